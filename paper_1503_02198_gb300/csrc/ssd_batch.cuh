// ssd_batch.cuh -- kernels of the batched form: many independent cases (each
// its own mesh, order, rotation rate and step size) advanced together, one
// launch per phase for all cases of a class (same compute type, N and viscous
// flag) instead of one per case.  Included by ssd_engine.cuh.
//
// A class's work for one stage is a list of items numbered across its cases,
// with per-case prefix sums: face-pass blocks (the mortar-flux blocks of a
// case first, then its face-point blocks) and volume / gradient tiles (the
// persistent kernels walk them through CaseList and gather the mortar
// contributions of their interface faces themselves).  Each
// case's stage view of the mesh (its stage clock and mortar table) and its
// volume arguments sit in device arrays, so a changed step size is a copy
// into those arrays, not a new graph.
#pragma once

namespace ssd {

// A class's point and block work of one stage.
struct BatchWork {
  const MeshDev *md;    // [n] each case's view of the stage
  const int *off_fblk;  // [n + 1] first block of each case in the fused face pass
  const int *nmb;       // [n] mortar-flux blocks of each case (its first blocks)
  int n;
};

// the last case c with off[c] <= x (off ascending, off[0] = 0)
__device__ __forceinline__ int case_of(const int *off, int n, int x) {
  int lo = 0, hi = n - 1;
  while (lo < hi) {
    const int mid = (lo + hi + 1) >> 1;
    if (__ldg(off + mid) <= x) lo = mid;
    else hi = mid - 1;
  }
  return lo;
}

// The face pass of every case of a class with the mortar flux of the same
// pass (the pairs of k_faces_mortar): a block belongs to one case; a case's
// first nmb blocks compute its mortar fluxes, the rest FB face points each.
template <typename T, int N, bool OTF, int MMODE, int FB>
__global__ void __launch_bounds__(FB) k_batch_faces(BatchWork w) {
  pdl_enter();
  static_assert(MortCfg<N>::THREADS <= FB, "mortar block");
  const int c = case_of(w.off_fblk, w.n, blockIdx.x);
  const int lb = (int)blockIdx.x - __ldg(w.off_fblk + c);
  const MeshDev &md = w.md[c];
  const int nmb = __ldg(w.nmb + c);
  if (!batch_check(md, lb >= 0 && nmb >= 0 && (lb < nmb || (lb - nmb) * FB < (md.nF + md.nB) * N))) return;
  if (lb < nmb) {
    mortar_flux_body<T, N, MMODE, MortCfg<N>::MPB>(md, lb);
    return;
  }
  const int t = (lb - nmb) * FB + threadIdx.x;
  if (t < md.nF * N) {
    if (MMODE == MORTAR_RUSANOV) k_face_point<T, N, OTF>(md, t);
    else if (MMODE == MORTAR_AVG_Q) k_face_cq_point<T, N>(md, t);
    else k_face_visc_point<T, N>(md, t);
  } else if (t < (md.nF + md.nB) * N) {
    const int tb = t - md.nF * N;
    if (MMODE == MORTAR_RUSANOV) k_bface_point<T, N, OTF>(md, tb);
    else if (MMODE == MORTAR_AVG_Q) k_bface_cq_point<T, N, OTF>(md, tb);
    else k_bface_visc_point<T, N, OTF>(md, tb);
  }
}

// Stage clocks and mortar tables of every stage of every case of a batch:
// block (interface ii, stage k, case c); the step's start time is the case's
// own clock's.
static __global__ void k_batch_merge(BatchMergeDev bm) {
  pdl_enter();
  const int ii = blockIdx.x, k = blockIdx.y, c = blockIdx.z;
  const MeshDev &base = bm.md[c];
  if (ii >= base.nI) return;
  const StageMerge &sm = bm.sm[c];
  clock_merge_body(bm.md_stage[(size_t)k * bm.ncase + c], ii, sm.c[k], bm.dt[c], sm.work_i[k], sm.work_d[k],
                   base.clk);
}

// Eq. xz of every mortar of every stage of every case (after k_batch_merge):
// block (x, stage k, case c)
static __global__ void __launch_bounds__(kXzBlock) k_batch_xz(BatchMergeDev bm) {
  pdl_enter();
  mortar_xz_body(bm.md_stage[(size_t)blockIdx.y * bm.ncase + blockIdx.z], blockIdx.x * kXzBlock + threadIdx.x);
}

// the end of a step of every case: t_n += dt
static __global__ void k_batch_advance(BatchMergeDev bm) {
  pdl_enter();
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c < bm.ncase) {
    DevClock *k = bm.md[c].clk;
    k->t_n = k->t_n + bm.dt[c];
  }
}

}  // namespace ssd
