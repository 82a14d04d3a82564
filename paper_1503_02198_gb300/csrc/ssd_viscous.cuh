// ssd_viscous.cuh -- viscous chain of the sliding-mesh SD residual (Sec. 2.1
// viscous fluxes; Sec. 3.1 common solution / common viscous flux on cell
// faces; Sec. 3.2 viscous mortar procedure).  Included by ssd_engine.cuh.
//
// Per stage, after the stage clock and mortar merge:
//   k_faces_cq                 common solution Q_c on conforming faces (average)
//                              and boundaries (the state on the boundary)
//   k_mortar_flux<MORTAR_AVG_Q>  Q_c on the interface: both sides projected
//                              to the mortars, averaged, projected back (summed
//                              into each face by the gradient kernel)
//   k_grad_trace               gradients of the conservative variables at the
//                              SPs (derivative of the degree-N polynomial through
//                              the FP values with Q_c at the end FPs, chain rule
//                              with the SP metrics), stored for k_volume_visc and
//                              interpolated to the faces
//   k_faces_visc               Rusanov + average of both sides' viscous normal
//                              flux evaluated with Q_c (boundaries: boundary state,
//                              interior gradient)
//   k_mortar_flux<MORTAR_RUSANOV_FV>: traces and the viscous normal flux of
//                              both sides projected to the mortars in one pass,
//                              Rusanov + average of the viscous fluxes, projected
//                              back as one sum (summed into each face by the
//                              viscous volume kernel)
//   k_volume_visc              inviscid + viscous fluxes at interior FPs (with
//                              the stored SP gradients), divergence, Runge-Kutta
//                              update, traces; persistent, tiles fed by 1-D
//                              bulk copies one tile ahead
#pragma once

namespace ssd {

// viscous fluxes of Sec. 2.1 (with the paper's leading minus sign) from Q and
// the physical gradients of the conservative variables; conduct = false drops
// the heat conduction (adiabatic walls)
template <typename T>
__device__ __forceinline__ void viscous_flux(const T *q, const T *qx, const T *qy, const MeshDev &md, T *F, T *G,
                                             bool conduct = true) {
  const T gm1 = pick<T>(md.gm1, md.gm1_f), mu = pick<T>(md.mu, md.mu_f);
  const T kr = conduct ? pick<T>(md.kcR, md.kcR_f) : T(0);  // conductivity / R
  const T ir = recip(q[0]);
  const T u = q[1] * ir, v = q[2] * ir;
  // velocity gradients rounded as products (mul_rn): they are summed with each
  // other below, where an FMA could otherwise take either one
  const T ux = mul_rn(qx[1] - u * qx[0], ir), uy = mul_rn(qy[1] - u * qy[0], ir);
  const T vx = mul_rn(qx[2] - v * qx[0], ir), vy = mul_rn(qy[2] - v * qy[0], ir);
  const T ke = T(0.5) * mul_add(u, u, v, v);
  const T p = gm1 * (q[3] - ke * q[0]);
  const T pr = p * ir;  // R T
  const T px = mul_rn(gm1, qx[3] - fma(u, qx[1], mul_sub(v, qx[2], ke, qx[0])));
  const T py = mul_rn(gm1, qy[3] - fma(u, qy[1], mul_sub(v, qy[2], ke, qy[0])));
  // R grad T = (grad p - R T grad rho) / rho; the heat flux takes k / R
  const T Tx = fma(-pr, qx[0], px) * ir, Ty = fma(-pr, qy[0], py) * ir;
  const T lam = T(-2) / T(3) * mu, dv = ux + vy;
  const T txx = mul_add(T(2) * mu, ux, lam, dv), tyy = mul_add(T(2) * mu, vy, lam, dv), txy = mu * (uy + vx);
  F[0] = 0;
  F[1] = -txx;
  F[2] = -txy;
  F[3] = -fma(u, txx, mul_add(v, txy, kr, Tx));
  G[0] = 0;
  G[1] = -txy;
  G[2] = -tyy;
  G[3] = -fma(u, txy, mul_add(v, tyy, kr, Ty));
}

// ---- common solution -------------------------------------------------------

template <typename T, int N>
__device__ __forceinline__ void k_face_cq_point(const MeshDev &md, int t) {
  const int fi = t / N, j = t - fi * N;
  const int4 fc = md.faces[fi];
  const int efA = fc.x, efB = fc.y, jB = fc.z ? N - 1 - j : j;
  const T *TR = (const T *)md.TR;
  T *CQ = (T *)md.CQ;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const T c = T(0.5) * (TR[((size_t)efA * 4 + v) * N + j] + TR[((size_t)efB * 4 + v) * N + jB]);
    CQ[((size_t)efA * 4 + v) * N + j] = c;
    CQ[((size_t)efB * 4 + v) * N + jB] = c;
  }
}

// boundary faces: the common solution is the state on the boundary
template <typename T, int N, bool OTF>
__device__ __forceinline__ void k_bface_cq_point(const MeshDev &md, int t) {
  const int b = t / N, j = t - b * N;
  const int4 bf = md.bfaces[b];
  const int ef = bf.x;
  const T *TR = (const T *)md.TR;
  T q[4], qg[4], qb[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) q[v] = TR[((size_t)ef * 4 + v) * N + j];
  T nx, ny, sS, vgn, ug, vg;
  bface_geom<T, N, OTF>(md, b, j, nx, ny, sS, vgn, ug, vg);
  boundary_states(md, bf.y, q, ug, vg, nx, ny, qg, qb);
#pragma unroll
  for (int v = 0; v < 4; ++v) ((T *)md.CQ)[((size_t)ef * 4 + v) * N + j] = qb[v];
}

// common solution at all face points of a stage (conforming, then boundary)
template <typename T, int N, bool OTF>
__global__ void k_faces_cq(MeshDev md) {
  pdl_enter();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < md.nF * N) k_face_cq_point<T, N>(md, t);
  else if (t < (md.nF + md.nB) * N) k_bface_cq_point<T, N, OTF>(md, t - md.nF * N);
}

// ---- gradients ---------------------------------------------------------------

// Elements per block of the viscous kernels (two threads per SP line pair:
// 2 N threads per element): chosen so that a block is whole warps.
template <typename T, int N>
struct VisCfg {
  static constexpr bool F = sizeof(T) == 4;
  static constexpr int EPB = N == 3 ? 16 : (N == 4 ? 8 : (N == 5 ? (F ? 16 : 8) : (F ? 8 : 4)));
  static constexpr int THREADS = EPB * 2 * N;
  // resident blocks per SM the register budget is set for: about 16 warps
  static constexpr int MINB = 16 / ((THREADS + 31) / 32) > 0 ? 16 / ((THREADS + 31) / 32) : 1;
};

// Gradients at the SPs of a tile (thread per SP line, then per SP): on
// return sDx / sDe hold Q_x / Q_y, and gsp (the tile's rows of GSP,
// [element][8][N^2]) the same.  The caller synchronises before and after.
template <typename T, int N, bool OTF>
__device__ __forceinline__ void tile_gradients(const MeshDev &md, int e0, int ne, T (*sQ)[4][N * N],
                                               T (*sCQ)[16 * N], T (*sDx)[4][N * N], T (*sDe)[4][N * N],
                                               const T *zt, const int *sEF, const T *sEG, T *gsp) {
  constexpr int NN = N * N, NT = VisCfg<T, N>::THREADS;
  const VolBasis<T, N> &B = cVB<T, N>;
  const int le = threadIdx.x / (2 * N);
  const int r = threadIdx.x - le * 2 * N;
  const int d = r / N, m = r - d * N;
  if (le < ne) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T val[N + 1], qv[N];
      val[0] = sCQ[le][((d == 0 ? 3 : 0) * 4 + v) * N + m];
      val[N] = sCQ[le][((d == 0 ? 1 : 2) * 4 + v) * N + m];
      // the line's N values, read once for all its flux points
#pragma unroll
      for (int k = 0; k < N; ++k) qv[k] = sQ[le][v][d == 0 ? m * N + k : k * N + m];
#pragma unroll
      for (int i = 1; i < N; ++i) {
        T acc = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) acc += qv[k] * B.Hf[i * N + k];
        val[i] = acc;
      }
#pragma unroll
      for (int k = 0; k < N; ++k) {
        T acc = 0;
#pragma unroll
        for (int i = 0; i <= N; ++i) acc += B.Dm[k * (N + 1) + i] * val[i];
        if (d == 0) sDx[le][v][m * N + k] = acc;   // d/dxi at SP (k, m)
        else sDe[le][v][k * N + m] = acc;          // d/deta at SP (m, k)
      }
    }
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < ne * NN; idx += NT) {
    const int l2 = idx / NN, sp = idx - l2 * NN;
    ElemGeo<T, N, OTF> G;
    G.load_rec(md, e0 + l2, sEF[l2], sEG + l2 * 8, zt);
    T xix, xiy, etx, ety;
    G.sp_grad(sp % N, sp / N, xix, xiy, etx, ety);
    T *g = gsp + (size_t)l2 * 8 * NN + sp;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      const T a = sDx[l2][v][sp], b = sDe[l2][v][sp];
      const T gx = mul_add(xix, a, etx, b), gy = mul_add(xiy, a, ety, b);
      sDx[l2][v][sp] = gx;
      sDe[l2][v][sp] = gy;
      g[v * NN] = gx;
      g[(4 + v) * NN] = gy;
    }
  }
}

// Shared-memory layout of the persistent gradient kernel: two stages of a
// tile's state (4 N^2 values per element) and common solution (16 N), one
// contiguous run each as in global memory; then the gradient arrays.
template <typename T, int N>
struct GradCfg {
  static constexpr int EPB = VisCfg<T, N>::EPB, THREADS = VisCfg<T, N>::THREADS, NN = N * N;
  static constexpr int QE = 4 * NN * (int)sizeof(T), CE = 16 * N * (int)sizeof(T);
  static constexpr int GEE = 8 * (int)sizeof(T);  // bilinear cell record
  static constexpr int O_Q = 0, O_C = O_Q + EPB * QE, O_EG = O_C + EPB * CE, O_EF = O_EG + EPB * GEE;
  static constexpr int STAGE = ((O_EF + EPB * 4) + 127) / 128 * 128;
  static constexpr int O_DX = 2 * STAGE, O_DE = O_DX + EPB * QE;
  static constexpr int O_BAR = ((O_DE + EPB * QE) + 15) / 16 * 16;
  static constexpr int SMEM = O_BAR + 2 * 8;
  static_assert(QE % 16 == 0 && CE % 16 == 0, "bulk-copy sizes and alignment");
  static_assert(SMEM <= 227 * 1024, "dynamic shared memory of one CTA");
};

// SP gradients GSP [E][8][N][N] and gradient traces GTR [E][4 faces][8][N]
// (component v = dQ_v/dx, 4 + v = dQ_v/dy).  Persistent: each CTA walks
// tiles; thread 0 issues the next tile's state and common solution (two 1-D
// bulk copies) into the other stage while the CTA computes the current one.
template <typename T, int N, bool OTF, class Src>
__global__ void __launch_bounds__(GradCfg<T, N>::THREADS) k_grad_trace(Src src, int nitems) {
  pdl_enter();
  using C = GradCfg<T, N>;
  constexpr int EPB = C::EPB, NT = C::THREADS, NN = N * N;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = (uint64_t *)(smem + C::O_BAR);
  T(*sDx)[4][NN] = (T(*)[4][NN])(smem + C::O_DX);
  T(*sDe)[4][NN] = (T(*)[4][NN])(smem + C::O_DE);
  // the state of the stage (the item's case's input state), the common
  // solution, the cell records (on-the-fly path) and flags; the flags are
  // copied in whole groups of 4 (16 bytes), within the tile-padded array
  auto issue = [&](int item, int st) {
    int cn, tl;
    src.item(item, cn, tl);
    const MeshDev &mn = src.mesh(cn);
    const T *Q = (const T *)src.args(cn).in.hi;
    unsigned char *sb = smem + st * C::STAGE;
    if (!batch_check(mn, tl >= 0 && tl * EPB < mn.E)) {
      mbar_expect_tx(&bar[st], 0);  // a work item outside its case: nothing copied
      return;
    }
    const size_t e0 = (size_t)tl * EPB;
    const uint32_t ne = (uint32_t)min(EPB, mn.E - (int)e0), nf = (ne + 3u) & ~3u;
    mbar_expect_tx(&bar[st], ne * (C::QE + C::CE + (OTF ? C::GEE : 0)) + nf * 4u);
    bulk_g2s(sb + C::O_Q, Q + e0 * 4 * NN, ne * C::QE, &bar[st]);
    bulk_g2s(sb + C::O_C, (const T *)mn.CQ + e0 * 16 * N, ne * C::CE, &bar[st]);
    if (OTF) bulk_g2s(sb + C::O_EG, (const T *)mn.egeo + e0 * 8, ne * C::GEE, &bar[st]);
    bulk_g2s(sb + C::O_EF, mn.eflag + e0, nf * 4u, &bar[st]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  __syncthreads();
  int item = blockIdx.x;
  if (threadIdx.x == 0 && item < nitems) issue(item, 0);
  const VolBasis<T, N> &B = cVB<T, N>;
  const int le = threadIdx.x / (2 * N);
  const int r = threadIdx.x - le * 2 * N;
  const int d = r / N, m = r - d * N;
  int it = 0;
  for (; item < nitems; item += gridDim.x, ++it) {
    const int st = it & 1;
    const int next = item + gridDim.x;
    int cs, tile;
    src.item(item, cs, tile);
    const MeshDev &md = src.mesh(cs);
    const T *zt = zone_tab<T>(md.clk);
    if (threadIdx.x == 0 && next < nitems) {
      fence_proxy_async_smem();
      issue(next, st ^ 1);
    }
    if (!cta_wait(&bar[st], (uint32_t)((it >> 1) & 1))) {
      if (threadIdx.x == 0) {
        atomicOr(&md.clk->flags, 4);
        if (next < nitems) mbar_wait_bounded(&bar[st ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
      }
      return;
    }
    unsigned char *sb = smem + st * C::STAGE;
    T(*sQ)[4][NN] = (T(*)[4][NN])(sb + C::O_Q);
    T(*sCQ)[16 * N] = (T(*)[16 * N])(sb + C::O_C);
    const T *sEG = (const T *)(sb + C::O_EG);
    const int *sEF = (const int *)(sb + C::O_EF);
    const int e0 = tile * EPB;
    const int ne = min(EPB, md.E - e0);
    // the tile's interface faces: their common solution from the mortar
    // contributions, also into CQ for the viscous mortar pass that follows
    if (gather_tile<T, N, GATHER_Q>(md, e0, ne, sEF, (T *)(sb + C::O_C), 16 * N, true, NT)) __syncthreads();
    // the SP gradients, also stored for the volume kernel of this stage
    tile_gradients<T, N, OTF>(md, e0, ne, sQ, sCQ, sDx, sDe, zt, sEF, sEG, (T *)md.GSP + (size_t)e0 * 8 * NN);
    __syncthreads();
    if (le < ne) {
      T *g = (T *)md.GTR + (size_t)(e0 + le) * 32 * N;
      const int fa = d == 0 ? 3 : 0, fb = d == 0 ? 1 : 2;
#pragma unroll
      for (int c = 0; c < 8; ++c) {
        const int v = c & 3;
        T a0 = 0, a1 = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const int sp = d == 0 ? m * N + k : k * N + m;
          const T val = c < 4 ? sDx[le][v][sp] : sDe[le][v][sp];
          a0 += val * B.H0[k];
          a1 += val * B.H1[k];
        }
        g[(fa * 8 + c) * N + m] = a0;
        g[(fb * 8 + c) * N + m] = a1;
      }
    }
    // every read of this tile's stage and of the gradient arrays is done
    // before they are refilled
    __syncthreads();
  }
}

// ---- common fluxes -------------------------------------------------------------

// normal viscous flux F_vis . n from Q and the 8 gradient components
template <typename T>
__device__ __forceinline__ void viscous_normal(const T *q, const T *g8, T nx, T ny, const MeshDev &md, T *fn,
                                               bool conduct = true) {
  T F[4], G[4];
  viscous_flux(q, g8, g8 + 4, md, F, G, conduct);
#pragma unroll
  for (int v = 0; v < 4; ++v) fn[v] = mul_add(F[v], nx, G[v], ny);
}

template <typename T, int N>
__device__ __forceinline__ void k_face_visc_point(const MeshDev &md, int t) {
  const int fi = t / N, j = t - fi * N;
  const int4 fc = md.faces[fi];
  const int efA = fc.x, efB = fc.y, jB = fc.z ? N - 1 - j : j;
  const T *TR = (const T *)md.TR, *CQ = (const T *)md.CQ, *GT = (const T *)md.GTR;
  T qA[4], qB[4], qc[4], gA[8], gB[8];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    qA[v] = TR[((size_t)efA * 4 + v) * N + j];
    qB[v] = TR[((size_t)efB * 4 + v) * N + jB];
    qc[v] = CQ[((size_t)efA * 4 + v) * N + j];
  }
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    gA[c] = GT[((size_t)efA * 8 + c) * N + j];
    gB[c] = GT[((size_t)efB * 8 + c) * N + jB];
  }
  const T *g = (const T *)md.fgeo + (size_t)fi * 5 * N;
  T nx = g[j], ny = g[N + j];
  const T sA = g[2 * N + j], sB = g[3 * N + j], vgn = g[4 * N + j];
  const int z = md.eflag[efA >> 2] & kZoneMask;
  if (z) {
    const T *zt = zone_tab<T>(md.clk);
    const T c = zt[z], s = zt[kZT + z];
    const T rx = mul_sub(c, nx, s, ny), ry = mul_add(s, nx, c, ny);
    nx = rx;
    ny = ry;
  }
  T Fn[4], va[4], vb[4];
  rusanov(qA, qB, nx, ny, vgn, pick<T>(md.gamma, md.gamma_f), Fn);
  viscous_normal(qc, gA, nx, ny, md, va);
  viscous_normal(qc, gB, nx, ny, md, vb);
  T *CF = (T *)md.CF;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    const T f = Fn[v] + T(0.5) * (va[v] + vb[v]);
    CF[((size_t)efA * 4 + v) * N + j] = sA * f;
    CF[((size_t)efB * 4 + v) * N + jB] = -sB * f;
  }
}

// boundary faces: Rusanov through the ghost state plus the viscous flux of the
// boundary state with the interior gradient
template <typename T, int N, bool OTF>
__device__ __forceinline__ void k_bface_visc_point(const MeshDev &md, int t) {
  const int b = t / N, j = t - b * N;
  const int4 bf = md.bfaces[b];
  const int ef = bf.x;
  const T *TR = (const T *)md.TR, *GT = (const T *)md.GTR;
  T q[4], qg[4], qb[4], g8[8];
#pragma unroll
  for (int v = 0; v < 4; ++v) q[v] = TR[((size_t)ef * 4 + v) * N + j];
#pragma unroll
  for (int c = 0; c < 8; ++c) g8[c] = GT[((size_t)ef * 8 + c) * N + j];
  T nx, ny, sS, vgn, ug, vg;
  bface_geom<T, N, OTF>(md, b, j, nx, ny, sS, vgn, ug, vg);
  boundary_states(md, bf.y, q, ug, vg, nx, ny, qg, qb);
  T Fn[4], fv[4];
  rusanov(q, qg, nx, ny, vgn, pick<T>(md.gamma, md.gamma_f), Fn);
  viscous_normal(qb, g8, nx, ny, md, fv, bf.y != SD_BC_ADIABATIC);
  T *CF = (T *)md.CF;
#pragma unroll
  for (int v = 0; v < 4; ++v) CF[((size_t)ef * 4 + v) * N + j] = sS * (Fn[v] + fv[v]);
}

// common inviscid + viscous fluxes at all face points of a stage
template <typename T, int N, bool OTF>
__global__ void k_faces_visc(MeshDev md) {
  pdl_enter();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < md.nF * N) k_face_visc_point<T, N>(md, t);
  else if (t < (md.nF + md.nB) * N) k_bface_visc_point<T, N, OTF>(md, t - md.nF * N);
}

// ---- volume ------------------------------------------------------------------

// Shared-memory layout of the persistent viscous volume kernel: two stages of
// a tile's state (4 N^2 values per element), SP gradients (8 N^2: x then y)
// and common fluxes (16 N), each one contiguous run as in global memory, so a
// tile arrives by three 1-D bulk copies; then the tile's transformed fluxes at
// the interior flux points and the interpolation / derivative weights.  One
// thread per interior flux point of every SP line of the tile: 2 N (N - 1)
// threads per element, so that a CTA holds few elements and many threads.
template <typename T, int N>
struct VisVolCfg {
  static constexpr int EPB = N == 3 ? 16 : (N == 4 ? 8 : 4);
  static constexpr int NN = N * N, LINES = EPB * 2 * N, THREADS = LINES * (N - 1);
  static constexpr int QE = 4 * NN * (int)sizeof(T), GE = 8 * NN * (int)sizeof(T), CE = 16 * N * (int)sizeof(T);
  static constexpr int GEE = 8 * (int)sizeof(T);  // bilinear cell record
  static constexpr int O_Q = 0, O_G = O_Q + EPB * QE, O_C = O_G + EPB * GE, O_EG = O_C + EPB * CE;
  static constexpr int O_EF = O_EG + EPB * GEE;
  static constexpr int STAGE = ((O_EF + EPB * 4) + 127) / 128 * 128;
  // fluxes [EPB][2 directions][N lines][LS]: a line's N - 1 interior points,
  // 4 values each; the odd line stride puts neighbouring lines in different banks
  static constexpr int LS = 4 * (N - 1) + 1;
  static constexpr int O_FL = 2 * STAGE;
  static constexpr int O_W = O_FL + (EPB * 2 * N * LS * (int)sizeof(T) + 15) / 16 * 16;  // Hf, then Dm
  static constexpr int O_BAR = (O_W + 2 * N * (N + 1) * (int)sizeof(T) + 15) / 16 * 16;
  static constexpr int SMEM = O_BAR + 2 * 8;
  static_assert(QE % 16 == 0 && GE % 16 == 0 && CE % 16 == 0, "bulk-copy sizes and alignment");
  static_assert(SMEM <= 227 * 1024 && THREADS <= 1024, "one CTA");
  // resident CTAs per SM the register budget is set for: about 24 warps, or
  // what the shared memory admits
  static constexpr int WARPS = (THREADS + 31) / 32;
  static constexpr int BY_WARPS = 32 / WARPS > 0 ? 32 / WARPS : 1;
  static constexpr int BY_SMEM = 228 * 1024 / (SMEM + 1024);
  static constexpr int MINB = BY_WARPS < BY_SMEM ? BY_WARPS : (BY_SMEM > 0 ? BY_SMEM : 1);
};

// Inviscid + viscous fluxes at the interior FPs with the stored SP gradients,
// common fluxes at the end FPs, divergence, Runge-Kutta stage, traces.
// Persistent: each CTA walks tiles of EPB elements; thread 0 issues the next
// tile's three bulk copies into the other stage while the CTA computes the
// current one.  Every wait is bounded (device flag bit 2 on timeout).
template <typename T, int N, int MODE, bool OTF, bool LO, class Src>
__global__ void __launch_bounds__(VisVolCfg<T, N>::THREADS, VisVolCfg<T, N>::MINB)
    k_volume_visc(Src src, int nitems) {
  pdl_enter();
  using C = VisVolCfg<T, N>;
  constexpr int EPB = C::EPB, NT = C::THREADS, NN = N * N;
  constexpr bool FF = std::is_same<T, float>::value;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = (uint64_t *)(smem + C::O_BAR);
  T *sFl = (T *)(smem + C::O_FL);
  T *sHf = (T *)(smem + C::O_W), *sDm = sHf + (N + 1) * N;
  const VolBasis<T, N> &B = cVB<T, N>;
  // the state, the SP gradients that k_grad_trace formed from it in this
  // stage, and the common fluxes of tile tl into stage st
  // with the cell records (on-the-fly path) and flags, the flags in whole
  // groups of 4 (16 bytes), within the tile-padded array
  auto issue = [&](int item, int st) {
    int cn, tl;
    src.item(item, cn, tl);
    const MeshDev &mn = src.mesh(cn);
    unsigned char *sb = smem + st * C::STAGE;
    if (!batch_check(mn, tl >= 0 && tl * EPB < mn.E)) {
      mbar_expect_tx(&bar[st], 0);  // a work item outside its case: nothing copied
      return;
    }
    const size_t e0 = (size_t)tl * EPB;
    const uint32_t ne = (uint32_t)min(EPB, mn.E - (int)e0), nf = (ne + 3u) & ~3u;
    mbar_expect_tx(&bar[st], ne * (C::QE + C::GE + C::CE + (OTF ? C::GEE : 0)) + nf * 4u);
    bulk_g2s(sb + C::O_Q, (const T *)src.args(cn).in.hi + e0 * 4 * NN, ne * C::QE, &bar[st]);
    bulk_g2s(sb + C::O_G, (const T *)mn.GSP + e0 * 8 * NN, ne * C::GE, &bar[st]);
    bulk_g2s(sb + C::O_C, (const T *)mn.CF + e0 * 16 * N, ne * C::CE, &bar[st]);
    if (OTF) bulk_g2s(sb + C::O_EG, (const T *)mn.egeo + e0 * 8, ne * C::GEE, &bar[st]);
    bulk_g2s(sb + C::O_EF, mn.eflag + e0, nf * 4u, &bar[st]);
  };
  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  // the interpolation and derivative weights, read per thread at different points
  for (int k = threadIdx.x; k < (N + 1) * N; k += NT) {
    sHf[k] = B.Hf[k];
    sDm[k] = B.Dm[k];
  }
  __syncthreads();
  int item = blockIdx.x;
  if (threadIdx.x == 0 && item < nitems) issue(item, 0);
  // phase-1 thread: interior flux point fi of SP line m in direction d of
  // tile element le; the threads with fi = 1 also take the line's traces
  const int fi = 1 + (int)threadIdx.x / C::LINES;
  const int t1 = (int)threadIdx.x - (fi - 1) * C::LINES;
  const int le = t1 / (2 * N);
  const int r = t1 - le * 2 * N;
  const int d = r / N, m = r - d * N;
  bool bad = false;
  int it = 0;
  for (; item < nitems; item += gridDim.x, ++it) {
    const int st = it & 1;
    const int next = item + gridDim.x;
    int cs, tile;
    src.item(item, cs, tile);
    const MeshDev &md = src.mesh(cs);
    const VolArgs<T> &va = src.args(cs);
    const StatePtr in = va.in, base = va.base, out = va.out;
    const RkCoef<T> rk = va.rk;
    const int has_base = va.has_base;
    T *const w_out = va.w_out;
    const T *const w_in = va.w_in;
    double *const Rout = va.R;
    const T *zt = zone_tab<T>(md.clk);
    const T gm1 = pick<T>(md.gm1, md.gm1_f);
    if (threadIdx.x == 0 && next < nitems) {
      // the other stage was last read before the previous iteration's closing
      // barrier; order those generic reads before the async writes
      fence_proxy_async_smem();
      issue(next, st ^ 1);
    }
    if (!cta_wait(&bar[st], (uint32_t)((it >> 1) & 1))) {
      if (threadIdx.x == 0) {
        atomicOr(&md.clk->flags, 4);
        // let the copy in flight land before the CTA exits
        if (next < nitems) mbar_wait_bounded(&bar[st ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
      }
      return;
    }
    unsigned char *sb = smem + st * C::STAGE;
    T(*sQ)[4][NN] = (T(*)[4][NN])(sb + C::O_Q);
    const T(*sG)[8][NN] = (const T(*)[8][NN])(sb + C::O_G);
    const T(*sCF)[16 * N] = (const T(*)[16 * N])(sb + C::O_C);
    const T *sEG = (const T *)(sb + C::O_EG);
    const int *sEF = (const int *)(sb + C::O_EF);
    const int e0 = tile * EPB;
    const int ne = min(EPB, md.E - e0);
    // the tile's interface faces: their common fluxes from the mortar contributions
    if (gather_tile<T, N, GATHER_FLUX>(md, e0, ne, sEF, (T *)(sb + C::O_C), 16 * N, false, NT)) __syncthreads();
    // ---- phase 1: one thread per interior flux point: Q and its gradients
    // interpolated to the point (Eq. Qt), the inviscid ALE flux and the
    // viscous flux (Sec. 2.1) transformed with the point's metric vector,
    // into the tile's flux array ----
    if (le < ne) {
      ElemGeo<T, N, OTF> G;
      G.load_rec(md, e0 + le, sEF[le], sEG + le * 8, zt);
      const T *h = sHf + fi * N;
      T qf[4], g8[8];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        T a = 0, bx = 0, by = 0;
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const int sp = d == 0 ? m * N + k : k * N + m;
          a = fma(sQ[le][v][sp], h[k], a);
          bx = fma(sG[le][v][sp], h[k], bx);
          by = fma(sG[le][4 + v][sp], h[k], by);
        }
        qf[v] = a;
        g8[v] = bx;
        g8[4 + v] = by;
      }
      T vx, vy, vg;
      if (d == 0) G.xi_fp(fi, m, vx, vy, vg);
      else G.eta_fp(m, fi, vx, vy, vg);
      const T p = pressure_of(qf, gm1);
      T f[4], Fv[4], Gv[4];
      normal_flux(qf, p, vx, vy, vg, f);
      viscous_flux(qf, g8, g8 + 4, md, Fv, Gv);
      T *o = sFl + ((le * 2 + d) * N + m) * C::LS + (fi - 1) * 4;
#pragma unroll
      for (int v = 0; v < 4; ++v) o[v] = fma(vx, Fv[v], fma(vy, Gv[v], f[v]));
    }
    __syncthreads();
    // (RF + RG)[v] at SP sp = (i, j) of element l2: each direction's
    // divergence over its line's flux points 0..N in order (Eqs. Ft, Gt), the
    // end points from the common fluxes
    auto divergence = [&](int l2, int sp, T *dsum) {
      const int i = sp % N, j = sp / N;
      const T *fx = sFl + ((l2 * 2 + 0) * N + j) * C::LS, *fe = sFl + ((l2 * 2 + 1) * N + i) * C::LS;
      const T *wx = sDm + i * (N + 1), *we = sDm + j * (N + 1);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        T a = mul_rn(wx[0], sCF[l2][(3 * 4 + v) * N + j]);
        T b = mul_rn(we[0], sCF[l2][(0 * 4 + v) * N + i]);
#pragma unroll
        for (int l = 1; l < N; ++l) {
          a = fma(wx[l], fx[(l - 1) * 4 + v], a);
          b = fma(we[l], fe[(l - 1) * 4 + v], b);
        }
        a = fma(wx[N], sCF[l2][(1 * 4 + v) * N + j], a);
        b = fma(we[N], sCF[l2][(2 * 4 + v) * N + i], b);
        dsum[v] = a + b;
      }
    };
    // ---- phase 2: dQ/dt at the SPs and the Runge-Kutta stage ----
    if constexpr (MODE == MODE_RK && FF) {
      // FP32: the base state and the lo planes of an SP come from global
      // memory; the next SP's loads are issued before this SP's stores (later
      // stages update the state in place, so the compiler keeps loads behind
      // earlier stores unless the program orders them first)
      auto fetch = [&](int idx, float *bh, float *kl, float *bl) {
        const int l2 = idx / NN, sp = idx - l2 * NN;
        const size_t gi = ((size_t)(e0 + l2) * 4) * NN + sp;
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          bh[v] = has_base ? ((const float *)base.hi)[gi + v * NN] : 0.0f;
          kl[v] = LO ? ((const float *)in.lo)[gi + v * NN] : 0.0f;
          bl[v] = (LO && has_base) ? ((const float *)base.lo)[gi + v * NN] : 0.0f;
        }
      };
      float bh[4], kl[4], bl[4];
      if ((int)threadIdx.x < ne * NN) fetch(threadIdx.x, bh, kl, bl);
      for (int idx = threadIdx.x; idx < ne * NN; idx += NT) {
        float nbh[4], nkl[4], nbl[4];
        if (idx + NT < ne * NN) fetch(idx + NT, nbh, nkl, nbl);
        const int l2 = idx / NN, sp = idx - l2 * NN;
        const T iJ = ElemGeo<T, N, OTF>::inv_jac_t0(md, sEF[l2], sEG + l2 * 8, sp % N, sp / N);
        const size_t gi = ((size_t)(e0 + l2) * 4) * NN + sp;
        T dsum[4];
        divergence(l2, sp, dsum);
        float hv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const size_t ii = gi + v * NN;
          const float R = -(float)(dsum[v] * iJ);
          const float h = (float)sQ[l2][v][sp];
          float inc = __fmul_rn((float)rk.bdt, R);
          if constexpr (LO) {
            const float l = kl[v];
            if (has_base) inc = fmaf((float)rk.a0, (bh[v] - h) + (bl[v] - l), inc);
            if (w_in) inc += (float)w_in[ii];
            float sum, err;
            two_sum(h, inc, sum, err);
            err += l;
            const float H = sum + err;
            ((float *)out.hi)[ii] = H;
            ((float *)out.lo)[ii] = err - (H - sum);
            hv[v] = H;
          } else {
            // single-float state: the stage result is rounded to float once
            if (has_base) inc = fmaf((float)rk.a0, bh[v] - h, inc);
            if (w_in) inc += (float)w_in[ii];
            const float H = h + inc;
            ((float *)out.hi)[ii] = H;
            hv[v] = H;
          }
          if (w_out) w_out[ii] = (T)fmaf(-(float)rk.g, inc, (float)rk.ddt * R);
        }
        bad |= !physical(hv);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          sQ[l2][v][sp] = (T)hv[v];
          bh[v] = nbh[v];
          kl[v] = nkl[v];
          bl[v] = nbl[v];
        }
      }
    } else
    for (int idx = threadIdx.x; idx < ne * NN; idx += NT) {
      const int l2 = idx / NN, sp = idx - l2 * NN;
      const T iJ = ElemGeo<T, N, OTF>::inv_jac_t0(md, sEF[l2], sEG + l2 * 8, sp % N, sp / N);
      const size_t gi = ((size_t)(e0 + l2) * 4) * NN + sp;
      T dsum[4];
      divergence(l2, sp, dsum);
      if (MODE == MODE_RESIDUAL) {
#pragma unroll
        for (int v = 0; v < 4; ++v) Rout[gi + v * NN] = -(double)(dsum[v] * iJ);
      } else if (!FF) {
        double qn[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const size_t ii = gi + v * NN;
          const double R = -(double)(dsum[v] * iJ);
          const double qk = (double)sQ[l2][v][sp];
          double inc = __dmul_rn((double)rk.bdt, R);
          if (has_base) inc = fma((double)rk.a0, ((const double *)base.hi)[ii] - qk, inc);
          if (w_in) inc += (double)w_in[ii];
          qn[v] = qk + inc;
          if (w_out) w_out[ii] = (T)mul_sub((double)rk.ddt, R, (double)rk.g, inc);
        }
        bad |= !physical(qn);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          ((double *)out.hi)[gi + v * NN] = qn[v];
          sQ[l2][v][sp] = (T)qn[v];
        }
      } else {
        float hv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const size_t ii = gi + v * NN;
          const float R = -(float)(dsum[v] * iJ);
          const float h = (float)sQ[l2][v][sp];
          float inc = __fmul_rn((float)rk.bdt, R);
          if constexpr (LO) {
            const float l = ((const float *)in.lo)[ii];
            if (has_base)
              inc = fmaf((float)rk.a0, (((const float *)base.hi)[ii] - h) + (((const float *)base.lo)[ii] - l), inc);
            if (w_in) inc += (float)w_in[ii];
            float sum, err;
            two_sum(h, inc, sum, err);
            err += l;
            const float H = sum + err;
            ((float *)out.hi)[ii] = H;
            ((float *)out.lo)[ii] = err - (H - sum);
            hv[v] = H;
          } else {
            // single-float state: the stage result is rounded to float once
            if (has_base) inc = fmaf((float)rk.a0, ((const float *)base.hi)[ii] - h, inc);
            if (w_in) inc += (float)w_in[ii];
            const float H = h + inc;
            ((float *)out.hi)[ii] = H;
            hv[v] = H;
          }
          if (w_out) w_out[ii] = (T)fmaf(-(float)rk.g, inc, (float)rk.ddt * R);
        }
        bad |= !physical(hv);
#pragma unroll
        for (int v = 0; v < 4; ++v) sQ[l2][v][sp] = (T)hv[v];
      }
    }
    if (MODE == MODE_RK) {
      __syncthreads();
      // ---- phase 3: face traces of the new state, one thread per SP line
      // and variable (all the CTA's threads take part) ----
      for (int q = threadIdx.x; q < 4 * C::LINES; q += NT) {
        const int v = q / C::LINES, ln = q - v * C::LINES;
        const int l3 = ln / (2 * N), r3 = ln - l3 * 2 * N;
        const int d3 = r3 / N, m3 = r3 - d3 * N;
        if (l3 < ne) {
          T *tr = (T *)md.TR + (size_t)(e0 + l3) * 16 * N;
          const int fa = d3 == 0 ? 3 : 0, fb = d3 == 0 ? 1 : 2;
          T a0 = 0, a1 = 0;
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const T qk = d3 == 0 ? sQ[l3][v][m3 * N + k] : sQ[l3][v][k * N + m3];
            a0 += qk * B.H0[k];
            a1 += qk * B.H1[k];
          }
          tr[(fa * 4 + v) * N + m3] = a0;
          tr[(fb * 4 + v) * N + m3] = a1;
        }
      }
    }
    // every read of this tile's stage is done before it is refilled (a batch
    // raises the non-physical flag on the tile's own case here)
    if constexpr (Src::kMulti) {
      if (__syncthreads_or(bad) && threadIdx.x == 0 && MODE == MODE_RK) atomicOr(&md.clk->flags, 1);
      bad = false;
    } else {
      __syncthreads();
    }
  }
  if constexpr (!Src::kMulti) {
    if (MODE == MODE_RK && __syncthreads_or(bad) && threadIdx.x == 0) atomicOr(&src.mesh(0).clk->flags, 1);
  }
}

}  // namespace ssd
