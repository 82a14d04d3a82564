// ssd_engine.cuh -- sm_103a kernels of the sliding-mesh spectral difference
// residual and its SSP Runge-Kutta stage update, templated on the compute
// type T (double: FP64 path; float: FP32 path) and on N (solution points per
// direction, Sec. 3.1).
//
// FP64 path: every value and every operation in double.  FP32 path: the
// interpolation, flux and divergence arithmetic in float; the state is kept
// as a double-float pair (hi + lo) and the Runge-Kutta accumulation uses exact
// two-sum arithmetic on the FP32 pipe (GB300's FP64 pipe runs at 1/64 of the
// FP32 rate); the rotation angles (double-double), the mortar node order and
// the mortar offsets and scales (Eq. xz) are extended FP64 in both paths; the
// FP32 path evaluates the interface normals and the Lagrange products of the
// projection weights in float (Sec. 3.2).
//
// Per step:      k_clock_merge_stages, one CTA per stage (stage time t_k)
//                   and interface: theta_z = omega_z t_k of every rotating
//                   zone; merge of the interface's rotated L node angles
//                   with its R node angles -> mortars, (o, s) of each mortar
//                   against its L and R face (Eq. xz), face ranges, into the
//                   stage's own clock record and mortar table.  Off the
//                   critical path: stages 1.. are merged beside stage 0's
//                   kernels, and stage 0 of the next step beside stage 1's
//                   (k_clock_merge: the same for one stage, e.g. a residual)
// Per stage:
//   k_faces         one launch for every face point: conforming and periodic
//                   faces (Rusanov common flux), then boundary faces (wall,
//                   slip, inlet, outlet, adiabatic: Rusanov through a ghost state)
//   k_mortar_flux   per mortar: L2 projection of both sides' face traces
//                   (Eq. prjQ2), Rusanov at the mortar SPs, back-projection
//                   weights of the common flux (Eq. prjF2)
//   k_volume        per element: the common fluxes of its interface faces as
//                   the deterministic sum over each face's mortars (the
//                   gather), SP -> FP interpolation (Eq. Qt), transformed
//                   ALE fluxes (Eq. transform_relation), common fluxes at the
//                   end FPs, divergence (Eqs. Ft, Gt), RK update and the face
//                   traces of the new state
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <cstdio>
#include <type_traits>

#include "ssd_internal.h"
#include "../../include/ssd.h"

namespace ssd {

// Programmatic dependent launch: the kernels of a step are launched with
// programmatic stream serialization (launch_pdl), so a grid may be scheduled
// as the blocks of the grid before it exit (no early trigger: dependent
// blocks parked beside a running grid slowed it down).  Every such kernel
// first waits until the grid before it has completed and its writes are
// visible; without the attribute the wait returns at once.  Since each grid
// waits for its predecessor before it can complete, the order of the whole
// stream is kept.
__device__ __forceinline__ void pdl_enter() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  attr[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kernel, args...);
}

// Debug build (-DSSD_DEBUG): indices read from the mesh and mortar tables are
// checked before use; a bad one raises device flag bit 3 (reported by sd_sync
// as SD_ERR_MESH) and the access is skipped.  Kernels never trap.  In the
// normal build the check is the constant true.
#ifdef SSD_DEBUG
__device__ __forceinline__ bool ssd_check(const MeshDev &md, bool ok) {
  if (!ok) atomicOr(&md.clk->flags, 8);
  return ok;
}
#else
__device__ __forceinline__ bool ssd_check(const MeshDev &, bool) { return true; }
#endif
// The same check in every build, for the work lists of the batched form (a
// work item or face block outside its case is reported and its
// memory accesses skipped).
__device__ __forceinline__ bool batch_check(const MeshDev &md, bool ok) {
  if (!ok) atomicOr(&md.clk->flags, 8);
  return ok;
}

// ---------------------------------------------------------------------------
// constants
// ---------------------------------------------------------------------------

template <typename T, int N>
struct VolBasis {
  T Hf[(N + 1) * N];  // h_k(X_{i+1/2}) [i][k]
  T Dm[N * (N + 1)];  // l'_{i+1/2}(X_k) [k][i]
  T H0[N], H1[N];     // h_k(0), h_k(1)
  T Xs[N], Xf[N + 1]; // solution and flux points
  // the same weights duplicated into float pairs for packed FP32x2 FMAs
  float2 Hf2[(N + 1) * N], Dm2[N * (N + 1)], H02[N], H12[N];
};

template <int N>
struct MortBasis {
  double zq[N], wq[N];  // Gauss-Legendre on [0,1]
  double Hz[N * N];     // h_j(z_q) [q][j]
  double wHz[N * N];    // w_q h_j(z_q) [q][j]
  double Minv[N * N];   // M^{-1}
  double Xs[N];         // solution points
  double cden[N];       // 1 / prod_{s != i}(X_i - X_s)
  // the same rounded to float, for the FP32 contractions
  float Hz_f[N * N], wHz_f[N * N], Minv_f[N * N];
};

template <typename T, int N>
__constant__ VolBasis<T, N> cVB;
template <int N>
__constant__ MortBasis<N> cMB;

// metric table of one element at t = 0 (words of type T)
template <int N>
struct GeoLayout {
  static constexpr int NF = N * (N + 1);
  static constexpr int ax = 0, ay = NF, gx = 2 * NF;           // xi-FPs [j][i]: (y_eta, -x_eta), V_g . a
  static constexpr int bx = 3 * NF, by = 4 * NF, gy = 5 * NF;  // eta-FPs [l][i]: (-y_xi, x_xi), V_g . b
  static constexpr int iJ = 6 * NF;                            // 1/|J| at SPs [j][i]
  static constexpr int grad = 6 * NF + N * N;                  // xi_x, xi_y, eta_x, eta_y at SPs [4][N*N]
  static constexpr int G = 6 * NF + 5 * N * N;
};

// a b + c d and a b - c d with one fixed rounding: the first product is fused
// into an FMA, the second rounded first.  Left to the compiler, either product
// of such a sum may be fused, and two kernels that inline the same expression
// (a single case's kernel and a batch class's) may choose differently and
// differ in the last bit; written out, every kernel computes the same bits.
template <typename T>
__device__ __forceinline__ T mul_add(T a, T b, T c, T d) {
  return fma(a, b, c * d);
}
template <typename T>
__device__ __forceinline__ T mul_sub(T a, T b, T c, T d) {
  return fma(a, b, -(c * d));
}
// a state value set that is physical: rho > 0, p > 0 and E finite.  With
// rho > 0, p = (gamma - 1) (E - |m|^2 / (2 rho)) > 0 is 2 E rho > |m|^2,
// which needs no division.
template <typename T>
__device__ __forceinline__ bool physical(const T *q) {
  return q[0] > T(0) && T(2) * q[3] * q[0] - mul_add(q[1], q[1], q[2], q[2]) > T(0) && isfinite(q[3]);
}

// a product that is never fused into a later addition
__device__ __forceinline__ float mul_rn(float a, float b) { return __fmul_rn(a, b); }
__device__ __forceinline__ double mul_rn(double a, double b) { return __dmul_rn(a, b); }

// a parameter in the compute type, taken from its float copy on the FP32
// path so that no FP64 instruction runs there
template <typename T>
__device__ __forceinline__ T pick(double d, float f) {
  if constexpr (std::is_same<T, float>::value) return f;
  else return (T)d;
}

// 1 / x in FP64 by Newton's iteration for the reciprocal, r <- r + r (1 - x r)
// (each step squares the relative error), started from the hardware's
// approximate reciprocal (rcp.approx.ftz.f64); two steps bring the seed's
// error below double round-off, leaving at most an ulp or so against the
// correctly rounded 1 / x.  For normal, finite, non-zero x (densities and
// Jacobians here); the FP64 pipe then spends four FMAs instead of a division.
__device__ __forceinline__ double recip_newton(double x) {
  double r;
  asm("rcp.approx.ftz.f64 %0, %1;" : "=d"(r) : "d"(x));
  r = fma(r, fma(-x, r, 1.0), r);
  r = fma(r, fma(-x, r, 1.0), r);
  return r;
}

// The same in FP32: one Newton step from rcp.approx.ftz.f32 (relative error
// about 2^-23) leaves the result within an ulp of the correctly rounded 1 / x,
// in three instructions.
__device__ __forceinline__ float recip_newton(float x) {
  float r;
  asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return fmaf(r, fmaf(-x, r, 1.0f), r);
}

// 1 / x in the compute type (densities and Jacobians)
template <typename T>
__device__ __forceinline__ T recip(T x) {
  return recip_newton(x);
}

// face f of an element: sign sigma_f with F~_end = sigma_f |S| F.n_out
__device__ __forceinline__ double face_sigma(int f) { return (f == 1 || f == 2) ? 1.0 : -1.0; }

// ---------------------------------------------------------------------------
// geometry (Sec. 3.1 iso-parametric cells; Sec. 2.3 metrics)
// ---------------------------------------------------------------------------

// Edge from P to Q at u in [0,1]: offset of the point from P and the
// parameter derivative.  An arc edge is the circle about the origin
// (coordinates are centre-relative); its offset uses the chord identity
// e(phi0 + d) - e(phi0) = 2 sin(d/2) e_perp(phi0 + d/2), which keeps full
// relative precision for short arcs far from the centre.
__device__ inline void edge_offset(double px, double py, double qx, double qy, bool arc, double u, double &ox,
                                   double &oy, double &dx, double &dy) {
  if (!arc) {
    ox = u * (qx - px);
    oy = u * (qy - py);
    dx = qx - px;
    dy = qy - py;
    return;
  }
  const double r = sqrt(px * px + py * py);
  const double phi0 = atan2(py, px);
  const double dphi = atan2(px * qy - py * qx, px * qx + py * qy);
  const double half = 0.5 * u * dphi;
  double sh, ch, sm, cm, sn, cs;
  sincos(half, &sh, &ch);
  sincos(phi0 + half, &sm, &cm);
  const double chord = 2.0 * r * sh;
  ox = -chord * sm;
  oy = chord * cm;
  sincos(phi0 + u * dphi, &sn, &cs);
  dx = -r * dphi * sn;
  dy = r * dphi * cs;
}

// Cubic edge (Sec. 3.1's 12-node cells) through P, M1, M2, Q at u = 0, 1/3,
// 2/3, 1: offset from P and derivative, with the cubic Lagrange basis in
// closed form, l1 = 27/2 u (u - 2/3)(u - 1), l2 = -27/2 u (u - 1/3)(u - 1),
// l3 = 9/2 u (u - 1/3)(u - 2/3).
__device__ inline void cubic_offset(double px, double py, const double *mid, double qx, double qy, double u,
                                    double &ox, double &oy, double &dx, double &dy) {
  const double a = u - 1.0 / 3.0, b = u - 2.0 / 3.0, c = u - 1.0;
  const double l1 = 13.5 * u * b * c, l2 = -13.5 * u * a * c, l3 = 4.5 * u * a * b;
  const double d1 = 13.5 * (b * c + u * c + u * b), d2 = -13.5 * (a * c + u * c + u * a),
               d3 = 4.5 * (a * b + u * b + u * a);
  const double x1 = mid[0] - px, y1 = mid[1] - py, x2 = mid[2] - px, y2 = mid[3] - py, x3 = qx - px, y3 = qy - py;
  ox = l1 * x1 + l2 * x2 + l3 * x3;
  oy = l1 * y1 + l2 * y2 + l3 * y3;
  dx = d1 * x1 + d2 * x2 + d3 * x3;
  dy = d1 * y1 + d2 * y2 + d3 * y3;
}

// edge f of a cell: cubic (bit 4 + f, edge nodes in cub[4 f ..]), arc (bit f) or straight
__device__ inline void cell_edge(int arcs, const double *cub, int f, double px, double py, double qx, double qy,
                                 double u, double &ox, double &oy, double &dx, double &dy) {
  if (arcs & (16 << f)) cubic_offset(px, py, cub + 4 * f, qx, qy, u, ox, oy, dx, dy);
  else edge_offset(px, py, qx, qy, arcs & (1 << f), u, ox, oy, dx, dy);
}

// Transfinite map of a cell with corners c[8] (x0 y0 .. x3 y3, centre
// relative), edge kind bits and cubic edge nodes (or null) at (xi, eta):
// out = x, y, x_xi, y_xi, x_eta, y_eta.  Evaluated about corner 0 (an exact
// shift in real arithmetic), so the round-off of the metrics scales with the
// cell, not with the coordinates.
__device__ inline void cell_map(const double *c, int arcs, const double *cub, double xi, double eta, double *out) {
  const double u1 = c[2] - c[0], v1 = c[3] - c[1];
  const double u2 = c[4] - c[0], v2 = c[5] - c[1];
  const double u3 = c[6] - c[0], v3 = c[7] - c[1];
  double bx, by, dbx, dby, tx, ty, dtx, dty, lx, ly, dlx, dly, rx, ry, drx, dry;
  cell_edge(arcs, cub, 0, c[0], c[1], c[2], c[3], xi, bx, by, dbx, dby);   // f0: n0 -> n1
  cell_edge(arcs, cub, 1, c[2], c[3], c[4], c[5], eta, rx, ry, drx, dry);  // f1: n1 -> n2
  cell_edge(arcs, cub, 2, c[6], c[7], c[4], c[5], xi, tx, ty, dtx, dty);   // f2: n3 -> n2
  cell_edge(arcs, cub, 3, c[0], c[1], c[6], c[7], eta, lx, ly, dlx, dly);  // f3: n0 -> n3
  rx += u1;
  ry += v1;
  tx += u3;
  ty += v3;
  const double a = 1.0 - xi, b = 1.0 - eta;
  // bilinear corner blend (corner 0 at the origin) and its derivatives
  const double cxv = xi * b * u1 + xi * eta * u2 + a * eta * u3;
  const double cyv = xi * b * v1 + xi * eta * v2 + a * eta * v3;
  const double cx_xi = b * u1 + eta * u2 - eta * u3;
  const double cy_xi = b * v1 + eta * v2 - eta * v3;
  const double cx_eta = -xi * u1 + xi * u2 + a * u3;
  const double cy_eta = -xi * v1 + xi * v2 + a * v3;
  out[0] = c[0] + (b * bx + eta * tx + a * lx + xi * rx - cxv);
  out[1] = c[1] + (b * by + eta * ty + a * ly + xi * ry - cyv);
  out[2] = b * dbx + eta * dtx - lx + rx - cx_xi;
  out[3] = b * dby + eta * dty - ly + ry - cy_xi;
  out[4] = -bx + tx + a * dlx + xi * drx - cx_eta;
  out[5] = -by + ty + a * dly + xi * dry - cy_eta;
}

// t = 0 metric tables (one thread per table; table t belongs to element tab_elem[t])
template <typename T, int N>
__global__ void k_geo(MeshDev md, const double *__restrict__ Xs, const double *__restrict__ Xf) {
  using L = GeoLayout<N>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= md.nTab) return;
  const int e = md.tab_elem[t];
  double c[8];
  for (int k = 0; k < 8; ++k) c[k] = md.corners[(size_t)e * 8 + k];
  const double *cub = md.cubic ? md.cubic + (size_t)e * 16 : nullptr;
  const int arcs = md.arcs[e];
  const double om = md.clk0->om[md.zone[e]];
  T *g = (T *)md.geo + (size_t)t * L::G;
  double m[6];
  for (int j = 0; j < N; ++j)
    for (int i = 0; i <= N; ++i) {
      // xi-FP (X_{i+1/2}, X_j)
      cell_map(c, arcs, cub, Xf[i], Xs[j], m);
      const double ax = m[5], ay = -m[4];
      g[L::ax + j * (N + 1) + i] = (T)ax;
      g[L::ay + j * (N + 1) + i] = (T)ay;
      g[L::gx + j * (N + 1) + i] = (T)(om * (-m[1] * ax + m[0] * ay));
      // eta-FP (X_j, X_{i+1/2}) stored at FP row i, column j
      cell_map(c, arcs, cub, Xs[j], Xf[i], m);
      const double bx = -m[3], by = m[2];
      g[L::bx + i * N + j] = (T)bx;
      g[L::by + i * N + j] = (T)by;
      g[L::gy + i * N + j] = (T)(om * (-m[1] * bx + m[0] * by));
    }
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) {
      cell_map(c, arcs, cub, Xs[i], Xs[j], m);
      const double J = m[2] * m[5] - m[4] * m[3];
      g[L::iJ + j * N + i] = (T)(1.0 / J);
      g[L::grad + 0 * N * N + j * N + i] = (T)(m[5] / J);   // xi_x
      g[L::grad + 1 * N * N + j * N + i] = (T)(-m[4] / J);  // xi_y
      g[L::grad + 2 * N * N + j * N + i] = (T)(-m[3] / J);  // eta_x
      g[L::grad + 3 * N * N + j * N + i] = (T)(m[2] / J);   // eta_y
    }
}

// Every cell: positive Jacobian at all SPs and FPs (folded or clockwise cells
// set flag bit 1), and the bilinear record x0, y0, e1 = x1 - x0, e3 = x3 - x0,
// d = x2 - x1 - x3 + x0 (centre-relative, differences formed in FP64) used for
// the on-the-fly metrics of straight cells.
template <typename T, int N>
__global__ void k_egeo(MeshDev md, const double *__restrict__ Xs, const double *__restrict__ Xf) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= md.E) return;
  double c[8], m[6];
  for (int k = 0; k < 8; ++k) c[k] = md.corners[(size_t)e * 8 + k];
  const double *cub = md.cubic ? md.cubic + (size_t)e * 16 : nullptr;
  const int arcs = md.arcs[e];
  bool bad = false;
  for (int j = 0; j < N; ++j) {
    for (int i = 0; i <= N; ++i) {
      cell_map(c, arcs, cub, Xf[i], Xs[j], m);  // xi-FP
      bad |= !(m[2] * m[5] - m[4] * m[3] > 0.0);
      cell_map(c, arcs, cub, Xs[j], Xf[i], m);  // eta-FP
      bad |= !(m[2] * m[5] - m[4] * m[3] > 0.0);
    }
    for (int i = 0; i < N; ++i) {
      cell_map(c, arcs, cub, Xs[i], Xs[j], m);  // SP
      bad |= !(m[2] * m[5] - m[4] * m[3] > 0.0);
    }
  }
  if (bad) atomicOr(&md.clk->flags, 2);
  if (md.egeo) {
    T *r = (T *)md.egeo + (size_t)e * 8;
    r[0] = (T)c[0];
    r[1] = (T)c[1];
    r[2] = (T)(c[2] - c[0]);
    r[3] = (T)(c[3] - c[1]);
    r[4] = (T)(c[6] - c[0]);
    r[5] = (T)(c[7] - c[1]);
    r[6] = (T)((c[4] - c[2]) - (c[6] - c[0]));
    r[7] = (T)((c[5] - c[3]) - (c[7] - c[1]));
  }
}

// t = 0 positions of boundary-face points (wall velocity of the rotating zone)
template <int N>
__global__ void k_bgeo(MeshDev md, const double *__restrict__ Xs, double *bxy) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= md.nB) return;
  const int ef = md.bfaces[b].x, e = ef >> 2, f = ef & 3;
  double c[8], m[6];
  for (int k = 0; k < 8; ++k) c[k] = md.corners[(size_t)e * 8 + k];
  const double *cub = md.cubic ? md.cubic + (size_t)e * 16 : nullptr;
  for (int j = 0; j < N; ++j) {
    const double xi = (f == 0 || f == 2) ? Xs[j] : (f == 1 ? 1.0 : 0.0);
    const double eta = (f == 1 || f == 3) ? Xs[j] : (f == 2 ? 1.0 : 0.0);
    cell_map(c, md.arcs[e], cub, xi, eta, m);
    bxy[((size_t)b * N + j) * 2] = m[0];
    bxy[((size_t)b * N + j) * 2 + 1] = m[1];
  }
}

// physical SP coordinates at time t, [E][N][N][2]
// y = recip(x) in the compute type, one thread per value (test of recip)
template <typename T>
__global__ void k_reciprocal(const double *x, double *y, int n) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y[i] = (double)recip<T>((T)x[i]);
}

template <int N>
__global__ void k_spxy(MeshDev md, const double *__restrict__ Xs, double t, double *out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= md.E) return;
  double c[8], m[6];
  for (int k = 0; k < 8; ++k) c[k] = md.corners[(size_t)e * 8 + k];
  const double *cub = md.cubic ? md.cubic + (size_t)e * 16 : nullptr;
  const int z = md.zone[e], fz = md.frame[e];
  const double cx = md.zpar[4 * fz], cy = md.zpar[4 * fz + 1];
  double cs = 1.0, sn = 0.0;
  if (z) sincos(md.zpar[4 * z + 2] * t, &sn, &cs);
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) {
      cell_map(c, md.arcs[e], cub, Xs[i], Xs[j], m);
      out[(((size_t)e * N + j) * N + i) * 2] = cx + (cs * m[0] - sn * m[1]);
      out[(((size_t)e * N + j) * N + i) * 2 + 1] = cy + (sn * m[0] + cs * m[1]);
    }
}

// The zone table [3][kZT] of a clock record in the compute type: cos theta_z,
// sin theta_z, omega_z of every zone (zone 0: 1, 0, 0).
template <typename T>
__device__ __forceinline__ const T *zone_tab(const DevClock *k) {
  if constexpr (std::is_same<T, double>::value) return k->c;
  else return k->cf;
}

// Metrics of one element at the current rotation of its zone (Sec. 2.3):
// either its t = 0 table rotated by R(theta_z), or, for a straight cell on the
// on-the-fly path, the bilinear map from its rotated record.  The
// grid-velocity coefficient V_g . a is rotation invariant.
template <typename T, int N, bool OTF>
struct ElemGeo {
  using L = GeoLayout<N>;
  const T *tab;
  T c, s, om;
  T x0, y0, e1x, e1y, e3x, e3y, dx, dy;

  // zt: a zone table (zone_tab of the stage's clock, or of the t = 0 clock)
  __device__ __forceinline__ void load(const MeshDev &md, int e, const T *zt) {
    load_rec(md, e, md.eflag[e], OTF ? (const T *)md.egeo + (size_t)e * 8 : nullptr, zt);
  }
  // the same with the flag and the bilinear record already at hand (e.g. in shared memory)
  __device__ __forceinline__ void load_rec(const MeshDev &md, int e, int f, const T *r, const T *zt) {
    const int z = f & kZoneMask;
    c = zt[z];
    s = zt[kZT + z];
    om = zt[2 * kZT + z];
    int ti = ((f & ~kIfaceBit) >> kZoneBits) - 1;
    if (!ssd_check(md, ti < md.nTab && (OTF || ti >= 0))) ti = 0;
    if (OTF && ti < 0) {
      tab = nullptr;
      T v0, v1, v2, v3, v4, v5, v6, v7;
      if constexpr (std::is_same<T, float>::value) {
        // the record is 16-byte aligned (32 bytes per cell, in global or shared memory)
        const float4 a = reinterpret_cast<const float4 *>(r)[0], b = reinterpret_cast<const float4 *>(r)[1];
        v0 = a.x, v1 = a.y, v2 = a.z, v3 = a.w, v4 = b.x, v5 = b.y, v6 = b.z, v7 = b.w;
      } else {
        v0 = r[0], v1 = r[1], v2 = r[2], v3 = r[3], v4 = r[4], v5 = r[5], v6 = r[6], v7 = r[7];
      }
      x0 = mul_sub(c, v0, s, v1);
      y0 = mul_add(s, v0, c, v1);
      e1x = mul_sub(c, v2, s, v3);
      e1y = mul_add(s, v2, c, v3);
      e3x = mul_sub(c, v4, s, v5);
      e3y = mul_add(s, v4, c, v5);
      dx = mul_sub(c, v6, s, v7);
      dy = mul_add(s, v6, c, v7);
    } else {
      tab = (const T *)md.geo + (size_t)ti * L::G;
    }
  }
  // xi-FP (X_{i+1/2}, X_j): a = (y_eta, -x_eta) and V_g . a
  __device__ __forceinline__ void xi_fp(int i, int j, T &vx, T &vy, T &g) const {
    if (OTF && tab == nullptr) {
      const T xi = cVB<T, N>.Xf[i], eta = cVB<T, N>.Xs[j];
      const T xe = e3x + xi * dx, ye = e3y + xi * dy;
      vx = ye;
      vy = -xe;
      g = T(0);
      if (om != T(0)) {
        const T px = x0 + xi * e1x + eta * xe, py = y0 + xi * e1y + eta * ye;
        g = om * mul_sub(px, vy, py, vx);
      }
    } else {
      const int k = j * (N + 1) + i;
      const T ax = tab[L::ax + k], ay = tab[L::ay + k];
      vx = mul_sub(c, ax, s, ay);
      vy = mul_add(s, ax, c, ay);
      g = tab[L::gx + k];
    }
  }
  // eta-FP (X_i, X_{l+1/2}): b = (-y_xi, x_xi) and V_g . b
  __device__ __forceinline__ void eta_fp(int i, int l, T &vx, T &vy, T &g) const {
    if (OTF && tab == nullptr) {
      const T xi = cVB<T, N>.Xs[i], eta = cVB<T, N>.Xf[l];
      const T xx = e1x + eta * dx, yx = e1y + eta * dy;
      vx = -yx;
      vy = xx;
      g = T(0);
      if (om != T(0)) {
        const T px = x0 + eta * e3x + xi * xx, py = y0 + eta * e3y + xi * yx;
        g = om * mul_sub(px, vy, py, vx);
      }
    } else {
      const int k = l * N + i;
      const T bx = tab[L::bx + k], by = tab[L::by + k];
      vx = mul_sub(c, bx, s, by);
      vy = mul_add(s, bx, c, by);
      g = tab[L::gy + k];
    }
  }
  // Metric vectors and V_g . a at the interior FPs 1..N-1 of SP line m in
  // direction d (0: xi line at eta = X_m, 1: eta line at xi = X_m), into
  // vx/vy/vg[1..N-1].  On straight cells both directions share one form:
  // with the line's coordinate u = X_{i+1/2}, the tangent of the cross
  // direction is t = A + u d (A = e3 for xi lines, e1 for eta lines), the
  // vector is (t_y, -t_x) or (-t_y, t_x), and the point is x0 + u B + X_m t
  // (B = e1 or e3); no branch depends on the FP.
  __device__ __forceinline__ void line_metrics(int d, int m, T *vx, T *vy, T *vg) const {
    if (OTF && tab == nullptr) {
      const T Ax = d == 0 ? e3x : e1x, Ay = d == 0 ? e3y : e1y;
      const T Bx = d == 0 ? e1x : e3x, By = d == 0 ? e1y : e3y;
      const T sg = d == 0 ? T(1) : T(-1), w = cVB<T, N>.Xs[m];
#pragma unroll
      for (int i = 1; i < N; ++i) {
        const T u = cVB<T, N>.Xf[i];
        const T tx = Ax + u * dx, ty = Ay + u * dy;
        vx[i] = sg * ty;
        vy[i] = -sg * tx;
        const T px = x0 + u * Bx + w * tx, py = y0 + u * By + w * ty;
        vg[i] = om * mul_sub(px, vy[i], py, vx[i]);
      }
    } else {
#pragma unroll
      for (int i = 1; i < N; ++i) {
        if (d == 0) xi_fp(i, m, vx[i], vy[i], vg[i]);
        else eta_fp(m, i, vx[i], vy[i], vg[i]);
      }
    }
  }
  // metric vector of the end FP at point j of face f
  __device__ __forceinline__ void face(int f, int j, T &vx, T &vy, T &g) const {
    if (f == 1) xi_fp(N, j, vx, vy, g);
    else if (f == 3) xi_fp(0, j, vx, vy, g);
    else if (f == 0) eta_fp(j, 0, vx, vy, g);
    else eta_fp(j, N, vx, vy, g);
  }
  // 1 / |J| at SP (X_i, X_j)
  __device__ __forceinline__ T inv_jac(int i, int j) const {
    if (OTF && tab == nullptr) {
      const T xi = cVB<T, N>.Xs[i], eta = cVB<T, N>.Xs[j];
      const T xx = e1x + eta * dx, yx = e1y + eta * dy, xe = e3x + xi * dx, ye = e3y + xi * dy;
      return recip(mul_sub(xx, ye, xe, yx));
    }
    return tab[L::iJ + j * N + i];
  }
  // 1 / |J| at SP (X_i, X_j) straight from the cell flag and the unrotated
  // record or table (|J| does not change under the rotation)
  static __device__ __forceinline__ T inv_jac_t0(const MeshDev &md, int f, const T *r, int i, int j) {
    const int ti = ((f & ~kIfaceBit) >> kZoneBits) - 1;
    if (OTF && ti < 0) {
      const T xi = cVB<T, N>.Xs[i], eta = cVB<T, N>.Xs[j];
      T r2, r3, r4, r5, r6, r7;
      if constexpr (std::is_same<T, float>::value) {
        const float4 a = reinterpret_cast<const float4 *>(r)[0], b = reinterpret_cast<const float4 *>(r)[1];
        r2 = a.z, r3 = a.w, r4 = b.x, r5 = b.y, r6 = b.z, r7 = b.w;
      } else {
        r2 = r[2], r3 = r[3], r4 = r[4], r5 = r[5], r6 = r[6], r7 = r[7];
      }
      const T xx = r2 + eta * r6, yx = r3 + eta * r7, xe = r4 + xi * r6, ye = r5 + xi * r7;
      return recip(mul_sub(xx, ye, xe, yx));
    }
    return ((const T *)md.geo + (size_t)ti * L::G)[L::iJ + j * N + i];
  }
  // gradients of xi and eta at SP (X_i, X_j): (xi_x, xi_y), (eta_x, eta_y)
  __device__ __forceinline__ void sp_grad(int i, int j, T &xix, T &xiy, T &etx, T &ety) const {
    if (OTF && tab == nullptr) {
      const T xi = cVB<T, N>.Xs[i], eta = cVB<T, N>.Xs[j];
      const T xx = e1x + eta * dx, yx = e1y + eta * dy, xe = e3x + xi * dx, ye = e3y + xi * dy;
      const T iJ = T(1) / mul_sub(xx, ye, xe, yx);
      xix = ye * iJ;
      xiy = -xe * iJ;
      etx = -yx * iJ;
      ety = xx * iJ;
    } else {
      const int k = j * N + i;
      const T a = tab[L::grad + k], b = tab[L::grad + N * N + k];
      const T c2 = tab[L::grad + 2 * N * N + k], d2 = tab[L::grad + 3 * N * N + k];
      xix = mul_sub(c, a, s, b);
      xiy = mul_add(s, a, c, b);
      etx = mul_sub(c, c2, s, d2);
      ety = mul_add(s, c2, c, d2);
    }
  }
};

// ---------------------------------------------------------------------------
// physics (Sec. 2)
// ---------------------------------------------------------------------------

// pressure from the conservative state with ir = 1 / rho at hand
template <typename T>
__device__ __forceinline__ T pressure_ir(const T *q, T ir, T gm1) {
  return gm1 * fma(-(T(0.5) * mul_add(q[1], q[1], q[2], q[2])), ir, q[3]);
}

template <typename T>
__device__ __forceinline__ T pressure_of(const T *q, T gm1) {
  return pressure_ir(q, recip(q[0]), gm1);
}

// normal ALE inviscid flux through a (not necessarily unit) vector (nx, ny):
// (F - u_g Q, G - v_g Q) . n  with vgn = V_g . n, ir = 1 / rho
template <typename T>
__device__ __forceinline__ void normal_flux_ir(const T *q, T ir, T p, T nx, T ny, T vgn, T *f) {
  const T un = mul_add(q[1], nx, q[2], ny) * ir;
  f[0] = mul_sub(q[0], un, vgn, q[0]);
  f[1] = fma(q[1], un, mul_sub(p, nx, vgn, q[1]));
  f[2] = fma(q[2], un, mul_sub(p, ny, vgn, q[2]));
  f[3] = mul_sub(q[3] + p, un, vgn, q[3]);
}

template <typename T>
__device__ __forceinline__ void normal_flux(const T *q, T p, T nx, T ny, T vgn, T *f) {
  normal_flux_ir(q, recip(q[0]), p, nx, ny, vgn, f);
}

// Rusanov common flux (Sec. 3.1) for unit normal n from L to R; one
// reciprocal density per side
template <typename T>
__device__ __forceinline__ void rusanov(const T *qL, const T *qR, T nx, T ny, T vgn, T gamma, T *Fn) {
  const T gm1 = gamma - T(1);
  const T irL = recip(qL[0]), irR = recip(qR[0]);
  const T pL = pressure_ir(qL, irL, gm1), pR = pressure_ir(qR, irR, gm1);
  T fL[4], fR[4];
  normal_flux_ir(qL, irL, pL, nx, ny, vgn, fL);
  normal_flux_ir(qR, irR, pR, nx, ny, vgn, fR);
  const T unL = mul_add(qL[1], nx, qL[2], ny) * irL, unR = mul_add(qR[1], nx, qR[2], ny) * irR;
  const T lL = fabs(unL - vgn) + sqrt(gamma * pL * irL);
  const T lR = fabs(unR - vgn) + sqrt(gamma * pR * irR);
  const T lam = lL > lR ? lL : lR;
#pragma unroll
  for (int v = 0; v < 4; ++v) Fn[v] = mul_sub(T(0.5), fL[v] + fR[v], T(0.5) * lam, qR[v] - qL[v]);
}

// ---------------------------------------------------------------------------
// per-stage coupling kernels
// ---------------------------------------------------------------------------

// Double-double angles (an unevaluated sum hi + lo, |lo| <= ulp(hi) / 2) for
// the sliding interface: a mortar offset o = (phi_m - phi_f) / width is a
// difference of two angles near pi divided by a small width, so the absolute
// round-off of FP64 angles (~1e-16) becomes ~1e-14 in o and reaches the
// residual of the interface cells amplified by the flux-derivative weights.
// The t = 0 face angles come from the host in long double; the rotation
// angle omega t is formed exactly and reduced with a double-double 2 pi.
struct ddang {
  double hi, lo;
};

// 2 pi = kTwoPiHi + kTwoPiLo to about 1e-32
constexpr double kTwoPiHi = 6.283185307179586476925286766559;
constexpr double kTwoPiLo = 2.4492935982947064e-16;

// s + e = a + b exactly (Knuth's two-sum)
__device__ __forceinline__ ddang dd_two_sum(double a, double b) {
  const double s = a + b;
  const double bb = s - a;
  return ddang{s, (a - (s - bb)) + (b - bb)};
}

__device__ __forceinline__ ddang dd_add(ddang a, ddang b) {
  const ddang s = dd_two_sum(a.hi, b.hi);
  const double lo = s.lo + (a.lo + b.lo);
  const double hi = s.hi + lo;
  return ddang{hi, lo - (hi - s.hi)};
}

__device__ __forceinline__ ddang dd_sub(ddang a, ddang b) { return dd_add(a, ddang{-b.hi, -b.lo}); }

__device__ __forceinline__ bool dd_lt(ddang a, ddang b) { return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo); }
__device__ __forceinline__ bool dd_le(ddang a, ddang b) { return a.hi < b.hi || (a.hi == b.hi && a.lo <= b.lo); }

// into [0, 2 pi) for an angle in [-2 pi, 4 pi)
__device__ __forceinline__ ddang dd_wrap_2pi(ddang a) {
  const ddang tp{kTwoPiHi, kTwoPiLo};
  if (dd_lt(a, ddang{0.0, 0.0})) return dd_add(a, tp);
  if (!dd_lt(a, tp)) return dd_sub(a, tp);
  return a;
}

// theta = omega t reduced to [0, 2 pi) as a double-double: the product is
// exact (p + e, with the FMA), k = floor(p / 2 pi) turns are taken off with
// the exact product k kTwoPiHi and k kTwoPiLo
constexpr double kInvTwoPi = 0.15915494309189535;  // 1 / (2 pi), rounded
__device__ __forceinline__ ddang dd_rotation_angle(double om, double t) {
  const double p = om * t;
  const double e = fma(om, t, -p);
  // any integer k near p / 2 pi will do: the reduction below is exact for it
  // and the final wrap brings the angle into [0, 2 pi)
  const double k = floor(p * kInvTwoPi);
  const double kh = k * kTwoPiHi;
  const double kl = fma(k, kTwoPiHi, -kh);
  const ddang r = dd_two_sum(p, -kh);
  const double small = (e - kl) - k * kTwoPiLo;
  const double lo = r.lo + small;
  const double hi = r.hi + lo;
  return dd_wrap_2pi(ddang{hi, lo - (hi - r.hi)});
}

// Stage clock and mortar table of interface ii (Sec. 3.2: connectivity
// updated at every stage).  Its mortar k is the interval between merged node
// positions k and k+1 (counter-clockwise, cyclic); nodes of both sides sorted
// by angle, L before R on ties.  One CTA per interface; the node angles
// (double-double) are searched in shared memory (dynamic, 2 (nL + nR) doubles
// of the interface: high parts, then low parts); work_i / work_d hold the
// merged positions and angles.  The CTA of interface 0 also writes the stage
// clock of every zone: theta_z = omega_z t_stage.  The offsets and scales of
// Eq. xz of each mortar against its faces are formed here too, for the mortar
// flux kernels of the stage.  The step's start time t_n is read from *tsrc
// (ahead: the next step's, t_n + dt, formed as k_advance forms it); the stage
// clock and the tables are written through md.
static __device__ void clock_merge_body(const MeshDev &md, int ii, double c, double dt, int *work_i,
                                        double *work_d, const DevClock *tsrc, bool ahead = false) {
  extern __shared__ double s_ang[];  // [nb] high parts (rotated L, then R), [nb] low parts
  __shared__ double s_th2, s_th2lo;
  __shared__ int s_k0;
  const double t0 = ahead ? tsrc->t_n + dt : tsrc->t_n;
  const double ts = t0 + c * dt;
  // the zone clocks on warp 1, beside warp 0's angle of this interface
  if (ii == 0 && threadIdx.x >= 32 && threadIdx.x < 32 + kZT) {
    DevClock *k = md.clk;
    const int z = threadIdx.x - 32;
    const double om = z ? md.zpar[4 * z + 2] : 0.0;
    double sn = 0.0, cs = 1.0;
    ddang th{0.0, 0.0};
    if (z) {
      th = dd_rotation_angle(om, ts);
      double sh, ch;
      sincos(th.hi, &sh, &ch);
      // R(theta) of the double-double angle: first order in the low part
      cs = ch - sh * th.lo;
      sn = sh + ch * th.lo;
    } else {
      k->t_stage = ts;
    }
    k->theta2[z] = th.hi;
    k->theta2_lo[z] = th.lo;
    k->c[z] = cs;
    k->s[z] = sn;
    k->om[z] = om;
    k->cf[z] = (float)cs;
    k->sf[z] = (float)sn;
    k->omf[z] = (float)om;
  }
  const int Lo = md.zoff[ii], Ro = md.zoff[kZT + ii];
  const int nL = md.zoff[ii + 1] - Lo, nR = md.zoff[kZT + ii + 1] - Ro, nb = nL + nR;
  const int Mo = Lo + Ro;
  if (threadIdx.x == 0) {
    const ddang th = dd_rotation_angle(md.zpar[4 * (ii + 1) + 2], ts);
    s_th2 = th.hi;
    s_th2lo = th.lo;
    s_k0 = 0;
  }
  __syncthreads();
  if (nL == 0) return;
  const ddang th2{s_th2, s_th2lo};
  double *sLh = s_ang, *sRh = s_ang + nL, *sLl = s_ang + nb, *sRl = s_ang + nb + nL;
  for (int k = threadIdx.x; k < nL; k += blockDim.x) {
    const ddang a = dd_wrap_2pi(dd_add(ddang{md.La[Lo + k], md.La_lo[Lo + k]}, th2));
    sLh[k] = a.hi;
    sLl[k] = a.lo;
  }
  for (int k = threadIdx.x; k < nR; k += blockDim.x) {
    sRh[k] = md.Ra[Ro + k];
    sRl[k] = md.Ra_lo[Ro + k];
  }
  __syncthreads();
  // rotated L angles are a cyclic shift of an ascending list; k0 = index of the minimum
  for (int k = threadIdx.x; k < nL; k += blockDim.x) {
    const int kp = k == 0 ? nL - 1 : k - 1;
    if (dd_lt(ddang{sLh[k], sLl[k]}, ddang{sLh[kp], sLl[kp]})) s_k0 = k;
  }
  __syncthreads();
  const int k0 = s_k0;
  const int nMall = md.nM;
  double *mAh = work_d + Mo;          // [nb] merged angles: high parts
  double *mAl = work_d + nMall + Mo;  // and low parts
  int *posL = work_i + 2 * Mo;    // [nL] merged position of L node k (t = 0 index)
  int *posR = posL + nL;          // [nR]
  int *otherL = posL + nb;        // [nL] R face containing the mortar that starts at L node k
  int *otherR = otherL + nL;      // [nR] L face containing the mortar that starts at R node k
  for (int k = threadIdx.x; k < nL; k += blockDim.x) {
    const ddang a{sLh[k], sLl[k]};
    const int rank = (k - k0 + nL) % nL;
    int lo = 0, hi = nR;  // number of R angles strictly below a
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (dd_lt(ddang{sRh[mid], sRl[mid]}, a)) lo = mid + 1; else hi = mid;
    }
    const int p = rank + lo;
    posL[k] = p;
    mAh[p] = a.hi;
    mAl[p] = a.lo;
    otherL[k] = lo == 0 ? nR - 1 : lo - 1;
  }
  for (int k = threadIdx.x; k < nR; k += blockDim.x) {
    const ddang a{sRh[k], sRl[k]};
    int lo = 0, hi = nL;  // number of rotated L angles <= a (L first on ties)
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      int idx = k0 + mid;
      if (idx >= nL) idx -= nL;
      if (dd_le(ddang{sLh[idx], sLl[idx]}, a)) lo = mid + 1; else hi = mid;
    }
    const int p = k + lo;
    posR[k] = p;
    mAh[p] = a.hi;
    mAl[p] = a.lo;
    otherR[k] = lo == 0 ? (k0 + nL - 1) % nL : (k0 + lo - 1) % nL;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nL; k += blockDim.x) {
    const int p = posL[k];
    md.mLf[Mo + p] = Lo + k;
    md.mRf[Mo + p] = Ro + otherL[k];
    const int cnt = (posL[k + 1 == nL ? 0 : k + 1] - p + nb) % nb;
    md.Lstart[Lo + k] = Mo + p;
    md.Lcount[Lo + k] = cnt == 0 ? nb : cnt;
  }
  for (int k = threadIdx.x; k < nR; k += blockDim.x) {
    const int p = posR[k];
    md.mRf[Mo + p] = Ro + k;
    md.mLf[Mo + p] = Lo + otherR[k];
    const int cnt = (posR[k + 1 == nR ? 0 : k + 1] - p + nb) % nb;
    md.Rstart[Ro + k] = Mo + p;
    md.Rcount[Ro + k] = cnt == 0 ? nb : cnt;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < nb; p += blockDim.x) {
    const ddang a{mAh[p], mAl[p]};
    const ddang b = p + 1 < nb ? ddang{mAh[p + 1], mAl[p + 1]}
                               : dd_add(ddang{mAh[0], mAl[0]}, ddang{kTwoPiHi, kTwoPiLo});
    const ddang d = dd_sub(b, a);
    md.mgeo[4 * (Mo + p)] = a.hi;
    md.mgeo[4 * (Mo + p) + 1] = a.lo;
    md.mgeo[4 * (Mo + p) + 2] = d.hi + d.lo;
    md.mgeo[4 * (Mo + p) + 3] = 0.0;
  }
}

// Eq. xz of mortar m against its face on side sd (0: L, 1: R) of a stage
// whose merge has run: the offset of the mortar's start from the face's
// start angle (the L face's turned by its zone's stage angle), a
// double-double difference taken into (-pi, pi], and the mortar's length,
// both over the face's angular width.  One thread per (mortar, side), so the
// FP64 work spreads over many SMs.
static __device__ __forceinline__ void mortar_xz_body(const MeshDev &md, int t) {
  if (t >= 2 * md.nM) return;
  const int sd = t >= md.nM, m = t - sd * md.nM;
  const double pi = 0.5 * kTwoPiHi;
  const ddang m0d{md.mgeo[4 * m], md.mgeo[4 * m + 1]};
  const double dm = md.mgeo[4 * m + 2];
  const int fq = sd ? md.mRf[m] : md.mLf[m];
  MortSide ms{};
  if (ssd_check(md, fq >= 0 && fq < (sd ? md.nR : md.nL))) {
    ddang fa{md.Ra[fq], md.Ra_lo[fq]};
    if (!sd) {
      // interface ifz[fq] belongs to zone ifz[fq] + 1
      const int z = md.ifz[fq] + 1;
      fa = dd_wrap_2pi(dd_add(ddang{md.La[fq], md.La_lo[fq]}, ddang{md.clk->theta2[z], md.clk->theta2_lo[z]}));
    }
    ddang offd = dd_sub(m0d, fa);
    if (offd.hi > pi) offd = dd_sub(offd, ddang{kTwoPiHi, kTwoPiLo});
    if (offd.hi <= -pi) offd = dd_add(offd, ddang{kTwoPiHi, kTwoPiLo});
    const double off = offd.hi + offd.lo;
    const double iw = sd ? md.RiW[fq] : md.LiW[fq];
    const int4 fc = sd ? md.Rface[fq] : md.Lface[fq];
    ms.o = off * iw;
    ms.s = dm * iw;
    ms.fa_hi = fa.hi;
    ms.fa_lo = fa.lo;
    ms.w = sd ? md.Rw[fq] : md.Lw[fq];
    ms.ef = fc.x;
    ms.rev = fc.y;
  }
  md.msd[t] = ms;
}

constexpr int kXzBlock = 128;

static __global__ void __launch_bounds__(kXzBlock) k_mortar_xz(MeshDev md) {
  pdl_enter();
  mortar_xz_body(md, blockIdx.x * kXzBlock + threadIdx.x);
}

// block (0, ii): interface ii of one stage
static __global__ void k_clock_merge(MeshDev md, double c, double dt, int *work_i, double *work_d) {
  pdl_enter();
  clock_merge_body(md, blockIdx.y, c, dt, work_i, work_d, md.clk);
}

// block (x, ii): the clock and interface ii's mortar table of stage b = b0 + x
// of a step (ahead: of the next step)
static __global__ void k_clock_merge_stages(MeshDev md, StageMerge sm, double dt, int b0, int ahead) {
  pdl_enter();
  const int b = b0 + (int)blockIdx.x;
  MeshDev m = md;
  m.clk = sm.clk[b];
  m.mLf = sm.mLf[b];
  m.mRf = sm.mRf[b];
  m.Lstart = sm.Lstart[b];
  m.Lcount = sm.Lcount[b];
  m.Rstart = sm.Rstart[b];
  m.Rcount = sm.Rcount[b];
  m.mgeo = sm.mgeo[b];
  clock_merge_body(m, blockIdx.y, sm.c[b], dt, sm.work_i[b], sm.work_d[b], md.clk, ahead != 0);
}

// block (x, y): Eq. xz of mortars [x kXzBlock / 2 ...) of stage b0 + y
static __global__ void __launch_bounds__(kXzBlock) k_mortar_xz_stages(MeshDev md, StageMerge sm, int b0) {
  pdl_enter();
  const int b = b0 + (int)blockIdx.y;
  MeshDev m = md;
  m.clk = sm.clk[b];
  m.mLf = sm.mLf[b];
  m.mRf = sm.mRf[b];
  m.mgeo = sm.mgeo[b];
  m.msd = sm.msd[b];
  mortar_xz_body(m, blockIdx.x * kXzBlock + threadIdx.x);
}

// t = 0 geometry of every conforming / periodic face point (one thread per point)
template <typename T, int N, bool OTF>
__global__ void k_fgeo(MeshDev md) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= md.nF * N) return;
  const int fi = t / N, j = t - fi * N;
  const int4 fc = md.faces[fi];
  const int efA = fc.x, efB = fc.y, jB = fc.z ? N - 1 - j : j;
  ElemGeo<T, N, OTF> GA, GB;
  GA.load(md, efA >> 2, zone_tab<T>(md.clk0));
  GB.load(md, efB >> 2, zone_tab<T>(md.clk0));
  T ax, ay, ag, bx, by, bg;
  GA.face(efA & 3, j, ax, ay, ag);
  GB.face(efB & 3, jB, bx, by, bg);
  const T SA = sqrt(ax * ax + ay * ay), SB = sqrt(bx * bx + by * by);
  const T sgA = (T)face_sigma(efA & 3), sgB = (T)face_sigma(efB & 3);
  T *g = (T *)md.fgeo + (size_t)fi * 5 * N;
  g[0 * N + j] = sgA * ax / SA;
  g[1 * N + j] = sgA * ay / SA;
  g[2 * N + j] = sgA * SA;
  g[3 * N + j] = sgB * SB;
  g[4 * N + j] = sgA * ag / SA;
}

// Conforming and periodic faces: one thread per face point; geometry from the
// t = 0 face table, the normal turned by R(theta_z) on rotating zone z (both
// sides of a conforming face lie in one zone).
template <typename T, int N, bool OTF>
__device__ __forceinline__ void k_face_point(const MeshDev &md, int t) {
  const int fi = t / N, j = t - fi * N;
  const int4 fc = md.faces[fi];
  const int efA = fc.x, efB = fc.y, jB = fc.z ? N - 1 - j : j;
  if (!ssd_check(md, efA >= 0 && efA < 4 * md.E && efB >= 0 && efB < 4 * md.E)) return;
  const T *TR = (const T *)md.TR;
  T qA[4], qB[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    qA[v] = TR[((size_t)efA * 4 + v) * N + j];
    qB[v] = TR[((size_t)efB * 4 + v) * N + jB];
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
  T Fn[4];
  rusanov(qA, qB, nx, ny, vgn, pick<T>(md.gamma, md.gamma_f), Fn);
  T *CF = (T *)md.CF;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    CF[((size_t)efA * 4 + v) * N + j] = sA * Fn[v];
    CF[((size_t)efB * 4 + v) * N + jB] = -sB * Fn[v];
  }
}

// conservative state from density, velocity and pressure
template <typename T>
__device__ __forceinline__ void from_primitive(T rho, T u, T v, T p, T gm1, T *q) {
  q[0] = rho;
  q[1] = rho * u;
  q[2] = rho * v;
  q[3] = p / gm1 + T(0.5) * rho * mul_add(u, u, v, v);
}

// Boundary conditions (Secs. 4.2-4.3 name them; these are the readings): the
// ghost state qg entering the Rusanov flux and the state qb on the boundary,
// the common solution of the viscous terms.  (ug, vg) is the grid velocity at
// the point, (nx, ny) the outward unit normal.
//   WALL   ghost velocity 2 V_g - V, wall temperature, interior pressure; qb has V_g
//   ADIABATIC  the same with the interior temperature; its viscous flux
//          carries no heat conduction
//   SLIP   normal velocity relative to the wall mirrored (qb: removed),
//          interior density and pressure
//   INLET  the free stream
//   OUTLET interior density and velocity, free-stream pressure
template <typename T>
__device__ __forceinline__ void boundary_states(const MeshDev &md, int tag, const T *q, T ug, T vg, T nx, T ny, T *qg,
                                                T *qb) {
  const T gm1 = pick<T>(md.gm1, md.gm1_f);
  const T p = pressure_of(q, gm1);
  const T u = q[1] / q[0], v = q[2] / q[0];
  if (tag == SD_BC_WALL || tag == SD_BC_ADIABATIC) {
    const T rho = tag == SD_BC_WALL ? p / pick<T>(md.RTw, md.RTw_f) : q[0];
    from_primitive(rho, T(2) * ug - u, T(2) * vg - v, p, gm1, qg);
    from_primitive(rho, ug, vg, p, gm1, qb);
  } else if (tag == SD_BC_SLIP) {
    const T wn = mul_add(u - ug, nx, v - vg, ny);
    from_primitive(q[0], u - T(2) * wn * nx, v - T(2) * wn * ny, p, gm1, qg);
    from_primitive(q[0], u - wn * nx, v - wn * ny, p, gm1, qb);
  } else if (tag == SD_BC_INLET) {
    const T ri = pick<T>(md.rho_inf, md.rho_inf_f), ui = pick<T>(md.u_inf, md.u_inf_f);
    const T vi = pick<T>(md.v_inf, md.v_inf_f), pi = pick<T>(md.p_inf, md.p_inf_f);
    from_primitive(ri, ui, vi, pi, gm1, qg);
    from_primitive(ri, ui, vi, pi, gm1, qb);
  } else {
    from_primitive(q[0], u, v, pick<T>(md.p_inf, md.p_inf_f), gm1, qg);
    from_primitive(q[0], u, v, pick<T>(md.p_inf, md.p_inf_f), gm1, qb);
  }
}

// Geometry of boundary point (b, j) at the current rotation: outward unit
// normal, |S| with the face sign, normal grid velocity and the grid velocity
// (from the t = 0 position of the point, rotated).
template <typename T, int N, bool OTF>
__device__ __forceinline__ void bface_geom(const MeshDev &md, int b, int j, T &nx, T &ny, T &sS, T &vgn, T &ug,
                                           T &vg) {
  const int ef = md.bfaces[b].x, e = ef >> 2, f = ef & 3;
  ElemGeo<T, N, OTF> G;
  G.load(md, e, zone_tab<T>(md.clk));
  T ax, ay, ag;
  G.face(f, j, ax, ay, ag);
  double uw = 0.0, vw = 0.0;
  const int z = md.eflag[e] & kZoneMask;
  if (z) {
    // wall velocity omega_z x (R(theta_z) x0), x0 relative to the zone's centre
    const double c = md.clk->c[z], s = md.clk->s[z], om = md.clk->om[z];
    const double x0 = md.bxy[((size_t)b * N + j) * 2], y0 = md.bxy[((size_t)b * N + j) * 2 + 1];
    uw = -om * mul_add(s, x0, c, y0);
    vw = om * mul_sub(c, x0, s, y0);
  }
  const T S = sqrt(mul_add(ax, ax, ay, ay)), sg = (T)face_sigma(f);
  nx = sg * ax / S;
  ny = sg * ay / S;
  vgn = sg * ag / S;
  sS = sg * S;
  ug = (T)uw;
  vg = (T)vw;
}

// Boundary faces: Rusanov through the ghost state of the face's condition.
template <typename T, int N, bool OTF>
__device__ __forceinline__ void k_bface_point(const MeshDev &md, int t) {
  const int b = t / N, j = t - b * N;
  const int4 bf = md.bfaces[b];
  const int ef = bf.x;
  if (!ssd_check(md, ef >= 0 && ef < 4 * md.E)) return;
  const T *TR = (const T *)md.TR;
  T q[4], qg[4], qb[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) q[v] = TR[((size_t)ef * 4 + v) * N + j];
  T nx, ny, sS, vgn, ug, vg;
  bface_geom<T, N, OTF>(md, b, j, nx, ny, sS, vgn, ug, vg);
  boundary_states(md, bf.y, q, ug, vg, nx, ny, qg, qb);
  T Fn[4];
  rusanov(q, qg, nx, ny, vgn, pick<T>(md.gamma, md.gamma_f), Fn);
  T *CF = (T *)md.CF;
#pragma unroll
  for (int v = 0; v < 4; ++v) CF[((size_t)ef * 4 + v) * N + j] = sS * Fn[v];
}

// One launch for all face points of a stage: threads [0, nF N) take the
// conforming and periodic faces, the next nB N threads the boundary faces.
template <typename T, int N, bool OTF>
__global__ void k_faces(MeshDev md) {
  pdl_enter();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < md.nF * N) k_face_point<T, N, OTF>(md, t);
  else if (t < (md.nF + md.nB) * N) k_bface_point<T, N, OTF>(md, t - md.nF * N);
}

// Mortar coupling of Sec. 3.2.  Thread (mortar, side, p): p is a quadrature
// point or a basis index depending on the phase.  Projections use the N-point
// Gauss-Legendre rule, exact for the degree 2N-2 integrands of Eqs. mortarM
// and mortarS; the (o, s)-dependent Lagrange values are FP64.
template <int N>
struct MortCfg {
  static constexpr int MPB = (128 / (2 * N)) > 0 ? 128 / (2 * N) : 1;
  static constexpr int THREADS = MPB * 2 * N;
};

// RUSANOV: inviscid common flux; AVG_Q: common solution (average); RUSANOV_FV:
// the inviscid common flux plus the average of both sides' viscous normal
// fluxes, both projected in one pass and back-projected as one sum (the
// back-projection is linear, Eq. prjF2)
enum { MORTAR_RUSANOV = 0, MORTAR_AVG_Q = 1, MORTAR_RUSANOV_FV = 2 };

// cos and sin of an angle formed in FP64 (an interface normal), evaluated in
// the compute type: in double on the FP64 path; on the FP32 path in float from
// the angle rounded to float (its absolute error, ~2.4e-7 over [0, 2 pi), is
// below the FP32 form's own round-off of the fluxes the normal multiplies)
template <typename T>
__device__ __forceinline__ void normal_of(double ang, T &cs, T &sn) {
  if constexpr (std::is_same<T, float>::value) {
    sincosf((float)ang, &sn, &cs);
  } else {
    sincos(ang, &sn, &cs);
  }
}

// The mortar flux of MPB mortars of block blk: thread (mortar lm < MPB, side,
// point); threads beyond MPB * 2 N only take part in the barriers.
template <typename T, int N, int MMODE, int MPB>
__device__ __forceinline__ void mortar_flux_body(const MeshDev &md, int blk) {
  constexpr int NV = MMODE == MORTAR_RUSANOV_FV ? 8 : 4;  // projected values per point
  // h_i(o + s z_q) and w_q h_i(o + s z_q) [q][i]: formed in FP64, stored in
  // the compute type once
  __shared__ T sH[MPB][2][N][N];
  __shared__ T sWH[MPB][2][N][N];
  __shared__ T sQf[MPB][2][NV][N];     // face values, CCW order (+ viscous normal flux)
  __shared__ T sA[MPB][2][NV][N];      // work arrays
  __shared__ T sB[MPB][2][NV][N];
  __shared__ T sF[MPB][4][N];          // common mortar flux at mortar SPs
  __shared__ T sFz[MPB][4][N];         // common flux at quadrature points
  const int lm = threadIdx.x / (2 * N);
  const int r = threadIdx.x - lm * 2 * N;
  const int sd = r / N, p = r - sd * N;
  const int m = blk * MPB + lm;
  const bool act = lm < MPB && m < md.nM;
  const MortBasis<N> &B = cMB<N>;
  double o = 0.0, s = 0.0;
  int ef = 0, rev = 0;
  double m0 = 0.0, dm = 0.0;
  if (act) {
    // Eq. xz: offset and scale of this mortar against its face on side sd,
    // formed by the stage's merge
    const MortSide ms = md.msd[(size_t)sd * md.nM + m];
    m0 = md.mgeo[4 * m];
    dm = md.mgeo[4 * m + 2];
    o = ms.o;
    s = ms.s;
    ef = ms.ef;
    rev = ms.rev;
    if (!ssd_check(md, ef >= 0 && ef < 4 * md.E)) ef = 0;
    const int jj = rev ? N - 1 - p : p;
    if (MMODE == MORTAR_RUSANOV_FV) {
      // viscous normal flux of this face point with the common solution and
      // the face's own gradient, along the radial normal (from L to R)
      const T *CQ = (const T *)md.CQ, *GT = (const T *)md.GTR;
      T q[4], g8[8], fn[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) q[v] = CQ[((size_t)ef * 4 + v) * N + jj];
#pragma unroll
      for (int c = 0; c < 8; ++c) g8[c] = GT[((size_t)ef * 8 + c) * N + jj];
      T sn, cs;
      normal_of<T>(ms.fa_hi + (ms.fa_lo + B.Xs[p] * ms.w), cs, sn);
      viscous_normal(q, g8, cs, sn, md, fn);
#pragma unroll
      for (int v = 0; v < 4; ++v) sQf[lm][sd][NV - 4 + v][p] = fn[v];
    }
    {
      const T *TR = (const T *)md.TR;
#pragma unroll
      for (int v = 0; v < 4; ++v) sQf[lm][sd][v][p] = TR[((size_t)ef * 4 + v) * N + jj];
    }
    // Lagrange values at the mapped quadrature point x = o + s z_p: x and its
    // distances to the SPs in FP64 (they cancel), the products in the compute
    // type (on the FP32 path each weight is then good to a few float ulps)
    const double x = fma(s, B.zq[p], o);
    T dif[N];
#pragma unroll
    for (int k = 0; k < N; ++k) dif[k] = (T)(x - B.Xs[k]);
#pragma unroll
    for (int i = 0; i < N; ++i) {
      T h = (T)B.cden[i];
#pragma unroll
      for (int k = 0; k < N; ++k)
        if (k != i) h *= dif[k];
      sH[lm][sd][p][i] = h;
      sWH[lm][sd][p][i] = (T)B.wq[p] * h;
    }
  }
  __syncthreads();
  // (A) face polynomial at the mapped quadrature points
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T acc = 0;
#pragma unroll
      for (int i = 0; i < N; ++i) acc += sQf[lm][sd][v][i] * sH[lm][sd][p][i];
      sA[lm][sd][v][p] = acc;
    }
  }
  __syncthreads();
  // (B) right-hand side of Eq. prjQ1: (S^T Q)_p = sum_q w_q h_p(z_q) Q(o + s z_q)
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T acc = 0;
#pragma unroll
      for (int q = 0; q < N; ++q) acc += pick<T>(B.wHz[q * N + p], B.wHz_f[q * N + p]) * sA[lm][sd][v][q];
      sB[lm][sd][v][p] = acc;
    }
  }
  __syncthreads();
  // (C) Q^Xi = M^{-1} S^T Q^Omega (Eq. prjQ2)
  if (act) {
#pragma unroll
    for (int v = 0; v < NV; ++v) {
      T acc = 0;
#pragma unroll
      for (int k = 0; k < N; ++k) acc += pick<T>(B.Minv[p * N + k], B.Minv_f[p * N + k]) * sB[lm][sd][v][k];
      sA[lm][sd][v][p] = acc;
    }
  }
  __syncthreads();
  // (D) Rusanov at mortar SP p with the radial normal (the grid velocity of
  // a rotation about the circle's centre is tangential: v_g . n = 0)
  if (act && sd == 0) {
    if (MMODE != MORTAR_AVG_Q) {
      T sn, cs;
      normal_of<T>(m0 + fma(B.Xs[p], dm, md.mgeo[4 * m + 1]), cs, sn);
      T qL[4], qR[4], Fn[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        qL[v] = sA[lm][0][v][p];
        qR[v] = sA[lm][1][v][p];
      }
      rusanov(qL, qR, (T)cs, (T)sn, T(0), pick<T>(md.gamma, md.gamma_f), Fn);
#pragma unroll
      for (int v = 0; v < 4; ++v)
        sF[lm][v][p] = MMODE == MORTAR_RUSANOV_FV ? Fn[v] + T(0.5) * (sA[lm][0][4 + v][p] + sA[lm][1][4 + v][p])
                                                  : Fn[v];
    } else {
      // common value on the mortar: average of both sides (Sec. 3.2)
#pragma unroll
      for (int v = 0; v < 4; ++v) sF[lm][v][p] = T(0.5) * (sA[lm][0][v][p] + sA[lm][1][v][p]);
    }
  }
  __syncthreads();
  // (E) mortar flux polynomial at the quadrature points
  if (act && sd == 0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T acc = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) acc += pick<T>(B.Hz[p * N + j], B.Hz_f[p * N + j]) * sF[lm][v][j];
      sFz[lm][v][p] = acc;
    }
  }
  __syncthreads();
  // (F) (S F)_p = sum_q w_q h_p(o + s z_q) F(z_q)
  if (act) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T acc = 0;
#pragma unroll
      for (int q = 0; q < N; ++q) acc += sWH[lm][sd][q][p] * sFz[lm][v][q];
      sB[lm][sd][v][p] = acc;
    }
  }
  __syncthreads();
  // (G) contribution s M^{-1} S F^Xi to the face (Eq. prjF2)
  if (act) {
    T *out = (T *)md.contrib + (((size_t)sd * md.nM + m) * 4) * N;
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T acc = 0;
#pragma unroll
      for (int k = 0; k < N; ++k) acc += pick<T>(B.Minv[p * N + k], B.Minv_f[p * N + k]) * sB[lm][sd][v][k];
      out[v * N + p] = (T)s * acc;
    }
  }
}

template <typename T, int N, int MMODE>
__global__ void __launch_bounds__(MortCfg<N>::THREADS) k_mortar_flux(MeshDev md) {
  pdl_enter();
  mortar_flux_body<T, N, MMODE, MortCfg<N>::MPB>(md, blockIdx.x);
}

// Sum of the mortar contributions of each interface face (fixed order: the
// face's mortars in counter-clockwise order), written as the face's common
// flux F~_end = sigma_f |S| F.n_out (n from L to R is outward for L, inward
// for R).  One thread per (side, face, point).
enum { GATHER_FLUX = 0, GATHER_Q = 1 };

// The common value at point p of interface face fq (L faces first, then R):
// the sum of the contributions of the face's mortars, in their
// counter-clockwise order -- the common solution (GATHER_Q) or, scaled by
// sigma_f |S| and the side's sign, the common flux (GATHER_FLUX).  Also gives
// the element face ef and its point j.  False for a bad table entry (debug
// build).
template <typename T, int N, int GMODE>
__device__ __forceinline__ bool gather_sum(const MeshDev &md, int fq, int p, T *out, int &ef, int &j) {
  const int sd = fq >= md.nL;
  const int k = sd ? fq - md.nL : fq;
  const int start = sd ? md.Rstart[k] : md.Lstart[k];
  const int cnt = sd ? md.Rcount[k] : md.Lcount[k];
  const int4 fc = sd ? md.Rface[k] : md.Lface[k];
  const T *cb = (const T *)md.contrib + (size_t)sd * md.nM * 4 * N;
  // the face's mortars run cyclically through its interface's mortar range [m0, m1)
  const int ii = md.ifz[fq];
  const int m0 = md.zoff[ii] + md.zoff[kZT + ii], m1 = md.zoff[ii + 1] + md.zoff[kZT + ii + 1];
  if (!ssd_check(md, start >= m0 && start < m1 && cnt >= 1 && cnt <= m1 - m0 && fc.x >= 0 && fc.x < 4 * md.E))
    return false;
  T acc[4] = {0, 0, 0, 0};
  int mi = start;
  for (int c = 0; c < cnt; ++c) {
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[v] += cb[((size_t)mi * 4 + v) * N + p];
    mi = mi + 1 == m1 ? m0 : mi + 1;
  }
  ef = fc.x;
  j = fc.y ? N - 1 - p : p;
  if (GMODE == GATHER_Q) {
#pragma unroll
    for (int v = 0; v < 4; ++v) out[v] = acc[v];
    return true;
  }
  const T S = (T)(sd ? md.RS[k] : md.LS[k]);
  const T sc = (T)face_sigma(ef & 3) * S * (sd ? T(-1) : T(1));
#pragma unroll
  for (int v = 0; v < 4; ++v) out[v] = sc * acc[v];
  return true;
}

// The gather inside the kernel that reads its result: the interface faces of
// the tile elements e0 + [0, ne) get their common values (per element 16 N
// values [face][variable][point], element stride `stride`) in the tile's
// shared copy; with `global` also in CQ / CF.  Returns whether the tile had
// an interface cell (then the caller synchronises before reading the tile).
template <typename T, int N, int GMODE>
__device__ __forceinline__ bool gather_tile(const MeshDev &md, int e0, int ne, const int *sEF, T *tile, int stride,
                                            bool global, int nthreads) {
  // the tile's flags in 16-byte groups (a tile's flags are copied in whole
  // groups of 4, the cells past the mesh's last carrying 0)
  int any = 0;
  for (int q = 0; q < (ne + 3) / 4; ++q) {
    const int4 f4 = reinterpret_cast<const int4 *>(sEF)[q];
    any |= f4.x | f4.y | f4.z | f4.w;
  }
  if (!(any & kIfaceBit)) return false;
  for (int u = threadIdx.x; u < ne * 4 * N; u += nthreads) {
    const int le = u / (4 * N), r = u - le * 4 * N, f = r / N, jj = r - f * N;
    if (!(sEF[le] & kIfaceBit)) continue;
    const int fq = md.efi[4 * (e0 + le) + f];
    if (fq < 0) continue;
    const int k = fq >= md.nL ? fq - md.nL : fq;
    const int rev = (fq >= md.nL ? md.Rface[k] : md.Lface[k]).y;
    T val[4];
    int ef, j;
    if (!gather_sum<T, N, GMODE>(md, fq, rev ? N - 1 - jj : jj, val, ef, j)) continue;
#pragma unroll
    for (int v = 0; v < 4; ++v) tile[le * stride + (f * 4 + v) * N + jj] = val[v];
    if (global) {
      T *dst = (T *)(GMODE == GATHER_Q ? md.CQ : md.CF);
#pragma unroll
      for (int v = 0; v < 4; ++v) dst[((size_t)ef * 4 + v) * N + j] = val[v];
    }
  }
  return true;
}


// ---------------------------------------------------------------------------
// state conversion and traces
// ---------------------------------------------------------------------------

// FP64 state -> double-float pair (hi = round(x), lo = round(x - hi))
static __global__ void k_split(const double *__restrict__ Q, float *hi, float *lo, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = Q[i];
  const float h = __double2float_rn(x);
  hi[i] = h;
  if (lo) lo[i] = __double2float_rn(x - (double)h);
}

static __global__ void k_join(const float *__restrict__ hi, const float *__restrict__ lo, double *Q, size_t n) {
  const size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  Q[i] = lo ? (double)hi[i] + (double)lo[i] : (double)hi[i];
}

// face traces [E][4][4][N] of a state (compute-precision values)
template <typename T, int N>
__global__ void k_trace(MeshDev md, const T *__restrict__ Q) {
  pdl_enter();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= md.E * 16 * N) return;
  const int e = t / (16 * N);
  const int r = t - e * 16 * N;
  const int f = r / (4 * N), v = (r / N) & 3, j = r % N;
  const VolBasis<T, N> &B = cVB<T, N>;
  const T *q = Q + ((size_t)e * 4 + v) * N * N;
  T acc = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    // f0 eta=0 / f2 eta=1: column j; f1 xi=1 / f3 xi=0: row j
    const T qk = (f == 0 || f == 2) ? q[k * N + j] : q[j * N + k];
    acc += qk * ((f == 1 || f == 2) ? B.H1[k] : B.H0[k]);
  }
  ((T *)md.TR)[t] = acc;
}

// ---------------------------------------------------------------------------
// volume kernel: persistent CTAs stream element tiles through shared memory
// with 1-D bulk TMA copies (cp.async.bulk + mbarrier), two stages deep, so the
// next tile's state, base state, common fluxes and cell records load while
// the current tile computes.  Every per-element array is padded to a whole
// number of tiles, so each copy is a full, 16-byte-aligned tile.
// ---------------------------------------------------------------------------

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done)
      : "r"(smem_u32(bar)), "r"(parity)
      : "memory");
  return done != 0;
}

// bounded wait: gives up after a fixed number of polls (each poll may suspend
// the thread for a hardware-defined time), so a lost copy cannot hang the GPU
constexpr int kWaitPolls = 1 << 22;
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, int polls = kWaitPolls) {
  for (int i = 0; i < polls; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}

__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// exact sum s + e = a + b (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  const float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// default elements per volume tile (a multiple of 4)
template <int N>
constexpr int vol_epb_default() { return N == 3 ? 16 : (N == 6 ? 8 : 12); }

template <typename T, int N, bool OTF, bool AUX = false, bool LO = true, int EPBX = 0, bool TC = false>
struct VolCfg {
  static constexpr int NN = N * N;
  static constexpr bool FF = std::is_same<T, float>::value;  // FP32 arithmetic (packed pairs)
  static constexpr bool DF = FF && LO;                       // double-float state (hi + lo planes)
  static constexpr int EPB = EPBX ? EPBX : vol_epb_default<N>();  // elements per tile (multiple of 4)
  static constexpr int THREADS = EPB * 2 * N;                  // one thread per SP line
  // element strides (values) of the tiles in shared memory: padded so that
  // the elements of a tile start in different banks (a stride of 4 N^2 or 16 N
  // words put the SP lines of neighbouring elements on the same banks); every
  // stride is a multiple of 16 bytes, as a bulk copy's destination must be
  static constexpr int PADQ = N == 3 ? 8 : (N == 4 ? 16 : (N == 5 ? 24 : 20));
  static constexpr int SE = 4 * NN + PADQ;  // state hi tile, work arrays
  static constexpr int SC = 16 * N + 8;     // common-flux tile
  // bytes one element moves per array
  static constexpr int QE = 4 * NN * (int)sizeof(T), CE = 16 * N * (int)sizeof(T);
  // double-buffered part of a tile (needed by the flux phase): state hi,
  // common fluxes, cell records, flags
  static constexpr int QHI = EPB * SE * (int)sizeof(T);
  static constexpr int CFB = EPB * SC * (int)sizeof(T);
  static constexpr int EGB = OTF ? EPB * 8 * (int)sizeof(T) : 0;
  static constexpr int EFB = EPB * 4;
  static constexpr int O_QHI = 0, O_CF = O_QHI + QHI, O_EG = O_CF + CFB, O_EF = O_EG + EGB;
  static constexpr int STAGE = ((O_EF + EFB) + 127) / 128 * 128;
  // single-buffered part (needed only by the Runge-Kutta phase): state lo,
  // base state hi and lo, carried increment; loaded at the start of each tile
  // behind the flux phase, unpadded (one copy per array lands sooner than one
  // per element; its reads are plain runs of consecutive words)
  static constexpr int QB = EPB * 4 * NN * (int)sizeof(T), QBL = DF ? EPB * 4 * NN * 4 : 0;
  static constexpr int AUXB = AUX ? QB : 0;  // increment carried from an earlier stage
  static constexpr int O_QLO = 2 * STAGE, O_NHI = O_QLO + QBL, O_NLO = O_NHI + QB, O_AUX = O_NLO + QBL;
  static constexpr int SINGLE_END = ((O_AUX + AUXB) + 127) / 128 * 128;
  // work arrays
  static constexpr int O_RF = SINGLE_END, O_RG = O_RF + QHI;
  static constexpr int O_BAR = ((O_RG + QHI) + 15) / 16 * 16;
  // the stage's zone table [3][kZT] (cos theta_z, sin theta_z, omega_z); two
  // slots, one per pipeline stage, for a batch whose next item is another case
  static constexpr int O_ZT = O_BAR + 32;
  // tensor-core variant: the tile's rows (direction, element, SP line,
  // variable) with 8 flux-point columns, for the interpolated values and then
  // the fluxes (the operands of the two contractions)
  static constexpr int TC_ROWS = 8 * EPB * N;
  static constexpr int O_TC = ((O_ZT + 2 * 3 * kZT * (int)sizeof(T)) + 127) / 128 * 128;
  static constexpr int SMEM = TC ? O_TC + TC_ROWS * 8 * 4 : O_ZT + 2 * 3 * kZT * (int)sizeof(T);
  // transaction bytes of the two barriers' copies
  static constexpr int TX_QHI = EPB * QE, TX_CF = EPB * CE;
  static_assert((SE * (int)sizeof(T)) % 16 == 0 && (SC * (int)sizeof(T)) % 16 == 0, "bulk-copy alignment");
  static_assert(QE % 16 == 0 && CE % 16 == 0 && QB % 16 == 0, "bulk-copy sizes");
  static_assert(EPB <= 32, "one warp-0 lane per element");
  // resident CTAs per SM the register budget is set for (228 KB of shared
  // memory per SM, 1 KB of it reserved per CTA)
  static constexpr int MINB = (228 * 1024 / (SMEM + 1024)) < 8 ? (228 * 1024 / (SMEM + 1024)) : 8;
};

// transformed ALE inviscid flux at one flux point: a.(F, G) - (V_g . a) Q
template <typename T>
__device__ __forceinline__ void point_flux(const T *q, T vx, T vy, T vg, T gm1, T *f) {
  const T ir = recip(q[0]);
  const T p = gm1 * (q[3] - T(0.5) * mul_add(q[1], q[1], q[2], q[2]) * ir);
  const T un = mul_add(q[1], vx, q[2], vy) * ir;
  f[0] = mul_sub(q[0], un, vg, q[0]);
  f[1] = fma(q[1], un, mul_sub(p, vx, vg, q[1]));
  f[2] = fma(q[2], un, mul_sub(p, vy, vg, q[2]));
  f[3] = mul_sub(q[3] + p, un, vg, q[3]);
}

// bounded wait by warp 0 only; the other warps wait at the barrier without issuing
__device__ __forceinline__ bool cta_wait(uint64_t *bar, uint32_t parity, int polls = kWaitPolls) {
  bool ok = true;
  if (threadIdx.x < 32) ok = mbar_wait_bounded(bar, parity, polls);
  return __syncthreads_and(ok) != 0;
}

// stage coefficients in the compute type
template <typename T>
struct RkCoef {
  T a0, bdt, g, ddt;
};

// Arguments of one case's volume launch: the states it reads and writes, the
// residual output (MODE_RESIDUAL), the stage coefficients and the increments
// carried between stages of the five-stage scheme.
template <typename T>
struct VolArgs {
  StatePtr in, base, out;
  double *R;
  RkCoef<T> rk;
  int has_base;
  T *w_out;
  const T *w_in;
};

// Work sources of the persistent kernels.  A work item is one tile of one
// case; the source names the case and its tile and gives that case's mesh
// view and launch arguments A.  OneCase: one handle, whose tiles are the
// items.  CaseList: the cases of a batch class, items numbered across all of
// them (off[c] = first item of case c, off[n] = all items), each case's view
// and arguments in device memory.
template <typename A>
struct OneCase {
  static constexpr bool kMulti = false;
  MeshDev md;
  A a;
  __device__ __forceinline__ void item(int it, int &c, int &tile) const {
    c = 0;
    tile = it;
  }
  __device__ __forceinline__ const MeshDev &mesh(int) const { return md; }
  __device__ __forceinline__ const A &args(int) const { return a; }
};

template <typename A>
struct CaseList {
  static constexpr bool kMulti = true;
  const MeshDev *md;
  const A *a;
  const int *off;
  int n;
  __device__ __forceinline__ void item(int it, int &c, int &tile) const {
    int lo = 0, hi = n - 1;  // the last case whose first item is <= it
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (__ldg(off + mid) <= it) lo = mid;
      else hi = mid - 1;
    }
    c = lo;
    tile = it - __ldg(off + lo);
  }
  __device__ __forceinline__ const MeshDev &mesh(int c) const { return md[c]; }
  __device__ __forceinline__ const A &args(int c) const { return a[c]; }
};

// ---- 3xTF32 tensor-core contractions (the optional path of the FP32 form) ----
// A float x is split into two TF32 values, x = big + small (+ the remainder
// below TF32 resolution); a product is taken as big_a big_b + big_a small_b +
// small_a big_b, three m16n8k8 TF32 MMAs accumulating in FP32, which keeps
// close to FP32 accuracy.

__device__ __forceinline__ uint32_t tf32_of(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return r;
}

__device__ __forceinline__ void tf32_split(float x, uint32_t &big, uint32_t &small) {
  big = tf32_of(x);
  small = tf32_of(x - __uint_as_float(big));
}

// D += A B for one m16n8k8 tile (A row-major 16 x 8, B column-major 8 x 8,
// TF32 inputs, FP32 accumulators; fragments as the PTX ISA lays them out)
__device__ __forceinline__ void mma_tf32(float *d, const uint32_t *a, uint32_t b0, uint32_t b1) {
  asm volatile("mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
               "{%0,%1,%2,%3};"
               : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
               : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// 3xTF32 product of one A fragment (four floats) with a split B fragment
__device__ __forceinline__ void mma_3xtf32(float *d, const float *af, const uint32_t *bb, const uint32_t *bs) {
  uint32_t ab[4], as[4];
#pragma unroll
  for (int q = 0; q < 4; ++q) tf32_split(af[q], ab[q], as[q]);
  mma_tf32(d, as, bb[0], bb[1]);
  mma_tf32(d, ab, bs[0], bs[1]);
  mma_tf32(d, ab, bb[0], bb[1]);
}

// Phase 1 of the FP32 volume kernel on the tensor cores.  Rows of the tile:
// r = ((d EPB + e) N + line) 4 + v (direction d, element e, SP line, variable
// v), 16 per MMA tile.  (1) interpolation: X[r][i] = sum_k Q[r][k] Hf[i][k]
// (Eq. Qt at the flux points i = 0..N, K = the N SPs of the line, padded to 8);
// (2) each line's thread forms the transformed fluxes at its interior flux
// points from X, the common fluxes at its end points, into the same rows;
// (3) divergence: R[r][k] = sum_i F[r][i] Dm[k][i] (Eqs. Ft, Gt), into the
// tile's divergence arrays.  Full warps take the MMA tiles; barriers between.
template <typename T, int N, bool OTF, class C>
__device__ __forceinline__ void volume_phase1_tc(const MeshDev &md, int e0, int ne, const T (*sQ)[C::SE],
                                                 const T (*sCF)[C::SC], const int *sEF, const T *sEG,
                                                 const T *sZT, T gm1, T (*sRF)[C::SE], T (*sRG)[C::SE],
                                                 float (*sX)[8]) {
  constexpr int EPB = C::EPB, NN = N * N, NT = C::THREADS, MT = C::TC_ROWS / 16, NW = NT / 32;
  const VolBasis<T, N> &B = cVB<T, N>;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int g = lane >> 2, t = lane & 3;
  // value of row r at K index k (the SP of the line), 0 beyond the N SPs
  auto qval = [&](int r, int k) -> float {
    const int v = r & 3, line = (r >> 2) % N, de = (r >> 2) / N, e = de % EPB, d = de / EPB;
    if (k >= N) return 0.0f;
    return (float)(d == 0 ? sQ[e][v * NN + line * N + k] : sQ[e][v * NN + k * N + line]);
  };
  // (1) interpolation, B[k][n] = Hf[n][k] (n = flux point)
  if (warp < NW) {
    uint32_t bb[2], bs[2];
    {
      const float h0 = (g <= N && t < N) ? (float)B.Hf[g * N + t] : 0.0f;
      const float h1 = (g <= N && t + 4 < N) ? (float)B.Hf[g * N + t + 4] : 0.0f;
      tf32_split(h0, bb[0], bs[0]);
      tf32_split(h1, bb[1], bs[1]);
    }
    for (int mt = warp; mt < MT; mt += NW) {
      const int r0 = mt * 16;
      float af[4] = {qval(r0 + g, t), qval(r0 + g + 8, t), qval(r0 + g, t + 4), qval(r0 + g + 8, t + 4)};
      float dd[4] = {0.f, 0.f, 0.f, 0.f};
      mma_3xtf32(dd, af, bb, bs);
      sX[r0 + g][2 * t] = dd[0];
      sX[r0 + g][2 * t + 1] = dd[1];
      sX[r0 + g + 8][2 * t] = dd[2];
      sX[r0 + g + 8][2 * t + 1] = dd[3];
    }
  }
  __syncthreads();
  // (2) fluxes, one thread per SP line (as the FFMA path)
  {
    const int d = threadIdx.x >= EPB * N ? 1 : 0;
    const int tl = threadIdx.x - d * EPB * N;
    const int le = tl / N, mline = tl - le * N;
    if (le < ne && threadIdx.x < 2 * EPB * N) {
      ElemGeo<T, N, OTF> G;
      G.load_rec(md, e0 + le, sEF[le], sEG + le * 8, sZT);
      T mvx[N + 1], mvy[N + 1], mvg[N + 1];
      G.line_metrics(d, mline, mvx, mvy, mvg);
      const int rb = ((d * EPB + le) * N + mline) * 4;
      const int fa = d == 0 ? 3 : 0, fb = d == 0 ? 1 : 2;
#pragma unroll
      for (int i = 1; i < N; ++i) {
        const float qf[4] = {sX[rb][i], sX[rb + 1][i], sX[rb + 2][i], sX[rb + 3][i]};
        float f[4];
        point_flux(qf, (float)mvx[i], (float)mvy[i], (float)mvg[i], (float)gm1, f);
#pragma unroll
        for (int v = 0; v < 4; ++v) sX[rb + v][i] = f[v];
      }
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        sX[rb + v][0] = (float)sCF[le][(fa * 4 + v) * N + mline];
        sX[rb + v][N] = (float)sCF[le][(fb * 4 + v) * N + mline];
      }
    }
  }
  __syncthreads();
  // (3) divergence, B[i][n] = Dm[n][i] (n = SP of the line)
  if (warp < NW) {
    uint32_t bb[2], bs[2];
    {
      const float w0 = (g < N && t <= N) ? (float)B.Dm[g * (N + 1) + t] : 0.0f;
      const float w1 = (g < N && t + 4 <= N) ? (float)B.Dm[g * (N + 1) + t + 4] : 0.0f;
      tf32_split(w0, bb[0], bs[0]);
      tf32_split(w1, bb[1], bs[1]);
    }
    for (int mt = warp; mt < MT; mt += NW) {
      const int r0 = mt * 16;
      float af[4] = {sX[r0 + g][t], sX[r0 + g + 8][t], sX[r0 + g][t + 4], sX[r0 + g + 8][t + 4]};
      float dd[4] = {0.f, 0.f, 0.f, 0.f};
      mma_3xtf32(dd, af, bb, bs);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int r = r0 + g + (q >> 1) * 8, k = 2 * t + (q & 1);
        if (k >= N) continue;
        const int v = r & 3, line = (r >> 2) % N, de = (r >> 2) / N, e = de % EPB, d = de / EPB;
        if (d == 0) sRF[e][v * NN + line * N + k] = (T)dd[q];
        else sRG[e][v * NN + k * N + line] = (T)dd[q];
      }
    }
  }
}

// The persistent volume kernel over the work items of src (see OneCase /
// CaseList): for a batch class the items of all its cases form one list, and
// the next item's copies are issued while the current one computes even when
// it belongs to another case.
template <typename T, int N, int MODE, bool OTF, bool AUX, bool LO, int EPBX, class Src, bool TC = false>
__global__ void __launch_bounds__(VolCfg<T, N, OTF, AUX, LO, EPBX, TC>::THREADS,
                                  VolCfg<T, N, OTF, AUX, LO, EPBX, TC>::MINB)
    k_volume(Src src, int nitems) {
  pdl_enter();
  using C = VolCfg<T, N, OTF, AUX, LO, EPBX, TC>;
  static_assert(!TC || (C::FF && LO), "the tensor-core contractions are a variant of the FP32 form");
  constexpr int EPB = C::EPB, NT = C::THREADS, NN = N * N;
  constexpr bool FF = C::FF, DF = C::DF;
  extern __shared__ __align__(128) unsigned char smem[];
  uint64_t *bar = (uint64_t *)(smem + C::O_BAR);  // [0], [1]: double-buffered part; [2]: single part
  T(*sRF)[C::SE] = (T(*)[C::SE])(smem + C::O_RF);
  T(*sRG)[C::SE] = (T(*)[C::SE])(smem + C::O_RG);
  const VolBasis<T, N> &B = cVB<T, N>;
  // the zone table of the item's case: one copy for a single case, a copy per
  // stage of the pipeline for a batch (the next item may be another case)
  T *sZT0 = (T *)(smem + C::O_ZT);

  // copies are issued by the lanes of warp 0, one element each, into the
  // padded tile; lane 0 first arms the barrier with the whole byte count
  auto issueA = [&](int item, int st, int lane) {
    int cn, tl;
    src.item(item, cn, tl);
    const MeshDev &mn = src.mesh(cn);
    const VolArgs<T> &an = src.args(cn);
    unsigned char *sb = smem + st * C::STAGE;
    if (!batch_check(mn, tl >= 0 && tl * EPB < mn.E)) {
      // a work item outside its case: the barrier is armed with nothing to
      // wait for and the tile computes on stale data, writing nothing
      if (lane == 0) mbar_expect_tx(&bar[st], 0);
      return;
    }
    const size_t e0 = (size_t)tl * EPB;
    // (the test switch of sd_test_wait_timeout arms work item 0 with more
    // bytes than its copies deliver; it is 0 otherwise)
    if (lane == 0) mbar_expect_tx(&bar[st], C::TX_QHI + C::TX_CF + C::EGB + C::EFB + (item == 0 ? mn.test_tx_extra : 0));
    __syncwarp();
    if (lane < EPB) {
      bulk_g2s(sb + C::O_QHI + lane * C::SE * sizeof(T), (const T *)an.in.hi + (e0 + lane) * 4 * NN, C::QE, &bar[st]);
      bulk_g2s(sb + C::O_CF + lane * C::SC * sizeof(T), (const T *)mn.CF + (e0 + lane) * 16 * N, C::CE, &bar[st]);
    }
    if (lane == 0) {
      if (OTF) bulk_g2s(sb + C::O_EG, (const T *)mn.egeo + e0 * 8, C::EGB, &bar[st]);
      bulk_g2s(sb + C::O_EF, mn.eflag + e0, C::EFB, &bar[st]);
    }
    if constexpr (Src::kMulti) {
      if (lane < 3 * kZT) sZT0[st * 3 * kZT + lane] = zone_tab<T>(mn.clk)[lane];
    }
  };
  auto txB_of = [&](const VolArgs<T> &a) -> uint32_t {
    return MODE == MODE_RK ? C::QBL + (a.has_base ? C::QB + C::QBL : 0) + C::AUXB : 0;
  };
  auto issueB = [&](const VolArgs<T> &a, int tl) {
    const size_t e0 = (size_t)tl * EPB;
    mbar_expect_tx(&bar[2], txB_of(a));
    if (DF) bulk_g2s(smem + C::O_QLO, (const float *)a.in.lo + e0 * 4 * NN, C::QBL, &bar[2]);
    if (a.has_base) {
      bulk_g2s(smem + C::O_NHI, (const T *)a.base.hi + e0 * 4 * NN, C::QB, &bar[2]);
      if (DF) bulk_g2s(smem + C::O_NLO, (const float *)a.base.lo + e0 * 4 * NN, C::QBL, &bar[2]);
    }
    if (AUX) bulk_g2s(smem + C::O_AUX, a.w_in + e0 * 4 * NN, C::AUXB, &bar[2]);
  };

  if (threadIdx.x == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    mbar_init(&bar[2], 1);
    fence_mbar_init();
  }
  if constexpr (!Src::kMulti) {
    if (threadIdx.x < 3 * kZT) sZT0[threadIdx.x] = zone_tab<T>(src.mesh(0).clk)[threadIdx.x];
  }
  __syncthreads();
  int item = blockIdx.x;
  if (threadIdx.x < 32 && item < nitems) issueA(item, 0, threadIdx.x);
  bool bad = false;
  int it = 0;
  for (; item < nitems; item += gridDim.x, ++it) {
    const int st = it & 1;
    const int next = item + gridDim.x;
    int cs, tile;
    src.item(item, cs, tile);
    const MeshDev &md = src.mesh(cs);
    const VolArgs<T> &va = src.args(cs);
    const uint32_t txB = txB_of(va);
    const bool use_base = MODE == MODE_RK && va.has_base;
    const T gm1 = pick<T>(md.gamma, md.gamma_f) - T(1);
    const T *sZT = Src::kMulti ? sZT0 + st * 3 * kZT : sZT0;
    if (threadIdx.x < 32) {
      // both refilled regions were last read before the previous iteration's
      // closing barrier; order those generic reads before the async writes
      fence_proxy_async_smem();
      if (next < nitems) issueA(next, st ^ 1, threadIdx.x);
      if (txB && threadIdx.x == 0) issueB(va, tile);
    }
    if (!cta_wait(&bar[st], (uint32_t)((it >> 1) & 1), (item == 0 && md.test_poll) ? md.test_poll : kWaitPolls)) {
      if (threadIdx.x == 0) {
        atomicOr(&md.clk->flags, 4);
        // let the copies in flight land before the CTA exits (full limits)
        if (next < nitems) mbar_wait_bounded(&bar[st ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
        if (txB) mbar_wait_bounded(&bar[2], (uint32_t)(it & 1));
      }
      return;
    }
    unsigned char *sb = smem + st * C::STAGE;
    T(*sQ)[C::SE] = (T(*)[C::SE])(sb + C::O_QHI);
    const T(*sCF)[C::SC] = (const T(*)[C::SC])(sb + C::O_CF);
    const int *sEF = (const int *)(sb + C::O_EF);
    const T *sEG = (const T *)(sb + C::O_EG);
    const int e0 = tile * EPB;
    const int ne = min(EPB, md.E - e0);
    // the tile's interface faces: their common fluxes from the mortar
    // contributions (the gather of Eq. prjF2 over each face's mortars)
    if (gather_tile<T, N, GATHER_FLUX>(md, e0, ne, sEF, (T *)(sb + C::O_CF), C::SC, false, NT)) __syncthreads();
    // ---- phase 1: one thread per SP line: threads [0, EPB N) take the xi
    // lines, the rest the eta lines, so that most warps run one direction ----
    const int d = threadIdx.x >= EPB * N ? 1 : 0;
    const int tl = threadIdx.x - d * EPB * N;
    const int le = tl / N, mline = tl - le * N;
    if constexpr (TC) {
      volume_phase1_tc<T, N, OTF, C>(md, e0, ne, sQ, sCF, sEF, sEG, sZT, gm1, sRF, sRG,
                                     (float(*)[8])(smem + C::O_TC));
    } else if (le < ne) {
      ElemGeo<T, N, OTF> G;
      G.load_rec(md, e0 + le, sEF[le], sEG + le * 8, sZT);
      T mvx[N + 1], mvy[N + 1], mvg[N + 1];
      G.line_metrics(d, mline, mvx, mvy, mvg);
      if constexpr (FF) {
        // FP32: variables packed in pairs (rho, rho u), (rho v, E); every
        // interpolation and divergence FMA is a packed FP32x2 FMA
        float2 q2[2][N], acc2[2][N];
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const int sp = d == 0 ? mline * N + k : k * N + mline;
          q2[0][k] = make_float2(sQ[le][(0) * NN + sp], sQ[le][(1) * NN + sp]);
          q2[1][k] = make_float2(sQ[le][(2) * NN + sp], sQ[le][(3) * NN + sp]);
          acc2[0][k] = make_float2(0.f, 0.f);
          acc2[1][k] = make_float2(0.f, 0.f);
        }
        // Q at every interior FP of the line at once (the SP index outermost,
        // so the 2 (N - 1) sums are independent chains), then the fluxes, then
        // the divergence; each sum keeps its order
        float2 s01[N + 1], s23[N + 1];
#pragma unroll
        for (int i = 1; i < N; ++i) {
          s01[i] = make_float2(0.f, 0.f);
          s23[i] = make_float2(0.f, 0.f);
        }
#pragma unroll
        for (int k = 0; k < N; ++k)
#pragma unroll
          for (int i = 1; i < N; ++i) {
            const float2 h = B.Hf2[i * N + k];
            s01[i] = __ffma2_rn(q2[0][k], h, s01[i]);
            s23[i] = __ffma2_rn(q2[1][k], h, s23[i]);
          }
        float2 f01[N + 1], f23[N + 1];
        {
          const int fa = d == 0 ? 3 : 0, fb = d == 0 ? 1 : 2;
          f01[0] = make_float2(sCF[le][(fa * 4 + 0) * N + mline], sCF[le][(fa * 4 + 1) * N + mline]);
          f23[0] = make_float2(sCF[le][(fa * 4 + 2) * N + mline], sCF[le][(fa * 4 + 3) * N + mline]);
          f01[N] = make_float2(sCF[le][(fb * 4 + 0) * N + mline], sCF[le][(fb * 4 + 1) * N + mline]);
          f23[N] = make_float2(sCF[le][(fb * 4 + 2) * N + mline], sCF[le][(fb * 4 + 3) * N + mline]);
        }
#pragma unroll
        for (int i = 1; i < N; ++i) {
          const float qf[4] = {s01[i].x, s01[i].y, s23[i].x, s23[i].y};
          float f[4];
          point_flux(qf, (float)mvx[i], (float)mvy[i], (float)mvg[i], (float)gm1, f);
          f01[i] = make_float2(f[0], f[1]);
          f23[i] = make_float2(f[2], f[3]);
        }
#pragma unroll
        for (int i = 0; i <= N; ++i)
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const float2 w = B.Dm2[k * (N + 1) + i];
            acc2[0][k] = __ffma2_rn(w, f01[i], acc2[0][k]);
            acc2[1][k] = __ffma2_rn(w, f23[i], acc2[1][k]);
          }
        if (d == 0) {
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const int sp = mline * N + k;
            sRF[le][(0) * NN + sp] = acc2[0][k].x;
            sRF[le][(1) * NN + sp] = acc2[0][k].y;
            sRF[le][(2) * NN + sp] = acc2[1][k].x;
            sRF[le][(3) * NN + sp] = acc2[1][k].y;
          }
        } else {
#pragma unroll
          for (int k = 0; k < N; ++k) {
            const int sp = k * N + mline;
            sRG[le][(0) * NN + sp] = acc2[0][k].x;
            sRG[le][(1) * NN + sp] = acc2[0][k].y;
            sRG[le][(2) * NN + sp] = acc2[1][k].x;
            sRG[le][(3) * NN + sp] = acc2[1][k].y;
          }
        }
      } else {
      T q[4][N];
#pragma unroll
      for (int k = 0; k < N; ++k)
#pragma unroll
        for (int v = 0; v < 4; ++v) q[v][k] = d == 0 ? sQ[le][(v) * NN + mline * N + k] : sQ[le][(v) * NN + k * N + mline];
      T acc[4][N];
#pragma unroll
      for (int k = 0; k < N; ++k)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[v][k] = 0;
#pragma unroll
      for (int i = 0; i <= N; ++i) {
        T f[4];
        if (i == 0 || i == N) {
          const int face = d == 0 ? (i == 0 ? 3 : 1) : (i == 0 ? 0 : 2);
#pragma unroll
          for (int v = 0; v < 4; ++v) f[v] = sCF[le][(face * 4 + v) * N + mline];
        } else {
          T qf[4];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            T s = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) s += q[v][k] * B.Hf[i * N + k];
            qf[v] = s;
          }
          point_flux(qf, mvx[i], mvy[i], mvg[i], gm1, f);
        }
#pragma unroll
        for (int k = 0; k < N; ++k) {
          const T w = B.Dm[k * (N + 1) + i];
#pragma unroll
          for (int v = 0; v < 4; ++v) acc[v][k] += w * f[v];
        }
      }
      if (d == 0) {
#pragma unroll
        for (int k = 0; k < N; ++k)
#pragma unroll
          for (int v = 0; v < 4; ++v) sRF[le][(v) * NN + mline * N + k] = acc[v][k];
      } else {
#pragma unroll
        for (int k = 0; k < N; ++k)
#pragma unroll
          for (int v = 0; v < 4; ++v) sRG[le][(v) * NN + k * N + mline] = acc[v][k];
      }
      }
    }
    // the single-buffered part (state lo, base state) must have landed too
    if (txB) {
      if (!cta_wait(&bar[2], (uint32_t)(it & 1))) {
        if (threadIdx.x == 0) {
          atomicOr(&md.clk->flags, 4);
          if (next < nitems) mbar_wait_bounded(&bar[st ^ 1], (uint32_t)(((it + 1) >> 1) & 1));
        }
        return;
      }
    } else {
      __syncthreads();
    }
    // ---- phase 2: dQ/dt at the SPs and the Runge-Kutta combination ----
    for (int idx = threadIdx.x; idx < ne * NN; idx += NT) {
      const int l2 = idx / NN, sp = idx - l2 * NN;
      const T iJ = ElemGeo<T, N, OTF>::inv_jac_t0(md, sEF[l2], sEG + l2 * 8, sp % N, sp / N);
      const size_t gi = ((size_t)(e0 + l2) * 4) * NN + sp;
      if (MODE == MODE_RESIDUAL) {
#pragma unroll
        for (int v = 0; v < 4; ++v) va.R[gi + v * NN] = -(double)((sRF[l2][(v) * NN + sp] + sRG[l2][(v) * NN + sp]) * iJ);
      } else if (!FF) {
        // FP64: inc = a0 (Q_base - Q_k) + w_in + bdt R;  Q_out = Q_k + inc
        const double(*sN)[4 * NN] = (const double(*)[4 * NN])(smem + C::O_NHI);
        const double(*sW)[4 * NN] = (const double(*)[4 * NN])(smem + C::O_AUX);
        double *qo = (double *)va.out.hi;
        double qn[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const double R = -(double)((sRF[l2][(v) * NN + sp] + sRG[l2][(v) * NN + sp]) * iJ);
          const double qk = (double)sQ[l2][(v) * NN + sp];
          double inc = __dmul_rn((double)va.rk.bdt, R);
          if (use_base) inc = fma((double)va.rk.a0, sN[l2][(v) * NN + sp] - qk, inc);
          if (AUX) inc += sW[l2][(v) * NN + sp];
          qn[v] = qk + inc;
          if (va.w_out) va.w_out[gi + v * NN] = (T)mul_sub((double)va.rk.ddt, R, (double)va.rk.g, inc);
        }
        bad |= !physical(qn);
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          qo[gi + v * NN] = qn[v];
          sQ[l2][(v) * NN + sp] = (T)qn[v];
        }
      } else {
        // FP32: the O(dt) increment inc = a0 (Q_base - Q_k) + w_in + bdt R is
        // formed in float; with a double-float state it is added to Q_k exactly
        // (two-sum), so the state keeps ~48 significant bits
        const float(*sKL)[4 * NN] = (const float(*)[4 * NN])(smem + C::O_QLO);
        const float(*sNH)[4 * NN] = (const float(*)[4 * NN])(smem + C::O_NHI);
        const float(*sNL)[4 * NN] = (const float(*)[4 * NN])(smem + C::O_NLO);
        const float(*sW)[4 * NN] = (const float(*)[4 * NN])(smem + C::O_AUX);
        float *oh = (float *)va.out.hi, *ol = (float *)va.out.lo;
        float hv[4];
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const float R = -(float)((sRF[l2][(v) * NN + sp] + sRG[l2][(v) * NN + sp]) * iJ);
          const float h = (float)sQ[l2][(v) * NN + sp];
          float inc = __fmul_rn((float)va.rk.bdt, R);
          if constexpr (DF) {
            const float l = sKL[l2][(v) * NN + sp];
            if (use_base) inc = fmaf((float)va.rk.a0, (sNH[l2][(v) * NN + sp] - h) + (sNL[l2][(v) * NN + sp] - l), inc);
            if (AUX) inc += sW[l2][(v) * NN + sp];
            float sum, err;
            two_sum(h, inc, sum, err);
            err += l;
            const float H = sum + err;
            oh[gi + v * NN] = H;
            ol[gi + v * NN] = err - (H - sum);
            hv[v] = H;
          } else {
            // single-float state: the stage result is rounded to float once
            if (use_base) inc = fmaf((float)va.rk.a0, sNH[l2][(v) * NN + sp] - h, inc);
            if (AUX) inc += sW[l2][(v) * NN + sp];
            const float H = h + inc;
            oh[gi + v * NN] = H;
            hv[v] = H;
          }
          if (va.w_out) va.w_out[gi + v * NN] = (T)fmaf(-(float)va.rk.g, inc, (float)va.rk.ddt * R);
        }
        bad |= !physical(hv);
#pragma unroll
        for (int v = 0; v < 4; ++v) sQ[l2][(v) * NN + sp] = (T)hv[v];
      }
    }
    if (MODE == MODE_RK) {
      __syncthreads();
      // ---- phase 3: face traces of the new state, one thread per SP line:
      // xi line j -> faces 3 (xi = 0) and 1 (xi = 1) at point j; eta line i ->
      // faces 0 (eta = 0) and 2 (eta = 1) at point i ----
      if (le < ne) {
        T *tr = (T *)md.TR + (size_t)(e0 + le) * 16 * N;
        const int fa = d == 0 ? 3 : 0, fb = d == 0 ? 1 : 2;
        if constexpr (FF) {
#pragma unroll
          for (int vp = 0; vp < 2; ++vp) {
            float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < N; ++k) {
              const int sp = d == 0 ? mline * N + k : k * N + mline;
              const float2 qk = make_float2(sQ[le][(2 * vp) * NN + sp], sQ[le][(2 * vp + 1) * NN + sp]);
              a0 = __ffma2_rn(qk, B.H02[k], a0);
              a1 = __ffma2_rn(qk, B.H12[k], a1);
            }
            tr[(fa * 4 + 2 * vp) * N + mline] = a0.x;
            tr[(fa * 4 + 2 * vp + 1) * N + mline] = a0.y;
            tr[(fb * 4 + 2 * vp) * N + mline] = a1.x;
            tr[(fb * 4 + 2 * vp + 1) * N + mline] = a1.y;
          }
        } else {
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            T a0 = 0, a1 = 0;
#pragma unroll
            for (int k = 0; k < N; ++k) {
              const T qk = d == 0 ? sQ[le][(v) * NN + mline * N + k] : sQ[le][(v) * NN + k * N + mline];
              a0 += qk * B.H0[k];
              a1 += qk * B.H1[k];
            }
            tr[(fa * 4 + v) * N + mline] = a0;
            tr[(fb * 4 + v) * N + mline] = a1;
          }
        }
      }
    }
    // every read of this tile's buffers is done before they are refilled (a
    // batch raises the non-physical flag on the tile's own case here)
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

#include "ssd_viscous.cuh"

namespace ssd {

// One launch for a face pass and the mortar flux of the same pass, which are
// independent: blocks [0, nmb) compute the mortar fluxes (MortCfg's MPB
// mortars each; the latency-bound mortar chain then runs under the face
// work), the rest one face point per thread.  MMODE selects the pair:
// RUSANOV with k_faces, AVG_Q with k_faces_cq, RUSANOV_FV with k_faces_visc.
constexpr int kFusedBlock = 256;

template <typename T, int N, bool OTF, int MMODE>
__global__ void __launch_bounds__(kFusedBlock) k_faces_mortar(MeshDev md, int nmb) {
  pdl_enter();
  static_assert(MortCfg<N>::THREADS <= kFusedBlock, "mortar block");
  if ((int)blockIdx.x < nmb) {
    mortar_flux_body<T, N, MMODE, MortCfg<N>::MPB>(md, blockIdx.x);
    return;
  }
  const int t = ((int)blockIdx.x - nmb) * kFusedBlock + threadIdx.x;
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

}  // namespace ssd

namespace ssd {

static __global__ void k_advance(DevClock *clk, double dt) {
  pdl_enter();
  clk->t_n = clk->t_n + dt;
}

}  // namespace ssd

#include "ssd_batch.cuh"

namespace ssd {

// ---------------------------------------------------------------------------
// engine
// ---------------------------------------------------------------------------
// LO: FP32 path with a double-float state (hi + lo planes); false: one float
// per value (FP32 state storage)
template <typename T, int N, bool LO = true>
struct EngineImpl : Engine {
  static constexpr bool OTF = std::is_same<T, float>::value;
  static constexpr bool DF = OTF && LO;
  using One = OneCase<VolArgs<T>>;
  using List = CaseList<VolArgs<T>>;

  template <int MODE, class Src>
  static cudaError_t visc_setup(int *occ) {
    using V = VisVolCfg<T, N>;
    auto *k = k_volume_visc<T, N, MODE, OTF, LO, Src>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, V::SMEM);
    if (err) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, V::THREADS, V::SMEM);
  }
  template <class Src>
  static cudaError_t grad_setup(int *occ) {
    using G = GradCfg<T, N>;
    auto *k = k_grad_trace<T, N, OTF, Src>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, G::SMEM);
    if (err) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, G::THREADS, G::SMEM);
  }

  // shared-memory attribute and resident CTAs per SM of one volume-kernel variant
  template <int MODE, bool AUX, int EPBX, class Src, bool TC = false>
  static cudaError_t vol_setup(int *occ) {
    using C = VolCfg<T, N, OTF, AUX, LO, EPBX, TC>;
    auto *k = k_volume<T, N, MODE, OTF, AUX, LO, EPBX, Src, TC>;
    cudaError_t err = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, C::SMEM);
    if (err) return err;
    return cudaOccupancyMaxActiveBlocksPerMultiprocessor(occ, k, C::THREADS, C::SMEM);
  }
  double *dXs = nullptr, *dXf = nullptr;
  int *scratch_i = nullptr;
  double *scratch_d = nullptr;
  void *sA[2] = {nullptr, nullptr}, *sB[2] = {nullptr, nullptr}, *sC[2] = {nullptr, nullptr};
  void *sW = nullptr;
  size_t nval = 0, nalloc_vals = 0;
  int merge_smem = 0;
  int grid_res = 1, grid_rk = 1, grid_aux = 1;  // persistent grid sizes of the volume kernel
  int grid_visc_res = 1, grid_visc_rk = 1;       // and of the viscous volume kernel
  int grid_grad = 1;                              // and of the gradient kernel
  bool fuse_faces_mortar = true;                  // mortar flux inside the face launch
  int sms = 1, occ_rk = 1;         // SM count, resident volume CTAs per SM
  int face_block = 256;            // block size of the conforming-face kernel
  bool tc = false;                 // volume contractions on the tensor cores (3xTF32, FP32 form)
  static constexpr bool kTC = OTF && LO;  // the engines that have the tensor-core variant
  int grid_tc_res = 1, grid_tc_rk = 1, grid_tc_aux = 1;
  int face_block_max = 256;        // the most threads per block its registers allow

  ~EngineImpl() override {
    cudaFree(dXs);
    cudaFree(dXf);
    cudaFree(scratch_i);
    cudaFree(scratch_d);
    for (int k = 0; k < 2; ++k) {
      cudaFree(sA[k]);
      cudaFree(sB[k]);
      cudaFree(sC[k]);
    }
    cudaFree(sW);
  }
  size_t geo_words() const override { return GeoLayout<N>::G; }
  size_t compute_word() const override { return sizeof(T); }
  bool metrics_on_the_fly() const override { return OTF; }

  cudaError_t alloc_state(int E, int Epad) override {
    nval = (size_t)E * 4 * N * N;
    const size_t nalloc = (size_t)Epad * 4 * N * N;
    nalloc_vals = nalloc;
    cudaError_t e;
    if ((e = cudaMalloc(&sA[0], sizeof(T) * nalloc))) return e;
    if ((e = cudaMalloc(&sB[0], sizeof(T) * nalloc))) return e;
    if (DF) {
      if ((e = cudaMalloc(&sA[1], sizeof(float) * nalloc))) return e;
      if ((e = cudaMalloc(&sB[1], sizeof(float) * nalloc))) return e;
    }
    return cudaSuccess;
  }
  StatePtr A() const override { return StatePtr{sA[0], sA[1]}; }
  StatePtr B() const override { return StatePtr{sB[0], sB[1]}; }

  void set_state(const MeshDev &, const double *Q, cudaStream_t s) override {
    if (DF)
      k_split<<<(unsigned)((nval + 255) / 256), 256, 0, s>>>(Q, (float *)sA[0], (float *)sA[1], nval);
    else if (OTF)
      k_split<<<(unsigned)((nval + 255) / 256), 256, 0, s>>>(Q, (float *)sA[0], nullptr, nval);
    else
      cudaMemcpyAsync(sA[0], Q, sizeof(double) * nval, cudaMemcpyDeviceToDevice, s);
  }
  void get_state(const MeshDev &, double *Q, cudaStream_t s) override {
    if (OTF)
      k_join<<<(unsigned)((nval + 255) / 256), 256, 0, s>>>((const float *)sA[0], (const float *)sA[1], Q, nval);
    else
      cudaMemcpyAsync(Q, sA[0], sizeof(double) * nval, cudaMemcpyDeviceToDevice, s);
  }

  cudaError_t init(const HostBasis &hb, const MeshDev &md, cudaStream_t s) override {
    VolBasis<T, N> vb;
    MortBasis<N> mb;
    for (int i = 0; i <= N; ++i)
      for (int k = 0; k < N; ++k) vb.Hf[i * N + k] = (T)hb.Hf[i * N + k];
    for (int k = 0; k < N; ++k)
      for (int i = 0; i <= N; ++i) vb.Dm[k * (N + 1) + i] = (T)hb.Dm[k * (N + 1) + i];
    for (int k = 0; k < N; ++k) {
      vb.H0[k] = (T)hb.H0[k];
      vb.H1[k] = (T)hb.H1[k];
      vb.Xs[k] = (T)hb.Xs[k];
      mb.zq[k] = hb.zq[k];
      mb.wq[k] = hb.wq[k];
      mb.Xs[k] = hb.Xs[k];
      mb.cden[k] = hb.cden[k];
    }
    for (int k = 0; k <= N; ++k) vb.Xf[k] = (T)hb.Xf[k];
    for (int k = 0; k < (N + 1) * N; ++k) {
      vb.Hf2[k] = make_float2((float)hb.Hf[k], (float)hb.Hf[k]);
      vb.Dm2[k] = make_float2((float)hb.Dm[k], (float)hb.Dm[k]);
    }
    for (int k = 0; k < N; ++k) {
      vb.H02[k] = make_float2((float)hb.H0[k], (float)hb.H0[k]);
      vb.H12[k] = make_float2((float)hb.H1[k], (float)hb.H1[k]);
    }
    for (int k = 0; k < N * N; ++k) {
      mb.Hz[k] = hb.Hz[k];
      mb.Minv[k] = hb.Minv[k];
      mb.wHz[k] = hb.wq[k / N] * hb.Hz[k];
      mb.Hz_f[k] = (float)mb.Hz[k];
      mb.wHz_f[k] = (float)mb.wHz[k];
      mb.Minv_f[k] = (float)mb.Minv[k];
    }
    cudaError_t err;
    if ((err = cudaMemcpyToSymbolAsync(cVB<T, N>, &vb, sizeof vb, 0, cudaMemcpyHostToDevice, s))) return err;
    if ((err = cudaMemcpyToSymbolAsync(cMB<N>, &mb, sizeof mb, 0, cudaMemcpyHostToDevice, s))) return err;
    if ((err = cudaMalloc(&dXs, sizeof(double) * N))) return err;
    if ((err = cudaMalloc(&dXf, sizeof(double) * (N + 1)))) return err;
    if ((err = cudaMemcpyAsync(dXs, hb.Xs, sizeof(double) * N, cudaMemcpyHostToDevice, s))) return err;
    if ((err = cudaMemcpyAsync(dXf, hb.Xf, sizeof(double) * (N + 1), cudaMemcpyHostToDevice, s))) return err;
    const int nb = md.nL + md.nR;
    if ((err = cudaMalloc(&scratch_i, sizeof(int) * (2 * nb + 1)))) return err;
    if ((err = cudaMalloc(&scratch_d, sizeof(double) * (2 * nb + 1)))) return err;
    merge_smem = (int)(2 * sizeof(double) * (md.nbmax > 0 ? md.nbmax : 1));  // one interface's angles
    if (merge_smem > 48 * 1024) {
      if ((err = cudaFuncSetAttribute(k_clock_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, merge_smem)))
        return err;
      if ((err = cudaFuncSetAttribute(k_clock_merge_stages, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                      merge_smem)))
        return err;
    }
    {
      // persistent volume kernel: as many CTAs as fit on the GPU at once
      using C = VolCfg<T, N, OTF, false, LO>;
      int dev = 0, occ0 = 0, occ1 = 0;
      if ((err = cudaGetDevice(&dev))) return err;
      if ((err = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev))) return err;
      int occ2 = 0;
      if ((err = vol_setup<MODE_RESIDUAL, false, 0, One>(&occ0))) return err;
      if ((err = vol_setup<MODE_RK, false, 0, One>(&occ1))) return err;
      if ((err = vol_setup<MODE_RK, true, 0, One>(&occ2))) return err;
      if constexpr (kTC) {
        int t0 = 0, t1 = 0, t2 = 0;
        if ((err = vol_setup<MODE_RESIDUAL, false, 0, One, true>(&t0))) return err;
        if ((err = vol_setup<MODE_RK, false, 0, One, true>(&t1))) return err;
        if ((err = vol_setup<MODE_RK, true, 0, One, true>(&t2))) return err;
        grid_tc_res = std::max(1, t0) * sms;
        grid_tc_rk = std::max(1, t1) * sms;
        grid_tc_aux = std::max(1, t2) * sms;
      }
      grid_res = std::max(1, occ0) * sms;
      occ_rk = std::max(1, occ1);
      grid_rk = occ_rk * sms;
      grid_aux = std::max(1, occ2) * sms;
      // the persistent viscous volume kernel likewise
      int ov0 = 0, ov1 = 0, og = 0;
      if ((err = visc_setup<MODE_RESIDUAL, One>(&ov0))) return err;
      if ((err = visc_setup<MODE_RK, One>(&ov1))) return err;
      grid_visc_res = std::max(1, ov0) * sms;
      grid_visc_rk = std::max(1, ov1) * sms;
      if ((err = grad_setup<One>(&og))) return err;
      grid_grad = std::max(1, og) * sms;
    }
    {
      cudaFuncAttributes fa;
      if ((err = cudaFuncGetAttributes(&fa, k_faces<T, N, OTF>))) return err;
      face_block_max = fa.maxThreadsPerBlock / 32 * 32;
      face_block = std::min(face_block, face_block_max);
    }
    if (md.nTab > 0) k_geo<T, N><<<(md.nTab + 127) / 128, 128, 0, s>>>(md, dXs, dXf);
    k_egeo<T, N><<<(md.E + 127) / 128, 128, 0, s>>>(md, dXs, dXf);
    if (md.nF > 0) k_fgeo<T, N, OTF><<<(md.nF * N + 127) / 128, 128, 0, s>>>(md);
    if (md.nB > 0) k_bgeo<N><<<(md.nB + 127) / 128, 128, 0, s>>>(md, dXs, (double *)md.bxy);
    return cudaGetLastError();
  }

  void trace(const MeshDev &md, StatePtr q, cudaStream_t s) override {
    const int n = md.E * 16 * N;
    launch_pdl(k_trace<T, N>, (n + 255) / 256, 256, 0, s, md, (const T *)q.hi);
  }

  void clock_merge(const MeshDev &md, double c, double dt, cudaStream_t s) override {
    launch_pdl(k_clock_merge, dim3(1, md.nI), 1024, merge_smem, s, md, c, dt, scratch_i, scratch_d);
    if (md.nM > 0) launch_pdl(k_mortar_xz, xz_blocks(md), kXzBlock, 0, s, md);
  }

  void clock_merge_into(const MeshDev &md, double c, double dt, int *work_i, double *work_d,
                        cudaStream_t s) override {
    launch_pdl(k_clock_merge, dim3(1, md.nI), 1024, merge_smem, s, md, c, dt, work_i, work_d);
    if (md.nM > 0) launch_pdl(k_mortar_xz, xz_blocks(md), kXzBlock, 0, s, md);
  }

  void merge_stages(const MeshDev &md, const StageMerge &sm, double dt, int first, int count, int ahead,
                    int threads, cudaStream_t s) override {
    if (count <= 0) return;
    launch_pdl(k_clock_merge_stages, dim3(count, md.nI), threads, merge_smem, s, md, sm, dt, first, ahead);
    if (md.nM > 0) launch_pdl(k_mortar_xz_stages, dim3(xz_blocks(md), count), kXzBlock, 0, s, md, sm, first);
  }
  static unsigned xz_blocks(const MeshDev &md) { return (unsigned)((2 * md.nM + kXzBlock - 1) / kXzBlock); }

  // the mortar flux as its own launch; the gather of its contributions into
  // each interface face is done by the kernel that reads the result
  // (gather_tile in k_volume, k_volume_visc, k_grad_trace)
  template <int MMODE>
  void mortar_flux(const MeshDev &md, cudaStream_t s) {
    constexpr int MPB = MortCfg<N>::MPB;
    launch_pdl(k_mortar_flux<T, N, MMODE>, (md.nM + MPB - 1) / MPB, MortCfg<N>::THREADS, 0, s, md);
  }

  // a face pass fused with the mortar flux of the same pass (meshes with an
  // interface)
  template <int MMODE>
  void fused_pass(const MeshDev &md, cudaStream_t s) {
    constexpr int MPB = MortCfg<N>::MPB;
    const int nmb = (md.nM + MPB - 1) / MPB;
    const int np = (md.nF + md.nB) * N;
    launch_pdl(k_faces_mortar<T, N, OTF, MMODE>, nmb + (np + kFusedBlock - 1) / kFusedBlock, kFusedBlock, 0, s, md,
               nmb);
  }
  bool fused(const MeshDev &md) const { return fuse_faces_mortar && md.nL > 0; }

  void faces(const MeshDev &md, StatePtr q, cudaStream_t s) override {
    const int np = (md.nF + md.nB) * N;
    if (!md.viscous) {
      if (fused(md)) fused_pass<MORTAR_RUSANOV>(md, s);
      else if (np > 0) launch_pdl(k_faces<T, N, OTF>, (np + face_block - 1) / face_block, face_block, 0, s, md);
      return;
    }
    // common solution, gradient traces, then common inviscid + viscous fluxes
    if (fused(md)) {
      fused_pass<MORTAR_AVG_Q>(md, s);
    } else {
      if (np > 0) launch_pdl(k_faces_cq<T, N, OTF>, (np + 255) / 256, 256, 0, s, md);
      if (md.nL > 0) mortar_flux<MORTAR_AVG_Q>(md, s);
    }
    using Gc = GradCfg<T, N>;
    const int ntg = (md.E + Gc::EPB - 1) / Gc::EPB;
    One src;
    src.md = md;
    src.a = vol_args(q, StatePtr{nullptr, nullptr}, StatePtr{nullptr, nullptr}, nullptr, RkArgs());
    launch_pdl(k_grad_trace<T, N, OTF, One>, std::min(ntg, grid_grad), Gc::THREADS, Gc::SMEM, s, src, ntg);
    if (fused(md)) fused_pass<MORTAR_RUSANOV_FV>(md, s);
    else if (np > 0) launch_pdl(k_faces_visc<T, N, OTF>, (np + 255) / 256, 256, 0, s, md);
  }

  // the mortar flux when it is not fused into the face pass (the gather is
  // done by the volume kernel)
  void mortars(const MeshDev &md, cudaStream_t s) override {
    if (md.nL > 0 && !fused(md)) {
      if (md.viscous) mortar_flux<MORTAR_RUSANOV_FV>(md, s);
      else mortar_flux<MORTAR_RUSANOV>(md, s);
    }
  }
  void set_fusion(bool on) override { fuse_faces_mortar = on; }

  static VolArgs<T> vol_args(StatePtr in, StatePtr base, StatePtr out, double *R, const RkArgs &rk) {
    VolArgs<T> a;
    a.in = in;
    a.base = base;
    a.out = out;
    a.R = R;
    a.rk = RkCoef<T>{(T)rk.a0, (T)rk.bdt, (T)rk.g, (T)rk.ddt};
    a.has_base = rk.has_base;
    a.w_out = (T *)rk.w_out;
    a.w_in = (const T *)rk.w_in;
    return a;
  }

  template <int MODE, bool AUX, bool TC = false>
  void launch_volume(const MeshDev &md, StatePtr in, StatePtr base, StatePtr out, double *R, const RkArgs &rk,
                     int grid, cudaStream_t s) {
    using C = VolCfg<T, N, OTF, AUX, LO, 0, TC>;
    const int ntiles = (md.E + C::EPB - 1) / C::EPB;
    One src;
    src.md = md;
    src.a = vol_args(in, base, out, R, rk);
    launch_pdl(k_volume<T, N, MODE, OTF, AUX, LO, 0, One, TC>, std::min(ntiles, grid), C::THREADS, C::SMEM, s, src,
               ntiles);
  }

  void volume(const MeshDev &md, StatePtr in, StatePtr base, StatePtr out, double *R, const RkArgs &rk, int mode,
              cudaStream_t s) override {
    if (md.viscous) {
      using V = VisVolCfg<T, N>;
      const int ntiles = (md.E + V::EPB - 1) / V::EPB;
      One src;
      src.md = md;
      src.a = vol_args(in, base, out, R, rk);
      if (mode == MODE_RESIDUAL)
        launch_pdl(k_volume_visc<T, N, MODE_RESIDUAL, OTF, LO, One>, std::min(ntiles, grid_visc_res), V::THREADS,
                   V::SMEM, s, src, ntiles);
      else
        launch_pdl(k_volume_visc<T, N, MODE_RK, OTF, LO, One>, std::min(ntiles, grid_visc_rk), V::THREADS, V::SMEM,
                   s, src, ntiles);
      return;
    }
    if constexpr (kTC) {
      if (tc) {
        if (mode == MODE_RESIDUAL) launch_volume<MODE_RESIDUAL, false, true>(md, in, base, out, R, rk, grid_tc_res, s);
        else if (rk.w_in) launch_volume<MODE_RK, true, true>(md, in, base, out, R, rk, grid_tc_aux, s);
        else launch_volume<MODE_RK, false, true>(md, in, base, out, R, rk, grid_tc_rk, s);
        return;
      }
    }
    if (mode == MODE_RESIDUAL) launch_volume<MODE_RESIDUAL, false>(md, in, base, out, R, rk, grid_res, s);
    else if (rk.w_in) launch_volume<MODE_RK, true>(md, in, base, out, R, rk, grid_aux, s);
    else launch_volume<MODE_RK, false>(md, in, base, out, R, rk, grid_rk, s);
  }
  bool set_tensor_cores(bool on) override {
    tc = kTC && on;
    return tc == on;
  }

  cudaError_t alloc_rk54() override {
    if (sC[0]) return cudaSuccess;
    const size_t nalloc = nalloc_vals;
    cudaError_t e;
    if ((e = cudaMalloc(&sC[0], sizeof(T) * nalloc))) return e;
    if (DF && (e = cudaMalloc(&sC[1], sizeof(float) * nalloc))) return e;
    if ((e = cudaMalloc(&sW, sizeof(T) * nalloc))) return e;
    return cudaSuccess;
  }
  StatePtr C() const override { return StatePtr{sC[0], sC[1]}; }
  void *W() const override { return sW; }

  // launch shapes chosen by the batch autotuner: volume CTAs per SM (capped
  // by occupancy; 0 keeps the current value) and the face-kernel block size
  void tuning(int *vol_ctas_per_sm, int *max_ctas_per_sm, int *fblock) override {
    if (max_ctas_per_sm) *max_ctas_per_sm = occ_rk;
    if (vol_ctas_per_sm) {
      if (*vol_ctas_per_sm > 0) grid_rk = std::min(*vol_ctas_per_sm, occ_rk) * sms;
      *vol_ctas_per_sm = grid_rk / sms;
    }
    if (fblock) {
      if (*fblock > 0) face_block = std::min(*fblock, face_block_max);
      *fblock = face_block;
    }
  }

  void advance(const MeshDev &md, double dt, cudaStream_t s) override {
    launch_pdl(k_advance, 1, 1, 0, s, md.clk, dt);
  }

  void sp_coords(const MeshDev &md, double t, double *xy, cudaStream_t s) override {
    k_spxy<N><<<(md.E + 127) / 128, 128, 0, s>>>(md, dXs, t, xy);
  }

  void reciprocal(const double *x, double *y, int n, cudaStream_t s) override {
    if (n > 0) k_reciprocal<T><<<(n + 255) / 256, 256, 0, s>>>(x, y, n);
  }

  // ---- batched form ----
  // elements per volume tile the batch autotuner chooses from: the default
  // tile and a smaller one (more, shorter work items)
  static constexpr int kEpbAlt = vol_epb_default<N>() >= 12 ? 8 : (vol_epb_default<N>() >= 8 ? 4 : 0);
  static constexpr int kFaceBlocks[3] = {128, 256, 512};
  static_assert(kElemPad % vol_epb_default<N>() == 0 && (kEpbAlt == 0 || kElemPad % kEpbAlt == 0) &&
                    kElemPad % VisCfg<T, N>::EPB == 0 && kElemPad % VisVolCfg<T, N>::EPB == 0,
                "every tile size divides the element padding");

  struct BatchImpl : BatchClass {
    int n = 0, nstages = 0, viscous = 0;
    std::vector<int> E, nF, nB, nM, nL, nR;  // per case
    std::vector<char> aux;                   // per stage: the stage carries an increment in (w_in)
    MeshDev *md = nullptr;                   // [nstages][n] stage views
    VolArgs<T> *va = nullptr;                // [nstages][n]
    int *off_tile = nullptr, *off_gtile = nullptr, *off_fblk = nullptr, *nmb = nullptr;
    int ntile = 0, ngtile = 0, nfblk = 0;
    int epb_alt = 0;       // 0: default tile, 1: the smaller tile
    int face_block = 256;  // face-pass block size
    int vol_ctas = 0;      // volume (or viscous volume) CTAs per SM
    int occ[2] = {1, 1};   // resident volume CTAs per SM for the default / smaller tile
    int occ_visc = 1, occ_grad = 1;
    std::vector<void *> allocs;
    ~BatchImpl() override {
      for (void *p : allocs) cudaFree(p);
    }
  };

  // debug build: after each batch launch outside a graph capture, wait and
  // name the launch if it failed
  static void dbg_sync(cudaStream_t s, const char *what) {
#ifdef SSD_DEBUG
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusNone) {
      cudaError_t e = cudaStreamSynchronize(s);
      if (e) fprintf(stderr, "ssd debug: N=%d %s: %s\n", N, what, cudaGetErrorString(e));
    }
#else
    (void)s;
    (void)what;
#endif
  }

  int batch_tile_choices(int *out) const override {
    out[0] = vol_epb_default<N>();
    if (kEpbAlt) out[1] = kEpbAlt;
    return kEpbAlt ? 2 : 1;
  }

  cudaError_t batch_offsets(BatchImpl &b, cudaStream_t s) {
    const int epb = b.epb_alt ? kEpbAlt : vol_epb_default<N>();
    const int vepb = b.viscous ? VisVolCfg<T, N>::EPB : epb;
    constexpr int MPB = MortCfg<N>::MPB;
    std::vector<int> ot(b.n + 1, 0), og(b.n + 1, 0), of(b.n + 1, 0), nm(b.n, 0);
    for (int c = 0; c < b.n; ++c) {
      ot[c + 1] = ot[c] + (b.E[c] + vepb - 1) / vepb;
      og[c + 1] = og[c] + (b.E[c] + GradCfg<T, N>::EPB - 1) / GradCfg<T, N>::EPB;
      nm[c] = (b.nM[c] + MPB - 1) / MPB;
      of[c + 1] = of[c] + nm[c] + ((b.nF[c] + b.nB[c]) * N + b.face_block - 1) / b.face_block;
    }
    b.ntile = ot[b.n];
    b.ngtile = og[b.n];
    b.nfblk = of[b.n];
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b.off_tile, ot.data(), sizeof(int) * (b.n + 1), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(b.off_gtile, og.data(), sizeof(int) * (b.n + 1), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(b.off_fblk, of.data(), sizeof(int) * (b.n + 1), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(b.nmb, nm.data(), sizeof(int) * b.n, cudaMemcpyHostToDevice, s))) return e;
    return cudaStreamSynchronize(s);  // the host vectors go out of scope
  }

  cudaError_t batch_args(BatchImpl &b, const std::vector<std::vector<BatchStageHost>> &stages, cudaStream_t s) {
    std::vector<MeshDev> mh((size_t)b.nstages * b.n);
    std::vector<VolArgs<T>> ah((size_t)b.nstages * b.n);
    for (int k = 0; k < b.nstages; ++k)
      for (int c = 0; c < b.n; ++c) {
        const BatchStageHost &h = stages[k][c];
        mh[(size_t)k * b.n + c] = h.md;
        ah[(size_t)k * b.n + c] = vol_args(h.in, h.base, h.out, nullptr, h.rk);
      }
    cudaError_t e;
    if ((e = cudaMemcpyAsync(b.md, mh.data(), sizeof(MeshDev) * mh.size(), cudaMemcpyHostToDevice, s))) return e;
    if ((e = cudaMemcpyAsync(b.va, ah.data(), sizeof(VolArgs<T>) * ah.size(), cudaMemcpyHostToDevice, s))) return e;
    return cudaStreamSynchronize(s);
  }

  BatchClass *batch_class(const std::vector<std::vector<BatchStageHost>> &stages, int viscous,
                          cudaStream_t s) override {
    BatchImpl *b = new BatchImpl();
    b->nstages = (int)stages.size();
    b->n = b->nstages ? (int)stages[0].size() : 0;
    b->viscous = viscous;
    for (int c = 0; c < b->n; ++c) {
      const MeshDev &m = stages[0][c].md;
      b->E.push_back(m.E);
      b->nF.push_back(m.nF);
      b->nB.push_back(m.nB);
      b->nM.push_back(m.nM);
      b->nL.push_back(m.nL);
      b->nR.push_back(m.nR);
    }
    for (int k = 0; k < b->nstages; ++k) b->aux.push_back(stages[k][0].rk.w_in != nullptr);
    auto al = [&](void **p, size_t bytes) {
      cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
      if (!e) b->allocs.push_back(*p);
      return e;
    };
    const size_t nk = (size_t)b->nstages * b->n;
    cudaError_t e = cudaSuccess;
    if (!e) e = al((void **)&b->md, sizeof(MeshDev) * nk);
    if (!e) e = al((void **)&b->va, sizeof(VolArgs<T>) * nk);
    if (!e) e = al((void **)&b->off_tile, sizeof(int) * (b->n + 1));
    if (!e) e = al((void **)&b->off_gtile, sizeof(int) * (b->n + 1));
    if (!e) e = al((void **)&b->off_fblk, sizeof(int) * (b->n + 1));
    if (!e) e = al((void **)&b->nmb, sizeof(int) * (b->n + 1));
    if (!e) e = batch_args(*b, stages, s);
    // resident CTAs per SM of the class's persistent kernels
    if (!e) e = vol_setup<MODE_RK, false, 0, List>(&b->occ[0]);
    if (!e) e = vol_setup<MODE_RK, true, 0, List>(&b->occ[0]);
    if (kEpbAlt) {
      if (!e) e = vol_setup<MODE_RK, false, kEpbAlt, List>(&b->occ[1]);
      if (!e) e = vol_setup<MODE_RK, true, kEpbAlt, List>(&b->occ[1]);
    }
    if (!e) e = visc_setup<MODE_RK, List>(&b->occ_visc);
    if (!e) e = grad_setup<List>(&b->occ_grad);
    if (!e) {
      b->vol_ctas = b->viscous ? b->occ_visc : b->occ[0];
      e = batch_offsets(*b, s);
    }
    if (e) {
      delete b;
      return nullptr;
    }
    return b;
  }

  cudaError_t batch_update(BatchClass *bc, const std::vector<std::vector<BatchStageHost>> &stages,
                           cudaStream_t s) override {
    return batch_args(*static_cast<BatchImpl *>(bc), stages, s);
  }

  void batch_tuning(BatchClass *bc, int *vol_ctas_per_sm, int *tile_elems, int *fblock, cudaStream_t s) override {
    BatchImpl &b = *static_cast<BatchImpl *>(bc);
    bool re = false;
    if (tile_elems && *tile_elems > 0 && !b.viscous) {
      const int alt = (kEpbAlt && *tile_elems == kEpbAlt) ? 1 : 0;
      re |= alt != b.epb_alt;
      b.epb_alt = alt;
    }
    const int occ = std::max(1, b.viscous ? b.occ_visc : b.occ[b.epb_alt]);
    if (vol_ctas_per_sm && *vol_ctas_per_sm > 0) b.vol_ctas = std::min(*vol_ctas_per_sm, occ);
    b.vol_ctas = std::max(1, std::min(b.vol_ctas, occ));
    if (fblock && *fblock > 0) {
      const int fb = *fblock <= 128 ? 128 : (*fblock <= 256 ? 256 : 512);
      re |= fb != b.face_block;
      b.face_block = fb;
    }
    if (re) batch_offsets(b, s);
    if (vol_ctas_per_sm) *vol_ctas_per_sm = b.vol_ctas;
    if (tile_elems) *tile_elems = b.viscous ? VisVolCfg<T, N>::EPB : (b.epb_alt ? kEpbAlt : vol_epb_default<N>());
    if (fblock) *fblock = b.face_block;
  }

  void batch_free(BatchClass *bc) override { delete static_cast<BatchImpl *>(bc); }

  template <int MMODE>
  void batch_face_pass(const BatchImpl &b, const BatchWork &w, cudaStream_t s) {
    if (b.nfblk == 0) return;
    if (b.face_block == 128) launch_pdl(k_batch_faces<T, N, OTF, MMODE, 128>, b.nfblk, 128, 0, s, w);
    else if (b.face_block == 256) launch_pdl(k_batch_faces<T, N, OTF, MMODE, 256>, b.nfblk, 256, 0, s, w);
    else launch_pdl(k_batch_faces<T, N, OTF, MMODE, 512>, b.nfblk, 512, 0, s, w);
    dbg_sync(s, "batch face pass");
  }


  template <bool AUX, int EPBX>
  void batch_volume(const BatchImpl &b, const List &src, cudaStream_t s) {
    using C = VolCfg<T, N, OTF, AUX, LO, EPBX>;
    launch_pdl(k_volume<T, N, MODE_RK, OTF, AUX, LO, EPBX, List>, std::max(1, std::min(b.ntile, b.vol_ctas * sms)),
               C::THREADS, C::SMEM, s, src, b.ntile);
    dbg_sync(s, "batch volume");
  }

  void batch_stage(BatchClass *bc, int k, cudaStream_t s) override {
    const BatchImpl &b = *static_cast<const BatchImpl *>(bc);
    BatchWork w{b.md + (size_t)k * b.n, b.off_fblk, b.nmb, b.n};
    List src;
    src.md = b.md + (size_t)k * b.n;
    src.a = b.va + (size_t)k * b.n;
    src.n = b.n;
    if (!b.viscous) {
      batch_face_pass<MORTAR_RUSANOV>(b, w, s);
      src.off = b.off_tile;
      const bool aux = b.aux[k];
      if (!b.epb_alt) {
        if (aux) batch_volume<true, 0>(b, src, s);
        else batch_volume<false, 0>(b, src, s);
      } else if (kEpbAlt) {
        if (aux) batch_volume<true, kEpbAlt>(b, src, s);
        else batch_volume<false, kEpbAlt>(b, src, s);
      }
      return;
    }
    // common solution, gradients and their traces, common fluxes, volume
    batch_face_pass<MORTAR_AVG_Q>(b, w, s);
    using G = GradCfg<T, N>;
    src.off = b.off_gtile;
    launch_pdl(k_grad_trace<T, N, OTF, List>, std::max(1, std::min(b.ngtile, std::max(1, b.occ_grad) * sms)),
               G::THREADS, G::SMEM, s, src, b.ngtile);
    dbg_sync(s, "batch gradients");
    batch_face_pass<MORTAR_RUSANOV_FV>(b, w, s);
    using V = VisVolCfg<T, N>;
    src.off = b.off_tile;
    launch_pdl(k_volume_visc<T, N, MODE_RK, OTF, LO, List>, std::max(1, std::min(b.ntile, b.vol_ctas * sms)),
               V::THREADS, V::SMEM, s, src, b.ntile);
    dbg_sync(s, "batch viscous volume");
  }

  void batch_merge(const BatchMergeDev &bm, cudaStream_t s) override {
    if (bm.smem > 48 * 1024) cudaFuncSetAttribute(k_batch_merge, cudaFuncAttributeMaxDynamicSharedMemorySize, bm.smem);
    launch_pdl(k_batch_merge, dim3(bm.max_iface, bm.nstages, bm.ncase), 1024, bm.smem, s, bm);
    dbg_sync(s, "batch merge");
    if (bm.max_nm > 0) {
      launch_pdl(k_batch_xz, dim3((2 * bm.max_nm + kXzBlock - 1) / kXzBlock, bm.nstages, bm.ncase), kXzBlock, 0, s,
                 bm);
      dbg_sync(s, "batch mortar offsets");
    }
  }

  void batch_advance(const BatchMergeDev &bm, cudaStream_t s) override {
    launch_pdl(k_batch_advance, (bm.ncase + 127) / 128, 128, 0, s, bm);
  }
};

template <typename T, bool LO = true>
Engine *make_engine_t(int N) {
  switch (N) {
    case 3: return new EngineImpl<T, 3, LO>();
    case 4: return new EngineImpl<T, 4, LO>();
    case 5: return new EngineImpl<T, 5, LO>();
    case 6: return new EngineImpl<T, 6, LO>();
    default: return nullptr;
  }
}

}  // namespace ssd
