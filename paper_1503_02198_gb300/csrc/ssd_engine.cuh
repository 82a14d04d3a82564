// ssd_engine.cuh -- sm_103a kernels of the sliding-mesh spectral difference
// residual and its SSP Runge-Kutta stage update, templated on the compute
// type T (double: FP64 path; float: FP32 path) and on N (solution points per
// direction, Sec. 3.1).  The state and the Runge-Kutta accumulation are FP64
// in both paths; so are the rotation angle, the mortar geometry and the
// mortar projection weights (Sec. 3.2).
//
// Per stage (stage time t_k):
//   k_clock_merge   1 CTA: theta = omega t_k; merge of the rotated L node
//                   angles with the R node angles -> mortars, (o, s) of each
//                   mortar against its L and R face (Eq. xz), face ranges
//   k_face          conforming and periodic faces: Rusanov common flux
//   k_bface         isothermal wall faces: Rusanov through a ghost state
//   k_mortar_flux   per mortar: L2 projection of both sides' face traces
//                   (Eq. prjQ2), Rusanov at the mortar SPs, back-projection
//                   weights of the common flux (Eq. prjF2)
//   k_mortar_gather per interface face point: deterministic sum over the
//                   face's mortars -> common flux of the face
//   k_volume        per element: SP -> FP interpolation (Eq. Qt), transformed
//                   ALE fluxes (Eq. transform_relation), common fluxes at the
//                   end FPs, divergence (Eqs. Ft, Gt), RK update and the face
//                   traces of the new state
#pragma once

#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include "ssd_internal.h"

namespace ssd {

// ---------------------------------------------------------------------------
// constants
// ---------------------------------------------------------------------------

template <typename T, int N>
struct VolBasis {
  T Hf[(N + 1) * N];  // h_k(X_{i+1/2}) [i][k]
  T Dm[N * (N + 1)];  // l'_{i+1/2}(X_k) [k][i]
  T H0[N], H1[N];     // h_k(0), h_k(1)
};

template <int N>
struct MortBasis {
  double zq[N], wq[N];  // Gauss-Legendre on [0,1]
  double Hz[N * N];     // h_j(z_q) [q][j]
  double Minv[N * N];   // M^{-1}
  double Xs[N];         // solution points
  double cden[N];       // 1 / prod_{s != i}(X_i - X_s)
};

template <typename T, int N>
__constant__ VolBasis<T, N> cVB;
template <int N>
__constant__ MortBasis<N> cMB;

// metric table of one element, t = 0 (words of type T)
template <int N>
struct GeoLayout {
  static constexpr int NF = N * (N + 1);
  static constexpr int ax = 0, ay = NF, gx = 2 * NF;      // xi-FPs [j][i]: (y_eta, -x_eta), V_g . a
  static constexpr int bx = 3 * NF, by = 4 * NF, gy = 5 * NF;  // eta-FPs [i'][i]: (-y_xi, x_xi), V_g . b
  static constexpr int iJ = 6 * NF;                       // 1/|J| at SPs [j][i]
  static constexpr int grad = 6 * NF + N * N;             // xi_x, xi_y, eta_x, eta_y at SPs [4][N*N]
  static constexpr int G = 6 * NF + 5 * N * N;
};

// face f of an element: sign sigma_f with F~_end = sigma_f |S| F.n_out
__device__ __forceinline__ double face_sigma(int f) { return (f == 1 || f == 2) ? 1.0 : -1.0; }

// ---------------------------------------------------------------------------
// geometry (Sec. 3.1 iso-parametric cells; Sec. 2.3 metrics)
// ---------------------------------------------------------------------------

// point and parameter derivative of the edge from P to Q at u in [0,1]; an arc
// edge is the circle about the origin (coordinates are centre-relative)
__device__ inline void edge_point(double px, double py, double qx, double qy, bool arc, double u, double &x,
                                  double &y, double &dx, double &dy) {
  if (!arc) {
    x = fma(u, qx - px, px);
    y = fma(u, qy - py, py);
    dx = qx - px;
    dy = qy - py;
    return;
  }
  const double r = sqrt(px * px + py * py);
  const double phi0 = atan2(py, px);
  const double dphi = atan2(px * qy - py * qx, px * qx + py * qy);
  double sn, cs;
  sincos(fma(u, dphi, phi0), &sn, &cs);
  x = r * cs;
  y = r * sn;
  dx = -r * dphi * sn;
  dy = r * dphi * cs;
}

// transfinite map of a cell with corners c[8] (x0 y0 .. x3 y3) and arc bits
// at (xi, eta): out = x, y, x_xi, y_xi, x_eta, y_eta
__device__ inline void cell_map(const double *c, int arcs, double xi, double eta, double *out) {
  double bx, by, dbx, dby, tx, ty, dtx, dty, lx, ly, dlx, dly, rx, ry, drx, dry;
  edge_point(c[0], c[1], c[2], c[3], arcs & 1, xi, bx, by, dbx, dby);    // f0: n0 -> n1
  edge_point(c[2], c[3], c[4], c[5], arcs & 2, eta, rx, ry, drx, dry);   // f1: n1 -> n2
  edge_point(c[6], c[7], c[4], c[5], arcs & 4, xi, tx, ty, dtx, dty);    // f2: n3 -> n2
  edge_point(c[0], c[1], c[6], c[7], arcs & 8, eta, lx, ly, dlx, dly);   // f3: n0 -> n3
  const double a = 1.0 - xi, b = 1.0 - eta;
  // bilinear corner blend and its derivatives
  const double cxv = a * b * c[0] + xi * b * c[2] + xi * eta * c[4] + a * eta * c[6];
  const double cyv = a * b * c[1] + xi * b * c[3] + xi * eta * c[5] + a * eta * c[7];
  const double cx_xi = -b * c[0] + b * c[2] + eta * c[4] - eta * c[6];
  const double cy_xi = -b * c[1] + b * c[3] + eta * c[5] - eta * c[7];
  const double cx_eta = -a * c[0] - xi * c[2] + xi * c[4] + a * c[6];
  const double cy_eta = -a * c[1] - xi * c[3] + xi * c[5] + a * c[7];
  out[0] = b * bx + eta * tx + a * lx + xi * rx - cxv;
  out[1] = b * by + eta * ty + a * ly + xi * ry - cyv;
  out[2] = b * dbx + eta * dtx - lx + rx - cx_xi;
  out[3] = b * dby + eta * dty - ly + ry - cy_xi;
  out[4] = -bx + tx + a * dlx + xi * drx - cx_eta;
  out[5] = -by + ty + a * dly + xi * dry - cy_eta;
}

// t = 0 metric tables of every element (one thread per element)
template <typename T, int N>
__global__ void k_geo(MeshDev md, const double *__restrict__ Xs, const double *__restrict__ Xf) {
  using L = GeoLayout<N>;
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= md.E) return;
  double c[8];
  for (int k = 0; k < 8; ++k) c[k] = md.corners[(size_t)e * 8 + k];
  const int arcs = md.arcs[e];
  const double om = md.zone[e] == 1 ? md.omega : 0.0;
  T *g = (T *)md.geo + (size_t)e * L::G;
  bool bad = false;
  double m[6];
  for (int j = 0; j < N; ++j)
    for (int i = 0; i <= N; ++i) {
      // xi-FP (X_{i+1/2}, X_j)
      cell_map(c, arcs, Xf[i], Xs[j], m);
      const double ax = m[5], ay = -m[4];
      g[L::ax + j * (N + 1) + i] = (T)ax;
      g[L::ay + j * (N + 1) + i] = (T)ay;
      g[L::gx + j * (N + 1) + i] = (T)(om * (-m[1] * ax + m[0] * ay));
      bad |= !(m[2] * m[5] - m[4] * m[3] > 0.0);
      // eta-FP (X_j, X_{i+1/2}) stored at FP row i, column j
      cell_map(c, arcs, Xs[j], Xf[i], m);
      const double bx = -m[3], by = m[2];
      g[L::bx + i * N + j] = (T)bx;
      g[L::by + i * N + j] = (T)by;
      g[L::gy + i * N + j] = (T)(om * (-m[1] * bx + m[0] * by));
      bad |= !(m[2] * m[5] - m[4] * m[3] > 0.0);
    }
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) {
      cell_map(c, arcs, Xs[i], Xs[j], m);
      const double J = m[2] * m[5] - m[4] * m[3];
      bad |= !(J > 0.0);
      g[L::iJ + j * N + i] = (T)(1.0 / J);
      g[L::grad + 0 * N * N + j * N + i] = (T)(m[5] / J);   // xi_x
      g[L::grad + 1 * N * N + j * N + i] = (T)(-m[4] / J);  // xi_y
      g[L::grad + 2 * N * N + j * N + i] = (T)(-m[3] / J);  // eta_x
      g[L::grad + 3 * N * N + j * N + i] = (T)(m[2] / J);   // eta_y
    }
  if (bad) atomicOr(&md.clk->flags, 2);
}

// t = 0 positions of boundary-face points (wall velocity of the rotating zone)
template <int N>
__global__ void k_bgeo(MeshDev md, const double *__restrict__ Xs, double *bxy) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= md.nB) return;
  const int ef = md.bfaces[b].x, e = ef >> 2, f = ef & 3;
  double c[8], m[6];
  for (int k = 0; k < 8; ++k) c[k] = md.corners[(size_t)e * 8 + k];
  for (int j = 0; j < N; ++j) {
    const double xi = (f == 0 || f == 2) ? Xs[j] : (f == 1 ? 1.0 : 0.0);
    const double eta = (f == 1 || f == 3) ? Xs[j] : (f == 2 ? 1.0 : 0.0);
    cell_map(c, md.arcs[e], xi, eta, m);
    bxy[((size_t)b * N + j) * 2] = m[0];
    bxy[((size_t)b * N + j) * 2 + 1] = m[1];
  }
}

// physical SP coordinates at time t, [E][N][N][2]
template <int N>
__global__ void k_spxy(MeshDev md, const double *__restrict__ Xs, double t, double cx, double cy, double *out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= md.E) return;
  double c[8], m[6];
  for (int k = 0; k < 8; ++k) c[k] = md.corners[(size_t)e * 8 + k];
  double cs = 1.0, sn = 0.0;
  if (md.zone[e] == 1) sincos(md.omega * t, &sn, &cs);
  for (int j = 0; j < N; ++j)
    for (int i = 0; i < N; ++i) {
      cell_map(c, md.arcs[e], Xs[i], Xs[j], m);
      out[(((size_t)e * N + j) * N + i) * 2] = cx + (cs * m[0] - sn * m[1]);
      out[(((size_t)e * N + j) * N + i) * 2 + 1] = cy + (sn * m[0] + cs * m[1]);
    }
}

// ---------------------------------------------------------------------------
// physics (Sec. 2)
// ---------------------------------------------------------------------------

template <typename T>
__device__ __forceinline__ T pressure_of(const T *q, T gm1) {
  return gm1 * (q[3] - T(0.5) * (q[1] * q[1] + q[2] * q[2]) / q[0]);
}

// normal ALE inviscid flux through a (not necessarily unit) vector (nx, ny):
// (F - u_g Q, G - v_g Q) . n  with vgn = V_g . n
template <typename T>
__device__ __forceinline__ void normal_flux(const T *q, T p, T nx, T ny, T vgn, T *f) {
  const T un = (q[1] * nx + q[2] * ny) / q[0];
  f[0] = q[0] * un - vgn * q[0];
  f[1] = q[1] * un + p * nx - vgn * q[1];
  f[2] = q[2] * un + p * ny - vgn * q[2];
  f[3] = (q[3] + p) * un - vgn * q[3];
}

// Rusanov common flux (Sec. 3.1) for unit normal n from L to R
template <typename T>
__device__ __forceinline__ void rusanov(const T *qL, const T *qR, T nx, T ny, T vgn, T gamma, T *Fn) {
  const T gm1 = gamma - T(1);
  const T pL = pressure_of(qL, gm1), pR = pressure_of(qR, gm1);
  T fL[4], fR[4];
  normal_flux(qL, pL, nx, ny, vgn, fL);
  normal_flux(qR, pR, nx, ny, vgn, fR);
  const T unL = (qL[1] * nx + qL[2] * ny) / qL[0], unR = (qR[1] * nx + qR[2] * ny) / qR[0];
  const T lL = fabs(unL - vgn) + sqrt(gamma * pL / qL[0]);
  const T lR = fabs(unR - vgn) + sqrt(gamma * pR / qR[0]);
  const T lam = lL > lR ? lL : lR;
#pragma unroll
  for (int v = 0; v < 4; ++v) Fn[v] = T(0.5) * (fL[v] + fR[v]) - T(0.5) * lam * (qR[v] - qL[v]);
}

// metric vector of the end FP at face f, point j, of an element's table
template <typename T, int N>
__device__ __forceinline__ void end_metric(const T *__restrict__ g, int f, int j, T &vx, T &vy, T &vg) {
  using L = GeoLayout<N>;
  int o0, o1, o2, idx;
  if (f == 1 || f == 3) {
    o0 = L::ax; o1 = L::ay; o2 = L::gx;
    idx = j * (N + 1) + (f == 1 ? N : 0);
  } else {
    o0 = L::bx; o1 = L::by; o2 = L::gy;
    idx = (f == 2 ? N : 0) * N + j;
  }
  vx = g[o0 + idx];
  vy = g[o1 + idx];
  vg = g[o2 + idx];
}

// ---------------------------------------------------------------------------
// per-stage coupling kernels
// ---------------------------------------------------------------------------

// Stage clock and mortar table (Sec. 3.2: connectivity updated at every
// stage).  Mortar k is the interval between merged node positions k and k+1
// (counter-clockwise, cyclic); nodes of both sides are sorted by angle, L
// before R on ties.  One CTA; loops cover any interface size.
__device__ __forceinline__ double wrap_2pi(double a) {
  const double tp = 6.283185307179586476925286766559;
  double r = fmod(a, tp);
  return r < 0.0 ? r + tp : r;
}

__device__ __forceinline__ double wrap_pi(double a) {
  const double pi = 3.14159265358979323846264338328;
  return wrap_2pi(a + pi) - pi;
}

static __global__ void k_clock_merge(MeshDev md, double c, double dt, int *scratch_i, double *scratch_d) {
  __shared__ double s_theta;
  __shared__ int s_k0;
  const int nL = md.nL, nR = md.nR, nb = nL + nR;
  if (threadIdx.x == 0) {
    DevClock *k = md.clk;
    const double ts = k->t_n + c * dt;
    const double th = md.omega * ts;
    k->t_stage = ts;
    k->theta = th;
    double sn, cs;
    sincos(th, &sn, &cs);
    k->c = cs;
    k->s = sn;
    s_theta = th;
    s_k0 = 0;
  }
  __syncthreads();
  if (nL == 0) return;
  const double th = s_theta;
  // rotated L angles: a cyclic shift of an ascending list; k0 = index of the minimum
  for (int k = threadIdx.x; k < nL; k += blockDim.x) {
    const double a = wrap_2pi(md.La[k] + th);
    scratch_d[k] = a;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nL; k += blockDim.x) {
    const int kp = k == 0 ? nL - 1 : k - 1;
    if (scratch_d[k] < scratch_d[kp]) s_k0 = k;
  }
  __syncthreads();
  const int k0 = s_k0;
  double *mAng = scratch_d + nL;  // [nb] merged angles
  int *posL = scratch_i;          // [nL] merged position of L node k (t=0 index)
  int *posR = scratch_i + nL;     // [nR]
  int *otherL = scratch_i + nb;   // [nL] R face containing the mortar that starts at L node k
  int *otherR = otherL + nL;      // [nR] L face (t=0 index) containing the mortar starting at R node k
  for (int k = threadIdx.x; k < nL; k += blockDim.x) {
    const double a = scratch_d[k];
    const int rank = (k - k0 + nL) % nL;
    // number of R angles strictly below a
    int lo = 0, hi = nR;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (md.Ra[mid] < a) lo = mid + 1; else hi = mid;
    }
    const int p = rank + lo;
    posL[k] = p;
    mAng[p] = a;
    otherL[k] = lo == 0 ? nR - 1 : lo - 1;
  }
  for (int k = threadIdx.x; k < nR; k += blockDim.x) {
    const double a = md.Ra[k];
    // number of rotated L angles <= a (L first on ties)
    int lo = 0, hi = nL;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (scratch_d[(k0 + mid) % nL] <= a) lo = mid + 1; else hi = mid;
    }
    const int p = k + lo;
    posR[k] = p;
    mAng[p] = a;
    otherR[k] = lo == 0 ? (k0 + nL - 1) % nL : (k0 + lo - 1) % nL;
  }
  __syncthreads();
  const double tp = 6.283185307179586476925286766559;
  for (int k = threadIdx.x; k < nL; k += blockDim.x) {
    const int p = posL[k];
    md.mLf[p] = k;
    md.mRf[p] = otherL[k];
    const int cnt = (posL[(k + 1) % nL] - p + nb) % nb;
    md.Lstart[k] = p;
    md.Lcount[k] = cnt == 0 ? nb : cnt;
  }
  for (int k = threadIdx.x; k < nR; k += blockDim.x) {
    const int p = posR[k];
    md.mRf[p] = k;
    md.mLf[p] = otherR[k];
    const int cnt = (posR[(k + 1) % nR] - p + nb) % nb;
    md.Rstart[k] = p;
    md.Rcount[k] = cnt == 0 ? nb : cnt;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < nb; p += blockDim.x) {
    const double a = mAng[p];
    const double b = p + 1 < nb ? mAng[p + 1] : mAng[0] + tp;
    const double d = b - a;
    const int fl = md.mLf[p], fr = md.mRf[p];
    const double aL = wrap_2pi(md.La[fl] + th);
    double *g = md.mgeo + (size_t)p * 6;
    g[0] = wrap_pi(a - aL) / md.Lw[fl];
    g[1] = d / md.Lw[fl];
    g[2] = wrap_pi(a - md.Ra[fr]) / md.Rw[fr];
    g[3] = d / md.Rw[fr];
    g[4] = a;
    g[5] = d;
  }
}

// Conforming and periodic faces: one thread per face point.
template <typename T, int N>
__global__ void k_face(MeshDev md) {
  using L = GeoLayout<N>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= md.nF * N) return;
  const int fi = t / N, j = t - fi * N;
  const int4 fc = md.faces[fi];
  const int efA = fc.x, efB = fc.y, jB = fc.z ? N - 1 - j : j;
  const int eA = efA >> 2, fA = efA & 3, eB = efB >> 2, fB = efB & 3;
  const T *TR = (const T *)md.TR;
  T qA[4], qB[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    qA[v] = TR[((size_t)efA * 4 + v) * N + j];
    qB[v] = TR[((size_t)efB * 4 + v) * N + jB];
  }
  const T *gA = (const T *)md.geo + (size_t)eA * L::G;
  const T *gB = (const T *)md.geo + (size_t)eB * L::G;
  T ax, ay, ag, bx, by, bg;
  end_metric<T, N>(gA, fA, j, ax, ay, ag);
  end_metric<T, N>(gB, fB, jB, bx, by, bg);
  if (md.zone[eA] == 1) {
    const T c = (T)md.clk->c, s = (T)md.clk->s;
    const T rx = c * ax - s * ay, ry = s * ax + c * ay;
    ax = rx;
    ay = ry;
  }
  const T SA = sqrt(ax * ax + ay * ay), SB = sqrt(bx * bx + by * by);
  const T sgA = (T)face_sigma(fA), sgB = (T)face_sigma(fB);
  const T nx = sgA * ax / SA, ny = sgA * ay / SA, vgn = sgA * ag / SA;
  T Fn[4];
  rusanov(qA, qB, nx, ny, vgn, (T)md.gamma, Fn);
  T *CF = (T *)md.CF;
#pragma unroll
  for (int v = 0; v < 4; ++v) {
    CF[((size_t)efA * 4 + v) * N + j] = sgA * SA * Fn[v];
    CF[((size_t)efB * 4 + v) * N + jB] = -sgB * SB * Fn[v];
  }
}

// Isothermal no-slip walls moving with their zone: Rusanov through a ghost
// state with velocity 2 V_w - V, the wall temperature and the interior pressure.
template <typename T, int N>
__global__ void k_bface(MeshDev md) {
  using L = GeoLayout<N>;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= md.nB * N) return;
  const int b = t / N, j = t - b * N;
  const int ef = md.bfaces[b].x, e = ef >> 2, f = ef & 3;
  const T *TR = (const T *)md.TR;
  T q[4], qg[4];
#pragma unroll
  for (int v = 0; v < 4; ++v) q[v] = TR[((size_t)ef * 4 + v) * N + j];
  const T *g = (const T *)md.geo + (size_t)e * L::G;
  T ax, ay, ag;
  end_metric<T, N>(g, f, j, ax, ay, ag);
  double uw = 0.0, vw = 0.0;
  if (md.zone[e] == 1) {
    const double c = md.clk->c, s = md.clk->s;
    const T rx = (T)c * ax - (T)s * ay, ry = (T)s * ax + (T)c * ay;
    ax = rx;
    ay = ry;
    const double x0 = md.bxy[((size_t)b * N + j) * 2], y0 = md.bxy[((size_t)b * N + j) * 2 + 1];
    const double x = c * x0 - s * y0, y = s * x0 + c * y0;
    uw = -md.omega * y;
    vw = md.omega * x;
  }
  const T S = sqrt(ax * ax + ay * ay), sg = (T)face_sigma(f);
  const T nx = sg * ax / S, ny = sg * ay / S, vgn = sg * ag / S;
  const T gm1 = (T)(md.gamma - 1.0);
  const T p = pressure_of(q, gm1);
  const T rho = p / (T)(md.Rgas * md.T_wall);
  const T gu = T(2) * (T)uw - q[1] / q[0], gv = T(2) * (T)vw - q[2] / q[0];
  qg[0] = rho;
  qg[1] = rho * gu;
  qg[2] = rho * gv;
  qg[3] = p / gm1 + T(0.5) * rho * (gu * gu + gv * gv);
  T Fn[4];
  rusanov(q, qg, nx, ny, vgn, (T)md.gamma, Fn);
  T *CF = (T *)md.CF;
#pragma unroll
  for (int v = 0; v < 4; ++v) CF[((size_t)ef * 4 + v) * N + j] = sg * S * Fn[v];
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

template <typename T, int N>
__global__ void __launch_bounds__(MortCfg<N>::THREADS) k_mortar_flux(MeshDev md) {
  constexpr int MPB = MortCfg<N>::MPB;
  __shared__ double sH[MPB][2][N][N];  // h_i(o + s z_q) [q][i]
  __shared__ T sQf[MPB][2][4][N];      // face values, CCW order
  __shared__ T sA[MPB][2][4][N];       // work arrays
  __shared__ T sB[MPB][2][4][N];
  __shared__ T sF[MPB][4][N];          // common mortar flux at mortar SPs
  __shared__ T sFz[MPB][4][N];         // common flux at quadrature points
  const int lm = threadIdx.x / (2 * N);
  const int r = threadIdx.x - lm * 2 * N;
  const int sd = r / N, p = r - sd * N;
  const int m = blockIdx.x * MPB + lm;
  const bool act = m < md.nM;
  const MortBasis<N> &B = cMB<N>;
  double o = 0.0, s = 0.0;
  int ef = 0, rev = 0;
  if (act) {
    const double *g = md.mgeo + (size_t)m * 6;
    o = g[sd ? 2 : 0];
    s = g[sd ? 3 : 1];
    const int4 fc = sd ? md.Rface[md.mRf[m]] : md.Lface[md.mLf[m]];
    ef = fc.x;
    rev = fc.y;
    const T *TR = (const T *)md.TR;
#pragma unroll
    for (int v = 0; v < 4; ++v) sQf[lm][sd][v][p] = TR[((size_t)ef * 4 + v) * N + (rev ? N - 1 - p : p)];
    // Lagrange values at the mapped quadrature point x = o + s z_p
    const double x = fma(s, B.zq[p], o);
    double dif[N];
#pragma unroll
    for (int k = 0; k < N; ++k) dif[k] = x - B.Xs[k];
#pragma unroll
    for (int i = 0; i < N; ++i) {
      double h = B.cden[i];
#pragma unroll
      for (int k = 0; k < N; ++k)
        if (k != i) h *= dif[k];
      sH[lm][sd][p][i] = h;
    }
  }
  __syncthreads();
  // (A) face polynomial at the mapped quadrature points
  if (act) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T acc = 0;
#pragma unroll
      for (int i = 0; i < N; ++i) acc += sQf[lm][sd][v][i] * (T)sH[lm][sd][p][i];
      sA[lm][sd][v][p] = acc;
    }
  }
  __syncthreads();
  // (B) right-hand side of Eq. prjQ1: (S^T Q)_p = sum_q w_q h_p(z_q) Q(o + s z_q)
  if (act) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T acc = 0;
#pragma unroll
      for (int q = 0; q < N; ++q) acc += (T)(B.wq[q] * B.Hz[q * N + p]) * sA[lm][sd][v][q];
      sB[lm][sd][v][p] = acc;
    }
  }
  __syncthreads();
  // (C) Q^Xi = M^{-1} S^T Q^Omega (Eq. prjQ2)
  if (act) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T acc = 0;
#pragma unroll
      for (int k = 0; k < N; ++k) acc += (T)B.Minv[p * N + k] * sB[lm][sd][v][k];
      sA[lm][sd][v][p] = acc;
    }
  }
  __syncthreads();
  // (D) Rusanov at mortar SP p with the radial normal (the grid velocity of
  // a rotation about the circle's centre is tangential: v_g . n = 0)
  if (act && sd == 0) {
    const double *g = md.mgeo + (size_t)m * 6;
    double sn, cs;
    sincos(fma(B.Xs[p], g[5], g[4]), &sn, &cs);
    T qL[4], qR[4], Fn[4];
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      qL[v] = sA[lm][0][v][p];
      qR[v] = sA[lm][1][v][p];
    }
    rusanov(qL, qR, (T)cs, (T)sn, T(0), (T)md.gamma, Fn);
#pragma unroll
    for (int v = 0; v < 4; ++v) sF[lm][v][p] = Fn[v];
  }
  __syncthreads();
  // (E) mortar flux polynomial at the quadrature points
  if (act && sd == 0) {
#pragma unroll
    for (int v = 0; v < 4; ++v) {
      T acc = 0;
#pragma unroll
      for (int j = 0; j < N; ++j) acc += (T)B.Hz[p * N + j] * sF[lm][v][j];
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
      for (int q = 0; q < N; ++q) acc += (T)(B.wq[q] * sH[lm][sd][q][p]) * sFz[lm][v][q];
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
      for (int k = 0; k < N; ++k) acc += (T)B.Minv[p * N + k] * sB[lm][sd][v][k];
      out[v * N + p] = (T)s * acc;
    }
  }
}

// Sum of the mortar contributions of each interface face (fixed order: the
// face's mortars in counter-clockwise order), written as the face's common
// flux F~_end = sigma_f |S| F.n_out (n from L to R is outward for L, inward
// for R).  One thread per (side, face, point).
template <typename T, int N>
__global__ void k_mortar_gather(MeshDev md) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nLR = md.nL + md.nR;
  if (t >= nLR * N) return;
  const int fq = t / N, p = t - fq * N;
  const int sd = fq >= md.nL;
  const int k = sd ? fq - md.nL : fq;
  const int start = sd ? md.Rstart[k] : md.Lstart[k];
  const int cnt = sd ? md.Rcount[k] : md.Lcount[k];
  const int4 fc = sd ? md.Rface[k] : md.Lface[k];
  const T *cb = (const T *)md.contrib + (size_t)sd * md.nM * 4 * N;
  T acc[4] = {0, 0, 0, 0};
  int mi = start;
  for (int c = 0; c < cnt; ++c) {
#pragma unroll
    for (int v = 0; v < 4; ++v) acc[v] += cb[((size_t)mi * 4 + v) * N + p];
    mi = mi + 1 == md.nM ? 0 : mi + 1;
  }
  const int ef = fc.x, f = ef & 3;
  const int j = fc.y ? N - 1 - p : p;
  const T S = (T)(sd ? md.RS[k] : md.LS[k]);
  const T sc = (T)face_sigma(f) * S * (sd ? T(-1) : T(1));
  T *CF = (T *)md.CF;
#pragma unroll
  for (int v = 0; v < 4; ++v) CF[((size_t)ef * 4 + v) * N + j] = sc * acc[v];
}

// ---------------------------------------------------------------------------
// traces of a state (used before the first stage and by the residual call)
// ---------------------------------------------------------------------------
template <typename T, int N>
__global__ void k_trace(MeshDev md, const double *__restrict__ Q) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= md.E * 16 * N) return;
  const int e = t / (16 * N);
  const int r = t - e * 16 * N;
  const int f = r / (4 * N), v = (r / N) & 3, j = r % N;
  const VolBasis<T, N> &B = cVB<T, N>;
  const double *q = Q + ((size_t)e * 4 + v) * N * N;
  T acc = 0;
#pragma unroll
  for (int k = 0; k < N; ++k) {
    // f0 eta=0 / f2 eta=1: column j; f1 xi=1 / f3 xi=0: row j
    const T qk = (T)((f == 0 || f == 2) ? q[k * N + j] : q[j * N + k]);
    acc += qk * ((f == 1 || f == 2) ? B.H1[k] : B.H0[k]);
  }
  ((T *)md.TR)[t] = acc;
}

// ---------------------------------------------------------------------------
// volume kernel
// ---------------------------------------------------------------------------
template <int N>
struct VolCfg {
  static constexpr int EPB = (128 / (2 * N)) > 0 ? 128 / (2 * N) : 1;  // elements per CTA
  static constexpr int THREADS = EPB * 2 * N;                          // one thread per line
};

template <typename T, int N, int MODE>
__global__ void __launch_bounds__(VolCfg<N>::THREADS)
    k_volume(MeshDev md, const double *Qin, const double *Qbase, double *Qout, double *Rout, double alpha,
             double beta, double dt) {
  using L = GeoLayout<N>;
  constexpr int EPB = VolCfg<N>::EPB, NT = VolCfg<N>::THREADS, NN = N * N;
  __shared__ T sQ[EPB][4][NN];
  __shared__ T sCF[EPB][16 * N];
  __shared__ T sRF[EPB][4][NN];
  __shared__ T sRG[EPB][4][NN];
  const VolBasis<T, N> &B = cVB<T, N>;
  const int e0 = blockIdx.x * EPB;
  const int ne = min(EPB, md.E - e0);
  // coalesced tile loads
  {
    const double *src = Qin + (size_t)e0 * 4 * NN;
    T *dst = &sQ[0][0][0];
    for (int i = threadIdx.x; i < ne * 4 * NN; i += NT) dst[i] = (T)src[i];
    const T *cf = (const T *)md.CF + (size_t)e0 * 16 * N;
    T *dcf = &sCF[0][0];
    for (int i = threadIdx.x; i < ne * 16 * N; i += NT) dcf[i] = cf[i];
  }
  __syncthreads();
  const T cth = (T)md.clk->c, sth = (T)md.clk->s;
  const T gam = (T)md.gamma, gm1 = (T)(md.gamma - 1.0);
  {
    const int le = threadIdx.x / (2 * N);
    const int r = threadIdx.x - le * 2 * N;
    const int d = r / N, mline = r - d * N;
    if (le < ne) {
      const int e = e0 + le;
      const bool rot = md.zone[e] == 1;
      const T *g = (const T *)md.geo + (size_t)e * L::G;
      T q[4][N];
#pragma unroll
      for (int k = 0; k < N; ++k)
#pragma unroll
        for (int v = 0; v < 4; ++v) q[v][k] = d == 0 ? sQ[le][v][mline * N + k] : sQ[le][v][k * N + mline];
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
          const int gi = d == 0 ? mline * (N + 1) + i : i * N + mline;
          T vx = g[(d == 0 ? L::ax : L::bx) + gi];
          T vy = g[(d == 0 ? L::ay : L::by) + gi];
          const T vg = g[(d == 0 ? L::gx : L::gy) + gi];
          if (rot) {
            const T rx = cth * vx - sth * vy, ry = sth * vx + cth * vy;
            vx = rx;
            vy = ry;
          }
          const T p = pressure_of(qf, gm1);
          normal_flux(qf, p, vx, vy, vg, f);
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
          for (int v = 0; v < 4; ++v) sRF[le][v][mline * N + k] = acc[v][k];
      } else {
#pragma unroll
        for (int k = 0; k < N; ++k)
#pragma unroll
          for (int v = 0; v < 4; ++v) sRG[le][v][k * N + mline] = acc[v][k];
      }
    }
  }
  __syncthreads();
  // divergence -> dQ/dt at the SPs; one thread per SP (all four variables)
  bool bad = false;
  for (int idx = threadIdx.x; idx < ne * NN; idx += NT) {
    const int le = idx / NN, sp = idx - le * NN;
    const int e = e0 + le;
    const T *g = (const T *)md.geo + (size_t)e * L::G;
    const T iJ = g[L::iJ + sp];
    const size_t base = (size_t)e * 4 * NN + sp;
    if (MODE == MODE_RESIDUAL) {
#pragma unroll
      for (int v = 0; v < 4; ++v) Rout[base + v * NN] = -(double)((sRF[le][v][sp] + sRG[le][v][sp]) * iJ);
    } else {
      double qn[4];
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        const double R = -(double)((sRF[le][v][sp] + sRG[le][v][sp]) * iJ);
        const double qk = Qin[base + v * NN];
        double val = beta * (qk + dt * R);
        if (alpha != 0.0) val = alpha * Qbase[base + v * NN] + val;
        qn[v] = val;
      }
      const double pr = (md.gamma - 1.0) * (qn[3] - 0.5 * (qn[1] * qn[1] + qn[2] * qn[2]) / qn[0]);
      bad |= !(qn[0] > 0.0) || !(pr > 0.0) || !isfinite(qn[3]);
#pragma unroll
      for (int v = 0; v < 4; ++v) {
        Qout[base + v * NN] = qn[v];
        sQ[le][v][sp] = (T)qn[v];
      }
    }
  }
  if (MODE == MODE_RK) {
    if (bad) atomicOr(&md.clk->flags, 1);
    __syncthreads();
    // face traces of the new state, coalesced [E][4][4][N]
    T *tr = (T *)md.TR + (size_t)e0 * 16 * N;
    for (int idx = threadIdx.x; idx < ne * 16 * N; idx += NT) {
      const int le = idx / (16 * N);
      const int r = idx - le * 16 * N;
      const int f = r / (4 * N), v = (r / N) & 3, j = r % N;
      T acc = 0;
#pragma unroll
      for (int k = 0; k < N; ++k) {
        const T qk = (f == 0 || f == 2) ? sQ[le][v][k * N + j] : sQ[le][v][j * N + k];
        acc += qk * ((f == 1 || f == 2) ? B.H1[k] : B.H0[k]);
      }
      tr[idx] = acc;
    }
  }
}

static __global__ void k_advance(DevClock *clk, double dt) { clk->t_n = clk->t_n + dt; }

// ---------------------------------------------------------------------------
// engine
// ---------------------------------------------------------------------------
template <typename T, int N>
struct EngineImpl : Engine {
  double *dXs = nullptr, *dXf = nullptr;
  int *scratch_i = nullptr;
  double *scratch_d = nullptr;

  ~EngineImpl() override {
    cudaFree(dXs);
    cudaFree(dXf);
    cudaFree(scratch_i);
    cudaFree(scratch_d);
  }
  size_t geo_words() const override { return GeoLayout<N>::G; }
  size_t compute_word() const override { return sizeof(T); }

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
      mb.zq[k] = hb.zq[k];
      mb.wq[k] = hb.wq[k];
      mb.Xs[k] = hb.Xs[k];
      mb.cden[k] = hb.cden[k];
    }
    for (int k = 0; k < N * N; ++k) {
      mb.Hz[k] = hb.Hz[k];
      mb.Minv[k] = hb.Minv[k];
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
    if ((err = cudaMalloc(&scratch_d, sizeof(double) * (md.nL + nb + 1)))) return err;
    k_geo<T, N><<<(md.E + 127) / 128, 128, 0, s>>>(md, dXs, dXf);
    if (md.nB > 0) k_bgeo<N><<<(md.nB + 127) / 128, 128, 0, s>>>(md, dXs, (double *)md.bxy);
    // the stream synchronises in the caller before the geometry flag is read
    return cudaSuccess;
  }

  void trace(const MeshDev &md, const double *Q, cudaStream_t s) override {
    const int n = md.E * 16 * N;
    k_trace<T, N><<<(n + 255) / 256, 256, 0, s>>>(md, Q);
  }

  void clock_merge(const MeshDev &md, double c, double dt, cudaStream_t s) override {
    k_clock_merge<<<1, 1024, 0, s>>>(md, c, dt, scratch_i, scratch_d);
  }

  void clock_merge_into(const MeshDev &md, double c, double dt, int *work_i, double *work_d,
                        cudaStream_t s) override {
    k_clock_merge<<<1, 1024, 0, s>>>(md, c, dt, work_i, work_d);
  }

  void faces(const MeshDev &md, cudaStream_t s) override {
    if (md.nF > 0) k_face<T, N><<<(md.nF * N + 255) / 256, 256, 0, s>>>(md);
    if (md.nB > 0) k_bface<T, N><<<(md.nB * N + 127) / 128, 128, 0, s>>>(md);
  }

  void mortars(const MeshDev &md, cudaStream_t s) override {
    if (md.nL > 0) {
      constexpr int MPB = MortCfg<N>::MPB;
      k_mortar_flux<T, N><<<(md.nM + MPB - 1) / MPB, MortCfg<N>::THREADS, 0, s>>>(md);
      const int n = (md.nL + md.nR) * N;
      k_mortar_gather<T, N><<<(n + 127) / 128, 128, 0, s>>>(md);
    }
  }

  void volume(const MeshDev &md, const double *Qin, const double *Qbase, double *Qout, double *R, double alpha,
              double beta, double dt, int mode, cudaStream_t s) override {
    constexpr int EPB = VolCfg<N>::EPB;
    const int grid = (md.E + EPB - 1) / EPB;
    if (mode == MODE_RESIDUAL)
      k_volume<T, N, MODE_RESIDUAL><<<grid, VolCfg<N>::THREADS, 0, s>>>(md, Qin, Qbase, Qout, R, alpha, beta, dt);
    else
      k_volume<T, N, MODE_RK><<<grid, VolCfg<N>::THREADS, 0, s>>>(md, Qin, Qbase, Qout, R, alpha, beta, dt);
  }

  void advance(const MeshDev &md, double dt, cudaStream_t s) override { k_advance<<<1, 1, 0, s>>>(md.clk, dt); }

  void sp_coords(const MeshDev &md, double t, double cx, double cy, double *xy, cudaStream_t s) override {
    k_spxy<N><<<(md.E + 127) / 128, 128, 0, s>>>(md, dXs, t, cx, cy, xy);
  }
};

template <typename T>
Engine *make_engine_t(int N) {
  switch (N) {
    case 3: return new EngineImpl<T, 3>();
    case 4: return new EngineImpl<T, 4>();
    case 5: return new EngineImpl<T, 5>();
    case 6: return new EngineImpl<T, 6>();
    default: return nullptr;
  }
}

}  // namespace ssd
