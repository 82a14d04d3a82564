/*
 * ssd_oracle.c -- plain, slow FP64 CPU oracle of the sliding-mesh spectral
 * difference (SSD) method of Zhang & Liang (arXiv:1503.02198).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the CPU
 * baseline leg of the benchmark load this file.  It shares no code, header,
 * table or constant with the CUDA library: every basis, geometry, flux and
 * projection below is written out here from the paper.
 *
 * It follows the paper's steps in order, element by element, in plain loops:
 *   Sec. 3.1: SPs (Chebyshev-Gauss) and FPs (Legendre-Gauss + end points),
 *             Lagrange bases (Eqs. hbasis, lbasis), solution polynomial
 *             (Eq. Qt) evaluated at the FPs,
 *   Sec. 2.1/2.2: inviscid fluxes with the grid-velocity terms of the
 *             rotating zone, viscous fluxes,
 *   Sec. 2.3: transformed fluxes (Eq. transform_relation),
 *   Sec. 3.1: Rusanov common flux on conforming faces,
 *   Sec. 3.2: mortars on the sliding interface: Eq. xz, projection of face
 *             data to mortars (Eqs. prjQ1-2, mortarM, mortarS), Rusanov on the
 *             mortar, projection of the common flux back (Eqs. prjF1-2), and the
 *             viscous mortar procedure,
 *   Sec. 3.1: divergence of the flux polynomials (Eqs. Ft, Gt) at the SPs,
 *   Sec. 3: explicit SSP Runge-Kutta (three-stage Shu-Osher form).
 *
 * Readings where the paper is silent (each listed in the design notes):
 *   - projections are defined by the integral statements prjQ1 / prjF1;
 *     the integrals use exact (N+2)-point Gauss-Legendre quadrature;
 *   - the quantity projected back is the physical normal flux per unit
 *     length, oriented from the rotating (L) side to the stationary (R) side;
 *     the element end-FP flux is then  sigma_f |S| F.n_out;
 *   - interface faces are exact circular arcs, parameterised linearly in
 *     angle, so o(t), s(t) are angle ratios;
 *   - a face whose parameter runs clockwise is handled by reversing its point
 *     order (the SP set is symmetric);
 *   - Rusanov wave speed max(|u_n - v_gn| + c) over both sides;
 *   - conforming viscous coupling: common Q = average, common viscous flux =
 *     average of both sides' viscous flux evaluated with the common Q;
 *   - isothermal moving walls through a ghost state (velocity 2 V_w - V,
 *     wall temperature, interior pressure);
 *   - the boundary conditions of the elliptic-cylinder case of Sec. 4
 *     (slip walls, Dirichlet inlet, fixed-pressure outlet) through ghost
 *     states as well: slip mirrors the velocity relative to the wall in the
 *     normal direction, the inlet ghost is the free stream, the outlet ghost is
 *     the interior state with the free-stream pressure.  For the viscous
 *     fluxes the common solution at a boundary point is the state on the
 *     boundary itself (slip: interior density and pressure with the normal
 *     relative velocity removed; inlet, outlet: the ghost state) and the
 *     viscous flux uses the interior gradient;
 *   - curved cells with 12 nodes (Sec. 3.1): an edge may be the cubic
 *     through its two corners and two edge nodes at face parameter 1/3 and
 *     2/3; the transfinite map with such edges spans exactly the 12-node
 *     serendipity cubic element;
 *   - several rotating zones (the paper has one per case): zone z >= 1 turns
 *     rigidly about its own centre at its own angular velocity and meets the
 *     stationary zone 0 across its own circular sliding interface; every
 *     interface is coupled by the procedure of Sec. 3.2 on its own.
 */
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

/* The real type of every value and operation.  The default build is FP64
 * (real = double), the oracle proper.  With -DOR_REAL_LONG the same source is
 * compiled with real = long double (64-bit significand on x86-64, IEEE
 * binary128 on AArch64): an extended-precision reference that shows how much
 * of the difference between two FP64 evaluations each one carries.  The math
 * functions are the type-generic ones of <tgmath.h>, so the FP64 build calls
 * the same double functions as a plain <math.h> build. */
#ifdef OR_REAL_LONG
typedef long double real;
#define OR_PI 3.141592653589793238462643383279502884L
#else
typedef double real;
#define OR_PI 3.14159265358979323846
#endif
#include <tgmath.h>
#undef I /* <complex.h> names the imaginary unit I; the code uses it for an interface */
#undef complex

#define OR_MAXN 12
#define OR_MAXZ 4 /* rotating zones */

/* ------------------------------------------------------------------------ */
/* parameters and mesh                                                       */
/* ------------------------------------------------------------------------ */

typedef struct {
  real gamma, Rgas, mu, prandtl, omega, T_wall;
  int viscous;
  real rho_inf, u_inf, v_inf, p_inf; /* free stream (inlet state, outlet pressure) */
} or_params;

/* boundary tags */
enum { BC_WALL = 1, BC_SLIP = 2, BC_INLET = 3, BC_OUTLET = 4, BC_ADIABATIC = 5 };
/* edge kinds */
enum { EDGE_STRAIGHT = 0, EDGE_ARC = 1, EDGE_CUBIC = 2 };

enum { FK_NONE = -1, FK_CONF = 0, FK_PERIODIC = 1, FK_BOUNDARY = 2, FK_IFACE_L = 3, FK_IFACE_R = 4 };

/* A rotating zone z >= 1: rigid rotation theta = omega t about its centre
 * (Sec. 2.2), and its circular sliding interface of radius rI with the
 * stationary zone 0 (Sec. 3.2), the rotating cells being the L side. */
typedef struct {
  real cx, cy, rI, omega;
  int nL, nR;                /* interface faces, sorted counter-clockwise */
  int *Lef, *Ref;            /* element-face index */
  real *La, *Lw, *Ra, *Rw; /* CCW start angle at t = 0 (in [0, 2pi)) and angular width */
  int *Lrev, *Rrev;          /* 1 if the face parameter runs clockwise */
} or_iface;

typedef struct {
  int N;
  real Xs[OR_MAXN];     /* solution points X_s, s = 1..N (stored 0-based) */
  real Xf[OR_MAXN + 1]; /* flux points X_{s+1/2}, s = 0..N */
  /* mesh */
  int nn, ne;
  real *xy;
  int *en, *zone, *arc;
  int *enode; /* [E][4][2]: edge nodes at face parameter 1/3, 2/3 of cubic edges, or NULL */
  int *azone; /* [E]: the zone whose centre the cell's arc edges are drawn about */
  /* per element face e*4+f */
  int *fkind, *fnbr, *frev, *ftag;
  int nz;               /* rotating zones 1..nz */
  or_iface zi[OR_MAXZ]; /* zi[z - 1]: zone z */
  or_params prm;
  char err[256];
} or_mesh;

/* ------------------------------------------------------------------------ */
/* Sec. 3.1: solution and flux points, Lagrange bases                         */
/* ------------------------------------------------------------------------ */

/* Legendre polynomial P_n and derivative on [-1, 1] (three-term recurrence) */
static void legendre(int n, real x, real *P, real *dP) {
  real p0 = 1.0, p1 = x;
  if (n == 0) { *P = 1.0; *dP = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    real p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = n * (x * p1 - p0) / (x * x - 1.0);
}

/* roots of P_n on [-1,1] in ascending order, by Newton iteration; weights of
 * the Gauss-Legendre rule 2 / ((1 - x^2) P_n'(x)^2) */
static void gauss_legendre(int n, real *x, real *w) {
  for (int k = 1; k <= n; ++k) {
    real r = cos(OR_PI * (k - 0.25) / (n + 0.5));
    for (int it = 0; it < 200; ++it) {
      real P, dP;
      legendre(n, r, &P, &dP);
      real dr = P / dP;
      r -= dr;
      if (fabs(dr) < 1e-17) break;
    }
    real P, dP;
    legendre(n, r, &P, &dP);
    x[n - k] = r; /* cos(...) decreases with k */
    w[n - k] = 2.0 / ((1.0 - r * r) * dP * dP);
  }
}

static void make_points(int N, real *Xs, real *Xf) {
  for (int s = 1; s <= N; ++s) Xs[s - 1] = 0.5 * (1.0 - cos((2.0 * s - 1.0) * OR_PI / (2.0 * N)));
  real z[OR_MAXN], w[OR_MAXN];
  Xf[0] = 0.0;
  Xf[N] = 1.0;
  if (N >= 2) {
    gauss_legendre(N - 1, z, w);
    for (int k = 0; k < N - 1; ++k) Xf[k + 1] = 0.5 * (1.0 + z[k]);
  }
}

/* Lagrange basis on nodes[0..n-1], product formula (Eqs. hbasis / lbasis) */
static real lag(const real *nodes, int n, int i, real x) {
  real v = 1.0;
  for (int s = 0; s < n; ++s)
    if (s != i) v *= (x - nodes[s]) / (nodes[i] - nodes[s]);
  return v;
}

static real lag_d(const real *nodes, int n, int i, real x) {
  real sum = 0.0;
  for (int m = 0; m < n; ++m) {
    if (m == i) continue;
    real v = 1.0 / (nodes[i] - nodes[m]);
    for (int s = 0; s < n; ++s)
      if (s != i && s != m) v *= (x - nodes[s]) / (nodes[i] - nodes[s]);
    sum += v;
  }
  return sum;
}

/* ------------------------------------------------------------------------ */
/* Geometry: iso-parametric map of each cell to [0,1]^2 (Sec. 3.1), rigid   */
/* rotation of the rotating zone (Sec. 2.2), metrics (Sec. 2.3)              */
/* ------------------------------------------------------------------------ */

static const int FACE_A[4] = {0, 1, 3, 0}; /* start corner of face f's parameter */
static const int FACE_B[4] = {1, 2, 2, 3}; /* end corner */

/* Edge curve from P to Q at parameter u: offset of the point from P, and the
 * derivative.  An arc is about the centre (cx, cy); it is written with the chord form
 * e(phi0 + d) - e(phi0) = 2 sin(d/2) (-sin(phi0 + d/2), cos(phi0 + d/2)),
 * so the offset keeps full relative precision for short arcs far from the
 * centre. */
static void edge_curve(const or_mesh *m, real cx, real cy, real px, real py, real qx, real qy, int arc,
                       const int *mid, real u, real *ox, real *oy, real *dx, real *dy) {
  if (arc == EDGE_CUBIC) {
    /* cubic Lagrange interpolation through P, M1, M2, Q at u = 0, 1/3, 2/3, 1,
     * written as offsets from P */
    static const real un[4] = {0.0, 1.0 / 3.0, 2.0 / 3.0, 1.0};
    real Dx[4] = {0.0, m->xy[2 * mid[0]] - px, m->xy[2 * mid[1]] - px, qx - px};
    real Dy[4] = {0.0, m->xy[2 * mid[0] + 1] - py, m->xy[2 * mid[1] + 1] - py, qy - py};
    *ox = *oy = *dx = *dy = 0.0;
    for (int k = 1; k < 4; ++k) {
      real l = lag(un, 4, k, u), ld = lag_d(un, 4, k, u);
      *ox += l * Dx[k];
      *oy += l * Dy[k];
      *dx += ld * Dx[k];
      *dy += ld * Dy[k];
    }
    return;
  }
  if (!arc) {
    *ox = u * (qx - px);
    *oy = u * (qy - py);
    *dx = qx - px;
    *dy = qy - py;
    return;
  }
  real ax = px - cx, ay = py - cy, bx = qx - cx, by = qy - cy;
  real r = sqrt(ax * ax + ay * ay);
  real phi0 = atan2(ay, ax);
  real dphi = atan2(ax * by - ay * bx, ax * bx + ay * by);
  real half = 0.5 * u * dphi, chord = 2.0 * r * sin(half);
  *ox = -chord * sin(phi0 + half);
  *oy = chord * cos(phi0 + half);
  real phi = phi0 + u * dphi;
  *dx = -r * dphi * sin(phi);
  *dy = r * dphi * cos(phi);
}

/* Transfinite (Coons) map of element e at (xi, eta) at t = 0: position and the
 * four derivatives.  With straight edges it is the 4-node bilinear map; an arc
 * edge is reproduced exactly.  It is evaluated about the cell's first corner
 * (an exact shift in real arithmetic) so that the round-off of the metrics
 * scales with the cell size rather than with the coordinates. */
static void map_t0(const or_mesh *m, int e, real xi, real eta, real *g) {
  const int *n = m->en + 4 * e;
  real X[4], Y[4];
  for (int k = 0; k < 4; ++k) {
    X[k] = m->xy[2 * n[k]];
    Y[k] = m->xy[2 * n[k] + 1];
  }
  real U[4], V[4]; /* corners relative to corner 0 */
  for (int k = 0; k < 4; ++k) {
    U[k] = X[k] - X[0];
    V[k] = Y[k] - Y[0];
  }
  const int *a = m->arc + 4 * e;
  const int *md = m->enode ? m->enode + 8 * e : NULL;
  const real cx = m->zi[m->azone[e] - 1].cx, cy = m->zi[m->azone[e] - 1].cy; /* centre of arc edges */
  real Bx, By, dBx, dBy, Tx, Ty, dTx, dTy, Lx, Ly, dLx, dLy, Rx, Ry, dRx, dRy;
  edge_curve(m, cx, cy, X[0], Y[0], X[1], Y[1], a[0], md ? md + 0 : NULL, xi, &Bx, &By, &dBx, &dBy);  /* f0 */
  edge_curve(m, cx, cy, X[1], Y[1], X[2], Y[2], a[1], md ? md + 2 : NULL, eta, &Rx, &Ry, &dRx, &dRy); /* f1 */
  edge_curve(m, cx, cy, X[3], Y[3], X[2], Y[2], a[2], md ? md + 4 : NULL, xi, &Tx, &Ty, &dTx, &dTy);  /* f2 */
  edge_curve(m, cx, cy, X[0], Y[0], X[3], Y[3], a[3], md ? md + 6 : NULL, eta, &Lx, &Ly, &dLx, &dLy); /* f3 */
  /* edge points relative to corner 0 */
  Rx += U[1]; Ry += V[1];
  Tx += U[3]; Ty += V[3];
  real x = (1 - eta) * Bx + eta * Tx + (1 - xi) * Lx + xi * Rx -
             (xi * (1 - eta) * U[1] + xi * eta * U[2] + (1 - xi) * eta * U[3]);
  real y = (1 - eta) * By + eta * Ty + (1 - xi) * Ly + xi * Ry -
             (xi * (1 - eta) * V[1] + xi * eta * V[2] + (1 - xi) * eta * V[3]);
  real x_xi = (1 - eta) * dBx + eta * dTx - Lx + Rx - ((1 - eta) * U[1] + eta * U[2] - eta * U[3]);
  real y_xi = (1 - eta) * dBy + eta * dTy - Ly + Ry - ((1 - eta) * V[1] + eta * V[2] - eta * V[3]);
  real x_eta = -Bx + Tx + (1 - xi) * dLx + xi * dRx - (-xi * U[1] + xi * U[2] + (1 - xi) * U[3]);
  real y_eta = -By + Ty + (1 - xi) * dLy + xi * dRy - (-xi * V[1] + xi * V[2] + (1 - xi) * V[3]);
  g[0] = X[0] + x; g[1] = Y[0] + y; g[2] = x_xi; g[3] = y_xi; g[4] = x_eta; g[5] = y_eta;
}

/* Map at time t: cells of rotating zone z are rotated rigidly about the
 * zone's centre by theta = omega_z t (Sec. 2.2: coordinates updated
 * analytically). */
static void map_at(const or_mesh *m, int e, real xi, real eta, real t, real *g) {
  map_t0(m, e, xi, eta, g);
  if (m->zone[e] >= 1) {
    const or_iface *Z = &m->zi[m->zone[e] - 1];
    real th = Z->omega * t, c = cos(th), s = sin(th);
    real dx = g[0] - Z->cx, dy = g[1] - Z->cy;
    g[0] = Z->cx + c * dx - s * dy;
    g[1] = Z->cy + s * dx + c * dy;
    for (int k = 2; k < 6; k += 2) {
      real vx = g[k], vy = g[k + 1];
      g[k] = c * vx - s * vy;
      g[k + 1] = s * vx + c * vy;
    }
  }
}

/* grid velocity (u_g, v_g) = omega_z x (r - centre_z) on rotating zone z, 0 elsewhere */
static void grid_velocity(const or_mesh *m, int e, real x, real y, real *ug, real *vg) {
  if (m->zone[e] >= 1) {
    const or_iface *Z = &m->zi[m->zone[e] - 1];
    *ug = -Z->omega * (y - Z->cy);
    *vg = Z->omega * (x - Z->cx);
  } else {
    *ug = 0.0;
    *vg = 0.0;
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 2: physical fluxes                                                    */
/* ------------------------------------------------------------------------ */

static real pressure(const or_params *p, const real *q) {
  return (p->gamma - 1.0) * (q[3] - 0.5 * (q[1] * q[1] + q[2] * q[2]) / q[0]);
}

/* inviscid fluxes with grid-velocity terms (Sec. 2.2) */
static void inviscid_flux(const or_params *p, const real *q, real ug, real vg, real *F, real *G) {
  real u = q[1] / q[0], v = q[2] / q[0], pr = pressure(p, q);
  F[0] = q[1];
  F[1] = q[1] * u + pr;
  F[2] = q[1] * v;
  F[3] = (q[3] + pr) * u;
  G[0] = q[2];
  G[1] = q[2] * u;
  G[2] = q[2] * v + pr;
  G[3] = (q[3] + pr) * v;
  for (int k = 0; k < 4; ++k) {
    F[k] -= ug * q[k];
    G[k] -= vg * q[k];
  }
}

/* viscous fluxes (Sec. 2.1) from Q and the physical gradients dQ/dx, dQ/dy of
 * the conservative variables; includes the leading minus sign of the paper */
static void viscous_flux(const or_params *p, const real *q, const real *qx, const real *qy, real *F,
                         real *G) {
  real rho = q[0], u = q[1] / rho, v = q[2] / rho;
  real ux = (qx[1] - u * qx[0]) / rho, uy = (qy[1] - u * qy[0]) / rho;
  real vx = (qx[2] - v * qx[0]) / rho, vy = (qy[2] - v * qy[0]) / rho;
  real pr = pressure(p, q);
  real T = pr / (rho * p->Rgas);
  real px = (p->gamma - 1.0) * (qx[3] - (u * qx[1] + v * qx[2] - 0.5 * (u * u + v * v) * qx[0]));
  real py = (p->gamma - 1.0) * (qy[3] - (u * qy[1] + v * qy[2] - 0.5 * (u * u + v * v) * qy[0]));
  real Tx = (px - p->Rgas * T * qx[0]) / (rho * p->Rgas);
  real Ty = (py - p->Rgas * T * qy[0]) / (rho * p->Rgas);
  real mu = p->mu, lam = -2.0 / 3.0 * mu;
  real kc = mu * p->gamma * p->Rgas / ((p->gamma - 1.0) * p->prandtl);
  real txx = 2.0 * mu * ux + lam * (ux + vy);
  real tyy = 2.0 * mu * vy + lam * (ux + vy);
  real txy = mu * (uy + vx);
  F[0] = 0.0;
  F[1] = -txx;
  F[2] = -txy;
  F[3] = -(u * txx + v * txy + kc * Tx);
  G[0] = 0.0;
  G[1] = -txy;
  G[2] = -tyy;
  G[3] = -(u * txy + v * tyy + kc * Ty);
}

/* conductive heat flux -k grad T from Q and its gradients (the part of the
 * energy viscous flux an adiabatic wall removes): returns k T_x, k T_y */
static void conduction(const or_params *p, const real *q, const real *qx, const real *qy, real *kTx,
                       real *kTy) {
  real rho = q[0], u = q[1] / rho, v = q[2] / rho;
  real T = pressure(p, q) / (rho * p->Rgas);
  real px = (p->gamma - 1.0) * (qx[3] - (u * qx[1] + v * qx[2] - 0.5 * (u * u + v * v) * qx[0]));
  real py = (p->gamma - 1.0) * (qy[3] - (u * qy[1] + v * qy[2] - 0.5 * (u * u + v * v) * qy[0]));
  real kc = p->mu * p->gamma * p->Rgas / ((p->gamma - 1.0) * p->prandtl);
  *kTx = kc * (px - p->Rgas * T * qx[0]) / (rho * p->Rgas);
  *kTy = kc * (py - p->Rgas * T * qy[0]) / (rho * p->Rgas);
}

/* Rusanov common normal flux (Sec. 3.1) across a face with unit normal n
 * pointing from L to R; vgn is the grid velocity normal to the face. */
static void rusanov(const or_params *p, const real *qL, const real *qR, real nx, real ny, real vgn,
                    real *Fn) {
  real FL[4], GL[4], FR[4], GR[4];
  inviscid_flux(p, qL, 0.0, 0.0, FL, GL);
  inviscid_flux(p, qR, 0.0, 0.0, FR, GR);
  real unL = (qL[1] * nx + qL[2] * ny) / qL[0], unR = (qR[1] * nx + qR[2] * ny) / qR[0];
  real cL = sqrt(p->gamma * pressure(p, qL) / qL[0]), cR = sqrt(p->gamma * pressure(p, qR) / qR[0]);
  real lamL = fabs(unL - vgn) + cL, lamR = fabs(unR - vgn) + cR;
  real lam = lamL > lamR ? lamL : lamR;
  for (int k = 0; k < 4; ++k) {
    real fL = FL[k] * nx + GL[k] * ny - vgn * qL[k];
    real fR = FR[k] * nx + GR[k] * ny - vgn * qR[k];
    Fn[k] = 0.5 * (fL + fR) - 0.5 * lam * (qR[k] - qL[k]);
  }
}

/* ------------------------------------------------------------------------ */
/* Sec. 3.2: mortar matrices                                                  */
/* ------------------------------------------------------------------------ */

/* M_ij = int_0^1 h_i h_j dz and S_ij = int_0^1 h_i(o + s z) h_j(z) dz (Eqs.
 * mortarM, mortarS), by (N+2)-point Gauss-Legendre on [0,1] (exact: the
 * integrands have degree 2N-2). */
static void mortar_MS(int N, const real *Xs, real o, real s, real *M, real *S) {
  int nq = N + 2;
  real z[OR_MAXN + 2], w[OR_MAXN + 2];
  gauss_legendre(nq, z, w);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      real mij = 0.0, sij = 0.0;
      for (int q = 0; q < nq; ++q) {
        real zq = 0.5 * (1.0 + z[q]), wq = 0.5 * w[q];
        mij += wq * lag(Xs, N, i, zq) * lag(Xs, N, j, zq);
        sij += wq * lag(Xs, N, i, o + s * zq) * lag(Xs, N, j, zq);
      }
      M[i * N + j] = mij;
      S[i * N + j] = sij;
    }
}

/* inverse of a small dense matrix by Gauss-Jordan with partial pivoting */
static int invert(int n, const real *A, real *Ainv) {
  real W[OR_MAXN * 2 * OR_MAXN];
  int w2 = 2 * n;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < w2; ++j) W[i * w2 + j] = j < n ? A[i * n + j] : (j - n == i ? 1.0 : 0.0);
  for (int c = 0; c < n; ++c) {
    int piv = c;
    for (int r = c + 1; r < n; ++r)
      if (fabs(W[r * w2 + c]) > fabs(W[piv * w2 + c])) piv = r;
    if (W[piv * w2 + c] == 0.0) return -1;
    if (piv != c)
      for (int j = 0; j < w2; ++j) {
        real tmp = W[c * w2 + j];
        W[c * w2 + j] = W[piv * w2 + j];
        W[piv * w2 + j] = tmp;
      }
    real d = W[c * w2 + c];
    for (int j = 0; j < w2; ++j) W[c * w2 + j] /= d;
    for (int r = 0; r < n; ++r) {
      if (r == c) continue;
      real f = W[r * w2 + c];
      for (int j = 0; j < w2; ++j) W[r * w2 + j] -= f * W[c * w2 + j];
    }
  }
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) Ainv[i * n + j] = W[i * w2 + n + j];
  return 0;
}

/* Projection matrices for a mortar with offset o and scale s relative to a face:
 *   forward  (Eq. prjQ1):  M Q^Xi = S^T Q^Omega  ->  Pf = M^-1 S^T
 *   backward (Eq. prjF1):  M F^Omega = sum_k s_k S_k F^Xi_k  ->  Pb = s M^-1 S  */
void or_projection(int N, real o, real s, real *Pf, real *Pb) {
  real Xs[OR_MAXN], Xf[OR_MAXN + 1], M[OR_MAXN * OR_MAXN], S[OR_MAXN * OR_MAXN], Mi[OR_MAXN * OR_MAXN];
  make_points(N, Xs, Xf);
  mortar_MS(N, Xs, o, s, M, S);
  invert(N, M, Mi);
  for (int i = 0; i < N; ++i)
    for (int j = 0; j < N; ++j) {
      real f = 0.0, b = 0.0;
      for (int k = 0; k < N; ++k) {
        f += Mi[i * N + k] * S[j * N + k];
        b += Mi[i * N + k] * S[k * N + j];
      }
      Pf[i * N + j] = f;
      Pb[i * N + j] = s * b;
    }
}

/* Rusanov common flux for tests: gamma, the two states (rho, rho u, rho v, E),
 * the unit normal from L to R and the normal grid velocity -> Fn[4]. */
void or_rusanov(real gamma, const real *qL, const real *qR, real nx, real ny, real vgn, real *Fn) {
  or_params p;
  memset(&p, 0, sizeof p);
  p.gamma = gamma;
  p.Rgas = 1.0;
  rusanov(&p, qL, qR, nx, ny, vgn, Fn);
}

/* ------------------------------------------------------------------------ */
/* mesh set-up: face table, interface lists                                   */
/* ------------------------------------------------------------------------ */

typedef struct { int a, b, ef; } edge_key;

static int cmp_edge(const void *x, const void *y) {
  const edge_key *p = x, *q = y;
  if (p->a != q->a) return p->a < q->a ? -1 : 1;
  if (p->b != q->b) return p->b < q->b ? -1 : 1;
  return p->ef < q->ef ? -1 : (p->ef > q->ef);
}

static void face_nodes(const or_mesh *m, int ef, int *na, int *nb) {
  int e = ef / 4, f = ef % 4;
  *na = m->en[4 * e + FACE_A[f]];
  *nb = m->en[4 * e + FACE_B[f]];
}

static real wrap2pi(real a) {
  real r = fmod(a, 2.0 * OR_PI);
  if (r < 0) r += 2.0 * OR_PI;
  return r;
}

/* signed angle in (-pi, pi] */
static real wrap_pi(real a) {
  real r = wrap2pi(a + OR_PI) - OR_PI;
  return r;
}

static int setup_interface_side(or_mesh *m, const or_iface *I, int n, const int *faces, int kind, int **ef_out,
                                real **a_out, real **w_out, int **rev_out) {
  int *ef = malloc(sizeof(int) * (n > 0 ? n : 1));
  real *a = malloc(sizeof(real) * (n > 0 ? n : 1)), *w = malloc(sizeof(real) * (n > 0 ? n : 1));
  int *rv = malloc(sizeof(int) * (n > 0 ? n : 1));
  for (int k = 0; k < n; ++k) {
    int e = faces[2 * k], f = faces[2 * k + 1], na, nb;
    ef[k] = 4 * e + f;
    face_nodes(m, ef[k], &na, &nb);
    real pa = atan2(m->xy[2 * na + 1] - I->cy, m->xy[2 * na] - I->cx);
    real pb = atan2(m->xy[2 * nb + 1] - I->cy, m->xy[2 * nb] - I->cx);
    real d = wrap_pi(pb - pa);
    if (d > 0) {
      a[k] = wrap2pi(pa);
      w[k] = d;
      rv[k] = 0;
    } else {
      a[k] = wrap2pi(pb);
      w[k] = -d;
      rv[k] = 1;
    }
    if (m->fkind[ef[k]] != FK_NONE) {
      snprintf(m->err, sizeof m->err, "interface face %d/%d already classified", e, f);
      *ef_out = ef; *a_out = a; *w_out = w; *rev_out = rv;
      return -1;
    }
    m->fkind[ef[k]] = kind;
  }
  /* sort counter-clockwise by start angle (insertion sort; plain) */
  for (int i = 1; i < n; ++i)
    for (int j = i; j > 0 && a[j] < a[j - 1]; --j) {
      real ta = a[j]; a[j] = a[j - 1]; a[j - 1] = ta;
      real tw = w[j]; w[j] = w[j - 1]; w[j - 1] = tw;
      int te = ef[j]; ef[j] = ef[j - 1]; ef[j - 1] = te;
      int tr = rv[j]; rv[j] = rv[j - 1]; rv[j - 1] = tr;
    }
  real total = 0.0;
  for (int k = 0; k < n; ++k) total += w[k];
  *ef_out = ef; *a_out = a; *w_out = w; *rev_out = rv;
  if (n > 0 && fabs(total - 2.0 * OR_PI) > 1e-9) {
    snprintf(m->err, sizeof m->err, "interface side does not close (%.12f)", (double)total);
    return -1;
  }
  *ef_out = ef; *a_out = a; *w_out = w; *rev_out = rv;
  return 0;
}

void or_destroy(or_mesh *m);

/* Zone 1 is given by (cx, cy, rI), prm_in's omega and the interface lists
 * Lf / Rf; zones 2 .. nxz + 1 by xz[k] = (cx, cy, rI, omega), xcnt[k] =
 * (nL, nR) and their lists, concatenated in xfaces (L then R, zone by zone).
 * azone (or NULL: the cell's own zone, zone 1 for stationary cells) names the
 * zone whose centre a cell's arc edges are drawn about. */
or_mesh *or_create(int nn, const real *xy, int ne, const int *en, const int *zone, const int *arc,
                   const int *enode, int nb,
                   const int *bfaces, int np, const int *pfaces, int nL, const int *Lf, int nR, const int *Rf,
                   real cx, real cy, real rI, int N, const real *prm_in, int nxz, const real *xz,
                   const int *xcnt, const int *xfaces, const int *azone, char *err, int errlen) {
  or_mesh *m = calloc(1, sizeof(or_mesh));
  m->N = N;
  make_points(N, m->Xs, m->Xf);
  m->nn = nn;
  m->ne = ne;
  m->xy = malloc(sizeof(real) * 2 * nn);
  memcpy(m->xy, xy, sizeof(real) * 2 * nn);
  m->en = malloc(sizeof(int) * 4 * ne);
  memcpy(m->en, en, sizeof(int) * 4 * ne);
  m->zone = malloc(sizeof(int) * ne);
  memcpy(m->zone, zone, sizeof(int) * ne);
  m->arc = malloc(sizeof(int) * 4 * ne);
  memcpy(m->arc, arc, sizeof(int) * 4 * ne);
  m->enode = NULL;
  if (enode) {
    m->enode = malloc(sizeof(int) * 8 * ne);
    memcpy(m->enode, enode, sizeof(int) * 8 * ne);
  }
  m->prm.gamma = prm_in[0];
  m->prm.Rgas = prm_in[1];
  m->prm.mu = prm_in[2];
  m->prm.prandtl = prm_in[3];
  m->prm.omega = prm_in[4];
  m->prm.viscous = (int)prm_in[5];
  m->prm.T_wall = prm_in[6];
  m->prm.rho_inf = prm_in[7];
  m->prm.u_inf = prm_in[8];
  m->prm.v_inf = prm_in[9];
  m->prm.p_inf = prm_in[10];
  int rc = 0;
  if (nxz < 0 || nxz + 1 > OR_MAXZ) {
    snprintf(m->err, sizeof m->err, "at most %d rotating zones", OR_MAXZ);
    rc = -1;
    nxz = 0;
  }
  m->nz = 1 + nxz;
  m->zi[0].cx = cx;
  m->zi[0].cy = cy;
  m->zi[0].rI = rI;
  m->zi[0].omega = m->prm.omega;
  for (int k = 0; k < nxz; ++k) {
    m->zi[1 + k].cx = xz[4 * k];
    m->zi[1 + k].cy = xz[4 * k + 1];
    m->zi[1 + k].rI = xz[4 * k + 2];
    m->zi[1 + k].omega = xz[4 * k + 3];
  }
  m->azone = malloc(sizeof(int) * (ne > 0 ? ne : 1));
  for (int e = 0; e < ne; ++e) {
    m->azone[e] = azone ? azone[e] : (zone[e] >= 1 ? zone[e] : 1);
    if (zone[e] < 0 || zone[e] > m->nz) {
      snprintf(m->err, sizeof m->err, "zone of element %d out of range", e);
      rc = -1;
    } else if (m->azone[e] < 1 || m->azone[e] > m->nz || (zone[e] >= 1 && m->azone[e] != zone[e])) {
      snprintf(m->err, sizeof m->err, "arc zone of element %d invalid", e);
      rc = -1;
    }
  }
  if (rc) m->nz = 0; /* nothing of the interfaces is allocated */
  int nf = 4 * ne;
  m->fkind = malloc(sizeof(int) * nf);
  m->fnbr = malloc(sizeof(int) * nf);
  m->frev = malloc(sizeof(int) * nf);
  m->ftag = malloc(sizeof(int) * nf);
  for (int k = 0; k < nf; ++k) { m->fkind[k] = FK_NONE; m->fnbr[k] = -1; m->frev[k] = 0; m->ftag[k] = 0; }
  /* edge kinds: a cubic edge needs its two edge nodes */
  for (int k = 0; k < 4 * ne && !rc; ++k) {
    if (arc[k] < EDGE_STRAIGHT || arc[k] > EDGE_CUBIC) {
      snprintf(m->err, sizeof m->err, "unknown edge kind");
      rc = -1;
    } else if (arc[k] == EDGE_CUBIC &&
               (!enode || enode[2 * k] < 0 || enode[2 * k] >= nn || enode[2 * k + 1] < 0 || enode[2 * k + 1] >= nn)) {
      snprintf(m->err, sizeof m->err, "cubic edge without valid edge nodes");
      rc = -1;
    }
  }
  /* boundary faces */
  for (int k = 0; k < nb && !rc; ++k) {
    int ef = 4 * bfaces[3 * k] + bfaces[3 * k + 1];
    int tag = bfaces[3 * k + 2];
    if (tag < BC_WALL || tag > BC_ADIABATIC) { snprintf(m->err, sizeof m->err, "unknown boundary tag"); rc = -1; }
    if (m->fkind[ef] != FK_NONE) { snprintf(m->err, sizeof m->err, "boundary face repeated"); rc = -1; }
    m->fkind[ef] = FK_BOUNDARY;
    m->ftag[ef] = bfaces[3 * k + 2];
  }
  /* periodic pairs: orientation from the translation between the faces */
  for (int k = 0; k < np && !rc; ++k) {
    int efA = 4 * pfaces[4 * k] + pfaces[4 * k + 1], efB = 4 * pfaces[4 * k + 2] + pfaces[4 * k + 3];
    int a0, a1, b0, b1;
    face_nodes(m, efA, &a0, &a1);
    face_nodes(m, efB, &b0, &b1);
    real dx = 0.5 * (m->xy[2 * b0] + m->xy[2 * b1] - m->xy[2 * a0] - m->xy[2 * a1]);
    real dy = 0.5 * (m->xy[2 * b0 + 1] + m->xy[2 * b1 + 1] - m->xy[2 * a0 + 1] - m->xy[2 * a1 + 1]);
    real ds = hypot(m->xy[2 * a0] + dx - m->xy[2 * b0], m->xy[2 * a0 + 1] + dy - m->xy[2 * b0 + 1]);
    real dr = hypot(m->xy[2 * a0] + dx - m->xy[2 * b1], m->xy[2 * a0 + 1] + dy - m->xy[2 * b1 + 1]);
    int rev = dr < ds;
    if (m->fkind[efA] != FK_NONE || m->fkind[efB] != FK_NONE) {
      snprintf(m->err, sizeof m->err, "periodic face repeated");
      rc = -1;
    }
    m->fkind[efA] = m->fkind[efB] = FK_PERIODIC;
    m->fnbr[efA] = efB;
    m->fnbr[efB] = efA;
    m->frev[efA] = m->frev[efB] = rev;
  }
  /* interfaces: the L side of zone z's interface lies in zone z, the R side in zone 0 */
  const int *xf = xfaces;
  for (int z = 1; z <= m->nz; ++z) {
    or_iface *I = &m->zi[z - 1];
    const int *fl = z == 1 ? Lf : xf, *fr;
    I->nL = z == 1 ? nL : xcnt[2 * (z - 2)];
    I->nR = z == 1 ? nR : xcnt[2 * (z - 2) + 1];
    if (z > 1) xf += 2 * I->nL;
    fr = z == 1 ? Rf : xf;
    if (z > 1) xf += 2 * I->nR;
    if (rc) continue;
    rc = setup_interface_side(m, I, I->nL, fl, FK_IFACE_L, &I->Lef, &I->La, &I->Lw, &I->Lrev);
    if (!rc) rc = setup_interface_side(m, I, I->nR, fr, FK_IFACE_R, &I->Ref, &I->Ra, &I->Rw, &I->Rrev);
    for (int k = 0; k < I->nL && !rc; ++k)
      if (zone[I->Lef[k] / 4] != z) {
        snprintf(m->err, sizeof m->err, "rotating-side face of interface %d not in zone %d", z, z);
        rc = -1;
      }
    for (int k = 0; k < I->nR && !rc; ++k)
      if (zone[I->Ref[k] / 4] != 0) {
        snprintf(m->err, sizeof m->err, "stationary-side face of interface %d not in zone 0", z);
        rc = -1;
      }
    if (!rc && (I->nL == 0) != (I->nR == 0)) {
      snprintf(m->err, sizeof m->err, "interface %d has faces on one side only", z);
      rc = -1;
    }
  }
  /* conforming faces by shared node pairs */
  if (!rc) {
    edge_key *keys = malloc(sizeof(edge_key) * nf);
    int nk = 0;
    for (int ef = 0; ef < nf; ++ef) {
      if (m->fkind[ef] != FK_NONE) continue;
      int a, b;
      face_nodes(m, ef, &a, &b);
      keys[nk].a = a < b ? a : b;
      keys[nk].b = a < b ? b : a;
      keys[nk].ef = ef;
      ++nk;
    }
    qsort(keys, nk, sizeof(edge_key), cmp_edge);
    for (int k = 0; k < nk && !rc; ++k) {
      if (k + 1 < nk && keys[k + 1].a == keys[k].a && keys[k + 1].b == keys[k].b) {
        if (k + 2 < nk && keys[k + 2].a == keys[k].a && keys[k + 2].b == keys[k].b) {
          snprintf(m->err, sizeof m->err, "edge shared by more than two cells");
          rc = -1;
          break;
        }
        int efA = keys[k].ef, efB = keys[k + 1].ef, a0, a1, b0, b1;
        face_nodes(m, efA, &a0, &a1);
        face_nodes(m, efB, &b0, &b1);
        m->fkind[efA] = m->fkind[efB] = FK_CONF;
        m->fnbr[efA] = efB;
        m->fnbr[efB] = efA;
        m->frev[efA] = m->frev[efB] = (a0 != b0);
        /* both sides must describe the same curve */
        int kA = m->arc[efA], kB = m->arc[efB];
        if (kA != kB) {
          snprintf(m->err, sizeof m->err, "edge kinds differ across a conforming face");
          rc = -1;
        } else if (kA == EDGE_CUBIC) {
          const int *pA = m->enode + 2 * efA, *pB = m->enode + 2 * efB;
          int same = m->frev[efA] ? (pA[0] == pB[1] && pA[1] == pB[0]) : (pA[0] == pB[0] && pA[1] == pB[1]);
          if (!same) {
            snprintf(m->err, sizeof m->err, "cubic edge nodes differ across a conforming face");
            rc = -1;
          }
        }
        if (m->zone[efA / 4] != m->zone[efB / 4]) {
          snprintf(m->err, sizeof m->err, "conforming face joins two zones");
          rc = -1;
        }
        ++k;
      } else {
        snprintf(m->err, sizeof m->err, "face %d of element %d has no neighbour and no boundary condition",
                 keys[k].ef % 4, keys[k].ef / 4);
        rc = -1;
      }
    }
    free(keys);
  }
  for (int ef = 0; ef < nf && !rc; ++ef) {
    int k = m->fkind[ef];
    if ((k == FK_PERIODIC || k == FK_IFACE_L || k == FK_IFACE_R) && m->arc[ef] == EDGE_CUBIC) {
      snprintf(m->err, sizeof m->err, "periodic and interface faces cannot be cubic edges");
      rc = -1;
    }
  }
  if (rc) {
    if (err) snprintf(err, errlen, "%s", m->err);
    or_destroy(m);
    return NULL;
  }
  return m;
}

void or_destroy(or_mesh *m) {
  if (!m) return;
  free(m->xy); free(m->en); free(m->zone); free(m->arc); free(m->enode); free(m->azone);
  free(m->fkind); free(m->fnbr); free(m->frev); free(m->ftag);
  for (int z = 0; z < m->nz; ++z) {
    or_iface *I = &m->zi[z];
    free(I->Lef); free(I->La); free(I->Lw); free(I->Lrev);
    free(I->Ref); free(I->Ra); free(I->Rw); free(I->Rrev);
  }
  free(m);
}

/* physical coordinates of the SPs at time t, [E][N][N][2] (row j = eta index) */
void or_sp_coords(const or_mesh *m, real t, real *out) {
  int N = m->N;
  real g[6];
  for (int e = 0; e < m->ne; ++e)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        map_at(m, e, m->Xs[i], m->Xs[j], t, g);
        out[((e * N + j) * N + i) * 2] = g[0];
        out[((e * N + j) * N + i) * 2 + 1] = g[1];
      }
}

/* |J| at the SPs, [E][N][N] */
void or_sp_jacobian(const or_mesh *m, real *out) {
  int N = m->N;
  real g[6];
  for (int e = 0; e < m->ne; ++e)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i < N; ++i) {
        map_t0(m, e, m->Xs[i], m->Xs[j], g);
        out[(e * N + j) * N + i] = g[2] * g[5] - g[4] * g[3];
      }
}

void or_points(int N, real *Xs, real *Xf) { make_points(N, Xs, Xf); }

void or_gauss_legendre(int n, real *x, real *w) { gauss_legendre(n, x, w); }

void or_lagrange(const real *nodes, int n, const real *x, int nx, real *val, real *der) {
  for (int p = 0; p < nx; ++p)
    for (int i = 0; i < n; ++i) {
      val[p * n + i] = lag(nodes, n, i, x[p]);
      der[p * n + i] = lag_d(nodes, n, i, x[p]);
    }
}

const char *or_face_info(const or_mesh *m, int *kind, int *nbr, int *rev) {
  for (int k = 0; k < 4 * m->ne; ++k) {
    kind[k] = m->fkind[k];
    nbr[k] = m->fnbr[k];
    rev[k] = m->frev[k];
  }
  return m->err;
}

/* ------------------------------------------------------------------------ */
/* residual                                                                   */
/* ------------------------------------------------------------------------ */

/* index helpers.  Q layout [E][4][N][N] with row j (eta) and column i (xi).
 * xi-FP arrays [E][4][N][N+1]: row j, FP i.  eta-FP arrays [E][4][N+1][N]:
 * FP row j, column i. */
#define IQ(e, v, j, i) ((((size_t)(e) * 4 + (v)) * N + (j)) * N + (i))
#define IXF(e, v, j, i) ((((size_t)(e) * 4 + (v)) * N + (j)) * (N + 1) + (i))
#define IEF(e, v, j, i) ((((size_t)(e) * 4 + (v)) * (N + 1) + (j)) * N + (i))

/* value at face point (f, j) of an xi-FP or eta-FP array */
static size_t face_index(int N, int e, int f, int v, int j) {
  switch (f) {
    case 0: return IEF(e, v, 0, j);
    case 1: return IXF(e, v, j, N);
    case 2: return IEF(e, v, N, j);
    default: return IXF(e, v, j, 0);
  }
}

static const real FACE_SIGMA[4] = {-1.0, 1.0, 1.0, -1.0};

/* geometry at face point j of face f of element e, time t: outward unit normal,
 * |S| (length of the contravariant vector), position */
static void face_geom(const or_mesh *m, int e, int f, int j, real t, real *nx, real *ny, real *S, real *x,
                      real *y) {
  real g[6], ax, ay;
  real xi = 0, eta = 0;
  switch (f) {
    case 0: xi = m->Xs[j]; eta = 0.0; break;
    case 1: xi = 1.0; eta = m->Xs[j]; break;
    case 2: xi = m->Xs[j]; eta = 1.0; break;
    default: xi = 0.0; eta = m->Xs[j]; break;
  }
  map_at(m, e, xi, eta, t, g);
  if (f == 1 || f == 3) { ax = g[5]; ay = -g[4]; }  /* (y_eta, -x_eta) */
  else { ax = -g[3]; ay = g[2]; }                    /* (-y_xi, x_xi) */
  real len = sqrt(ax * ax + ay * ay);
  *S = len;
  *nx = FACE_SIGMA[f] * ax / len;
  *ny = FACE_SIGMA[f] * ay / len;
  *x = g[0];
  *y = g[1];
}

typedef struct {
  int nm;            /* number of non-degenerate mortars */
  int *lf, *rf;      /* index into the sorted L / R lists */
  real *oL, *sL, *oR, *sR, *m0, *dm;
} or_mortars;

/* Sec. 3.2: mortars of interface I at stage time t.  Its rotating (L) side
 * is turned by theta = omega t; the mortars are the intervals between
 * consecutive node angles of both sides, in counter-clockwise order. */
static void build_mortars(const or_iface *I, real t, or_mortars *mo) {
  int nL = I->nL, nR = I->nR, nb = nL + nR;
  real th = I->omega * t;
  real *ang = malloc(sizeof(real) * (nb > 0 ? nb : 1));
  for (int k = 0; k < nL; ++k) ang[k] = wrap2pi(I->La[k] + th);
  for (int k = 0; k < nR; ++k) ang[nL + k] = I->Ra[k];
  for (int i = 1; i < nb; ++i)
    for (int j = i; j > 0 && ang[j] < ang[j - 1]; --j) { real tt = ang[j]; ang[j] = ang[j - 1]; ang[j - 1] = tt; }
  mo->nm = 0;
  int na = nb > 0 ? nb : 1;
  mo->lf = malloc(sizeof(int) * na); mo->rf = malloc(sizeof(int) * na);
  mo->oL = malloc(sizeof(real) * na); mo->sL = malloc(sizeof(real) * na);
  mo->oR = malloc(sizeof(real) * na); mo->sR = malloc(sizeof(real) * na);
  mo->m0 = malloc(sizeof(real) * na); mo->dm = malloc(sizeof(real) * na);
  for (int k = 0; k < nb; ++k) {
    real a = ang[k], b = (k + 1 < nb) ? ang[k + 1] : ang[0] + 2.0 * OR_PI;
    real d = b - a;
    if (d <= 1e-13) continue;
    real mid = a + 0.5 * d;
    int fl = -1, fr = -1;
    real oL = 0, oR = 0;
    for (int q = 0; q < nL; ++q) {
      real st = wrap2pi(I->La[q] + th);
      real off = wrap2pi(mid - st);
      if (off < I->Lw[q]) { fl = q; oL = wrap_pi(a - st); break; }
    }
    for (int q = 0; q < nR; ++q) {
      real off = wrap2pi(mid - I->Ra[q]);
      if (off < I->Rw[q]) { fr = q; oR = wrap_pi(a - I->Ra[q]); break; }
    }
    if (fl < 0 || fr < 0) continue;
    int n = mo->nm++;
    mo->lf[n] = fl;
    mo->rf[n] = fr;
    mo->oL[n] = oL / I->Lw[fl];
    mo->sL[n] = d / I->Lw[fl];
    mo->oR[n] = oR / I->Rw[fr];
    mo->sR[n] = d / I->Rw[fr];
    mo->m0[n] = a;
    mo->dm[n] = d;
  }
  free(ang);
}

static void free_mortars(or_mortars *mo) {
  free(mo->lf); free(mo->rf); free(mo->oL); free(mo->sL); free(mo->oR); free(mo->sR); free(mo->m0); free(mo->dm);
}

/* Read the N values (per variable) at the face points of element face ef from
 * an FP array in counter-clockwise order (reversed if the face runs clockwise). */
static void gather_ccw(const or_mesh *m, const real *arr_xi, const real *arr_eta, int ef, int rev, int nv,
                       real *out) {
  int N = m->N, e = ef / 4, f = ef % 4;
  for (int v = 0; v < nv; ++v)
    for (int j = 0; j < N; ++j) {
      int jj = rev ? N - 1 - j : j;
      size_t idx = face_index(N, e, f, v, jj);
      out[v * N + j] = (f == 1 || f == 3) ? arr_xi[idx] : arr_eta[idx];
    }
}

/* Mortar coupling of one family of face fields (nv variables per point):
 *   mode 0: inviscid common flux: project Q^Omega of both sides to each mortar
 *           (Eq. prjQ2), Rusanov at the mortar SPs with the radial normal
 *           (Sec. 3.2), project the common flux back to both sides (Eq. prjF2);
 *   mode 1: common solution: project, average both sides, project back;
 *   mode 2: viscous flux: project the face values of F_vis . n (supplied per
 *           face point in Lval / Rval), average both sides, project back.
 * Lin/Rin: per sorted L/R face, nv*N values in CCW order.  Lout/Rout receive the
 * projected-back values in CCW order. */
static void mortar_couple(const or_mesh *m, const or_iface *I, const or_mortars *mo, int mode, const real *Lin,
                          const real *Rin, real *Lout, real *Rout) {
  int N = m->N;
  int nv = 4;
  memset(Lout, 0, sizeof(real) * I->nL * nv * N);
  memset(Rout, 0, sizeof(real) * I->nR * nv * N);
  real PfL[OR_MAXN * OR_MAXN], PbL[OR_MAXN * OR_MAXN], PfR[OR_MAXN * OR_MAXN], PbR[OR_MAXN * OR_MAXN];
  for (int k = 0; k < mo->nm; ++k) {
    int fl = mo->lf[k], fr = mo->rf[k];
    or_projection(N, mo->oL[k], mo->sL[k], PfL, PbL);
    or_projection(N, mo->oR[k], mo->sR[k], PfR, PbR);
    real qL[4 * OR_MAXN], qR[4 * OR_MAXN], fm[4 * OR_MAXN];
    for (int v = 0; v < nv; ++v)
      for (int i = 0; i < N; ++i) {
        real sl = 0.0, sr = 0.0;
        for (int j = 0; j < N; ++j) {
          sl += PfL[i * N + j] * Lin[(fl * nv + v) * N + j];
          sr += PfR[i * N + j] * Rin[(fr * nv + v) * N + j];
        }
        qL[v * N + i] = sl;
        qR[v * N + i] = sr;
      }
    if (mode == 0) {
      for (int i = 0; i < N; ++i) {
        real phi = mo->m0[k] + m->Xs[i] * mo->dm[k];
        real a[4], b[4], Fn[4];
        for (int v = 0; v < 4; ++v) { a[v] = qL[v * N + i]; b[v] = qR[v * N + i]; }
        /* on a circle about its zone's centre the grid velocity is tangential */
        rusanov(&m->prm, a, b, cos(phi), sin(phi), 0.0, Fn);
        for (int v = 0; v < 4; ++v) fm[v * N + i] = Fn[v];
      }
    } else {
      for (int x = 0; x < nv * N; ++x) fm[x] = 0.5 * (qL[x] + qR[x]);
    }
    for (int v = 0; v < nv; ++v)
      for (int i = 0; i < N; ++i) {
        real sl = 0.0, sr = 0.0;
        for (int j = 0; j < N; ++j) {
          sl += PbL[i * N + j] * fm[v * N + j];
          sr += PbR[i * N + j] * fm[v * N + j];
        }
        Lout[(fl * nv + v) * N + i] += sl;
        Rout[(fr * nv + v) * N + i] += sr;
      }
  }
}

/* conservative state from density, velocity and pressure */
static void from_primitive(const or_params *p, real rho, real u, real v, real pr, real *q) {
  q[0] = rho;
  q[1] = rho * u;
  q[2] = rho * v;
  q[3] = pr / (p->gamma - 1.0) + 0.5 * rho * (u * u + v * v);
}

/* Boundary conditions (readings; the paper names them only): the ghost state
 * qg that enters the Rusanov flux and the state qb on the boundary itself,
 * which is the common solution of the viscous terms.  (ug, vg) is the grid
 * velocity at the point, (nx, ny) the outward unit normal.
 *   wall   (isothermal, no slip, moving with its zone): ghost velocity
 *          2 V_g - V, wall temperature, interior pressure; on the wall V_g;
 *   adiabatic wall (no slip, moving with its zone; the stirred tank's
 *          blades, Sec. 4): as the isothermal wall with the interior
 *          temperature (interior density) instead of the wall temperature;
 *          its viscous flux carries no heat conduction;
 *   slip:  ghost velocity with the normal velocity relative to the wall
 *          mirrored, interior density and pressure; on the wall that
 *          normal component is zero;
 *   inlet  (Dirichlet): the free stream;
 *   outlet (fixed pressure): interior density and velocity, free-stream
 *          pressure. */
static void boundary_states(const or_params *p, int tag, const real *qi, real ug, real vg, real nx,
                            real ny, real *qg, real *qb) {
  real pr = pressure(p, qi), u = qi[1] / qi[0], v = qi[2] / qi[0];
  if (tag == BC_WALL) {
    real rho = pr / (p->Rgas * p->T_wall);
    from_primitive(p, rho, 2.0 * ug - u, 2.0 * vg - v, pr, qg);
    from_primitive(p, rho, ug, vg, pr, qb);
  } else if (tag == BC_ADIABATIC) {
    from_primitive(p, qi[0], 2.0 * ug - u, 2.0 * vg - v, pr, qg);
    from_primitive(p, qi[0], ug, vg, pr, qb);
  } else if (tag == BC_SLIP) {
    real wn = (u - ug) * nx + (v - vg) * ny;
    from_primitive(p, qi[0], u - 2.0 * wn * nx, v - 2.0 * wn * ny, pr, qg);
    from_primitive(p, qi[0], u - wn * nx, v - wn * ny, pr, qb);
  } else if (tag == BC_INLET) {
    from_primitive(p, p->rho_inf, p->u_inf, p->v_inf, p->p_inf, qg);
    from_primitive(p, p->rho_inf, p->u_inf, p->v_inf, p->p_inf, qb);
  } else {
    from_primitive(p, qi[0], u, v, p->p_inf, qg);
    from_primitive(p, qi[0], u, v, p->p_inf, qb);
  }
}

typedef struct {
  real *Qxi, *Qeta;   /* Q at xi / eta FPs */
  real *Fxi, *Geta;   /* transformed fluxes at xi / eta FPs */
  real *cQxi, *cQeta; /* common solution at face points (viscous) */
  real *gxi, *geta;   /* physical gradient at FPs: [E][8][..] as two 4-var blocks */
} or_work;

/* Residual; when scale is not NULL it also receives, per SP and variable,
 * (sum_i |l'_i(X_k)| |F~_i| + sum_i |l'_i(X_j)| |G~_i|) / |J|: the magnitude of
 * the terms the divergence adds up, which bounds its round-off. */
int or_residual_ex(or_mesh *m, const real *Q, real t, real *dQdt, real *scale);

int or_residual(or_mesh *m, const real *Q, real t, real *dQdt) { return or_residual_ex(m, Q, t, dQdt, NULL); }

int or_residual_ex(or_mesh *m, const real *Q, real t, real *dQdt, real *scale) {
  int N = m->N, ne = m->ne;
  const or_params *P = &m->prm;
  size_t nxf = (size_t)ne * 4 * N * (N + 1);
  real *Qxi = calloc(nxf, sizeof(real)), *Qeta = calloc(nxf, sizeof(real));
  real *Fxi = calloc(nxf, sizeof(real)), *Geta = calloc(nxf, sizeof(real));
  real *cQxi = NULL, *cQeta = NULL, *Gxx = NULL, *Gxy = NULL, *Gex = NULL, *Gey = NULL;
  real hf[(OR_MAXN + 1) * OR_MAXN], dl[OR_MAXN * (OR_MAXN + 1)];
  /* h_k(X_{i+1/2}) and l'_{i+1/2}(X_k) */
  for (int i = 0; i <= N; ++i)
    for (int k = 0; k < N; ++k) hf[i * N + k] = lag(m->Xs, N, k, m->Xf[i]);
  for (int k = 0; k < N; ++k)
    for (int i = 0; i <= N; ++i) dl[k * (N + 1) + i] = lag_d(m->Xf, N + 1, i, m->Xs[k]);

  /* step 1: solution polynomial (Eq. Qt) at all FPs */
  for (int e = 0; e < ne; ++e)
    for (int v = 0; v < 4; ++v)
      for (int j = 0; j < N; ++j)
        for (int i = 0; i <= N; ++i) {
          real sx = 0.0, se = 0.0;
          for (int k = 0; k < N; ++k) {
            sx += Q[IQ(e, v, j, k)] * hf[i * N + k];
            se += Q[IQ(e, v, k, j)] * hf[i * N + k];
          }
          Qxi[IXF(e, v, j, i)] = sx;
          Qeta[IEF(e, v, i, j)] = se;
        }

  /* step 2: inviscid fluxes (with grid velocity) at the FPs, transformed by
   * Eq. transform_relation: F~ = y_eta F - x_eta G, G~ = -y_xi F + x_xi G */
  for (int e = 0; e < ne; ++e)
    for (int j = 0; j < N; ++j)
      for (int i = 0; i <= N; ++i) {
        real g[6], q[4], F[4], G[4], ug, vg;
        map_at(m, e, m->Xf[i], m->Xs[j], t, g);
        grid_velocity(m, e, g[0], g[1], &ug, &vg);
        for (int v = 0; v < 4; ++v) q[v] = Qxi[IXF(e, v, j, i)];
        inviscid_flux(P, q, ug, vg, F, G);
        for (int v = 0; v < 4; ++v) Fxi[IXF(e, v, j, i)] = g[5] * F[v] - g[4] * G[v];
        map_at(m, e, m->Xs[j], m->Xf[i], t, g);
        grid_velocity(m, e, g[0], g[1], &ug, &vg);
        for (int v = 0; v < 4; ++v) q[v] = Qeta[IEF(e, v, i, j)];
        inviscid_flux(P, q, ug, vg, F, G);
        for (int v = 0; v < 4; ++v) Geta[IEF(e, v, i, j)] = -g[3] * F[v] + g[2] * G[v];
      }

  /* mortars of every interface at this stage time */
  or_mortars mos[OR_MAXZ];
  real *Lins[OR_MAXZ], *Rins[OR_MAXZ], *Louts[OR_MAXZ], *Routs[OR_MAXZ];
  memset(mos, 0, sizeof mos);
  for (int z = 0; z < m->nz; ++z) {
    const or_iface *I = &m->zi[z];
    Lins[z] = Rins[z] = Louts[z] = Routs[z] = NULL;
    if (I->nL == 0) continue;
    build_mortars(I, t, &mos[z]);
    Lins[z] = malloc(sizeof(real) * I->nL * 4 * N);
    Rins[z] = malloc(sizeof(real) * I->nR * 4 * N);
    Louts[z] = malloc(sizeof(real) * I->nL * 4 * N);
    Routs[z] = malloc(sizeof(real) * I->nR * 4 * N);
  }

  /* viscous: common solution, gradients, viscous fluxes at the FPs */
  real *Fv_face = NULL; /* common viscous normal flux per element face point [E*4][4][N] (outward) */
  if (P->viscous) {
    cQxi = calloc(nxf, sizeof(real));
    cQeta = calloc(nxf, sizeof(real));
    Gxx = calloc(nxf, sizeof(real)); Gxy = calloc(nxf, sizeof(real));
    Gex = calloc(nxf, sizeof(real)); Gey = calloc(nxf, sizeof(real));
    /* (a) common solution at every face point */
    for (int e = 0; e < ne; ++e)
      for (int f = 0; f < 4; ++f) {
        int ef = 4 * e + f, kind = m->fkind[ef];
        for (int j = 0; j < N; ++j) {
          real qi[4], qc[4];
          for (int v = 0; v < 4; ++v) {
            size_t id = face_index(N, e, f, v, j);
            qi[v] = (f == 1 || f == 3) ? Qxi[id] : Qeta[id];
          }
          if (kind == FK_CONF || kind == FK_PERIODIC) {
            int eb = m->fnbr[ef] / 4, fb = m->fnbr[ef] % 4, jb = m->frev[ef] ? N - 1 - j : j;
            for (int v = 0; v < 4; ++v) {
              size_t id = face_index(N, eb, fb, v, jb);
              real qo = (fb == 1 || fb == 3) ? Qxi[id] : Qeta[id];
              qc[v] = 0.5 * (qi[v] + qo);
            }
          } else if (kind == FK_BOUNDARY) {
            real nx, ny, S, x, y, ug, vg, qg[4];
            face_geom(m, e, f, j, t, &nx, &ny, &S, &x, &y);
            grid_velocity(m, e, x, y, &ug, &vg);
            boundary_states(P, m->ftag[ef], qi, ug, vg, nx, ny, qg, qc);
          } else {
            continue; /* interface: below */
          }
          for (int v = 0; v < 4; ++v) {
            size_t id = face_index(N, e, f, v, j);
            if (f == 1 || f == 3) cQxi[id] = qc[v]; else cQeta[id] = qc[v];
          }
        }
      }
    for (int z = 0; z < m->nz; ++z) {
      const or_iface *I = &m->zi[z];
      const int nL = I->nL, nR = I->nR;
      real *Lin = Lins[z], *Rin = Rins[z], *Lout = Louts[z], *Rout = Routs[z];
      const or_mortars *mo = &mos[z];
      if (nL == 0) continue;
      for (int k = 0; k < nL; ++k) gather_ccw(m, Qxi, Qeta, I->Lef[k], I->Lrev[k], 4, Lin + (size_t)k * 4 * N);
      for (int k = 0; k < nR; ++k) gather_ccw(m, Qxi, Qeta, I->Ref[k], I->Rrev[k], 4, Rin + (size_t)k * 4 * N);
      mortar_couple(m, I, mo, 1, Lin, Rin, Lout, Rout);
      for (int side = 0; side < 2; ++side) {
        int n = side ? nR : nL;
        for (int k = 0; k < n; ++k) {
          int ef = side ? I->Ref[k] : I->Lef[k], rev = side ? I->Rrev[k] : I->Lrev[k];
          const real *src = (side ? Rout : Lout) + (size_t)k * 4 * N;
          int e = ef / 4, f = ef % 4;
          for (int v = 0; v < 4; ++v)
            for (int j = 0; j < N; ++j) {
              int jj = rev ? N - 1 - j : j;
              size_t id = face_index(N, e, f, v, jj);
              if (f == 1 || f == 3) cQxi[id] = src[v * N + j]; else cQeta[id] = src[v * N + j];
            }
        }
      }
    }
    /* (b) gradients at the SPs: derivative of the degree-N polynomial through
     * the FP values, with the common solution at the end FPs; mapped to x, y
     * with the metrics at the SP (chain rule). */
    real *Qx = calloc((size_t)ne * 4 * N * N, sizeof(real)), *Qy = calloc((size_t)ne * 4 * N * N, sizeof(real));
    for (int e = 0; e < ne; ++e)
      for (int j = 0; j < N; ++j)
        for (int k = 0; k < N; ++k) {
          real g[6];
          map_at(m, e, m->Xs[k], m->Xs[j], t, g);
          real J = g[2] * g[5] - g[4] * g[3];
          for (int v = 0; v < 4; ++v) {
            real dxi = 0.0, deta = 0.0;
            for (int i = 0; i <= N; ++i) {
              real ax = (i == 0 || i == N) ? cQxi[IXF(e, v, j, i)] : Qxi[IXF(e, v, j, i)];
              real ae = (i == 0 || i == N) ? cQeta[IEF(e, v, i, k)] : Qeta[IEF(e, v, i, k)];
              dxi += ax * dl[k * (N + 1) + i];
              deta += ae * dl[j * (N + 1) + i];
            }
            /* SP (k, j): xi derivative along row j, eta derivative along column k */
            Qx[IQ(e, v, j, k)] = (g[5] * dxi - g[3] * deta) / J;
            Qy[IQ(e, v, j, k)] = (-g[4] * dxi + g[2] * deta) / J;
          }
        }
    /* (c) gradients interpolated to the FPs */
    for (int e = 0; e < ne; ++e)
      for (int v = 0; v < 4; ++v)
        for (int j = 0; j < N; ++j)
          for (int i = 0; i <= N; ++i) {
            real a = 0, b = 0, c = 0, d = 0;
            for (int k = 0; k < N; ++k) {
              a += Qx[IQ(e, v, j, k)] * hf[i * N + k];
              b += Qy[IQ(e, v, j, k)] * hf[i * N + k];
              c += Qx[IQ(e, v, k, j)] * hf[i * N + k];
              d += Qy[IQ(e, v, k, j)] * hf[i * N + k];
            }
            Gxx[IXF(e, v, j, i)] = a;
            Gxy[IXF(e, v, j, i)] = b;
            Gex[IEF(e, v, i, j)] = c;
            Gey[IEF(e, v, i, j)] = d;
          }
    free(Qx);
    free(Qy);
    /* (d) viscous fluxes at the interior FPs, transformed and added */
    for (int e = 0; e < ne; ++e)
      for (int j = 0; j < N; ++j)
        for (int i = 1; i < N; ++i) {
          real g[6], q[4], qx[4], qy[4], F[4], G[4];
          map_at(m, e, m->Xf[i], m->Xs[j], t, g);
          for (int v = 0; v < 4; ++v) { q[v] = Qxi[IXF(e, v, j, i)]; qx[v] = Gxx[IXF(e, v, j, i)]; qy[v] = Gxy[IXF(e, v, j, i)]; }
          viscous_flux(P, q, qx, qy, F, G);
          for (int v = 0; v < 4; ++v) Fxi[IXF(e, v, j, i)] += g[5] * F[v] - g[4] * G[v];
          map_at(m, e, m->Xs[j], m->Xf[i], t, g);
          for (int v = 0; v < 4; ++v) { q[v] = Qeta[IEF(e, v, i, j)]; qx[v] = Gex[IEF(e, v, i, j)]; qy[v] = Gey[IEF(e, v, i, j)]; }
          viscous_flux(P, q, qx, qy, F, G);
          for (int v = 0; v < 4; ++v) Geta[IEF(e, v, i, j)] += -g[3] * F[v] + g[2] * G[v];
        }
    /* (e) common viscous normal flux at the face points */
    Fv_face = calloc((size_t)ne * 4 * 4 * N, sizeof(real));
    for (int e = 0; e < ne; ++e)
      for (int f = 0; f < 4; ++f) {
        int ef = 4 * e + f, kind = m->fkind[ef];
        for (int j = 0; j < N; ++j) {
          real nx, ny, S, x, y, qc[4], gx[4], gy[4], F[4], G[4], fo[4];
          face_geom(m, e, f, j, t, &nx, &ny, &S, &x, &y);
          for (int v = 0; v < 4; ++v) {
            size_t id = face_index(N, e, f, v, j);
            int isx = (f == 1 || f == 3);
            qc[v] = isx ? cQxi[id] : cQeta[id];
            gx[v] = isx ? Gxx[id] : Gex[id];
            gy[v] = isx ? Gxy[id] : Gey[id];
          }
          viscous_flux(P, qc, gx, gy, F, G);
          for (int v = 0; v < 4; ++v) fo[v] = F[v] * nx + G[v] * ny; /* own side, outward */
          if (kind == FK_CONF || kind == FK_PERIODIC) {
            int eb = m->fnbr[ef] / 4, fb = m->fnbr[ef] % 4, jb = m->frev[ef] ? N - 1 - j : j;
            real gbx[4], gby[4], Fb[4], Gb[4];
            for (int v = 0; v < 4; ++v) {
              size_t id = face_index(N, eb, fb, v, jb);
              int isx = (fb == 1 || fb == 3);
              gbx[v] = isx ? Gxx[id] : Gex[id];
              gby[v] = isx ? Gxy[id] : Gey[id];
            }
            viscous_flux(P, qc, gbx, gby, Fb, Gb);
            for (int v = 0; v < 4; ++v) Fv_face[((size_t)ef * 4 + v) * N + j] = 0.5 * (fo[v] + Fb[v] * nx + Gb[v] * ny);
          } else if (kind == FK_BOUNDARY) {
            if (m->ftag[ef] == BC_ADIABATIC) {
              /* no heat through the wall: remove the conduction term of the energy flux */
              real kTx, kTy;
              conduction(P, qc, gx, gy, &kTx, &kTy);
              fo[3] += kTx * nx + kTy * ny;
            }
            for (int v = 0; v < 4; ++v) Fv_face[((size_t)ef * 4 + v) * N + j] = fo[v];
          } else {
            /* interface: store F_vis . n with n oriented from L to R, in the
             * face's own point order; projected below */
            real sgn = (kind == FK_IFACE_L) ? 1.0 : -1.0;
            for (int v = 0; v < 4; ++v) Fv_face[((size_t)ef * 4 + v) * N + j] = sgn * fo[v];
          }
        }
      }
    for (int z = 0; z < m->nz; ++z) {
      const or_iface *I = &m->zi[z];
      const int nL = I->nL, nR = I->nR;
      real *Lout = Louts[z], *Rout = Routs[z];
      const or_mortars *mo = &mos[z];
      if (nL == 0) continue;
      real *vL = calloc((size_t)nL * 4 * N, sizeof(real)), *vR = calloc((size_t)nR * 4 * N, sizeof(real));
      for (int side = 0; side < 2; ++side) {
        int n = side ? nR : nL;
        for (int k = 0; k < n; ++k) {
          int ef = side ? I->Ref[k] : I->Lef[k], rev = side ? I->Rrev[k] : I->Lrev[k];
          real *dst = (side ? vR : vL) + (size_t)k * 4 * N;
          for (int v = 0; v < 4; ++v)
            for (int j = 0; j < N; ++j) dst[v * N + j] = Fv_face[((size_t)ef * 4 + v) * N + (rev ? N - 1 - j : j)];
        }
      }
      mortar_couple(m, I, mo, 2, vL, vR, Lout, Rout);
      for (int side = 0; side < 2; ++side) {
        int n = side ? nR : nL;
        for (int k = 0; k < n; ++k) {
          int ef = side ? I->Ref[k] : I->Lef[k], rev = side ? I->Rrev[k] : I->Lrev[k];
          const real *src = (side ? Rout : Lout) + (size_t)k * 4 * N;
          real sgn = side ? -1.0 : 1.0; /* back to outward orientation */
          for (int v = 0; v < 4; ++v)
            for (int j = 0; j < N; ++j) Fv_face[((size_t)ef * 4 + v) * N + (rev ? N - 1 - j : j)] = sgn * src[v * N + j];
        }
      }
      free(vL);
      free(vR);
    }
  }

  /* step 3: common inviscid flux at every face point (Rusanov on conforming and
   * periodic faces and through boundary ghost states); end FP value
   * F~ = sigma_f |S| (F_inv + F_vis).n_out */
  for (int e = 0; e < ne; ++e)
    for (int f = 0; f < 4; ++f) {
      int ef = 4 * e + f, kind = m->fkind[ef];
      if (kind == FK_IFACE_L || kind == FK_IFACE_R) continue;
      for (int j = 0; j < N; ++j) {
        real nx, ny, S, x, y, ug, vg, qi[4], qo[4], Fn[4];
        face_geom(m, e, f, j, t, &nx, &ny, &S, &x, &y);
        grid_velocity(m, e, x, y, &ug, &vg);
        real vgn = ug * nx + vg * ny;
        for (int v = 0; v < 4; ++v) {
          size_t id = face_index(N, e, f, v, j);
          qi[v] = (f == 1 || f == 3) ? Qxi[id] : Qeta[id];
        }
        if (kind == FK_CONF || kind == FK_PERIODIC) {
          int eb = m->fnbr[ef] / 4, fb = m->fnbr[ef] % 4, jb = m->frev[ef] ? N - 1 - j : j;
          for (int v = 0; v < 4; ++v) {
            size_t id = face_index(N, eb, fb, v, jb);
            qo[v] = (fb == 1 || fb == 3) ? Qxi[id] : Qeta[id];
          }
        } else {
          real qb[4];
          boundary_states(P, m->ftag[ef], qi, ug, vg, nx, ny, qo, qb);
        }
        rusanov(P, qi, qo, nx, ny, vgn, Fn);
        for (int v = 0; v < 4; ++v) {
          real fv = Fv_face ? Fv_face[((size_t)ef * 4 + v) * N + j] : 0.0;
          size_t id = face_index(N, e, f, v, j);
          real val = FACE_SIGMA[f] * S * (Fn[v] + fv);
          if (f == 1 || f == 3) Fxi[id] = val; else Geta[id] = val;
        }
      }
    }
  /* sliding interface: Eqs. prjQ2 -> Rusanov -> prjF2 */
  for (int z = 0; z < m->nz; ++z) {
    const or_iface *I = &m->zi[z];
    const int nL = I->nL, nR = I->nR;
    real *Lin = Lins[z], *Rin = Rins[z], *Lout = Louts[z], *Rout = Routs[z];
    const or_mortars *mo = &mos[z];
    if (nL == 0) continue;
    for (int k = 0; k < nL; ++k) gather_ccw(m, Qxi, Qeta, I->Lef[k], I->Lrev[k], 4, Lin + (size_t)k * 4 * N);
    for (int k = 0; k < nR; ++k) gather_ccw(m, Qxi, Qeta, I->Ref[k], I->Rrev[k], 4, Rin + (size_t)k * 4 * N);
    mortar_couple(m, I, mo, 0, Lin, Rin, Lout, Rout);
    for (int side = 0; side < 2; ++side) {
      int n = side ? nR : nL;
      for (int k = 0; k < n; ++k) {
        int ef = side ? I->Ref[k] : I->Lef[k], rev = side ? I->Rrev[k] : I->Lrev[k];
        int e = ef / 4, f = ef % 4;
        const real *src = (side ? Rout : Lout) + (size_t)k * 4 * N;
        real sgn = side ? -1.0 : 1.0; /* L -> R normal is outward for L, inward for R */
        for (int j = 0; j < N; ++j) {
          int jj = rev ? N - 1 - j : j;
          real nx, ny, S, x, y;
          face_geom(m, e, f, jj, t, &nx, &ny, &S, &x, &y);
          for (int v = 0; v < 4; ++v) {
            real fv = Fv_face ? Fv_face[((size_t)ef * 4 + v) * N + jj] : 0.0;
            size_t id = face_index(N, e, f, v, jj);
            real val = FACE_SIGMA[f] * S * (sgn * src[v * N + j] + fv);
            if (f == 1 || f == 3) Fxi[id] = val; else Geta[id] = val;
          }
        }
      }
    }
  }

  /* step 4: divergence of the flux polynomials (Eqs. Ft, Gt) at the SPs;
   * dQ/dt = -(dF~/dxi + dG~/deta) / |J| */
  for (int e = 0; e < ne; ++e)
    for (int j = 0; j < N; ++j)
      for (int k = 0; k < N; ++k) {
        real g[6];
        map_t0(m, e, m->Xs[k], m->Xs[j], g);
        real J = g[2] * g[5] - g[4] * g[3];
        for (int v = 0; v < 4; ++v) {
          real dF = 0.0, dG = 0.0;
          for (int i = 0; i <= N; ++i) {
            dF += Fxi[IXF(e, v, j, i)] * dl[k * (N + 1) + i];
            dG += Geta[IEF(e, v, i, k)] * dl[j * (N + 1) + i];
          }
          dQdt[IQ(e, v, j, k)] = -(dF + dG) / J;
          if (scale) {
            real a = 0.0;
            for (int i = 0; i <= N; ++i)
              a += fabs(Fxi[IXF(e, v, j, i)] * dl[k * (N + 1) + i]) + fabs(Geta[IEF(e, v, i, k)] * dl[j * (N + 1) + i]);
            scale[IQ(e, v, j, k)] = a / fabs(J);
          }
        }
      }

  free(Qxi); free(Qeta); free(Fxi); free(Geta);
  free(cQxi); free(cQeta); free(Gxx); free(Gxy); free(Gex); free(Gey); free(Fv_face);
  for (int z = 0; z < m->nz; ++z)
    if (m->zi[z].nL > 0) { free(Lins[z]); free(Rins[z]); free(Louts[z]); free(Routs[z]); free_mortars(&mos[z]); }
  return 0;
}

/* Three-stage SSP Runge-Kutta (Shu-Osher form), stage times t, t+dt, t+dt/2 */
int or_step(or_mesh *m, real *Q, real *t, real dt, int nsteps) {
  size_t n = (size_t)m->ne * 4 * m->N * m->N;
  real *q1 = malloc(n * sizeof(real)), *q2 = malloc(n * sizeof(real)), *r = malloc(n * sizeof(real));
  for (int s = 0; s < nsteps; ++s) {
    real tn = *t;
    or_residual(m, Q, tn, r);
    for (size_t i = 0; i < n; ++i) q1[i] = Q[i] + dt * r[i];
    or_residual(m, q1, tn + dt, r);
    for (size_t i = 0; i < n; ++i) q2[i] = 0.75 * Q[i] + 0.25 * (q1[i] + dt * r[i]);
    or_residual(m, q2, tn + 0.5 * dt, r);
    for (size_t i = 0; i < n; ++i) Q[i] = Q[i] / 3.0 + 2.0 / 3.0 * (q2[i] + dt * r[i]);
    *t = tn + dt;
  }
  free(q1); free(q2); free(r);
  return 0;
}

/* Five-stage, fourth-order SSP Runge-Kutta (the integrator of Sec. 4; the
 * paper cites Spiteri & Ruuth for it without printing coefficients).  Shu-Osher
 * form with the published coefficients:
 *   u1 = u + c10 dt L(u)
 *   u2 = a20 u + a21 u1 + c21 dt L(u1)
 *   u3 = a30 u + a32 u2 + c32 dt L(u2)
 *   u4 = a40 u + a43 u3 + c43 dt L(u3)
 *   u+ = a52 u2 + a53 u3 + c53 dt L(u3) + a54 u4 + c54 dt L(u4)
 * Stage times follow from the coefficients (or_rk54_tableau). */
static const real RK54_C10 = 0.391752226571890;
static const real RK54_A20 = 0.444370493651235, RK54_A21 = 0.555629506348765, RK54_C21 = 0.368410593050371;
static const real RK54_A30 = 0.620101851488403, RK54_A32 = 0.379898148511597, RK54_C32 = 0.251891774271694;
static const real RK54_A40 = 0.178079954393132, RK54_A43 = 0.821920045606868, RK54_C43 = 0.544974750228521;
static const real RK54_A52 = 0.517231671970585, RK54_A53 = 0.096059710526147, RK54_C53 = 0.063692468666290;
static const real RK54_A54 = 0.386708617503269, RK54_C54 = 0.226007483236906;

/* Butcher tableau (A 5x5 row-major, b 5, c 5) of the scheme above, for tests:
 * every stage value is expanded as u + dt sum_j A_ij k_j with k_j = L(stage j). */
void or_rk54_tableau(real *A, real *b, real *c) {
  /* coefficient of dt k_j in stage i (stage 1 = u) */
  real S[6][5];
  memset(S, 0, sizeof S);
  /* S[1] = u1 */
  S[1][0] = RK54_C10;
  for (int j = 0; j < 5; ++j) S[2][j] = RK54_A21 * S[1][j];
  S[2][1] += RK54_C21;
  for (int j = 0; j < 5; ++j) S[3][j] = RK54_A32 * S[2][j];
  S[3][2] += RK54_C32;
  for (int j = 0; j < 5; ++j) S[4][j] = RK54_A43 * S[3][j];
  S[4][3] += RK54_C43;
  for (int j = 0; j < 5; ++j) S[5][j] = RK54_A52 * S[2][j] + RK54_A53 * S[3][j] + RK54_A54 * S[4][j];
  S[5][3] += RK54_C53;
  S[5][4] += RK54_C54;
  memset(A, 0, sizeof(real) * 25);
  for (int i = 0; i < 5; ++i) {
    real ci = 0.0;
    for (int j = 0; j < 5; ++j) {
      A[i * 5 + j] = i == 0 ? 0.0 : S[i][j];
      ci += A[i * 5 + j];
    }
    c[i] = ci;
  }
  for (int j = 0; j < 5; ++j) b[j] = S[5][j];
}

int or_step_rk54(or_mesh *m, real *Q, real *t, real dt, int nsteps) {
  size_t n = (size_t)m->ne * 4 * m->N * m->N;
  real *u1 = malloc(n * sizeof(real)), *u2 = malloc(n * sizeof(real)), *u3 = malloc(n * sizeof(real));
  real *u4 = malloc(n * sizeof(real)), *r = malloc(n * sizeof(real)), *r3 = malloc(n * sizeof(real));
  real A[25], b[5], c[5];
  or_rk54_tableau(A, b, c);
  for (int s = 0; s < nsteps; ++s) {
    real tn = *t;
    or_residual(m, Q, tn + c[0] * dt, r);
    for (size_t i = 0; i < n; ++i) u1[i] = Q[i] + RK54_C10 * dt * r[i];
    or_residual(m, u1, tn + c[1] * dt, r);
    for (size_t i = 0; i < n; ++i) u2[i] = RK54_A20 * Q[i] + RK54_A21 * u1[i] + RK54_C21 * dt * r[i];
    or_residual(m, u2, tn + c[2] * dt, r);
    for (size_t i = 0; i < n; ++i) u3[i] = RK54_A30 * Q[i] + RK54_A32 * u2[i] + RK54_C32 * dt * r[i];
    or_residual(m, u3, tn + c[3] * dt, r3);
    for (size_t i = 0; i < n; ++i) u4[i] = RK54_A40 * Q[i] + RK54_A43 * u3[i] + RK54_C43 * dt * r3[i];
    or_residual(m, u4, tn + c[4] * dt, r);
    for (size_t i = 0; i < n; ++i)
      Q[i] = RK54_A52 * u2[i] + RK54_A53 * u3[i] + RK54_C53 * dt * r3[i] + RK54_A54 * u4[i] + RK54_C54 * dt * r[i];
    *t = tn + dt;
  }
  free(u1); free(u2); free(u3); free(u4); free(r); free(r3);
  return 0;
}

/* mortar list of zone z's interface at time t, for tests: returns the number
 * of mortars (-1 for no such zone); arrays must hold nL + nR entries */
int or_mortar_list_zone(const or_mesh *m, int z, real t, int *lf, int *rf, real *oL, real *sL, real *oR,
                        real *sR) {
  if (z < 1 || z > m->nz) return -1;
  or_mortars mo;
  build_mortars(&m->zi[z - 1], t, &mo);
  for (int k = 0; k < mo.nm; ++k) {
    lf[k] = mo.lf[k]; rf[k] = mo.rf[k]; oL[k] = mo.oL[k]; sL[k] = mo.sL[k]; oR[k] = mo.oR[k]; sR[k] = mo.sR[k];
  }
  int n = mo.nm;
  free_mortars(&mo);
  return n;
}

/* the same for zone 1 */
int or_mortar_list(const or_mesh *m, real t, int *lf, int *rf, real *oL, real *sL, real *oR, real *sR) {
  return or_mortar_list_zone(m, 1, t, lf, rf, oL, sL, oR, sR);
}
