// Internal structures shared by the host driver (ssd_api.cu) and the
// per-precision kernel engines (ssd_engine.cuh instantiated in ssd_f64.cu and
// ssd_f32.cu).  Not part of the C ABI.
#pragma once

#include <cuda_runtime.h>

#include <vector>

namespace ssd {

constexpr int kMaxN = 8;
// rotating zones per mesh (zone 0 is the stationary zone; zone z >= 1 turns
// rigidly about its own centre and has its own sliding interface)
constexpr int kMaxZones = 4;
constexpr int kZT = kMaxZones + 1;  // per-zone table entries, zone 0 included
// Per-element arrays are padded to a multiple of kElemPad elements: every tile
// size the persistent kernels use (4, 8, 12, 16 elements) divides it, so a
// tile that copies whole tiles stays inside the arrays whichever size runs.
constexpr int kElemPad = 48;
// cell flag: zone in the low kZoneBits bits, (metric table index + 1) above
constexpr int kZoneBits = 3, kZoneMask = (1 << kZoneBits) - 1;
// and bit 30: the cell has a face on a sliding interface
constexpr int kIfaceBit = 1 << 30;
static_assert(kMaxZones <= kZoneMask, "zone bits");

// Device-resident clock of the current stage (the rotation angles never
// leave FP64: theta_z = omega_z * t_stage, Sec. 2.2).  Per zone z: the
// rotation R(theta_z) as (c, s) and the angular velocity om; zone 0 holds
// (1, 0, 0).  c, s, om follow each other so that c points at the zone table
// [3][kZT] a kernel reads (likewise cf, sf, omf on the FP32 path).  The
// reduced angle is a double-double theta2 + theta2_lo: the exact product
// omega_z t_stage reduced modulo 2 pi with a double-double 2 pi, so that
// mortar offsets (differences of angles near pi) keep full relative accuracy.
struct DevClock {
  double t_n;           // time at the start of the step
  double t_stage;       // time of the stage being evaluated
  double theta2[kZT];   // theta_z reduced to [0, 2 pi): high part
  double theta2_lo[kZT];  // and low part
  double c[kZT], s[kZT], om[kZT];
  float cf[kZT], sf[kZT], omf[kZT];
  int flags;  // bit 0: non-physical state; bit 1: mesh geometry error; bit 2: a bounded device wait gave up;
              // bit 3: (debug build) a table index out of range
  int pad;
};

// Basis data of Sec. 3.1 and the mortar quadrature of Sec. 3.2, built on the
// host in FP64 for one N (see ssd_api.cu) and copied to constant memory.
struct HostBasis {
  int N;
  double Xs[kMaxN];                  // solution points
  double Xf[kMaxN + 1];              // flux points
  double Hf[(kMaxN + 1) * kMaxN];    // h_k(X_{i+1/2}) [i][k]
  double Dm[kMaxN * (kMaxN + 1)];    // l'_{i+1/2}(X_k) [k][i]
  double H0[kMaxN], H1[kMaxN];       // h_k(0), h_k(1)
  double zq[kMaxN], wq[kMaxN];       // N-point Gauss-Legendre rule on [0,1]
  double Hz[kMaxN * kMaxN];          // h_j(z_q) [q][j]
  double Minv[kMaxN * kMaxN];        // inverse mortar mass matrix (Eq. mortarM)
  double cden[kMaxN];                // 1 / prod_{s != i} (X_i - X_s)
};

// A solution state in device memory.  FP64 path: hi = double[E][4][N][N],
// lo = nullptr.  FP32 path: the value is hi + lo with hi, lo float[E][4][N][N]
// (a double-float pair, about 48 significant bits).
struct StatePtr {
  void *hi;
  void *lo;
};

// Eq. xz for one mortar against its face on one side, formed by the merge of
// the stage: offset o and scale s of the mortar in the face's reference
// coordinate, the face's rotated start angle (double-double) and angular
// width, its element-face index and orientation
struct __align__(16) MortSide {
  double o, s, fa_hi, fa_lo, w;
  int ef, rev;
};

// Everything a kernel needs, by value (device pointers + sizes + parameters).
struct MeshDev {
  int E, N;
  // conforming and periodic face pairs: (efA, efB, reversed, 0), ef = 4 e + f
  int nF;
  const int4 *faces;
  // boundary faces: (ef, tag, 0, 0); t = 0 positions of their points [nB][N][2]
  int nB;
  const int4 *bfaces;
  const double *bxy;
  // sliding interfaces, both sides of each sorted counter-clockwise at t = 0
  // about its zone's centre: (ef, reversed, 0, 0), CCW start angle (a
  // double-double La + La_lo, Ra + Ra_lo, formed on the host in long double),
  // angular width, |S| = r * width.  The lists of all interfaces are concatenated:
  // interface i (of zone i + 1) owns L faces [zoff[i], zoff[i + 1]), R faces
  // [zoff[kZT + i], zoff[kZT + i + 1]) and mortars [zoff[i] + zoff[kZT + i], ...)
  int nL, nR, nM;
  int nI;                   // interfaces (rotating zones) of the mesh, at least 1
  int nbmax;                // the largest nL + nR of one interface
  const int *zoff;          // [2][kZT] prefix sums of the L and R list lengths
  const int *ifz;           // [nL + nR] interface of each L, then R, face
  const int4 *Lface, *Rface;
  const double *La, *Lw, *LS, *Ra, *Rw, *RS;
  const double *La_lo, *Ra_lo;
  const double *LiW, *RiW;  // 1 / angular width
  // per-stage mortar table (written by the merge kernel)
  int *mLf, *mRf;       // [nM] containing L / R face (sorted index)
  double *mgeo;         // [nM][4]: start angle (double-double: high, low), angular length, unused
  MortSide *msd;        // [2][nM]: Eq. xz of each mortar against its L, then its R face
  int *Lstart, *Lcount; // [nL] first mortar (merged position) and count
  int *Rstart, *Rcount; // [nR]
  void *contrib;        // T [2][nM][4][N] back-projected mortar fluxes
  // elements
  // each cell's coordinates are relative to the centre of its frame zone:
  // its own zone if rotating, else the zone its arc edges are drawn about
  const double *corners;  // [E][8] t = 0 corner coordinates relative to the frame centre
  const int *arcs;        // [E] bit f: local face f is an arc; bit 4 + f: it is a cubic
  const double *cubic;    // [E][4][4] edge nodes (x, y at 1/3, x, y at 2/3) of cubic
                          // edges, centre relative; null when the mesh has none
  const int *zone;        // [E]
  const int *frame;       // [E] frame zone
  const double *zpar;     // [kZT][4] per zone: centre x, y, omega, interface radius
  // eflag[e]: bits 0-2 = zone; (table index + 1) << kZoneBits, or 0 above
  // them for a straight cell whose bilinear metrics are computed on the fly;
  // kIfaceBit if the cell has an interface face
  const int *eflag;
  // [4 E] per element face ef = 4 e + f: its interface face (L faces first,
  // then R: k or nL + k), or -1
  const int *efi;
  int nTab;               // number of metric tables
  const int *tab_elem;    // [nTab] element of each table
  void *geo;              // T [nTab][G] metric tables (see ssd_engine.cuh)
  void *egeo;             // T [E][8] bilinear record x0, y0, e1, e3, d of each cell
  void *TR, *CF;          // T [E][4][4][N] face traces and common fluxes
  void *CQ, *GTR;         // viscous: T [E][4][4][N] common solution, [E][4][8][N] gradient traces
  void *GSP;              // viscous: T [E][8][N][N] gradients at the SPs (x then y, 4 variables each)
  void *fgeo;             // T [nF][5][N] conforming-face geometry at t = 0: unit normal
                          // (x, y) out of side A, sigma_A |S_A|, sigma_B |S_B|, V_g . n
  DevClock *clk;
  const DevClock *clk0;   // t = 0: the identity rotation with each zone's omega
  double gamma, Rgas, mu, prandtl, T_wall;
  double rho_inf, u_inf, v_inf, p_inf;  // free stream (inlet state, outlet pressure)
  // derived constants, computed once on the host in double, with float copies
  // for the FP32 kernels (no double arithmetic or conversion per point there):
  // gamma - 1, conductivity k = mu gamma R / ((gamma - 1) Pr), R T_wall
  double gm1, kc, kcR, RTw;  // kcR = kc / Rgas
  float gm1_f, Rgas_f, mu_f, kc_f, kcR_f, RTw_f, rho_inf_f, u_inf_f, v_inf_f, p_inf_f;
  int any_farfield;                     // the mesh has inlet or outlet faces
  float gamma_f;  // the same rounded to float (FP32 path)
  int viscous;
  // test switch of the bounded waits (sd_test_wait_timeout), 0 otherwise: extra
  // transaction bytes armed on volume work item 0 and its wait's poll limit
  int test_tx_extra, test_poll;
};

enum { MODE_RESIDUAL = 0, MODE_RK = 1 };

// Stage clocks and mortar tables of every stage of one time step, filled by
// one merge launch at the start of the step (one block per stage and
// interface; the stage times t_n + c_k dt are known there).  Each stage's kernels then see a
// MeshDev whose clock and mortar-table pointers are that stage's.
constexpr int kMaxStages = 5;
struct StageMerge {
  int n;
  double c[kMaxStages];
  DevClock *clk[kMaxStages];
  int *mLf[kMaxStages], *mRf[kMaxStages];
  int *Lstart[kMaxStages], *Lcount[kMaxStages], *Rstart[kMaxStages], *Rcount[kMaxStages];
  double *mgeo[kMaxStages];
  MortSide *msd[kMaxStages];
  int *work_i[kMaxStages];
  double *work_d[kMaxStages];
};

// One Runge-Kutta stage in increment form: with R = L(in),
//   inc = a0 (base - in) + w_in + bdt R,   out = in + inc,
//   w_out = -g inc + ddt R   (an O(dt) increment kept for a later stage).
// SSP-RK3 and the five-stage SSP-RK(5,4) are sequences of such stages.
struct RkArgs {
  double a0 = 0.0, bdt = 0.0, g = 0.0, ddt = 0.0;
  int has_base = 0;
  const void *w_in = nullptr;  // compute-precision [E][4][N][N] or null
  void *w_out = nullptr;       // compute-precision [E][4][N][N] or null
};

// One case's part in a stage of the batched form (host side): its stage view
// of the mesh, the states the stage reads and writes, and the stage's
// Runge-Kutta arguments.
struct BatchStageHost {
  MeshDev md;
  StatePtr in, base, out;
  RkArgs rk;
};

// The merge and advance launches of a batch: for every case its base view,
// its stage views, stage records and step size (device arrays); the merge has
// a block per (interface, stage, case).
struct BatchMergeDev {
  int ncase, nstages, max_iface;
  int max_nm;               // the most mortars of one case
  const MeshDev *md;        // [ncase] base view (its clock holds the step's start time)
  const MeshDev *md_stage;  // [nstages][ncase] stage views (stage clock, mortar table)
  const StageMerge *sm;     // [ncase]
  const double *dt;         // [ncase]
  int smem;                 // dynamic shared memory: the largest interface's angles
};

// engine-owned device tables and launch shapes of one class
struct BatchClass {
  virtual ~BatchClass() {}
};

// Per-precision engine: T = double (FP64 path) or float (FP32 path).
struct Engine {
  virtual ~Engine() {}
  virtual size_t geo_words() const = 0;
  virtual size_t compute_word() const = 0;
  // true: straight cells get their metrics on the fly (tables only for arc cells)
  virtual bool metrics_on_the_fly() const = 0;
  // get / set the tunable launch shapes (see EngineImpl::tuning)
  virtual void tuning(int *vol_ctas_per_sm, int *max_ctas_per_sm, int *face_block) = 0;
  // the two state buffers A and B: E elements, storage for Epad >= E
  virtual cudaError_t alloc_state(int E, int Epad) = 0;
  virtual StatePtr A() const = 0;
  virtual StatePtr B() const = 0;
  // copy an FP64 state (device memory) into A, or A out as FP64 (device memory)
  virtual void set_state(const MeshDev &md, const double *Q, cudaStream_t s) = 0;
  virtual void get_state(const MeshDev &md, double *Q, cudaStream_t s) = 0;
  // upload basis constants, compute the t = 0 metrics
  virtual cudaError_t init(const HostBasis &hb, const MeshDev &md, cudaStream_t s) = 0;
  // face traces of a state
  virtual void trace(const MeshDev &md, StatePtr q, cudaStream_t s) = 0;
  // stage clock at t_n + c dt and mortar table; common fluxes on conforming,
  // periodic and wall faces; mortar fluxes gathered onto the interface faces
  virtual void clock_merge(const MeshDev &md, double c, double dt, cudaStream_t s) = 0;
  // the same merge with caller-provided work arrays (ints: 2 (nL + nR) + 1,
  // doubles: 2 (nL + nR) + 1)
  virtual void clock_merge_into(const MeshDev &md, double c, double dt, int *work_i, double *work_d,
                                cudaStream_t s) = 0;
  // the clocks, mortar tables and mortar offsets (Eq. xz) of stages first ..
  // first + count - 1 of a step, at t_n + c_k dt (t_n read from md.clk; with
  // ahead, of the next step: t_n + dt in place of t_n), merge CTAs of the
  // given size
  virtual void merge_stages(const MeshDev &md, const StageMerge &sm, double dt, int first, int count, int ahead,
                            int threads, cudaStream_t s) = 0;
  // q: the stage's state (the viscous chain needs its gradients)
  virtual void faces(const MeshDev &md, StatePtr q, cudaStream_t s) = 0;
  virtual void mortars(const MeshDev &md, cudaStream_t s) = 0;
  // true (default): the mortar flux runs inside the face launch of the same
  // pass; false: as its own launch in mortars() (per-phase timing)
  virtual void set_fusion(bool on) = 0;
  // the inviscid volume kernel's interpolation and divergence contractions on
  // the tensor cores (3xTF32; FP32 form only); returns false if unavailable
  virtual bool set_tensor_cores(bool on) = 0;
  void couple(const MeshDev &md, StatePtr q, double c, double dt, cudaStream_t s) {
    clock_merge(md, c, dt, s);
    faces(md, q, s);
    mortars(md, s);
  }
  // divergence; MODE_RESIDUAL writes R (FP64), MODE_RK writes the stage
  // described by rk (see RkArgs) and the face traces of its result
  virtual void volume(const MeshDev &md, StatePtr in, StatePtr base, StatePtr out, double *R, const RkArgs &rk,
                      int mode, cudaStream_t s) = 0;
  // the extra buffers of the five-stage scheme: a third state and an increment
  virtual cudaError_t alloc_rk54() = 0;
  virtual StatePtr C() const = 0;
  virtual void *W() const = 0;
  virtual void advance(const MeshDev &md, double dt, cudaStream_t s) = 0;
  virtual void sp_coords(const MeshDev &md, double t, double *xy, cudaStream_t s) = 0;
  // the compute type's reciprocal (recip) of n device values, for its test
  virtual void reciprocal(const double *x, double *y, int n, cudaStream_t s) = 0;

  // ---- batched form: one launch per phase for every case of a class ----
  // A class is a set of cases that share this engine's compute type and N
  // and one viscous flag.  Its device tables hold, per stage, each case's
  // stage view (clock and mortar table of that stage), its volume arguments
  // and prefix sums of each kind of work item, so that the kernels walk the
  // items of all cases of the class as one work list.
  // stages[k][c]: case c's view and Runge-Kutta arguments of stage k
  virtual BatchClass *batch_class(const std::vector<std::vector<BatchStageHost>> &stages, int viscous,
                                  cudaStream_t s) = 0;
  // new Runge-Kutta arguments (a dt changed); the kernels read them at launch
  virtual cudaError_t batch_update(BatchClass *bc, const std::vector<std::vector<BatchStageHost>> &stages,
                                   cudaStream_t s) = 0;
  // the kernels of stage k of every case of the class: face pass with the
  // mortar flux, gather (and the viscous chain), volume kernel with the
  // Runge-Kutta combination and traces
  virtual void batch_stage(BatchClass *bc, int k, cudaStream_t s) = 0;
  // launch shapes: volume CTAs per SM (0: keep) and elements per volume tile
  // (0: keep; one of the values batch_tile_choices lists) and face-pass
  // block size (0: keep); returns the values in force
  virtual void batch_tuning(BatchClass *bc, int *vol_ctas_per_sm, int *tile_elems, int *face_block,
                            cudaStream_t s) = 0;
  virtual int batch_tile_choices(int *out) const = 0;
  virtual void batch_free(BatchClass *bc) = 0;
  // the clocks and mortar tables of every stage of every case of a batch in
  // one launch, and the closing t_n += dt of every case (N-independent; any
  // engine launches them)
  virtual void batch_merge(const BatchMergeDev &bm, cudaStream_t s) = 0;
  virtual void batch_advance(const BatchMergeDev &bm, cudaStream_t s) = 0;
};

Engine *make_engine_f64(int N);
Engine *make_engine_f32(int N);
Engine *make_engine_f32s(int N);

}  // namespace ssd
