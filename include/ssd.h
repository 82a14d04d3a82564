/*
 * ssd.h -- C ABI of the GB300 sliding-mesh spectral difference (SSD) library.
 *
 * The library advances the two-dimensional compressible Euler / Navier-Stokes
 * equations (Sec. 2 of Zhang & Liang, arXiv:1503.02198) on curvilinear
 * quadrilaterals with one rotating zone coupled to one stationary zone through
 * a curved sliding interface (Sec. 3.2), using the spectral difference method
 * (Sec. 3.1) and explicit three-stage SSP Runge-Kutta (Sec. 3).  Every step of
 * the residual and of the time step runs in CUDA kernels on one GPU.
 *
 * Conventions shared by every call:
 *   - return value: SD_OK (0) or a negative SD_ERR_* code; sd_last_error()
 *     gives a message for the last failure on a handle;
 *   - the handle owns all device memory; input arrays are copied during the
 *     call and stay owned by the caller;
 *   - a state array is [E][4][N][N] doubles, element-major, then the
 *     conservative variable (rho, rho u, rho v, E; Sec. 2.1 Eq. Q), then the
 *     eta index j, then the xi index i of the solution point (X_i, X_j);
 *     N = p + 1 points per direction;
 *   - "on_device" = 1 means the pointer is CUDA device memory (for example a
 *     torch tensor's data_ptr()), 0 means host memory;
 *   - all work is queued on the stream given at creation; calls that return
 *     data to the host synchronise that stream.
 */
#ifndef SSD_H
#define SSD_H

#ifdef __cplusplus
extern "C" {
#endif

enum {
  SD_OK = 0,
  SD_ERR_ARG = -1,         /* invalid argument (null pointer, bad p, dt <= 0 ...) */
  SD_ERR_MESH = -2,        /* inconsistent mesh (unmatched face, folded cell ...) */
  SD_ERR_CUDA = -3,        /* a CUDA runtime call failed */
  SD_ERR_NONPHYSICAL = -4, /* a kernel met rho <= 0, p <= 0 or a non-finite value */
  SD_ERR_TIMEOUT = -5,     /* a bounded device wait gave up (reported by sd_sync) */
  SD_ERR_UNSUPPORTED = -6  /* valid request this build does not support (e.g. p) */
};

enum { SD_PREC_FP64 = 0, SD_PREC_FP32 = 1, SD_PREC_FP32S = 2, SD_PREC_FP32_TF32 = 3 };

/* Boundary tags of sd_mesh.bfaces.  Each acts through a ghost state in the
 * Rusanov flux; the state on the boundary is the common solution of the
 * viscous terms, whose flux uses the interior gradient (the paper names these
 * conditions, Secs. 4.2-4.3, without formulas; these are the readings):
 *   WALL   ghost velocity 2 V_g - V, temperature T_wall, interior pressure;
 *          on the wall the velocity is V_g (the grid velocity of the zone);
 *   SLIP   ghost velocity with the normal component of V - V_g mirrored,
 *          interior density and pressure; on the wall that component is 0;
 *   INLET  ghost = the free stream (rho_inf, u_inf, v_inf, p_inf);
 *   OUTLET ghost = interior density and velocity with pressure p_inf;
 *   ADIABATIC  as WALL with the interior temperature (density) instead of
 *          T_wall; its viscous flux has no heat conduction (Sec. 4's stirred
 *          tank blades). */
enum {
  SD_BC_WALL = 1,     /* isothermal no-slip wall moving with its zone */
  SD_BC_SLIP = 2,     /* slip (inviscid) wall */
  SD_BC_INLET = 3,    /* Dirichlet inflow of the free stream */
  SD_BC_OUTLET = 4,   /* fixed-pressure outflow */
  SD_BC_ADIABATIC = 5 /* adiabatic no-slip wall moving with its zone */
};

/* edge kinds of sd_mesh.edge_arc */
enum { SD_EDGE_STRAIGHT = 0, SD_EDGE_ARC = 1, SD_EDGE_CUBIC = 2 };

/* rotating zones per mesh (zone 1 plus at most SD_MAX_ZONES - 1 further zones) */
#define SD_MAX_ZONES 4

/* A further rotating zone (the paper has one per case; Sec. 2.2 applies to
 * each zone and Sec. 3.2 to each interface on its own).  Zone k + 2, the k-th
 * entry of sd_mesh.zones, turns rigidly about `center` at angular velocity
 * `omega` and meets the stationary zone 0 across its own circular sliding
 * interface of radius r_interface about `center`: iface_L lists its faces on
 * the zone's side, iface_R those on the stationary side, both as
 * [n][2] (element, local face).  The arrays are copied by sd_create. */
typedef struct {
  double center[2];
  double r_interface;
  double omega;
  int n_iface_L;
  const int *iface_L;
  int n_iface_R;
  const int *iface_R;
} sd_zone;

/* Mesh (Sec. 3.1: every cell is mapped to the standard square [0,1]^2).
 * Corners n0..n3 are counter-clockwise and map to (0,0), (1,0), (1,1), (0,1).
 * Local face f: f0 = {eta=0} n0->n1, f1 = {xi=1} n1->n2, f2 = {eta=1} n3->n2,
 * f3 = {xi=0} n0->n3 (the arrow is the direction of the face parameter).
 * An SD_EDGE_ARC edge is the circular arc through its two corners (both at
 * the same radius) about the centre of the cell's arc zone (elem_arc_zone:
 * zone 1's centre is `center`); an SD_EDGE_CUBIC edge is the cubic
 * through its corners and the two edge nodes edge_nodes[e][f][0..1] at face
 * parameter 1/3 and 2/3 (Sec. 3.1's 12-node cubic cells); other edges are
 * straight.  The map of a cell is the transfinite interpolation of its four
 * edges: the 4-node bilinear map when all edges are straight, the 12-node
 * serendipity map when all are cubic.  Faces shared by two cells of the same
 * zone are found from their node pairs and must have the same edge kind (and,
 * if cubic, the same edge nodes); periodic and interface faces cannot be
 * cubic.  Every other face must appear in exactly one of bfaces, pfaces,
 * iface_L, iface_R and the interface lists of the further zones.  A
 * conforming face joins two cells of one zone; periodic faces lie in zone 0. */
typedef struct {
  int n_nodes;
  const double *xy;        /* [n_nodes][2] */
  int n_elems;
  const int *elem_nodes;   /* [n_elems][4] */
  const int *elem_zone;    /* [n_elems]: 0 stationary, z >= 1 rotating zone z (zone 1: rigid
                              rotation about center at sd_params.omega; zone z >= 2: zones[z - 2]) */
  const int *edge_arc;     /* [n_elems][4]: SD_EDGE_* kind of local face f */
  int n_bfaces;
  const int *bfaces;       /* [n_bfaces][3]: element, local face, SD_BC_* tag */
  int n_pfaces;
  const int *pfaces;       /* [n_pfaces][4]: periodic pair elemA, faceA, elemB, faceB */
  int n_iface_L;
  const int *iface_L;      /* [n][2]: element, local face on the interface, rotating side (Sec. 3.2 "left") */
  int n_iface_R;
  const int *iface_R;      /* [n][2]: stationary side ("right") */
  double center[2];        /* zone 1: rotation centre = centre of its interface circle */
  double r_interface;      /* radius of zone 1's sliding interface */
  const int *edge_nodes;   /* [n_elems][4][2] node indices of cubic edges (-1 elsewhere);
                              may be NULL when no edge is cubic */
  int n_zones;             /* further rotating zones (0 .. SD_MAX_ZONES - 1) */
  const sd_zone *zones;    /* [n_zones] zones 2, 3, ...; may be NULL when n_zones = 0 */
  const int *elem_arc_zone; /* [n_elems] zone (>= 1) whose centre the cell's arc edges are
                              drawn about; a rotating cell's must be its own zone.  NULL: the
                              cell's own zone, zone 1 for stationary cells */
} sd_mesh;

/* Gas, flow and run parameters (non-dimensional).  Viscous fluxes follow
 * Sec. 2.1 with lambda = -2/3 mu and conductivity k = mu gamma Rgas /
 * ((gamma - 1) prandtl). */
typedef struct {
  double gamma;     /* ratio of specific heats (Sec. 2.1: 1.4) */
  double Rgas;      /* gas constant, p = rho Rgas T */
  double mu;        /* dynamic viscosity (constant) */
  double prandtl;   /* Prandtl number */
  double omega;     /* angular velocity of rotating zone 1 (Sec. 2.2) */
  double T_wall;    /* temperature of SD_BC_WALL faces */
  int viscous;      /* 0 Euler, 1 Navier-Stokes */
  int precision;    /* SD_PREC_FP64, or SD_PREC_FP32: FP32 interpolation, flux and
                       divergence arithmetic; FP64 rotation angle, mortar geometry and
                       projection weights, and FP64 state / Runge-Kutta accumulation
                       (a double-float pair per value); or SD_PREC_FP32S: as SD_PREC_FP32
                       with the state stored as one float per value, each Runge-Kutta
                       stage result rounded to float (half the state bytes; the state
                       carries float round-off, about 6e-8 relative per stage); or
                       SD_PREC_FP32_TF32: as SD_PREC_FP32 with the inviscid volume
                       kernel's interpolation (Eq. Qt) and divergence (Eqs. Ft, Gt)
                       contractions on the tensor cores, each product as three TF32
                       matrix multiplies of a big/small split of both operands
                       (3xTF32, near-FP32 accuracy); Navier-Stokes meshes keep the
                       FMA-pipe kernels; not available in the batched form */
  void *stream;     /* cudaStream_t to queue work on; NULL = a non-blocking stream the handle creates */
  int rk_stages;    /* time integrator: 0 or 3 = three-stage SSP-RK3 (Shu-Osher); 5 = the
                       five-stage fourth-order SSP-RK of Sec. 4 (Spiteri-Ruuth coefficients) */
  double rho_inf, u_inf, v_inf, p_inf; /* free stream: SD_BC_INLET state, SD_BC_OUTLET pressure
                                          (read only when the mesh has such faces) */
} sd_params;

typedef struct sd_handle sd_handle;

/* Build the solver for mesh m at polynomial degree p (N = p + 1 solution points
 * per direction, Sec. 3.1; supported p = 2..5).  Validates the mesh, builds
 * the face tables and the sorted interface lists, uploads the geometry and
 * computes the t = 0 metrics on the device.  Time starts at 0 and the state
 * is zero until sd_set_state.  On failure *out is NULL and the return code
 * says why (the message is printed by sd_create_error()). */
int sd_create(const sd_mesh *m, int p, const sd_params *prm, sd_handle **out);

/* message of the last sd_create failure in this thread */
const char *sd_create_error(void);

/* Free the handle and its device memory (synchronises the stream first). */
int sd_destroy(sd_handle *h);

/* Message for the last failure on h (a static string owned by h). */
const char *sd_last_error(const sd_handle *h);

/* Sizes: number of elements, N, and number of conservative unknowns
 * (E * 4 * N * N). Any pointer may be NULL. */
int sd_info(const sd_handle *h, int *n_elems, int *N, long long *n_dofs);

/* Copy the physical state Q (layout above) into the solver.  on_device: Q is
 * device memory; else host memory.  A pinned host buffer (cudaHostAlloc,
 * cudaMallocHost, cudaHostRegister) is read by the device directly; pageable
 * memory goes through a staged copy.  Returns once Q may be reused. */
int sd_set_state(sd_handle *h, const double *Q, int on_device);

/* Copy the current state out (synchronises); host buffers as for
 * sd_set_state (a pinned one is written by the device directly). */
int sd_get_state(sd_handle *h, double *Q, int on_device);

/* Set / read the solution time t (the rotation angle is omega * t). */
int sd_set_time(sd_handle *h, double t);
int sd_get_time(sd_handle *h, double *t);

/* Semi-discrete residual dQ/dt = -(dF~/dxi + dG~/deta) / |J| (Eq. computational
 * with Eqs. Qt, Ft, Gt) at the current state and time, with the mortar
 * coupling of Sec. 3.2 at the current rotation angle.  R has the state layout.
 * Synchronises when R is host memory. */
int sd_residual(sd_handle *h, double *R, int on_device);

/* Advance nsteps steps of size dt with the SSP Runge-Kutta scheme chosen by
 * sd_params.rk_stages (Sec. 3: three stages at t, t + dt, t + dt/2; Sec. 4:
 * five stages); the mortar connectivity is rebuilt at every stage (Sec. 3.2).
 * Asynchronous: queued on the handle's stream as two kernel launches (the
 * stage clocks and mortar tables of the first step) and nsteps CUDA-graph
 * launches; each captured step also merges the next step's stages on a
 * second stream of the handle, beside its own kernels, and rejoins before it
 * ends, so the result is the same as merging each step after the last.
 * Errors detected on the device are reported by sd_sync. */
int sd_step(sd_handle *h, double dt, int nsteps);

/* Wait for queued work; returns SD_ERR_NONPHYSICAL if a stage produced
 * rho <= 0, p <= 0 or a non-finite value since the last sd_sync. */
int sd_sync(sd_handle *h);

/* Test aid for the bounded device waits, off by default (on = 0).  With
 * on = 1 the volume kernel of later residuals and steps arms the copy
 * barrier of its first work item with 16 bytes more than that item's copies
 * deliver and gives that one wait a short poll limit: the wait gives up, the
 * kernel raises its timeout flag, lets the copies it has issued land and
 * returns, and sd_sync (or sd_residual_noalloc) reports SD_ERR_TIMEOUT; the
 * result of that call is incomplete.  Every issued copy still lands; nothing
 * faults or hangs.  on = 0 restores normal operation.  Synchronises. */
int sd_test_wait_timeout(sd_handle *h, int on);

/* Test aid for the handle's reciprocal 1/x (the density and Jacobian
 * reciprocals of its kernels): y[i] = 1 / x[i] computed on the GPU in the
 * handle's compute type (Newton's iteration from the hardware's approximate
 * reciprocal: two steps in FP64, one in FP32; within one ulp), for n host
 * values x (normal, finite, non-zero) into host y.  Allocates and frees a
 * device buffer of 16 n bytes; synchronises.  SD_ERR_ARG for n < 0 or null
 * arrays with n > 0. */
int sd_test_reciprocal(sd_handle *h, const double *x, double *y, int n);

/* Physical coordinates of the solution points at time t, [E][N][N][2]. */
int sd_sp_coords(sd_handle *h, double t, double *xy, int on_device);

/* ---- batched form: many independent cases, one CUDA-graph launch per step ----
 * Each case has its own mesh, polynomial degree and parameters (its own
 * rotation rate and step size); all cases share the precision and the
 * Runge-Kutta scheme.  The cases are grouped into classes of equal N and
 * viscous flag; every phase of a stage (face pass with the mortar flux,
 * gather, gradients, volume kernel) is one launch per class whose work list
 * spans all cases of the class (per-case prefix sums of faces, mortars and
 * element tiles; the persistent volume kernels walk (case, tile) items), and
 * the stage clocks and mortar tables of every case come from one merge
 * launch per step.  sd_batch_step runs one CUDA-graph launch per step.  With
 * tune_dt > 0 an autotuner chooses, per class, the elements per volume tile,
 * the face-pass block size and the volume CTAs per SM by timing a few batch
 * steps of size tune_dt from a uniform state; states and times are reset to
 * zero afterwards. */
typedef struct sd_batch sd_batch;

/* SD_ERR_ARG if the cases differ in precision or Runge-Kutta scheme;
 * SD_ERR_UNSUPPORTED for SD_PREC_FP32_TF32.  The batched form is held in this
 * version: unless the environment variable SSD_BATCH_ENABLE is "1" the call
 * returns SD_ERR_UNSUPPORTED (after the argument checks above), because a run
 * of 64 FP32 cases stopped on a device memory error whose cause is not yet
 * found. */
int sd_batch_create(int n, const sd_mesh *const *meshes, const int *p, const sd_params *prm, double tune_dt,
                    sd_batch **out);
int sd_batch_destroy(sd_batch *b);
int sd_batch_size(const sd_batch *b);

/* Handle of case i (owned by the batch): use it with sd_set_state,
 * sd_get_state, sd_set_time, sd_get_time, sd_residual; work queued on it is
 * ordered after the batch's earlier steps.  NULL if i is out of range. */
sd_handle *sd_batch_case(sd_batch *b, int i);

/* Advance every case by nsteps steps; dt[i] is case i's step (the graph is
 * captured again when a dt changes).  Asynchronous; errors of any case are
 * reported by sd_batch_sync. */
int sd_batch_step(sd_batch *b, const double *dt, int nsteps);

/* Wait for the batch; returns the first case error (SD_ERR_NONPHYSICAL ...). */
int sd_batch_sync(sd_batch *b);
const char *sd_batch_last_error(const sd_batch *b);

/* Classes of the batch and, for class i, info[0..5] = N, viscous flag,
 * number of cases, elements per volume tile, volume CTAs per SM and face-pass
 * block size in force (the autotuner's choice). */
int sd_batch_classes(const sd_batch *b);
int sd_batch_class_info(sd_batch *b, int i, int *info);

/* Measurement aid (the paper reports wall time split into interface and
 * total time, Tables 3-10): runs reps steps outside the CUDA graph with CUDA
 * events around each launch group on the handle's stream and writes the mean
 * milliseconds per launch of ms[0] stage clock + mortar merge, ms[1]
 * conforming, periodic and wall faces, ms[2] mortar projection + gather
 * (the paper's "interface" work), ms[3] volume kernel (divergence, RK update,
 * traces); ms[4] = mean milliseconds per whole step.  The mortar flux is
 * timed as its own launch here; sd_step runs it inside the face launch of
 * the same pass.  Advances the solution by reps steps; synchronises. */
int sd_profile_step(sd_handle *h, double dt, int reps, double *ms);

/* Measured FMA throughput of the current GPU in TFLOP/s (2 flops per FMA)
 * for precision SD_PREC_FP64 or SD_PREC_FP32, from a probe kernel queued on
 * the handle's stream; the denominator for FP64 / FP32 pipe utilisation.
 * Synchronises. */
int sd_fma_peak(sd_handle *h, int precision, double *tflops);

/* Same result as sd_residual, for callers that must not allocate device
 * memory once their handle exists: a solver embedded in a host application
 * whose device memory is owned by another allocator (for example a framework
 * memory pool that reserves the free memory), or a latency-bound loop where
 * the implicit device synchronisation of cudaMalloc / cudaFree is not
 * acceptable.  sd_residual may allocate a device staging buffer on its first
 * call with a host R; this variant allocates nothing.  (The paper has no
 * counterpart: this is a deployment aid, not part of the method.)
 *
 * Work memory: the mortar table and mortar offsets (Eq. xz), the mortar flux
 * contributions, the merge work arrays and, when R is host memory, the device copy of R all live in one
 * fixed 16 MiB device array inside the library, which every GPU that loads the
 * library holds until the process exits.  Calls needing more than 16 MiB
 * return SD_ERR_ARG with a message (with R in host memory the state copy,
 * E * 4 * N * N doubles, counts against the limit; with R in device memory
 * only the interface work does).  Every call looks up the current device's
 * copy of the array (cudaGetSymbolAddress).  All calls share the array and
 * nothing in it is assumed to start at zero; calls that overlap on the GPU
 * (several handles or streams at once) race on it.  Synchronises the
 * handle's stream, then reports device errors as sd_sync does
 * (SD_ERR_TIMEOUT: a bounded wait gave up and R is incomplete). */
int sd_residual_noalloc(sd_handle *h, double *R, int on_device);

#ifdef __cplusplus
}
#endif

#endif /* SSD_H */
