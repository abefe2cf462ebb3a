/*
 * lbm2p — GPU solver for the double-distribution lattice Boltzmann model of two-phase
 * Darcy flow of Chai, Liang, Du and Shi (arXiv 1808.07554).  C ABI.
 *
 * The model (Sec. 2, Eqs. 2-15 and 2-18) couples a Poisson equation for the global
 * pressure P and a convection-diffusion equation for the wetting saturation S:
 *     div(D_p grad P) + F_p = 0,   D_p = K lambda_t(S)
 *     phi dS/dt = div(D_s grad S) + F_s + div(lambda_w K grad P)
 * P is carried by a D2Q9 distribution f relaxed in pseudo time until steady (Eq. 3-1,
 * Eq. 3-3); grad P and the Darcy velocity u = -K lambda_t grad P are read locally from
 * f's first moment (Eq. 3-10); S is carried by a second D2Q9 distribution g (Eq. 3-2,
 * Eq. 3-4, Eq. 3-8).  One physical step (Sec. 3):
 *   1. stream g, S^n (Eq. 3-9b), tau_f(x) from D_p(S^n, K) (Eq. 3-11a, Remark IV);
 *   2. sweep f (stream + collide, Eq. 3-1) until the pressure increment satisfies the
 *      stopping rule below, or replay a given number of sweeps;
 *   3. stream f once more for grad P (Eq. 3-10a); stream g, collide it with both sources
 *      (Eq. 3-2) and keep the post-collision populations.
 *
 * Units and layout.  All host arrays are row-major [ny][nx] (node (i, j) at index
 * j*nx + i), cell centred: node (i, j) sits at ((i + 1/2) dx, (j + 1/2) dx) and walls
 * lie half-way between a boundary node and its missing neighbour.  Host inputs are FP64
 * and are copied (the caller keeps ownership); the library computes in FP32 on the GPU
 * and accumulates the residual in FP64.  Device outputs are FP32.
 *
 * Memory.  The handle owns all device memory.  It is obtained through params.alloc /
 * params.release when given (for instance a framework's caching allocator), otherwise
 * with cudaMalloc / cudaFree.  All work is enqueued on params.stream (a cudaStream_t;
 * NULL is the legacy default stream); calls that return host data synchronise that
 * stream.  A handle must be used by one host thread at a time.
 *
 * Errors.  Every call returns an lbm2p_status; lbm2p_last_error(handle) (or
 * lbm2p_last_error(NULL) after a failed create) gives a one-line description.
 * LBM2P_ENOTCONVERGED still advances the state.  LBM2P_ENONFINITE from lbm2p_step rolls
 * the failing step back: the state after the call (lbm2p_get_state, the fields) is the state
 * before that step, bit for bit, so the caller may fix its inputs and step again.
 */
#ifndef LBM2P_H
#define LBM2P_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM2P_ABI_VERSION 7
/* Sparse wells passed to the sweep kernels as launch arguments (more wells: error). */
#define LBM2P_MAX_WELLS 16

typedef struct lbm2p lbm2p;

typedef enum {
    LBM2P_OK = 0,
    LBM2P_EINVAL = 1,          /* bad argument; nothing was changed */
    LBM2P_ENOMEM = 2,          /* device or host allocation failed */
    LBM2P_ECUDA = 3,           /* a CUDA call failed; the handle should be destroyed */
    LBM2P_ENOTCONVERGED = 4,   /* max_sub_iters reached before the residual met tol */
    LBM2P_ENONFINITE = 5,      /* the pressure residual became NaN (e.g. NaN sources); a
                                  step that meets it is rolled back */
    LBM2P_ENOTIMPL = 6         /* requested option is not implemented by the library */
} lbm2p_status;

/* Wall kinds of Sec. 4: bounce-back for no-flux, anti-bounce-back for Dirichlet. */
typedef enum { LBM2P_BC_PERIODIC = 0, LBM2P_BC_NOFLUX = 1, LBM2P_BC_DIRICHLET = 2 } lbm2p_bc_kind;
typedef enum { LBM2P_XMIN = 0, LBM2P_XMAX = 1, LBM2P_YMIN = 2, LBM2P_YMAX = 3 } lbm2p_side;

/* Mobility laws lambda_w(S), lambda_t(S):
 *   QUADRATIC: k_rw = S^2, k_rn = (1-S)^2, lambda_a = k_ra / mu_a (Eq. 2-9, Sec. 4.3);
 *   DECOUPLED: lambda_t = lambda_w = 1/mu_w, independent of S (Sec. 4.1);
 *   RATIONAL:  lambda_t = 1/(0.5 - 0.2 S), lambda_w = S lambda_t (Eq. 4-4, K = 1). */
typedef enum { LBM2P_MOB_QUADRATIC = 0, LBM2P_MOB_DECOUPLED = 1, LBM2P_MOB_RATIONAL = 2 } lbm2p_mobility;

/* Pressure pseudo-time scale s (Eq. 3-1 is iterated in a pseudo time of its own, Sec. 3):
 * tau_f(x) = 1/2 + 3 s D_p(x) (Eq. 3-11a), and the source enters as s dx^2 F_p.
 *   REFERENCE:   s = (tau_p - 1/2) / (3 D_ref); D_ref = params.D_ref when > 0, else the
 *                geometric mean of D_p(K, S0) over the grid at t = 0 (fixed for the run);
 *   PHYSICAL_DT: s = dt / dx^2 (pseudo step equal to the physical step, as in Sec. 4). */
typedef enum { LBM2P_TAU_REFERENCE = 0, LBM2P_TAU_PHYSICAL_DT = 1 } lbm2p_tau_mode;

/* Single-sweep pressure kernels.  All compute bit for bit the same populations:
 *   VEC4:   four nodes per thread, 128-bit loads and stores;
 *   SCALAR: one node per thread;
 *   ROWS:   a block marches down a strip of rows whose input rows are staged in shared memory
 *           by bulk asynchronous copies (cp.async.bulk) several rows ahead.
 * AUTO lets create time them on the lattice and keep the fastest. */
typedef enum { LBM2P_SWEEP_AUTO = 0, LBM2P_SWEEP_VEC4 = 1, LBM2P_SWEEP_SCALAR = 2,
               LBM2P_SWEEP_ROWS = 3 } lbm2p_sweep_kernel;

/* Population storage during the pressure sub-iteration.
 *   FP32:     the FP32 deviations n_i = f_i^+ - w_i R (see lbm2p_state_count), 72 B per node
 *             and sweep.
 *   FP16_DEV: each solve narrows them to FP16 scaled by a power of two chosen from max |n_i|,
 *             sweeps with R moved to the node's new pressure after every sweep (so the
 *             stored values are the post-collision non-equilibrium parts f_i^+ - w_i P), and
 *             widens the result back; arithmetic FP32, residual FP64; 44 B per node and
 *             sweep.  The state between steps stays FP32.  FP16 rounding puts a floor under
 *             the relative increment r: use a tolerance above it or replayed sweep counts.
 *             Sweeps are launched from the host (no graph) by an FP16 one-node-per-thread
 *             kernel or an FP16 staged-rows kernel, timed at create (sweep_kernel SCALAR or
 *             ROWS pins one; lbm2p_autotune_report lists "fp16_scalar" and "fp16_rows"
 *             lines); not available in batches. */
typedef enum { LBM2P_STORE_FP32 = 0, LBM2P_STORE_FP16_DEV = 1 } lbm2p_storage;

/* A point well at node (i, j) with total rate q >= 0 (per unit depth): the node's cell
 * receives F_p = +q/dx^2 and F_s = +q/dx^2 (injector) or F_p = -q/dx^2 and
 * F_s = -f_w(S*) q/dx^2 (producer), f_w = lambda_w/lambda_t, S* = sum_i g_i / phi. */
typedef struct {
    int i, j;
    double q;
    int is_producer;
} lbm2p_well;

typedef struct {
    int nx, ny;                 /* lattice size, >= 1 each (Dirichlet sides need >= 3 nodes) */
    double dx, dt;              /* lattice spacing and physical time step */
    double phi, beta;           /* porosity; Eq. 3-4 parameter, phi/2 <= beta <= 2 phi */
    int mobility;               /* lbm2p_mobility */
    double mu_w, mu_n;          /* viscosities of the mobility law */
    double D_s;                 /* saturation diffusivity (constant): Eq. 3-11b gives tau_g */
    int tau_mode;               /* lbm2p_tau_mode */
    double tau_p, D_ref;        /* REFERENCE mode: typical tau_f and its diffusivity */
    double tol;                 /* pressure stopping tolerance on r (see lbm2p_step) */
    int max_sub_iters;          /* cap on sweeps per pressure solve */
    int check_every;            /* sweeps between residual checks, >= 1 */
    int bc[4];                  /* lbm2p_bc_kind per side (XMIN, XMAX, YMIN, YMAX); a
                                   periodic side must be paired with its opposite */
    int storage;                /* lbm2p_storage */
    int fuse_sweeps;            /* pressure sweeps fused per kernel launch: 0 = automatic,
                                   1 = one sweep per launch, 2 or 4 = that many.  Results are
                                   identical bit for bit whatever the choice; fusion reads and
                                   writes the populations once per fused group of sweeps.
                                   Within the choice, create times the candidate kernels and
                                   tile shapes on the lattice and keeps the fastest; with 0 a
                                   fused form replaces single sweeps only when its time per
                                   sweep is at most 0.95 of the best single sweep's (these
                                   timings favour the fused forms a little).  Fused
                                   kernels: T = 2 or 4 sweeps on shared-memory stages, and, on
                                   lattices with walls on every side, 2 sweeps on rows staged
                                   by bulk copies and 2 sweeps with direct loads (fuse_sweeps
                                   2 with sweep_kernel ROWS pins the former, with SCALAR the
                                   latter). */
    int sweep_kernel;           /* lbm2p_sweep_kernel: the single-sweep kernel (AUTO: timed) */
    int sat_lattice;            /* saturation lattice: 9 (D2Q9, Eq. 3-4) or 5 (D2Q5, Remark V,
                                   Eq. 3-4b, weights 1/3 and 1/6; needs beta <= 1.5 phi) */
    double D_c;                 /* saturation-dependent diffusivity (Remark IV):
                                   D_s(x, S) = D_s + D_c K lambda_w lambda_n / lambda_t, the
                                   D_s of Eq. 2-16 with a linear capillary pressure of scale
                                   D_c; tau_g then varies per node (Eq. 3-11b).  0: constant */
    int warm_start;             /* start of each step's pressure solve.  0: the previous
                                   step's populations as they are (continuation, the paper's
                                   pseudo-time reading).  1: their equilibrium part moved to the
                                   pressure extrapolated linearly in time, 2 P^n - P^{n-1}
                                   (f_i += f_i^eq(P^n - P^{n-1}), Eq. 3-3), the non-equilibrium
                                   part kept.  Each solve still runs to the same stopping rule;
                                   only its starting iterate changes (far fewer sweeps). */
    void *stream;               /* cudaStream_t the work is enqueued on */
    void *(*alloc)(size_t bytes, void *ctx);            /* optional device allocator */
    void (*release)(void *ptr, size_t bytes, void *ctx); /* its matching free */
    void *alloc_ctx;
} lbm2p_params;

typedef struct {
    const double *K;            /* [ny][nx] absolute permeability, required */
    const double *S0;           /* [ny][nx] initial saturation, required */
    const double *P0;           /* [ny][nx] initial pressure guess, or NULL (zero) */
    const double *Fp, *Fs;      /* [ny][nx] dense sources at t = 0, or NULL (zero) */
    const lbm2p_well *wells;    /* n_wells entries, or NULL */
    int n_wells;                /* 0 .. LBM2P_MAX_WELLS */
    /* Dirichlet wall traces for each side whose kind is DIRICHLET: the wall value at the
       points k dx / 2, k = 0 .. 2n (n = ny for XMIN/XMAX, nx for YMIN/YMAX); a link of a
       boundary node crosses the wall at one of these points.  NULL means zero. */
    const double *P_b[4];
    const double *S_b[4];
    const int *init_replay;     /* NULL: iterate the t = 0 pressure to tol; else that
                                   exact number of sweeps */
} lbm2p_inputs;

typedef struct {
    int sub_iters;              /* pressure sweeps run in this step */
    int status;                 /* lbm2p_status of this step */
    double residual;            /* last evaluated r (NaN when no check ran) */
    float sweep_ms;             /* device time of the pressure sweeps (timing on), else -1 */
    float step_ms;              /* device time of the whole step (timing on), else -1 */
} lbm2p_step_stats;

/* ABI version of the loaded library (LBM2P_ABI_VERSION). */
int lbm2p_abi_version(void);

/* Fill params with defaults: phi = 0.2, beta = 0.4, quadratic mobility with mu_w = 1,
   mu_n = 2, D_s = 0.01, REFERENCE mode with tau_p = 1, tol = 1e-8, check_every = 8,
   max_sub_iters = 10^7, no-flux walls, FP32 storage, cudaMalloc, default stream. */
void lbm2p_default_params(lbm2p_params *p);

/* Create a solver and run the t = 0 initialisation of Sec. 4: f = f^eq(P0) (Eq. 3-3),
 * tau_f from S0, the pressure solve, then g(0) = g^eq(S0) + eps g^(1) (Eqs. gini, gneq;
 * grad S0 by second-order central differences, grad P by Eq. 3-10a) followed by the t = 0
 * collision of g.  init_stats (may be NULL) receives the t = 0 solve's statistics; its
 * step_ms is the device time of that solve alone (CUDA events around it, whatever the
 * timing setting; the create-time kernel tuning and the uploads are not in it).
 * Returns EINVAL for inconsistent parameters (nothing allocated, *out = NULL). */
lbm2p_status lbm2p_create(lbm2p **out, const lbm2p_params *p, const lbm2p_inputs *in,
                          lbm2p_step_stats *init_stats);

/* Replace the dense sources F_p, F_s (host [ny][nx] FP64, NULL = zero) used from the next
   step on (Eq. 2-17 sources evaluated at the new time level). */
lbm2p_status lbm2p_set_sources(lbm2p *h, const double *Fp, const double *Fs);

/* Replace a Dirichlet side's wall traces (host FP64, 2n+1 values, NULL = zero). */
lbm2p_status lbm2p_set_dirichlet(lbm2p *h, int side, const double *P_b, const double *S_b);

/* Advance nsteps physical steps (Sec. 3 order, see the top of this file).
 * Pressure stopping rule: every check_every-th sweep k >= 2 of a step computes
 *     r_k = ||dP - mean(dP)||_2 / ||P^k - mean(P^k)||_2,   dP = P^k - P^{k-1},
 * and the iteration stops when r_k <= tol, or at max_sub_iters (ENOTCONVERGED).
 * replay: NULL, or nsteps sweep counts (>= 0) to run exactly instead.
 * stats: NULL or nsteps entries.  Returns the worst status over the steps.
 * A step reads the state and writes spare buffers (a third set of pressure populations, a
 * second set of R, 1/tau_f and the warm start's previous pressure), which become the state
 * when the step ends.  When a residual check finds a value that is not a number the step
 * stops: no saturation update runs, the state stays the one before the step, and the call
 * returns LBM2P_ENONFINITE without running the remaining steps (a replayed count detects
 * it only when it is >= 2, at the final check). */
lbm2p_status lbm2p_step(lbm2p *h, int nsteps, const int *replay, lbm2p_step_stats *stats);

/* Run exactly nsweeps pressure sweeps (Eq. 3-1) with the current tau_f and sources, no
   stopping test; residual (may be NULL) receives r of the last sweep when nsweeps >= 2.
   The populations after the call are those the sweeps produced, also when they are not
   finite (ENONFINITE): no rollback here. */
lbm2p_status lbm2p_pressure_sweeps(lbm2p *h, int nsweeps, double *residual);

/* Darcy velocity u = -K lambda_t(S) grad P (Eq. 3-10b) of the current time level into
   caller buffers of ny*nx floats (device pointers if on_device, else host). */
lbm2p_status lbm2p_velocity(lbm2p *h, float *ux, float *uy, int on_device);

/* Pressure (Eq. 3-9a; minus its mean when mean_free_P) and saturation S^n (Eq. 3-9b) of
   the current time level into ny*nx float buffers (either may be NULL). */
lbm2p_status lbm2p_fields(lbm2p *h, float *P, float *S, int mean_free_P, int on_device);

/* Number of floats in a state image: 20 planes of ny*nx, in order
 *   n_1..n_8  pressure populations, stored as deviations n_i = f_i^+ - w_i R from the
 *             reference pressure R below (f_i^+ the post-collision populations of Eq. 3-1),
 *   g_0..g_8  post-collision saturation populations (Eq. 3-2),
 *   1/tau_f, S, R.
 * The library keeps f in this form on the device: R is the pressure of the last converged
 * step, so the stored values are small and FP32 resolves them finely. */
size_t lbm2p_state_count(const lbm2p *h);

/* Copy the state out / in (checkpoint and restart; count must equal lbm2p_state_count). */
lbm2p_status lbm2p_get_state(lbm2p *h, float *buf, size_t count, int on_device);
lbm2p_status lbm2p_set_state(lbm2p *h, const float *buf, size_t count, int on_device);

/* Warm start of the next pressure solve from a caller's pressure field (for instance a learned
   predictor's): P_guess, ny*nx floats (device pointer if on_device, else host), becomes the
   equilibrium part of the pressure populations (their non-equilibrium part is kept), exactly
   as warm_start = 1 does with its extrapolated field.  The solve's stopping rule is unchanged.
   A constant offset in P_guess is harmless where P is defined up to a constant (no Dirichlet
   side).  Combined with warm_start = 1, the extrapolation is applied on top at the next step. */
lbm2p_status lbm2p_warm_start(lbm2p *h, const float *P_guess, int on_device);

/* Record CUDA events around each step and its sweeps (fills sweep_ms / step_ms). */
lbm2p_status lbm2p_set_timing(lbm2p *h, int enable);

/* How the pressure sweeps run on this handle, as chosen at create: sweeps fused per launch
   (1, 2 or 4); the single-sweep kernel (an lbm2p_sweep_kernel value, never AUTO); the tile
   of the kernel that runs the sweeps: for fused sweeps its threads per block (columns per
   block for the two-sweep row-walking kernels: 120 or 240) and rows per block, for the ROWS
   kernel its strip width and rows per block, otherwise 0 and 0. */
lbm2p_status lbm2p_sweep_config(const lbm2p *h, int *fused, int *kind, int *tile_w, int *tile_h);

/* Which fused kernel runs the sweeps when lbm2p_sweep_config reports fused > 1. */
typedef enum {
    LBM2P_FUSED_NONE = 0,        /* single sweeps */
    LBM2P_FUSED_STAGES = 1,      /* T sweeps on shared-memory stages (T = 2 or 4) */
    LBM2P_FUSED_STAGED_ROWS = 2, /* two sweeps on rows staged by bulk copies */
    LBM2P_FUSED_DIRECT = 3       /* two sweeps, inputs loaded directly (lattices held in L2) */
} lbm2p_fused_form;
int lbm2p_fused_form_of(const lbm2p *h);

/* Pin the two-sweep launch shape instead of the one create chose: form STAGED_ROWS (warps 4
   or 8 consumer warps; slots 6 or 8 with 4 warps, 4 or 6 with 8, or 6 + LBM2P_ROWS2_DENSE: 4
   warps and 6 slots with the register cap that keeps seven plain blocks per SM; rows 16, 32, 64
   or 128) or DIRECT (warps 4 or 8, slots 0, rows 2, 4, 8, 16 or 32); rows above ny mean ny.
   Every shape computes the same populations bit for bit; only the speed differs.  The lattice
   needs walls on every side and FP32 storage (the graph-resident loop uses the shape when
   check_every is a multiple of 4, the host-driven loop always).  Waits for the
   handle's stream and drops its solve graphs (rebuilt on the next solve); a batch created
   before keeps the shape it was built with.  EINVAL (handle unchanged) for any other value. */
#define LBM2P_ROWS2_DENSE 16
lbm2p_status lbm2p_set_fused_shape(lbm2p *h, int form, int warps, int slots, int rows);

/* The candidates create timed to choose the sweep kernel, one line each:
 *   "single_vec4 <grid> 0 0 0 <us>", "single_scalar <grid> 0 0 0 <us>",
 *   "single_rows <strip width> <ring slots> <rows per block> <grid> <us>",
 *   "fused <sweeps per launch> <threads per block> <rows per block> <grid> <us>",
 *   "fused_rows <consumer warps> <ring slots> <rows per block> <grid> <us>",
 *   "fused_direct <warps> 0 <rows per block> <grid> <us>"
 * with <us> the time per sweep inside the solve loop: a check period of check_every sweeps
 * timed as its plain launches plus the one launch that also sums the residual (the first two
 * kinds once per grid tried: the resident-block capacity of the GPU down to half of it).  Owned by h; valid until the next create-time tuning. */
const char *lbm2p_autotune_report(const lbm2p *h);

/* Running totals since creation: kernels launched by the library, pressure sweeps run. */
lbm2p_status lbm2p_counters(const lbm2p *h, long long *launches, long long *sweeps);

/* ---- Batched realisations --------------------------------------------------------------
 * Independent lattices (for instance Monte Carlo realisations of the permeability field,
 * each with its own size, coefficients and sources) advanced together: one CUDA graph per
 * physical step runs steps 1-3 above for every member, each kernel covering the tiles of
 * all members, and the sub-iteration continues while any member is still above its
 * tolerance (members that met theirs stop sweeping).  The paper solves one realisation at
 * a time; this is the same per-member computation scheduled so that small lattices fill
 * the GPU together: they share one sweep kernel over a tile list, while the members of 512^2
 * nodes or more on lattices with walls on every side share a two-sweeps-per-launch kernel
 * over a list of their blocks, beside the shared sweep (when check_every is a multiple of 4).
 *
 * members: count handles made by lbm2p_create on the current device, all on one stream,
 * all with one even check_every that divides each member's max_sub_iters; each handle
 * appears once.  The batch keeps pointers to the members' device memory: destroy the
 * batch before any member, and while it exists step members only through the batch
 * (lbm2p_batch_step returns EINVAL if a member was stepped alone).  Between batch steps
 * a member may be read (fields, velocity, get_state, counters) and its sources, wall
 * values and state replaced (set_sources, set_dirichlet, set_state).  The batch owns a
 * little device memory of its own (a descriptor per member, 36 bytes per tile of 256
 * nodes), allocated with cudaMalloc. */
typedef struct lbm2p_batch lbm2p_batch;
lbm2p_status lbm2p_batch_create(lbm2p_batch **out, lbm2p *const *members, int count);

/* Advance every member nsteps physical steps.  Member m's stopping rule is its own tol
 * and max_sub_iters.  replay: NULL, or nsteps*count sweep counts (step-major: entry
 * s*count + m), each a multiple of check_every, run exactly.  stats: NULL or nsteps*count
 * entries in the same order (step_ms is the whole batched step; sweep_ms is -1).  Each
 * member's state after a step is bit-identical to lbm2p_step on that handle alone with the
 * same sweep count.  Returns the worst status (ENONFINITE stops at the failing step). */
lbm2p_status lbm2p_batch_step(lbm2p_batch *b, int nsteps, const int *replay,
                              lbm2p_step_stats *stats);

/* Kernels launched by the batch so far, and the tiles (256 nodes) of one batched sweep. */
lbm2p_status lbm2p_batch_counters(const lbm2p_batch *b, long long *launches, int *total_tiles);

/* One-line description of the batch's last error (NULL: that of the last failed create). */
const char *lbm2p_batch_last_error(const lbm2p_batch *b);

/* Free the batch (not its members; NULL is ignored).  Synchronises the stream first. */
void lbm2p_batch_destroy(lbm2p_batch *b);

/* ---- Pressure sweep for callers that cannot allocate device memory -------------------
 * The paper has no counterpart of this call: it exists for host programs that must not
 * call cudaMalloc while running (codes that give all device memory to their own pool at
 * start-up, real-time loops that forbid allocation after initialisation, plug-ins inside
 * an application that owns the device allocator).  Such callers cannot create a handle,
 * but can run the solver's pressure sweep on buffers they already own.
 *
 * One fused pressure sweep (the kernel lbm2p_step uses), then the residual r of the
 * stopping rule, for one lattice whose planes the caller owns on the current device:
 *   n_in[8]  pressure populations in the library's deviation form n_i = f_i^+ - w_i R,
 *            directions c_1..c_8, each a [ny][pitch] FP32 plane (read);
 *   n_out[8] the populations after the sweep (written; no output plane may be an input
 *            plane, another output plane, R, inv_tau, Fp or dP: EINVAL);
 *   R        reference pressure, inv_tau = 1/tau_f, Fp = dense pressure source already in
 *            lattice units (s dx^2 F_p) or NULL: [ny][pitch] FP32 planes (read);
 *   P_b[4]   Dirichlet wall traces (FP32, 2n+1 values) for sides whose bc is DIRICHLET;
 *   dP       [ny][pitch] FP32: on entry the pressure increment P - R of the previous
 *            sweep, on exit that of this sweep (so calls chain; the first call's residual
 *            compares with whatever dP held); not R, inv_tau, Fp or an input plane (EINVAL);
 *   residual host double: r = ||dP_new - dP_old - mean|| / ||P_new - mean P_new||.
 * pitch is a multiple of 4 floats and every plane pointer is 16-byte aligned.  Wells are
 * not taken: put their sources into Fp.
 * Memory: allocates nothing.  The residual scratch (four FP64 partials per row tile of 1024
 * nodes, the finalize output and two shifts) is a static device array sized for
 * LBM2P_NOALLOC_MAX_TILES tiles (2 MiB), held by every GPU that loads the library until the
 * process exits; lattices with more row tiles (ceil(nx / 1024) * ny) are rejected with
 * LBM2P_EINVAL before anything is launched.  The first call on each device (and again the
 * first after that device's context is re-created, e.g. by cudaDeviceReset) looks up the
 * array's device address with that device current.  Every call shares the one array and
 * each call clears what must start at zero, so calls whose work overlaps on the GPU (other
 * streams, other host threads) race on it: serialise them.  Each call synchronises `stream`
 * (a cudaStream_t) to return the residual to the host, so it cannot be used inside a stream
 * capture.  Errors: lbm2p_last_error(NULL) describes the failure. */
#define LBM2P_NOALLOC_MAX_TILES 65536
lbm2p_status lbm2p_pressure_sweep_noalloc(int nx, int ny, int pitch, const int bc[4],
                                          const float *const n_in[8], float *const n_out[8],
                                          const float *R, const float *inv_tau, const float *Fp,
                                          const float *const P_b[4], float *dP, double *residual,
                                          void *stream);

/* One-line description of the last error of h (or of the last failed create if h NULL). */
const char *lbm2p_last_error(const lbm2p *h);

/* Free every resource of h (NULL is ignored).  Synchronises the stream first. */
void lbm2p_destroy(lbm2p *h);

#ifdef __cplusplus
}
#endif

#endif /* LBM2P_H */
