/*
 * pplbm -- GB300 (sm_103a) pseudopotential thermal lattice Boltzmann step for
 * flow boiling in a narrow channel, after Mukherjee, Basu & Mondal, "Mesoscopic
 * Characterization of Bubble Dynamics in Flow Boiling following A
 * Pseudopotential-based Approach" (arXiv 2009.05264).
 *
 * C ABI.  Plain pointers and sizes only; no exceptions cross it.  Every call
 * returns an lbm_status; lbm_last_error() gives the text of the last failure
 * of a context.  All quantities are lattice units (dx = dt = 1, c_s^2 = 1/3).
 *
 * Lattice (Sec. 2.A, Fig. 1): D2Q9 with velocities
 *   0 (0,0) 1 (1,0) 2 (0,1) 3 (-1,0) 4 (0,-1) 5 (1,1) 6 (-1,1) 7 (-1,-1) 8 (1,-1)
 * and weights 4/9, 1/9 (i = 1..4), 1/36 (i = 5..8).
 * Grid: fluid nodes x = 0..nx-1 (inlet x = 0, outlet x = nx-1), y = 0..ny-1.
 * Walls lie halfway between rows: solid rows y = -1 (bottom, carries the
 * microheater) and y = ny (top).
 *
 * Host arrays crossing this interface are row-major, index y*nx + x; population
 * arrays are 9 such planes, index (i*ny + y)*nx + x.  They are owned by the
 * caller and only read or written during the call.
 *
 * Threading: a context is used by one host thread at a time.  Work is ordered
 * on the context's CUDA stream.
 */
#ifndef PPLBM_H
#define PPLBM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 2

typedef struct lbm_ctx lbm_ctx;
typedef struct lbm_batch lbm_batch;

typedef enum {
  LBM_OK = 0,
  LBM_EINVAL = 1,    /* bad argument: NULL pointer, size mismatch, parameter out of range */
  LBM_ENOMEM = 2,    /* device or host allocation failed, or caller buffer too small */
  LBM_EUNSTABLE = 3, /* the lattice left the EOS domain: rho <= 0, rho >= 1/b, NaN, or a
                        negative psi radicand (Eq. 11).  State is kept for inspection. */
  LBM_ETIMEOUT = 4,  /* a bounded device wait gave up */
  LBM_ECUDA = 5,     /* a CUDA runtime call failed (text in lbm_last_error) */
  LBM_EBUDGET = 6,   /* admission refused: device memory budget exceeded */
  LBM_ESTATE = 7,    /* call out of order (e.g. lbm_step before lbm_set_params) */
  LBM_EBOUNDS = 8    /* only from a library compiled with -DLBM_BOUNDS_CHECK (a test build): a
                        kernel formed an element index outside the buffer it addresses; the
                        access was skipped, so the lattice state is undefined */
} lbm_status;

typedef enum { LBM_FP32 = 0, LBM_FP64 = 1 } lbm_precision;

enum {
  LBM_GEOM_PERIODIC = 0, /* periodic in x and y (static droplet / bubble tests) */
  LBM_GEOM_CHANNEL = 1,  /* Sec. 2.C: velocity inlet x = 0, pressure outlet x = nx-1, walls */
  LBM_GEOM_WALLS = 2,    /* walls at y = -1 and y = ny, periodic in x */
  LBM_GEOM_POOL = 3      /* pool boiling (Sec. 2.D): periodic in x, bottom wall (heater) at y = -1, and a
                            free-surface top read as a constant-pressure boundary: Zou-He rho = rho_out,
                            u_x = 0 on row ny-1, zero temperature gradient; needs ny >= 3 */
};

enum { LBM_INIT_UNIFORM = 0, LBM_INIT_DISK = 1 };

/* Diagnostics record of one step, computed from that step's moments: each CTA sums its nodes in
 * FP64, and the CTA sums are added as signed 64-bit fixed-point totals with 52 - ceil(log2 m)
 * fraction bits (m = nx*ny for mass, energy and the vapour counts, nx for the heater row, ny for
 * the inlet and outlet columns).  Integer addition makes a record independent of the order in
 * which CTAs finish; rounding adds at most 2^-(53 - ceil(log2 m)) per CTA.  A CTA sum outside the
 * totals' range (per-node terms above 1024 in magnitude: a diverged run) or a NaN sets the
 * unstable status. */
enum {
  LBM_D_STEP = 0,    /* step index n */
  LBM_D_MASS,        /* sum of rho over fluid nodes (Eq. 4) */
  LBM_D_ENERGY,      /* sum of T over fluid nodes (Eq. 17) */
  LBM_D_RHO_AVG,     /* mass / (nx*ny): the rho_avg the buoyancy of step n+1 uses (Eq. 14) */
  LBM_D_DP,          /* centreline pressure drop p(1, ny/2) - p(nx-2, ny/2) (Sec. 3.B, Fig. 12b) */
  LBM_D_DTSTAR,      /* (T_wall - T_next_to_heater)/(T_wall - T_bulk) (Sec. 3.B, Fig. 12c); 0 if heater off */
  LBM_D_FLUX_IN,     /* sum over y of rho * u_act,x at x = 0 */
  LBM_D_FLUX_OUT,    /* sum over y of rho * u_act,x at x = nx-1 */
  LBM_D_VAPOR_AREA,  /* nodes with rho < rho_vapor: bubble area (Sec. 3.A, Fig. 8); this and the next
                        three records need params.bubble_stats = 1 */
  LBM_D_WALL_VAPOR,  /* of those, nodes on the row next to the bottom wall: the vapour footprint,
                        i.e. the contact-line extent in 2D (Sec. 3.E, Fig. 17) */
  LBM_D_HEATER_VAPOR,/* of those, nodes above heater sites: non-zero while a bubble sits on the heater */
  LBM_D_ZONE_VAPOR,  /* vapour nodes in the columns x_h - n_h <= x < x_h + 2 n_h: the bubble at the heater,
                        without the earlier bubbles the stream has carried off */
  LBM_D_COUNT
};

/* Problem parameters (lattice units).  `size` must be sizeof(lbm_params).
 * lbm_default_params() fills the paper's values; see each field. */
typedef struct lbm_params {
  uint32_t size;
  int32_t geometry;   /* LBM_GEOM_* */
  int32_t thermal;    /* 1: evolve the temperature distribution g (Eq. 16); 0: T fixed at T0 */
  int32_t multiphase; /* 1: Shan-Chen (Eq. 9) + wetting (Eq. 15) forces with the PR EOS;
                         0: single-phase lattice gas p = rho/3 (duct-flow validation, Sec. 2.D) */
  double tau_f;       /* relaxation time of f (Eq. 2); nu = (tau_f - 1/2)/3.  Default 1 */
  double tau_g;       /* relaxation time of g (Eq. 16); alpha_T = (tau_g - 1/2)/3.  Default 0.6 (with
                         tau_g >= 1 thermal runs between walls grow a wall mode and diverge) */
  double a, b, R;     /* Peng-Robinson constants of Eq. 12: 2/49, 2/21, 1 */
  double omega;       /* acentric factor (Eq. 12): 0.32 (R134a) */
  double beta;        /* force mixing weight of Eq. 8: 1.16 */
  double c0;          /* Eq. 11: 6 */
  double G;           /* interaction strength g of Eqs. 10-11 (g1 = 2G, g2 = G/2): -1 */
  double T0_R;        /* initial temperature / Tc (Eq. 13): 0.9 */
  double Tin_R;       /* inlet and wall temperature / Tc: 0.9 */
  double dTheat_R;    /* heater superheat / Tc: 0.3 (Sec. 3.A) */
  double u_in;        /* inlet velocity (x) */
  double rho_out;     /* outlet density (channel), top density (pool) */
  double rho_w;       /* false wall density of Eq. 15 (sets the contact angle): 5.95 */
  double G_wet;       /* wetting strength of Eq. 15: 9 (1 + beta) G, so that a wall whose false density
                         equals the fluid's exerts no net force on uniform fluid under the beta-mixed
                         Eq. 9 (18 G at beta = 1, where G_wet w_i is the Eq. 10 stencil) */
  double g_a;         /* gravitational acceleration magnitude, acting along -y (Eq. 14): 5e-5 */
  double c_v;         /* specific heat at constant volume in the source of Eq. 19: 6 */
  int32_t heater_x0;  /* first heated bottom-wall site; -1 = nx/5 */
  int32_t heater_len; /* number of heated sites: 5 */
  int64_t heat_on_step; /* first step whose boundary condition heats: 10000 */
  int32_t init_kind;  /* LBM_INIT_UNIFORM: rho = init_rho_out everywhere;
                         LBM_INIT_DISK: init_rho_in inside a centred disk of init_radius,
                         tanh interface of init_width, times (1 + perturb_amp * xi) with
                         xi = splitmix64 hash of (seed, node) in [-1, 1).  u = 0, T = T0. */
  int32_t reserved0;
  double init_rho_in, init_rho_out, init_radius, init_width, perturb_amp;
  uint64_t seed;
  double rho_vapor;   /* bubble diagnostics count a node as vapour when rho < rho_vapor: 3.2
                         (about the midpoint of the coexisting densities 0.59 and 5.88 at 0.9 Tc) */
  int32_t source_model; /* energy source of Eq. 16: LBM_SOURCE_GONG_CHENG (second Eq. 19, the paper's
                           choice, default) or LBM_SOURCE_HAZI_MARKUS (first Eq. 19, with the temporal
                           density gradient rho^n - rho^(n-1); the context keeps rho^(n-1) per node,
                           equal to the initial or injected density before the first step) */
  int32_t bubble_stats; /* 1: count vapour nodes every step (the LBM_D_*_VAPOR records); 0 (default):
                           those records stay 0 and the step runs its leaner form */
} lbm_params;

enum { LBM_SOURCE_GONG_CHENG = 0, LBM_SOURCE_HAZI_MARKUS = 1 };

/* Fill *p with the defaults listed above (and p->size). */
void lbm_default_params(lbm_params* p);

/* Device bytes a context of this size needs (state double buffers, reductions). */
size_t lbm_required_bytes(int32_t nx, int32_t ny, lbm_precision prec);

/* Create a context for an nx x ny lattice on CUDA device `device`.
 * prec: LBM_FP64 stores and computes populations in FP64; LBM_FP32 stores them in
 * FP32 as deviations from the rest-state weights (w_i rho_out, w_i T0) and
 * computes in FP32, with FP64 global reductions.
 * cuda_stream: a cudaStream_t to order all work on, or NULL for a stream the
 * context creates and owns.  The context allocates its device memory.
 * Errors: LBM_EINVAL (nx, ny < 1, or 9 * ny * pitch >= 2^31 elements, pitch = nx rounded
 * up to 32: about 238 M nodes), LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_create(lbm_ctx** out, int32_t nx, int32_t ny, lbm_precision prec, int32_t device,
                      void* cuda_stream);

/* As lbm_create, but the state lives in caller-owned device memory dev_buf of
 * dev_bytes >= lbm_required_bytes(); it must outlive the context.  dev_buf
 * must be 256-byte aligned.  Errors as lbm_create, LBM_ENOMEM if dev_bytes is short. */
lbm_status lbm_create_ex(lbm_ctx** out, int32_t nx, int32_t ny, lbm_precision prec, int32_t device,
                         void* cuda_stream, void* dev_buf, size_t dev_bytes);

/* Validate and store parameters, then initialise the lattice from p->init_kind
 * (f = f^eq(rho, 0), Eq. 3; g = g^eq(T0, 0), Eq. 18) at step 0.
 * Errors: LBM_EINVAL (p NULL, p->size wrong, geometry too small: channel needs
 * nx >= 3, ny >= 2; walls need ny >= 2; tau <= 1/2; non-positive c_v ...). */
lbm_status lbm_set_params(lbm_ctx* ctx, const lbm_params* p);

/* Start from host fields (n = nx*ny each, row-major): f = f^eq(rho, u) (Eq. 3),
 * g = g^eq(T, u) (Eq. 18); T is the absolute lattice temperature (T_R * Tc) and
 * may be NULL (T0 everywhere).  Sets step 0; the buoyancy mean of the previous
 * step (Eq. 14) is the mean density of the initialised populations, summed on the
 * device (FP64: the mean of rho up to rounding; FP32: of rho as stored).  Returns
 * once the populations are in place.  Requires lbm_set_params. */
lbm_status lbm_init_fields(lbm_ctx* ctx, const double* rho, const double* ux, const double* uy,
                           const double* T, size_t n);

/* Advance nsteps time steps (Eqs. 1-19 and the Sec. 2.C boundary conditions),
 * fused into one kernel per step, then wait and return the stability status.
 * Errors: LBM_ESTATE (no params), LBM_EUNSTABLE, LBM_ECUDA. */
lbm_status lbm_step(lbm_ctx* ctx, int64_t nsteps);

/* Enqueue nsteps steps without waiting; lbm_sync() waits and reports status. */
lbm_status lbm_step_async(lbm_ctx* ctx, int64_t nsteps);
lbm_status lbm_sync(lbm_ctx* ctx);

/* Macroscopic fields of the current state, FP64, into caller host arrays of n =
 * nx*ny: rho (Eq. 4), the actual velocity u_act (Eq. 7) and T (Eq. 17).  Any
 * pointer may be NULL.  Errors: LBM_EINVAL (n != nx*ny), LBM_ESTATE, LBM_ECUDA. */
lbm_status lbm_read_fields(lbm_ctx* ctx, double* rho, double* ux, double* uy, double* T, size_t n);

/* Post-stream populations f^n, g^n of the current state in FP64 (n = 9*nx*ny
 * per array; g may be NULL).  In FP32 mode the stored deviations are widened
 * and the rest-state weights added back. */
lbm_status lbm_get_populations(lbm_ctx* ctx, double* f, double* g, size_t n);

/* Replace the state by post-stream populations f^n, g^n (n = 9*nx*ny; g NULL
 * keeps g^eq(T0, 0)), at time step `step`, with the previous step's mean density
 * rho_avg_prev (Eq. 14); pass NaN to use the mean of the given populations. */
lbm_status lbm_set_populations(lbm_ctx* ctx, const double* f, const double* g, size_t n, int64_t step,
                               double rho_avg_prev);

/* Diagnostics record of the most recent step: out[LBM_D_COUNT]. */
lbm_status lbm_read_diagnostics(lbm_ctx* ctx, double* out, size_t n);

/* Records of the steps first, first + 1, ..., first + count - 1 (oldest first) into the
 * host array out[count][LBM_D_COUNT].  The context keeps the records of its last 1024
 * steps; LBM_EINVAL if a requested step is not held (not yet taken, or more than 1024
 * steps back) or count < 0.  Waits for the context's stream. */
lbm_status lbm_read_diagnostics_range(lbm_ctx* ctx, int64_t first, int64_t count, double* out);

/* Checkpoint / resume: raw state (a header with the step, buoyancy mean and
 * parameters; then f and g as 9 planes of ny x nx each in storage precision; then the
 * per-node density history of the Hazi-Markus source, 1 plane).  lbm_state_bytes()
 * gives the buffer size; resume is bitwise. */
size_t lbm_state_bytes(const lbm_ctx* ctx);
lbm_status lbm_save_state(lbm_ctx* ctx, void* host_buf, size_t bytes);
lbm_status lbm_load_state(lbm_ctx* ctx, const void* host_buf, size_t bytes);

/* Tile shape of the fused kernel: columns per CTA (64, 128 or 256; a CTA writes
 * cols - 8 columns, the other 8 cover halo columns; the scalar kernel runs cols
 * threads, the paired kernel cols / 2) and rows per CTA (>= 4, or the full height).
 * Results do not depend on the shape except through the per-CTA sums of the
 * domain-mean density (Eq. 14) and their rounding to the fixed-point totals; only speed differs.  0 = default: the band plan of
 * lbm_default_band_plan for the CTA slots of the current device and kernel form. */
lbm_status lbm_set_tiling(lbm_ctx* ctx, int32_t cols, int32_t rows);

/* Time trial_steps steps of each candidate tiling (64, 128 and 256 columns, each with the
 * default plan and with uniform bands of 4, 7, 10, 16, 24, 32 and 48 rows where the lattice
 * is that high) and keep the fastest; the chosen columns and rows (0 = default plan) go to
 * *cols and *rows (either may be NULL).  The trials advance the lattice: re-initialise it
 * afterwards if its state matters.  Results depend on the tiling only through the per-CTA
 * sums of the domain-mean density.  Errors: LBM_EINVAL (trial_steps < 1), LBM_ESTATE (no
 * parameters), LBM_EUNSTABLE, LBM_ECUDA. */
lbm_status lbm_autotune(lbm_ctx* ctx, int32_t trial_steps, int32_t* cols, int32_t* rows);

/* The context's current step tiling: CTA columns, and per strip of cols - 8 columns
 * tall_count bands of tall_rows from the bottom followed by bands of short_rows up to the
 * top (the last possibly lower); uniform tilings have tall_count = 0.  Any output pointer
 * may be NULL.  LBM_EINVAL if ctx is NULL. */
lbm_status lbm_get_tiling(const lbm_ctx* ctx, int32_t* cols, int32_t* tall_rows, int32_t* tall_count,
                          int32_t* short_rows);

/* The default step tiling of an nx x ny lattice with `cols`-column CTAs when `slots` CTAs
 * (SMs x resident CTAs per SM) fit on the device at once: one cost model (row-iterations
 * per CTA slot, each tile charged its rows, 4 halo rows and one row of fixed cost, plus
 * half a tile of the class dispatched last) compares uniform bands of the balanced heights
 * ceil(ny / bands) >= 4 rows (every band charged that height; ny itself when ny <= 4) with
 * two-level plans: bands of 2h rows dispatched first and about one wave (ceil(slots /
 * strips) per strip) of h-row bands dispatched last, h >= 4.
 * Output as lbm_get_tiling.  Host-only (no device needed).  LBM_EINVAL for nx, ny < 1,
 * cols not 64, 128 or 256, or slots < 1. */
lbm_status lbm_default_band_plan(int32_t nx, int32_t ny, int32_t cols, int64_t slots, int32_t* tall_rows,
                                 int32_t* tall_count, int32_t* short_rows);

/* Form of the FP32 step kernel.  All forms compute the same step (Sec. 2; boundary
 * conditions of Sec. 2.C) and agree to FP32 rounding.
 *   LBM_KERNEL_SCALAR (and LBM_KERNEL_AUTO, the default): one column per thread; each
 *     thread stages the populations it pulls with per-element asynchronous copies
 *     (cp.async).  Handles every option.  The fastest form on GB300.
 *   LBM_KERNEL_PAIRED: each thread updates two adjacent columns with packed FP32
 *     arithmetic (two nodes per add / multiply / fused multiply-add) and 8-byte stores;
 *     about 40 % fewer instructions per node but fewer warps per SM, slower on GB300.
 *     Lattices with the Hazi-Markus source take the scalar form.
 *   LBM_KERNEL_TMA: one column per thread; one thread per CTA stages whole rows of
 *     every population plane with bulk tensor copies (cp.async.bulk.tensor, completion
 *     on mbarriers), which removes the per-thread copy work from the step.  Needs
 *     128-column tiles and the step's lean form (no pool geometry, Hazi-Markus source
 *     or bubble statistics); other lattices take the scalar form.  A bulk copy that does
 *     not complete within a bounded wait (lbm_set_wait_limit) makes lbm_sync return
 *     LBM_ETIMEOUT.  Its results
 *     are bit-identical to the scalar form's; on GB300 it runs about 9 % slower (its
 *     warps wait on rows that arrive later than the per-thread copies do).
 * FP64 lattices, and lbm_step_noalloc on caller-laid-out buffers, always use the scalar
 * form.  LBM_EINVAL for other values. */
enum { LBM_KERNEL_AUTO = 0, LBM_KERNEL_SCALAR = 1, LBM_KERNEL_PAIRED = 2, LBM_KERNEL_TMA = 3, LBM_KERNEL_INTERIOR = 4 };
lbm_status lbm_set_kernel(lbm_ctx* ctx, int32_t kernel);
/* The form (LBM_KERNEL_SCALAR, _PAIRED or _TMA) the context's step launches take
 * with its current kernel request, precision, parameters and tiling; -1 if ctx is NULL. */
int32_t lbm_step_kernel(const lbm_ctx* ctx);

/* How lbm_step / lbm_step_async advance the lattice (a calling convention of the library;
 * the paper's time loop, Sec. 2 and Fig. 2, is the same either way).
 *   LBM_LOOP_LAUNCHES: one step-kernel launch per step.
 *   LBM_LOOP_PERSISTENT: one cooperative launch per call advances all nsteps steps (nsteps >= 2;
 *     a single step is one launch).  Where the step tiling fits in one wave, each CTA keeps
 *     its tile and the CTAs meet at a grid-wide barrier between steps.  Where it needs more
 *     CTAs than are resident, and the geometry is a channel, walls or periodic box, the
 *     launch overlaps consecutive steps (reported as LBM_LOOP_OVERLAPPED): the CTAs draw
 *     (step, tile) tickets in order, and a tile starts as soon as the tiles around it (the
 *     rows and columns its pulls read) have finished the previous step, the step before that
 *     is complete, and the inlet and outlet tiles of the previous step have posted the mass
 *     that crossed the open ends; its
 *     buoyancy mean (Eq. 14) is the mean density two steps back plus that mass over the
 *     nodes, which is the previous step's mean up to the rounding of one collision.  Otherwise
 *     (the pool geometry) the CTAs draw each step's tiles from a counter and meet at a
 *     barrier between steps.  Every wait is bounded: a CTA that waits longer than 5 s (or
 *     than the poll limit of lbm_set_wait_limit) gives up, the launch ends, and the next
 *     lbm_sync returns LBM_ETIMEOUT; the lattice state is then undefined until it is
 *     initialised again (lbm_set_params, lbm_init_fields, lbm_set_populations or
 *     lbm_load_state), and the CUDA context stays usable.  Only the one-column step forms
 *     (LBM_KERNEL_SCALAR, LBM_KERNEL_INTERIOR) have a persistent form.
 *   LBM_LOOP_AUTO (default): persistent where the step tiling fits in one wave of the
 *     persistent kernel (small lattices, whose steps are short enough for the launch gap and
 *     the kernel boundary to count) or where it takes at least two and a half waves and the
 *     launch can overlap the steps, else one launch per step.
 * Results are the same either way up to the rounding of separately compiled kernels (and,
 * overlapped, of one collision in the buoyancy mean).  LBM_EINVAL for other values. */
enum { LBM_LOOP_AUTO = 0, LBM_LOOP_LAUNCHES = 1, LBM_LOOP_PERSISTENT = 2, LBM_LOOP_OVERLAPPED = 3 };
lbm_status lbm_set_step_loop(lbm_ctx* ctx, int32_t loop);
/* The loop a multi-step call takes now: LBM_LOOP_LAUNCHES, _PERSISTENT (a barrier between
 * steps) or _OVERLAPPED (a persistent launch that overlaps the steps); -1 if ctx is NULL. */
int32_t lbm_step_loop(lbm_ctx* ctx);
/* Poll limit of the step's bounded device waits: the persistent launch's grid-barrier waits
 * (default: 5 s of polling) and the TMA form's waits for its staged rows (default: 2^22
 * polls); a wait gives up after max_polls polls (0 restores the defaults).  A test sets 1 to
 * make a wait run out while the work it waits for is still under way, and checks that
 * lbm_sync reports LBM_ETIMEOUT, that nothing faults, and that the context recovers after a
 * new initialisation (a TMA wait that gives up still lets its row's copies land before the
 * CTA ends).  LBM_EINVAL for max_polls < 0 or >= 2^32. */
lbm_status lbm_set_wait_limit(lbm_ctx* ctx, int64_t max_polls);

int64_t lbm_get_step(const lbm_ctx* ctx);
/* Kernel launches enqueued by this context since creation (all kinds). */
int64_t lbm_launch_count(const lbm_ctx* ctx);
/* The CUDA stream the context orders its work on (a cudaStream_t). */
void* lbm_get_stream(const lbm_ctx* ctx);
/* Critical temperature of the parameters' Eq. 12: Tc = 0.0778 a / (0.45724 b R). */
double lbm_critical_temperature(const lbm_params* p);

/* ---------------------------------------------------------------------------
 * Batches: many independent lattices of uneven size and parameters advanced
 * together, one fused launch per step over all members' tiles (replayed from a
 * captured CUDA graph in runs of 16 steps).  Members share the batch's precision,
 * thermal flag, device and stream; each member is an lbm_ctx owned by the batch,
 * reachable through lbm_batch_member() for initialisation and readback (do not
 * step a member on its own while the batch is stepping it).  A member's results
 * are those of the same lattice run alone with the batch's tiling.
 * ------------------------------------------------------------------------- */

/* Create an empty batch.  cuda_stream NULL: the batch creates and owns a stream. */
lbm_status lbm_batch_create(lbm_batch** out, lbm_precision prec, int32_t thermal, int32_t device,
                            void* cuda_stream);
/* Add an nx x ny member with parameters p (p->thermal must match the batch), initialised
 * as lbm_set_params does; *slot receives its index (freed slots are reused).
 * Allocates the member's device memory (lbm_required_bytes). */
lbm_status lbm_batch_add(lbm_batch* b, int32_t nx, int32_t ny, const lbm_params* p, int32_t* slot);
/* Remove a member and free its device memory (waits for the batch's stream). */
lbm_status lbm_batch_remove(lbm_batch* b, int32_t slot);
/* The member's context, or NULL for a free slot.  Owned by the batch. */
lbm_ctx* lbm_batch_member(lbm_batch* b, int32_t slot);
int32_t lbm_batch_size(const lbm_batch* b);
/* Tiling of the batched launch: columns per CTA (64, 128, 256) and rows per band
 * (0 = each member's default, else >= 4). */
lbm_status lbm_batch_set_tiling(lbm_batch* b, int32_t cols, int32_t rows);
/* Step kernel form of the batched launch (as lbm_set_kernel). */
lbm_status lbm_batch_set_kernel(lbm_batch* b, int32_t kernel);
lbm_status lbm_batch_get_tiling(const lbm_batch* b, int32_t* cols, int32_t* rows);
/* Time trial_steps of every candidate tiling on the current members and keep the
 * fastest (reported in *cols, *rows; either may be NULL).  The trials advance the
 * members: re-initialise them afterwards if their state matters. */
lbm_status lbm_batch_autotune(lbm_batch* b, int32_t trial_steps, int32_t* cols, int32_t* rows);
/* Advance every member nsteps steps, then wait and check every member's status
 * (LBM_EUNSTABLE if any member left the EOS domain). */
lbm_status lbm_batch_step(lbm_batch* b, int64_t nsteps);
/* Enqueue without waiting; lbm_batch_sync waits, returns the first failing member's
 * status and its slot in *unstable_slot (-1 if none; may be NULL). */
lbm_status lbm_batch_step_async(lbm_batch* b, int64_t nsteps);
lbm_status lbm_batch_sync(lbm_batch* b, int32_t* unstable_slot);
/* The step loop of the batch's multi-step calls (LBM_LOOP_* as lbm_set_step_loop): one
 * cooperative launch per call over every member's tiles, which overlaps consecutive steps
 * (each member's tiles wait only for that member's neighbouring tiles, its step two back and
 * its open-end balance) where every member is a channel, walls or periodic lattice and the
 * tiling needs more CTAs than are resident, and otherwise meets at bounded grid barriers
 * between steps; or one launch per step replayed from CUDA graphs.  LBM_LOOP_AUTO takes the
 * overlapped launch from two and a half waves of tiles up and the graph-replayed launches
 * below (measured faster for small served mixes).  A wait that gives up sets LBM_ETIMEOUT on
 * the member whose tile gave up; lbm_batch_sync reports it. */
lbm_status lbm_batch_set_step_loop(lbm_batch* b, int32_t loop);
/* The loop a multi-step call takes now (LBM_LOOP_LAUNCHES, _PERSISTENT or _OVERLAPPED); -1 on
 * error. */
int32_t lbm_batch_step_loop(lbm_batch* b);
/* As lbm_set_wait_limit, for the batch's persistent and TMA launches. */
lbm_status lbm_batch_set_wait_limit(lbm_batch* b, int64_t max_polls);
/* lbm_read_fields of one member. */
lbm_status lbm_batch_read_fields(lbm_batch* b, int32_t slot, double* rho, double* ux, double* uy, double* T,
                                 size_t n);
int64_t lbm_batch_launch_count(const lbm_batch* b);
void* lbm_batch_get_stream(const lbm_batch* b);
const char* lbm_batch_last_error(const lbm_batch* b);
/* Destroy the batch and every member.  NULL-safe. */
lbm_status lbm_batch_destroy(lbm_batch* b);

/* One fused step without any device allocation, for callers that cannot call
 * cudaMalloc: code that runs inside a process whose device memory is owned by
 * another allocator or budgeted to the last byte, or a plug-in that may only use
 * the buffers its host hands it.  The paper has no counterpart; this is a calling
 * convention of the library.
 *
 * Populations are caller-owned device arrays in the library's storage form:
 * 9 planes of ny rows of nx elements (no padding), element type float for
 * LBM_FP32 and double for LBM_FP64.  FP32 stores deviations from the rest state,
 * f_i - w_i rho_ref and g_i - w_i T0 (rho_ref = p->rho_out for a channel, else
 * p->init_rho_out; T0 = p->T0_R * Tc); FP64 stores the populations themselves.
 * in_post_stream = 1: f_in, g_in hold post-stream populations f^n (an initial
 * state); 0: they hold the previous call's output, which this call streams.
 * f_out, g_out receive the post-collision populations of step `step` and must not
 * alias the inputs; g_in and g_out may be NULL when p->thermal is 0.
 * rho_avg_prev is the domain-mean density of step - 1 (buoyancy, Eq. 14);
 * diag_out (host, LBM_D_COUNT doubles, may be NULL) receives this step's record,
 * whose LBM_D_RHO_AVG is the rho_avg_prev of the next call.  The call waits for
 * the step on cuda_stream (a cudaStream_t; NULL = the default stream).
 *
 * Scratch: a fixed 0.36 MB device array inside the library, which every GPU that
 * loads the library holds until the process exits.  Every call looks up that array's
 * device address on the current device (cudaGetSymbolAddress), so a device reset or a
 * recreated context between calls is safe.  Every call reuses the same array and
 * overwrites the previous call's contents (the parts that must start at zero are
 * cleared by each call), so calls that overlap on the GPU (other streams, other host
 * threads) race and must be serialised by the caller.  The call allocates nothing:
 * no cudaMalloc, cudaFree or allocating library routine; it copies two small
 * descriptors from host memory, launches, reads the step's state back and waits.  Sizes beyond the array's capacity are rejected:
 * the lattice is cut into ceil(nx / 120) column strips and at most 8192 tiles,
 * so nx > 983040, or 9 * nx * ny >= 2^31, returns LBM_EINVAL.
 * Errors: LBM_EINVAL (invalid parameters, sizes, NULL or aliased buffers),
 * LBM_EUNSTABLE (as lbm_step), LBM_ECUDA. */
lbm_status lbm_step_noalloc(const lbm_params* p, int32_t nx, int32_t ny, lbm_precision prec, const void* f_in,
                            const void* g_in, void* f_out, void* g_out, int32_t in_post_stream, int64_t step,
                            double rho_avg_prev, double* diag_out, void* cuda_stream);

/* Measurement helper, not part of the paper's method: the fused multiply-add rate
 * (floating-point operations per second, two per FMA) that a plain kernel of independent
 * FMA chains reaches on the current device, in FP64 (fp64 = 1) or FP32 (fp64 = 0), over
 * iters FMAs per chain (1 <= iters <= 2^30; 2^16 runs for milliseconds).  The FP64 step is
 * bounded by this rate, which the benchmark reports its FP64 roofline against.  Allocates
 * a small output buffer on cuda_stream (a cudaStream_t; NULL = the default stream) and waits
 * for the probe.  LBM_EINVAL for bad arguments, LBM_ENOMEM, LBM_ECUDA. */
lbm_status lbm_probe_fma_rate(int32_t fp64, int64_t iters, void* cuda_stream, double* flops_per_s);

/* Free the context and its device memory (not caller-provided memory).  NULL-safe. */
lbm_status lbm_destroy(lbm_ctx* ctx);

const char* lbm_status_string(lbm_status s);
const char* lbm_last_error(const lbm_ctx* ctx);

#ifdef __cplusplus
}
#endif
#endif /* PPLBM_H */
