/*
 * C ABI of the GB300 D2Q9 pseudopotential MRT lattice Boltzmann solver with the
 * finite-difference energy equation (Zhao, Xu & Zhang, arXiv:1803.01756,
 * Section 2, Eqs. 1-18; channel problem of Section 3.3).
 *
 * Conventions shared by every entry point:
 *  - A lattice has nx * ny fluid nodes.  Host field arrays are row-major
 *    [ny][nx] doubles (x fastest), owned by the caller.
 *  - "stream" is a cudaStream_t passed as void*; NULL means the legacy default
 *    stream.  Calls enqueue their GPU work on it; calls that return host data
 *    synchronise that stream before returning.
 *  - Time t counts completed lattice updates.  The populations of time t carry
 *    the inlet velocity u_amp sin(2 pi t / u_period) and step t multiplies the
 *    body force by cos(g_omega t).
 *  - Every call returns LBM_OK (0) or a negative LBM_ERR_* code.  A failed call
 *    leaves the handle usable for lbm_read_* and lbm_destroy.
 *  - Temperatures in lbm_params_t are in units of the critical temperature Tc of
 *    Eq. 11 (Tc = 0.0778 a / (0.45724 b R)); field temperatures are absolute.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_OK 0
#define LBM_ERR_ARG -1       /* invalid argument or size */
#define LBM_ERR_OOM -2       /* device or host allocation failed */
#define LBM_ERR_CUDA -3      /* a CUDA runtime call or launch failed */
#define LBM_ERR_UNSTABLE -4  /* device status bits set (see LBM_ST_*) */
#define LBM_ERR_TIMEOUT -5   /* a host-side wait passed its deadline */
#define LBM_ERR_BUSY -6      /* admission refused */
#define LBM_ERR_STATE -7     /* malformed checkpoint */

/* device status bits, OR-ed by the kernels (never a trap) */
#define LBM_ST_NAN 1u        /* NaN in a stored population or temperature */
#define LBM_ST_PSI_NEG 2u    /* negative argument of the square root of Eq. 10 (psi set to 0) */
#define LBM_ST_RHO_NONPOS 4u /* density <= 0 */
#define LBM_ST_EOS_POLE 8u   /* b rho >= 1, the pole of Eq. 11 */
#define LBM_ST_T_NONPOS 16u  /* temperature <= 0 */

#define LBM_X_PERIODIC 0
#define LBM_X_INLET_OUTLET 1 /* Zou-He velocity inlet at x=0, density outlet at x=nx-1 */
#define LBM_X_PRESSURE_INLET 2 /* Zou-He pressure inlet at x=0, density outlet at x=nx-1 */
#define LBM_Y_PERIODIC 0
#define LBM_Y_WALLS 1        /* half-way bounce-back walls below y=0 and above y=ny-1 */

#define LBM_STORAGE_F32 0    /* populations stored as FP32 f_i - w_i rho_ref */
#define LBM_STORAGE_BF16 1   /* stored as BF16 f_i / w_i - rho_ref (FP32 arithmetic) */
#define LBM_STORAGE_F16 2    /* stored as FP16 f_i / w_i - rho_ref (FP32 arithmetic) */

#define LBM_KERNEL_AUTO 0    /* the library's choice: with the energy equation on, the two-pass
                                path for lattices of at most 2^18 nodes, else the fused kernel */
#define LBM_KERNEL_SPLIT 1   /* density/psi, collide, energy: three launches per update */
#define LBM_KERNEL_FUSED 2   /* one launch per update; the library picks the columns per thread */
#define LBM_KERNEL_FUSED_1COL 3 /* the fused kernel with one lattice column per thread */
#define LBM_KERNEL_FUSED_2COL 4 /* the fused kernel with two lattice columns per thread */
#define LBM_KERNEL_TWOPASS 5 /* two launches per update: streaming and collision (Eqs. 6-15),
                                then the RK4 energy update (Eqs. 16-18) */

/* Problem parameters, copied by value at lbm_create (the caller keeps ownership). */
typedef struct lbm_params {
  double eos_a, eos_b, eos_R, eos_omega; /* Peng-Robinson EOS, Eq. 11 */
  double G;                              /* fluid-fluid interaction strength, Eq. 9 (< 0) */
  double Gw;                             /* fluid-wall strength, Eq. 14 */
  double rho_w;                          /* Eq. 14 wall density; <= 0: psi_w = local psi */
  double theta;                          /* Li forcing constant, Eq. 8 */
  double tau_g, tau_l, rho_g, rho_l;     /* Eq. 5; rho_g is also the rho_v of Eq. 15 */
  double s_e, s_zeta, s_q;               /* Eq. 3 rates of the e, epsilon and q moments */
  double Cv, lambda;                     /* Eq. 16 heat capacity and conductivity */
  double gx, gy, g_omega;                /* Eq. 15 body force (rho-rho_g) g cos(g_omega t) */
  double T0, T_wall_left, T_wall_right, T_inlet; /* units of Tc; wall T linear in x */
  int x_bc, y_bc;                        /* LBM_X_*, LBM_Y_* */
  double u_amp, u_period;                /* inlet velocity; u_period = 0 gives u_amp */
  double rho_out;                        /* outlet density */
  int thermal;                           /* 1: advance T with Eqs. 16-18 (RK4) */
  int multiphase;                        /* 1: pseudopotential forces, Eqs. 9, 14 */
  int storage;                           /* LBM_STORAGE_* */
  double rho_ref;                        /* deviation reference density; <= 0: rho_g, else rho_out, else 1 */
  int kernel;                            /* LBM_KERNEL_* */
  double p_amp_frac;                     /* pressure inlet (Section 3.3): p = p0 (1 + p_amp_frac
                                            sin(2 pi t / u_period)), p0 = P_EOS(rho_out, T_inlet),
                                            imposed as the vapour-branch density of that pressure */
  /* Section 3.2 walls.  The top wall's temperature profile (units of Tc, linear in x; both 0
     selects T_wall_left/right for the top wall too) and, per wall, the columns [x0, x1) that
     are isothermal; the rest of that wall is adiabatic: the energy equation's ghost copies the
     fluid node across the wall (zero normal gradient of T).  x1 <= x0 makes the whole wall
     isothermal.  Adiabatic columns need periodic x ends (LBM_ERR_ARG otherwise). */
  double T_top_left, T_top_right;
  int top_iso_x0, top_iso_x1;
  int bot_iso_x0, bot_iso_x1;
} lbm_params_t;

typedef struct lbm_lattice *lbm_h;

typedef struct lbm_info {
  int nx, ny, pitch;          /* pitch: row stride of the device arrays, in elements */
  long long t;                /* completed updates */
  double Tc;                  /* critical temperature from Eq. 11 */
  double T_ref, rho_ref;      /* deviation references of the stored T and populations */
  size_t device_bytes;        /* device memory held by the handle */
  int kernel;                 /* kernel path in use (LBM_KERNEL_SPLIT, _FUSED or _TWOPASS) */
  int tile_cols, tile_rows;   /* fused kernel (two-pass path: its first pass): most output
                                 columns and rows of one CTA's tile (0 on the split path) */
  int cols_per_thread;        /* fused kernel: lattice columns each thread sweeps (1 or 2;
                                 0 on the split path) */
} lbm_info_t;

/* Create a lattice of nx * ny nodes with parameters *p.  Allocates all device
   memory of the handle on the current device; the populations start at the
   equilibrium of rho_g at rest and T = T0.  LBM_ERR_ARG for nx or ny outside
   [1, 2^20], nx < 2 with open x ends, or invalid parameters (checked before any
   device call); LBM_ERR_OOM if allocation fails. */
int lbm_create(int nx, int ny, const lbm_params_t *p, lbm_h *out);

/* Set the state at the current time from host fields: populations f = f^eq(rho, u = 0)
   (the second-order D2Q9 equilibrium), with the open-boundary rules of the current time
   applied to the boundary columns; T (absolute, may be NULL for uniform T0) as given.
   rho: [ny][nx] host doubles.  Synchronises the stream.  A page-locked host array
   (cudaHostAlloc, cudaMallocHost or cudaHostRegister memory) is read by the kernels
   directly over the host link; any other is first copied to a device staging array. */
int lbm_write_fields(lbm_h h, const double *rho, const double *T, void *stream);

/* Advance nsteps lattice updates (Eqs. 1-18 per update): pull-streaming with bounce-back
   and Zou-He rules, density, pseudopotential (Eqs. 10-11), forces (Eqs. 9, 14, 15),
   velocity (Eq. 13), moment-space collision with Li forcing (Eqs. 6-8) and the RK4
   temperature update (Eqs. 16-18).  Asynchronous: enqueues work on the stream; on the
   fused path the updates go in chunks of 16, each preceded by a 192-byte copy of its
   boundary scalars from pinned host memory, and the host may wait for the copy of the
   chunk before last.  Calls on different streams must be ordered by the caller (they
   share the lattice state).  LBM_ERR_ARG if the stream is being captured into a CUDA
   graph: each call stages the boundary scalars of its own updates, so a captured call
   could not be replayed (lbm_set_graph replays whole chunks instead). */
int lbm_step(lbm_h h, long nsteps, void *stream);

/* enable != 0 (the default): lbm_step replays each full chunk of 16 fused updates from a
   CUDA graph captured on first use (one per buffer parity); 0: one launch per update.
   Per-launch timing (lbm_timing_enable) always launches one by one; the split path never
   uses graphs.  Results are identical either way. */
int lbm_set_graph(lbm_h h, int enable);

/* Copy the fields of the current time t to host arrays (any may be NULL): rho = sum f,
   u = (sum e f + F/2) / rho (Eq. 13, force of time t), T absolute.  Synchronises the
   stream.  Returns LBM_ERR_UNSTABLE if device status bits are set (fields still written).
   Page-locked host arrays are written by the kernels directly, others through a device
   staging array and a copy. */
int lbm_read_fields(lbm_h h, double *rho, double *ux, double *uy, double *T, void *stream);

/* FP64 sums over all nodes of rho (the density of Eq. 13, sum_i f_i) and of rho Cv T
   (the internal energy per unit volume whose balance Eq. 16 states) at the current time:
   *mass and *heat (either may be NULL).  The per-node values are formed in FP32 on the
   device and summed in FP64 (warp shuffles, then one pass over per-block partials).
   Synchronises the stream; LBM_ERR_CUDA if a launch or copy fails. */
int lbm_reduce(lbm_h h, double *mass, double *heat, void *stream);

/* Device status bits (LBM_ST_*) accumulated since creation; clears them when clear != 0.
   The bits flag states outside the domain of the model's equations: a negative argument of
   the square root of Eq. 10, b rho at or beyond the pole of Eq. 11, rho <= 0 (Eq. 13 divides
   by it), T <= 0 (the sqrt(T/Tc) of Eq. 11 and the RK4 stages of Eqs. 16-18), or a NaN.
   *bits written on return.  Synchronises the stream; LBM_ERR_ARG for NULL pointers. */
int lbm_status(lbm_h h, unsigned *bits, int clear, void *stream);

/* Checkpoint of the complete state of the update (Eqs. 1-18 advance the populations f_i of
   Eq. 1 and the temperature of Eq. 16; every other field is recomputed from them): the stored
   post-collision populations, the temperature and the time t as one opaque byte string of
   lbm_state_bytes() bytes (a header with the sizes, pitch, storage and t, then the device
   arrays as stored).  The caller owns buf.  lbm_read_state copies the current state out;
   lbm_write_state restores it into a handle of the same nx, ny and storage, after which
   lbm_step continues bit for bit as the original would.  Both synchronise the stream.
   LBM_ERR_ARG for NULL pointers or a buffer smaller than lbm_state_bytes() on read;
   LBM_ERR_STATE for a short or foreign byte string on write. */
int lbm_state_bytes(lbm_h h, size_t *bytes);
int lbm_read_state(lbm_h h, void *buf, size_t bytes, void *stream);
int lbm_write_state(lbm_h h, const void *buf, size_t bytes, void *stream);

/* Sizes, time, the critical temperature of Eq. 11 and the deviation references of the
   handle, its device footprint and kernel tiling, written to the caller's *info.  Host
   only (no device call).  LBM_ERR_ARG for NULL pointers. */
int lbm_info(lbm_h h, lbm_info_t *info);

/* Per-kernel CUDA-event timing of lbm_step launches.  enable != 0 starts recording
   (events are placed around every launch, which serialises nothing but costs host time).
   lbm_timing_get writes up to n (name, total ms, launches) triples for kernels launched
   since the last reset and synchronises the stream. */
int lbm_timing_enable(lbm_h h, int enable);
int lbm_timing_get(lbm_h h, const char **names, double *total_ms, long *launches, int n,
                   int *count, void *stream);

/* Free everything the handle owns.  NULL is ignored. */
void lbm_destroy(lbm_h h);

const char *lbm_strerror(int code);

/* Critical temperature of Eq. 11 for the given parameters. */
double lbm_critical_temperature(const lbm_params_t *p);

/* Density that the pressure inlet (Section 3.3, LBM_X_PRESSURE_INLET) imposes on column 0
   at time t: the root on the vapour branch of the Peng-Robinson isotherm (Eq. 11) at
   T_inlet of P(rho) = p0 (1 + p_amp_frac sin(2 pi t / u_period)), p0 = P(rho_out, T_inlet);
   the vapour branch runs from 0 to the isotherm's first maximum (to 0.999 / b above Tc),
   and a target above its top pressure gives the branch end.  Host-only: no device call,
   usable without a GPU.  *rho written in FP64.  LBM_ERR_ARG for NULL pointers or
   parameters outside the ranges lbm_create accepts for this inlet. */
int lbm_pressure_inlet_density(const lbm_params_t *p, long long t, double *rho);

/* Droplet statistics of a density field (the condensate on the channel walls of Section 3.3,
   whose droplet count and spacing the paper's closing wettability discussion compares).
   Liquid nodes have rho > threshold (for example the mean of the coexistence densities);
   droplets are 8-connected liquid components that touch a wall row (y = 0: bottom, y = ny - 1:
   top; a component touching both counts for both); a droplet's position is the mean x of its
   nodes (the circular mean when x is periodic).  rho: host [ny][nx] doubles, caller-owned.
   Host-only (no device call, usable without a GPU).  LBM_ERR_ARG for NULL pointers, sizes
   outside [1, 2^20] or a NaN threshold. */
typedef struct lbm_droplet_stats {
  int count[2];            /* droplets on the bottom and on the top wall */
  double spacing[2];       /* mean x distance between neighbouring droplet positions on each wall,
                              (last - first) / (count - 1); nx / count with periodic x; 0 for
                              fewer than two droplets */
  double condensed_mass;   /* sum over liquid nodes of (rho - rho_v) */
  long long liquid_nodes;  /* nodes with rho > threshold */
  int detached;            /* liquid components touching neither wall */
} lbm_droplet_stats_t;
int lbm_droplet_stats(const double *rho, int nx, int ny, double threshold, double rho_v,
                      int periodic_x, lbm_droplet_stats_t *out);

/* ---- batched updates of many lattices (one persistent launch per step) ----
   A batch groups lattices that share the boundary modes (x_bc class, y_bc), the
   thermal and multiphase switches and the storage, and that use the fused kernel or
   the two-pass path (LBM_KERNEL_AUTO gives one of the two);
   sizes and all other parameters may differ.  Each step is one launch whose
   resident CTAs take tiles of all lattices from one work-list (largest lattices
   first) through an atomic counter.  The batch borrows the lattices: they stay
   owned by the caller, must outlive the batch, and while batched should be advanced
   only through lbm_batch_step (their own t, buffers and status words advance).
   A lattice's fields after lbm_batch_step equal those after lbm_step alone. */
typedef struct lbm_batch *lbm_batch_h;

/* LBM_ERR_ARG if a lattice is NULL, repeated, on another device, on the split path, or
   differs in modes or storage from the first. */
int lbm_batch_create(lbm_h *lattices, int n, lbm_batch_h *out);
/* Advance every lattice of the batch by nsteps updates (enqueued on the stream).
   LBM_ERR_ARG if the stream is being captured into a CUDA graph, as for lbm_step. */
int lbm_batch_step(lbm_batch_h b, long nsteps, void *stream);
/* enable != 0: replay whole chunks of 16 steps from one captured CUDA graph. */
int lbm_batch_set_graph(lbm_batch_h b, int enable);
/* Output rows per tile (the work-list granularity).  The default, chosen at creation, is the
   height among 128, 96, 64, 48, 32, 24 and 16 rows whose work-list a greedy schedule over
   the resident CTAs finishes first; if that leaves fewer tiles than SMs, heights down to
   1 row compete, with row steps slower the more tiles share an SM.  A launch has one CTA
   per tile when there are fewer tiles than resident CTAs. */
int lbm_batch_set_tile_rows(lbm_batch_h b, int rows);
/* Set the tiling: output rows and columns per tile and lattice columns per thread (1, or 2
   when the batch's modes include the energy equation and the pseudopotential forces; cols
   at most 118 with one column per thread, an even number up to 244 with two).
   LBM_ERR_ARG otherwise.  Results do not depend on the tiling. */
int lbm_batch_set_tiling(lbm_batch_h b, int rows, int cols, int cols_per_thread);
int lbm_batch_tiling(lbm_batch_h b, int *rows, int *cols, int *cols_per_thread);
/* The library's autotuner: times tilings with steps_per_candidate timed updates each (plus
   two warm-up updates) and keeps the fastest.  Candidates: tile heights 16, 24, 32, 48, 64,
   96 and 128 rows at the widest tiles, for one column per thread and, where the modes allow
   it, two; then tiles of three quarters and half that width at the winner's height and
   column count.  These are real updates: every lattice advances by
   (7 k + 2) * (steps_per_candidate + 2) steps, k the number of column counts tried (1 or 2).
   Writes the winning height to *best_rows (may be NULL; lbm_batch_tiling gives all three).
   Synchronises the stream. */
int lbm_batch_autotune(lbm_batch_h b, int steps_per_candidate, int *best_rows, void *stream);
int lbm_batch_info(lbm_batch_h b, int *ntiles, int *grid, int *tile_rows);
/* Synchronises the device, frees the batch's tables; the lattices are untouched. */
void lbm_batch_destroy(lbm_batch_h b);

/* ---- serving: continuous batching of simulation jobs ----
   A server owns one CUDA stream and one worker thread on `device`.  Jobs (lattice
   size, parameters, initial density, number of updates) are submitted at any time
   and queue first come, first served.  The worker admits queued jobs while fewer
   than max_active run and their device footprint (populations, temperature and
   scratch of lbm_create) fits in hbm_budget bytes; it then advances all running
   jobs that share modes together in batched launches (lbm_batch_*; a group's batch is
   kept across rounds while its jobs stay the same), and each job of 2^20 nodes or more,
   which fills the GPU alone, with lbm_step, chunk_steps updates per round (fewer when a
   job has fewer left); it reads every job's status word with one synchronisation, reads
   finished jobs' fields back to host memory and frees their device memory, which admits
   the next jobs.
   A job's fields equal those of the same job run alone (lbm_step) within the FP32
   parity bound. */
#define LBM_JOB_QUEUED 0
#define LBM_JOB_RUNNING 1
#define LBM_JOB_DONE 2  /* other final states are negative LBM_ERR_* codes */

typedef struct lbm_server_config {
  int device;          /* CUDA device the worker uses */
  size_t hbm_budget;   /* bytes of device memory all running jobs may hold */
  int max_active;      /* running jobs at most */
  long chunk_steps;    /* updates per scheduling round */
} lbm_server_config_t;

typedef struct lbm_server_stats {
  long queued, active, completed, failed, rounds;
  size_t bytes_in_use, peak_bytes;
} lbm_server_stats_t;

typedef struct lbm_server *lbm_server_h;

int lbm_server_create(const lbm_server_config_t *cfg, lbm_server_h *out);
/* Queue a job; rho0 ([ny][nx] host doubles, copied) may be NULL for rest at rho_g.
   Never blocks.  LBM_ERR_BUSY if the job alone exceeds hbm_budget. */
int lbm_submit(lbm_server_h s, int nx, int ny, const lbm_params_t *p, const double *rho0,
               long nsteps, long *job_id);
/* Non-blocking: *state = LBM_JOB_* or a negative error.  When LBM_JOB_DONE, copies the
   final fields into any non-NULL [ny][nx] host arrays and the submit-to-done time. */
int lbm_poll(lbm_server_h s, long job_id, int *state, double *rho, double *ux, double *uy,
             double *T, double *latency_s);
/* Block until the job leaves the queued and running states or timeout_s passes
   (LBM_ERR_TIMEOUT). */
int lbm_wait(lbm_server_h s, long job_id, double timeout_s, int *state);
int lbm_server_stats(lbm_server_h s, lbm_server_stats_t *st);
/* Stops the worker after its current round; queued and running jobs are cancelled
   (state LBM_ERR_ARG). */
void lbm_server_destroy(lbm_server_h s);

/* Largest nx or ny that lbm_mass_heat_noalloc accepts. */
#define LBM_NOALLOC_MAX_DIM (1 << 20)

/* FP64 sums of rho and of rho * Cv * (T_dev + T_ref) over an nx * ny field pair, for
   callers that cannot allocate device memory: a host framework or serving loop that
   owns the whole device-memory budget and hands out buffers only from its own pool,
   or a latency-critical loop that must not risk the device-wide synchronisation that
   cudaMalloc and cudaFree can cause.  This entry point has no counterpart in the paper;
   it is a service of this library.
   rho, T_dev: device arrays of FP32, row y at element offset y * pitch (pitch >= nx).
   out: device memory for two doubles, written with {sum rho, sum rho Cv T}.
   Enqueued on the stream; nothing is allocated and nothing is synchronised.
   The two-stage reduction keeps its per-block partial sums in one fixed array of
   1216 pairs (19 KB) in this library's device memory, which every GPU that loads the
   library holds until the process exits; the first call on a device looks up that
   array's address (make that first call before any stream capture).  All calls on a
   device share the array: calls whose kernels overlap on the GPU (different streams
   without ordering) race and may return wrong sums.  Each call overwrites every
   partial pair it reads, so nothing needs clearing between calls.
   Returns LBM_ERR_ARG for NULL pointers, nx or ny outside [1, LBM_NOALLOC_MAX_DIM] or
   pitch outside [nx, 2 * LBM_NOALLOC_MAX_DIM]; LBM_ERR_CUDA if a CUDA call fails. */
int lbm_mass_heat_noalloc(const float *rho, const float *T_dev, int nx, int ny, int pitch,
                          double T_ref, double Cv, double *out, void *stream);

#ifdef __cplusplus
}
#endif
#endif
