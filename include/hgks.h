/*
 * hgks.h -- C ABI of the GB300 (sm_103a) FP64 hybrid WENO-AO gas-kinetic solver.
 *
 * The library advances the finite-volume semi-discretisation W_t = L(W) of the
 * 1D / 2D Euler or Navier-Stokes equations (arXiv 2304.05572, Sec. 2, Eq. (1))
 * on a uniform structured grid with the two-stage fourth-order (S2O4) time
 * integrator of Sec. 2.2.  Each stage evaluates, for every interface, the
 * extreme-point troubled-cell indicator (Sec. 2.3.1, Steps 1-4), linear-upwind
 * or characteristic WENO-AO reconstruction of the values and normal and
 * tangential derivatives at the interface Gauss points (Sec. 2.3.1 Step 5,
 * Eqs. (26)-(45); Sec. 2.3.3), the kinetic weighting of the equilibrium
 * (Eqs. (46)-(47)) and the time-integrated second-order gas-kinetic flux
 * (Sec. 2.1, Eqs. (6)-(12)).  All arithmetic is IEEE FP64 on the GPU.
 *
 * Conventions (all entry points):
 *   - Return 0 (HGKS_OK) or a negative HGKS_E* code; no exception crosses the ABI.
 *   - The state is the conservative cell averages W, laid out [nv][ny][nx] in C
 *     order (nv = 3 in 1D: rho, rho U, rho E; nv = 4 in 2D: rho, rho U, rho V, rho E),
 *     FP64.  Caller-provided buffers stay owned by the caller; the library never
 *     keeps a pointer to them after the call returns.
 *   - A solver owns its device memory and works on the CUDA stream given at
 *     creation (NULL = the legacy default stream).  A solver is not thread-safe;
 *     distinct solvers on distinct streams may be used from distinct threads.
 *   - hgks_last_error(s) returns a static, human-readable description of the
 *     last failure on s (or, when s is NULL, of the calling thread's last failed
 *     hgks_create_solver / hgks_batch_create / hgks_step_noalloc call).
 */
#ifndef HGKS_H
#define HGKS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define HGKS_OK 0
#define HGKS_EINVAL (-1)         /* invalid argument or configuration */
#define HGKS_ENOMEM (-2)         /* device or host allocation failed */
#define HGKS_ENONPHYSICAL (-3)   /* rho <= 0, p <= 0 or non-finite state detected on the device */
#define HGKS_ETIMEOUT (-4)       /* a bounded device wait ran out (reserved: no kernel of this library waits) */
#define HGKS_ECUDA (-5)          /* a CUDA runtime call failed */

/* boundary conditions (Sec. 3: periodic, non-reflecting, reflecting, symmetric, no-slip adiabatic;
 * Sec. 3.5, double Mach reflection: a prescribed inflow state, a wall that starts at x = shock_x0
 * with the inflow state ahead of it, and a top boundary that follows the exact motion of the
 * oblique shock).  All ghost values are set at the ghost cell's centre (x_c, y_c), at the time of
 * the stage being evaluated (t^n for the first stage, t^n + dt/2 for the second):
 *   HGKS_BC_INFLOW:      ghost = bc_state[side]
 *   HGKS_BC_SHOCK_WALL:  (y-lo, 2D) x_c < shock_x0: bc_state[side]; else reflecting
 *   HGKS_BC_SHOCK_TRACK: (y-lo or y-hi, 2D) x_c < shock_x0 + shock_cot (y_c + shock_speed t):
 *                        bc_state[side] (behind the shock); else shock_pre (ahead of it) */
enum { HGKS_BC_PERIODIC = 0, HGKS_BC_EXTRAP = 1, HGKS_BC_REFLECT = 2, HGKS_BC_SYMMETRY = 3, HGKS_BC_NOSLIP = 4,
       HGKS_BC_INFLOW = 5, HGKS_BC_SHOCK_WALL = 6, HGKS_BC_SHOCK_TRACK = 7 };
/* reconstruction: hybrid (the paper's method), linear upwind only, WENO-AO everywhere (Sec. 3, Tables 1 and 4) */
enum { HGKS_RECON_HYBRID = 0, HGKS_RECON_LINEAR = 1, HGKS_RECON_WENOAO = 2 };
/* readings of zeta1 = "5/17 dx" in Step 1 (Sec. 2.3.1): A = (5/17) dx, B = 5/(17 dx) (default), C = 5/17 in cell units */
enum { HGKS_ZETA1_A = 0, HGKS_ZETA1_B = 1, HGKS_ZETA1_C = 2 };

typedef struct hgks_config {
    int dim;                  /* 1 or 2 */
    int nx, ny;               /* interior cells; ny = 1 in 1D */
    double x0, x1, y0, y1;    /* domain [x0,x1] x [y0,y1] */
    double gamma;             /* ratio of specific heats (Sec. 3: 1.4) */
    int viscous;              /* 0: Euler, tau = c1 dt + c2 |pl-pr|/(pl+pr) dt; 1: Navier-Stokes, tau = mu/p + c2 ... (Sec. 3) */
    double mu, prandtl;       /* dynamic viscosity (1/Re); Prandtl number.  The paper's BGK flux has Pr = 1;
                                 for viscous runs with Pr != 1 the energy flux gains (1/Pr - 1) q, q the
                                 time-integrated heat flux of the interface distribution of Eq. (10) relative
                                 to the equilibrium velocity (an extension; Pr = 1 leaves the flux untouched) */
    double c1, c2;            /* collision-time constants (Sec. 3) */
    double cfl;               /* dt = cfl min(h/(|U|+a), h^2/(4 nu)), h = min(dx, dy), nu = mu/rho */
    double fixed_dt;          /* > 0: use this dt instead of the CFL rule (Sec. 3.1 uses dt = 0.2 dx) */
    int tau_zero;             /* 1: tau = 0 (Sec. 3.1, 3.3) */
    int bc[4];                /* x-lo, x-hi, y-lo, y-hi: HGKS_BC_* */
    int recon_mode;           /* HGKS_RECON_* */
    int zeta1_mode;           /* HGKS_ZETA1_* */
    double gamma_hi, gamma_lo;/* WENO-AO linear weights, Eq. (35) (0.85, 0.85) */
    double eps;               /* WENO-AO epsilon, Eq. (37) (1e-8) */
    double bc_state[4][4];    /* conservative state [side][component] for HGKS_BC_INFLOW / _SHOCK_* sides */
    double shock_pre[4];      /* conservative state ahead of the shock (HGKS_BC_SHOCK_TRACK) */
    double shock_x0, shock_cot, shock_speed;   /* shock line x = shock_x0 + shock_cot (y + shock_speed t) */
} hgks_config;

typedef struct hgks_stats {
    long long steps;          /* S2O4 steps taken since set_state */
    double t;                 /* simulation time */
    double last_dt;           /* dt of the last step */
    int status;               /* 0 or the HGKS_E* code latched on the device */
    int pad_;
    /* troubled counts accumulated over all steps: [stage][sweep x/y][0 = normal cells, 1 = tangential passes] */
    long long troubled[2][2][2];
    /* number of candidates counted by troubled[][][] (cells resp. passes examined) */
    long long examined[2][2][2];
    /* kernels this solver enqueued since the last hgks_set_state (host-side count) */
    long long launches;
} hgks_stats;

typedef struct hgks_solver hgks_solver;

/* Fill *cfg with the paper's defaults (gamma 1.4, c1 0.01, c2 1, CFL 0.5, hybrid, reading B,
 * gamma_hi = gamma_lo = 0.85, eps 1e-8, periodic boundaries).  Returns HGKS_EINVAL on NULL. */
int hgks_config_default(hgks_config* cfg);

/* Validate *cfg and allocate the solver and its device buffers on the current
 * CUDA device.  stream: a cudaStream_t cast to void* (NULL = default stream).
 * On success *out owns the solver; free it with hgks_destroy_solver.
 * Errors: HGKS_EINVAL (bad config, see hgks_last_error(NULL)), HGKS_ENOMEM, HGKS_ECUDA. */
int hgks_create_solver(const hgks_config* cfg, void* stream, hgks_solver** out);

/* Release every resource of s (NULL is a no-op).  Synchronises s's stream first. */
void hgks_destroy_solver(hgks_solver* s);

/* Copy the conservative cell averages W ([nv][ny][nx], FP64) into the solver,
 * reset time to t0 and the step and troubled counters to zero and clear the
 * latched status.  on_device = 0: W is host memory (pageable or pinned);
 * 1: W is device memory of the solver's device.  The copy is ordered on the
 * solver's stream; the call returns after W may be reused by the caller. */
int hgks_set_state(hgks_solver* s, const double* W, int on_device, double t0);

/* Advance by whole S2O4 steps until the time reaches t_end (the last step is
 * shortened to land on it; the run stops once t_end - t <= 1e-12 max(1, |t_end|))
 * or max_steps steps were taken.  All work is enqueued on the solver's stream;
 * dt is computed and clipped on the device.  If steps_done is non-NULL the call
 * waits for the stream and stores the number of steps actually taken; with
 * steps_done == NULL it returns after enqueueing (errors latched on the device
 * surface at the next waiting call).  Returns HGKS_ENONPHYSICAL if a
 * non-physical state was detected (the solver then stops advancing; the state
 * the failing step leaves holds NaN wherever a Gauss-point flux met a
 * non-physical state, the same bits however the solver was stepped). */
int hgks_step(hgks_solver* s, double t_end, int max_steps, int* steps_done);

/* Copy the state out ([nv][ny][nx], FP64) to host (on_device = 0) or device (1)
 * memory.  Waits for the solver's stream. */
int hgks_get_state(hgks_solver* s, double* W, int on_device);

/* Current simulation time (waits for the stream). */
int hgks_get_time(hgks_solver* s, double* t);

/* Step count, last dt, latched status and troubled-cell counters (waits for the stream). */
int hgks_get_stats(hgks_solver* s, hgks_stats* st);

/* Troubled flags of the last step (parity hook).  stage 0/1, sweep 0 (x) / 1 (y),
 * kind 0: final (Step-4 spread) flag of every cell the normal reconstruction of
 * the sweep visits, laid out [nt+6][nn+2] (2D) or [1][nn+2] (1D), entry
 * [t+3][n+1] for line t in [-3, nt+2] and cell n in [-1, nn];
 * kind 1 (2D only): bits 0..3 = final flags of the tangential passes of
 * Q^l, Q^r, Q^l_n, Q^r_n at interface m of line t, laid out [nt][nn+1].
 * nn / nt = cell counts normal / tangential to the sweep (x: nn = nx, nt = ny).
 * Flags are recorded only when hgks_set_flag_capture(s, 1) is active.
 * out must hold the stated number of bytes (see hgks_flags_size). */
int hgks_set_flag_capture(hgks_solver* s, int enable);
size_t hgks_flags_size(const hgks_solver* s, int sweep, int kind);
int hgks_get_flags(hgks_solver* s, int stage, int sweep, int kind, uint8_t* out);

/* Per-kernel-class timing (CUDA events on the solver's stream), for profiling.
 * enable = 1 records an event pair around every launch of every class; the
 * totals are summed until reset.  names: kernel class names, ms: total ms,
 * calls: launches; returns the number of classes written (<= cap). */
int hgks_set_timing(hgks_solver* s, int enable);
int hgks_get_timing(hgks_solver* s, int cap, const char** names, double* ms, long long* calls);

/* Description of the last error on s (or of the last create/validation error if s is NULL). */
const char* hgks_last_error(const hgks_solver* s);

/* Number of device bytes a solver of this configuration allocates (for admission control). */
size_t hgks_footprint_bytes(const hgks_config* cfg);

/* ------------------------------------------------------------------------ */
/* Batched execution: many independent solvers advanced by the same launches.*/
/* ------------------------------------------------------------------------ */

typedef struct hgks_batch hgks_batch;

#define HGKS_BATCH_GRAPH 1      /* replay one captured batched step (needs a non-NULL stream) */
#define HGKS_BATCH_AUTOTUNE 2   /* choose the block size of each kernel class on the first steps (see hgks_batch_step) */

/* Group n >= 1 solvers of the same dimension on the current device.  One
 * batched step issues one launch per kernel class (24 per step in 2D, the sweep
 * classes covering both sweeps) whose blocks cover every solver's interfaces;
 * each block works for exactly one solver (and one sweep) with that solver's own
 * arithmetic, so every result is bit-identical
 * to stepping the solver alone.  The solvers keep their own state, dt, time and
 * counters; they must stay alive, and must not be stepped on their own, while
 * the batch exists.  stream: cudaStream_t cast to void* for all batched work.
 * A solver's own stream is ordered with the batch stream by events: work
 * enqueued on it before hgks_batch_step (hgks_set_state, ...) runs before the
 * batched steps, work enqueued on it afterwards (hgks_get_state, ...) after them.
 * The batch's own device memory is O(n) (descriptors, block tables).
 * The paper describes one solve at a time; batching is this library's way of
 * filling one GPU with many small solves.  Errors: HGKS_EINVAL, HGKS_ENOMEM, HGKS_ECUDA. */
int hgks_batch_create(hgks_solver* const* solvers, int n, void* stream, hgks_batch** out);

/* Replace the batch's solvers by solvers[0..n) (n >= 1, the batch's dimension and
 * device), keeping its stream and the block sizes chosen by the autotuner: for a
 * scheduler whose set of resident solves changes between groups of steps.  Waits
 * for the batch's stream and the new solvers' streams; the device arrays are
 * reused while n fits the largest membership so far (grown by doubling
 * otherwise); a captured graph is re-captured at the next graph step and the
 * executable graph updated in place (the kernel sequence is the same) instead of
 * re-instantiated.  The end times start at 0: pass t_end to the next
 * hgks_batch_step.  Results stay bit-identical to stepping each solver alone.
 * Errors: HGKS_EINVAL, HGKS_ENOMEM, HGKS_ECUDA (message in hgks_batch_last_error(b)). */
int hgks_batch_update(hgks_batch* b, hgks_solver* const* solvers, int n);

/* Enqueue nsteps batched S2O4 steps.  t_end (length n, may be NULL to keep the
 * previous values; initially 0) is each solver's end time with hgks_step's
 * clipping rule; solvers at their end time or with a latched error are left
 * unchanged by further steps.  flags: HGKS_BATCH_GRAPH | HGKS_BATCH_AUTOTUNE.
 * With HGKS_BATCH_AUTOTUNE on a batch not tuned yet, the first (up to) 4 of the
 * nsteps steps are taken one at a time with a wait after each: one with the
 * default block sizes, then one with each of three candidate sizes per kernel
 * class, timed per class with CUDA events; the fastest size of each class is
 * kept for the rest of the batch's life.  These are real steps (results do not
 * depend on the block size).  Otherwise the call returns after enqueueing (no
 * wait); use hgks_batch_sync to wait.  A graph captured earlier is rebuilt
 * after tuning. */
int hgks_batch_step(hgks_batch* b, const double* t_end, int nsteps, int flags);

/* Wait for the batch's stream.  *n_active (may be NULL) = solvers that have not
 * reached their t_end and have no latched error; *n_failed (may be NULL) =
 * solvers with a latched HGKS_ENONPHYSICAL (they stopped at the step that
 * produced the state, exactly as hgks_step would; hgks_get_stats tells which).
 * A failed solver does not stop the others, and is not an error of the batch:
 * returns HGKS_OK unless a CUDA call failed (HGKS_ECUDA). */
int hgks_batch_sync(hgks_batch* b, int* n_active, int* n_failed);

/* Per-solver time, latched status (0 or HGKS_ENONPHYSICAL) and step count as of the
 * last hgks_batch_sync, in batch order; no wait, no device access.  Each output
 * array (length n) may be NULL.  Lets a scheduler retire solvers without a
 * round trip per solver. */
int hgks_batch_status(const hgks_batch* b, double* t, int* status, long long* steps);

/* Block size chosen for each kernel class (up to cap entries) and the number of
 * batched steps enqueued so far; returns the number of kernel classes. */
int hgks_batch_info(const hgks_batch* b, int* tpb, int cap, long long* steps_enqueued);

const char* hgks_batch_last_error(const hgks_batch* b);
void hgks_batch_destroy(hgks_batch* b);

/* ------------------------------------------------------------------------ */
/* Debug build (the paper has no counterpart).                               */
/* ------------------------------------------------------------------------ */

/* A library built with HGKS_DEBUG_BOUNDS (paper_2304_05572_gb300/_build.py, debug=True:
 * _lib/libhgks_debug.so) checks every global-memory load and store of its kernels against
 * the range of the solver's device buffers; an access outside it is skipped (a load returns
 * 0) and counted, and the address of the first one is kept; no kernel traps.  Returns 1 and
 * the process-wide *count and *first_address (0 if none) in a debug build, 0 (both set to 0)
 * in the normal build.  Waits for the device.  Errors: HGKS_EINVAL (NULL argument),
 * HGKS_ECUDA. */
int hgks_debug_bounds(unsigned long long* count, unsigned long long* first_address);

/* ------------------------------------------------------------------------ */
/* FP64 rate probe (measurement helper; the paper has no counterpart).       */
/* ------------------------------------------------------------------------ */

/* Measure the FP64 fused-multiply-add rate of the current device: 8 blocks of
 * 256 threads per SM each run 8 independent DFMA chains (4 launches of about
 * 70 ms each at the nominal rate, CUDA events on `stream`, NULL = default
 * stream; the call waits for them).
 * *tflops = 2 x DFMA per second / 1e12, *ms (may be NULL) the time of the 4 launches,
 * *sms (may be NULL) the device's SM count.  Errors: HGKS_EINVAL (tflops NULL),
 * HGKS_ECUDA (message in hgks_last_error(NULL)). */
int hgks_probe_fp64(void* stream, double* tflops, double* ms, int* sms);

/* Check of the flux's reciprocal and reciprocal square root (a measurement
 * helper like the probe above; the paper has no counterpart).  The flux forms 1/x
 * and 1/sqrt(x) as the hardware's approximations refined by two Newton-Raphson
 * steps instead of a division or square root; this evaluates both on n >= 1
 * arguments spread log-uniformly over 1e-8..1e8 (both signs for 1/x) on the
 * current device (default stream; the call waits) and stores in max_ulp[0] the
 * largest distance of 1/x, in units in the last place, from the correctly
 * rounded IEEE quotient, in max_ulp[1] that of 1/sqrt(x) from IEEE division by
 * the IEEE square root (itself up to one rounding away).  max_ulp: 2 entries.
 * Errors: HGKS_EINVAL (n < 1, max_ulp NULL), HGKS_ECUDA. */
int hgks_check_reciprocal(long long n, unsigned long long* max_ulp);

/* ------------------------------------------------------------------------ */
/* Allocation-free single step.                                              */
/* ------------------------------------------------------------------------ */

/* Size of the static device scratch used by hgks_step_noalloc (8 MiB). */
#define HGKS_NOALLOC_SCRATCH_BYTES (8u * 1024u * 1024u)

/* One S2O4 step of the state W_in into W_out, for callers that must not
 * allocate device memory: a process whose memory manager already owns the
 * GPU's memory (a framework's caching allocator, an embedding host that hands
 * the library only buffers it owns), or a loop that cannot afford the
 * device-wide synchronisation cudaMalloc/cudaFree may cause.  The paper has no
 * counterpart; the arithmetic is exactly that of hgks_step on a solver created
 * from *cfg (same kernels, dt from the CFL rule or cfg->fixed_dt, no t_end
 * clipping), so the result is bit-identical to that step.  The step starts at
 * t = 0: boundaries that move with time (HGKS_BC_SHOCK_TRACK) take their t = 0
 * position.
 *
 * W_in, W_out: device memory of the current device, [nv][ny][nx] FP64 as
 * everywhere in this ABI, owned by the caller; they may be the same buffer.
 * status: NULL, or one int the device can be copied to (device memory, or
 * host memory); when the stream reaches the end of the step it holds 0, or
 * HGKS_ENONPHYSICAL if the step met a non-physical state (rho <= 0, p <= 0 or
 * non-finite; W_out is then not a valid state).  The copy is a cudaMemcpyAsync
 * with cudaMemcpyDefault on the stream: with device or pinned host memory the
 * call does not wait, with pageable host memory it waits for the step.
 * Without a status word a non-physical step goes unreported.
 * stream: cudaStream_t cast to void* (NULL = default stream).  The call
 * enqueues the work and returns; W_out (and *status) are ready when the stream
 * reaches them.
 *
 * Every intermediate buffer lives in one file-scope device array of
 * HGKS_NOALLOC_SCRATCH_BYTES that every GPU loading this library holds until
 * the process exits; no cudaMalloc, cudaFree or other allocation is made.  A
 * configuration whose buffers do not fit (hgks_footprint_bytes(cfg) greater
 * than HGKS_NOALLOC_SCRATCH_BYTES: square 2D grids above 74 x 74 cells, 1D
 * grids above 37 105 cells) is rejected with HGKS_EINVAL.  The first call on a device
 * looks up the array's device address (cudaGetSymbolAddress, with that device
 * current); make that first call before any stream capture.  All calls share
 * the one array: calls whose work overlaps on the GPU race and corrupt each
 * other, so issue them one after another (for example on one stream).  Each
 * call clears the array before use.
 * Errors: HGKS_EINVAL (bad config, NULL buffer, grid too large), HGKS_ECUDA;
 * the message is in hgks_last_error(NULL), kept per calling thread. */
int hgks_step_noalloc(const hgks_config* cfg, const double* W_in, double* W_out, int* status, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* HGKS_H */
