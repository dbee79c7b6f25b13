/*
 * tfsph.h - C ABI of the GB300 SPH-IDIC library.
 *
 * One time step of two-fluid smoothed particle hydrodynamics (TFSPH) for a
 * gas-dust mixture whose stiff interphase drag is solved implicitly per Euler
 * cell ("drag in cell", SPH-IDIC), after Stoyanovskaya, Glushko, Snytnikov
 * and Snytnikov, arXiv:1908.01682:
 *   - carrier (gas) and dispersed (dust) phases as two particle sets,
 *     momentum equations in the K form of Eq. 7, drag f = rho_d (v-u)/t_stop
 *     (Eq. 3);
 *   - gas pressure acceleration as the symmetric SPH sum of the first term of
 *     Eq. 19, with the summation density rho^n;
 *   - the domain split into disjoint cells holding N gas and L dust
 *     particles (Sec. 2.3), eps* = m_d L / (m_g N) (Eq. 17), K* with
 *     K* / rho*_g = eps* / t*_stop and K* / rho*_d = 1 / t*_stop (Eq. 18);
 *   - the implicit first-order update of Eqs. 19-20 against the new cell
 *     means of Eq. 21, which conserves each cell's momentum.
 *
 * Conventions for every call:
 *   - Return value: TFSPH_OK (0) or one of the TFSPH_E_* codes below; no call
 *     aborts, throws or traps the GPU. tfsph_last_error() gives a message.
 *   - Floating-point arrays are of the context's precision: float for
 *     TFSPH_FP32, double for TFSPH_FP64.
 *   - mem_kind tells whether a pointer is host memory (TFSPH_MEM_HOST) or
 *     device memory of the current CUDA device (TFSPH_MEM_DEVICE).
 *   - Ownership: the library deep-copies inputs and owns all its device state;
 *     the caller owns every output buffer. Pointers are only read during the
 *     call (asynchronously on the context's stream for device pointers, so the
 *     caller keeps them alive until that stream has reached the call).
 *   - Concurrency: a context is used from one host thread at a time; all its
 *     GPU work is issued on the stream given to tfsph_set_stream (default:
 *     the legacy default stream). tfsph_step makes no host synchronisation.
 *   - Particle identity: particle i of the arrays given to tfsph_init has id
 *     i. Inside the library particles are kept sorted by (cell key, id).
 */
#ifndef TFSPH_H
#define TFSPH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define TFSPH_OK              0
#define TFSPH_E_INVALID_ARG   1  /* bad parameter, size, pointer or enum */
#define TFSPH_E_NONFINITE     2  /* NaN/Inf input, or t_stop <= 0 */
#define TFSPH_E_OUT_OF_DOMAIN 3  /* a moving particle outside [lo, hi) at set-up */
#define TFSPH_E_CUDA          4  /* a CUDA runtime call failed */
#define TFSPH_E_OOM           5  /* device or host allocation failed */
#define TFSPH_E_INTERNAL      6  /* a device-side consistency check failed */
#define TFSPH_E_TIMEOUT       7  /* a bounded device-side wait ran out (batched persistent step) */

#define TFSPH_MEM_HOST   0
#define TFSPH_MEM_DEVICE 1

#define TFSPH_FP32 0  /* float state and pair sums */
#define TFSPH_FP64 1  /* double everywhere */

#define TFSPH_EOS_ISOTHERMAL 0  /* p = cs^2 rho */
#define TFSPH_EOS_ADIABATIC  1  /* p = (gamma - 1) rho e, with an energy equation */

#define TFSPH_KERNEL_CUBIC 0    /* M4 cubic spline, support 2h */

#define TFSPH_TSTAR_ARITHMETIC 0 /* t*_stop = mean of the cell's t_j */
#define TFSPH_TSTAR_HARMONIC   1 /* t*_stop = L / sum 1/t_j */

#define TFSPH_CELL_ACC_FP32 0   /* per-cell sums and drag solve in float */
#define TFSPH_CELL_ACC_FP64 1   /* per-cell sums and drag solve in double */

/* drag scheme (tfsph_params.drag). K = rho_d / t_stop (Eq. 7) with the
 * per-particle stopping times throughout. */
#define TFSPH_DRAG_IDIC 0  /* implicit drag in cell (Sec. 2.3, Eqs. 17-21) */
#define TFSPH_DRAG_ISPH 1  /* semi-implicit SPH interpolation (Sec. 2.2, Eqs. 11-16): per particle,
                              the other phase's velocity, density and K interpolated at it */
#define TFSPH_DRAG_MK   2  /* explicit pairwise drag (Sec. 2.1, Eqs. 8-10); stable only for
                              tau below t_stop (Eq. 5) */

/* fields for tfsph_fields; vector fields are written component-major, out[k*n + i] */
#define TFSPH_FIELD_POS_G    0  /* dim x n_gas */
#define TFSPH_FIELD_VEL_G    1  /* dim x n_gas */
#define TFSPH_FIELD_ENERGY_G 2  /* n_gas, specific internal energy (adiabatic) */
#define TFSPH_FIELD_RHO_G    3  /* n_gas, summation density at the current positions */
#define TFSPH_FIELD_POS_D    4  /* dim x n_dust */
#define TFSPH_FIELD_VEL_D    5  /* dim x n_dust */
#define TFSPH_FIELD_TSTOP_D  6  /* n_dust */
#define TFSPH_FIELD_RHO_D    7  /* n_dust, dust summation density at the current positions */

#define TFSPH_ORDER_ORIGINAL 0  /* out[i] belongs to the particle with id i */
#define TFSPH_ORDER_CELL     1  /* out[s] belongs to storage slot s (sorted by cell, id) */

/* debug exports for tfsph_debug; all refer to the binning of the current positions */
#define TFSPH_DEBUG_KEYS_G       0  /* uint32[n_gas]  cell key per storage slot */
#define TFSPH_DEBUG_KEYS_D       1  /* uint32[n_dust] */
#define TFSPH_DEBUG_PERM_G       2  /* uint32[n_gas]  particle id per storage slot */
#define TFSPH_DEBUG_PERM_D       3  /* uint32[n_dust] */
#define TFSPH_DEBUG_CSTART_G     4  /* uint32[n_cells + 1] first slot of each cell */
#define TFSPH_DEBUG_CSTART_D     5  /* uint32[n_cells + 1] */
#define TFSPH_DEBUG_NEIGH_COUNT  6  /* int32[n_gas] gas neighbours (r < 2h, self included) */
#define TFSPH_DEBUG_NEIGH_FPRINT 7  /* uint64[n_gas] sum over neighbours of (id+1)*0x9E3779B97F4A7C15 */
#define TFSPH_DEBUG_ACC_G        8  /* T[dim x n_gas] pressure acceleration of the last step, storage order */

typedef struct tfsph_ctx tfsph_ctx;

/* Problem parameters. Cells form a uniform grid from lo with
 * n_d = max(1, floor((hi_d - lo_d) / cell_size)) cells along axis d; the
 * same cells serve the drag (Sec. 2.3) and the neighbour search. */
typedef struct {
    int32_t dim;          /* 1, 2 or 3 */
    int32_t precision;    /* TFSPH_FP32 | TFSPH_FP64 */
    int32_t kernel;       /* TFSPH_KERNEL_CUBIC */
    int32_t eos;          /* TFSPH_EOS_* */
    int32_t periodic[3];  /* 1 = periodic axis, 0 = open axis (walls are frozen gas particles) */
    int32_t tstar_mode;   /* TFSPH_TSTAR_* */
    int32_t cell_acc;     /* TFSPH_CELL_ACC_*; forced to FP64 when precision is FP64 */
    int32_t drag;         /* TFSPH_DRAG_*: IDIC (Sec. 2.3, 0), ISPH (Sec. 2.2) or MK (Sec. 2.1) */
    double lo[3], hi[3];  /* box; periodic axes need hi - lo >= 4h */
    double h;             /* smoothing length (> 0), kernel support 2h */
    double cell_size;     /* requested cell edge (> 0) */
    double m_gas, m_dust; /* particle masses (> 0) */
    double cs;            /* isothermal sound speed (> 0) */
    double gamma;         /* adiabatic index (> 1 when adiabatic) */
    double av_alpha, av_beta; /* Monaghan artificial viscosity (>= 0; 0, 0 = off) */
} tfsph_params;

typedef struct {
    int64_t n_gas, n_dust;
    int32_t n_cells[3];
    int32_t reach[3];      /* neighbour-search reach in cells per axis */
    int64_t n_cells_total;
    int64_t steps;         /* steps taken since init or the last set_state */
    int64_t device_bytes;  /* device memory held by the context */
    int64_t launches;      /* kernels launched by tfsph_step since init */
} tfsph_info_t;

/* phases timed by tfsph_profile_read */
#define TFSPH_PROF_COUNT   0  /* cell counts (atomics) */
#define TFSPH_PROF_SCAN    1  /* exclusive scan of the counts: cell ranges */
#define TFSPH_PROF_SCATTER 2  /* slot per particle */
#define TFSPH_PROF_GATHER  3  /* rank in cell by id, copy into cell order */
#define TFSPH_PROF_DENSITY 4  /* gas summation density and p/rho^2 */
#define TFSPH_PROF_FORCE   5  /* gas pressure (+ viscous) acceleration */
#define TFSPH_PROF_DRAG    6  /* implicit cell drag, particle update, next keys */
#define TFSPH_PROF_NPHASE  7

/* Create a context from a particle state (Sec. 2.3 set-up).
 *   gas[]:  2*dim arrays of n_gas values, x_0..x_{dim-1}, v_0..v_{dim-1},
 *           then, for TFSPH_EOS_ADIABATIC, the specific energy e.
 *   dust[]: 2*dim + 1 arrays of n_dust values, x.., u.., then t_stop (> 0).
 *   frozen: nullable, n_gas bytes; nonzero marks a wall particle that enters
 *           the SPH sums but never moves and takes no part in the drag.
 * Moving particles must lie in [lo, hi) on every axis. n_gas, n_dust may be
 * 0 and must be < 2^31. Errors: INVALID_ARG, NONFINITE, OUT_OF_DOMAIN, OOM,
 * CUDA. On error *out is NULL. */
int tfsph_init(tfsph_ctx **out, const tfsph_params *p,
               const void *const *gas, int64_t n_gas,
               const void *const *dust, int64_t n_dust,
               const uint8_t *frozen, int mem_kind);

/* Replace the whole particle state (same counts and layout as tfsph_init). */
int tfsph_set_state(tfsph_ctx *c, const void *const *gas, const void *const *dust,
                    const uint8_t *frozen, int mem_kind);

/* Use `stream` (a cudaStream_t, may be NULL for the default stream) for all
 * later work of this context. */
int tfsph_set_stream(tfsph_ctx *c, void *stream);

/* Advance the mixture by one step tau (> 0) under gravity g[3] (Eqs. 19-21):
 * bin both phases into cells, gas summation density and pressure force,
 * per-cell eps*, t*_stop and mean velocities, implicit drag, new velocities
 * and positions x' = x + tau v' (periodic axes wrapped).
 *   t_stop: nullable; n_dust new stopping times in id order (memory of
 *           mem_kind) replacing the resident ones from this step on.
 * Asynchronous: a bad value inside a device t_stop array is reported by the
 * next tfsph_sync / tfsph_fields as NONFINITE. */
int tfsph_step(tfsph_ctx *c, double tau, const void *t_stop, int mem_kind, const double g[3]);

/* Reverse-mode derivative of one tfsph_step taken from the context's current
 * state (the state is not changed), for the isothermal gas without
 * artificial viscosity (INVALID_ARG otherwise). It differentiates the step of
 * Eqs. 19-21 as computed here: the implicit cell drag and particle update,
 * the SPH pressure force and the summation density; cell membership is
 * piecewise constant and has no derivative.
 *   In:  lam_gx, lam_gv = dLoss/d(x', v') of the gas after the step,
 *        lam_dx, lam_du = dLoss/d(x', u') of the dust after the step.
 *   Out: lam_gx, lam_gv, lam_du overwritten with dLoss/d(x, v, u) before the
 *        step (lam_dx passes through unchanged: dust positions enter the step
 *        only through cell membership); lam_ts (n_dust) is ADDED
 *        dLoss/dt_stop of this step.
 * All arrays component-major in id order, of the context's precision, in
 * memory of mem_kind (host arrays are copied and the call synchronises).
 * Rolling out several steps: restore the state at the start of each step
 * (tfsph_set_state) and call this in reverse order, carrying the lambdas. */
int tfsph_step_adjoint(tfsph_ctx *c, double tau, const double g[3], void *lam_gx, void *lam_gv,
                       void *lam_dx, void *lam_du, void *lam_ts, int mem_kind);

/* Checkpoint / resume: a raw snapshot of the context's particle state
 * (positions, velocities, energies, stopping times, ids, in the library's
 * storage order), its step count, and the state's forward quantities (cell
 * ranges, gas densities and pressure accelerations, Eqs. 17-19), which
 * tfsph_save_state computes first if the context does not hold them yet.
 * Loading a snapshot leaves the context as a step finds it after binning,
 * density and force, so the next tfsph_step or tfsph_step_adjoint starts
 * from the update (this is what makes a checkpointed reverse pass cost one
 * force evaluation per step). tfsph_state_bytes gives the size; save and
 * load copy to/from a caller-owned buffer of mem_kind (device copies are
 * asynchronous on the context's stream, one kernel launch, and need a
 * 4-byte-aligned buffer; host copies synchronise). A snapshot
 * loads only into a context of the same counts, dimension, precision and
 * cell grid: INVALID_ARG from a host buffer; for a device buffer the header
 * is checked on the device and a mismatch is reported by the next
 * tfsph_sync (INTERNAL). Loading a device snapshot keeps the context's step
 * count. */
int tfsph_state_bytes(const tfsph_ctx *c, int64_t *bytes);
int tfsph_save_state(tfsph_ctx *c, void *buf, int mem_kind);
int tfsph_load_state(tfsph_ctx *c, const void *buf, int mem_kind);

/* Courant step (Eq. 4): *tau_out = cfl * h / max over moving gas of
 * max(|v_a|, c_a). Synchronises the stream. */
int tfsph_max_dt(tfsph_ctx *c, double cfl, double *tau_out);

/* Copy one field (TFSPH_FIELD_*) into `out` in the given order
 * (TFSPH_ORDER_*). Density fields are computed at the current positions.
 * Synchronises the stream when `out` is host memory. */
int tfsph_fields(tfsph_ctx *c, int field, void *out, int mem_kind, int order);

/* Debug exports (TFSPH_DEBUG_*), for tests. Synchronises for host output. */
int tfsph_debug(tfsph_ctx *c, int what, void *out, int mem_kind);

/* Sizes and counters of a context. */
int tfsph_info(const tfsph_ctx *c, tfsph_info_t *out);

/* Start (enable = 1, clearing the totals) or stop (0) timing the phases of
 * tfsph_step with CUDA events recorded on the context's stream. */
int tfsph_profile(tfsph_ctx *c, int enable);

/* Synchronise and read the accumulated time per phase (TFSPH_PROF_*, ms,
 * TFSPH_PROF_NPHASE doubles), the number of timed steps and the kernels
 * those steps launched. Any pointer may be NULL. */
int tfsph_profile_read(tfsph_ctx *c, double *ms, int64_t *steps, int64_t *launches);

/* Wait for the context's stream and report any error raised on the device
 * since the last call (NONFINITE for bad t_stop values, INTERNAL otherwise). */
int tfsph_sync(tfsph_ctx *c);

/* Message of the last error of `c` (or of the last failed tfsph_init when c
 * is NULL). The string lives until the next call on the same context. */
const char *tfsph_last_error(const tfsph_ctx *c);

/* Static name of a status code. */
const char *tfsph_status_string(int code);

/* Free the context and its device memory (NULL is allowed). */
void tfsph_destroy(tfsph_ctx *c);

/* Library version, major * 10000 + minor * 100 + patch. */
int tfsph_version(void);

/* ------------------------------------------------------------------------
 * Binned dust density and a squared-error loss on it, with the loss's
 * gradient: the loss of the differentiable rollout (tfsph_step_adjoint). The
 * paper's test problems compare profiles of the dust density (Sec. 3); this
 * is the cloud-in-cell form of such a profile.
 *   grid: nbins[k] bins of width D_k = (hi_k - lo_k)/nbins[k] on each axis
 *     k < dim (1 <= nbins[k] <= 65536, at most 2^26 bins), bin b = i_0 +
 *     nbins[0] (i_1 + nbins[1] i_2). A particle at x (s = (x - lo)/D - 1/2,
 *     i = floor(s), f = s - i per axis) adds mass * prod_k (1 - f_k or f_k)
 *     to the 2^dim bins (i_k or i_k + 1); periodic axes wrap the bin index,
 *     other axes clamp it to [0, nbins - 1]; rho_b = deposited mass / bin
 *     volume. NaN positions are skipped.
 *   x:      device positions of n particles, component-major (dim, n), of the
 *           spec's precision (as tfsph_fields exports them).
 *   rho:    device double[nbins] (caller-owned), the profile.
 *   target: device double[nbins] or NULL. With a target, loss (device double,
 *           or NULL) receives sum_b (rho_b - target_b)^2 and lam_x (device,
 *           (dim, n), spec precision, or NULL) is overwritten with d loss /
 *           d x (the derivative of the linear piece that holds x).
 *   stream: cudaStream_t (NULL = legacy default stream); asynchronous.
 * The deposit accumulates in binary64 with atomics, so the last bits of rho
 * may depend on the order of the particles' additions.
 * Errors: INVALID_ARG, CUDA; the message is in tfsph_last_error(NULL). */
typedef struct {
    int dim;
    double lo[3], hi[3];
    int periodic[3];
    int nbins[3];
    double mass;      /* mass of every particle */
    int precision;    /* TFSPH_FP32 or TFSPH_FP64: the type of x and lam_x */
} tfsph_grid_spec;

int tfsph_dust_profile(const tfsph_grid_spec *grid, const void *x, int64_t n, const void *target, void *rho,
                       void *loss, void *lam_x, void *stream);

/* Cell ranges of a set of cell keys, computed without allocating any device
 * memory. The paper has no counterpart: this is an entry point for callers
 * that cannot call cudaMalloc, such as applications whose device memory is
 * handed out by their own fixed pool, or loops that must not allocate (or
 * pay the device synchronisation an allocation can bring) once running.
 *   keys:   n device cell keys (uint32); keys >= n_cells are not counted.
 *   starts: n_cells + 1 device values (caller-owned). starts[c] is the
 *           number of counted keys below c, starts[n_cells] the number of
 *           counted keys; keys sorted ascending make [starts[c],
 *           starts[c+1]) the slots of cell c.
 *   stream: cudaStream_t (NULL = legacy default stream); asynchronous.
 * The scratch (2^21 cell counters and the scan's block totals, 8 MiB in all)
 * is one static device array that every GPU loading the library holds until
 * the process exits; n_cells above 2^21 is rejected with INVALID_ARG. The
 * first call on a device looks up that array's device address (with the
 * device current); make that first call before any stream capture. All calls
 * on a device share that device's array and each clears the counters it
 * uses first, so calls that overlap on the same GPU (on different streams)
 * race: order them on one stream. The device address is kept for the life
 * of the process: calls after cudaDeviceReset are not supported. A CUDA
 * error already pending when the call starts is returned as CUDA and left
 * pending. Errors: INVALID_ARG, CUDA; the message is in
 * tfsph_last_error(NULL). */
int tfsph_cell_ranges_noalloc(const uint32_t *keys, int64_t n, uint32_t n_cells, uint32_t *starts,
                              void *stream);

/* ------------------------------------------------------------------------
 * Batched ensembles: many independent instances of the step (Sec. 2.3) in
 * one context, each with its own box, particle counts, h, cell grid,
 * masses, sound speed, t_stop values, tau and g. All instances share dim,
 * tstar_mode and cell_acc, and the batch runs FP32 state (precision must be
 * TFSPH_FP32). Each instance computes exactly what a single context with
 * its parameters computes; only the order in which neighbour terms are
 * summed may differ (rounding).
 *
 * A step of the whole batch is replayed from a captured CUDA graph in one of
 * two launch forms:
 *   TFSPH_BATCH_PERSISTENT: one cooperative launch per step; its phases are
 *     separated by grid barriers whose waits are bounded (a wait that runs
 *     out makes the next tfsph_batch_sync return TFSPH_E_TIMEOUT; the
 *     context stays usable);
 *   TFSPH_BATCH_KERNELS: one launch per phase (the default); the gas pair
 *     sums walk each particle's candidate cells in global memory;
 *   TFSPH_BATCH_TILED: one launch per phase, and the gas pair sums stage the
 *     candidate cells of each chunk of CTA-size particles (a window of
 *     consecutive cells) in shared memory. 1D batches of isothermal gas
 *     without viscosity only (INVALID_ARG otherwise).
 * The CTA size (128, 256 or 512) is also the tile of the tiled form: the
 * number of consecutive particles whose window is staged together.
 * tfsph_batch_autotune times the forms and CTA sizes on the current state
 * (which it restores) and keeps the fastest.
 * ---------------------------------------------------------------------- */
typedef struct tfsph_batch tfsph_batch;

#define TFSPH_BATCH_KERNELS    0
#define TFSPH_BATCH_PERSISTENT 1
#define TFSPH_BATCH_TILED      2

typedef struct {
    int32_t n_inst, dim;
    int64_t n_gas, n_dust;   /* totals over the instances */
    int64_t n_cells;         /* total cells (instance grids concatenated) */
    int32_t mode;            /* TFSPH_BATCH_* */
    int32_t block;           /* threads per CTA */
    int32_t grid;            /* CTAs of the persistent launch (0 otherwise) */
    int32_t graph;           /* 1 when steps replay a captured CUDA graph */
    int64_t steps;           /* steps taken since init */
    int64_t launches;        /* kernel launches of those steps (graph kernel nodes count) */
    int64_t device_bytes;    /* device memory held */
} tfsph_batch_info_t;

/* Creates a batch of n_inst instances. params[i], n_gas[i], n_dust[i]
 * describe instance i (each is checked like tfsph_init's). gas and dust list
 * the same component arrays as tfsph_init, each holding every instance's
 * particles concatenated in instance order (instance i's gas occupies
 * [sum_{k<i} n_gas[k], sum_{k<=i} n_gas[k])); the energy array is present
 * when any instance is adiabatic. frozen (nullable) flags wall gas particles
 * in the same concatenated order. The particle ids of field exports follow
 * the concatenated order. Errors: INVALID_ARG, NONFINITE, OUT_OF_DOMAIN,
 * OOM, CUDA; the message is in tfsph_batch_last_error(NULL). */
int tfsph_batch_init(tfsph_batch **out, const tfsph_params *params, const int64_t *n_gas, const int64_t *n_dust,
                     int32_t n_inst, const void *const *gas, const void *const *dust, const uint8_t *frozen,
                     int mem_kind);

/* Work goes on this stream (cudaStream_t; NULL = legacy default stream). */
int tfsph_batch_set_stream(tfsph_batch *b, void *stream);

/* Advances every instance by nsteps steps. tau: n_inst host values (> 0),
 * required on the first call, NULL keeps the previous ones; g: 3 * n_inst
 * host values (instance-major, components beyond dim ignored), NULL keeps
 * the previous ones (initially 0). Asynchronous, except that a changed tau
 * or g is uploaded before the call returns. nsteps = 0 only sets tau, g. */
int tfsph_batch_step(tfsph_batch *b, const double *tau, const double *g, int32_t nsteps);

/* Selects the launch form: mode TFSPH_BATCH_*, block in {128, 256, 512}
 * threads per CTA, blocks_per_sm in [1, 16] (persistent form: CTAs per SM,
 * capped by what fits), barrier_timeout_ms >= 0 (how long a persistent grid
 * barrier waits before it gives up). */
int tfsph_batch_config(tfsph_batch *b, int32_t mode, int32_t block, int32_t blocks_per_sm, double barrier_timeout_ms);

/* Times every launch form for `steps` steps from the current state (after
 * one warm-up step each), restores the state and keeps the fastest; returns
 * its mode, block, blocks_per_sm and time per step (any output may be
 * NULL). Synchronises. tau must have been set. */
int tfsph_batch_autotune(tfsph_batch *b, int32_t steps, int32_t *mode, int32_t *block, int32_t *blocks_per_sm,
                         float *ms_per_step);

/* Copies one field of every instance, concatenated in instance order and
 * in input order inside each instance (TFSPH_FIELD_POS_G, VEL_G, ENERGY_G,
 * RHO_G, POS_D, VEL_D, TSTOP_D; RHO_G bins the current state first). Host
 * copies synchronise. */
int tfsph_batch_fields(tfsph_batch *b, int field, void *out, int mem_kind);

int tfsph_batch_info(const tfsph_batch *b, tfsph_batch_info_t *out);

/* Waits for the batch's work and reports device-side errors (TIMEOUT,
 * INTERNAL), clearing them. */
int tfsph_batch_sync(tfsph_batch *b);

/* Message of the last failed call on b (b = NULL: of the last failed
 * tfsph_batch_init on this thread). */
const char *tfsph_batch_last_error(const tfsph_batch *b);

void tfsph_batch_destroy(tfsph_batch *b);

#ifdef __cplusplus
}
#endif

#endif /* TFSPH_H */
