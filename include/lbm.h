/*
 * lbm.h -- C ABI of the GB300 (sm_103a) coupled multiphase lattice Boltzmann step.
 *
 * Method: Otomo et al., "Lattice Boltzmann models for the hydrodynamic equations
 * in multiphase flow with high density ratio" (arXiv 2512.01027), Sec. II:
 *   - phase-field LB for the conservative Allen-Cahn equation, populations h_i
 *     (Eq. LB_phi_filter_col, h_eq with Gamma_i, theta and the delta-theta
 *     correction);
 *   - hydrodynamic LB of the pressure P and velocity u, populations g_i, with the
 *     LKS-mapped moments (Eq. Kiterm and the P, u definitions), the equilibrium of
 *     Eq. BGK_LBeq_hydroeq (surface-tension force, density-gradient stress term,
 *     bulk term B) and the filter collision (Eqs. momentum_flux0/1, LB_filter_col).
 * One time step of lbm_step advances both populations at every site, by default
 * in two kernel launches (the split form: moments, then stencils and
 * collisions; see lbm_set_tuning for the fused and persistent forms).
 *
 * Conventions (all entry points):
 *   - Every function returns an int status: LBM_OK (0) or one of the LBM_ERR_*
 *     codes.  On error, lbm_last_error(handle) describes the failure.
 *   - A handle owns all device memory it allocates; the caller owns every host
 *     array it passes.  Host arrays are never retained after a call returns.
 *   - Grid: nx * ny * nz = N sites, x fastest, then y, then z.  2D lattices need
 *     nz == 1.  Host scalar fields are double[N]; host vector fields are
 *     double[3][N] (three component planes; the z plane is ignored on input and
 *     zero on output for 2D lattices).
 *   - Non-periodic axes are closed by solid sites just outside the grid.  Solid
 *     sites (grid.solid) are never updated; halfway bounce-back applies on every
 *     link into a solid site (paper: no-slip walls).
 *   - Work is enqueued on the handle's stream (default: the legacy default
 *     stream, or the stream set by lbm_set_stream).  Functions that return host
 *     data synchronise that stream.
 *   - There is no CPU fallback: without a usable CUDA device, lbm_create returns
 *     LBM_ERR_CUDA.
 *   - Not thread-safe per handle; distinct handles may be used from distinct
 *     threads.
 */
#ifndef LBM_GB300_H
#define LBM_GB300_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define LBM_ABI_VERSION 1

/* Status codes. */
#define LBM_OK 0
#define LBM_ERR_INVALID_ARG 1   /* bad pointer, size, enum or parameter value */
#define LBM_ERR_OOM 2           /* device allocation failed (cudaMalloc or the allocator hook) */
#define LBM_ERR_CUDA 3          /* a CUDA runtime call or kernel launch failed */
#define LBM_ERR_NONFINITE 4     /* a step produced a non-finite phi, P or u */
#define LBM_ERR_UNSUPPORTED 5   /* a valid request the library does not implement */
#define LBM_ERR_TIMEOUT 6       /* a bounded wait inside a kernel ran out; the step's results are invalid */

typedef struct lbm_ctx *lbm_handle;

/* Lattices (Sec. II: the paper uses D3Q19; D2Q9 and D3Q27 use the same
 * formulas with T = 1/3). */
typedef enum { LBM_D2Q9 = 0, LBM_D3Q19 = 1, LBM_D3Q27 = 2 } lbm_lattice;

/* Population storage.  F64: FP64 storage and arithmetic.  F32: FP32 storage
 * and arithmetic.  F16DEV / BF16DEV: populations stored in 16 bits as scaled
 * deviations from the lattice weights, collided in FP32; P and u in FP32. */
typedef enum {
    LBM_STORE_F64 = 0,
    LBM_STORE_F32 = 1,
    LBM_STORE_F16DEV = 2,
    LBM_STORE_BF16DEV = 3
} lbm_storage;

typedef struct {
    int32_t nx, ny, nz;       /* sites per axis (>= 1) */
    int32_t periodic[3];      /* 1: periodic axis; 0: closed by solid outside the grid */
    const uint8_t *solid;     /* host, N bytes (1 = solid) or NULL for no solid sites */
} lbm_grid;

/* Physical parameters (lattice units).  Defaults from Sec. II/III are given
 * by lbm_default_params.  struct_size must be sizeof(lbm_params). */
typedef struct {
    uint64_t struct_size;
    double rho_w;          /* heavy-phase density (phi = 1), rho_water */
    double rho_a;          /* light-phase density (phi = 0), rho_air = rho_ref */
    double nu_w, nu_a;     /* kinematic viscosities; tau_k = nu_k / T + 1/2 (Eq. tau_interpolate) */
    double sigma;          /* surface tension in the chemical potential mu */
    double M;              /* mobility; tau_phi = M / T + 1/2 (Eq. LB_phi_filter_col) */
    double W;              /* interface thickness */
    double lambda_b;       /* bulk viscosity (paper: 1/6) */
    double gamma, phi_n, phi_m, D, eps;   /* delta-theta constants (paper: -22.5, 0.8, 0.2, 1e-4, 1e-10) */
    double g_ext[3];       /* body acceleration; F_ext = rho * g_ext */
    int32_t clamp_phi_props;   /* 1: clamp phi to [0,1] for rho, tau_mix and omega (default) */
    int32_t filter_full_trace; /* 0: filter carries the trace-free part of Pi (default);
                                  1: the full Pi as printed (linearly unstable at low nu) */
    int32_t storage;           /* lbm_storage of the populations (default LBM_STORE_F32) */
    int32_t inplace;           /* 0: two population stores (ping-pong, default); 1: one store
                                  updated in place with the AA streaming pattern (half the
                                  population memory; steps run in the two-launch split form) */
    int32_t coupling_unew;     /* 0: the omega-term of the pressure formula (Sec. II) takes
                                  u^n(x - c_i), the previous step's velocity (default);
                                  1: u^{n+1}(x - c_i) of the same step, the alternative
                                  reading, linearly unstable at nu < 5e-3 (split form and
                                  batches only: the fused, persistent and cluster forms
                                  return LBM_ERR_UNSUPPORTED) */
} lbm_params;

/* Fill *p with the paper's defaults: rho_w = 1, rho_a = 1e-3, nu_w = 0.0167,
 * nu_a = 0.167, sigma = 1e-3, M = 0.166, W = 4, lambda_b = 1/6, gamma = -22.5,
 * phi_n = 0.8, phi_m = 0.2, D = 1e-4, eps = 1e-10, g_ext = 0, clamp on,
 * trace-free filter, FP32 storage. */
int lbm_default_params(lbm_params *p);

/* Direction table of a lattice, in the library's population order (rest
 * first, then pairs (c, -c)): c[3*i + a] and w[i] for i < Q.  Either output
 * may be NULL.  *d and *Q receive the dimension and the number of directions. */
int lbm_lattice_info(int lattice, int *d, int *Q, int *c, double *w);

/* Create a lattice state on the current CUDA device.  grid->solid is copied.
 * Returns LBM_ERR_INVALID_ARG for bad sizes/parameters (rho_a <= 0,
 * rho_w <= rho_a, nu <= 0, M <= 0, W <= 0), LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_create(const lbm_grid *grid, int lattice, const lbm_params *params, lbm_handle *out);

/* Release all device memory of h (after synchronising its stream). */
int lbm_destroy(lbm_handle h);

/* Stream for all later work of h (a cudaStream_t passed as void*; NULL = legacy default). */
int lbm_set_stream(lbm_handle h, void *cuda_stream);

/* Device-memory hooks used by later lbm_create calls in this process: alloc
 * returns a device pointer of at least `bytes` (256-byte aligned) or NULL;
 * free releases it.  Pass NULLs to restore cudaMalloc/cudaFree. */
typedef void *(*lbm_alloc_fn)(size_t bytes, void *ctx);
typedef void (*lbm_free_fn)(void *ptr, void *ctx);
int lbm_set_allocator(lbm_alloc_fn alloc, lbm_free_fn free_fn, void *ctx);

/* Initial state from host fields phi[N], P[N], u[3][N]: populations start at
 * equilibrium (Sec. I: "f_i in the initial condition is assumed to be the
 * equilibrium state"), h* = h_eq, g* = g_eq built from these fields and their
 * stencils; P^0 = P, u^0 = u.  Resets the step counter.  Returns after the
 * host arrays have been read (the caller may reuse them).
 *
 * Staging of the host-array calls (lbm_init_fields, lbm_read_fields,
 * lbm_get_state, lbm_probe): the data pass through a device buffer.  With no
 * allocator hook it comes from one stream-ordered memory pool per device that
 * keeps its memory for later calls of any handle on that device: it holds the
 * largest staging size used so far (40 B per site for the fields, 16 Q + 32 B
 * per site for lbm_get_state) until the process exits.  With a hook
 * (lbm_set_allocator) it comes from the hook and is released before the call
 * returns.  Neither is counted by lbm_footprint. */
int lbm_init_fields(lbm_handle h, const double *phi, const double *P, const double *u);

/* Same from device arrays (double, same layout) already on the handle's device. */
int lbm_init_fields_device(lbm_handle h, const double *d_phi, const double *d_P, const double *d_u);

/* Advance n >= 0 time steps (asynchronous on the handle's stream). */
int lbm_step(lbm_handle h, int64_t n);

/* Current fields into host arrays (any may be NULL): phi^n = sum_i h*_i,
 * P^n, u^n (double[3][N]); solid sites read 0.  Synchronises the stream and
 * returns LBM_ERR_NONFINITE if any step since lbm_init_fields produced a
 * non-finite value. */
int lbm_read_fields(lbm_handle h, double *phi, double *P, double *u);

/* Same into device double arrays (no synchronisation). */
int lbm_read_fields_device(lbm_handle h, double *d_phi, double *d_P, double *d_u);

/* Steps taken since the last lbm_init_fields / lbm_load_state. */
int lbm_steps_done(lbm_handle h, int64_t *steps);

/* Synchronise and report LBM_ERR_NONFINITE if a non-finite value was seen. */
int lbm_check(lbm_handle h);

/* FP64 global reductions over fluid sites (Sec. II: sum h_eq = phi makes sum
 * phi a conserved quantity): out[0] = sum phi, out[1..3] = sum rho(phi) u,
 * out[4] = number of fluid sites.  Synchronises the stream. */
int lbm_reduce(lbm_handle h, double out[5]);

/* Laplace pressure jump (Sec. III.A): mean P over fluid sites with
 * |x - center| < r_in minus mean P over fluid sites with |x - center| > r_out
 * (distances on the periodic grid; FP64 accumulation).  Synchronises. */
int lbm_pressure_jump(lbm_handle h, const double center[3], double r_in, double r_out, double *dP);

/* Decoded populations as double[Q][N] in the library's direction order
 * (lbm_lattice_info), plus P^n and u^n[3][N]; any pointer may be NULL.
 * Synchronises. */
int lbm_get_state(lbm_handle h, double *h_pop, double *g_pop, double *P, double *u);

/* State at n chosen sites (linear indices x + nx (y + ny z)): decoded
 * populations h_pop[n][Q], g_pop[n][Q], P[n] and u[n][3] as doubles, in the
 * library's direction order; any output may be NULL.  Solid sites hold no
 * state and read as zeros.  For probes (pressure sensors) and for sampled
 * checks of large lattices.  Synchronises. */
int lbm_probe(lbm_handle h, int64_t n, const int64_t *sites, double *h_pop, double *g_pop, double *P, double *u);

/* Checkpoint: a 40-byte header (lattice, storage, layout, grid), then the
 * raw state (populations in storage format and store layout, P, u, step
 * counter).  lbm_state_bytes gives the size; save/load copy through a host
 * buffer of exactly that size.  A state loads only into a handle of the same
 * lattice, grid, storage and layout (in-place or not); anything else is
 * LBM_ERR_INVALID_ARG and leaves the handle unchanged.
 * With BF16 storage the split form keeps part of g (its first-order odd
 * part) in FP32 beside the populations; saving a state first folds it into
 * the stored BF16 populations (one rounding), so the handle continues from
 * the saved state exactly as one that loads it.  Reading populations
 * (lbm_get_state, lbm_probe) adds that part on the fly and changes nothing. */
int lbm_state_bytes(lbm_handle h, size_t *bytes);
int lbm_save_state(lbm_handle h, void *host_buf, size_t bytes);
int lbm_load_state(lbm_handle h, const void *host_buf, size_t bytes);

/* Launch tuning of the step (used by the autotuner).  variant: 0 =
 * automatic (the split form), 1 = fused plane-synchronous kernel, 2 = fused
 * pipelined kernel (3D lattices with 4-byte populations, else
 * LBM_ERR_UNSUPPORTED), 3 = split form (two launches per step: moments, then
 * stencils + collisions), 4 = persistent split form (both phases in one
 * launch per step: blocks take plane-ordered work items so that the
 * collision of a plane follows the moments of the next one while their data
 * is in L2; FP32 arithmetic and Q x sites < 2^32, else LBM_ERR_UNSUPPORTED),
 * 5 = cluster step (one launch per step: a CTA owns one row of sites and
 * marches in z, a thread-block cluster of CTAs on consecutive rows shares
 * the moments of each plane through distributed shared memory, so the
 * moments reach the stencils without passing through HBM; 3D lattices,
 * ping-pong store, nx a multiple of 32 and at most 256, ny a multiple of
 * the cluster rows (lbm_set_cluster), 2 nx a multiple of 32 x rows,
 * Q x sites < 2^32, FP64, FP32 or FP16 storage; else LBM_ERR_UNSUPPORTED).
 * An in-place handle always uses a split form (variants 1 and 2 are
 * LBM_ERR_UNSUPPORTED there).  zchunk: z planes per
 * block of the fused kernels and per CTA of the cluster step (0 =
 * automatic); it never changes results.
 * Every variant evaluates the same formulas in the same order: with FP64
 * storage (built without FMA contraction) all variants agree bit for bit;
 * with FP32 arithmetic the compiler may contract a product and a sum into
 * one FMA differently in different kernels, so variants agree to rounding. */
int lbm_set_tuning(lbm_handle h, int variant, int zchunk);

/* Shape of the cluster step (variant 5).  rows: CTAs per thread-block
 * cluster, one of 2, 4, 8, 16, or 0 for automatic (the largest the lattice
 * fits, 16 only where the device allows clusters of that non-portable
 * size).  staged: with FP32 arithmetic (FP32 or FP16 storage), 1 stages
 * the population rows each plane pulls in shared memory by bulk asynchronous
 * copies two planes ahead; 0 or -1 (default) reads them from the store (on
 * GB300 the staged form, one CTA per SM for its shared memory, was the
 * slower one).
 * Neither changes results.  LBM_ERR_INVALID_ARG for other values,
 * LBM_ERR_UNSUPPORTED when the lattice does not meet the cluster step's
 * requirements with that many rows. */
int lbm_set_cluster(lbm_handle h, int rows, int staged);

/* Testing aid for the failure path of the persistent split step (variant
 * 4): while set, its moments launch leaves the z-plane `plane` uncounted, so
 * the collisions that need that plane wait until their bounded wait runs out
 * (1 s on the GPU's timer); the step then ends, its results are invalid, and
 * lbm_check / lbm_read_fields report LBM_ERR_TIMEOUT.  The handle stays
 * usable: clear the aid (plane < 0) and initialise it again.  plane >= nz is
 * LBM_ERR_INVALID_ARG.  No other variant looks at it. */
int lbm_debug_stall(lbm_handle h, int plane);

/* Device bytes held by h, and the bytes one step reads and writes at minimum
 * (algorithmic traffic: both population sets in and out, P and u in and out). */
int lbm_footprint(lbm_handle h, size_t *device_bytes, size_t *step_bytes);

/* Device bytes lbm_create would hold for (grid, lattice, params), computed
 * on the host without a device and without allocating: for admission
 * control (a server admits a lattice when its footprint fits in free HBM).
 * Equals lbm_footprint's device_bytes of the created handle. */
int lbm_estimate_footprint(const lbm_grid *grid, int lattice, const lbm_params *params, size_t *device_bytes);

/* Allocation-free FP64 sums of caller-owned device fields; the paper has no
 * counterpart (it is a service for callers, not a step of the method).
 * For callers that cannot allocate device memory where they need the sums:
 * real-time loops that must not block in an allocator (cudaMalloc and
 * cudaFree can synchronise the device), and hosts whose device memory
 * belongs to a pool they do not own, where an allocation of the library's
 * own would escape the pool's accounting.
 * Inputs: d_phi[n], d_u[3][n] (device doubles, e.g. from
 * lbm_read_fields_device), d_solid[n] (device bytes, 1 = solid, or NULL),
 * rho_w > rho_a > 0 and clamp_phi_props as in lbm_params.  Output: d_out[5]
 * (device doubles) = sum phi, sum rho(phi) u (3 components), fluid sites,
 * summed over non-solid sites in the same order as lbm_reduce, so with
 * FP64 storage the two agree bit for bit.  Enqueued on `stream` (a
 * cudaStream_t, NULL = legacy default); no synchronisation.
 * No cudaMalloc, cudaFree or allocating library call is made: the per-block
 * partial sums live in one fixed 40 KB array (1024 blocks x 5 doubles) in
 * device global memory that every GPU loading this library holds until the
 * process exits.  Limit: 1 <= n <= 2^31 - 1 sites; larger n (or n <= 0)
 * returns LBM_ERR_INVALID_ARG, as do NULL d_phi, d_u or d_out and densities
 * other than rho_w > rho_a > 0.  The first call with a given device current
 * looks up the array's device address (cudaGetSymbolAddress) and caches it
 * for as long as that device's context lives (after cudaDeviceReset the
 * library must be loaded again).  All calls share the array and it keeps the last call's contents
 * (each call overwrites every partial it reads, so nothing needs clearing);
 * calls that overlap on the GPU (different streams, or different host
 * threads) race on it.  LBM_ERR_CUDA when a launch fails; the error state
 * of the calling thread is read without clearing it, so an error pending
 * from earlier work is reported too and stays pending for the caller. */
int lbm_reduce_fields_noalloc(const double *d_phi, const double *d_u, const uint8_t *d_solid, int64_t n,
                              double rho_w, double rho_a, int32_t clamp_phi_props, double *d_out, void *stream);

/* Description of the last error on h (or of the last lbm_create failure when
 * h is NULL).  Never NULL. */
const char *lbm_last_error(lbm_handle h);

/* ------------------------------------------------------------------------
 * Autotuner.  Times `trial_steps` steps of every launch form the handle
 * supports (split form; persistent split form; fused plane-synchronous
 * kernel; fused pipelined kernel at several z-chunks; cluster step with
 * clusters of 4, 8 and 16 rows, staged or not, where available) on the
 * handle's own state,
 * keeps the fastest with lbm_set_tuning and restores the state it started
 * from (through a host copy of lbm_state_bytes bytes), so the results of the
 * following steps are those of the chosen variant from the same state.
 * Outputs (any may be NULL): the chosen variant and zchunk and its measured
 * milliseconds per step.  An in-place handle tries the split forms only.
 * Synchronises; 1 <= trial_steps <= 1000. */
int lbm_autotune(lbm_handle h, int trial_steps, int *variant, int *zchunk, double *ms_per_step);

/* ------------------------------------------------------------------------
 * Batches: many independent lattices advanced together, two kernel launches
 * per time step for the whole set (no per-lattice launches), on a
 * persistent grid.  Work items are blocks of consecutive sites of one
 * member; a device table lists the members, so one CUDA graph of `chunk`
 * steps, captured once, serves any membership.  Members are ordinary
 * handles (their own grid, parameters, walls, storage layout and state),
 * created with lbm_create and initialised as usual, all of the batch's
 * lattice and storage.  Each member carries a step budget; a batch step
 * advances every member by min(n, its remaining budget).  The per-site
 * arithmetic is the split form's, so a member's results do not depend on
 * which other lattices share the batch.
 *
 * While in a batch, lbm_step on the member returns LBM_ERR_INVALID_ARG;
 * reading, probing, reductions and checkpoints work as usual (call them
 * between batch steps).  lbm_destroy of a member removes it from its batch. */
typedef struct lbm_batch_ctx *lbm_batch;

/* A batch for lattices of one DdQq and storage, on the current device, with
 * its own non-blocking stream. */
int lbm_batch_create(int lattice, int storage, lbm_batch *out);

/* Detaches every member (the handles stay valid) and frees the batch. */
int lbm_batch_destroy(lbm_batch b);

/* Stream of the batch's work (a cudaStream_t, not the legacy default
 * stream: graphs need a capturable stream).  NULL restores the own stream. */
int lbm_batch_set_stream(lbm_batch b, void *stream);

/* chunk: steps per graph launch, 1..64 (default 16); use_graph: 0 launches
 * the kernels one by one (same results). */
int lbm_batch_set_tuning(lbm_batch b, int chunk, int use_graph);

/* Launch shape of the batch kernels: span = consecutive blocks of 128 sites
 * (one thread a site) that one work item covers, 1..16 (default 1; a longer
 * item pays the member lookup and the load of the member's arguments once
 * for more sites, a shorter one spreads small members over more blocks);
 * blocks_per_sm = persistent blocks per SM, 0 (default: as many as fit) to
 * 32 (capped at what fits).  Neither changes results. */
int lbm_batch_set_shape(lbm_batch b, int span, int blocks_per_sm);

/* Autotuner of the batch: times `trial_steps` steps (rounded up to whole
 * chunks) of the current members for each launch shape it tries (chunk 8,
 * 16, 32; span 1, 2, 4, 8; all resident blocks or one block per SM fewer),
 * keeps the fastest (lbm_batch_set_tuning / lbm_batch_set_shape), then
 * restores every member's state (through host copies of lbm_state_bytes
 * bytes, as lbm_autotune does) and its step budget, so the following steps
 * give the results they would have given without the trials.  Outputs (any
 * may be NULL): the chosen chunk, span, blocks per SM and the measured
 * milliseconds per step.  LBM_ERR_INVALID_ARG for an empty batch or
 * trial_steps outside 1..1000.  Synchronises. */
int lbm_batch_autotune(lbm_batch b, int trial_steps, int *chunk, int *span, int *blocks_per_sm,
                       double *ms_per_step);

/* Adds h with a budget of `steps` steps (>= 0).  h must match the batch's
 * lattice and storage and belong to no other batch (else
 * LBM_ERR_INVALID_ARG); members index their populations in 32 bits, so
 * Q x sites must stay below 2^32 (else LBM_ERR_UNSUPPORTED). */
int lbm_batch_add(lbm_batch b, lbm_handle h, int64_t steps);

/* Removes h (its state stays as the last completed step left it). */
int lbm_batch_remove(lbm_batch b, lbm_handle h);

/* Advances every member by min(n, remaining budget) steps (n >= 0), chunk by
 * chunk, and returns when the GPU work is done.  *finished (may be NULL):
 * members whose budget is now 0. */
int lbm_batch_step(lbm_batch b, int64_t n, int *finished);

/* Remaining budget of member h. */
int lbm_batch_remaining(lbm_batch b, lbm_handle h, int64_t *steps_left);

/* Pauses (paused = 1) or resumes (0) member h: a paused member takes no
 * steps in lbm_batch_step and keeps its budget, its state and its device
 * memory; the others step as before.  A serving loop uses it to give the
 * GPU to the members with the least work left.  Members join unpaused.
 * LBM_ERR_INVALID_ARG if h is not a member or paused is not 0 or 1. */
int lbm_batch_pause(lbm_batch b, lbm_handle h, int32_t paused);

/* Members and kernel launches issued so far (either may be NULL). */
int lbm_batch_info(lbm_batch b, int *members, int64_t *launches);

/* Description of the batch's last error.  Never NULL. */
const char *lbm_batch_last_error(lbm_batch b);

#ifdef __cplusplus
}
#endif

#endif /* LBM_GB300_H */
