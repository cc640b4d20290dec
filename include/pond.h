/*
 * pond.h -- C ABI of libpond: the GB300 (sm_103a) time step of the two-population
 * "Particles on Demand" (PonD) kinetic model of a van der Waals fluid
 * (Reyhanian, Dorschner & Karlin, "Thermokinetic model of compressible multiphase
 * flows", arXiv:2002.09217).
 *
 * One time step per node (all on the GPU, no CPU fallback):
 *   1. frame search: predictor = the node's previous gauge lambda = (theta, u);
 *      corrector = re-stream with theta = max(p, p_floor)/(rho T_L) and u from the
 *      streamed moments (shifted velocities v_i = sqrt(theta) c_i + u, Eq. particle
 *      velocity) until the relative change is <= tol or max_iter streams were done;
 *   2. semi-Lagrangian streaming of f and g from x - v_i dt (Eqs. f/g streaming):
 *      each stencil neighbour's populations are carried into the arrival gauge by the
 *      moment-matching transfer matrix (SM "Transfer matrix") and combined with the
 *      4x4 cubic Lagrange stencil (SM "Reconstruction");
 *   3. moments rho, rho u, 2 rho E (moments Eq.), e -> T by the vdW energy
 *      e = C_v T - a rho, and the BGK collision of f and g with the Korteweg force
 *      source S_i, the heat-flux correction and the forced g equilibrium
 *      (Eqs. f/g collision, S-i, korteweg, gtilde, new geq).
 * The non-local terms (force F = -div K, interface energy, heat-flux source M_0)
 * use the previous step's density and temperature.
 *
 * Conventions
 *   - Lattices (the model holds for any tensor lattice C1 x C1, W_i = W_jx W_jy,
 *     T_L = sum W c^2; SM "Equilibrium"):
 *       POND_D2Q9 (the paper's): C1 = {-1, 0, 1}, population index i = 3*(cy+1) + (cx+1),
 *         W_0 = 2/3, W_+-1 = 1/6, T_L = 1/3;
 *       POND_D3Q27 (three dimensions, D = 3 in the energy equilibrium and the heat-flux
 *         correction): C1^3 with C1 = {-1, 0, 1}, index i = 9*(cz+1) + 3*(cy+1) + (cx+1),
 *         W = product of 1/6, 2/3, 1/6, T_L = 1/3; the 4x4x4 cubic stencil;
 *       POND_D2Q16: C1 = the roots -+sqrt(3 +- sqrt 6) of He_4(c) = c^4 - 6 c^2 + 3 in
 *         increasing order, index i = 4*jy + jx, Gauss-Hermite weights (3 - sqrt 6)/12
 *         (outer) and (3 + sqrt 6)/12 (inner), T_L = 1; the transfer map is the product
 *         of two 4-node Lagrange maps.  Q = 9 or 16 populations per family.
 *     The non-local terms use the isotropic D2Q9 difference stencils on the grid with
 *     either lattice.
 *   - Grids are nx * ny nodes, Delta x = 1, row-major with x fastest: node = y*nx + x.
 *   - Host arrays are always caller-owned; they are read or written during the call
 *     only.  Device memory is owned by the context; it is taken from the caller's
 *     allocator callbacks when given (e.g. PyTorch's caching allocator), else from
 *     cudaMalloc.
 *   - All work is enqueued on the context's stream (opts.stream, NULL = the legacy
 *     default stream).  Calls that return host data synchronise that stream.
 *   - Errors are returned as pond_status; pond_last_error() gives a message.  Device
 *     conditions (non-converged frame search, pressure floor hit, NaN) are counted on
 *     the device (pond_stats() reads the counts) and raised as sticky flags that the
 *     synchronising calls pond_moments, pond_moments3 and pond_conservation return as
 *     their status: POND_ETIMEOUT if a bounded device wait ran out, else
 *     POND_ENAN while the state holds non-finite values, else POND_ENONCONV, else
 *     POND_ETHETA for conditions that occurred since the previous report.  ENONCONV and ETHETA are warnings: the call has completed and its
 *     outputs are written; the report clears both flags.  There is no CPU fallback: a
 *     missing or unusable GPU is POND_ECUDA.
 *   - A context is not thread safe; distinct contexts may be used concurrently.
 */
#ifndef POND_H
#define POND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct pond_ctx pond_ctx;
typedef struct pond_batch pond_batch;

typedef enum {
    POND_OK = 0,
    POND_EINVAL = 1,    /* invalid argument or parameter out of range             */
    POND_ENOMEM = 2,    /* device allocation failed                               */
    POND_ECUDA = 3,     /* CUDA runtime error (message in pond_last_error)         */
    POND_ENONCONV = 4,  /* warning: a frame search hit max_iter since the last
                           report (sticky flag; outputs are still written)         */
    POND_ETHETA = 5,    /* warning: the pressure floor was hit since the last
                           report (sticky flag; outputs are still written)         */
    POND_ENAN = 6,      /* a NaN/Inf appeared in the state (see pond_stats)        */
    POND_ETIMEOUT = 7   /* a bounded wait of the D2Q9 step for a tile's staging
                           copies (TMA) ran out: the tile was skipped, the state
                           is incomplete (sticky, reported at the sync points)     */
} pond_status;

enum { POND_PERIODIC = 0, POND_ZEROGRAD = 1 };     /* boundary per axis               */
enum { POND_D2Q9 = 0, POND_D2Q16 = 1, POND_D3Q27 = 2 };   /* lattice                  */
enum { POND_VDW = 0, POND_IDEAL = 1, POND_DIETERICI = 2, POND_SIMPLIFIED = 3 };   /* see pond_eos */
enum { POND_FP64 = 0, POND_MIXED = 1 };            /* arithmetic / storage form       */
enum { POND_NONLOCAL_LAGGED = 0, POND_NONLOCAL_CURRENT = 1 };   /* see pond_opts.nonlocal */

/* Grid: nx, ny >= 1; bc_x, bc_y, bc_z: POND_PERIODIC, or POND_ZEROGRAD (index clamp).
 * nz: nodes along z, >= 1 on POND_D3Q27 (node = (z*ny + y)*nx + x), 0 or 1 on the
 * two-dimensional lattices; bc_z is read on D3Q27 only. */
typedef struct { int32_t nx, ny; int32_t bc_x, bc_y; int32_t nz, bc_z; } pond_grid;

typedef struct { int32_t kind; } pond_lattice;     /* kind = POND_D2Q9, D2Q16 or D3Q27 */

/* Equation of state.  POND_VDW: van der Waals p = rho R T/(1 - b rho) - a rho^2 with
 * e = (R/delta) T - a rho (main text; SM "Thermodynamics"); 0 < delta <= 2/3.
 * POND_IDEAL: the same with a = b = 0 forced.  POND_DIETERICI: p = rho R T/(1 - b rho)
 * exp(-a rho/(R T)) (SM "Coexistence curve").  POND_SIMPLIFIED: the near-critical
 * double well of the SM's speed-of-sound study, p = p0 + rho E0' - E0 with
 * E0 = beta (rho - rho_l)^2 (rho - rho_v)^2 (fields beta, rho_l, rho_v, p0; p0 > 0 is a
 * background pressure the printed form lacks, which keeps theta = p/(rho T_L) positive).
 * Neither has a closed caloric equation here, so both require isothermal = 1.
 * isothermal = 1 holds T at T_iso > 0 everywhere (the SM's isothermal runs): the gauge
 * temperature comes from p(rho, T_iso) and the energy population then plays no part in
 * the flow; the initial T field should equal T_iso. */
typedef struct {
    int32_t kind;
    double a, b, R, delta;
    int32_t isothermal;
    double T_iso;
    double beta, rho_l, rho_v, p0;
} pond_eos;

/* Options.  precision: POND_FP64 (all FP64) or POND_MIXED (FP32 populations and
 * streaming/collision arithmetic; e->T, EoS and the conserved sums in float-float, i.e.
 * pairs of FP32 values carrying ~48 bits; the storage-rounding remainders of mass,
 * momentum and energy kept beside each node).
 * dt: time step (Delta x = 1), 0 < dt <= 1.  tol / max_iter: frame search stop rule.
 * k_cond: conductivity; < 0 selects k = mu (C_v + R), mu = (tau - 1/2) P dt.
 * p_floor: pressure floor of the gauge temperature theta = max(p, p_floor)/(rho T_L).
 * stream: a cudaStream_t (NULL = default stream).
 * dalloc/dfree/alloc_ctx: optional device allocator (both or neither).
 * lanes_per_node: threads cooperating on one node in the step kernel, 8 or 16 (0 = 8).
 * tile_x: width of the step kernel's tile of 16 nodes, 1, 2, 4, 8 or 16 (tile height
 * 16 / tile_x; 0 = 16 for grids of fewer than 4 rows, else 4).  Both are performance
 * knobs (autotuning) of the D2Q9 kernel; results are the same to rounding.  The D2Q16
 * kernel (one thread per node) ignores them.
 * In the mixed form on D2Q16 the moments, e->T, EoS and frame-search residual are FP64;
 * the storage-rounding remainders of mass, momentum and energy are kept beside each
 * node as on D2Q9.
 * nonlocal: time level of the Korteweg force, interface energy and heat-flux source,
 * which the paper leaves open.  POND_NONLOCAL_LAGGED (0): from rho, T at t - dt (one
 * launch per step).  POND_NONLOCAL_CURRENT (1): two passes per step, the first a lagged
 * step predicting rho, T at t, the second the step redone from the same state with the
 * terms of that prediction; it holds a third state buffer, and such a context cannot join
 * a batch. */
typedef struct {
    int32_t precision;
    int32_t max_iter;
    double tol;
    double dt;
    double k_cond;
    double p_floor;
    void *stream;
    void *(*dalloc)(size_t bytes, void *alloc_ctx);
    void (*dfree)(void *ptr, void *alloc_ctx);
    void *alloc_ctx;
    int32_t lanes_per_node;
    int32_t tile_x;
    int32_t nonlocal;
} pond_opts;

/* Device counters accumulated since the last pond_stats() call that reset them. */
typedef struct {
    int64_t steps;         /* time steps taken by this context                  */
    int64_t node_updates;  /* nx*ny*steps                                       */
    int64_t streams;       /* streaming passes (frame-search iterations) summed */
    int64_t nonconverged;  /* node updates whose frame search hit max_iter      */
    int64_t clamped;       /* node updates with p < p_floor                     */
    int64_t nonfinite;     /* node updates that produced NaN/Inf                */
    int64_t stalled;       /* mixed form: frame searches stopped at the FP32
                              rounding floor (residual no longer halving)      */
    int64_t block_streams; /* streaming passes summed over kernel blocks (a block
                              of 32 nodes streams until all its nodes stop)    */
    int64_t max_streams;   /* largest streaming-pass count of any block        */
    int64_t timeouts;      /* tiles skipped because a bounded wait for their
                              staging copies ran out (reported as POND_ETIMEOUT) */
    int64_t region_nodes;  /* stencil-region nodes carried into the arrival gauge,
                              summed over streams (the union of a node's 4x4
                              (4x4x4) departure stencils: 16..64 per stream on
                              D2Q9, 16..36 on D2Q16, 64..216 on D3Q27, less the
                              node's own entry in a first stream)              */
    int64_t pair_streams;  /* streams of regions wider than 8 nodes (D2Q9) or 6
                              nodes (D2Q16, D3Q27), which take the per-direction,
                              per-stencil-node path                            */
} pond_stats_t;

/* Create a context and allocate its device state (two state buffers holding one record
 * per node, 32 values on D2Q9 and 44 on D2Q16, in FP32 or FP64; a 5-plane FP64 staging
 * buffer and reduction partials; on D2Q16 also 9 FP64 planes of non-local terms).
 * lattice: POND_D2Q9 or POND_D2Q16 (else POND_EINVAL).  kappa >= 0: Korteweg coefficient
 * (Eq. korteweg); tau > 1/2: BGK relaxation time, omega = 1/tau.  On success *out owns
 * the context. */
pond_status pond_create(const pond_grid *grid, const pond_lattice *lattice, const pond_eos *eos,
                        double kappa, double tau, const pond_opts *opts, pond_ctx **out);

/* Equilibrium initial state from host fields rho, ux, uy, T (nx*ny doubles each):
 * f_i = rho W_i, g_i = the co-moving g equilibrium (Eq. geq) including the interface
 * energy kappa |grad rho|^2 / 2, gauge theta = max(p, p_floor)/(rho T_L).
 * Requires rho > 0, b rho < 1, T > 0 everywhere (POND_EINVAL otherwise). */
pond_status pond_init_fields(pond_ctx *ctx, const double *rho, const double *ux,
                             const double *uy, const double *T);

/* Same with a z velocity (D3Q27; nx*ny*nz doubles each, host arrays).  On the
 * two-dimensional lattices uz is ignored; pond_init_fields and the device form take
 * u_z = 0. */
pond_status pond_init_fields3(pond_ctx *ctx, const double *rho, const double *ux, const double *uy,
                              const double *uz, const double *T);

/* Same with device pointers (nx*ny doubles each, read on the context stream). */
pond_status pond_init_fields_device(pond_ctx *ctx, const double *d_rho, const double *d_ux,
                                    const double *d_uy, const double *d_T);

/* Advance n >= 0 time steps (asynchronous on the context stream). */
pond_status pond_step(pond_ctx *ctx, int64_t n);

/* Macroscopic fields to host arrays (nx*ny doubles each, NULL skips a field):
 * rho, fluid velocity uhat = u + F dt/(2 rho), T, p (vdW EoS).  Synchronises.
 * Returns the sticky device flags (POND_ENONCONV, POND_ETHETA, POND_ENAN, see the
 * conventions above); with ENONCONV or ETHETA the fields are written. */
pond_status pond_moments(pond_ctx *ctx, double *rho, double *ux, double *uy, double *T,
                         double *p);

/* With the z component of uhat (zero on the two-dimensional lattices); host arrays of
 * nx*ny*nz doubles, NULL skips a field.  Synchronises; returns the sticky device flags
 * as pond_moments does. */
pond_status pond_moments3(pond_ctx *ctx, double *rho, double *ux, double *uy, double *uz, double *T,
                          double *p);

/* Same into device arrays (asynchronous, so it reports no device flags; no u_z). */
pond_status pond_moments_device(pond_ctx *ctx, double *d_rho, double *d_ux, double *d_uy,
                                double *d_T, double *d_p);

/* Global sums in FP64 with compensated summation: out = {sum rho, sum rho uhat_x,
 * sum rho uhat_y, sum_nodes sum_i g_i / 2 (total energy)}, the kept FP32 energy
 * remainders included; on D3Q27 the z momentum is not among them.  Synchronises;
 * returns the sticky device flags as pond_moments does (out is written with ENONCONV or
 * ETHETA). */
pond_status pond_conservation(pond_ctx *ctx, double out[4]);

/* Full state as 2Q + 7 host planes of nx*ny doubles (25 on D2Q9, 39 on D2Q16):
 * f_0..f_(Q-1), g_0..g_(Q-1), theta, u_x, u_y (the gauge the populations are stored in),
 * rho, T, uhat_x, uhat_y; on D3Q27 63 planes of nx*ny*nz doubles: f, g, theta, u_x, u_y,
 * u_z, rho, T, uhat_x, uhat_y, uhat_z (its FP32 remainders folded in as on D2Q16, the
 * momentum part as W_i c_i . J / (sqrt(theta) T_L)).
 * pond_get_state synchronises; pond_set_state replaces the current state.  In the mixed
 * form the library keeps, beside each node's FP32 populations, what storage rounding
 * took from mass, energy and momentum: f_4 and g_4 are exchanged with it (as doubles;
 * set_state splits them again), the momentum part (below one FP32 ulp of the
 * populations) is not exchanged and set_state clears it.  On D2Q16 (mixed) all four
 * remainders are exchanged folded into the populations (mass and momentum as
 * W_i (m + (c_ix J_x + c_iy J_y)/sqrt(theta)) on f, energy as W_i G on g) and set_state
 * recovers them from what the FP32 populations leave out. */
pond_status pond_get_state(pond_ctx *ctx, double *state);
pond_status pond_set_state(pond_ctx *ctx, const double *state);

/* One time step (its launches: the fused step kernel on D2Q9; the two non-local kernels
 * and the node step on D2Q16) bracketed by CUDA events on the
 * context stream; *ms_out = its duration in milliseconds.  Synchronises (a tracing
 * aid; pond_step is the fast path). */
pond_status pond_step_timed(pond_ctx *ctx, double *ms_out);

/* Read (and, if reset != 0, zero) the device counters.  Synchronises.  Returns
 * POND_ENAN while the counters hold non-finite node updates, else POND_OK; a reset also
 * clears the sticky flags. */
pond_status pond_stats(pond_ctx *ctx, pond_stats_t *out, int32_t reset);

/* Conservation sums without any allocation, for callers that cannot allocate device
 * memory themselves or through the library: code running where cudaMalloc is not
 * allowed, such as inside a region whose memory budget is fixed up front, or a host
 * that hands the library only pre-placed buffers.  The paper has no counterpart; this
 * is a service of the library.
 *
 * d_planes: device pointer to a D2Q9 state in the 25-plane FP64 layout of pond_get_state
 * (plane p of node n at p*n_nodes + n), caller-owned and only read.  Only D2Q9 states
 * are summed correctly: the plane indices of the D2Q16 (39) and D3Q27 (63) layouts
 * differ, and the library cannot tell them apart from the pointer.  The pointer and
 * n_nodes are not checked against the allocation either (the C ABI cannot see it): the
 * caller must pass at least 25 * n_nodes doubles on the current device.  out: host array of
 * 4 doubles {sum rho, sum rho uhat_x, sum rho uhat_y, sum_nodes sum_i g_i / 2}, summed in
 * FP64 with compensated summation as pond_conservation does.  stream: cudaStream_t of
 * the work (NULL = default stream); the call synchronises it before returning.
 *
 * Scratch: the block partials live in a file-scope device array of the library
 * (32,776 doubles, 256 KiB, held on every device that loads the library until the
 * process exits), so n_nodes may be at most 8,388,608; larger n_nodes, n_nodes < 1 or
 * NULL pointers return POND_EINVAL.  The array's device address is looked up on the
 * first call on each device (that call should come before any stream capture) and
 * kept for the life of the process, which assumes the device's primary context is not
 * reset (cudaDeviceReset) in between.  All
 * calls share the one array: calls that overlap on the GPU (different streams, threads
 * or processes sharing a context) race on it; every slot a call reads it has written
 * itself first.  Returns POND_ECUDA on a CUDA error. */
pond_status pond_conservation_noalloc(const double *d_planes, int64_t n_nodes, double out[4],
                                      void *stream);

/* Bytes of device memory the context holds (state + scratch). */
size_t pond_device_bytes(const pond_ctx *ctx);

/* Destroy the context and release its device memory (NULL is a no-op). */
void pond_destroy(pond_ctx *ctx);

/* Last error message of the context (never NULL; "" after success). */
const char *pond_last_error(const pond_ctx *ctx);

/* ---- Batches: many simulations advanced together -------------------------------
 * A batch steps all its D2Q9 contexts with one launch of the step kernel per time step
 * and per group of contexts that share precision and lanes_per_node; the launch walks a
 * device work-list of (context, tile) pairs, so contexts of different grid sizes and
 * parameters share it.  D2Q16 contexts are stepped by their own three launches on the
 * batch stream.  Two consecutive steps of the whole batch are captured once in a CUDA
 * graph (when the batch stream is not the legacy default stream) and replayed.
 * Per-node arithmetic does not depend on the batch: a context gives the same result
 * stepped alone or in any batch.  The paper has no counterpart (serving layer).
 *
 * stream: cudaStream_t of the batch's work (NULL = legacy default stream, no graphs).
 * Contexts keep their own streams for everything else; calls on a batched context
 * wait for the batch's work first.  pond_step on a batched context is POND_EINVAL. */
pond_status pond_batch_create(void *stream, pond_batch **out);

/* Add an initialised context (same device); waits for the context's queued work.  A
 * two-pass (current-time) context and a D3Q27 context are POND_EINVAL. */
pond_status pond_batch_add(pond_batch *batch, pond_ctx *ctx);

/* Remove a context (waits for the batch's work); the context may be stepped alone again. */
pond_status pond_batch_remove(pond_batch *batch, pond_ctx *ctx);

/* Advance every context of the batch by n >= 0 steps (asynchronous on the batch stream). */
pond_status pond_batch_step(pond_batch *batch, int64_t n);

/* Number of contexts in the batch. */
int32_t pond_batch_size(const pond_batch *batch);

/* Admission by device memory: pond_batch_add refuses (POND_ENOMEM, the context stays
 * valid and outside the batch) a context whose pond_device_bytes would take the sum over
 * the members above `bytes`, unless the batch is empty (a lone member may exceed the
 * budget, so that no context is refused for ever); 0 (the default) sets no limit.  A
 * budget below what the members already hold is POND_EINVAL. */
pond_status pond_batch_set_budget(pond_batch *batch, size_t bytes);

/* Sum of pond_device_bytes over the batch's members. */
size_t pond_batch_bytes(const pond_batch *batch);

/* Completion poll without blocking: *done = 1 when all work enqueued by the batch's
 * last pond_batch_step has completed on the device (also before any step), else 0.
 * POND_ECUDA if that work failed. */
pond_status pond_batch_poll(pond_batch *batch, int32_t *done);

/* Last error message of the batch (never NULL). */
const char *pond_batch_last_error(const pond_batch *batch);

/* Destroy the batch (its contexts stay valid and leave the batch). */
void pond_batch_destroy(pond_batch *batch);

/* Library version string. */
const char *pond_version(void);

/* Measurement utility (no counterpart in the paper): the arithmetic peak of this GPU's
 * fused multiply-add pipes, for the roofline of the step kernel, which is bound by plain
 * FP32 (mixed form) or FP64 (FP64 form) arithmetic.  Runs a kernel of 8 independent FMA
 * chains per thread, iters FMAs each, on 8 blocks of 256 threads per SM, timed with CUDA
 * events on `stream` (NULL = default stream); *tflops_out = 2 x FMAs / time in TFLOP/s.
 * precision: POND_MIXED (FP32) or POND_FP64.  It allocates and frees a small device
 * buffer and synchronises the stream.  Errors: POND_EINVAL (bad precision, iters < 1,
 * NULL output), POND_ECUDA. */
pond_status pond_fma_peak(int32_t precision, int32_t iters, void *stream, double *tflops_out);

#ifdef __cplusplus
}
#endif

#endif /* POND_H */
