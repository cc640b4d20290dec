// pond.cu -- host side of libpond: the C ABI declared in include/pond.h.
//
// A context owns two state buffers of one 32-value record per node (ping-pong), a
// 5-plane FP64 staging buffer
// for host <-> device field copies, the block partials of the conservation sums and a
// small block of device counters.  Every call enqueues on the context stream; one time
// step is one launch of the fused kernel k_pond_step (pond_step.cuh).
#include "pond.h"

#include <cuda_runtime.h>
#include <cudaTypedefs.h>   // PFN_cuTensorMapEncodeTiled

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "pond_kernels.cuh"
#include "pond_step.cuh"
#include "pond_q16.cuh"
#include "pond_q27.cuh"

using namespace pond;

cudaEvent_t batch_done_event(pond_batch *b);   // defined with the batches below

struct pond_ctx {
    pond_grid grid{};
    pond_eos eos{};
    pond_opts opts{};
    double kappa = 0.0, tau = 1.0;
    int device = 0;
    size_t N = 0, esize = 0;
    void *state[2] = {nullptr, nullptr};
    int cur = 0;
    double *stage = nullptr;       // 6 planes of double
    double *part = nullptr;        // conservation partials (nblk * 8) + out[4]
    int red_blocks = 0;
    DevStats *dstats = nullptr;
    cudaStream_t stream = nullptr;
    int64_t steps = 0;
    int lanes = 8;                 // lanes per node of the step kernel (8 or 16)
    bool initialised = false;
    pond_batch *batch = nullptr;   // batch that steps this context, if any
    int nonlocal = 0;              // 1: current-time non-local terms (two passes per step)
    void *pred = nullptr;          // first pass's state (nonlocal = 1)
    DevStats *dstats_pred = nullptr;
    int lattice = POND_D2Q9;       // POND_D2Q16: node records of SLQ values; POND_D3Q27: SL27
    Grid3 g3{1, 0};                // z extent and boundary (D3Q27)
    double *nlbuf = nullptr;       // D2Q16: NL_PLANES FP64 planes of non-local terms
    std::string err;
    size_t bytes = 0;
    DevParams dp{};
    // device counters already reported by a sync point's status (sticky flags: a
    // condition is reported once, by the first sync point after it occurred)
    unsigned long long rep_nonconv = 0, rep_clamped = 0, rep_timeouts = 0;
    // D2Q9: tensor maps of the two state buffers for the TMA staging of interior tiles
    CUtensorMap tmap[2];
    int use_tma = 0;
};

namespace {

pond_status fail(pond_ctx *c, pond_status st, const std::string &msg)
{
    if (c) c->err = msg;
    return st;
}

pond_status cuda_fail(pond_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, POND_ECUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call, where)                                 \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, where); \
    } while (0)

void *dev_alloc(pond_ctx *c, size_t bytes)
{
    void *p = nullptr;
    if (c->opts.dalloc) {
        p = c->opts.dalloc(bytes, c->opts.alloc_ctx);
    } else if (cudaMalloc(&p, bytes) != cudaSuccess) {
        p = nullptr;
    }
    if (p) c->bytes += bytes;
    return p;
}

void dev_free(pond_ctx *c, void *p)
{
    if (!p) return;
    if (c->opts.dfree) c->opts.dfree(p, c->opts.alloc_ctx);
    else cudaFree(p);
}

inline unsigned blocks_for(size_t n, unsigned bs) { return (unsigned)((n + bs - 1) / bs); }

// cuTensorMapEncodeTiled from the driver, looked up once (null if unavailable).
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess && q == cudaDriverEntryPointSuccess)
            fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
        cudaGetLastError();
    });
    return fn;
}

// Tensor maps of a D2Q9 context's state buffers: the records as a 3-D tensor
// [ny][nx][SL] of R, box = the staged slot values x the staged row pitch x the halo'd tile
// height, so that a box lands in shared memory exactly as the step kernel's staged tile.
// Leaves use_tma = 0 (every tile copied per chunk) if the maps cannot be made.
void make_tensor_maps(pond_ctx *c)
{
    c->use_tma = 0;
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc || c->lattice != POND_D2Q9) return;
    const bool f32 = c->opts.precision == POND_MIXED;
    const int TS = f32 ? Slot<float>::stride : Slot<double>::stride;
    const int PT = step_row_pitch(c->dp.tile_x, TS), HT = STEP_NB / c->dp.tile_x + 2 * HALO;
    if (PT > c->grid.nx || HT > c->grid.ny) return;   // no interior tile
    const cuuint64_t dims[3] = {(cuuint64_t)SL, (cuuint64_t)c->grid.nx, (cuuint64_t)c->grid.ny};
    const cuuint64_t strides[2] = {(cuuint64_t)SL * c->esize, (cuuint64_t)SL * c->esize * c->grid.nx};
    const cuuint32_t box[3] = {(cuuint32_t)TS, (cuuint32_t)PT, (cuuint32_t)HT};
    const cuuint32_t estr[3] = {1, 1, 1};
    for (int k = 0; k < 2; ++k)
        if (enc(&c->tmap[k], f32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_FLOAT64, 3,
                c->state[k], dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return;
    c->use_tma = 1;
}

bool mixed(const pond_ctx *c) { return c->opts.precision == POND_MIXED; }

// Tiles of 16 nodes of the D2Q9 step kernel over the grid.
int step_tiles(const pond_ctx *c)
{
    const int ty = STEP_NB / c->dp.tile_x;
    return c->dp.tiles_x * ((c->grid.ny + ty - 1) / ty);
}

// Largest dynamic shared memory of a step block over the tile shapes, for lanes per node.
template <typename R>
size_t step_smem_max(int lanes)
{
    size_t m = 0;
    for (int tx = 1; tx <= STEP_NB; tx *= 2)
        m = std::max(m, step_smem_bytes(tx, Slot<R>::stride, (int)sizeof(R), lanes));
    return m;
}

// Lets the step kernels of type R use more than the default 48 KB of dynamic shared
// memory on the current device (idempotent; not a stream operation).
template <typename R>
cudaError_t allow_step_smem()
{
    cudaError_t e = cudaFuncSetAttribute(k_pond_step<R, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)step_smem_max<R>(8));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pond_step<R, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)step_smem_max<R>(16));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pond_step_batch<R, 8>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)step_smem_max<R>(8));
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_pond_step_batch<R, 16>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)step_smem_max<R>(16));
    return e;
}

// D2Q16: the non-local terms of state `src` into nlbuf, then the node step in -> out.
template <typename R>
void launch_q16_pass(pond_ctx *c, const R *in, const R *src, R *out, DevStats *stats,
                     cudaStream_t strm)
{
    const unsigned nb = blocks_for(c->N, 256);
    k_q16_nonlocal1<R><<<nb, 256, 0, strm>>>(c->dp, src, c->nlbuf);
    k_q16_nonlocal2<<<nb, 256, 0, strm>>>(c->dp, c->nlbuf);
    // 32 x 4 node patches (128 x 1 strips on grids of fewer than 4 rows)
    const dim3 blk = c->grid.ny < 4 ? dim3(128, 1) : dim3(32, 4);
    const dim3 grd(blocks_for((size_t)c->grid.nx, blk.x), blocks_for((size_t)c->grid.ny, blk.y));
    k_q16_step<R><<<grd, blk, 0, strm>>>(c->dp, in, c->nlbuf, out, stats);
}

template <typename R>
pond_status launch_step_q16(pond_ctx *c, cudaEvent_t *ev)
{
    const R *in = (const R *)c->state[c->cur];
    R *out = (R *)c->state[1 - c->cur];
    if (ev) cudaEventRecord(ev[0], c->stream);
    const R *nl = in;
    if (c->nonlocal) {
        // pass 1 predicts rho, T at t (lagged terms); pass 2 redoes the step with the
        // non-local terms of that prediction
        launch_q16_pass<R>(c, in, in, (R *)c->pred, c->dstats_pred, c->stream);
        nl = (const R *)c->pred;
    }
    launch_q16_pass<R>(c, in, nl, out, c->dstats, c->stream);
    if (ev) cudaEventRecord(ev[1], c->stream);
    c->cur = 1 - c->cur;
    return POND_OK;
}

// D3Q27: the non-local terms of state `src`, then the node step in -> out.
template <typename R>
void launch_q27_pass(pond_ctx *c, const R *in, const R *src, R *out, DevStats *stats)
{
    const unsigned nb = blocks_for(c->N, 256);
    k_q27_nonlocal1<R><<<nb, 256, 0, c->stream>>>(c->dp, c->g3, src, c->nlbuf);
    k_q27_nonlocal2<<<nb, 256, 0, c->stream>>>(c->dp, c->g3, c->nlbuf);
    const dim3 blk = c->grid.ny < 4 ? dim3(128, 1) : dim3(32, 4);
    const dim3 grd(blocks_for((size_t)c->grid.nx, blk.x), blocks_for((size_t)c->grid.ny, blk.y), (unsigned)c->g3.nz);
    k_q27_step<R><<<grd, blk, 0, c->stream>>>(c->dp, c->g3, in, c->nlbuf, out, stats);
}

template <typename R>
pond_status launch_step_q27(pond_ctx *c, cudaEvent_t *ev)
{
    const R *in = (const R *)c->state[c->cur];
    R *out = (R *)c->state[1 - c->cur];
    if (ev) cudaEventRecord(ev[0], c->stream);
    const R *nl = in;
    if (c->nonlocal) {
        launch_q27_pass<R>(c, in, in, (R *)c->pred, c->dstats_pred);
        nl = (const R *)c->pred;
    }
    launch_q27_pass<R>(c, in, nl, out, c->dstats);
    if (ev) cudaEventRecord(ev[1], c->stream);
    c->cur = 1 - c->cur;
    return POND_OK;
}

template <typename R>
pond_status launch_step(pond_ctx *c, cudaEvent_t *ev = nullptr)
{
    if (c->lattice == POND_D2Q16) return launch_step_q16<R>(c, ev);
    if (c->lattice == POND_D3Q27) return launch_step_q27<R>(c, ev);
    const R *in = (const R *)c->state[c->cur];
    R *out = (R *)c->state[1 - c->cur];
    const unsigned nb = (unsigned)step_tiles(c);
    const size_t smem = step_smem_bytes(c->dp.tile_x, Slot<R>::stride, (int)sizeof(R), c->lanes);
    const CUtensorMap &tm = c->tmap[c->cur];
    if (ev) cudaEventRecord(ev[0], c->stream);
    const R *nl = in;
    if (c->nonlocal) {
        // pass 1: the lagged step predicts rho, T at t (its counters kept apart); pass 2
        // redoes the step from the same state with the non-local terms of that prediction
        R *pred = (R *)c->pred;
        if (c->lanes == 16) k_pond_step<R, 16><<<nb, STEP_NB * 16, smem, c->stream>>>(c->dp, in, pred, c->dstats_pred, in, tm, c->use_tma);
        else k_pond_step<R, 8><<<nb, STEP_NB * 8, smem, c->stream>>>(c->dp, in, pred, c->dstats_pred, in, tm, c->use_tma);
        nl = pred;
    }
    if (c->lanes == 16) k_pond_step<R, 16><<<nb, STEP_NB * 16, smem, c->stream>>>(c->dp, in, out, c->dstats, nl, tm, c->use_tma);
    else k_pond_step<R, 8><<<nb, STEP_NB * 8, smem, c->stream>>>(c->dp, in, out, c->dstats, nl, tm, c->use_tma);
    if (ev) cudaEventRecord(ev[1], c->stream);
    c->cur = 1 - c->cur;
    return POND_OK;
}

template <typename R>
void launch_init(pond_ctx *c, const double *rho, const double *ux, const double *uy, const double *uz,
                 const double *T)
{
    if (c->lattice == POND_D3Q27) {
        k_q27_init<R><<<blocks_for(c->N, 256), 256, 0, c->stream>>>(c->dp, c->g3, rho, ux, uy, uz, T,
                                                                    (R *)c->state[c->cur], c->dstats);
        return;
    }
    if (c->lattice == POND_D2Q16) {
        k_q16_init<R><<<blocks_for(c->N, 256), 256, 0, c->stream>>>(c->dp, rho, ux, uy, T,
                                                                    (R *)c->state[c->cur], c->dstats);
        return;
    }
    k_init<R><<<blocks_for(c->N, 256), 256, 0, c->stream>>>(c->dp, rho, ux, uy, T,
                                                             (R *)c->state[c->cur], c->dstats);
}

template <typename R>
void launch_moments(pond_ctx *c, double *rho, double *ux, double *uy, double *uz, double *T, double *p)
{
    if (c->lattice == POND_D3Q27) {
        k_q27_moments<R><<<blocks_for(c->N, 256), 256, 0, c->stream>>>(c->dp, (const R *)c->state[c->cur],
                                                                       rho, ux, uy, uz, T, p);
        return;
    }
    if (c->lattice == POND_D2Q16) {
        k_q16_moments<R><<<blocks_for(c->N, 256), 256, 0, c->stream>>>(c->dp, (const R *)c->state[c->cur],
                                                                       rho, ux, uy, T, p);
        return;
    }
    k_moments<R><<<blocks_for(c->N, 256), 256, 0, c->stream>>>(c->dp, (const R *)c->state[c->cur],
                                                                rho, ux, uy, T, p);
}

template <typename R>
void launch_conserve(pond_ctx *c)
{
    if (c->lattice == POND_D3Q27)
        k_q27_conserve1<R><<<c->red_blocks, 256, 0, c->stream>>>(c->dp, (const R *)c->state[c->cur], c->part);
    else if (c->lattice == POND_D2Q16)
        k_q16_conserve1<R><<<c->red_blocks, 256, 0, c->stream>>>(c->dp, (const R *)c->state[c->cur], c->part);
    else
        k_conserve1<R><<<c->red_blocks, 256, 0, c->stream>>>(c->dp, (const R *)c->state[c->cur], c->part);
    k_conserve2<<<1, 32, 0, c->stream>>>(c->part, c->red_blocks, c->part + 8 * c->red_blocks);
}

// D2Q16 nodes and weights on the host (the same closed forms as the device's)
void lattice16(double c[4], double w[4])
{
    const double s6 = std::sqrt(6.0), ci = std::sqrt(3.0 - s6), co = std::sqrt(3.0 + s6);
    c[0] = -co; c[1] = -ci; c[2] = ci; c[3] = co;
    w[0] = w[3] = (3.0 - s6) / 12.0;
    w[1] = w[2] = (3.0 + s6) / 12.0;
}

pond_status check_ctx(pond_ctx *c)
{
    if (!c) return POND_EINVAL;
    c->err.clear();
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    // work of a batch this context belongs to comes first on the context's stream
    if (c->batch) {
        e = cudaStreamWaitEvent(c->stream, batch_done_event(c->batch), 0);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamWaitEvent");
    }
    return POND_OK;
}

// Status of a sync point from the device counters hs (read after the context stream
// was synchronised): POND_ENAN while the state holds non-finite values; otherwise
// POND_ENONCONV if frame searches hit max_iter since the last report, else POND_ETHETA if
// the pressure floor was hit since the last report, else POND_OK.  A report clears both
// flags (the counts stay readable through pond_stats).
pond_status report_flags(pond_ctx *c, const DevStats &hs)
{
    if (hs.timeouts > c->rep_timeouts) {
        c->rep_timeouts = hs.timeouts;
        return fail(c, POND_ETIMEOUT, "a bounded wait for a tile's staging copies ran out (" +
                                          std::to_string(hs.timeouts) + " tiles skipped; the state is incomplete)");
    }
    if (hs.nonfinite)
        return fail(c, POND_ENAN, "non-finite values in the state (" + std::to_string(hs.nonfinite) +
                                      " node updates; see pond_stats)");
    const unsigned long long nc = hs.nonconv - std::min(hs.nonconv, c->rep_nonconv);
    const unsigned long long cl = hs.clamped - std::min(hs.clamped, c->rep_clamped);
    c->rep_nonconv = hs.nonconv;
    c->rep_clamped = hs.clamped;
    if (nc)
        return fail(c, POND_ENONCONV, "frame search hit max_iter at " + std::to_string(nc) +
                                          " node updates since the last report (results are returned)");
    if (cl)
        return fail(c, POND_ETHETA, "pressure floor hit at " + std::to_string(cl) +
                                        " node updates since the last report (results are returned)");
    return POND_OK;
}

// Enqueue the copy of the device counters into hs (read it after synchronising).
cudaError_t fetch_stats(pond_ctx *c, DevStats *hs)
{
    return cudaMemcpyAsync(hs, c->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream);
}

pond_status init_common(pond_ctx *c, const double *d_rho, const double *d_ux, const double *d_uy,
                        const double *d_uz, const double *d_T)
{
    CK(cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->stream), "cudaMemsetAsync");
    if (mixed(c)) launch_init<float>(c, d_rho, d_ux, d_uy, d_uz, d_T);
    else launch_init<double>(c, d_rho, d_ux, d_uy, d_uz, d_T);
    CK(cudaGetLastError(), "k_init launch");
    DevStats hs{};
    CK(cudaMemcpyAsync(&hs, c->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream), "cudaMemcpyAsync");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    CK(cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->stream), "cudaMemsetAsync");
    if (hs.bad_init)
        return fail(c, POND_EINVAL, "init fields need rho > 0, b*rho < 1 and T > 0 at every node ("
                                        + std::to_string(hs.bad_init) + " nodes violate it)");
    c->initialised = true;
    c->steps = 0;
    c->rep_nonconv = c->rep_clamped = c->rep_timeouts = 0;
    return POND_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free conservation sums.  Scratch for the block partials lives in this
// file-scope device array instead of memory the caller or the library allocates: every
// device that loads the library holds these NOALLOC_SCRATCH_DOUBLES doubles until the
// process exits.  Host code may not pass the symbol itself to a kernel (it is a host-side
// stand-in, not a device address); the device address is looked up once per device.
constexpr int NOALLOC_SPAN = 2048;          // nodes summed by one block
constexpr int NOALLOC_MAX_BLOCKS = 4096;    // => at most 8,388,608 nodes per call
constexpr int NOALLOC_SCRATCH_DOUBLES = 8 * NOALLOC_MAX_BLOCKS + 8;
static __device__ __align__(256) double g_noalloc_scratch[NOALLOC_SCRATCH_DOUBLES];

constexpr int NOALLOC_MAX_DEVICES = 64;
std::mutex g_noalloc_mutex;
double *g_noalloc_ptr[NOALLOC_MAX_DEVICES] = {nullptr};

// Device address of g_noalloc_scratch on the current device, looked up on first use.
cudaError_t noalloc_scratch(double **ptr)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= NOALLOC_MAX_DEVICES) return cudaErrorInvalidDevice;
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess) return e;
        g_noalloc_ptr[dev] = (double *)p;
    }
    *ptr = g_noalloc_ptr[dev];
    return cudaSuccess;
}

}  // namespace

namespace {
// 8 independent chains a = a * m + c per thread (m, c chosen so that values stay finite
// and the compiler cannot fold them); one value per thread is written so that nothing
// is eliminated.
template <typename R>
__global__ void k_fma_chains(R *out, int iters, R m, R c)
{
    R a[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) a[k] = R(threadIdx.x + k) * R(1e-3);
    for (int it = 0; it < iters; ++it) {
#pragma unroll
        for (int k = 0; k < 8; ++k) a[k] = fma(a[k], m, c);
    }
    R s = 0;
#pragma unroll
    for (int k = 0; k < 8; ++k) s += a[k];
    out[(size_t)blockIdx.x * blockDim.x + threadIdx.x] = s;
}

template <typename R>
pond_status fma_peak(int iters, cudaStream_t s, double *tflops)
{
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
        return POND_ECUDA;
    const int blocks = 8 * sms, threads = 256;
    R *out = nullptr;
    if (cudaMalloc((void **)&out, (size_t)blocks * threads * sizeof(R)) != cudaSuccess) return POND_ECUDA;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    k_fma_chains<R><<<blocks, threads, 0, s>>>(out, iters / 10 + 1, R(0.999999), R(1e-6));   // warm-up
    cudaEventRecord(e0, s);
    k_fma_chains<R><<<blocks, threads, 0, s>>>(out, iters, R(0.999999), R(1e-6));
    cudaEventRecord(e1, s);
    cudaError_t e = cudaEventSynchronize(e1);
    float ms = 0.0f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
    if (e == cudaSuccess) e = cudaGetLastError();
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaFree(out);
    if (e != cudaSuccess || !(ms > 0.0f)) return POND_ECUDA;
    *tflops = 2.0 * 8.0 * (double)iters * blocks * threads / (ms * 1e-3) / 1e12;
    return POND_OK;
}
}  // namespace

extern "C" {

pond_status pond_conservation_noalloc(const double *d_planes, int64_t n_nodes, double out[4],
                                      void *stream)
{
    if (!d_planes || !out || n_nodes < 1) return POND_EINVAL;
    if (n_nodes > (int64_t)NOALLOC_SPAN * NOALLOC_MAX_BLOCKS) return POND_EINVAL;
    double *scratch = nullptr;
    if (noalloc_scratch(&scratch) != cudaSuccess) return POND_ECUDA;
    cudaStream_t s = (cudaStream_t)stream;
    const int nb = (int)((n_nodes + NOALLOC_SPAN - 1) / NOALLOC_SPAN);
    // launch errors are peeked right after each launch (a sticky error left by other work
    // is neither taken nor cleared here); the stream's synchronisation decides the result
    k_conserve_planes1<<<nb, 256, 0, s>>>(d_planes, (long long)n_nodes, NOALLOC_SPAN, scratch);
    if (cudaPeekAtLastError() != cudaSuccess) return POND_ECUDA;
    k_conserve2<<<1, 32, 0, s>>>(scratch, nb, scratch + 8 * NOALLOC_MAX_BLOCKS);
    if (cudaPeekAtLastError() != cudaSuccess) return POND_ECUDA;
    if (cudaMemcpyAsync(out, scratch + 8 * NOALLOC_MAX_BLOCKS, 4 * sizeof(double),
                        cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return POND_ECUDA;
    return cudaStreamSynchronize(s) == cudaSuccess ? POND_OK : POND_ECUDA;
}


const char *pond_version(void) { return "pond-gb300 0.1 (sm_103a)"; }


pond_status pond_fma_peak(int32_t precision, int32_t iters, void *stream, double *tflops_out)
{
    if (!tflops_out || iters < 1 || (precision != POND_MIXED && precision != POND_FP64)) return POND_EINVAL;
    cudaStream_t s = (cudaStream_t)stream;
    return precision == POND_MIXED ? fma_peak<float>(iters, s, tflops_out)
                                   : fma_peak<double>(iters, s, tflops_out);
}

const char *pond_last_error(const pond_ctx *ctx) { return ctx ? ctx->err.c_str() : "null context"; }

size_t pond_device_bytes(const pond_ctx *ctx) { return ctx ? ctx->bytes : 0; }

pond_status pond_create(const pond_grid *grid, const pond_lattice *lattice, const pond_eos *eos,
                        double kappa, double tau, const pond_opts *opts, pond_ctx **out)
{
    if (!out) return POND_EINVAL;
    *out = nullptr;
    if (!grid || !lattice || !eos || !opts) return POND_EINVAL;
    if (grid->nx < 1 || grid->ny < 1) return POND_EINVAL;
    if ((grid->bc_x != POND_PERIODIC && grid->bc_x != POND_ZEROGRAD) ||
        (grid->bc_y != POND_PERIODIC && grid->bc_y != POND_ZEROGRAD))
        return POND_EINVAL;
    if (lattice->kind != POND_D2Q9 && lattice->kind != POND_D2Q16 && lattice->kind != POND_D3Q27)
        return POND_EINVAL;
    // z extent: 0 or 1 on the two-dimensional lattices; >= 1 on D3Q27
    if (grid->nz < 0 || (lattice->kind != POND_D3Q27 && grid->nz > 1)) return POND_EINVAL;
    if (lattice->kind == POND_D3Q27 && (grid->nz < 1 || (grid->bc_z != POND_PERIODIC && grid->bc_z != POND_ZEROGRAD)))
        return POND_EINVAL;
    if (eos->kind != POND_VDW && eos->kind != POND_IDEAL && eos->kind != POND_DIETERICI &&
        eos->kind != POND_SIMPLIFIED)
        return POND_EINVAL;
    if (eos->kind == POND_SIMPLIFIED &&
        (!eos->isothermal || !(eos->beta > 0.0) || !(eos->rho_v > 0.0) || !(eos->rho_l > eos->rho_v) ||
         !(eos->p0 > 0.0)))
        return POND_EINVAL;
    if (eos->isothermal != 0 && eos->isothermal != 1) return POND_EINVAL;
    if (eos->isothermal && !(eos->T_iso > 0.0 && std::isfinite(eos->T_iso))) return POND_EINVAL;
    if (eos->kind == POND_DIETERICI && (!eos->isothermal || !(eos->a > 0.0) || !(eos->b > 0.0)))
        return POND_EINVAL;
    if (!(eos->R > 0.0) || !(eos->delta > 0.0) || !(eos->delta <= 2.0 / 3.0 + 1e-12)) return POND_EINVAL;
    if (eos->kind == POND_VDW && (!(eos->a >= 0.0) || !(eos->b >= 0.0))) return POND_EINVAL;
    if (!(kappa >= 0.0) || !(tau > 0.5) || !std::isfinite(tau) || !std::isfinite(kappa)) return POND_EINVAL;
    if (opts->precision != POND_FP64 && opts->precision != POND_MIXED) return POND_EINVAL;
    if (!(opts->dt > 0.0) || !(opts->dt <= 1.0)) return POND_EINVAL;
    if (!(opts->tol > 0.0) || opts->max_iter < 1 || opts->max_iter > 1000) return POND_EINVAL;
    if (!(opts->p_floor > 0.0)) return POND_EINVAL;
    if ((opts->dalloc == nullptr) != (opts->dfree == nullptr)) return POND_EINVAL;
    if (opts->lanes_per_node != 0 && opts->lanes_per_node != 8 && opts->lanes_per_node != 16)
        return POND_EINVAL;
    if (opts->nonlocal != POND_NONLOCAL_LAGGED && opts->nonlocal != POND_NONLOCAL_CURRENT)
        return POND_EINVAL;
    if (opts->tile_x != 0 && opts->tile_x != 1 && opts->tile_x != 2 && opts->tile_x != 4 &&
        opts->tile_x != 8 && opts->tile_x != 16)
        return POND_EINVAL;

    pond_ctx *c = new pond_ctx();
    c->grid = *grid;
    c->eos = *eos;
    if (eos->kind == POND_IDEAL) { c->eos.a = 0.0; c->eos.b = 0.0; }
    c->opts = *opts;
    c->lattice = lattice->kind;
    c->kappa = kappa;
    c->tau = tau;
    c->stream = (cudaStream_t)opts->stream;
    c->N = (size_t)grid->nx * (size_t)grid->ny * (size_t)(grid->nz > 1 ? grid->nz : 1);
    if (c->lattice == POND_D3Q27) c->g3 = Grid3{grid->nz, grid->bc_z};
    c->esize = opts->precision == POND_MIXED ? sizeof(float) : sizeof(double);
    // 8 lanes per node unless the caller picks 16 (measured faster on every grid tried so
    // far; the choice is exposed for the autotuner).
    c->lanes = opts->lanes_per_node ? opts->lanes_per_node : 8;
    // tile of the step kernel: a 16 x 1 strip for grids of few rows, 4 x 4 otherwise
    int tile_x = opts->tile_x ? opts->tile_x : (grid->ny < 4 ? 16 : 4);
    cudaError_t e = cudaGetDevice(&c->device);
    if (e == cudaSuccess)
        e = opts->precision == POND_MIXED ? allow_step_smem<float>() : allow_step_smem<double>();
    if (e != cudaSuccess) {
        delete c;
        return POND_ECUDA;
    }
    DevParams &d = c->dp;
    d.nx = grid->nx; d.ny = grid->ny; d.bcx = grid->bc_x; d.bcy = grid->bc_y;
    d.N = (long long)c->N;
    d.a = c->eos.a; d.b = c->eos.b; d.R = c->eos.R; d.delta = c->eos.delta; d.cv = c->eos.R / c->eos.delta;
    d.kappa = kappa; d.tau = tau; d.omega = 1.0 / tau; d.dt = opts->dt; d.k_cond = opts->k_cond;
    d.p_floor = opts->p_floor; d.tol = opts->tol; d.max_iter = opts->max_iter;
    d.tile_x = tile_x; d.tiles_x = (grid->nx + tile_x - 1) / tile_x;
    d.pd.a = d.a; d.pd.b = d.b; d.pd.R = d.R; d.pd.cv = d.cv; d.pd.inv_cv = 1.0 / d.cv;
    d.pd.kappa = d.kappa; d.pd.p_floor = d.p_floor; d.pd.dt = d.dt; d.pd.omega = d.omega;
    d.pd.mu_coef = (d.tau - 0.5) * d.dt; d.pd.cvR = d.cv + d.R; d.pd.k_cond = d.k_cond;
    d.pf.a = (float)d.pd.a; d.pf.b = (float)d.pd.b; d.pf.R = (float)d.pd.R; d.pf.cv = (float)d.pd.cv;
    d.pf.inv_cv = (float)d.pd.inv_cv; d.pf.kappa = (float)d.pd.kappa; d.pf.p_floor = (float)d.pd.p_floor;
    d.pf.dt = (float)d.pd.dt; d.pf.omega = (float)d.pd.omega; d.pf.mu_coef = (float)d.pd.mu_coef;
    d.pf.cvR = (float)d.pd.cvR; d.pf.k_cond = (float)d.pd.k_cond;
    auto split = [](double x, float out[2]) {
        out[0] = (float)x;
        out[1] = (float)(x - (double)out[0]);
    };
    split(d.a, d.ff_a); split(d.b, d.ff_b); split(d.R, d.ff_R); split(d.pd.inv_cv, d.ff_icv);
    split(d.p_floor, d.ff_pfl);
    d.tol_f = (float)d.tol;
    d.eos_kind = c->eos.kind == POND_DIETERICI ? 2 : (c->eos.kind == POND_SIMPLIFIED ? 3 : 0);
    d.sp[0] = c->eos.beta; d.sp[1] = c->eos.rho_l; d.sp[2] = c->eos.rho_v; d.sp[3] = c->eos.p0;
    for (int k = 0; k < 4; ++k) d.spf[k] = (float)d.sp[k];
    split(d.sp[3], d.ff_p0);
    d.isothermal = c->eos.isothermal;
    d.T_iso = c->eos.isothermal ? c->eos.T_iso : 0.0;
    split(d.T_iso, d.ff_Tiso);

    c->red_blocks = (int)std::min<size_t>(1024, std::max<size_t>(1, (c->N + 255) / 256));
    size_t sb = (size_t)(c->lattice == POND_D2Q16 ? SLQ : (c->lattice == POND_D3Q27 ? SL27 : SL)) * c->N * c->esize;
    c->state[0] = dev_alloc(c, sb);
    c->state[1] = dev_alloc(c, sb);
    c->stage = (double *)dev_alloc(c, 6 * c->N * sizeof(double));
    c->part = (double *)dev_alloc(c, (8 * (size_t)c->red_blocks + 8) * sizeof(double));
    c->dstats = (DevStats *)dev_alloc(c, sizeof(DevStats));
    if (c->lattice == POND_D2Q16) c->nlbuf = (double *)dev_alloc(c, (size_t)NL_PLANES * c->N * sizeof(double));
    if (c->lattice == POND_D3Q27) c->nlbuf = (double *)dev_alloc(c, (size_t)N3_PLANES * c->N * sizeof(double));
    c->nonlocal = opts->nonlocal;
    if (c->nonlocal) {
        c->pred = dev_alloc(c, sb);
        c->dstats_pred = (DevStats *)dev_alloc(c, sizeof(DevStats));
    }
    if (!c->state[0] || !c->state[1] || !c->stage || !c->part || !c->dstats ||
        (c->nonlocal && (!c->pred || !c->dstats_pred)) || (c->lattice != POND_D2Q9 && !c->nlbuf)) {
        pond_destroy(c);
        return POND_ENOMEM;
    }
    if (cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->stream) != cudaSuccess) {
        pond_destroy(c);
        return POND_ECUDA;
    }
    make_tensor_maps(c);
    *out = c;
    return POND_OK;
}

void pond_destroy(pond_ctx *c)
{
    if (!c) return;
    if (c->batch) pond_batch_remove(c->batch, c);
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    else cudaDeviceSynchronize();
    dev_free(c, c->state[0]);
    dev_free(c, c->state[1]);
    dev_free(c, c->stage);
    dev_free(c, c->part);
    dev_free(c, c->dstats);
    dev_free(c, c->pred);
    dev_free(c, c->dstats_pred);
    dev_free(c, c->nlbuf);
    delete c;
}

pond_status pond_init_fields(pond_ctx *c, const double *rho, const double *ux, const double *uy,
                             const double *T)
{
    pond_status st = check_ctx(c);
    if (st) return st;
    if (!rho || !ux || !uy || !T) return fail(c, POND_EINVAL, "null field pointer");
    size_t bytes = c->N * sizeof(double);
    const double *src[4] = {rho, ux, uy, T};
    for (int k = 0; k < 4; ++k)
        CK(cudaMemcpyAsync(c->stage + k * c->N, src[k], bytes, cudaMemcpyHostToDevice, c->stream),
           "cudaMemcpyAsync H2D");
    CK(cudaMemsetAsync(c->stage + 4 * c->N, 0, bytes, c->stream), "cudaMemsetAsync");   // u_z = 0
    return init_common(c, c->stage, c->stage + c->N, c->stage + 2 * c->N, c->stage + 4 * c->N,
                       c->stage + 3 * c->N);
}

pond_status pond_init_fields3(pond_ctx *c, const double *rho, const double *ux, const double *uy,
                              const double *uz, const double *T)
{
    pond_status st = check_ctx(c);
    if (st) return st;
    if (!rho || !ux || !uy || !uz || !T) return fail(c, POND_EINVAL, "null field pointer");
    size_t bytes = c->N * sizeof(double);
    const double *src[5] = {rho, ux, uy, T, uz};
    for (int k = 0; k < 5; ++k)
        CK(cudaMemcpyAsync(c->stage + k * c->N, src[k], bytes, cudaMemcpyHostToDevice, c->stream),
           "cudaMemcpyAsync H2D");
    return init_common(c, c->stage, c->stage + c->N, c->stage + 2 * c->N, c->stage + 4 * c->N,
                       c->stage + 3 * c->N);
}

pond_status pond_init_fields_device(pond_ctx *c, const double *d_rho, const double *d_ux,
                                    const double *d_uy, const double *d_T)
{
    pond_status st = check_ctx(c);
    if (st) return st;
    if (!d_rho || !d_ux || !d_uy || !d_T) return fail(c, POND_EINVAL, "null field pointer");
    CK(cudaMemsetAsync(c->stage + 4 * c->N, 0, c->N * sizeof(double), c->stream), "cudaMemsetAsync");
    return init_common(c, d_rho, d_ux, d_uy, c->stage + 4 * c->N, d_T);
}

pond_status pond_step(pond_ctx *c, int64_t n)
{
    pond_status st = check_ctx(c);
    if (st) return st;
    if (n < 0) return fail(c, POND_EINVAL, "negative step count");
    if (!c->initialised) return fail(c, POND_EINVAL, "state not initialised");
    if (c->batch) return fail(c, POND_EINVAL, "context belongs to a batch: step it with pond_batch_step");
    for (int64_t k = 0; k < n; ++k) {
        if (mixed(c)) launch_step<float>(c);
        else launch_step<double>(c);
    }
    CK(cudaGetLastError(), "step launch");
    c->steps += n;
    return POND_OK;
}

pond_status pond_step_timed(pond_ctx *c, double *ms_out)
{
    pond_status st = check_ctx(c);
    if (st) return st;
    if (!ms_out) return fail(c, POND_EINVAL, "null output");
    if (!c->initialised) return fail(c, POND_EINVAL, "state not initialised");
    cudaEvent_t ev[2];
    for (int k = 0; k < 2; ++k) CK(cudaEventCreate(&ev[k]), "cudaEventCreate");
    if (mixed(c)) launch_step<float>(c, ev);
    else launch_step<double>(c, ev);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaEventSynchronize(ev[1]);
    float ms = 0.f;
    if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, ev[0], ev[1]);
    *ms_out = ms;
    for (int k = 0; k < 2; ++k) cudaEventDestroy(ev[k]);
    if (e != cudaSuccess) return cuda_fail(c, e, "pond_step_timed");
    c->steps += 1;
    return POND_OK;
}

pond_status pond_moments_device(pond_ctx *c, double *rho, double *ux, double *uy, double *T, double *p)
{
    pond_status st = check_ctx(c);
    if (st) return st;
    if (!c->initialised) return fail(c, POND_EINVAL, "state not initialised");
    if (mixed(c)) launch_moments<float>(c, rho, ux, uy, nullptr, T, p);
    else launch_moments<double>(c, rho, ux, uy, nullptr, T, p);
    CK(cudaGetLastError(), "k_moments launch");
    return POND_OK;
}

pond_status pond_moments(pond_ctx *c, double *rho, double *ux, double *uy, double *T, double *p)
{
    pond_status st = check_ctx(c);
    if (st) return st;
    if (!c->initialised) return fail(c, POND_EINVAL, "state not initialised");
    double *host[5] = {rho, ux, uy, T, p};
    double *dev[5];
    for (int k = 0; k < 5; ++k) dev[k] = host[k] ? c->stage + k * c->N : nullptr;
    st = pond_moments_device(c, dev[0], dev[1], dev[2], dev[3], dev[4]);
    if (st) return st;
    for (int k = 0; k < 5; ++k)
        if (host[k])
            CK(cudaMemcpyAsync(host[k], dev[k], c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
               "cudaMemcpyAsync D2H");
    DevStats hs{};
    CK(fetch_stats(c, &hs), "cudaMemcpyAsync D2H");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    return report_flags(c, hs);
}

pond_status pond_moments3(pond_ctx *c, double *rho, double *ux, double *uy, double *uz, double *T,
                          double *p)
{
    pond_status st = check_ctx(c);
    if (st) return st;
    if (!c->initialised) return fail(c, POND_EINVAL, "state not initialised");
    double *host[6] = {rho, ux, uy, uz, T, p};
    double *dev[6];
    for (int k = 0; k < 6; ++k) dev[k] = host[k] ? c->stage + k * c->N : nullptr;
    if (c->lattice == POND_D3Q27) {
        if (mixed(c)) launch_moments<float>(c, dev[0], dev[1], dev[2], dev[3], dev[4], dev[5]);
        else launch_moments<double>(c, dev[0], dev[1], dev[2], dev[3], dev[4], dev[5]);
    } else {
        // two-dimensional lattices: u_z = 0
        if (mixed(c)) launch_moments<float>(c, dev[0], dev[1], dev[2], nullptr, dev[4], dev[5]);
        else launch_moments<double>(c, dev[0], dev[1], dev[2], nullptr, dev[4], dev[5]);
        if (dev[3]) CK(cudaMemsetAsync(dev[3], 0, c->N * sizeof(double), c->stream), "cudaMemsetAsync");
    }
    CK(cudaGetLastError(), "k_moments launch");
    for (int k = 0; k < 6; ++k)
        if (host[k])
            CK(cudaMemcpyAsync(host[k], dev[k], c->N * sizeof(double), cudaMemcpyDeviceToHost, c->stream),
               "cudaMemcpyAsync D2H");
    DevStats hs{};
    CK(fetch_stats(c, &hs), "cudaMemcpyAsync D2H");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    return report_flags(c, hs);
}

pond_status pond_conservation(pond_ctx *c, double out[4])
{
    pond_status st = check_ctx(c);
    if (st) return st;
    if (!out) return fail(c, POND_EINVAL, "null output");
    if (!c->initialised) return fail(c, POND_EINVAL, "state not initialised");
    if (mixed(c)) launch_conserve<float>(c);
    else launch_conserve<double>(c);
    CK(cudaGetLastError(), "conservation launch");
    CK(cudaMemcpyAsync(out, c->part + 8 * c->red_blocks, 4 * sizeof(double), cudaMemcpyDeviceToHost,
                       c->stream), "cudaMemcpyAsync D2H");
    DevStats hs{};
    CK(fetch_stats(c, &hs), "cudaMemcpyAsync D2H");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    return report_flags(c, hs);
}

pond_status pond_get_state(pond_ctx *c, double *state)
{
    pond_status st = check_ctx(c);
    if (st) return st;
    if (!state) return fail(c, POND_EINVAL, "null output");
    if (!c->initialised) return fail(c, POND_EINVAL, "state not initialised");
    if (c->lattice == POND_D3Q27) {
        const size_t N = c->N, rec = (size_t)SL27 * N;
        std::vector<double> d(mixed(c) ? 0 : rec);
        std::vector<float> f(mixed(c) ? rec : 0);
        void *dst = mixed(c) ? (void *)f.data() : (void *)d.data();
        CK(cudaMemcpyAsync(dst, c->state[c->cur], rec * c->esize, cudaMemcpyDeviceToHost, c->stream),
           "cudaMemcpyAsync D2H");
        CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        for (int p = 0; p < NP27; ++p) {
            const int o = rec27_off(p);
            for (size_t n = 0; n < N; ++n)
                state[(size_t)p * N + n] = mixed(c) ? (double)f[n * SL27 + o] : d[n * SL27 + o];
        }
        if (mixed(c)) {
            // kept remainders folded into the exchanged populations: W_i (m + c_i.J/(s T_L))
            // on f, W_i G on g
            const double w1[3] = {1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0};
            for (size_t n = 0; n < N; ++n) {
                const float *r = &f[n * SL27];
                const double sq = std::sqrt((double)r[R_TH]);
                const double m = r[R_MLO], gl = r[R_GLO];
                const double J[3] = {r[R_JLO], r[R_JLO + 1], r[R_JLO + 2]};
                for (int i = 0; i < Q27; ++i) {
                    const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
                    const double w = w1[cx + 1] * w1[cy + 1] * w1[cz + 1];
                    state[(size_t)i * N + n] += w * (m + (cx * J[0] + cy * J[1] + cz * J[2]) / (sq * (1.0 / 3.0)));
                    state[(size_t)(Q27 + i) * N + n] += w * gl;
                }
            }
        }
        return POND_OK;
    }
    if (c->lattice == POND_D2Q16) {
        // node records on the device, planes on the host
        const size_t N = c->N, rec = (size_t)SLQ * N;
        std::vector<double> d(mixed(c) ? 0 : rec);
        std::vector<float> f(mixed(c) ? rec : 0);
        void *dst = mixed(c) ? (void *)f.data() : (void *)d.data();
        CK(cudaMemcpyAsync(dst, c->state[c->cur], rec * c->esize, cudaMemcpyDeviceToHost, c->stream),
           "cudaMemcpyAsync D2H");
        CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        for (int p = 0; p < NP16; ++p)
            for (size_t n = 0; n < N; ++n)
                state[(size_t)p * N + n] = mixed(c) ? (double)f[n * SLQ + p] : d[n * SLQ + p];
        if (mixed(c)) {
            // the kept remainders go into the exchanged populations: mass and momentum as
            // W_i (m + (c_ix J_x + c_iy J_y)/s) on f (its sum is m, its momentum m u + J),
            // energy as W_i G on g
            double cq[4], wq[4];
            lattice16(cq, wq);
            for (size_t n = 0; n < N; ++n) {
                const float *r = &f[n * SLQ];
                const double sq = std::sqrt((double)r[Q_TH]);
                const double m = r[Q_MLO], jx = r[Q_JXLO], jy = r[Q_JYLO], gl = r[Q_GLO];
                for (int i = 0; i < Q16; ++i) {
                    const double w = wq[i & 3] * wq[i >> 2];
                    state[(size_t)(Q_F + i) * N + n] += w * (m + (cq[i & 3] * jx + cq[i >> 2] * jy) / sq);
                    state[(size_t)(Q_G + i) * N + n] += w * gl;
                }
            }
        }
        return POND_OK;
    }
    const size_t N = c->N, rec = (size_t)SL * N;
    std::vector<double> d(mixed(c) ? 0 : rec);
    std::vector<float> f(mixed(c) ? rec : 0);
    void *dst = mixed(c) ? (void *)f.data() : (void *)d.data();
    CK(cudaMemcpyAsync(dst, c->state[c->cur], rec * c->esize, cudaMemcpyDeviceToHost, c->stream),
       "cudaMemcpyAsync D2H");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    for (int p = 0; p < NPL; ++p) {
        const int o = rec_off(p);
        for (size_t n = 0; n < N; ++n)
            state[(size_t)p * N + n] = mixed(c) ? (double)f[n * SL + o] : d[n * SL + o];
    }
    // the rest populations with their kept low parts (the momentum low parts, below one
    // ulp of the populations, are not part of the exchanged state)
    for (int k = 0; k < 2; ++k) {
        const int p = k == 0 ? P_F + 4 : P_G + 4, lo = k == 0 ? P_F4LO : P_G4LO;
        for (size_t n = 0; n < N; ++n)
            state[(size_t)p * N + n] += mixed(c) ? (double)f[n * SL + lo] : d[n * SL + lo];
    }
    return POND_OK;
}

pond_status pond_set_state(pond_ctx *c, const double *state)
{
    pond_status st = check_ctx(c);
    if (st) return st;
    if (!state) return fail(c, POND_EINVAL, "null input");
    if (c->lattice == POND_D3Q27) {
        const size_t N = c->N, rec = (size_t)SL27 * N;
        std::vector<double> d(mixed(c) ? 0 : rec, 0.0);
        std::vector<float> f(mixed(c) ? rec : 0, 0.0f);
        for (int p = 0; p < NP27; ++p) {
            const int o = rec27_off(p);
            for (size_t n = 0; n < N; ++n) {
                if (mixed(c)) f[n * SL27 + o] = (float)state[(size_t)p * N + n];
                else d[n * SL27 + o] = state[(size_t)p * N + n];
            }
        }
        if (mixed(c))
            for (size_t n = 0; n < N; ++n) {
                // what the FP32 populations leave out becomes the kept remainders again
                float *r = &f[n * SL27];
                const double sq = std::sqrt((double)r[R_TH]);
                double m = 0.0, S[3] = {0, 0, 0}, gl = 0.0;
                for (int i = 0; i < Q27; ++i) {
                    const double rf = state[(size_t)i * N + n] - (double)r[R_F + i];
                    m += rf;
                    S[0] += rf * (i % 3 - 1); S[1] += rf * ((i / 3) % 3 - 1); S[2] += rf * (i / 9 - 1);
                    gl += state[(size_t)(Q27 + i) * N + n] - (double)r[R_G + i];
                }
                r[R_MLO] = (float)m;
                for (int a = 0; a < 3; ++a) r[R_JLO + a] = (float)(sq * S[a]);
                r[R_GLO] = (float)gl;
            }
        const void *src = mixed(c) ? (const void *)f.data() : (const void *)d.data();
        CK(cudaMemcpyAsync(c->state[c->cur], src, rec * c->esize, cudaMemcpyHostToDevice, c->stream),
           "cudaMemcpyAsync H2D");
        CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        c->initialised = true;
        return POND_OK;
    }
    if (c->lattice == POND_D2Q16) {
        const size_t N = c->N, rec = (size_t)SLQ * N;
        std::vector<double> d(mixed(c) ? 0 : rec, 0.0);
        std::vector<float> f(mixed(c) ? rec : 0, 0.0f);
        for (int p = 0; p < NP16; ++p)
            for (size_t n = 0; n < N; ++n) {
                if (mixed(c)) f[n * SLQ + p] = (float)state[(size_t)p * N + n];
                else d[n * SLQ + p] = state[(size_t)p * N + n];
            }
        if (mixed(c)) {
            // what the FP32 populations leave out becomes the kept remainders again: mass
            // sum r_i, momentum s sum r_i c_i (beyond the mass part's u m), energy sum r_gi
            double cq[4], wq[4];
            lattice16(cq, wq);
            for (size_t n = 0; n < N; ++n) {
                float *r = &f[n * SLQ];
                const double sq = std::sqrt((double)r[Q_TH]);
                double m = 0.0, sx = 0.0, sy = 0.0, gl = 0.0;
                for (int i = 0; i < Q16; ++i) {
                    const double rf = state[(size_t)(Q_F + i) * N + n] - (double)r[Q_F + i];
                    m += rf;
                    sx += rf * cq[i & 3];
                    sy += rf * cq[i >> 2];
                    gl += state[(size_t)(Q_G + i) * N + n] - (double)r[Q_G + i];
                }
                r[Q_MLO] = (float)m;
                r[Q_JXLO] = (float)(sq * sx);
                r[Q_JYLO] = (float)(sq * sy);
                r[Q_GLO] = (float)gl;
            }
        }
        const void *src = mixed(c) ? (const void *)f.data() : (const void *)d.data();
        CK(cudaMemcpyAsync(c->state[c->cur], src, rec * c->esize, cudaMemcpyHostToDevice, c->stream),
           "cudaMemcpyAsync H2D");
        CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
        c->initialised = true;
        return POND_OK;
    }
    const size_t N = c->N, rec = (size_t)SL * N;
    std::vector<double> d(mixed(c) ? 0 : rec, 0.0);
    std::vector<float> f(mixed(c) ? rec : 0, 0.0f);
    for (int p = 0; p < NPL; ++p) {
        const int o = rec_off(p);
        for (size_t n = 0; n < N; ++n) {
            if (mixed(c)) f[n * SL + o] = (float)state[(size_t)p * N + n];
            else d[n * SL + o] = state[(size_t)p * N + n];
        }
    }
    // FP32 form: the rest populations keep the part below their float as the low word
    if (mixed(c))
        for (int k = 0; k < 2; ++k) {
            const int p = k == 0 ? P_F + 4 : P_G + 4, lo = k == 0 ? P_F4LO : P_G4LO;
            for (size_t n = 0; n < N; ++n)
                f[n * SL + lo] = (float)(state[(size_t)p * N + n] - (double)f[n * SL + p]);
        }
    const void *src = mixed(c) ? (const void *)f.data() : (const void *)d.data();
    CK(cudaMemcpyAsync(c->state[c->cur], src, rec * c->esize, cudaMemcpyHostToDevice, c->stream),
       "cudaMemcpyAsync H2D");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    c->initialised = true;
    return POND_OK;
}

pond_status pond_stats(pond_ctx *c, pond_stats_t *out, int32_t reset)
{
    pond_status st = check_ctx(c);
    if (st) return st;
    if (!out) return fail(c, POND_EINVAL, "null output");
    DevStats hs{};
    CK(cudaMemcpyAsync(&hs, c->dstats, sizeof(DevStats), cudaMemcpyDeviceToHost, c->stream),
       "cudaMemcpyAsync D2H");
    if (reset) CK(cudaMemsetAsync(c->dstats, 0, sizeof(DevStats), c->stream), "cudaMemsetAsync");
    CK(cudaStreamSynchronize(c->stream), "cudaStreamSynchronize");
    if (reset) c->rep_nonconv = c->rep_clamped = c->rep_timeouts = 0;
    out->steps = c->steps;
    out->node_updates = c->steps * (int64_t)c->N;
    out->streams = (int64_t)hs.streams;
    out->nonconverged = (int64_t)hs.nonconv;
    out->clamped = (int64_t)hs.clamped;
    out->nonfinite = (int64_t)hs.nonfinite;
    out->stalled = (int64_t)hs.stalled;
    out->block_streams = (int64_t)hs.block_streams;
    out->max_streams = (int64_t)hs.max_streams;
    out->timeouts = (int64_t)hs.timeouts;
    out->region_nodes = (int64_t)hs.region_nodes;
    out->pair_streams = (int64_t)hs.pair_streams;
    return hs.nonfinite ? fail(c, POND_ENAN, "non-finite values in the state") : POND_OK;
}

// ---------------------------------------------------------------------------
// Batches: many simulations stepped by one launch per (precision, lanes) group and step.

}  // extern "C"

struct pond_batch {
    int device = 0;
    cudaStream_t stream = nullptr;
    std::vector<pond_ctx *> sims;
    bool dirty = true;
    int64_t since_build = 0;          // batch steps since the device lists were built
    cudaEvent_t done = nullptr;       // recorded after every batch step call
    std::string err;
    struct Group {
        int precision = 0, lanes = 8;
        std::vector<pond_ctx *> sims;
        void *desc[2] = {nullptr, nullptr};   // SimDesc arrays for even / odd steps
        int2 *work = nullptr;
        size_t desc_cap = 0, work_cap = 0;
        int nwork = 0;
        size_t smem = 0;
    };
    Group g[4];                       // (fp64, mixed) x (8, 16 lanes)
    // D2Q16 contexts: stepped by their own three launches on the batch stream; cur0 is
    // the context's current buffer when the lists were built
    struct Q16 { pond_ctx *c; int cur0; };
    std::vector<Q16> q16;
    cudaGraphExec_t graph = nullptr;  // two steps (even, odd) of every group
    bool graph_ok = false;
    size_t budget = 0;                // device bytes the members may hold (0: no limit)
    size_t member_bytes = 0;          // sum of the members' pond_device_bytes
};

cudaEvent_t batch_done_event(pond_batch *b) { return b->done; }

namespace {

pond_status bfail(pond_batch *b, pond_status st, const std::string &m)
{
    b->err = m;
    return st;
}


template <typename R>
cudaError_t build_group(pond_batch *b, pond_batch::Group &G)
{
    const size_t ns = G.sims.size();
    std::vector<SimDesc<R>> d0(ns), d1(ns);
    std::vector<int2> work;
    G.smem = 0;
    for (size_t k = 0; k < ns; ++k) {
        pond_ctx *c = G.sims[k];
        d0[k].p = c->dp; d0[k].in = (const R *)c->state[c->cur]; d0[k].out = (R *)c->state[1 - c->cur];
        d0[k].stats = c->dstats;
        d1[k] = d0[k]; d1[k].in = (const R *)c->state[1 - c->cur]; d1[k].out = (R *)c->state[c->cur];
        const int ty = STEP_NB / c->dp.tile_x;
        const int tiles = c->dp.tiles_x * ((c->grid.ny + ty - 1) / ty);
        for (int t = 0; t < tiles; ++t) work.push_back(make_int2((int)k, t));
        G.smem = std::max(G.smem, step_smem_bytes(c->dp.tile_x, Slot<R>::stride, (int)sizeof(R), G.lanes));
    }
    G.nwork = (int)work.size();
    cudaError_t e = cudaSuccess;
    if (ns * sizeof(SimDesc<R>) > G.desc_cap) {
        for (int k = 0; k < 2; ++k) { cudaFree(G.desc[k]); G.desc[k] = nullptr; }
        G.desc_cap = 2 * ns * sizeof(SimDesc<R>);
        for (int k = 0; k < 2 && e == cudaSuccess; ++k) e = cudaMalloc(&G.desc[k], G.desc_cap);
        if (e != cudaSuccess) { G.desc_cap = 0; return e; }
    }
    if (work.size() * sizeof(int2) > G.work_cap) {
        cudaFree(G.work); G.work = nullptr;
        G.work_cap = 2 * work.size() * sizeof(int2);
        e = cudaMalloc((void **)&G.work, G.work_cap);
        if (e != cudaSuccess) { G.work_cap = 0; return e; }
    }
    if (ns) {
        e = cudaMemcpyAsync(G.desc[0], d0.data(), ns * sizeof(SimDesc<R>), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(G.desc[1], d1.data(), ns * sizeof(SimDesc<R>), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(G.work, work.data(), work.size() * sizeof(int2), cudaMemcpyHostToDevice, b->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);   // host vectors go out of scope
    }
    return e;
}

template <typename R>
void launch_group(pond_batch *b, pond_batch::Group &G, int parity)
{
    if (!G.nwork) return;
    const SimDesc<R> *d = (const SimDesc<R> *)G.desc[parity];
    if (G.lanes == 16)
        k_pond_step_batch<R, 16><<<G.nwork, STEP_NB * 16, G.smem, b->stream>>>(d, G.work);
    else
        k_pond_step_batch<R, 8><<<G.nwork, STEP_NB * 8, G.smem, b->stream>>>(d, G.work);
}

template <typename R>
void launch_q16_entry(pond_batch *b, const pond_batch::Q16 &e, int parity)
{
    pond_ctx *c = e.c;
    const int ci = e.cur0 ^ parity;
    const R *in = (const R *)c->state[ci];
    launch_q16_pass<R>(c, in, in, (R *)c->state[1 - ci], c->dstats, b->stream);
}

void launch_all(pond_batch *b, int parity)
{
    for (int k = 0; k < 4; ++k) {
        if (b->g[k].precision == POND_MIXED) launch_group<float>(b, b->g[k], parity);
        else launch_group<double>(b, b->g[k], parity);
    }
    for (const pond_batch::Q16 &e : b->q16) {
        if (mixed(e.c)) launch_q16_entry<float>(b, e, parity);
        else launch_q16_entry<double>(b, e, parity);
    }
}

pond_status batch_build(pond_batch *b)
{
    for (int k = 0; k < 4; ++k) {
        b->g[k].precision = (k & 1) ? POND_MIXED : POND_FP64;
        b->g[k].lanes = (k & 2) ? 16 : 8;
        b->g[k].sims.clear();
    }
    b->q16.clear();
    for (pond_ctx *c : b->sims) {
        if (c->lattice == POND_D2Q16) {
            b->q16.push_back({c, c->cur});
            continue;
        }
        const int k = (c->opts.precision == POND_MIXED ? 1 : 0) | (c->lanes == 16 ? 2 : 0);
        b->g[k].sims.push_back(c);
    }
    for (int k = 0; k < 4; ++k) {
        cudaError_t e = (k & 1) ? build_group<float>(b, b->g[k]) : build_group<double>(b, b->g[k]);
        if (e != cudaSuccess) return bfail(b, POND_ECUDA, std::string("batch build: ") + cudaGetErrorString(e));
    }
    if (b->graph) { cudaGraphExecDestroy(b->graph); b->graph = nullptr; }
    b->graph_ok = false;
    // capture two steps (even then odd parity) of every group once; replays step the batch
    if (b->stream) {
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
            launch_all(b, 0);
            launch_all(b, 1);
            cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
            if (e == cudaSuccess && graph && cudaGraphInstantiate(&b->graph, graph, 0) == cudaSuccess)
                b->graph_ok = true;
            if (graph) cudaGraphDestroy(graph);
        }
        cudaGetLastError();   // a failed capture falls back to plain launches
    }
    b->dirty = false;
    b->since_build = 0;
    return POND_OK;
}

}  // namespace

extern "C" {

pond_status pond_batch_create(void *stream, pond_batch **out)
{
    if (!out) return POND_EINVAL;
    *out = nullptr;
    pond_batch *b = new pond_batch();
    b->stream = (cudaStream_t)stream;
    if (cudaGetDevice(&b->device) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming) != cudaSuccess) {
        delete b;
        return POND_ECUDA;
    }
    *out = b;
    return POND_OK;
}

pond_status pond_batch_add(pond_batch *b, pond_ctx *c)
{
    if (!b || !c) return POND_EINVAL;
    b->err.clear();
    if (c->batch) return bfail(b, POND_EINVAL, "context already belongs to a batch");
    if (!c->initialised) return bfail(b, POND_EINVAL, "context state not initialised");
    if (c->nonlocal) return bfail(b, POND_EINVAL, "two-pass (current-time) contexts are stepped alone");
    if (c->lattice == POND_D3Q27) return bfail(b, POND_EINVAL, "D3Q27 contexts are stepped alone");
    if (c->device != b->device) return bfail(b, POND_EINVAL, "context lives on another device");
    // a lone member may exceed the budget, so that no context is refused for ever
    if (b->budget && !b->sims.empty() && b->member_bytes + c->bytes > b->budget)
        return bfail(b, POND_ENOMEM, "the context's " + std::to_string(c->bytes) + " device bytes exceed the batch budget (" +
                                         std::to_string(b->member_bytes) + " of " + std::to_string(b->budget) + " in use)");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, POND_ECUDA, "cudaSetDevice");
    // the context's queued work (its initialisation) completes before the batch uses it
    if (cudaStreamSynchronize(c->stream) != cudaSuccess) return bfail(b, POND_ECUDA, "cudaStreamSynchronize");
    b->sims.push_back(c);
    b->member_bytes += c->bytes;
    c->batch = b;
    b->dirty = true;
    return POND_OK;
}

pond_status pond_batch_remove(pond_batch *b, pond_ctx *c)
{
    if (!b || !c) return POND_EINVAL;
    auto it = std::find(b->sims.begin(), b->sims.end(), c);
    if (it == b->sims.end()) return bfail(b, POND_EINVAL, "context is not in this batch");
    cudaSetDevice(b->device);
    if (cudaStreamSynchronize(b->stream) != cudaSuccess) return bfail(b, POND_ECUDA, "cudaStreamSynchronize");
    b->sims.erase(it);
    b->member_bytes -= std::min(b->member_bytes, c->bytes);
    c->batch = nullptr;
    b->dirty = true;
    return POND_OK;
}

int32_t pond_batch_size(const pond_batch *b) { return b ? (int32_t)b->sims.size() : 0; }

pond_status pond_batch_set_budget(pond_batch *b, size_t bytes)
{
    if (!b) return POND_EINVAL;
    b->err.clear();
    if (bytes && bytes < b->member_bytes)
        return bfail(b, POND_EINVAL, "budget below the members' current device bytes");
    b->budget = bytes;
    return POND_OK;
}

size_t pond_batch_bytes(const pond_batch *b) { return b ? b->member_bytes : 0; }

pond_status pond_batch_poll(pond_batch *b, int32_t *done)
{
    if (!b || !done) return POND_EINVAL;
    b->err.clear();
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, POND_ECUDA, "cudaSetDevice");
    const cudaError_t e = cudaEventQuery(b->done);
    if (e == cudaSuccess) { *done = 1; return POND_OK; }
    if (e == cudaErrorNotReady) { *done = 0; return POND_OK; }
    return bfail(b, POND_ECUDA, std::string("batch poll: ") + cudaGetErrorString(e));
}

pond_status pond_batch_step(pond_batch *b, int64_t n)
{
    if (!b) return POND_EINVAL;
    b->err.clear();
    if (n < 0) return bfail(b, POND_EINVAL, "negative step count");
    if (cudaSetDevice(b->device) != cudaSuccess) return bfail(b, POND_ECUDA, "cudaSetDevice");
    if (b->sims.empty() || n == 0) return POND_OK;
    if (b->dirty) {
        pond_status st = batch_build(b);
        if (st) return st;
    }
    int64_t k = 0;
    // whole graph replays when the next step is an even one
    if (b->graph_ok && (b->since_build % 2) == 0)
        for (; k + 2 <= n; k += 2)
            if (cudaGraphLaunch(b->graph, b->stream) != cudaSuccess)
                return bfail(b, POND_ECUDA, "cudaGraphLaunch");
    for (; k < n; ++k) launch_all(b, (int)((b->since_build + k) % 2));
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return bfail(b, POND_ECUDA, std::string("batch step: ") + cudaGetErrorString(e));
    b->since_build += n;
    for (pond_ctx *c : b->sims) {
        if (n % 2) c->cur = 1 - c->cur;
        c->steps += n;
    }
    if (cudaEventRecord(b->done, b->stream) != cudaSuccess) return bfail(b, POND_ECUDA, "cudaEventRecord");
    return POND_OK;
}

const char *pond_batch_last_error(const pond_batch *b) { return b ? b->err.c_str() : "null batch"; }

void pond_batch_destroy(pond_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaStreamSynchronize(b->stream);
    for (pond_ctx *c : b->sims) c->batch = nullptr;
    for (auto &G : b->g) {
        for (int k = 0; k < 2; ++k) cudaFree(G.desc[k]);
        cudaFree(G.work);
    }
    if (b->graph) cudaGraphExecDestroy(b->graph);
    cudaEventDestroy(b->done);
    delete b;
}

}  // extern "C"
