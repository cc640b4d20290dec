// pond_step.cuh -- the fused time-step kernel of the PonD van der Waals model (sm_103a).
//
// One launch per time step.  A block owns NB = 16 nodes; each node is served by a group
// of LPN = 8 or 16 lanes of one warp.  Per node:
//   phase 0  non-local terms from the previous step's rho and T (radius 2): lane l of the
//            group takes the l-th non-rest neighbour, builds the Korteweg stress K and the
//            heat flux q there from the 8 differences around it, and the group sums
//            W c . K and W c . q into F = -div K and M_0 = 2 div q (Eq. korteweg, Eq. gtilde).
//   phase 1  frame search (block lockstep): the group streams all 9 directions x 16 stencil
//            nodes (each lane 16/LPN stencil positions of every direction), keeps each
//            lane's partial increments in shared memory and reduces only the four moment
//            sums per stream; warp 0 (one lane per node) takes the moments, inverts
//            e -> T, evaluates the EoS and the residual, in FP64 in the FP64 form and in
//            float-float (pairs of FP32) in the mixed form.
//   phase 2  BGK collision with the force source, heat-flux correction and forced g
//            equilibrium, one population per lane; the rest population takes the exact
//            remainder of mass and energy, and what storage rounding takes from the
//            conserved sums is kept beside the record.
//
// Staging.  Each block owns a tile of tile_x x (16 / tile_x) nodes and first copies the
// records of the tile plus a halo of HALO = 3 nodes (their first 24 values) into shared
// memory with 16-byte cp.async copies, one record slot per unwrapped coordinate, so that
// periodic and zero-gradient boundaries need no special case.  All stencil reads of the
// step come from there; a departure point farther than the halo (|v| dt >= 1) falls back
// to a global load.
//
// Increment form.  With f~_i = sum_n A_n [G_n f(n)]_i and sum_n A_n = 1,
//   f~_i = f_i(x) + sum_n A_n ( [G_n (f(n) - f(x))]_i + [(G_n - I) f(x)]_i ),
// where G_n is the transfer map from the gauge of stencil node n into the arrival gauge
// (SM "Transfer matrix", separable per axis) and (G_n - I) is evaluated from the gauge
// differences directly, so equal gauges give exactly the identity and a uniform region
// reproduces itself exactly.  The FP32 rounding error of a step is then proportional to
// the local differences, not to the populations, and does not accumulate as a bias.
#pragma once

#include <cuda.h>   // CUtensorMap (the tensor-map type of the TMA tile copies)

#include "pond_kernels.cuh"

namespace pond {

constexpr int STEP_NB = 16;   // nodes per block (lanes per node LPN = 8 or 16 is a template
                              // parameter: more lanes per node for grids too small to fill
                              // the GPU with 8); 16 nodes per block keep small grids spread
                              // evenly over the 152 SMs
constexpr unsigned STEP_NB_MASK = STEP_NB == 32 ? 0xffffffffu : ((1u << STEP_NB) - 1u);
constexpr int HALO = 3;       // staged halo width (stencil reach for |v| dt < 1)
// Largest side of a node's stencil region (the union of its 9 directions' 4x4 stencils)
// that the region stream handles: 4 + the spread of the departure points' floors, 5 for
// |v| dt < 1; wider regions take the per-pair stream.
constexpr int REGION_MAX = 8;
// Mixed form: a frame-search residual below this multiple of tol that no longer halves is
// taken as the FP32 rounding floor (the EoS cancels up to ~200x inside interfaces).
constexpr float STALL_TOL_FACTOR = 16.0f;
// resident blocks per SM the register budget is sized for: in FP32 five blocks of 128
// threads (8 lanes per node, about 96 registers) or two of 256 (16 lanes); in FP64 three
// of 128 (168 registers, 2 % faster than two of 198) or one of 256, so that its wider
// values stay in registers
#define STEP_MIN_BLOCKS(R, LPN) (sizeof(R) == 8 ? ((LPN) == 8 ? 3 : 1) : ((LPN) == 8 ? 5 : 2))

// Shared-memory record slot: the first 24 values of a node record (f, g, theta, u, pad,
// rho, T), padded to a 16-byte multiple that spreads consecutive slots over the banks.
// slot words past the 24 staged values: p and p/rho of the staged node (shared memory only)
constexpr int S_PR = 24, S_PRR = 25;
template <typename R> struct Slot;
template <> struct Slot<float> { static constexpr int stride = 28, chunks = 6; };
template <> struct Slot<double> { static constexpr int stride = 26, chunks = 12; };

// Slots per staged row: the tile width plus halos, rounded up (FP32 slots of 28 words) to
// 4 mod 8 so that vertically adjacent slots start 16 banks apart and the two stencil rows
// a lane group reads fall on disjoint banks.
__host__ __device__ constexpr int step_row_pitch(int tile_x, int slot_words)
{
    return slot_words == 28 ? ((tile_x + 2 * HALO + 3) / 8) * 8 + 4 : tile_x + 2 * HALO;
}

// Slots of the step kernel's staged tile (tile_x columns).
__host__ __device__ constexpr int step_tile_slots(int tile_x, int slot_words)
{
    return step_row_pitch(tile_x, slot_words) * (STEP_NB / tile_x + 2 * HALO);
}

// Per-lane partial increments of the 18 streamed populations of every node, behind the
// staged tile: node j's row d (0..8 f, 9..17 g) holds its lanes' partials at
// [j * step_part_stride(LPN) + d * LPN + lane]; the extra LPN per node offsets
// neighbouring groups of a warp onto other banks.
__host__ __device__ constexpr int step_part_stride(int lpn) { return 19 * lpn; }

// Dynamic shared memory of one step block: staged tile + halo, then the partials.
__host__ __device__ constexpr size_t step_smem_bytes(int tile_x, int slot_words, int elem_bytes, int lpn)
{
    return ((size_t)step_tile_slots(tile_x, slot_words) * slot_words +
            (size_t)STEP_NB * step_part_stride(lpn)) * elem_bytes;
}

__device__ __forceinline__ void cp_async16(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all()
{
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;\n" ::: "memory");
}

// ---- TMA tile copies (cp.async.bulk.tensor) completed on an mbarrier ----------------
__device__ __forceinline__ unsigned smem_u32(const void *p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long *bar, unsigned count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    // make the initialised barrier visible to the async (TMA) proxy
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}

// One arrival that also expects `bytes` of asynchronous copies on the barrier.
__device__ __forceinline__ void mbar_arrive_expect_tx(unsigned long long *bar, unsigned bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// Copy the box at coordinates (c0, c1, c2) of a 3-D tensor map into shared memory dst
// (the box lands densely, innermost dimension first), completing on bar.
__device__ __forceinline__ void tma_load_3d(void *dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            unsigned long long *bar)
{
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3, %4}], [%5];\n" ::"r"(smem_u32(dst)),
        "l"(reinterpret_cast<unsigned long long>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_u32(bar))
        : "memory");
}

// Wait for phase `parity` of bar to complete, for at most limit_ns nanoseconds of the
// global timer; returns false if the limit ran out (the caller then gives up the tile
// instead of hanging).
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long *bar, unsigned parity,
                                                  unsigned long long limit_ns)
{
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t0));
    for (;;) {
        unsigned done;
        asm volatile(
            "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\nselp.u32 %0, 1, 0, p;\n}\n"
            : "=r"(done) : "r"(smem_u32(bar)), "r"(parity) : "memory");
        if (done) return true;
        unsigned long long t;
        asm volatile("mov.u64 %0, %%globaltimer;\n" : "=l"(t));
        if (t - t0 > limit_ns) return false;
    }
}
constexpr unsigned long long TMA_WAIT_LIMIT_NS = 1000000000ull;   // one second

template <typename R>
struct StepShared {
    R dsum[STEP_NB][4];        // sum dF, sum dF cx, sum dF cy, sum dG of the current stream
    R lam[STEP_NB][3];         // current arrival gauge (theta, ux, uy)
    R nl[STEP_NB][3];          // lagged F_x, F_y, rho E_lambda of the node
    R mac[STEP_NB][10];        // rho, u*x, u*y, uhx, uhy, E, T, P, theta*, p
    R dlam[STEP_NB][3];        // theta* - theta, u*x - ux, u*y - uy (from FP64)
    R hilo[STEP_NB][4];        // rho and sum g~ as (hi, lo) pairs of R
    R mom[STEP_NB][4];         // sum f~ c_x, sum f~ c_y (gauge units) as (hi, lo) pairs
    R bhi[STEP_NB][4];         // sums of the node's stored f, f cx, f cy, g, error-free as
    R blo[STEP_NB][4];         //   unevaluated (hi, lo) pairs of R
    // Lagrange weights of the current stream per axis and region column (row) c, one per
    // direction of that axis: wt[j][axis][c][k] = a_(c - o_k)(xi_k), zero outside the
    // 4-node stencil of direction k (o_k its offset in the node's region)
    R wt[STEP_NB][2][REGION_MAX][4];
    int active[STEP_NB];
    int any_active;
    int nreg[STEP_NB];         // region nodes streamed by node j (summed over its streams)
    int npair[STEP_NB];        // streams of node j that took the per-pair path
};

// 1-D transfer-map increment E = l_k(c_a + e) - l_k(c_a) for target index k (c = k-1),
// source offset e (in units of the target spacing s) and source index a (c_a = a-1).
template <typename R>
__device__ __forceinline__ R ell_inc(int k, int a, R e)
{
    R two_c = R(2 * (a - 1));
    if (k == 1) return -e * (two_c + e);
    if (k == 0) return R(0.5) * e * (two_c + e - R(1));
    return R(0.5) * e * (two_c + e + R(1));
}

// ell_inc for a target index k known only at run time: the same arithmetic, with the
// k = 0 / k = 2 forms joined through their sign
template <typename R>
__device__ __forceinline__ R ell_inc_rt(int k, int a, R e)
{
    const R base = R(2 * (a - 1)) + e;
    return k == 1 ? -e * base : R(0.5) * e * (base + R(k - 1));
}

// 1-D lattice weights W_-1, W_0, W_+1 = 1/6, 2/3, 1/6 as values of type R whose sum is
// exactly one: in FP32 the nearest floats to 1/6 and 2/3 sum to 1 + 3e-8, a bias that every
// collision would add to the mass and energy; W_+-1 = 1/6 rounded down and W_0 = 1 - 2 W_+-1
// (both exact floats) sum to one exactly.
template <typename R> __device__ __forceinline__ R wlat(int a);
template <> __device__ __forceinline__ float wlat<float>(int a)
{
    return a == 1 ? 0x1.555556p-1f : 0x1.555554p-3f;
}
template <> __device__ __forceinline__ double wlat<double>(int a)
{
    return a == 1 ? 1.0 - 2.0 * (1.0 / 6.0) : 1.0 / 6.0;
}

// Stencil weight W_i of the isotropic D2Q9 difference operators, as a constant of type R.
template <typename R>
__device__ __forceinline__ R wst(int ex, int ey)
{
    return (ex == 0 ? R(2.0 / 3.0) : R(1.0 / 6.0)) * (ey == 0 ? R(2.0 / 3.0) : R(1.0 / 6.0));
}

// One cubic Lagrange basis function a_j(xi) on nodes 0..3 (SM "Reconstruction").
template <typename R>
__device__ __forceinline__ R lag1(int j, R xi)
{
    R t0 = xi, t1 = xi - R(1), t2 = xi - R(2), t3 = xi - R(3);
    if (j == 0) return -(t1 * t2 * t3) * R(1.0 / 6.0);
    if (j == 1) return t0 * t2 * t3 * R(0.5);
    if (j == 2) return -(t0 * t1 * t3) * R(0.5);
    return t0 * t1 * t2 * R(1.0 / 6.0);
}

// A departure offset (in nodes) limited to +-2^20, NaN mapped to the lower bound: keeps
// stencil indices derived from it in int range whatever the gauge (fmax returns the
// non-NaN operand).
template <typename R>
__device__ __forceinline__ R clamp_offset(R d)
{
    return fmin(fmax(d, R(-1048576)), R(1048576));
}

// a_j(xi) for a run-time j: the three factors (xi - m), m != j, picked by selects.
template <typename R>
__device__ __forceinline__ R lag1_rt(int j, R xi)
{
    const R t0 = xi, t1 = xi - R(1), t2 = xi - R(2), t3 = xi - R(3);
    const R a = j == 0 ? t1 : t0;
    const R b = j <= 1 ? t2 : t1;
    const R c = j <= 2 ? t3 : t2;
    const R inv = j == 0 ? R(-1.0 / 6.0) : (j == 1 ? R(0.5) : (j == 2 ? R(-0.5) : R(1.0 / 6.0)));
    return a * b * c * inv;
}

// a[i] for a run-time i without local-memory indexing (unrolled selects).
template <typename R, int K>
__device__ __forceinline__ R pick(const R (&a)[K], int i)
{
    R r = a[0];
#pragma unroll
    for (int j = 1; j < K; ++j) r = (i == j) ? a[j] : r;
    return r;
}

// 1/x in FP64 from the FP32 reciprocal and two Newton steps (relative error ~1e-28
// before the final rounding); x must lie in the FP32 normal range.
__device__ __forceinline__ double rcp_d(double x)
{
    double r = (double)__frcp_rn((float)x);
    r = r * (2.0 - x * r);
    return r * (2.0 - x * r);
}

// a / b for operands of moderate range (transfer-map offsets, collision coefficients):
// the fast FP32 quotient, or a times the Newton reciprocal in FP64.
template <typename R> __device__ __forceinline__ R fdiv_(R a, R b);
template <> __device__ __forceinline__ float fdiv_(float a, float b) { return __fdividef(a, b); }
template <> __device__ __forceinline__ double fdiv_(double a, double b) { return a * rcp_d(b); }
template <typename R> __device__ __forceinline__ R frcp_(R b);
template <> __device__ __forceinline__ float frcp_(float b) { return __frcp_rn(b); }
template <> __device__ __forceinline__ double frcp_(double b) { return rcp_d(b); }

// Error-free sum of two values of type R (Knuth TwoSum).
template <typename R>
__device__ __forceinline__ void two_sum_(R a, R b, R &s, R &e)
{
    s = a + b;
    R bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Float-float ("double-word") arithmetic for the FP32 form's frame-search EoS: a value is
// an unevaluated pair hi + lo of floats.  Sums use Knuth's TwoSum, products the exact FMA
// product error (Dekker's TwoProduct with a fused multiply-add), each result renormalised
// with Dekker's Fast2Sum; relative error ~2^-44 per operation, far below the FP32 form's
// needs, on the FP32 pipes (GB300 runs FP64 at 1/64 of the FP32 rate).
struct ffv {
    float hi, lo;
};
__device__ __forceinline__ ffv ff_norm(float a, float b)   // |a| >= |b| or a == 0
{
    const float s = a + b;
    return {s, b - (s - a)};
}
__device__ __forceinline__ ffv ff_pair(float a, float b)   // any a, b
{
    ffv r;
    two_sum_(a, b, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ ffv ff_add(ffv a, ffv b)
{
    float s, e;
    two_sum_(a.hi, b.hi, s, e);
    return ff_norm(s, e + (a.lo + b.lo));
}
__device__ __forceinline__ ffv ff_add(ffv a, float b)
{
    float s, e;
    two_sum_(a.hi, b, s, e);
    return ff_norm(s, e + a.lo);
}
__device__ __forceinline__ ffv ff_neg(ffv a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ ffv ff_mul(ffv a, ffv b)
{
    const float p = __fmul_rn(a.hi, b.hi);   // never contracted into the sum below
    float e = fmaf(a.hi, b.hi, -p);
    e = fmaf(a.hi, b.lo, e);
    e = fmaf(a.lo, b.hi, e);
    return ff_norm(p, e);
}
__device__ __forceinline__ ffv ff_mul(ffv a, float b)
{
    const float p = __fmul_rn(a.hi, b);
    float e = fmaf(a.hi, b, -p);
    e = fmaf(a.lo, b, e);
    return ff_norm(p, e);
}
// 1/a: the FP32 reciprocal and one Newton step r + r (1 - a r) with the residual in
// float-float (Newton doubles the ~24 correct bits)
__device__ __forceinline__ ffv ff_rcp(ffv a)
{
    const float r = __frcp_rn(a.hi);
    const ffv ar = ff_mul(a, r);
    const float res = (1.0f - ar.hi) - ar.lo;
    return ff_norm(r, r * res);
}

// The 21 streamed values of node nd's record (f[9], g[9], theta, u_x, u_y, plus rho and T
// in [22..23]) with 16-byte loads through the read-only path.
__device__ __forceinline__ void load_rec24(const float *__restrict__ b, float v[24])
{
    const float4 *q = reinterpret_cast<const float4 *>(b);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float4 t = __ldg(q + k);
        v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
    }
}
__device__ __forceinline__ void load_rec24(const double *__restrict__ b, double v[24])
{
    const double2 *q = reinterpret_cast<const double2 *>(b);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 t = __ldg(q + k);
        v[2 * k] = t.x; v[2 * k + 1] = t.y;
    }
}

// The same 24 values from a shared-memory slot.
__device__ __forceinline__ void load_slot24(const float *sl, float v[24])
{
    const float4 *q = reinterpret_cast<const float4 *>(sl);
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float4 t = q[k];
        v[4 * k] = t.x; v[4 * k + 1] = t.y; v[4 * k + 2] = t.z; v[4 * k + 3] = t.w;
    }
}
__device__ __forceinline__ void load_slot24(const double *sl, double v[24])
{
    const double2 *q = reinterpret_cast<const double2 *>(sl);
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        const double2 t = q[k];
        v[2 * k] = t.x; v[2 * k + 1] = t.y;
    }
}

// Contribution of stencil node `nd` to direction (jx, jy) of the arrival node, in the
// increment form.
//
// With the per-axis maps written as G = I + E (E = transfer increments, zero for equal
// gauges), [G (f_n - f_x) + (G - I) f_x]_(jx,jy) regroups exactly into
//   (f_n - f_x)_(jx,jy) + t_jy + sum_b Ey[b] (f_n(jx, b) + t_b),   t_b = sum_a Ex[a] f_n(a, b):
// the difference of the two nodes' populations plus increments that multiply the source
// values by the small E only, so the rounding stays relative to the differences and equal
// gauges still give f_n - f_x exactly.
template <typename R>
__device__ __forceinline__ R sel3(int k, R a0, R a1, R a2)
{
    return k == 0 ? a0 : (k == 1 ? a1 : a2);
}

// fxj, gxj: the arrival node's own populations of direction (jx, jy).  jx must be a
// compile-time constant after unrolling; jy may vary at run time (selects, no indexing).
template <typename R>
__device__ __forceinline__ void pair_inc(const R v[24], int jx, int jy, R th, R s, R inv_s, R ux,
                                         R uy, R fxj, R gxj, R &tf, R &tg)
{
    const R thn = v[P_TH];
    const R sn = v[P_SQ];
    // (s_n - s)/s: in FP32 without cancellation, in FP64 directly (its rounding, ~1e-16 of
    // s_n/s, stays far below what the result needs, and saves a reciprocal per pair)
    const R qm1 = sizeof(R) == 8 ? sn * inv_s - R(1) : fdiv_(thn - th, (sn + s) * s);
    const R wx = (v[P_UX] - ux) * inv_s;
    const R wy = (v[P_UY] - uy) * inv_s;
    R Ex[3], Ey[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) {
        Ex[a] = ell_inc<R>(jx, a, qm1 * R(a - 1) + wx);
        Ey[a] = ell_inc<R>(jy, a, qm1 * R(a - 1) + wy);
    }
    if constexpr (sizeof(R) == 8) {
        // FP64: the transfer applied directly, [G_n f_n]_(jx,jy) - f_x (its rounding is far
        // below what the FP64 form needs; the increment form is for FP32)
        R Gx[3], Gy[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Gx[a] = Ex[a] + (a == jx ? R(1) : R(0));
            Gy[a] = Ey[a];
        }
        R rf[3], rg[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            rf[b] = Gx[0] * v[P_F + 3 * b] + Gx[1] * v[P_F + 3 * b + 1] + Gx[2] * v[P_F + 3 * b + 2];
            rg[b] = Gx[0] * v[P_G + 3 * b] + Gx[1] * v[P_G + 3 * b + 1] + Gx[2] * v[P_G + 3 * b + 2];
        }
        // Gy = Ey + delta(b, jy): the delta picks row jy
        R sf = sel3(jy, rf[0], rf[1], rf[2]) - fxj, sg = sel3(jy, rg[0], rg[1], rg[2]) - gxj;
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            sf += Gy[b] * rf[b];
            sg += Gy[b] * rg[b];
        }
        tf = sf;
        tg = sg;
        return;
    }
    R txf[3], txg[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        txf[b] = Ex[0] * v[P_F + 3 * b] + Ex[1] * v[P_F + 3 * b + 1] + Ex[2] * v[P_F + 3 * b + 2];
        txg[b] = Ex[0] * v[P_G + 3 * b] + Ex[1] * v[P_G + 3 * b + 1] + Ex[2] * v[P_G + 3 * b + 2];
    }
    R sf = (sel3(jy, v[P_F + jx], v[P_F + 3 + jx], v[P_F + 6 + jx]) - fxj) + sel3(jy, txf[0], txf[1], txf[2]);
    R sg = (sel3(jy, v[P_G + jx], v[P_G + 3 + jx], v[P_G + 6 + jx]) - gxj) + sel3(jy, txg[0], txg[1], txg[2]);
#pragma unroll
    for (int b = 0; b < 3; ++b) {
        sf += Ey[b] * (v[P_F + 3 * b + jx] + txf[b]);
        sg += Ey[b] * (v[P_G + 3 * b + jx] + txg[b]);
    }
    tf = sf;
    tg = sg;
}

// One stencil node of a node's region carried into the arrival gauge for all nine
// directions of one population family, weighted and accumulated:
//   acc[(k, l)] += wx[k] wy[l] ([G_n f_n](k, l) - f_x(k, l))
// with G_n = (I + Ex) (x) (I + Ey) the separable transfer map from the stencil node's
// gauge into the arrival gauge (SM "Transfer matrix"), Ex[k][a] = l_k increments at the
// source velocities.  In FP32 the increment form (see pair_inc) keeps the rounding
// relative to the differences: (f_n - f_x)(k, l) + t(k, l) + sum_b Ey[l][b] (f_n(k, b) +
// t(k, b)), t(k, b) = sum_a Ex[k][a] f_n(a, b); in FP64 the map is applied directly.
// All indices are compile-time: each stencil node is transformed once for every
// direction whose stencil contains it.
template <typename R>
__device__ __forceinline__ void region_family(const R *v, const R *own, const R (&Ex)[3][3],
                                              const R (&Ey)[3][3], const R (&wx)[3], const R (&wy)[3],
                                              R (&acc)[9])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        R t[3], u[3];
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            t[b] = Ex[k][0] * v[3 * b] + Ex[k][1] * v[3 * b + 1] + Ex[k][2] * v[3 * b + 2];
            if constexpr (sizeof(R) == 8) t[b] += v[3 * b + k];
            u[b] = sizeof(R) == 8 ? t[b] : v[3 * b + k] + t[b];
        }
#pragma unroll
        for (int l = 0; l < 3; ++l) {
            const int i = 3 * l + k;
            R o = sizeof(R) == 8 ? t[l] - own[i] : (v[i] - own[i]) + t[l];
            o += Ey[l][0] * u[0] + Ey[l][1] * u[1] + Ey[l][2] * u[2];
            acc[i] += (wx[k] * wy[l]) * o;
        }
    }
}

// The double-well constants in the arithmetic type of a kernel.
template <typename R> __device__ __forceinline__ const R *typed_sp(const DevParams &p);
template <> __device__ __forceinline__ const float *typed_sp<float>(const DevParams &p) { return p.spf; }
template <> __device__ __forceinline__ const double *typed_sp<double>(const DevParams &p) { return p.sp; }

// Results of one corrector evaluation (moments, e -> T, EoS) of a node, in R.
template <typename R>
struct EosOut {
    R rho_hi, rho_lo;   // rho as a (hi, lo) pair
    R gs_hi, gs_lo;     // sum of the streamed g as a (hi, lo) pair (= 2 rho E)
    R uxs, uys;         // streamed velocity u* (the next gauge velocity)
    R uhx, uhy;         // actual fluid velocity uhat = u* + F dt / (2 rho)
    R E, T, P, pr;      // total energy per mass, temperature, floored and vdW pressure
    R ths;              // theta* = P / (rho T_L)
    R dth, dux, duy;    // theta* - theta, u* - u (the gauge change)
    R mx_hi, mx_lo, my_hi, my_lo;   // sum f~ c_x, sum f~ c_y as (hi, lo) pairs
};

// FP64 form: the streamed moments are the stored sums (hi + lo, rounded to FP64) plus the
// stream's increments (moments Eq.; SM "Thermodynamics": e = E - uhat^2/2 - E_lambda,
// T = (e + a rho)/C_v, p = rho R T/(1 - b rho) - a rho^2, theta = max(p, p_floor)/(rho T_L)).
__device__ __forceinline__ void eos_update(const DevParams &p, const double *bhi, const double *blo,
                                           const double *dsum, const double *nl, const double *lam,
                                           double sr, EosOut<double> &o)
{
    const double dt = p.dt;
    const double Fxd = nl[0], Fyd = nl[1], rEd = nl[2];
    const double thd = lam[0], uxd = lam[1], uyd = lam[2];
    const double rho = (bhi[0] + blo[0]) + dsum[0];
    const double irho = rcp_d(rho);
    const double mx = (bhi[1] + blo[1]) + dsum[1], my = (bhi[2] + blo[2]) + dsum[2];
    const double dux = sr * mx * irho;
    const double duy = sr * my * irho;
    o.mx_hi = mx; o.mx_lo = 0.0; o.my_hi = my; o.my_lo = 0.0;
    const double uxs = uxd + dux, uys = uyd + duy;
    const double uhx = uxs + 0.5 * Fxd * dt * irho, uhy = uys + 0.5 * Fyd * dt * irho;
    const double gs = (bhi[3] + blo[3]) + dsum[3];
    const double E = 0.5 * gs * irho;
    const double e = E - 0.5 * (uhx * uhx + uhy * uhy) - rEd * irho;
    const double T = p.isothermal ? p.T_iso : (e + p.a * rho) * p.pd.inv_cv;
    const double pr = p.eos_kind == 2
        ? rho * p.R * T * rcp_d(1.0 - p.b * rho) * exp(-p.a * rho * rcp_d(p.R * T))
        : (p.eos_kind == 3 ? p.sp[3] + well_pressure<double>(p.sp, rho)
                           : rho * p.R * T * rcp_d(1.0 - p.b * rho) - p.a * rho * rho);
    const double P = pr > p.p_floor ? pr : p.p_floor;
    const double ths = P * irho * 3.0;
    o.rho_hi = rho; o.rho_lo = 0.0; o.gs_hi = gs; o.gs_lo = 0.0;
    o.uxs = uxs; o.uys = uys; o.uhx = uhx; o.uhy = uhy;
    o.E = E; o.T = T; o.P = P; o.pr = pr; o.ths = ths;
    o.dth = ths - thd; o.dux = dux; o.duy = duy;
}

// FP32 form: the same formulas in float-float from the exact (hi, lo) stored sums and the
// FP32 increments; the results are rounded to FP32 once (the pairs of rho and sum g are
// kept for the collision's exact remainders).
__device__ __forceinline__ void eos_update(const DevParams &p, const float *bhi, const float *blo,
                                           const float *dsum, const float *nl, const float *lam,
                                           float sr, EosOut<float> &o)
{
    const float dt = p.pf.dt;
    const ffv a = {p.ff_a[0], p.ff_a[1]}, b = {p.ff_b[0], p.ff_b[1]};
    const ffv Rg = {p.ff_R[0], p.ff_R[1]}, icv = {p.ff_icv[0], p.ff_icv[1]};
    const ffv rho = ff_add(ff_pair(bhi[0], blo[0]), dsum[0]);
    const ffv irho = ff_rcp(rho);
    const ffv mx = ff_add(ff_pair(bhi[1], blo[1]), dsum[1]);
    const ffv my = ff_add(ff_pair(bhi[2], blo[2]), dsum[2]);
    const ffv dux = ff_mul(ff_mul(mx, irho), sr), duy = ff_mul(ff_mul(my, irho), sr);
    const ffv uxs = ff_add(dux, lam[1]), uys = ff_add(duy, lam[2]);
    const ffv uhx = ff_add(uxs, 0.5f * nl[0] * dt * irho.hi);
    const ffv uhy = ff_add(uys, 0.5f * nl[1] * dt * irho.hi);
    const ffv gs = ff_add(ff_pair(bhi[3], blo[3]), dsum[3]);
    const ffv E = ff_mul(ff_mul(gs, irho), 0.5f);
    const ffv kin = ff_mul(ff_add(ff_mul(uhx, uhx), ff_mul(uhy, uhy)), 0.5f);
    const ffv e = ff_add(ff_add(E, ff_neg(kin)), ff_neg(ff_mul(irho, nl[2])));
    const ffv T = p.isothermal ? ffv{p.ff_Tiso[0], p.ff_Tiso[1]} : ff_mul(ff_add(e, ff_mul(rho, a)), icv);
    const ffv den = ff_add(ff_neg(ff_mul(rho, b)), 1.0f);
    const ffv pre = ff_mul(ff_mul(ff_mul(rho, Rg), T), ff_rcp(den));
    // Dieterici: a product with no cancellation, so its exponential factor in FP32 (a few
    // ulps) is enough; van der Waals: the difference in float-float
    // double well: p0 (a float pair) plus a small polynomial part, which FP32 carries
    const ffv pr = p.eos_kind == 2
        ? ff_mul(pre, expf(-(p.pf.a * rho.hi) / (p.pf.R * T.hi)))
        : (p.eos_kind == 3 ? ff_add(ffv{p.ff_p0[0], p.ff_p0[1]}, well_pressure<float>(p.spf, rho.hi))
                           : ff_add(pre, ff_neg(ff_mul(ff_mul(rho, rho), a))));
    const bool floored = !(pr.hi > p.ff_pfl[0] || (pr.hi == p.ff_pfl[0] && pr.lo > p.ff_pfl[1]));
    const ffv P = floored ? ffv{p.ff_pfl[0], p.ff_pfl[1]} : pr;
    const ffv ths = ff_mul(ff_mul(P, irho), 3.0f);
    o.rho_hi = rho.hi; o.rho_lo = rho.lo; o.gs_hi = gs.hi; o.gs_lo = gs.lo;
    o.mx_hi = mx.hi; o.mx_lo = mx.lo; o.my_hi = my.hi; o.my_lo = my.lo;
    o.uxs = uxs.hi; o.uys = uys.hi; o.uhx = uhx.hi; o.uhy = uhy.hi;
    o.E = E.hi; o.T = T.hi; o.P = P.hi; o.pr = pr.hi; o.ths = ths.hi;
    o.dth = (ths.hi - lam[0]) + ths.lo;
    o.dux = dux.hi; o.duy = duy.hi;
}

// Issue (without waiting) the 16-byte cp.async copies of tile `tile_idx` and its halo of
// HALO nodes (the first 24 values of each record) into the staged tile `tile`, one slot per
// unwrapped coordinate (periodic wrap or zero-gradient clamp applied to the source), and
// commit them as one group.
template <typename R>
__device__ __forceinline__ void stage_issue(const DevParams &p, const R *__restrict__ in, R *tile, int tile_idx)
{
    constexpr int TS = Slot<R>::stride, CH = Slot<R>::chunks;
    const int TX = p.tile_x, TY = STEP_NB / TX;
    const int X0 = (tile_idx % p.tiles_x) * TX, Y0 = (tile_idx / p.tiles_x) * TY;
    const int WT = TX + 2 * HALO, HT = TY + 2 * HALO;
    const int PT = step_row_pitch(TX, TS);
    const int total = WT * HT * CH;
    // k / WT through the float reciprocal: exact for k < 2^20 (the quotient's fraction
    // stays >= 0.5 / WT away from an integer)
    const float iwt = 1.0f / (float)WT;
    for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
        const int k = idx / CH, ch = idx - k * CH;
        const int cv = (int)(((float)k + 0.5f) * iwt), cu = k - cv * WT;
        const int gxw = bc_wrap(X0 - HALO + cu, p.nx, p.bcx);
        const int gyw = bc_wrap(Y0 - HALO + cv, p.ny, p.bcy);
        const R *src = in + ((size_t)gyw * p.nx + gxw) * SL + ch * (16 / sizeof(R));
        cp_async16(tile + (cv * PT + cu) * TS + ch * (16 / sizeof(R)), src);
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
}

// One time step of one tile (block) of a simulation: the body of both step kernels.
// tile: the block's staged tile (`staged`: its copies were issued and waited for by the
// caller, else they are issued here); part: the per-lane partials.
template <typename R, int LPN>
__device__ __forceinline__ void step_tile(const DevParams &p, const R *__restrict__ in,
                                          R *__restrict__ out, DevStats *stats, int tile_idx,
                                          const R *nlsrc, R *tile, R *part_base, bool staged,
                                          const CUtensorMap *tmap = nullptr)
{
    static_assert(LPN == 8 || LPN == 16, "8 or 16 lanes per node");
    constexpr int PPL = 16 / LPN;   // stencil positions per lane and direction
    __shared__ StepShared<R> sh;
    constexpr int TS = Slot<R>::stride;
    const TypedParams<R> &q = typed<R>(p);
    const int grp = threadIdx.x / LPN, lane = threadIdx.x % LPN;
    const unsigned gmask = (LPN == 8 ? 0xffu : 0xffffu) << (LPN * (grp % (32 / LPN)));
    // tile of TX x TY nodes; node grp at (tx, ty) of the tile
    const int TX = p.tile_x, TY = STEP_NB / TX;
    const int X0 = (tile_idx % p.tiles_x) * TX, Y0 = (tile_idx / p.tiles_x) * TY;
    const int WT = TX + 2 * HALO, HT = TY + 2 * HALO;
    const int PT = step_row_pitch(TX, TS);   // slots per staged row (>= WT)
    const int tx = grp % TX, ty = grp / TX;
    const bool valid = X0 + tx < p.nx && Y0 + ty < p.ny;
    const int X = min(X0 + tx, p.nx - 1), Y = min(Y0 + ty, p.ny - 1);
    const long long n = (long long)Y * p.nx + X;
    // slot of the unwrapped coordinate (u, v) in the staged tile, or -1 outside it
    auto slot_of = [&](int u, int v) -> int {
        const int cu = u - (X0 - HALO), cv = v - (Y0 - HALO);
        return (cu >= 0 && cu < WT && cv >= 0 && cv < HT) ? cv * PT + cu : -1;
    };

    // ---------------- staging: tile + halo records into shared memory --------------
    {
        const float iwt = 1.0f / (float)WT;
        // A tile whose halo'd box (PT x HT slots) lies inside the grid is one TMA copy of a
        // box of the record tensor [ny][nx][SL] (first TS values of each record); tiles at
        // the grid edges need the periodic wrap or zero-gradient clamp and take the
        // per-chunk cp.async copies.
        const bool tma = tmap != nullptr && X0 - HALO >= 0 && X0 - HALO + PT <= p.nx &&
                         Y0 - HALO >= 0 && Y0 - HALO + HT <= p.ny && (smem_u32(tile) & 127u) == 0;
        if (tma) {
            __shared__ __align__(8) unsigned long long tma_bar;
            __shared__ int tma_ok;
            if (threadIdx.x == 0) {
                mbar_init(&tma_bar, 1);
                mbar_arrive_expect_tx(&tma_bar, (unsigned)(PT * HT * TS * sizeof(R)));
                tma_load_3d(tile, tmap, 0, X0 - HALO, Y0 - HALO, &tma_bar);
                tma_ok = mbar_wait_bounded(&tma_bar, 0, TMA_WAIT_LIMIT_NS) ? 1 : 0;
                if (!tma_ok) atomicAdd(&stats->timeouts, 1ull);
            }
            __syncthreads();
            if (!tma_ok) return;     // the tile is skipped; the sync points report POND_ETIMEOUT
            // every thread observes the completed phase (returns at once), which orders the
            // copied data before its reads
            if (threadIdx.x != 0) mbar_wait_bounded(&tma_bar, 0, TMA_WAIT_LIMIT_NS);
        } else if (!staged) {
            stage_issue<R>(p, in, tile, tile_idx);
            cp_async_wait_all();
            __syncthreads();
        }
        // per staged node, once per step: sqrt(theta) into the slot's spare value, and the
        // vdW pressure and p/rho of the stored rho, T (for the non-local terms) into the
        // slot words past the staged values
        for (int k = threadIdx.x; k < WT * HT; k += blockDim.x) {
            const int cv = (int)(((float)k + 0.5f) * iwt), cu = k - cv * WT;
            R *sl = tile + (cv * PT + cu) * TS;
            sl[P_SQ] = sqrt_(sl[P_TH]);
            R r = sl[P_RHO], t = sl[P_T];
            if (nlsrc != in) {
                // current-time non-local terms: rho, T of the first pass's prediction
                const size_t g = ((size_t)bc_wrap(Y0 - HALO + cv, p.ny, p.bcy) * p.nx +
                                  bc_wrap(X0 - HALO + cu, p.nx, p.bcx)) * SL;
                r = nlsrc[g + P_RHO];
                t = nlsrc[g + P_T];
                sl[P_RHO] = r;
                sl[P_T] = t;
            }
            const R pr = eos_pressure<R>(p.eos_kind, q.a, q.b, q.R, r, t, typed_sp<R>(p));
            sl[S_PR] = pr;
            sl[S_PRR] = fdiv_(pr, r);
        }
        __syncthreads();
    }

    // ---------------- phase 0: non-local terms, own populations --------------------
    R Fx = 0, Fy = 0, M0 = 0, rEl = 0;
    {
        // lane -> non-rest neighbour (cx, cy); index skips the rest direction 4, so the
        // opposite neighbour (-cx, -cy) sits on lane 7 - l
        const int l8 = lane & 7;
        const int dir = l8 < 4 ? l8 : l8 + 1;
        const int cx = dir % 3 - 1, cy = dir / 3 - 1;
        // the neighbour in unwrapped tile coordinates; a zero-gradient edge clamps it onto
        // the grid first (its stencil is that of the boundary node itself)
        const int mx = p.bcx == 0 ? X0 + tx + cx : bc_wrap(X0 + tx + cx, p.nx, 1);
        const int my = p.bcy == 0 ? Y0 + ty + cy : bc_wrap(Y0 + ty + cy, p.ny, 1);
        // mx + ex, my + ey (|e| <= 1) lie within 2 nodes of the tile, inside the staged
        // halo: slots by direct offsets from the neighbour's own slot
        const int s0 = (my - (Y0 - HALO)) * PT + (mx - (X0 - HALO));
        const R *c0 = tile + s0 * TS;
        const R r0 = c0[P_RHO], t0 = c0[P_T];
        const R pr0 = c0[S_PR], prr0 = c0[S_PRR];
        // gradients from differences to the centre value (sum_i W_i c_i = 0), which keeps
        // their FP32 rounding proportional to the differences
        R grx = 0, gry = 0, lap = 0, ghx = 0, ghy = 0, gTx = 0, gTy = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const int ex = i % 3 - 1, ey = i / 3 - 1;
            if (ex == 0 && ey == 0) continue;
            const R *cm = c0 + (ey * PT + ex) * TS;
            const R w = wst<R>(ex, ey);
            const R r = cm[P_RHO], t = cm[P_T];
            const R dr = r - r0, dT = t - t0;
            const R dh = q.cv * dT - q.a * dr + (cm[S_PRR] - prr0);
            grx += w * R(ex) * dr;
            gry += w * R(ey) * dr;
            lap += w * dr;
            ghx += w * R(ex) * dh;
            ghy += w * R(ey) * dh;
            gTx += w * R(ex) * dT;
            gTy += w * R(ey) * dT;
        }
        grx *= R(3); gry *= R(3); lap *= R(6);
        ghx *= R(3); ghy *= R(3); gTx *= R(3); gTy *= R(3);
        const R kap = q.kappa;
        const R iso = -kap * (r0 * lap + R(0.5) * (grx * grx + gry * gry));
        const R Kxx = iso + kap * grx * grx, Kxy = kap * grx * gry, Kyy = iso + kap * gry * gry;
        const R P0 = pr0 > q.p_floor ? pr0 : q.p_floor;
        const R mu = q.mu_coef * P0;
        const R kc = q.k_cond >= R(0) ? q.k_cond : mu * q.cvR;
        const R qx = -mu * ghx + kc * gTx, qy = -mu * ghy + kc * gTy;
        const R w = lane < 8 ? wst<R>(cx, cy) : R(0);
        // divergences from the difference to the opposite neighbour (lane 7 - l); each
        // opposite pair is counted by both of its lanes, hence the halved factors
        const int opp = 7 - l8;
        const R Kxx_o = __shfl_sync(gmask, Kxx, opp, LPN), Kxy_o = __shfl_sync(gmask, Kxy, opp, LPN);
        const R Kyy_o = __shfl_sync(gmask, Kyy, opp, LPN);
        const R qx_o = __shfl_sync(gmask, qx, opp, LPN), qy_o = __shfl_sync(gmask, qy, opp, LPN);
        const R r_o = __shfl_sync(gmask, r0, opp, LPN);
        Fx = -R(1.5) * w * (R(cx) * (Kxx - Kxx_o) + R(cy) * (Kxy - Kxy_o));
        Fy = -R(1.5) * w * (R(cx) * (Kxy - Kxy_o) + R(cy) * (Kyy - Kyy_o));
        M0 = R(3) * w * (R(cx) * (qx - qx_o) + R(cy) * (qy - qy_o));
        R gxn = R(1.5) * w * R(cx) * (r0 - r_o), gyn = R(1.5) * w * R(cy) * (r0 - r_o);
#pragma unroll
        for (int o = LPN / 2; o > 0; o >>= 1) {
            Fx += __shfl_xor_sync(gmask, Fx, o, LPN);
            Fy += __shfl_xor_sync(gmask, Fy, o, LPN);
            M0 += __shfl_xor_sync(gmask, M0, o, LPN);
            gxn += __shfl_xor_sync(gmask, gxn, o, LPN);
            gyn += __shfl_xor_sync(gmask, gyn, o, LPN);
        }
        rEl = R(0.5) * kap * (gxn * gxn + gyn * gyn);
    }
    const R *own = tile + slot_of(X0 + tx, Y0 + ty) * TS;
    // the node's own populations are read from its staged slot where needed (holding
    // them in 18 registers through the stream loop cost more than the shared loads)
    if (lane == 0) {
        sh.lam[grp][0] = own[P_TH];
        sh.lam[grp][1] = own[P_UX];
        sh.lam[grp][2] = own[P_UY];
        sh.nl[grp][0] = Fx;
        sh.nl[grp][1] = Fy;
        sh.nl[grp][2] = rEl;
        sh.active[grp] = valid ? 1 : 0;
        sh.nreg[grp] = 0;
        sh.npair[grp] = 0;
    }
    if (threadIdx.x < STEP_NB) {
        // exact FP64 sums of node j's stored populations, one node per lane of warp 0
        // (error-free in R: TwoSum cascades, each sum kept as an unevaluated (hi, lo) pair
        // and rounded once to FP64, which keeps the FP64 pipe free in the FP32 form)
        const R *rj = tile + slot_of(X0 + threadIdx.x % TX, Y0 + threadIdx.x / TX) * TS;
        // the stored low parts of mass, momentum and energy (not staged) start the error terms
        const R *gj = in + ((size_t)min(Y0 + (int)threadIdx.x / TX, p.ny - 1) * p.nx +
                            min(X0 + (int)threadIdx.x % TX, p.nx - 1)) * SL;
        R hi[4] = {R(0), R(0), R(0), R(0)}, lo[4] = {gj[P_F4LO], gj[P_JXLO], gj[P_JYLO], gj[P_G4LO]};
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            const R f = rj[P_F + i], gv = rj[P_G + i];
            const R terms[4] = {f, R(i % 3 - 1) * f, R(i / 3 - 1) * f, gv};
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                if (k == 1 && i % 3 == 1) continue;
                if (k == 2 && i / 3 == 1) continue;
                R e;
                two_sum_(hi[k], terms[k], hi[k], e);
                lo[k] += e;
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            sh.bhi[threadIdx.x][k] = hi[k];
            sh.blo[threadIdx.x][k] = lo[k];
        }
    }
    if (threadIdx.x == 0) sh.any_active = 1;
    __syncthreads();

    // ---------------- phase 1: frame search (block lockstep) -----------------------
    // part: this lane's partial increments of the node's 18 populations in the latest stream
    R *part = part_base + grp * step_part_stride(LPN) + lane;
    int it = 0;                                   // iterations of this block
    int my_it = 0, my_conv = 0, my_stall = 0;     // warp-0 lane bookkeeping for node threadIdx.x
    float my_res = 3.0e38f;                       // previous residual of that node
    const int kk = lane & 3, m1 = (lane >> 2) & 3, m2 = m1 + 2;
    while (sh.any_active && it < p.max_iter) {
        ++it;
        if (sh.active[grp]) {
            const R th = sh.lam[grp][0], ux = sh.lam[grp][1], uy = sh.lam[grp][2];
            const R s = sqrt_(th), inv_s = R(1) / s;
            R a0 = 0, a1 = 0, a2 = 0, a3 = 0;
            // Departure points x - v_i dt of the directions of each axis (the x part depends
            // on jx only, the y part on jy only): stencil start floor(.) - 1 and the
            // Lagrange coordinate xi in [1, 2).  The node's region is the union of its
            // directions' 4x4 stencils: (4 + spread of the floors) per axis.
            // Offsets are clamped to +-2^20 nodes first (a NaN offset goes to the bound):
            // with a non-finite or runaway gauge the floors and their spread stay in int
            // range, so the region is always 4..8 wide when taken and its indices stay
            // inside the weight tables.
            int fl[2][3];
            R xi[2][3];
#pragma unroll
            for (int ax = 0; ax < 2; ++ax)
#pragma unroll
                for (int j = 0; j < 3; ++j) {
                    const R d = clamp_offset(-(s * R(j - 1) + (ax == 0 ? ux : uy)) * q.dt);
                    const R f = floor(d);
                    fl[ax][j] = (int)f;
                    xi[ax][j] = d - f + R(1);
                }
            const int lo_x = min(fl[0][0], min(fl[0][1], fl[0][2]));
            const int lo_y = min(fl[1][0], min(fl[1][1], fl[1][2]));
            const int ncols = 4 + max(fl[0][0], max(fl[0][1], fl[0][2])) - lo_x;
            const int nrows = 4 + max(fl[1][0], max(fl[1][1], fl[1][2])) - lo_y;
            if (ncols <= REGION_MAX && nrows <= REGION_MAX) {
                // weight tables: lane c < 8 fills region column c and region row c
                if (lane < REGION_MAX) {
#pragma unroll
                    for (int ax = 0; ax < 2; ++ax) {
                        const int n_ax = ax == 0 ? ncols : nrows, lo = ax == 0 ? lo_x : lo_y;
                        if (lane < n_ax) {
                            R w4[4];
#pragma unroll
                            for (int j = 0; j < 3; ++j) {
                                const int kk2 = lane - (fl[ax][j] - lo);
                                w4[j] = (kk2 >= 0 && kk2 < 4) ? lag1_rt<R>(kk2, xi[ax][j]) : R(0);
                            }
                            w4[3] = R(0);
                            R *dst = sh.wt[grp][ax][lane];
#pragma unroll
                            for (int j = 0; j < 4; ++j) dst[j] = w4[j];
                        }
                    }
                }
                __syncwarp(gmask);
                if (lane == 0) sh.nreg[grp] += ncols * nrows - ((it == 1 && lo_x <= 1 && 1 - lo_x < ncols &&
                                                                   lo_y <= 1 && 1 - lo_y < nrows) ? 1 : 0);
                R accf[9], accg[9];
#pragma unroll
                for (int i = 0; i < 9; ++i) accf[i] = accg[i] = R(0);
                const int x_lo = X + lo_x - 1, y_lo = Y + lo_y - 1;
                // In the first stream the arrival gauge is the node's own stored gauge, so
                // its own region entry is carried by the identity and adds exactly nothing
                // in the FP32 increment form (about 1e-16 in FP64): it is skipped, which
                // makes the usual 5 x 5 region 24 entries, three full passes of 8 lanes.
                const int own_r = (1 - lo_y) * ncols + (1 - lo_x);
                const bool skip_own = it == 1 && lo_x <= 1 && 1 - lo_x < ncols && lo_y <= 1 && 1 - lo_y < nrows;
                const int nreg = ncols * nrows - (skip_own ? 1 : 0);
                const float inc = 1.0f / (float)ncols;
                // the whole region inside the staged tile (always for |v| dt < 1): slots by
                // direct indexing from its corner, else per node with a global fallback
                const int cu0 = x_lo - (X0 - HALO), cv0 = y_lo - (Y0 - HALO);
                const bool staged_region = cu0 >= 0 && cu0 + ncols <= WT && cv0 >= 0 && cv0 + nrows <= HT;
                const R *corner = staged_region ? tile + (cv0 * PT + cu0) * TS : tile;
                // region nodes round-robin over the group's lanes
#pragma unroll 1
                for (int rr = lane; rr < nreg; rr += LPN) {
                    const int r = rr + (skip_own && rr >= own_r ? 1 : 0);
                    const int cy = (int)(((float)r + 0.5f) * inc), cx = r - cy * ncols;
                    R v[24];
                    if (staged_region) {
                        load_slot24(corner + (cy * PT + cx) * TS, v);
                    } else {
                        const int sl = slot_of(x_lo + cx, y_lo + cy);
                        if (sl >= 0) {
                            load_slot24(tile + sl * TS, v);
                        } else {
                            const size_t nd = (size_t)bc_wrap(y_lo + cy, p.ny, p.bcy) * p.nx +
                                              bc_wrap(x_lo + cx, p.nx, p.bcx);
                            load_rec24(in + nd * SL, v);
                            v[P_SQ] = sqrt_(v[P_TH]);
                        }
                    }
                    const R thn = v[P_TH], sn = v[P_SQ];
                    const R qm1 = sizeof(R) == 8 ? sn * inv_s - R(1) : fdiv_(thn - th, (sn + s) * s);
                    const R wxg = (v[P_UX] - ux) * inv_s, wyg = (v[P_UY] - uy) * inv_s;
                    // transfer increments per axis from h = e/2 and p = h (2 c_a + e):
                    // E_0 = p - h, E_1 = -2 p, E_2 = p + h (the three l_k increments)
                    R Ex[3][3], Ey[3][3];
#pragma unroll
                    for (int a = 0; a < 3; ++a) {
                        const R ex = qm1 * R(a - 1) + wxg, ey = qm1 * R(a - 1) + wyg;
                        const R hx = R(0.5) * ex, hy = R(0.5) * ey;
                        const R px = hx * (R(2 * (a - 1)) + ex), py = hy * (R(2 * (a - 1)) + ey);
                        Ex[0][a] = px - hx; Ex[1][a] = R(-2) * px; Ex[2][a] = px + hx;
                        Ey[0][a] = py - hy; Ey[1][a] = R(-2) * py; Ey[2][a] = py + hy;
                    }
                    R wx[3], wy[3];
                    {
                        const R *px = sh.wt[grp][0][cx], *py = sh.wt[grp][1][cy];
#pragma unroll
                        for (int j = 0; j < 3; ++j) {
                            wx[j] = px[j];
                            wy[j] = py[j];
                        }
                    }
                    // the node's own populations from its staged slot (16-byte loads)
                    R ov[24];
                    load_slot24(own, ov);
                    region_family<R>(v + P_F, ov + P_F, Ex, Ey, wx, wy, accf);
                    region_family<R>(v + P_G, ov + P_G, Ex, Ey, wx, wy, accg);
                }
#pragma unroll
                for (int i = 0; i < 9; ++i) {
                    part[i * LPN] = accf[i];
                    part[(9 + i) * LPN] = accg[i];
                    a0 += accf[i];
                    if (i % 3 == 0) a1 -= accf[i];
                    if (i % 3 == 2) a1 += accf[i];
                    a2 += accf[i] * R(i / 3 - 1);
                    a3 += accg[i];
                }
            } else {
            if (lane == 0) sh.npair[grp] += 1;
            // per-pair stream for wide regions (|v| dt of 2 nodes or more): rows of
            // directions (jy) in a rolled loop, the three directions of a row unrolled so
            // that their transfer coefficients are compile-time selections
#pragma unroll 1
            for (int jy = 0; jy < 3; ++jy) {
                R fxr[3], gxr[3];   // own populations of this row of directions
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    fxr[a] = own[P_F + 3 * jy + a];
                    gxr[a] = own[P_G + 3 * jy + a];
                }
                const R dy = clamp_offset(-(s * R(jy - 1) + uy) * q.dt);
                const R fly = floor(dy);
                const int y0 = Y + (int)fly - 1;
                const R eta = dy - fly + R(1);
#pragma unroll
                for (int jx = 0; jx < 3; ++jx) {
                    const int i = 3 * jy + jx;
                    const R dx = clamp_offset(-(s * R(jx - 1) + ux) * q.dt);
                    const R flx = floor(dx);
                    const int x0 = X + (int)flx - 1;
                    const R ax = lag1<R>(kk, dx - flx + R(1));
                    R vf = 0, vg = 0;
#pragma unroll
                    for (int pp = 0; pp < PPL; ++pp) {
                        const int mm = pp == 0 ? m1 : m2;
                        const int sl = slot_of(x0 + kk, y0 + mm);
                        R v[24];
                        if (sl >= 0) {
                            load_slot24(tile + sl * TS, v);
                        } else {
                            const size_t nd = (size_t)bc_wrap(y0 + mm, p.ny, p.bcy) * p.nx +
                                              bc_wrap(x0 + kk, p.nx, p.bcx);
                            load_rec24(in + nd * SL, v);
                            v[P_SQ] = sqrt_(v[P_TH]);
                        }
                        R tf, tg;
                        pair_inc<R>(v, jx, jy, th, s, inv_s, ux, uy, fxr[jx], gxr[jx], tf, tg);
                        const R ay = lag1<R>(mm, eta);
                        vf += ay * tf;
                        vg += ay * tg;
                    }
                    vf *= ax;
                    vg *= ax;
                    // this lane's partials: kept for the collision (the node's last stream
                    // leaves them in place) and summed into the moments right away
                    part[i * LPN] = vf;
                    part[(9 + i) * LPN] = vg;
                    a0 += vf;
                    if (jx == 0) a1 -= vf;
                    if (jx == 2) a1 += vf;
                    a2 += vf * R(jy - 1);
                    a3 += vg;
                }
            }
            }
#pragma unroll
            for (int o = LPN / 2; o > 0; o >>= 1) {
                a0 += __shfl_xor_sync(gmask, a0, o, LPN);
                a1 += __shfl_xor_sync(gmask, a1, o, LPN);
                a2 += __shfl_xor_sync(gmask, a2, o, LPN);
                a3 += __shfl_xor_sync(gmask, a3, o, LPN);
            }
            if (lane == 0) {
                sh.dsum[grp][0] = a0; sh.dsum[grp][1] = a1; sh.dsum[grp][2] = a2; sh.dsum[grp][3] = a3;
            }
        }
        __syncthreads();
        // warp 0: moments, e -> T, EoS, residual for node j = threadIdx.x, in FP64 (FP64
        // form) or float-float (FP32 form)
        if (threadIdx.x < STEP_NB) {
            const int j = threadIdx.x;
            if (sh.active[j]) {
                const R thr = sh.lam[j][0];
                const R sr = sqrt_(thr);
                EosOut<R> o;
                eos_update(p, sh.bhi[j], sh.blo[j], sh.dsum[j], sh.nl[j], sh.lam[j], sr, o);
                // relative change of the gauge
                const float rth = fabsf((float)o.dth) / (float)thr;
                const float rux = fabsf((float)o.dux) / (float)sr, ruy = fabsf((float)o.duy) / (float)sr;
                const float res = fmaxf(rth, fmaxf(rux, ruy));
                const bool conv = sizeof(R) == 4 ? res <= p.tol_f : (double)res <= p.tol;
                const bool bad = !(res == res);
                // FP32 form only: the streamed moments carry FP32 rounding that the EoS
                // cancellation inside interfaces can lift above tol; once a corrector no
                // longer halves the residual the iteration has reached that floor and stops.
                // Only a residual within STALL_TOL_FACTOR x tol counts as that floor: a larger
                // one that fails to halve once (the pressure floor's kink in
                // theta* = max(p, p_floor)/(rho T_L) can do that) keeps iterating, since
                // stopping there left the gauge up to 8 % off and single steps 3.6e-3 off the
                // converged result inside a compressed sub-spinodal droplet.
                const bool stall = sizeof(R) == 4 && it >= 2 && !conv && res > 0.5f * my_res &&
                                   res < STALL_TOL_FACTOR * p.tol_f;
                my_res = res;
                my_it = it;
                if (conv || bad || stall || it >= p.max_iter) {
                    sh.active[j] = 0;
                    my_conv = conv || stall;
                    my_stall = stall;
                    R *m = sh.mac[j];
                    m[0] = o.rho_hi; m[1] = o.uxs; m[2] = o.uys; m[3] = o.uhx; m[4] = o.uhy;
                    m[5] = o.E; m[6] = o.T; m[7] = o.P; m[8] = o.ths; m[9] = o.pr;
                    sh.dlam[j][0] = o.dth; sh.dlam[j][1] = o.dux; sh.dlam[j][2] = o.duy;
                    sh.hilo[j][0] = o.rho_hi; sh.hilo[j][1] = o.rho_lo;
                    sh.hilo[j][2] = o.gs_hi; sh.hilo[j][3] = o.gs_lo;
                    sh.mom[j][0] = o.mx_hi; sh.mom[j][1] = o.mx_lo;
                    sh.mom[j][2] = o.my_hi; sh.mom[j][3] = o.my_lo;
                } else {
                    sh.lam[j][0] = o.ths;
                    sh.lam[j][1] = o.uxs;
                    sh.lam[j][2] = o.uys;
                }
            }
            const int any = __any_sync(STEP_NB_MASK, sh.active[j]);
            if (j == 0) sh.any_active = any;
        }
        __syncthreads();
    }

    // ---------------- phase 2: collision (one population per lane) -----------------
    if (valid) {
        // Population `pop` of this lane.  The rest population (4) is stored as the exact
        // remainder of mass and energy, so with 8 lanes per node lane 4 takes population 8
        // instead; with 16, lanes 0..8 take their own index (lane 4's result is replaced).
        const int pop = (LPN == 8 && lane == 4) ? 8 : (lane < 9 ? lane : 8);
        const bool owner = lane < 9 && pop != 4;
        // its increment from the node's final stream: the sum of the lanes' partials, read
        // in a lane-rotated order so that the rows fall on different banks
        R my_df = 0, my_dg = 0;
        {
            const R *row = part - lane;
#pragma unroll
            for (int l = 0; l < LPN; ++l) {
                const int ll = (l + lane) & (LPN - 1);
                my_df += row[pop * LPN + ll];
                my_dg += row[(9 + pop) * LPN + ll];
            }
        }
        const R th = sh.lam[grp][0], ux = sh.lam[grp][1], uy = sh.lam[grp][2];
        const R s = sqrt_(th), inv_s = R(1) / s;
        const R *m = sh.mac[grp];
        const R rr = m[0], uxr = m[1], uyr = m[2], uhxr = m[3], uhyr = m[4], Er = m[5];
        const R Pr = m[7], thsr = m[8];
        const R sst = sqrt_(thsr);
        const R qm1 = sizeof(R) == 8 ? sst * inv_s - R(1) : fdiv_(sh.dlam[grp][0], (sst + s) * s);
        const R wsx = sh.dlam[grp][1] * inv_s, wsy = sh.dlam[grp][2] * inv_s;
        const R dtr = q.dt, om = q.omega;
        const R irr = frcp_(rr), iP2 = frcp_(R(2) * Pr);
        const R dvx = Fx * dtr * irr * inv_s, dvy = Fy * dtr * irr * inv_s;
        const R W1[3] = {wlat<R>(0), wlat<R>(1), wlat<R>(2)};
        // transfer increments from lambda* = (ths, u*) into the streaming gauge, and from the
        // force-shifted frame (ths, u* + F dt/rho) (Eq. S-i), for the row k of one axis:
        // E[a] = l_k increments at the source velocities, Ws = sum_a E[a] W_a, Wh = the
        // force-shifted frame's extra weight
        auto row = [&](int k, R w, R dv, R (&E)[3], R &Ws, R &Wh) {
            Ws = 0;
            Wh = 0;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                E[a] = ell_inc_rt<R>(k, a, qm1 * R(a - 1) + w);
                Ws += E[a] * W1[a];
                Wh += (ell_inc_rt<R>(k, a, qm1 * R(a - 1) + w + dv) - E[a]) * W1[a];
            }
        };
        // g: forced equilibrium (Eq. new geq), heat-flux correction (Eq. gtilde) and the
        // force-work source 2 W_i uhat.F, all in lambda*, in every lane (9 values)
        const R H = Er + Pr * irr;
        const R Ixx = R(2) * uhxr * Fx + dtr * Fx * Fx * Er * iP2;
        const R Ixy = uhxr * Fy + Fx * uhyr + dtr * Fx * Fy * Er * iP2;
        const R Iyy = R(2) * uhyr * Fy + dtr * Fy * Fy * Er * iP2;
        const R cM = R(2) * dtr * rr * iP2;
        const R Mx = cM * (Fx * H - (Ixx * uxr + Ixy * uyr));
        const R My = cM * (Fy * H - (Ixy * uxr + Iyy * uyr));
        const R cN = dtr * rr * iP2;
        const R Nxx = rr + cN * Ixx, Nxy = cN * Ixy, Nyy = rr + cN * Iyy;
        // P/rho in the g equilibrium as sqrt(theta*)^2 times the lattice temperature of
        // the weights in use (sum_i W_i c_ix^2 = 2 W_+-1), so that the equilibrium's zeroth
        // moment is 2 rho E to rounding also in FP32 (sum_i W_i (v_x^2 - P/rho - u_x^2) = 0)
        const R Pd = sst * sst * (R(2) * W1[0]);
        const R work = R(2) * (uhxr * Fx + uhyr * Fy);
        // X*_i for this lane's population(s) only, then gathered across the group
        auto xstar = [&](int i) -> R {
            const int ix = i % 3, iy = i / 3;
            const R cx = R(ix - 1), cy = R(iy - 1);
            const R w = pick(W1, ix) * pick(W1, iy);
            const R ccx = sst * cx, ccy = sst * cy;                  // v - u* in lambda*
            const R Axx = ccx * ccx + R(2) * ccx * uxr - Pd;          // v v - P/rho I - u u
            const R Axy = ccx * ccy + ccx * uyr + ccy * uxr;
            const R Ayy = ccy * ccy + R(2) * ccy * uyr - Pd;
            const R geq = w * (R(2) * rr * Er + Mx * ccx + My * ccy + Nxx * Axx + R(2) * Nxy * Axy + Nyy * Ayy);
            const R vx = ccx + uxr, vy = ccy + uyr;
            const R uc = uxr * cx + uyr * cy;
            const R gc = M0 * w * (R(1) + rr * uc * uc * iP2 * R(3)
                                   - rr * (vx * vx + vy * vy) * iP2 + R(1));
            return om * geq + dtr * (gc + w * work);
        };
        const R my_x = xstar(pop);
        const R x4 = LPN == 8 ? xstar(4) : R(0);   // no lane holds population 4 then
        R Xs[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            if (LPN == 8) Xs[k] = k == 4 ? x4 : __shfl_sync(gmask, my_x, k == 8 ? 4 : k, LPN);
            else Xs[k] = __shfl_sync(gmask, my_x, k, LPN);
        }
        R fo, go;
        {
            {
                const int i = pop;
                const int kx = i % 3, ky = i / 3;
                const R ft = own[P_F + i] + my_df, gt = own[P_G + i] + my_dg;
                R exk[3], eyl[3], Wsk, Wsl, Whk, Whl;
                row(kx, wsx, dvx, exk, Wsk, Whk);
                row(ky, wsy, dvy, eyl, Wsl, Whl);
                const R W1k = pick(W1, kx), W1l = pick(W1, ky);
                const R Wx = W1k + Wsk, Wy = W1l + Wsl;
                // f^eq - f~ with the frame-offset increments kept apart from the O(1)
                // weights: W + Ws rounded in FP32 would keep only the increment's leading
                // bits (Ws ~ the gauge change of one step, a few ulps of W), and always the
                // same way, since W is a constant
                const R dfeq = (rr * W1k * W1l - ft) + rr * (Wsk * W1l + W1k * Wsl + Wsk * Wsl);
                const R S = rr * (Whk * (Wy + Whl) + Wx * Whl);
                fo = ft + om * dfeq + S;
                // carry X* into the streaming gauge: X = X* + (G* - I) X*
                R acc = pick(Xs, i);
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    R gyc = 0;
#pragma unroll
                    for (int b = 0; b < 3; ++b) gyc += (eyl[b] + (b == ky ? R(1) : R(0))) * Xs[a + 3 * b];
                    acc += exk[a] * gyc;
                }
                R xcol[3];
#pragma unroll
                for (int b = 0; b < 3; ++b)
                    xcol[b] = kx == 0 ? Xs[3 * b] : (kx == 1 ? Xs[3 * b + 1] : Xs[3 * b + 2]);
#pragma unroll
                for (int b = 0; b < 3; ++b) acc += eyl[b] * xcol[b];
                go = (R(1) - om) * gt + acc;
            }
        }
        // The collision conserves mass exactly and changes the energy by dt (M_0 + 2 uhat.F);
        // the rest population (i = 4) takes the remainder, summed error-free as (hi, lo)
        // pairs, so that the stored populations keep these sums up to one rounding.
        // The stored momentum (exact pair sums of the stored populations) falls short of the
        // exact post-collision momentum sum f~ c + F dt / s by its storage rounding; that
        // difference is kept beside the populations too.
        R f4 = 0, g4 = 0, f4lo = 0, g4lo = 0, jxlo = 0, jylo = 0;
        {
            R fh = owner ? fo : R(0), fl = 0;
            R gh = owner ? go : R(0), gl = 0;
            R xh = owner ? R(pop % 3 - 1) * fo : R(0), xl = 0;
            R yh = owner ? R(pop / 3 - 1) * fo : R(0), yl = 0;
#pragma unroll
            for (int o = LPN / 2; o > 0; o >>= 1) {
                const R fh2 = __shfl_xor_sync(gmask, fh, o, LPN), fl2 = __shfl_xor_sync(gmask, fl, o, LPN);
                const R gh2 = __shfl_xor_sync(gmask, gh, o, LPN), gl2 = __shfl_xor_sync(gmask, gl, o, LPN);
                const R xh2 = __shfl_xor_sync(gmask, xh, o, LPN), xl2 = __shfl_xor_sync(gmask, xl, o, LPN);
                const R yh2 = __shfl_xor_sync(gmask, yh, o, LPN), yl2 = __shfl_xor_sync(gmask, yl, o, LPN);
                R e;
                two_sum_(fh, fh2, fh, e);
                fl = fl + fl2 + e;
                two_sum_(gh, gh2, gh, e);
                gl = gl + gl2 + e;
                two_sum_(xh, xh2, xh, e);
                xl = xl + xl2 + e;
                two_sum_(yh, yh2, yh, e);
                yl = yl + yl2 + e;
            }
            if (lane == 4) {
                // target sums: rho (hi, lo) and sum g~ + dt (M_0 + work)
                R th_, tl_;
                two_sum_(sh.hilo[grp][2], dtr * (M0 + work), th_, tl_);
                tl_ += sh.hilo[grp][3];
                // the remainders as (hi, lo) pairs: hi is stored as the population, lo
                // beside it for the next step's sums
                R s1, e1;
                two_sum_(sh.hilo[grp][0], -fh, s1, e1);
                two_sum_(s1, e1 + (sh.hilo[grp][1] - fl), f4, f4lo);
                two_sum_(th_, -gh, s1, e1);
                two_sum_(s1, e1 + (tl_ - gl), g4, g4lo);
                jxlo = ((sh.mom[grp][0] - xh) + (sh.mom[grp][1] - xl)) + Fx * dtr * inv_s;
                jylo = ((sh.mom[grp][2] - yh) + (sh.mom[grp][3] - yl)) + Fy * dtr * inv_s;
            }
        }
        if (owner) {
            REC(out, n, P_F + pop) = fo;
            REC(out, n, P_G + pop) = go;
        }
        if (lane == 4) {
            REC(out, n, P_F + 4) = f4;
            REC(out, n, P_G + 4) = g4;
            REC(out, n, P_F4LO) = f4lo;
            REC(out, n, P_G4LO) = g4lo;
            REC(out, n, P_JXLO) = jxlo;
            REC(out, n, P_JYLO) = jylo;
        }
        if (lane == 0) {
            REC(out, n, P_TH) = th;
            REC(out, n, P_UX) = ux;
            REC(out, n, P_UY) = uy;
            REC(out, n, P_RHO) = rr;
            REC(out, n, P_T) = m[6];
            REC(out, n, P_UHX) = uhxr;
            REC(out, n, P_UHY) = uhyr;
        }
    }
    // ---------------- statistics (warp 0, one lane per node) -----------------------
    if (threadIdx.x < STEP_NB) {
        const int j = threadIdx.x;
        const bool v = X0 + j % TX < p.nx && Y0 + j / TX < p.ny;
        const R T = sh.mac[j][6], rr = sh.mac[j][0], pr = sh.mac[j][9];
        warp_add(&stats->streams, v ? my_it : 0);
        warp_add(&stats->region_nodes, v ? sh.nreg[j] : 0);
        warp_add(&stats->pair_streams, v ? sh.npair[j] : 0);
        warp_add(&stats->nonconv, (v && !my_conv) ? 1 : 0);
        warp_add(&stats->stalled, (v && my_stall) ? 1 : 0);
        warp_add(&stats->clamped, (v && pr < q.p_floor) ? 1 : 0);
        const bool bad = v && (!(rr == rr) || !(T == T) || isinf(rr) || isinf(T));
        warp_add(&stats->nonfinite, bad ? 1 : 0);
        if (j == 0) {
            atomicAdd(&stats->block_streams, (unsigned long long)it);
            atomicMax(&stats->max_streams, (unsigned long long)it);
        }
    }
}

// One time step of one simulation: one block per tile.  (A persistent variant that
// prefetched its next tile into a second staging buffer was slower on GB300: 2.64 against
// 2.41 ms on the 2048 x 1024 droplet-shock; the block scheduler already overlaps one
// block's staging with the others' work, and the second buffer takes L1 capacity.)
// tmap: tensor map of `in` for the TMA staging of interior tiles (use_tma = 0: every tile
// takes the per-chunk copies).
template <typename R, int LPN>
__global__ void __launch_bounds__(STEP_NB *LPN, STEP_MIN_BLOCKS(R, LPN)) k_pond_step(DevParams p, const R *__restrict__ in,
                                                             R *__restrict__ out, DevStats *stats,
                                                             const R *nlsrc, const __grid_constant__ CUtensorMap tmap,
                                                             int use_tma)
{
    extern __shared__ __align__(128) unsigned char step_dyn_smem[];
    R *tile = reinterpret_cast<R *>(step_dyn_smem);
    step_tile<R, LPN>(p, in, out, stats, blockIdx.x, nlsrc, tile,
                      tile + (size_t)step_tile_slots(p.tile_x, Slot<R>::stride) * Slot<R>::stride, false,
                      use_tma ? &tmap : nullptr);
}

// A simulation of a batch as one launch sees it: parameters, the buffers this step reads
// and writes, and its counters.
template <typename R>
struct SimDesc {
    DevParams p;
    const R *in;
    R *out;
    DevStats *stats;
};

// One time step of every simulation of a batch in one launch: block b steps tile
// work[b].y of simulation work[b].x (a device work-list of (simulation, tile) pairs).
template <typename R, int LPN>
__global__ void __launch_bounds__(STEP_NB *LPN, STEP_MIN_BLOCKS(R, LPN)) k_pond_step_batch(const SimDesc<R> *__restrict__ descs,
                                                                   const int2 *__restrict__ work)
{
    __shared__ DevParams sp;
    __shared__ const R *s_in;
    __shared__ R *s_out;
    __shared__ DevStats *s_stats;
    const int2 w = work[blockIdx.x];
    if (threadIdx.x == 0) {
        sp = descs[w.x].p;
        s_in = descs[w.x].in;
        s_out = descs[w.x].out;
        s_stats = descs[w.x].stats;
    }
    __syncthreads();
    extern __shared__ __align__(128) unsigned char step_dyn_smem[];
    R *tile = reinterpret_cast<R *>(step_dyn_smem);
    step_tile<R, LPN>(sp, s_in, s_out, s_stats, w.y, s_in, tile,
                      tile + (size_t)step_tile_slots(sp.tile_x, Slot<R>::stride) * Slot<R>::stride, false);
}

}  // namespace pond
