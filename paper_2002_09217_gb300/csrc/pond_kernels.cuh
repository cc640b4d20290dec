// pond_kernels.cuh -- device code of the PonD van der Waals time step for sm_103a.
//
// Layout: a state buffer holds one record of SL = 32 values per node (node = y*nx + x),
// 128 bytes in FP32 so that a node is one cache line and its 21 streamed values are read
// with six 16-byte loads:
//   [0..8] f_0..f_8, [9..17] g_0..g_8, [18] theta, [19] u_x, [20] u_y, [21] spare,
//   [22] rho, [23] T, [24] uhat_x, [25] uhat_y, [26] f_4 lo, [27] g_4 lo, [28] j_x lo,
//   [29] j_y lo, [30..31] unused
// where the lo values are what storage rounding took from the conserved sums: f_4 lo and
// g_4 lo the remainders of the rest populations (which hold the exact remainder of mass
// and energy), j lo the difference between the exact post-collision momentum and that of
// the stored populations.  The next step's exact sums add them back, so changes smaller
// than half an ulp of the populations (which FP32 storage alone would drop every step at
// the weak edge of a wave) are kept.
// with population index i = 3*(cy+1) + (cx+1).  R = float (mixed form) or double.
// The ABI's state planes (f, g, theta, u_x, u_y, rho, T, uhat_x, uhat_y) map to record
// offsets by rec_off().
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pond {

constexpr int NPL = 25;   // planes of the ABI state
constexpr int SL = 32;    // values per node record on the device
enum : int { P_F = 0, P_G = 9, P_TH = 18, P_UX = 19, P_UY = 20, P_SQ = 21, P_RHO = 22, P_T = 23,
             P_UHX = 24, P_UHY = 25, P_F4LO = 26, P_G4LO = 27, P_JXLO = 28, P_JYLO = 29 };
// (P_SQ: sqrt(theta) in the staged copies)
__host__ __device__ constexpr int rec_off(int plane) { return plane < 21 ? plane : plane + 1; }
// value `off` of node n's record
#define REC(buf, n, off) (buf)[(size_t)(n) * SL + (off)]

// Model constants in the arithmetic type of a kernel (float copies keep FP64 work out of
// the FP32 paths).
template <typename T>
struct TypedParams {
    T a, b, R, cv, inv_cv, kappa, p_floor, dt, omega;
    T mu_coef;   // (tau - 1/2) dt, so that mu = mu_coef * P
    T cvR;       // C_v + R (default conductivity k = mu (C_v + R))
    T k_cond;    // >= 0: fixed conductivity
};

struct DevParams {
    int nx, ny, bcx, bcy;
    long long N;
    double a, b, R, delta, cv;
    double kappa, tau, omega, dt, k_cond, p_floor, tol;
    int max_iter;
    int tile_x, tiles_x;   // step kernel tile: tile_x by (16 / tile_x) nodes; tiles per row
    TypedParams<float> pf;
    TypedParams<double> pd;
    // the FP32 form's frame-search EoS constants as (hi, lo) float pairs (hi + lo = the
    // FP64 value to ~2^-48), and its tolerance
    float ff_a[2], ff_b[2], ff_R[2], ff_icv[2], ff_pfl[2];
    float tol_f;
    // equation of state: 0 van der Waals, 2 Dieterici (isothermal only); isothermal runs
    // hold T at T_iso (and ff_Tiso, its float pair)
    int eos_kind, isothermal;
    double T_iso;
    float ff_Tiso[2];
    // double-well constants (eos_kind 3): beta, rho_l, rho_v, p0 (and float copies)
    double sp[4];
    float spf[4], ff_p0[2];
};

template <typename R> __device__ __forceinline__ R exp_(R x);
template <> __device__ __forceinline__ float exp_(float x) { return expf(x); }
template <> __device__ __forceinline__ double exp_(double x) { return exp(x); }

// Pressure part rho E0' - E0 of the double well E0 = beta (rho - rho_l)^2 (rho - rho_v)^2
// (SM "Speed of sound"), from sp = {beta, rho_l, rho_v, p0}.
template <typename R>
__device__ __forceinline__ R well_pressure(const R *sp, R r)
{
    const R dl = r - sp[1], dv = r - sp[2];
    return r * (R(2) * sp[0] * dl * dv * (dl + dv)) - sp[0] * dl * dl * dv * dv;
}

// Pressure p(rho, T) of the run's equation of state in type R: van der Waals
// rho R T/(1 - b rho) - a rho^2 (main text), Dieterici rho R T/(1 - b rho) exp(-a rho/(R T))
// (SM "Coexistence curve") or the double well p0 + rho E0' - E0 (SM "Speed of sound").
template <typename R>
__device__ __forceinline__ R eos_pressure(int kind, R a, R b, R Rg, R r, R t, const R *sp)
{
    if (kind == 2) return r * Rg * t / (R(1) - b * r) * exp_(-a * r / (Rg * t));
    if (kind == 3) return sp[3] + well_pressure<R>(sp, r);
    return r * Rg * t / (R(1) - b * r) - a * r * r;
}

template <typename R> __device__ __forceinline__ const TypedParams<R> &typed(const DevParams &p);
template <> __device__ __forceinline__ const TypedParams<float> &typed<float>(const DevParams &p) { return p.pf; }
template <> __device__ __forceinline__ const TypedParams<double> &typed<double>(const DevParams &p) { return p.pd; }

struct DevStats {
    unsigned long long streams, nonconv, clamped, nonfinite, bad_init, stalled, block_streams, max_streams;
    unsigned long long timeouts;   // tiles skipped because a bounded wait for their copies ran out
    unsigned long long region_nodes;   // D2Q9 step: stencil-region nodes transformed, summed over streams
    unsigned long long pair_streams;   // D2Q9 step: streams that took the per-pair path (wide regions)
};

// lattice temperature T_L = 1/3 and 1-D weights W_-1, W_0, W_+1 (SM "Equilibrium")
#define POND_TL (1.0 / 3.0)
__device__ __forceinline__ double w1d(int a) { return a == 1 ? 2.0 / 3.0 : 1.0 / 6.0; }

// Index of a node after the boundary rule: periodic wrap or zero-gradient clamp.
__device__ __forceinline__ int bc_wrap(int i, int n, int bc)
{
    if (bc == 0) {
        if (i >= 0 && i < n) return i;
        if (i < 0 && i >= -n) return i + n;
        if (i >= n && i < 2 * n) return i - n;
        i %= n;
        return i < 0 ? i + n : i;
    }
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

template <typename R> __device__ __forceinline__ R sqrt_(R x);
template <> __device__ __forceinline__ float sqrt_(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double sqrt_(double x) { return sqrt(x); }

// ---------------------------------------------------------------------------
// Initial state: co-moving equilibrium of host-given (rho, u, T) (Eq. geq with the
// interface energy kappa |grad rho|^2 / 2 in the total energy).
template <typename R>
__global__ void k_init(DevParams p, const double *__restrict__ rho, const double *__restrict__ ux,
                       const double *__restrict__ uy, const double *__restrict__ T,
                       R *__restrict__ st, DevStats *stats)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    int X = (int)(n % p.nx), Y = (int)(n / p.nx);
    double gx = 0.0, gy = 0.0;
    for (int i = 0; i < 9; ++i) {
        int cx = i % 3 - 1, cy = i / 3 - 1;
        long long m = (long long)bc_wrap(Y + cy, p.ny, p.bcy) * p.nx + bc_wrap(X + cx, p.nx, p.bcx);
        double w = w1d(cx + 1) * w1d(cy + 1);
        gx += w * cx * rho[m];
        gy += w * cy * rho[m];
    }
    gx *= 3.0;
    gy *= 3.0;
    double r = rho[n], t = T[n];
    if (!(r > 0.0) || !(p.b * r < 1.0) || !(t > 0.0)) atomicAdd(&stats->bad_init, 1ull);
    double pr = eos_pressure<double>(p.eos_kind, p.a, p.b, p.R, r, t, p.sp);
    double P = pr > p.p_floor ? pr : p.p_floor;
    double th = P / (r * POND_TL), s = sqrt(th);
    double e = p.cv * t - p.a * r;
    double lam_e = p.kappa * (gx * gx + gy * gy);
    for (int i = 0; i < 9; ++i) {
        int cx = i % 3 - 1, cy = i / 3 - 1;
        double w = w1d(cx + 1) * w1d(cy + 1);
        double vx = s * cx + ux[n], vy = s * cy + uy[n];
        REC(st, n, P_F + i) = (R)(r * w);
        REC(st, n, P_G + i) = (R)(r * w * (2.0 * e - 2.0 * P / r + vx * vx + vy * vy) + w * lam_e);
    }
    REC(st, n, P_TH) = (R)th;
    REC(st, n, P_UX) = (R)ux[n];
    REC(st, n, P_UY) = (R)uy[n];
    REC(st, n, P_RHO) = (R)r;
    REC(st, n, P_T) = (R)t;
    REC(st, n, P_UHX) = (R)ux[n];
    REC(st, n, P_UHY) = (R)uy[n];
    REC(st, n, P_F4LO) = (R)0;
    REC(st, n, P_G4LO) = (R)0;
    REC(st, n, P_JXLO) = (R)0;
    REC(st, n, P_JYLO) = (R)0;
}

template <typename T>
__device__ __forceinline__ void warp_add(unsigned long long *dst, T v)
{
    unsigned mask = __activemask();
    unsigned long long x = (unsigned long long)v;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    if ((threadIdx.x & 31) == (__ffs(mask) - 1) && x) atomicAdd(dst, x);
}


// ---------------------------------------------------------------------------
// Output fields: rho, uhat, T, p (vdW EoS) in FP64.
template <typename R>
__global__ void k_moments(DevParams p, const R *__restrict__ st, double *rho, double *ux,
                          double *uy, double *T, double *pr)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    double r = (double)REC(st, n, P_RHO), t = (double)REC(st, n, P_T);
    if (rho) rho[n] = r;
    if (ux) ux[n] = (double)REC(st, n, P_UHX);
    if (uy) uy[n] = (double)REC(st, n, P_UHY);
    if (T) T[n] = t;
    if (pr) pr[n] = eos_pressure<double>(p.eos_kind, p.a, p.b, p.R, r, t, p.sp);
}

// Error-free sum of two doubles (Knuth TwoSum).
__device__ __forceinline__ void two_sum(double a, double b, double &s, double &e)
{
    s = a + b;
    double bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// Compensated (sum, error) pairs added together.
__device__ __forceinline__ void pair_add(double &s, double &c, double s2, double c2)
{
    double t, e;
    two_sum(s, s2, t, e);
    s = t;
    c += c2 + e;
}

// Conservation sums, stage 1: per-block compensated partials of
// {rho, rho uhat_x, rho uhat_y, sum_i g_i / 2}.  part holds gridDim.x * 8 doubles.
template <typename R>
__global__ void k_conserve1(DevParams p, const R *__restrict__ st, double *part)
{
    const long long N = p.N;
    double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        double r = (double)REC(st, n, P_RHO);
        double eg = 0.0;
        for (int i = 0; i < 9; ++i) eg += (double)REC(st, n, P_G + i);
        eg += (double)REC(st, n, P_G4LO);
        double v[4] = {r, r * (double)REC(st, n, P_UHX), r * (double)REC(st, n, P_UHY), 0.5 * eg};
        for (int k = 0; k < 4; ++k) pair_add(s[k], c[k], v[k], 0.0);
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 4; ++k) {
            double s2 = __shfl_xor_sync(0xffffffffu, s[k], o);
            double c2 = __shfl_xor_sync(0xffffffffu, c[k], o);
            pair_add(s[k], c[k], s2, c2);
        }
    __shared__ double sh[32][8];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) { sh[warp][2 * k] = s[k]; sh[warp][2 * k + 1] = c[k]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < 4; ++k) {
            double ss = sh[0][2 * k], cc = sh[0][2 * k + 1];
            for (int w = 1; w < nw; ++w) pair_add(ss, cc, sh[w][2 * k], sh[w][2 * k + 1]);
            part[blockIdx.x * 8 + 2 * k] = ss;
            part[blockIdx.x * 8 + 2 * k + 1] = cc;
        }
    }
}

// Stage 1 over the ABI's 25-plane FP64 state layout (plane p of node n at p*N + n), with
// each block summing a fixed span of `span` nodes so that the number of partials is
// ceil(N / span): {rho, rho uhat_x, rho uhat_y, sum_i g_i / 2} as in k_conserve1.
__global__ void k_conserve_planes1(const double *__restrict__ planes, long long N, int span, double *part)
{
    double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    const long long lo = (long long)blockIdx.x * span;
    const long long hi = lo + span < N ? lo + span : N;
    for (long long n = lo + threadIdx.x; n < hi; n += blockDim.x) {
        const double r = planes[21 * N + n];
        double eg = 0.0;
        for (int i = 0; i < 9; ++i) eg += planes[(9 + i) * N + n];
        const double v[4] = {r, r * planes[23 * N + n], r * planes[24 * N + n], 0.5 * eg};
        for (int k = 0; k < 4; ++k) pair_add(s[k], c[k], v[k], 0.0);
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 4; ++k) {
            double s2 = __shfl_xor_sync(0xffffffffu, s[k], o);
            double c2 = __shfl_xor_sync(0xffffffffu, c[k], o);
            pair_add(s[k], c[k], s2, c2);
        }
    __shared__ double sh[32][8];
    int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) { sh[warp][2 * k] = s[k]; sh[warp][2 * k + 1] = c[k]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < 4; ++k) {
            double ss = sh[0][2 * k], cc = sh[0][2 * k + 1];
            for (int w = 1; w < nw; ++w) pair_add(ss, cc, sh[w][2 * k], sh[w][2 * k + 1]);
            part[blockIdx.x * 8 + 2 * k] = ss;
            part[blockIdx.x * 8 + 2 * k + 1] = cc;
        }
    }
}

// Stage 2: one thread folds the block partials into out[4].
__global__ void k_conserve2(const double *part, int nblocks, double *out)
{
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    for (int k = 0; k < 4; ++k) {
        double ss = 0.0, cc = 0.0;
        for (int b = 0; b < nblocks; ++b) pair_add(ss, cc, part[b * 8 + 2 * k], part[b * 8 + 2 * k + 1]);
        out[k] = ss + cc;
    }
}

}  // namespace pond
