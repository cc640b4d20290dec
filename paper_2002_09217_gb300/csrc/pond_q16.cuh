// pond_q16.cuh -- the PonD van der Waals time step on the D2Q16 lattice for sm_103a.
//
// The model holds for any tensor lattice C1 x C1 with weights W_i = W_jx W_jy and lattice
// temperature T_L = sum W c^2 (SM "Equilibrium").  D2Q16 takes for C1 the four roots
// -+sqrt(3 +- sqrt 6) of the Hermite polynomial He_4(c) = c^4 - 6 c^2 + 3 with the
// Gauss-Hermite weights (3 -+ sqrt 6)/12, so that T_L = 1.  The transfer map
// G = M_lambda'^-1 M_lambda (SM "Transfer matrix") is then the product of two 4-node
// Lagrange maps, one per axis, and keeps the sixteen moments M_mn, m, n <= 3.
//
// Layout: one record of SLQ = 40 values per node (node = y*nx + x), in the ABI state's
// plane order:
//   [0..15] f_0..f_15, [16..31] g_0..g_15, [32] theta, [33] u_x, [34] u_y, [35] rho,
//   [36] T, [37] uhat_x, [38] uhat_y, [39] mass lo, [40] momentum_x lo,
//   [41] momentum_y lo, [42] energy lo, [43] unused
// with population i = 4*jy + jx, c_i = (C1[jx], C1[jy]).  Each row of four populations
// and the gauge (theta, u_x, u_y, rho) start on 16-byte boundaries (176-byte records in
// FP32, 352 in FP64), so a stencil node is read with nine 16-byte loads (FP32) at fixed
// offsets from one address.  The lo values (FP32 form only; zero in FP64) are what the
// storage rounding of the populations took from the node's exact post-collision mass,
// momentum (sum f v) and energy (sum g); the next step's moments add them back, so that
// changes below half an ulp of the populations (the weak edge of an acoustic pulse) are
// not lost.
//
// One step is three launches: the Korteweg stress K and heat-flux vector q of the state
// the non-local terms come from, their divergences F = -div K and M_0 = 2 div q, and the
// node step (frame search with semi-Lagrangian streaming, then BGK collision with the
// force, heat-flux and force-work sources).  R = float (FP32 storage and streaming /
// collision arithmetic, FP64 moments, EoS and frame-search residual) or double.
#pragma once

#include "pond_kernels.cuh"
#include "pond_step.cuh"   // float-float values (ffv) and TwoSum

namespace pond {

constexpr int Q16 = 16;
constexpr int NP16 = 2 * Q16 + 7;   // planes of a D2Q16 state
enum : int { Q_F = 0, Q_G = 16, Q_TH = 32, Q_UX = 33, Q_UY = 34, Q_RHO = 35, Q_T = 36, Q_UHX = 37,
             Q_UHY = 38 };
// planes of the non-local scratch (FP64): K_xx, K_xy, K_yy, q_x, q_y, rho E_lambda, F_x, F_y, M_0
enum : int { NL_KXX = 0, NL_KXY, NL_KYY, NL_QX, NL_QY, NL_REL, NL_FX, NL_FY, NL_M0, NL_PLANES };

constexpr int SLQ = 44;   // values per node record (43 used, padded to 16-byte rows)
enum : int { Q_MLO = 39, Q_JXLO = 40, Q_JYLO = 41, Q_GLO = 42 };
// value `off` of node n's record, and plane `plane` of the FP64 non-local scratch
#define REC16(buf, n, off) (buf)[(size_t)(n) * SLQ + (off)]
#define NLP(buf, plane, n, N) (buf)[(size_t)(plane) * (size_t)(N) + (size_t)(n)]

// Four consecutive record values starting on a 16-byte boundary: one 16-byte load (FP32)
// or two (FP64), through the read-only path; and the matching stores.
__device__ __forceinline__ void ld4(const float *p, float (&o)[4])
{
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld4(const double *p, double (&o)[4])
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}
__device__ __forceinline__ void st4(float *p, float a, float b, float c, float d)
{
    *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}
__device__ __forceinline__ void st4(double *p, double a, double b, double c, double d)
{
    reinterpret_cast<double2 *>(p)[0] = make_double2(a, b);
    reinterpret_cast<double2 *>(p)[1] = make_double2(c, d);
}

// C1, its weights, and per node k: 1 / prod_{j != k} (c_k - c_j) (the Lagrange
// denominator), the three other nodes o_m (in increasing order) and 1 / (c_k - o_m).
template <typename A>
struct Lat16 {
    A c[4], w[4], inv_den[4];
    A o0[4], o1[4], o2[4], r0[4], r1[4], r2[4];
};

template <typename A>
__device__ __forceinline__ Lat16<A> make_lat16()
{
    const double s6 = sqrt(6.0);
    const double ci = sqrt(3.0 - s6), co = sqrt(3.0 + s6);
    const double c[4] = {-co, -ci, ci, co};
    const double wi = (3.0 + s6) / 12.0, wo = (3.0 - s6) / 12.0;
    Lat16<A> L;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        double d = 1.0;
#pragma unroll
        for (int j = 0; j < 4; ++j)
            if (j != k) d *= c[k] - c[j];
        L.c[k] = (A)c[k];
        L.w[k] = (A)((k == 0 || k == 3) ? wo : wi);
        L.inv_den[k] = (A)(1.0 / d);
        const double o0 = k == 0 ? c[1] : c[0], o1 = k <= 1 ? c[2] : c[1], o2 = k <= 2 ? c[3] : c[2];
        L.o0[k] = (A)o0; L.o1[k] = (A)o1; L.o2[k] = (A)o2;
        L.r0[k] = (A)(1.0 / (c[k] - o0)); L.r1[k] = (A)(1.0 / (c[k] - o1)); L.r2[k] = (A)(1.0 / (c[k] - o2));
    }
    return L;
}

// element k (runtime, 0..3) of a 4-array held in registers
template <typename A>
__device__ __forceinline__ A sel4(const A (&v)[4], int k)
{
    return k == 0 ? v[0] : (k == 1 ? v[1] : (k == 2 ? v[2] : v[3]));
}

// Row k of a per-axis transfer map in increment form.  With the source velocities at
// xi_j = c_j + eps_j in the target's units, G[k][j] = l_k(c_j + eps_j) and the increment
// D[k][j] = G[k][j] - delta_kj is
//   j != k: inv_den_k prod_m ((c_j - o_m) + eps_j)   (one factor is eps_j exactly),
//   j == k: prod_m (1 + eps_k / (c_k - o_m)) - 1, expanded in the three small terms,
// so that it carries full relative precision however small the gauge change is (FP32
// arithmetic would otherwise lose the change under the rounding of G ~ I).
template <typename A>
struct IncRow {
    A id, r0, r1, r2;
    A d[4][3];   // c_j - o_m (exactly 0 where o_m = c_j)
    int k;
    // the whole row at the offsets eps[0..3]
    __device__ __forceinline__ void row(const A (&eps)[4], A (&out)[4]) const
    {
        const A ek = sel4(eps, k);
        const A t0 = ek * r0, t1 = ek * r1, t2 = ek * r2;
        const A diag = (t0 + t1 + t2) + (t0 * t1 + t0 * t2 + t1 * t2) + t0 * t1 * t2;
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            const A off = id * ((d[j][0] + eps[j]) * (d[j][1] + eps[j]) * (d[j][2] + eps[j]));
            out[j] = j == k ? diag : off;
        }
    }
};

template <typename A>
__device__ __forceinline__ IncRow<A> inc_row(const Lat16<A> &L, int k)
{
    IncRow<A> b;
    b.id = sel4(L.inv_den, k);
    const A o0 = sel4(L.o0, k), o1 = sel4(L.o1, k), o2 = sel4(L.o2, k);
    b.r0 = sel4(L.r0, k); b.r1 = sel4(L.r1, k); b.r2 = sel4(L.r2, k);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        b.d[j][0] = L.c[j] - o0;
        b.d[j][1] = L.c[j] - o1;
        b.d[j][2] = L.c[j] - o2;
    }
    b.k = k;
    return b;
}

// Cubic Lagrange weights on the nodes 0, 1, 2, 3 at xi (SM "Reconstruction").
template <typename A>
__device__ __forceinline__ void cubic_weights(A xi, A a[4])
{
    const A x0 = xi, x1 = xi - A(1), x2 = xi - A(2), x3 = xi - A(3);
    a[0] = -(x1 * x2 * x3) / A(6);
    a[1] = (x0 * x2 * x3) / A(2);
    a[2] = -(x0 * x1 * x3) / A(2);
    a[3] = (x0 * x1 * x2) / A(6);
}

// Departure stencil along one axis of a node at integer coordinate X for the velocity v:
// the departure point X - v dt lies at stencil coordinate xi in [1, 2) of the four nodes
// x0 .. x0 + 3 (x0 = floor(X - v dt) - 1); computed from the displacement so that FP32
// keeps full precision on large grids.
template <typename A>
__device__ __forceinline__ int departure(int X, A v, A dt, A w[4])
{
    const A d = -v * dt;
    const A fl = floor(d);
    cubic_weights<A>(d - fl + A(1), w);
    return X + (int)fl - 1;
}

// Pressure, energy and enthalpy of the run's EoS in FP64.
__device__ __forceinline__ double q16_p(const DevParams &p, double r, double t)
{
    return eos_pressure<double>(p.eos_kind, p.a, p.b, p.R, r, t, p.sp);
}

// ---------------------------------------------------------------------------
// Initial state: co-moving equilibrium of host-given (rho, u, T) (Eq. geq with the
// interface energy kappa |grad rho|^2 / 2 in the total energy), D2Q16 weights, T_L = 1.
template <typename R>
__global__ void k_q16_init(DevParams p, const double *__restrict__ rho, const double *__restrict__ ux,
                           const double *__restrict__ uy, const double *__restrict__ T,
                           R *__restrict__ st, DevStats *stats)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const Lat16<double> L = make_lat16<double>();
    const int X = (int)(n % p.nx), Y = (int)(n / p.nx);
    double gx = 0.0, gy = 0.0;
    for (int i = 0; i < 9; ++i) {
        const int cx = i % 3 - 1, cy = i / 3 - 1;
        const long long m = (long long)bc_wrap(Y + cy, p.ny, p.bcy) * p.nx + bc_wrap(X + cx, p.nx, p.bcx);
        const double w = w1d(cx + 1) * w1d(cy + 1);
        gx += w * cx * rho[m];
        gy += w * cy * rho[m];
    }
    gx *= 3.0;
    gy *= 3.0;
    const double r = rho[n], t = T[n];
    if (!(r > 0.0) || !(p.b * r < 1.0) || !(t > 0.0)) atomicAdd(&stats->bad_init, 1ull);
    const double pr = q16_p(p, r, t);
    const double P = pr > p.p_floor ? pr : p.p_floor;
    const double th = P / r, s = sqrt(th);
    const double e = p.cv * t - p.a * r;
    const double lam_e = p.kappa * (gx * gx + gy * gy);
    for (int i = 0; i < Q16; ++i) {
        const int jx = i & 3, jy = i >> 2;
        const double w = L.w[jx] * L.w[jy];
        const double vx = s * L.c[jx] + ux[n], vy = s * L.c[jy] + uy[n];
        REC16(st, n, Q_F + i) = (R)(r * w);
        REC16(st, n, Q_G + i) = (R)(r * w * (2.0 * e - 2.0 * P / r + vx * vx + vy * vy) + w * lam_e);
    }
    REC16(st, n, Q_TH) = (R)th;
    REC16(st, n, Q_UX) = (R)ux[n];
    REC16(st, n, Q_UY) = (R)uy[n];
    REC16(st, n, Q_RHO) = (R)r;
    REC16(st, n, Q_T) = (R)t;
    REC16(st, n, Q_UHX) = (R)ux[n];
    REC16(st, n, Q_UHY) = (R)uy[n];
    for (int k = Q_MLO; k < SLQ; ++k) REC16(st, n, k) = (R)0;
}

// ---------------------------------------------------------------------------
// Non-local terms, stage 1 (from the rho, T planes of `src`): with the isotropic D2Q9
// grid stencils grad = 3 sum W c phi(x + c), lap = 6 sum W (phi(x + c) - phi(x)),
//   K = -kappa (rho lap rho + |grad rho|^2 / 2) I + kappa grad rho (x) grad rho  (Eq. korteweg)
//   q = -mu grad h + k grad T, mu = (tau - 1/2) P dt, h = e + p/rho              (Eq. gtilde)
//   rho E_lambda = kappa |grad rho|^2 / 2.
template <typename R>
__global__ void k_q16_nonlocal1(DevParams p, const R *__restrict__ src, double *__restrict__ nl)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const long long N = p.N;
    const int X = (int)(n % p.nx), Y = (int)(n / p.nx);
    double gr[2] = {0.0, 0.0}, gh[2] = {0.0, 0.0}, gT[2] = {0.0, 0.0}, lap = 0.0;
    const double r0 = (double)REC16(src, n, Q_RHO), t0 = (double)REC16(src, n, Q_T);
    for (int i = 0; i < 9; ++i) {
        const int cx = i % 3 - 1, cy = i / 3 - 1;
        const long long m = (long long)bc_wrap(Y + cy, p.ny, p.bcy) * p.nx + bc_wrap(X + cx, p.nx, p.bcx);
        const double w = w1d(cx + 1) * w1d(cy + 1);
        const double r = (double)REC16(src, m, Q_RHO), t = (double)REC16(src, m, Q_T);
        const double h = p.cv * t - p.a * r + q16_p(p, r, t) / r;
        gr[0] += w * cx * r; gr[1] += w * cy * r;
        gh[0] += w * cx * h; gh[1] += w * cy * h;
        gT[0] += w * cx * t; gT[1] += w * cy * t;
        lap += w * (r - r0);
    }
    for (int k = 0; k < 2; ++k) { gr[k] *= 3.0; gh[k] *= 3.0; gT[k] *= 3.0; }
    lap *= 6.0;
    const double pr = q16_p(p, r0, t0);
    const double Pg = pr > p.p_floor ? pr : p.p_floor;
    const double mu = (p.tau - 0.5) * Pg * p.dt;
    const double kc = p.k_cond >= 0.0 ? p.k_cond : mu * (p.cv + p.R);
    const double g2 = gr[0] * gr[0] + gr[1] * gr[1];
    const double iso = -p.kappa * (r0 * lap + 0.5 * g2);
    NLP(nl, NL_KXX, n, N) = iso + p.kappa * gr[0] * gr[0];
    NLP(nl, NL_KXY, n, N) = p.kappa * gr[0] * gr[1];
    NLP(nl, NL_KYY, n, N) = iso + p.kappa * gr[1] * gr[1];
    NLP(nl, NL_QX, n, N) = -mu * gh[0] + kc * gT[0];
    NLP(nl, NL_QY, n, N) = -mu * gh[1] + kc * gT[1];
    NLP(nl, NL_REL, n, N) = 0.5 * p.kappa * g2;
}

// Stage 2: F = -div K and M_0 = 2 div q with the same gradient stencil.
__global__ void k_q16_nonlocal2(DevParams p, double *__restrict__ nl)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const long long N = p.N;
    const int X = (int)(n % p.nx), Y = (int)(n / p.nx);
    double dxx = 0.0, dxy_x = 0.0, dxy_y = 0.0, dyy = 0.0, dqx = 0.0, dqy = 0.0;
    for (int i = 0; i < 9; ++i) {
        const int cx = i % 3 - 1, cy = i / 3 - 1;
        const long long m = (long long)bc_wrap(Y + cy, p.ny, p.bcy) * p.nx + bc_wrap(X + cx, p.nx, p.bcx);
        const double w = w1d(cx + 1) * w1d(cy + 1);
        dxx += w * cx * NLP(nl, NL_KXX, m, N);
        dxy_x += w * cx * NLP(nl, NL_KXY, m, N);
        dxy_y += w * cy * NLP(nl, NL_KXY, m, N);
        dyy += w * cy * NLP(nl, NL_KYY, m, N);
        dqx += w * cx * NLP(nl, NL_QX, m, N);
        dqy += w * cy * NLP(nl, NL_QY, m, N);
    }
    NLP(nl, NL_FX, n, N) = -3.0 * (dxx + dxy_y);
    NLP(nl, NL_FY, n, N) = -3.0 * (dxy_x + dyy);
    NLP(nl, NL_M0, n, N) = 6.0 * (dqx + dqy);
}

// ---------------------------------------------------------------------------
// Semi-Lagrangian streaming into node (X, Y) in gauge (th, ux, uy) (Eqs. f/g streaming):
// for direction i the departure point x - v_i dt is reconstructed from the 4 x 4 nodes
// around it, each node's populations first carried from its own gauge into (th, u) by
// the transfer map.  Only component i of G f is needed: with the per-axis maps
// Gx[ix][jx] = l_ix((s' c_jx + u'_x - u_x)/s) (s' = sqrt(theta') and u' the neighbour's
// gauge) it is sum_jy Gy[iy][jy] sum_jx Gx[ix][jx] f_(4 jy + jx), evaluated as f_i plus
// increments (G = I + D per axis).  Returns the increments fi, gi of the streamed
// populations over the node's own stored f_i, g_i (streamed f_i = own f_i + fi[i]).
template <typename R>
__device__ void q16_stream(const DevParams &p, const Lat16<R> &L, const R *__restrict__ in, int X,
                           int Y, R th, R ux, R uy, R *fi, R *gi)
{
    const long long nself = (long long)Y * p.nx + X;
    const R s = sqrt_(th), is = R(1) / s, dt = (R)p.dt;
#pragma unroll 1
    for (int iy = 0; iy < 4; ++iy) {
        const IncRow<R> by = inc_row(L, iy);
        R ay[4];
        const int y0 = departure<R>(Y, s * sel4(L.c, iy) + uy, dt, ay);
        long long rows[4];
#pragma unroll
        for (int m = 0; m < 4; ++m) rows[m] = (long long)bc_wrap(y0 + m, p.ny, p.bcy) * p.nx;
#pragma unroll 1
        for (int ix = 0; ix < 4; ++ix) {
            const IncRow<R> bx = inc_row(L, ix);
            R ax[4];
            const int x0 = departure<R>(X, s * sel4(L.c, ix) + ux, dt, ax);
            int cols[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) cols[k] = bc_wrap(x0 + k, p.nx, p.bcx);
            // interpolated as ref + sum w (v - ref) with ref = the node's own f_i, g_i: the
            // weights' rounded sum then only scales the small differences
            const int i = 4 * iy + ix;
            const R refF = REC16(in, nself, Q_F + i), refG = REC16(in, nself, Q_G + i);
            R sf = R(0), sg = R(0);
            // the 16 stencil nodes as a loop unrolled by two only (fully unrolled, the body
            // overflows the instruction cache; two iterations give independent chains)
#pragma unroll 2
            for (int mk = 0; mk < 16; ++mk) {
                const int m = mk >> 2, k = mk & 3;
                const R *rec = in + (size_t)(sel4(rows, m) + sel4(cols, k)) * SLQ;
                R gv[4];   // theta, u_x, u_y, rho of the stencil node
                ld4(rec + Q_TH, gv);
                const R ths = gv[0];
                const R ds = (ths - th) / (sqrt_(ths) + s) * is;   // (s' - s)/s
                const R ex = (gv[1] - ux) * is, ey = (gv[2] - uy) * is;
                R epx[4], epy[4], gx[4], gy[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    epx[j] = ds * L.c[j] + ex;
                    epy[j] = ds * L.c[j] + ey;
                }
                bx.row(epx, gx);
                by.row(epy, gy);
                // per row jy: base = f_(jy, ix), inc = sum_jx Dx[ix][jx] f_(jy, jx)
                R bf[4], bg[4], xf[4], xg[4];
#pragma unroll
                for (int jy = 0; jy < 4; ++jy) {
                    R fr[4], gr[4];
                    ld4(rec + Q_F + 4 * jy, fr);
                    ld4(rec + Q_G + 4 * jy, gr);
                    R df = R(0), dg = R(0);
#pragma unroll
                    for (int jx = 0; jx < 4; ++jx) { df += gx[jx] * fr[jx]; dg += gx[jx] * gr[jx]; }
                    bf[jy] = sel4(fr, ix); bg[jy] = sel4(gr, ix);
                    xf[jy] = df; xg[jy] = dg;
                }
                R df = R(0), dg = R(0);
#pragma unroll
                for (int jy = 0; jy < 4; ++jy) {
                    df += gy[jy] * (bf[jy] + xf[jy]);
                    dg += gy[jy] * (bg[jy] + xg[jy]);
                }
                // [G f]_i - ref = (f_i - ref) + x-increment of row iy + y-increment
                const R wgt = sel4(ax, k) * sel4(ay, m);
                sf += wgt * (((sel4(bf, iy) - refF) + sel4(xf, iy)) + df);
                sg += wgt * (((sel4(bg, iy) - refG) + sel4(xg, iy)) + dg);
            }
            fi[4 * iy + ix] = sf;
            gi[4 * iy + ix] = sg;
        }
    }
}

// The FP32 form's population sums in float-float on the FP32 pipes (GB300 runs FP64 at
// 1/64 of the FP32 rate, and these sums were most of the step's FP64 work).  C1's outer and
// inner nodes co = sqrt(3 + sqrt 6), ci = sqrt(3 - sqrt 6) as hi + lo (hi their FP32
// rounding, lo the FP32 rounding of the rest: together within 2^-48 relative).
__device__ __forceinline__ ffv q16_co() { return {0x1.2ace16p+1f, -0x1.b3aab0p-26f}; }
__device__ __forceinline__ ffv q16_ci() { return {0x1.7be2aep-1f, -0x1.4e69e0p-26f}; }

// Moments of 16 FP32 values v (i = 4 jy + jx), returned as doubles: out[0] = sum v and,
// with WEIGHTED, out[1] = sum v c_jx and out[2] = sum v c_jy, from the column sums C_k and
// row sums R_r (sum v c_jx = co (C_3 - C_0) + ci (C_2 - C_1), the same over rows for y).
// Each float-float addition is exact up to ~2^-48 of its result (TwoSum, the error terms
// added in FP32), far below what the kept remainders resolve (FP32 storage rounding).
template <bool WEIGHTED>
__device__ __forceinline__ void q16_ff_moments(const float *v, double *out)
{
    ffv C[4], Rw[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        C[k] = {v[k], 0.0f};
#pragma unroll
        for (int r = 1; r < 4; ++r) C[k] = ff_add(C[k], v[4 * r + k]);
    }
    const ffv s = ff_add(ff_add(C[0], C[1]), ff_add(C[2], C[3]));
    out[0] = (double)s.hi + (double)s.lo;
    if (WEIGHTED) {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            Rw[r] = {v[4 * r], 0.0f};
#pragma unroll
            for (int k = 1; k < 4; ++k) Rw[r] = ff_add(Rw[r], v[4 * r + k]);
        }
        const ffv co = q16_co(), ci = q16_ci();
        const ffv sx = ff_add(ff_mul(ff_add(C[3], ff_neg(C[0])), co), ff_mul(ff_add(C[2], ff_neg(C[1])), ci));
        const ffv sy = ff_add(ff_mul(ff_add(Rw[3], ff_neg(Rw[0])), co), ff_mul(ff_add(Rw[2], ff_neg(Rw[1])), ci));
        out[1] = (double)sx.hi + (double)sx.lo;
        out[2] = (double)sy.hi + (double)sy.lo;
    }
}

// Sums of a node's own stored populations and its kept remainders (FP64; float-float in
// the FP32 form):
// own[0] = sum f + mass lo, own[1] = sum f c_x, own[2] = sum f c_y, own[3] = sum g +
// energy lo, own[4], own[5] = the momentum lo (absolute, sum f v units).
template <typename R>
__device__ __forceinline__ void q16_own_sums(const Lat16<double> &L, const R *rec, double own[6])
{
    double s0 = 0.0, sx = 0.0, sy = 0.0, sg = 0.0;
    if constexpr (sizeof(R) == 4) {
        float f[Q16], g[Q16];
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            float q[4];
            ld4(rec + Q_F + 4 * r, q);
#pragma unroll
            for (int k = 0; k < 4; ++k) f[4 * r + k] = q[k];
            ld4(rec + Q_G + 4 * r, q);
#pragma unroll
            for (int k = 0; k < 4; ++k) g[4 * r + k] = q[k];
        }
        double m[3], mg[1];
        q16_ff_moments<true>(f, m);
        q16_ff_moments<false>(g, mg);
        s0 = m[0]; sx = m[1]; sy = m[2]; sg = mg[0];
    } else {
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            R f[4], g[4];
            ld4(rec + Q_F + 4 * r, f);
            ld4(rec + Q_G + 4 * r, g);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                s0 += (double)f[k];
                sx += (double)f[k] * L.c[k];
                sy += (double)f[k] * L.c[r];
                sg += (double)g[k];
            }
        }
    }
    R lo[4];
    ld4(rec + Q_T, lo);       // T, uhat_x, uhat_y, mass lo
    R lo2[4];
    ld4(rec + Q_JXLO, lo2);   // momentum_x lo, momentum_y lo, energy lo, unused
    own[0] = s0 + (double)lo[3];
    own[1] = sx;
    own[2] = sy;
    own[3] = sg + (double)lo2[2];
    own[4] = (double)lo2[0];
    own[5] = (double)lo2[1];
}

// Macroscopic fields of the streamed populations (own + increments) in gauge (th, ux, uy)
// (moments Eq.), FP64: out = rho, u_x, u_y, uhat_x, uhat_y, E, e, T, p,
// P = max(p, p_floor), theta* = P/rho.
template <typename R>
__device__ __forceinline__ void q16_macro(const DevParams &p, const Lat16<double> &L, R th, R ux,
                                          R uy, const double own[6], const R *fi, const R *gi,
                                          double Fx, double Fy, double rEl, double out[11])
{
    const double s = sqrt((double)th);
    double d0 = 0.0, dx = 0.0, dy = 0.0, dg = 0.0;
    if constexpr (sizeof(R) == 4) {
        double m[3], mg[1];
        q16_ff_moments<true>(fi, m);
        q16_ff_moments<false>(gi, mg);
        d0 = m[0]; dx = m[1]; dy = m[2]; dg = mg[0];
    } else {
#pragma unroll
        for (int i = 0; i < Q16; ++i) {
            const double f = (double)fi[i];
            d0 += f;
            dx += f * L.c[i & 3];
            dy += f * L.c[i >> 2];
            dg += (double)gi[i];
        }
    }
    // sum f v = s sum f c + u sum f, for the stored part and the increments
    const double rho = own[0] + d0;
    const double jx = s * (own[1] + dx) + (double)ux * rho + own[4];
    const double jy = s * (own[2] + dy) + (double)uy * rho + own[5];
    const double sg = own[3] + dg;
    const double irho = 1.0 / rho;   // one FP64 division, the quotients by rho multiply
    const double u_x = jx * irho, u_y = jy * irho;
    const double uhx = u_x + (0.5 * p.dt) * Fx * irho, uhy = u_y + (0.5 * p.dt) * Fy * irho;
    const double E = 0.5 * sg * irho;
    const double e = E - 0.5 * (uhx * uhx + uhy * uhy) - rEl * irho;
    const double T = p.isothermal ? p.T_iso : (e + p.a * rho) / p.cv;
    const double pr = q16_p(p, rho, T);
    const double P = pr > p.p_floor ? pr : p.p_floor;
    out[0] = rho; out[1] = u_x; out[2] = u_y; out[3] = uhx; out[4] = uhy;
    out[5] = E; out[6] = e; out[7] = T; out[8] = pr; out[9] = P; out[10] = P * irho;
}

// Per-axis transfer map from gauge (s_src, u_src) into (s_dst, u_dst) in increment
// form: D[i][j] = l_i(c_j + eps_j) - delta_ij with eps_j = ((s_src - s_dst) c_j + du)/s_dst;
// ds = (s_src - s_dst)/s_dst and du / s_dst are passed in.
template <typename A>
__device__ __forceinline__ void axis_inc(const Lat16<A> &L, A ds, A du, A D[4][4])
{
    A eps[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) eps[j] = ds * L.c[j] + du;
#pragma unroll
    for (int i = 0; i < 4; ++i) inc_row(L, i).row(eps, D[i]);
}

// Increment of (I + Dy) (x) (I + Dx) applied to h: out_(4 iy + ix) = [G h]_i - h_i.
template <typename A>
__device__ __forceinline__ void apply_inc(const A Dx[4][4], const A Dy[4][4], const A h[16], A out[16])
{
    A t[16];
#pragma unroll
    for (int jy = 0; jy < 4; ++jy)
#pragma unroll
        for (int ix = 0; ix < 4; ++ix) {
            A a = A(0);
#pragma unroll
            for (int jx = 0; jx < 4; ++jx) a += Dx[ix][jx] * h[4 * jy + jx];
            t[4 * jy + ix] = a;
        }
#pragma unroll
    for (int iy = 0; iy < 4; ++iy)
#pragma unroll
        for (int ix = 0; ix < 4; ++ix) {
            A a = A(0);
#pragma unroll
            for (int jy = 0; jy < 4; ++jy) a += Dy[iy][jy] * (h[4 * jy + ix] + t[4 * jy + ix]);
            out[4 * iy + ix] = t[4 * iy + ix] + a;
        }
}

// ---------------------------------------------------------------------------
// Region stream.  On a tensor lattice the union of a node's sixteen 4 x 4 departure
// stencils is the product of the per-axis unions: W x H nodes with W (H) = 4 + the spread
// of the four departure floors along the axis, 5 x 5 while |v| dt < 1 in every direction.
// Each region node is carried into the arrival gauge once for all sixteen directions
// (G f = f + [(I + Dy) (x) (I + Dx) - I] f), and direction i takes its Lagrange-weighted
// share of component i.  The arithmetic per (direction, stencil node) pair is that of
// q16_stream, so the two agree up to the rounding of zero-weight terms; the region form
// transforms about 25 nodes per stream against 256 pairs.

// Largest region side the region stream takes; wider regions take q16_stream.
constexpr int Q16_REGION_MAX = 6;
constexpr int Q16_THREADS = 128;   // threads of a k_q16_step block
// FP32: f and g of a region node in one pass (two rolled passes, one population set each,
// measured 4 % slower on the 2048 x 1024 droplet-shock); FP64 always takes two passes
// (one pass exceeds the register file).  Three FP32 blocks per SM (168 registers): two
// (232 registers) and four (128, with spills) measured slower.
constexpr bool Q16_ONE_PASS = true;
constexpr int Q16_MIN_BLOCKS = 3;

// Lagrange weight tables of the region stream, one column of entries per thread (entry e
// of thread t at w[e][t]: consecutive threads in consecutive banks).  Entry
// (axis * 4 + k) * Q16_REGION_MAX + c is the weight of region column (row) c in the
// stencil of axis component k, zero outside that stencil.
template <typename R>
struct Q16Weights {
    R w[2 * 4 * Q16_REGION_MAX][Q16_THREADS];
};

// Departure floors and Lagrange weights of the four axis components for the gauge
// velocity u along one axis (as in `departure`), the table entries of that axis, and the
// region's first coordinate lo (= X + min floor - 1) and side. False, with nothing
// written, when the side exceeds Q16_REGION_MAX or a floor is not finite or not within
// 2^20 (the floors are checked as reals before any conversion to int).
template <typename R>
__device__ __forceinline__ bool q16_region_axis(const Lat16<R> &L, int X, R s, R u, R dt, R *wt, int &lo,
                                                int &side)
{
    R fl[4], a[4][4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const R d = -(s * L.c[k] + u) * dt;
        fl[k] = floor(d);
        cubic_weights<R>(d - fl[k] + R(1), a[k]);
    }
    const R flo = fmin(fmin(fl[0], fl[1]), fmin(fl[2], fl[3]));
    const R fhi = fmax(fmax(fl[0], fl[1]), fmax(fl[2], fl[3]));
    if (!(fhi - flo <= R(Q16_REGION_MAX - 4)) || !(fabs(flo) <= R(1 << 20)) || !(fabs(fhi) <= R(1 << 20)))
        return false;
    lo = X + (int)flo - 1;
    side = (int)(fhi - flo) + 4;
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        const int o = (int)(fl[k] - flo);   // 0 .. side - 4
#pragma unroll
        for (int c = 0; c < Q16_REGION_MAX; ++c) {
            const int j = c - o;
            wt[(k * Q16_REGION_MAX + c) * Q16_THREADS] =
                j == 0 ? a[k][0] : (j == 1 ? a[k][1] : (j == 2 ? a[k][2] : (j == 3 ? a[k][3] : R(0))));
        }
    }
    return true;
}

// One population set (16 values at v) of a region node: x-increments t = (I (x) Dx) h, the
// y-increment of each component, and acc_i += wx_ix wy_iy ((h_i - ref_i) + t_i + dy_i).
template <typename R>
__device__ __forceinline__ void q16_region_pop(const R (&Dx)[4][4], const R (&Dy)[4][4], const R *v,
                                               const R (&ref)[Q16], const R (&wx)[4], const R (&wy)[4],
                                               R (&acc)[Q16])
{
    R h[Q16], t[Q16];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        R q[4];
        ld4(v + 4 * r, q);
#pragma unroll
        for (int k = 0; k < 4; ++k) h[4 * r + k] = q[k];
    }
#pragma unroll
    for (int jy = 0; jy < 4; ++jy)
#pragma unroll
        for (int ix = 0; ix < 4; ++ix) {
            R a = R(0);
#pragma unroll
            for (int jx = 0; jx < 4; ++jx) a += Dx[ix][jx] * h[4 * jy + jx];
            t[4 * jy + ix] = a;
        }
#pragma unroll
    for (int iy = 0; iy < 4; ++iy)
#pragma unroll
        for (int ix = 0; ix < 4; ++ix) {
            R dy = R(0);
#pragma unroll
            for (int jy = 0; jy < 4; ++jy) dy += Dy[iy][jy] * (h[4 * jy + ix] + t[4 * jy + ix]);
            const int i = 4 * iy + ix;
            acc[i] += (wx[ix] * wy[iy]) * (((h[i] - ref[i]) + t[i]) + dy);
        }
}

// The region pass over the W x H region at (xlo, ylo), skipping region entry `skip` (-1:
// none): the increments of the streamed populations over the node's own (irec) for the
// population set at record offset `off` (Q_F or Q_G) into out0, and with BOTH (off = Q_F)
// those of g into out1 as well.
template <typename R, bool BOTH>
__device__ __forceinline__ void q16_region_pass(const DevParams &p, const Lat16<R> &L, const R *__restrict__ in,
                                                const R *irec, int xlo, int ylo, int W, int H, int skip,
                                                R th, R ux, R uy, const R *wt, int off, R *out0, R *out1)
{
    const R s = sqrt_(th), is = R(1) / s;
    R ref0[Q16], ref1[Q16], acc0[Q16], acc1[Q16];
#pragma unroll
    for (int r = 0; r < 4; ++r) {
        R q[4];
        ld4(irec + off + 4 * r, q);
#pragma unroll
        for (int k = 0; k < 4; ++k) ref0[4 * r + k] = q[k];
        if (BOTH) {
            ld4(irec + Q_G + 4 * r, q);
#pragma unroll
            for (int k = 0; k < 4; ++k) ref1[4 * r + k] = q[k];
        }
    }
#pragma unroll
    for (int i = 0; i < Q16; ++i) { acc0[i] = R(0); acc1[i] = R(0); }
#pragma unroll 1
    for (int cy = 0; cy < H; ++cy) {
        const long long row = (long long)bc_wrap(ylo + cy, p.ny, p.bcy) * p.nx;
        R wy[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) wy[k] = wt[((4 + k) * Q16_REGION_MAX + cy) * Q16_THREADS];
#pragma unroll 1
        for (int cx = 0; cx < W; ++cx) {
            if (cy * W + cx == skip) continue;
            const R *rec = in + (size_t)(row + bc_wrap(xlo + cx, p.nx, p.bcx)) * SLQ;
            R wx[4], gv[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) wx[k] = wt[(k * Q16_REGION_MAX + cx) * Q16_THREADS];
            ld4(rec + Q_TH, gv);   // theta, u_x, u_y, rho of the region node
            const R ds = (gv[0] - th) / (sqrt_(gv[0]) + s) * is;   // (s' - s)/s
            R Dx[4][4], Dy[4][4];
            axis_inc<R>(L, ds, (gv[1] - ux) * is, Dx);
            axis_inc<R>(L, ds, (gv[2] - uy) * is, Dy);
            q16_region_pop<R>(Dx, Dy, rec + off, ref0, wx, wy, acc0);
            if (BOTH) q16_region_pop<R>(Dx, Dy, rec + Q_G, ref1, wx, wy, acc1);
        }
    }
#pragma unroll
    for (int i = 0; i < Q16; ++i) {
        out0[i] = acc0[i];
        if (BOTH) out1[i] = acc1[i];
    }
}

// Streaming of node (X, Y) into gauge (th, ux, uy) by the region stream where the region
// fits, else by q16_stream; skip_own leaves out the node's own region entry (valid when
// the gauge is the node's stored gauge: the map is then the identity and the entry adds
// exactly zero).  Adds the region entries transformed to nreg, or 1 to npair.
template <typename R>
__device__ __forceinline__ void q16_stream_any(const DevParams &p, const Lat16<R> &L, const R *__restrict__ in,
                                               int X, int Y, R th, R ux, R uy, bool skip_own, R *wt, R *fi,
                                               R *gi, unsigned long long &nreg, unsigned long long &npair)
{
    const R s = sqrt_(th), dt = (R)p.dt;
    int xlo, ylo, W, H;
    if (q16_region_axis<R>(L, X, s, ux, dt, wt, xlo, W) &&
        q16_region_axis<R>(L, Y, s, uy, dt, wt + 4 * Q16_REGION_MAX * Q16_THREADS, ylo, H)) {
        const int cxo = X - xlo, cyo = Y - ylo;
        const int skip = (skip_own && cxo >= 0 && cxo < W && cyo >= 0 && cyo < H) ? cyo * W + cxo : -1;
        const R *irec = in + ((size_t)Y * p.nx + X) * SLQ;
        if (Q16_ONE_PASS && sizeof(R) == 4) {
            q16_region_pass<R, true>(p, L, in, irec, xlo, ylo, W, H, skip, th, ux, uy, wt, Q_F, fi, gi);
        } else {
            // one population set per pass, the pass's code once (a rolled loop)
#pragma unroll 1
            for (int ps = 0; ps < 2; ++ps)
                q16_region_pass<R, false>(p, L, in, irec, xlo, ylo, W, H, skip, th, ux, uy, wt,
                                          ps == 0 ? Q_F : Q_G, ps == 0 ? fi : gi, nullptr);
        }
        nreg += (unsigned long long)(W * H - (skip >= 0 ? 1 : 0));
    } else {
        q16_stream<R>(p, L, in, X, Y, th, ux, uy, fi, gi);
        npair += 1;
    }
}

// ---------------------------------------------------------------------------
// The node step.  in: state at t - dt; nl: non-local terms (F, rho E_lambda, M_0) of the
// state they are taken from; out: state at t.  Frame search: predictor = the node's
// stored gauge; corrector = re-stream with (theta*, u) of the streamed moments until the
// relative change is <= tol or after max_iter streams.  Collision: equilibria built in
// the co-moving frame lambda* = (theta*, u) and carried into the streaming gauge (Eqs.
// f collision with S_i, g collision with gtilde and phi, new geq).
template <typename R>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? Q16_MIN_BLOCKS : 1) k_q16_step(DevParams p, const R *__restrict__ in,
                                                  const double *__restrict__ nl, R *__restrict__ out,
                                                  DevStats *stats)
{
    const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y * blockDim.y + threadIdx.y;
    const bool valid = X < p.nx && Y < p.ny;
    const long long N = p.N, n = valid ? (long long)Y * p.nx + X : 0;
    unsigned long long its = 0, nonconv = 0, clamped = 0, nonfinite = 0, nreg = 0, npair = 0;
    __shared__ Q16Weights<R> qw;
    R *wt = &qw.w[0][threadIdx.y * blockDim.x + threadIdx.x];
    if (valid) {
        const Lat16<R> L = make_lat16<R>();
        const Lat16<double> Ld = make_lat16<double>();
        const double Fx = NLP(nl, NL_FX, n, N), Fy = NLP(nl, NL_FY, n, N);
        const double rEl = NLP(nl, NL_REL, n, N), M0 = NLP(nl, NL_M0, n, N);
        R th = REC16(in, n, Q_TH), ux = REC16(in, n, Q_UX), uy = REC16(in, n, Q_UY);
        const R *irec = in + (size_t)n * SLQ;
        double own[6];
        q16_own_sums<R>(Ld, irec, own);
        R ft[Q16], gt[Q16];   // increments during the search, streamed populations after it
        double mac[11];
        int it = 0;
        bool conv = false;
        for (;;) {
            ++it;
            // the first stream uses the node's stored gauge: its own region entry adds zero
            q16_stream_any<R>(p, L, in, X, Y, th, ux, uy, it == 1, wt, ft, gt, nreg, npair);
            q16_macro<R>(p, Ld, th, ux, uy, own, ft, gt, Fx, Fy, rEl, mac);
            const double ist0 = 1.0 / sqrt((double)th);   // 1/s of the streaming gauge
            const double r0 = fabs(mac[10] - (double)th) * (ist0 * ist0);
            const double r1 = fabs(mac[1] - (double)ux) * ist0, r2 = fabs(mac[2] - (double)uy) * ist0;
            const double r = fmax(fmax(r0, r1), r2);
            if (r <= p.tol) { conv = true; break; }
            if (it >= p.max_iter || !(r == r)) break;
            th = (R)mac[10]; ux = (R)mac[1]; uy = (R)mac[2];
        }
        its = (unsigned long long)it;
        nonconv = conv ? 0ull : 1ull;
        clamped = mac[8] < p.p_floor ? 1ull : 0ull;
#pragma unroll
        for (int r = 0; r < 4; ++r) {
            R f[4], g[4];
            ld4(irec + Q_F + 4 * r, f);
            ld4(irec + Q_G + 4 * r, g);
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                ft[4 * r + k] += f[k];
                gt[4 * r + k] += g[k];
            }
        }

        // ---- collision in type R, equilibria as increments over their co-moving form
        const TypedParams<R> &q = typed<R>(p);
        const R rho = (R)mac[0], u_x = (R)mac[1], u_y = (R)mac[2], uhx = (R)mac[3], uhy = (R)mac[4];
        const R E = (R)mac[5], Pg = (R)mac[9], ths = (R)mac[10];
        const R fx = (R)Fx, fy = (R)Fy, m0 = (R)M0, dt = q.dt, om = q.omega;
        const double sd = sqrt((double)th), ssd = sqrt(mac[10]);
        const double isd = 1.0 / sd;
        const R is = (R)isd, sst = (R)ssd;
        const R ds = (R)((mac[10] - (double)th) / (ssd + sd) * isd);   // (s* - s)/s
        const R dux = (R)(mac[1] - (double)ux) * is, duy = (R)(mac[2] - (double)uy) * is;
        const R shx = fx * dt / rho * is, shy = fy * dt / rho * is;   // du of the force
        R Dx[4][4], Dy[4][4], Ex[4][4], Ey[4][4];
        axis_inc<R>(L, ds, dux, Dx);                                  // lambda* -> lambda
        axis_inc<R>(L, ds, duy, Dy);
        axis_inc<R>(L, ds, dux + shx, Ex);                            // lambda* + du -> lambda
        axis_inc<R>(L, ds, duy + shy, Ey);
        R h[Q16], eqi[Q16], shi[Q16];
#pragma unroll
        for (int i = 0; i < Q16; ++i) h[i] = rho * (L.w[i & 3] * L.w[i >> 2]);
        apply_inc<R>(Dx, Dy, h, eqi);
        apply_inc<R>(Ex, Ey, h, shi);
        // Collision keeps the mass and adds F dt to the momentum: sum_i f_out = rho and
        // sum_i f_out v_i = rho u + F dt exactly.  The stored values are made to carry both
        // (their FP64 sums are compared with the exact ones; the mass defect, which the
        // rounded weights and products would otherwise add every step in the same
        // direction, is spread by W_i, the momentum defect by W_i s c_i / theta, which has
        // no mass).  Zero in exact arithmetic.
        R fo[Q16];
        double sf = 0.0, sjx = 0.0, sjy = 0.0;
#pragma unroll
        for (int i = 0; i < Q16; ++i) fo[i] = ft[i] + om * ((h[i] - ft[i]) + eqi[i]) + (shi[i] - eqi[i]);
        if constexpr (sizeof(R) == 4) {
            double m[3];
            q16_ff_moments<true>(fo, m);
            sf = m[0]; sjx = m[1]; sjy = m[2];
        } else {
#pragma unroll
            for (int i = 0; i < Q16; ++i) {
                const double f = (double)fo[i];
                sf += f;
                sjx += f * Ld.c[i & 3];
                sjy += f * Ld.c[i >> 2];
            }
        }
        // momentum of the stored values in the streaming gauge: sum f (s c + u)
        sjx = sd * sjx + sf * (double)ux;
        sjy = sd * sjy + sf * (double)uy;
        const double mdef = mac[0] - sf;
        const R fdef = (R)mdef;
        // W_i s c_i J / theta = W_i c_i J / s (sum_i W_i c_i^2 = T_L = 1); the mass part
        // W_i mdef already carries the momentum mdef u
        const R jxdef = (R)((mac[0] * mac[1] + Fx * p.dt - sjx - mdef * (double)ux) * isd);
        const R jydef = (R)((mac[0] * mac[2] + Fy * p.dt - sjy - mdef * (double)uy) * isd);
        R *orec = out + (size_t)n * SLQ;
#pragma unroll
        for (int i = 0; i < Q16; ++i)
            fo[i] += (L.w[i & 3] * L.w[i >> 2]) * (fdef + jxdef * L.c[i & 3] + jydef * L.c[i >> 2]);
        // what the stored values still miss (below their rounding) is kept beside them
        double mlo = 0.0, jxlo = 0.0, jylo = 0.0;
        if constexpr (sizeof(R) == 4) {
            double m[3];
            q16_ff_moments<true>(fo, m);
            const double s0 = m[0], cx = m[1], cy = m[2];
            mlo = mac[0] - s0;
            // the mass lo carries momentum u mlo in the next step's sums
            jxlo = (mac[0] * mac[1] + Fx * p.dt) - (sd * cx + (double)ux * s0) - mlo * (double)ux;
            jylo = (mac[0] * mac[2] + Fy * p.dt) - (sd * cy + (double)uy * s0) - mlo * (double)uy;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) st4(orec + Q_F + 4 * r, fo[4 * r], fo[4 * r + 1], fo[4 * r + 2], fo[4 * r + 3]);

        // the quotients by P and rho as products with two reciprocals
        const R irh = R(1) / rho, ihP = R(1) / (R(2) * Pg);   // 1/rho, 1/(2P)
        const R Prh = Pg * irh, k2 = dt * rho * ihP;            // P/rho, dt rho/(2P)
        const R H = E + Prh;
        const R Ixx = R(2) * uhx * fx + dt * fx * fx * E * ihP;
        const R Ixy = uhx * fy + fx * uhy + dt * fx * fy * E * ihP;
        const R Iyy = R(2) * uhy * fy + dt * fy * fy * E * ihP;
        const R Mx = (R(2) * k2) * (fx * H - (Ixx * u_x + Ixy * u_y));
        const R My = (R(2) * k2) * (fy * H - (Ixy * u_x + Iyy * u_y));
        const R Nxx = rho + k2 * Ixx;
        const R Nxy = k2 * Ixy;
        const R Nyy = rho + k2 * Iyy;
        const R phi = R(2) * (uhx * fx + uhy * fy);
        const R rhP = rho * ihP;                                // rho/(2P)
#pragma unroll
        for (int i = 0; i < Q16; ++i) {
            const R cx = L.c[i & 3], cy = L.c[i >> 2], W = L.w[i & 3] * L.w[i >> 2];
            const R vx = sst * cx + u_x, vy = sst * cy + u_y;
            const R Axx = vx * vx - Prh - u_x * u_x;
            const R Axy = vx * vy - u_x * u_y;
            const R Ayy = vy * vy - Prh - u_y * u_y;
            const R geq = W * (R(2) * rho * E + Mx * (vx - u_x) + My * (vy - u_y) + Nxx * Axx +
                               R(2) * Nxy * Axy + Nyy * Ayy);
            const R uc = u_x * cx + u_y * cy;
            const R gc = m0 * W * (R(1) + rhP * (uc * uc) - rhP * (vx * vx + vy * vy) + R(1));
            h[i] = om * geq + dt * (gc + W * phi);
        }
        R ginc[Q16];
        apply_inc<R>(Dx, Dy, h, ginc);
        // energy: sum_i g_out = sum_i g~ + dt (M_0 + 2 uhat . F) exactly (the heat-flux
        // correction sums to M_0, the force work to 2 uhat . F); the same defect spreading
        R go[Q16];
        double sg = 0.0;
#pragma unroll
        for (int i = 0; i < Q16; ++i) go[i] = gt[i] - om * gt[i] + (h[i] + ginc[i]);
        if constexpr (sizeof(R) == 4) {
            q16_ff_moments<false>(go, &sg);
        } else {
#pragma unroll
            for (int i = 0; i < Q16; ++i) sg += (double)go[i];
        }
        const double g_tot = 2.0 * mac[0] * mac[5] + p.dt * (M0 + 2.0 * (mac[3] * Fx + mac[4] * Fy));
        const R gdef = (R)(g_tot - sg);
#pragma unroll
        for (int i = 0; i < Q16; ++i) go[i] += gdef * (L.w[i & 3] * L.w[i >> 2]);
        double glo = 0.0;
        if constexpr (sizeof(R) == 4) {
            double s1;
            q16_ff_moments<false>(go, &s1);
            glo = g_tot - s1;
        }
#pragma unroll
        for (int r = 0; r < 4; ++r) st4(orec + Q_G + 4 * r, go[4 * r], go[4 * r + 1], go[4 * r + 2], go[4 * r + 3]);
        st4(orec + Q_TH, th, ux, uy, rho);
        st4(orec + Q_T, (R)mac[7], uhx, uhy, (R)mlo);
        st4(orec + Q_JXLO, (R)jxlo, (R)jylo, (R)glo, R(0));
        const double chk = mac[0] + mac[7] + (double)ginc[0] + (double)eqi[0];
        nonfinite = (chk - chk == 0.0) ? 0ull : 1ull;
    }
    // counters: warp sums (every thread of the block reaches here; the warp's lanes are
    // its linear thread indices, whatever the block's x extent), one atomic per warp
    unsigned long long v[6] = {its, nonconv, clamped, nonfinite, nreg, npair}, mx = its;
    for (int o = 16; o > 0; o >>= 1) {
#pragma unroll
        for (int k = 0; k < 6; ++k) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
        const unsigned long long m2 = __shfl_xor_sync(0xffffffffu, mx, o);
        mx = m2 > mx ? m2 : mx;
    }
    if ((threadIdx.x + threadIdx.y * blockDim.x) % 32 == 0) {
        if (v[0]) atomicAdd(&stats->streams, v[0]);
        if (v[1]) atomicAdd(&stats->nonconv, v[1]);
        if (v[2]) atomicAdd(&stats->clamped, v[2]);
        if (v[3]) atomicAdd(&stats->nonfinite, v[3]);
        // the region-stream counters of the D2Q9 step, filled the same way here
        if (v[4]) atomicAdd(&stats->region_nodes, v[4]);
        if (v[5]) atomicAdd(&stats->pair_streams, v[5]);
        if (mx) atomicMax(&stats->max_streams, mx);
    }
}

// Output fields: rho, uhat, T, p in FP64.
template <typename R>
__global__ void k_q16_moments(DevParams p, const R *__restrict__ st, double *rho, double *ux,
                              double *uy, double *T, double *pr)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const double r = (double)REC16(st, n, Q_RHO), t = (double)REC16(st, n, Q_T);
    if (rho) rho[n] = r;
    if (ux) ux[n] = (double)REC16(st, n, Q_UHX);
    if (uy) uy[n] = (double)REC16(st, n, Q_UHY);
    if (T) T[n] = t;
    if (pr) pr[n] = q16_p(p, r, t);
}

// Conservation sums, stage 1: per-block compensated partials of
// {rho, rho uhat_x, rho uhat_y, sum_i g_i / 2} (stage 2 is k_conserve2).
template <typename R>
__global__ void k_q16_conserve1(DevParams p, const R *__restrict__ st, double *part)
{
    const long long N = p.N;
    double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const double r = (double)REC16(st, n, Q_RHO);
        double eg = (double)REC16(st, n, Q_GLO);
        for (int i = 0; i < Q16; ++i) eg += (double)REC16(st, n, Q_G + i);
        const double v[4] = {r, r * (double)REC16(st, n, Q_UHX), r * (double)REC16(st, n, Q_UHY), 0.5 * eg};
        for (int k = 0; k < 4; ++k) pair_add(s[k], c[k], v[k], 0.0);
    }
    for (int o = 16; o > 0; o >>= 1)
        for (int k = 0; k < 4; ++k) {
            const double s2 = __shfl_xor_sync(0xffffffffu, s[k], o);
            const double c2 = __shfl_xor_sync(0xffffffffu, c[k], o);
            pair_add(s[k], c[k], s2, c2);
        }
    __shared__ double sh[32][8];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0)
        for (int k = 0; k < 4; ++k) { sh[warp][2 * k] = s[k]; sh[warp][2 * k + 1] = c[k]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        const int nw = (blockDim.x + 31) >> 5;
        for (int k = 0; k < 4; ++k) {
            double ss = sh[0][2 * k], cc = sh[0][2 * k + 1];
            for (int w = 1; w < nw; ++w) pair_add(ss, cc, sh[w][2 * k], sh[w][2 * k + 1]);
            part[blockIdx.x * 8 + 2 * k] = ss;
            part[blockIdx.x * 8 + 2 * k + 1] = cc;
        }
    }
}

}  // namespace pond
