// pond_kernels.cuh -- device code of the PonD van der Waals time step for sm_103a.
//
// Layout: a state buffer holds 25 planes of N = nx*ny values (x fastest):
//   f_0..f_8, g_0..g_8, theta, u_x, u_y, rho, T, uhat_x, uhat_y
// with population index i = 3*(cy+1) + (cx+1).  R = float (mixed form) or double.
// Scratch holds 9 planes: K_xx, K_xy, K_yy, q_x, q_y, rho*E_lambda, F_x, F_y, M_0.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

namespace pond {

constexpr int NPL = 25;
enum : int { P_F = 0, P_G = 9, P_TH = 18, P_UX = 19, P_UY = 20, P_RHO = 21, P_T = 22,
             P_UHX = 23, P_UHY = 24 };
enum : int { S_KXX = 0, S_KXY = 1, S_KYY = 2, S_QX = 3, S_QY = 4, S_REL = 5, S_FX = 6,
             S_FY = 7, S_M0 = 8, NSC = 9 };

struct DevParams {
    int nx, ny, bcx, bcy;
    long long N;
    double a, b, R, delta, cv;
    double kappa, tau, omega, dt, k_cond, p_floor, tol;
    int max_iter;
};

struct DevStats {
    unsigned long long streams, nonconv, clamped, nonfinite, bad_init;
};

// lattice temperature T_L = 1/3 and 1-D weights W_-1, W_0, W_+1 (SM "Equilibrium")
#define POND_TL (1.0 / 3.0)
__device__ __forceinline__ double w1d(int a) { return a == 1 ? 2.0 / 3.0 : 1.0 / 6.0; }

// Index of a node after the boundary rule: periodic wrap or zero-gradient clamp.
__device__ __forceinline__ int bc_wrap(int i, int n, int bc)
{
    if (bc == 0) {
        i %= n;
        return i < 0 ? i + n : i;
    }
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

// Cubic Lagrange basis at xi on nodes 0..3 (SM "Reconstruction").
template <typename R>
__device__ __forceinline__ void lagrange4(R xi, R a[4])
{
    R x1 = xi - R(1), x2 = xi - R(2), x3 = xi - R(3);
    a[0] = -(x1 * x2 * x3) * R(1.0 / 6.0);
    a[1] = xi * x2 * x3 * R(0.5);
    a[2] = -(xi * x1 * x3) * R(0.5);
    a[3] = xi * x1 * x2 * R(1.0 / 6.0);
}

// 1-D transfer coefficient: the Lagrange basis polynomial of target velocity index k
// (c = k - 1) on the target velocities {u' - s, u', u' + s}, evaluated at a source
// velocity v, with d = v - u' and inv_th = 1/s^2.  Moment matching of orders 0..2
// per axis makes the 2-D transfer matrix the tensor product of these
// (SM "Transfer matrix": G = M_{lambda'}^{-1} M_lambda).
template <typename R>
__device__ __forceinline__ R ell(int k, R d, R s, R inv_th)
{
    if (k == 1) return R(1) - d * d * inv_th;
    if (k == 0) return d * (d - s) * (R(0.5) * inv_th);
    return d * (d + s) * (R(0.5) * inv_th);
}

template <typename R> __device__ __forceinline__ R rsqrt_(R x);
template <> __device__ __forceinline__ float rsqrt_(float x) { return sqrtf(x); }
template <> __device__ __forceinline__ double rsqrt_(double x) { return sqrt(x); }

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
    const long long N = p.N;
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
    double pr = r * p.R * t / (1.0 - p.b * r) - p.a * r * r;
    double P = pr > p.p_floor ? pr : p.p_floor;
    double th = P / (r * POND_TL), s = sqrt(th);
    double e = p.cv * t - p.a * r;
    double lam_e = p.kappa * (gx * gx + gy * gy);
    for (int i = 0; i < 9; ++i) {
        int cx = i % 3 - 1, cy = i / 3 - 1;
        double w = w1d(cx + 1) * w1d(cy + 1);
        double vx = s * cx + ux[n], vy = s * cy + uy[n];
        st[(P_F + i) * N + n] = (R)(r * w);
        st[(P_G + i) * N + n] = (R)(r * w * (2.0 * e - 2.0 * P / r + vx * vx + vy * vy) + w * lam_e);
    }
    st[P_TH * N + n] = (R)th;
    st[P_UX * N + n] = (R)ux[n];
    st[P_UY * N + n] = (R)uy[n];
    st[P_RHO * N + n] = (R)r;
    st[P_T * N + n] = (R)t;
    st[P_UHX * N + n] = (R)ux[n];
    st[P_UHY * N + n] = (R)uy[n];
}

// ---------------------------------------------------------------------------
// Non-local terms from the previous step's rho and T, pass 1 (per node):
//   K = -kappa (rho lap rho + |grad rho|^2/2) I + kappa grad rho grad rho (Eq. korteweg)
//   q = -mu grad h + k grad T, mu = (tau - 1/2) P dt, h = e + p/rho  (Eq. gtilde)
//   rho E_lambda = kappa |grad rho|^2 / 2
// with grad = 3 sum W_i c_i phi(x + c_i), lap = 6 sum W_i (phi(x + c_i) - phi(x)).
template <typename R>
__global__ void k_nonlocal1(DevParams p, const R *__restrict__ st, R *__restrict__ sc)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const long long N = p.N;
    int X = (int)(n % p.nx), Y = (int)(n / p.nx);
    const R *rho = st + P_RHO * N, *T = st + P_T * N;
    R r0 = rho[n];
    R grx = 0, gry = 0, lap = 0, ghx = 0, ghy = 0, gTx = 0, gTy = 0;
    R pr0 = 0;
    for (int i = 0; i < 9; ++i) {
        int cx = i % 3 - 1, cy = i / 3 - 1;
        long long m = (long long)bc_wrap(Y + cy, p.ny, p.bcy) * p.nx + bc_wrap(X + cx, p.nx, p.bcx);
        R w = (R)(w1d(cx + 1) * w1d(cy + 1));
        R r = rho[m], t = T[m];
        R pr = r * (R)p.R * t / (R(1) - (R)p.b * r) - (R)p.a * r * r;
        R h = (R)p.cv * t - (R)p.a * r + pr / r;
        if (i == 4) pr0 = pr;
        grx += w * R(cx) * r;
        gry += w * R(cy) * r;
        lap += w * (r - r0);
        ghx += w * R(cx) * h;
        ghy += w * R(cy) * h;
        gTx += w * R(cx) * t;
        gTy += w * R(cy) * t;
    }
    grx *= R(3); gry *= R(3); lap *= R(6);
    ghx *= R(3); ghy *= R(3); gTx *= R(3); gTy *= R(3);
    R kap = (R)p.kappa;
    R iso = -kap * (r0 * lap + R(0.5) * (grx * grx + gry * gry));
    sc[S_KXX * N + n] = iso + kap * grx * grx;
    sc[S_KXY * N + n] = kap * grx * gry;
    sc[S_KYY * N + n] = iso + kap * gry * gry;
    R P0 = pr0 > (R)p.p_floor ? pr0 : (R)p.p_floor;
    R mu = (R)(p.tau - 0.5) * P0 * (R)p.dt;
    R kc = p.k_cond >= 0.0 ? (R)p.k_cond : mu * (R)(p.cv + p.R);
    sc[S_QX * N + n] = -mu * ghx + kc * gTx;
    sc[S_QY * N + n] = -mu * ghy + kc * gTy;
    sc[S_REL * N + n] = R(0.5) * kap * (grx * grx + gry * gry);
}

// Pass 2: F = -div K and M_0 = 2 div q at each node.
template <typename R>
__global__ void k_nonlocal2(DevParams p, R *__restrict__ sc)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const long long N = p.N;
    int X = (int)(n % p.nx), Y = (int)(n / p.nx);
    R dKxx = 0, dKxy_x = 0, dKxy_y = 0, dKyy = 0, dqx = 0, dqy = 0;
    for (int i = 0; i < 9; ++i) {
        int cx = i % 3 - 1, cy = i / 3 - 1;
        if (cx == 0 && cy == 0) continue;
        long long m = (long long)bc_wrap(Y + cy, p.ny, p.bcy) * p.nx + bc_wrap(X + cx, p.nx, p.bcx);
        R w = (R)(w1d(cx + 1) * w1d(cy + 1));
        dKxx += w * R(cx) * sc[S_KXX * N + m];
        dKxy_x += w * R(cx) * sc[S_KXY * N + m];
        dKxy_y += w * R(cy) * sc[S_KXY * N + m];
        dKyy += w * R(cy) * sc[S_KYY * N + m];
        dqx += w * R(cx) * sc[S_QX * N + m];
        dqy += w * R(cy) * sc[S_QY * N + m];
    }
    sc[S_FX * N + n] = -R(3) * (dKxx + dKxy_y);
    sc[S_FY * N + n] = -R(3) * (dKxy_x + dKyy);
    sc[S_M0 * N + n] = R(6) * (dqx + dqy);
}

// ---------------------------------------------------------------------------
// Streaming of direction (jx, jy) into node (X, Y) in the arrival gauge (s, ux, uy):
// departure point x - v dt; each node of the 4x4 stencil is carried into the arrival
// gauge (separable transfer map) and weighted by the cubic Lagrange basis.
template <typename R>
__device__ __forceinline__ void stream_dir(const DevParams &p, const R *__restrict__ st, int X,
                                           int Y, R s, R inv_th, R ux, R uy, int jx, int jy,
                                           R &fo, R &go)
{
    const long long N = p.N;
    R dx = -(s * R(jx - 1) + ux) * (R)p.dt;
    R dy = -(s * R(jy - 1) + uy) * (R)p.dt;
    R flx = floor(dx), fly = floor(dy);
    int x0 = X + (int)flx - 1, y0 = Y + (int)fly - 1;
    R ax[4], ay[4];
    lagrange4<R>(dx - flx + R(1), ax);
    lagrange4<R>(dy - fly + R(1), ay);
    R accf = 0, accg = 0;
#pragma unroll 1
    for (int m = 0; m < 4; ++m) {
        int yy = bc_wrap(y0 + m, p.ny, p.bcy);
        R rf = 0, rg = 0;
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            long long idx = (long long)yy * p.nx + bc_wrap(x0 + k, p.nx, p.bcx);
            R thn = st[P_TH * N + idx];
            R sn = rsqrt_(thn);
            R dux = st[P_UX * N + idx] - ux, duy = st[P_UY * N + idx] - uy;
            R gx[3], gy[3];
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                gx[a] = ell<R>(jx, sn * R(a - 1) + dux, s, inv_th);
                gy[a] = ell<R>(jy, sn * R(a - 1) + duy, s, inv_th);
            }
            R fv = 0, gv = 0;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                R tf = 0, tg = 0;
#pragma unroll
                for (int a = 0; a < 3; ++a) {
                    tf += gx[a] * st[(P_F + 3 * b + a) * N + idx];
                    tg += gx[a] * st[(P_G + 3 * b + a) * N + idx];
                }
                fv += gy[b] * tf;
                gv += gy[b] * tg;
            }
            rf += ax[k] * fv;
            rg += ax[k] * gv;
        }
        accf += ay[m] * rf;
        accg += ay[m] * rg;
    }
    fo = accf;
    go = accg;
}

template <typename T>
__device__ __forceinline__ void warp_add(unsigned long long *dst, T v)
{
    unsigned mask = __activemask();
    unsigned long long x = (unsigned long long)v;
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(mask, x, o);
    if ((threadIdx.x & 31) == (__ffs(mask) - 1) && x) atomicAdd(dst, x);
}

// One time step of one node: frame search (stream / moments / EoS / residual),
// then the BGK collision with forcing, all in registers.
template <typename R>
__global__ void __launch_bounds__(128) k_step(DevParams p, const R *__restrict__ in,
                                              R *__restrict__ out, const R *__restrict__ sc,
                                              DevStats *stats)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const long long N = p.N;
    int X = (int)(n % p.nx), Y = (int)(n / p.nx);
    const double dt = p.dt;
    const double Fx = (double)sc[S_FX * N + n], Fy = (double)sc[S_FY * N + n];
    const double rEl = (double)sc[S_REL * N + n], M0 = (double)sc[S_M0 * N + n];

    R th = in[P_TH * N + n], ux = in[P_UX * N + n], uy = in[P_UY * N + n];
    R ft[9], gt[9];
    double rho = 0, uxs = 0, uys = 0, uhx = 0, uhy = 0, E = 0, T = 0, pr = 0, P = 0, ths = 0;
    int it = 0;
    bool conv = false;
    for (;;) {
        ++it;
        R s = rsqrt_(th), inv_th = R(1) / th;
#pragma unroll
        for (int i = 0; i < 9; ++i) stream_dir<R>(p, in, X, Y, s, inv_th, ux, uy, i % 3, i / 3, ft[i], gt[i]);
        // moments (moments Eq.): rho, rho (u - u_gauge) = s sum f c, 2 rho E
        R r = 0, mx = 0, my = 0, sg = 0;
#pragma unroll
        for (int i = 0; i < 9; ++i) {
            r += ft[i];
            mx += ft[i] * R(i % 3 - 1);
            my += ft[i] * R(i / 3 - 1);
            sg += gt[i];
        }
        rho = (double)r;
        uxs = (double)ux + (double)s * (double)mx / rho;
        uys = (double)uy + (double)s * (double)my / rho;
        uhx = uxs + Fx * dt / (2.0 * rho);
        uhy = uys + Fy * dt / (2.0 * rho);
        E = (double)sg / (2.0 * rho);
        double e = E - 0.5 * (uhx * uhx + uhy * uhy) - rEl / rho;
        T = (e + p.a * rho) / p.cv;
        pr = rho * p.R * T / (1.0 - p.b * rho) - p.a * rho * rho;
        P = pr > p.p_floor ? pr : p.p_floor;
        ths = P / (rho * POND_TL);
        double thd = (double)th, sd = (double)s;
        double res = fabs(ths - thd) / thd;
        res = fmax(res, fabs(uxs - (double)ux) / sd);
        res = fmax(res, fabs(uys - (double)uy) / sd);
        if (res <= p.tol) { conv = true; break; }
        if (it >= p.max_iter || !(res == res)) break;
        th = (R)ths;
        ux = (R)uxs;
        uy = (R)uys;
    }

    // ---- collision in the streaming gauge (th, ux, uy); equilibria built in the
    //      co-moving frame lambda* = (ths, uxs, uys) and carried by the transfer map.
    const R om = (R)p.omega, dtr = (R)dt;
    const R s = rsqrt_(th), inv_th = R(1) / th;
    const R sst = rsqrt_((R)ths);
    const R dux = (R)(uxs - (double)ux), duy = (R)(uys - (double)uy);
    const R dvx = (R)(Fx * dt / rho), dvy = (R)(Fy * dt / rho);
    const R W1[3] = {R(1.0 / 6.0), R(2.0 / 3.0), R(1.0 / 6.0)};
    R Gx[3][3], Gy[3][3], Wx[3], Wy[3], Wxs[3], Wys[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        Wx[k] = Wy[k] = Wxs[k] = Wys[k] = 0;
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Gx[k][a] = ell<R>(k, sst * R(a - 1) + dux, s, inv_th);
            Gy[k][a] = ell<R>(k, sst * R(a - 1) + duy, s, inv_th);
            Wx[k] += Gx[k][a] * W1[a];
            Wy[k] += Gy[k][a] * W1[a];
            Wxs[k] += ell<R>(k, sst * R(a - 1) + dux + dvx, s, inv_th) * W1[a];
            Wys[k] += ell<R>(k, sst * R(a - 1) + duy + dvy, s, inv_th) * W1[a];
        }
    }
    const R rr = (R)rho;
    // f: f* = f~ + omega (f^eq - f~) + S,  S = G_{u+du}[rho W] - f^eq  (Eq. S-i)
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        int kx = i % 3, ky = i / 3;
        R feq = rr * Wx[kx] * Wy[ky];
        R fsh = rr * Wxs[kx] * Wys[ky];
        out[(P_F + i) * N + n] = ft[i] + om * (feq - ft[i]) + (fsh - feq);
    }
    // g: forced equilibrium (Eq. new geq), heat-flux correction (Eq. gtilde) and the
    // force-work source phi_i = 2 W_i uhat.F, all in lambda*, then carried into the gauge.
    const R Pr = (R)P, Er = (R)E, uxr = (R)uxs, uyr = (R)uys, uhxr = (R)uhx, uhyr = (R)uhy;
    const R Fxr = (R)Fx, Fyr = (R)Fy, M0r = (R)M0;
    const R H = Er + Pr / rr;
    const R Ixx = R(2) * uhxr * Fxr + dtr * Fxr * Fxr * Er / (R(2) * Pr);
    const R Ixy = uhxr * Fyr + Fxr * uhyr + dtr * Fxr * Fyr * Er / (R(2) * Pr);
    const R Iyy = R(2) * uhyr * Fyr + dtr * Fyr * Fyr * Er / (R(2) * Pr);
    const R cM = dtr * rr / Pr;
    const R Mx = cM * (Fxr * H - (Ixx * uxr + Ixy * uyr));
    const R My = cM * (Fyr * H - (Ixy * uxr + Iyy * uyr));
    const R cN = dtr * rr / (R(2) * Pr);
    const R Nxx = rr + cN * Ixx, Nxy = cN * Ixy, Nyy = rr + cN * Iyy;
    const R Pd = Pr / rr;
    const R work = R(2) * (uhxr * Fxr + uhyr * Fyr);
    R Xs[9];
#pragma unroll
    for (int i = 0; i < 9; ++i) {
        R cx = R(i % 3 - 1), cy = R(i / 3 - 1);
        R w = W1[i % 3] * W1[i / 3];
        R vx = sst * cx + uxr, vy = sst * cy + uyr;
        R Axx = vx * vx - Pd - uxr * uxr, Axy = vx * vy - uxr * uyr, Ayy = vy * vy - Pd - uyr * uyr;
        R geq = w * (R(2) * rr * Er + Mx * (vx - uxr) + My * (vy - uyr) + Nxx * Axx
                     + R(2) * Nxy * Axy + Nyy * Ayy);
        R uc = uxr * cx + uyr * cy;
        R gc = M0r * w * (R(1) + rr * uc * uc / (R(2) * Pr * R(POND_TL))
                          - rr * (vx * vx + vy * vy) / (R(2) * Pr) + R(1));
        Xs[i] = om * geq + dtr * (gc + w * work);
    }
#pragma unroll
    for (int l = 0; l < 3; ++l) {
        R tmp[3];
#pragma unroll
        for (int a = 0; a < 3; ++a)
            tmp[a] = Gy[l][0] * Xs[a] + Gy[l][1] * Xs[3 + a] + Gy[l][2] * Xs[6 + a];
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            int i = 3 * l + k;
            R X_ = Gx[k][0] * tmp[0] + Gx[k][1] * tmp[1] + Gx[k][2] * tmp[2];
            out[(P_G + i) * N + n] = (R(1) - om) * gt[i] + X_;
        }
    }
    out[P_TH * N + n] = th;
    out[P_UX * N + n] = ux;
    out[P_UY * N + n] = uy;
    out[P_RHO * N + n] = rr;
    out[P_T * N + n] = (R)T;
    out[P_UHX * N + n] = uhxr;
    out[P_UHY * N + n] = uhyr;

    warp_add(&stats->streams, it);
    warp_add(&stats->nonconv, conv ? 0 : 1);
    warp_add(&stats->clamped, pr < p.p_floor ? 1 : 0);
    bool bad = !(rho == rho) || !(T == T) || isinf(rho) || isinf(T);
    warp_add(&stats->nonfinite, bad ? 1 : 0);
}

// ---------------------------------------------------------------------------
// Output fields: rho, uhat, T, p (vdW EoS) in FP64.
template <typename R>
__global__ void k_moments(DevParams p, const R *__restrict__ st, double *rho, double *ux,
                          double *uy, double *T, double *pr)
{
    long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const long long N = p.N;
    double r = (double)st[P_RHO * N + n], t = (double)st[P_T * N + n];
    if (rho) rho[n] = r;
    if (ux) ux[n] = (double)st[P_UHX * N + n];
    if (uy) uy[n] = (double)st[P_UHY * N + n];
    if (T) T[n] = t;
    if (pr) pr[n] = r * p.R * t / (1.0 - p.b * r) - p.a * r * r;
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
        double r = (double)st[P_RHO * N + n];
        double eg = 0.0;
        for (int i = 0; i < 9; ++i) eg += (double)st[(P_G + i) * N + n];
        double v[4] = {r, r * (double)st[P_UHX * N + n], r * (double)st[P_UHY * N + n], 0.5 * eg};
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
