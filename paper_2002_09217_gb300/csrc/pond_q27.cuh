// pond_q27.cuh -- the PonD van der Waals time step in three dimensions on the D3Q27
// lattice for sm_103a.
//
// The model is written for D dimensions (D enters the energy equilibrium and the
// heat-flux correction); D3Q27 = C1 x C1 x C1 with C1 = {-1, 0, 1}, weights 1/6, 2/3,
// 1/6 per axis and T_L = 1/3.  The transfer map G = M_lambda'^-1 M_lambda over the 27
// moments M_lmn (l, m, n <= 2) is the product of three 3-node Lagrange maps, one per axis
// (SM "Transfer matrix"); reconstruction uses the 4 x 4 x 4 cubic stencil (one cubic
// factor per axis, SM "Reconstruction").  The forced g equilibrium takes its 3-D tensors
// I_ab = uhat_a F_b + F_a uhat_b + dt F_a F_b E/(2P), M_a = (dt rho/P)(F_a H - I_ab u_b),
// N_ab = rho delta_ab + (dt rho/(2P)) I_ab.
//
// Layout: one record of SL27 = 72 values per node (node = (z*ny + y)*nx + x):
//   [0] theta, [1..3] u, [4..30] f_0..f_26, [31..57] g_0..g_26, [58] rho, [59] T,
//   [60..62] uhat, [63] mass lo, [64..66] momentum lo, [67] energy lo, [68..71] unused
// with population i = 9*jz + 3*jy + jx, c = j - 1.  The gauge is one 16-byte load and
// the 54 populations fourteen more.  The lo values (FP32 form only) are what storage
// rounding took from the node's exact mass, momentum and energy (as on D2Q9 and D2Q16).
//
// One step is three launches: the Korteweg stress and heat-flux vector of the state the
// non-local terms come from, their divergences, and the node step (one thread per node).
#pragma once

#include "pond_kernels.cuh"

namespace pond {

constexpr int Q27 = 27;
constexpr int NP27 = 2 * Q27 + 9;   // planes of the exchanged D3Q27 state
constexpr int SL27 = 72;
enum : int { R_TH = 0, R_UX = 1, R_F = 4, R_G = 31, R_RHO = 58, R_T = 59, R_UHX = 60, R_MLO = 63,
             R_JLO = 64, R_GLO = 67 };
// FP64 scratch planes of the non-local terms
enum : int { N3_K = 0 /* xx, xy, xz, yy, yz, zz */, N3_Q = 6, N3_REL = 9, N3_F = 10, N3_M0 = 13, N3_PLANES = 14 };

// record offset of plane p of the exchanged state (f, g, theta, u, rho, T, uhat)
__host__ __device__ constexpr int rec27_off(int p) { return p < 54 ? p + 4 : (p < 58 ? p - 54 : p); }

#define REC27(buf, n, off) (buf)[(size_t)(n) * SL27 + (off)]
#define NL3(buf, plane, n, N) (buf)[(size_t)(plane) * (size_t)(N) + (size_t)(n)]

struct Grid3 {
    int nz, bcz;
};

__device__ __forceinline__ long long node27(const DevParams &p, const Grid3 &g, int x, int y, int z)
{
    return ((long long)bc_wrap(z, g.nz, g.bcz) * p.ny + bc_wrap(y, p.ny, p.bcy)) * p.nx + bc_wrap(x, p.nx, p.bcx);
}

template <typename A>
__device__ __forceinline__ A sel3(const A (&v)[3], int k)
{
    return k == 0 ? v[0] : (k == 1 ? v[1] : v[2]);
}

// Row k of a per-axis 3-node transfer map in increment form (nodes -1, 0, 1 in the
// target's units; source velocities at c_j + eps_j): D[k][j] = l_k(c_j + eps_j) - delta_kj,
// off-diagonal entries carry the exact factor eps_j, the diagonal is
// (1 + eps_k/(c_k - o0))(1 + eps_k/(c_k - o1)) - 1 expanded.
template <typename A>
__device__ __forceinline__ void inc_row3(int k, const A (&eps)[3], A (&out)[3])
{
    // l_k(xi) = prod_{m != k} (xi - c_m) / (c_k - c_m), c = -1, 0, 1: the inverse
    // denominators (1/2, -1, 1/2) and 1/(c_k - o_m) are exact binary constants
    const A id = k == 1 ? A(-1) : A(0.5);
    const A r0 = k == 0 ? A(-1) : (k == 1 ? A(1) : A(0.5));     // 1/(c_k - o0), o0 < o1
    const A r1 = k == 0 ? A(-0.5) : (k == 1 ? A(-1) : A(1));    // 1/(c_k - o1)
    const A ek = sel3(eps, k);
    const A t0 = ek * r0, t1 = ek * r1;
    const A diag = (t0 + t1) + t0 * t1;
#pragma unroll
    for (int j = 0; j < 3; ++j) {
        // the factors (c_j - c_m) + eps_j for m = 0, 1, 2 (the one with m = j is eps_j)
        const A f0 = A(j) + eps[j], f1 = A(j - 1) + eps[j], f2 = A(j - 2) + eps[j];
        const A prod = k == 0 ? f1 * f2 : (k == 1 ? f0 * f2 : f0 * f1);
        out[j] = j == k ? diag : id * prod;
    }
}

template <typename A>
__device__ __forceinline__ void cubic_w(A xi, A a[4])
{
    const A x0 = xi, x1 = xi - A(1), x2 = xi - A(2), x3 = xi - A(3);
    a[0] = -(x1 * x2 * x3) / A(6);
    a[1] = (x0 * x2 * x3) * A(0.5);
    a[2] = -(x0 * x1 * x3) * A(0.5);
    a[3] = (x0 * x1 * x2) / A(6);
}

template <typename A>
__device__ __forceinline__ int depart(int X, A v, A dt, A w[4])
{
    const A d = -v * dt;
    const A fl = floor(d);
    cubic_w<A>(d - fl + A(1), w);
    return X + (int)fl - 1;
}

__device__ __forceinline__ double w27(int i) { return w1d(i % 3) * w1d((i / 3) % 3) * w1d(i / 9); }

__device__ __forceinline__ void ld4r(const float *p, float (&o)[4])
{
    const float4 t = __ldg(reinterpret_cast<const float4 *>(p));
    o[0] = t.x; o[1] = t.y; o[2] = t.z; o[3] = t.w;
}
__device__ __forceinline__ void ld4r(const double *p, double (&o)[4])
{
    const double2 a = __ldg(reinterpret_cast<const double2 *>(p));
    const double2 b = __ldg(reinterpret_cast<const double2 *>(p) + 1);
    o[0] = a.x; o[1] = a.y; o[2] = b.x; o[3] = b.y;
}

// ---------------------------------------------------------------------------
// Initial state: co-moving equilibrium of host-given (rho, u, T) with the interface
// energy (Eq. geq, D = 3).
template <typename R>
__global__ void k_q27_init(DevParams p, Grid3 g3, const double *__restrict__ rho, const double *__restrict__ ux,
                           const double *__restrict__ uy, const double *__restrict__ uz,
                           const double *__restrict__ T, R *__restrict__ st, DevStats *stats)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const int X = (int)(n % p.nx), Y = (int)((n / p.nx) % p.ny), Z = (int)(n / ((long long)p.nx * p.ny));
    double gr[3] = {0.0, 0.0, 0.0};
    for (int i = 0; i < Q27; ++i) {
        const int cx = i % 3 - 1, cy = (i / 3) % 3 - 1, cz = i / 9 - 1;
        const double v = rho[node27(p, g3, X + cx, Y + cy, Z + cz)], w = w27(i);
        gr[0] += w * cx * v; gr[1] += w * cy * v; gr[2] += w * cz * v;
    }
    for (int k = 0; k < 3; ++k) gr[k] *= 3.0;
    const double r = rho[n], t = T[n];
    if (!(r > 0.0) || !(p.b * r < 1.0) || !(t > 0.0)) atomicAdd(&stats->bad_init, 1ull);
    const double pr = eos_pressure<double>(p.eos_kind, p.a, p.b, p.R, r, t, p.sp);
    const double P = pr > p.p_floor ? pr : p.p_floor;
    const double th = P / (r * POND_TL), s = sqrt(th);
    const double e = p.cv * t - p.a * r;
    const double lam_e = p.kappa * (gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
    const double u[3] = {ux[n], uy[n], uz[n]};
    for (int i = 0; i < Q27; ++i) {
        const double w = w27(i);
        const double vx = s * (i % 3 - 1) + u[0], vy = s * ((i / 3) % 3 - 1) + u[1], vz = s * (i / 9 - 1) + u[2];
        REC27(st, n, R_F + i) = (R)(r * w);
        REC27(st, n, R_G + i) = (R)(r * w * (2.0 * e - 3.0 * P / r + vx * vx + vy * vy + vz * vz) + w * lam_e);
    }
    REC27(st, n, R_TH) = (R)th;
    for (int a = 0; a < 3; ++a) {
        REC27(st, n, R_UX + a) = (R)u[a];
        REC27(st, n, R_UHX + a) = (R)u[a];
    }
    REC27(st, n, R_RHO) = (R)r;
    REC27(st, n, R_T) = (R)t;
    for (int k = R_MLO; k < SL27; ++k) REC27(st, n, k) = (R)0;
}

// ---------------------------------------------------------------------------
// Non-local terms, stage 1 (rho, T of `src`, isotropic D3Q27 stencils
// grad = 3 sum W c phi(x + c), lap = 6 sum W (phi(x + c) - phi(x))):
// K = -kappa (rho lap rho + |grad rho|^2/2) I + kappa grad rho (x) grad rho,
// q = -mu grad h + k grad T, rho E_lambda = kappa |grad rho|^2 / 2.
template <typename R>
__global__ void k_q27_nonlocal1(DevParams p, Grid3 g3, const R *__restrict__ src, double *__restrict__ nl)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const long long N = p.N;
    const int X = (int)(n % p.nx), Y = (int)((n / p.nx) % p.ny), Z = (int)(n / ((long long)p.nx * p.ny));
    double gr[3] = {0, 0, 0}, gh[3] = {0, 0, 0}, gT[3] = {0, 0, 0}, lap = 0.0;
    const double r0 = (double)REC27(src, n, R_RHO), t0 = (double)REC27(src, n, R_T);
    for (int i = 0; i < Q27; ++i) {
        const int c[3] = {i % 3 - 1, (i / 3) % 3 - 1, i / 9 - 1};
        const long long m = node27(p, g3, X + c[0], Y + c[1], Z + c[2]);
        const double w = w27(i);
        const double r = (double)REC27(src, m, R_RHO), t = (double)REC27(src, m, R_T);
        const double h = p.cv * t - p.a * r + eos_pressure<double>(p.eos_kind, p.a, p.b, p.R, r, t, p.sp) / r;
        for (int a = 0; a < 3; ++a) {
            gr[a] += w * c[a] * r;
            gh[a] += w * c[a] * h;
            gT[a] += w * c[a] * t;
        }
        lap += w * (r - r0);
    }
    for (int a = 0; a < 3; ++a) { gr[a] *= 3.0; gh[a] *= 3.0; gT[a] *= 3.0; }
    lap *= 6.0;
    const double pr = eos_pressure<double>(p.eos_kind, p.a, p.b, p.R, r0, t0, p.sp);
    const double Pg = pr > p.p_floor ? pr : p.p_floor;
    const double mu = (p.tau - 0.5) * Pg * p.dt;
    const double kc = p.k_cond >= 0.0 ? p.k_cond : mu * (p.cv + p.R);
    const double g2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
    const double iso = -p.kappa * (r0 * lap + 0.5 * g2);
    const int ab[6][2] = {{0, 0}, {0, 1}, {0, 2}, {1, 1}, {1, 2}, {2, 2}};
    for (int k = 0; k < 6; ++k) {
        const int a = ab[k][0], b = ab[k][1];
        NL3(nl, N3_K + k, n, N) = (a == b ? iso : 0.0) + p.kappa * gr[a] * gr[b];
    }
    for (int a = 0; a < 3; ++a) NL3(nl, N3_Q + a, n, N) = -mu * gh[a] + kc * gT[a];
    NL3(nl, N3_REL, n, N) = 0.5 * p.kappa * g2;
}

// Stage 2: F_a = -d_b K_ab and M_0 = 2 div q.
__global__ void k_q27_nonlocal2(DevParams p, Grid3 g3, double *__restrict__ nl)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const long long N = p.N;
    const int X = (int)(n % p.nx), Y = (int)((n / p.nx) % p.ny), Z = (int)(n / ((long long)p.nx * p.ny));
    // symmetric K index of (a, b)
    const int kidx[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
    double F[3] = {0, 0, 0}, dq = 0.0;
    for (int i = 0; i < Q27; ++i) {
        const int c[3] = {i % 3 - 1, (i / 3) % 3 - 1, i / 9 - 1};
        const long long m = node27(p, g3, X + c[0], Y + c[1], Z + c[2]);
        const double w = w27(i);
        for (int a = 0; a < 3; ++a) {
            double dk = 0.0;
            for (int b = 0; b < 3; ++b) dk += c[b] * NL3(nl, N3_K + kidx[a][b], m, N);
            F[a] += w * dk;
            dq += w * c[a] * NL3(nl, N3_Q + a, m, N);
        }
    }
    for (int a = 0; a < 3; ++a) NL3(nl, N3_F + a, n, N) = -3.0 * F[a];
    NL3(nl, N3_M0, n, N) = 6.0 * dq;
}

// ---------------------------------------------------------------------------
// Streaming into node (X, Y, Z) in gauge (th, u): for direction i = (ix, iy, iz) the
// departure point x - v_i dt is reconstructed from the 4 x 4 x 4 nodes around it, each
// carried into the arrival gauge by the three per-axis maps in increment form.  Returns
// the increments of the streamed f_i, g_i over the node's own stored values.
template <typename R>
__device__ void q27_stream(const DevParams &p, const Grid3 &g3, const R *__restrict__ in, int X, int Y,
                           int Z, R th, const R (&u)[3], R *fi, R *gi)
{
    const long long nself = ((long long)Z * p.ny + Y) * p.nx + X;
    const R s = sqrt_(th), is = R(1) / s, dt = (R)p.dt;
#pragma unroll 1
    for (int i = 0; i < Q27; ++i) {
        const int ix = i % 3, iy = (i / 3) % 3, iz = i / 9;
        R ax[4], ay[4], az[4];
        const int x0 = depart<R>(X, s * R(ix - 1) + u[0], dt, ax);
        const int y0 = depart<R>(Y, s * R(iy - 1) + u[1], dt, ay);
        const int z0 = depart<R>(Z, s * R(iz - 1) + u[2], dt, az);
        const R refF = REC27(in, nself, R_F + i), refG = REC27(in, nself, R_G + i);
        R sf = R(0), sg = R(0);
#pragma unroll 2
        for (int q = 0; q < 64; ++q) {
            const int k = q & 3, m = (q >> 2) & 3, l = q >> 4;
            const R wgt = ax[k] * ay[m] * az[l];
            const R *rec = in + (size_t)node27(p, g3, x0 + k, y0 + m, z0 + l) * SL27;
            R gv[4];
            ld4r(rec + R_TH, gv);
            const R ths = gv[0];
            const R ds = (ths - th) / (sqrt_(ths) + s) * is;   // (s' - s)/s
            R ex[3], ey[3], ez[3];
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                ex[j] = ds * R(j - 1) + (gv[1] - u[0]) * is;
                ey[j] = ds * R(j - 1) + (gv[2] - u[1]) * is;
                ez[j] = ds * R(j - 1) + (gv[3] - u[2]) * is;
            }
            R Dx[3], Dy[3], Dz[3];
            inc_row3<R>(ix, ex, Dx);
            inc_row3<R>(iy, ey, Dy);
            inc_row3<R>(iz, ez, Dz);
            R v[56];
#pragma unroll
            for (int c = 0; c < 14; ++c) {
                R t[4];
                ld4r(rec + R_F + 4 * c, t);
#pragma unroll
                for (int e = 0; e < 4; ++e) v[4 * c + e] = t[e];
            }
#pragma unroll
            for (int pg = 0; pg < 2; ++pg) {
                const R *f = v + 27 * pg;
                // rows (jz, jy): base f_(jz, jy, ix) and x-increment
                R b[3][3], xr[3][3];
#pragma unroll
                for (int jz = 0; jz < 3; ++jz)
#pragma unroll
                    for (int jy = 0; jy < 3; ++jy) {
                        const R r0 = f[9 * jz + 3 * jy], r1 = f[9 * jz + 3 * jy + 1], r2 = f[9 * jz + 3 * jy + 2];
                        const R row[3] = {r0, r1, r2};
                        b[jz][jy] = sel3(row, ix);
                        xr[jz][jy] = Dx[0] * r0 + Dx[1] * r1 + Dx[2] * r2;
                    }
                // y-increment per jz plane, then the z-increment
                R yz[3], tz[3];
#pragma unroll
                for (int jz = 0; jz < 3; ++jz) {
                    R a = R(0);
#pragma unroll
                    for (int jy = 0; jy < 3; ++jy) a += Dy[jy] * (b[jz][jy] + xr[jz][jy]);
                    yz[jz] = a;
                    const R bb[3] = {b[jz][0], b[jz][1], b[jz][2]}, xx[3] = {xr[jz][0], xr[jz][1], xr[jz][2]};
                    tz[jz] = sel3(bb, iy) + sel3(xx, iy) + a;
                }
                const R zinc = Dz[0] * tz[0] + Dz[1] * tz[1] + Dz[2] * tz[2];
                // [G f]_i - ref = (f_i - ref) + x-inc + y-inc + z-inc of row (iz, iy)
                R bi, xi_, yi;
                {
                    const R b0[3] = {b[0][0], b[0][1], b[0][2]}, b1[3] = {b[1][0], b[1][1], b[1][2]},
                            b2[3] = {b[2][0], b[2][1], b[2][2]};
                    const R x0r[3] = {xr[0][0], xr[0][1], xr[0][2]}, x1r[3] = {xr[1][0], xr[1][1], xr[1][2]},
                            x2r[3] = {xr[2][0], xr[2][1], xr[2][2]};
                    const R bsel[3] = {sel3(b0, iy), sel3(b1, iy), sel3(b2, iy)};
                    const R xsel[3] = {sel3(x0r, iy), sel3(x1r, iy), sel3(x2r, iy)};
                    bi = sel3(bsel, iz);
                    xi_ = sel3(xsel, iz);
                    yi = sel3(yz, iz);
                }
                const R ref = pg == 0 ? refF : refG;
                const R dv = ((bi - ref) + xi_) + yi + zinc;
                if (pg == 0) sf += wgt * dv;
                else sg += wgt * dv;
            }
        }
        fi[i] = sf;
        gi[i] = sg;
    }
}

// Exact FP64 sums of the node's own stored populations and kept remainders:
// own[0] = sum f + mass lo, own[1..3] = sum f c, own[4] = sum g + energy lo,
// own[5..7] = momentum lo.
template <typename R>
__device__ __forceinline__ void q27_own(const R *rec, double own[8])
{
    double s0 = 0.0, sc[3] = {0, 0, 0}, sg = 0.0;
    for (int i = 0; i < Q27; ++i) {
        const double f = (double)rec[R_F + i];
        s0 += f;
        sc[0] += f * (i % 3 - 1);
        sc[1] += f * ((i / 3) % 3 - 1);
        sc[2] += f * (i / 9 - 1);
        sg += (double)rec[R_G + i];
    }
    own[0] = s0 + (double)rec[R_MLO];
    own[1] = sc[0]; own[2] = sc[1]; own[3] = sc[2];
    own[4] = sg + (double)rec[R_GLO];
    own[5] = (double)rec[R_JLO]; own[6] = (double)rec[R_JLO + 1]; own[7] = (double)rec[R_JLO + 2];
}

// out: rho, u (3), uhat (3), E, e, T, p, P, theta*   (13 values), FP64
template <typename R>
__device__ __forceinline__ void q27_macro(const DevParams &p, R th, const R (&u)[3], const double own[8],
                                          const R *fi, const R *gi, const double F[3], double rEl,
                                          double out[13])
{
    const double s = sqrt((double)th);
    double d0 = 0.0, dc[3] = {0, 0, 0}, dg = 0.0;
    for (int i = 0; i < Q27; ++i) {
        const double f = (double)fi[i];
        d0 += f;
        dc[0] += f * (i % 3 - 1);
        dc[1] += f * ((i / 3) % 3 - 1);
        dc[2] += f * (i / 9 - 1);
        dg += (double)gi[i];
    }
    const double rho = own[0] + d0;
    double uu[3], uh[3];
    for (int a = 0; a < 3; ++a) {
        const double j = s * (own[1 + a] + dc[a]) + (double)u[a] * rho + own[5 + a];
        uu[a] = j / rho;
        uh[a] = uu[a] + F[a] * p.dt / (2.0 * rho);
    }
    const double E = (own[4] + dg) / (2.0 * rho);
    const double e = E - 0.5 * (uh[0] * uh[0] + uh[1] * uh[1] + uh[2] * uh[2]) - rEl / rho;
    const double T = p.isothermal ? p.T_iso : (e + p.a * rho) / p.cv;
    const double pr = eos_pressure<double>(p.eos_kind, p.a, p.b, p.R, rho, T, p.sp);
    const double P = pr > p.p_floor ? pr : p.p_floor;
    out[0] = rho;
    for (int a = 0; a < 3; ++a) { out[1 + a] = uu[a]; out[4 + a] = uh[a]; }
    out[7] = E; out[8] = e; out[9] = T; out[10] = pr; out[11] = P; out[12] = P / (rho * POND_TL);
}

// full per-axis increment map D[k][j] at offsets eps_j = ds c_j + du
template <typename A>
__device__ __forceinline__ void axis3(A ds, A du, A D[3][3])
{
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const A eps[3] = {-ds + du, du, ds + du};
        inc_row3<A>(k, eps, D[k]);
    }
}

// increment of (I + Dz)(I + Dy)(I + Dx) applied to h (27 values)
template <typename A>
__device__ __forceinline__ void apply3_inc(const A Dx[3][3], const A Dy[3][3], const A Dz[3][3], const A *h,
                                           A *out)
{
    A t1[27], t2[27];
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const int ix = i % 3, r = i - ix;
        t1[i] = Dx[ix][0] * h[r] + Dx[ix][1] * h[r + 1] + Dx[ix][2] * h[r + 2];
    }
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const int iy = (i / 3) % 3, r = i - 3 * iy;
        t2[i] = Dy[iy][0] * (h[r] + t1[r]) + Dy[iy][1] * (h[r + 3] + t1[r + 3]) + Dy[iy][2] * (h[r + 6] + t1[r + 6]);
    }
#pragma unroll
    for (int i = 0; i < 27; ++i) {
        const int iz = i / 9, r = i - 9 * iz;
        const A z = Dz[iz][0] * (h[r] + t1[r] + t2[r]) + Dz[iz][1] * (h[r + 9] + t1[r + 9] + t2[r + 9]) +
                    Dz[iz][2] * (h[r + 18] + t1[r + 18] + t2[r + 18]);
        out[i] = t1[i] + t2[i] + z;
    }
}

// ---------------------------------------------------------------------------
// Region stream.  On the tensor lattice the union of a node's 27 departure stencils
// (4 x 4 x 4 each) is the product of the per-axis unions: W x H x D nodes, each side 4 +
// the spread of its axis's three departure floors (5 x 5 x 5 while |v| dt < 1).  Each
// region node is carried into the arrival gauge once for all 27 directions and every
// direction adds its Lagrange-weighted share, with the per-(direction, node) arithmetic of
// q27_stream: the region form transforms about 125 nodes per stream against 1,728 pairs.

// Largest region side the region stream takes; wider regions take q27_stream.
constexpr int Q27_REGION_MAX = 6;
constexpr int Q27_THREADS = 128;   // threads of a k_q27_step block

// Per-thread Lagrange weight tables in shared memory, one column of entries per thread
// (entry e of thread t at w[e][t]).  Entries 0..17: x, (k * Q27_REGION_MAX + c) = weight
// of region column c in the stencil of x component k (c_x = k - 1), zero outside it;
// entries 18..41: y then z, (18 + (axis - 1) * 12 + k * 4 + j) = cubic weight j of
// component k, placed by the component's offset in the region (kept in registers).
constexpr int Q27_WT_ENTRIES = 3 * Q27_REGION_MAX + 2 * 12;
template <typename R>
struct Q27Weights {
    R w[Q27_WT_ENTRIES][Q27_THREADS];
};

// Departure floors and cubic weights of the three components of one axis (as in
// `depart`) for the gauge velocity u; the region's first coordinate lo = X + min floor - 1,
// its side, and each component's offset in it.  False, with nothing written, when the side
// exceeds Q27_REGION_MAX or a floor is not finite or not within 2^20 (checked as reals
// before any conversion to int).  PADDED: zero-padded table entries (x), else the four
// weights per component.
template <typename R, bool PADDED>
__device__ __forceinline__ bool q27_region_axis(int X, R s, R u, R dt, R *wt, int &lo, int &side, int (&off)[3])
{
    R fl[3], a[3][4];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const R d = -(s * R(k - 1) + u) * dt;
        fl[k] = floor(d);
        cubic_w<R>(d - fl[k] + R(1), a[k]);
    }
    const R flo = fmin(fmin(fl[0], fl[1]), fl[2]);
    const R fhi = fmax(fmax(fl[0], fl[1]), fl[2]);
    if (!(fhi - flo <= R(Q27_REGION_MAX - 4)) || !(fabs(flo) <= R(1 << 20)) || !(fabs(fhi) <= R(1 << 20)))
        return false;
    lo = X + (int)flo - 1;
    side = (int)(fhi - flo) + 4;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        off[k] = (int)(fl[k] - flo);   // 0 .. side - 4
        if (PADDED) {
#pragma unroll
            for (int c = 0; c < Q27_REGION_MAX; ++c) {
                const int j = c - off[k];
                wt[(k * Q27_REGION_MAX + c) * Q27_THREADS] =
                    j == 0 ? a[k][0] : (j == 1 ? a[k][1] : (j == 2 ? a[k][2] : (j == 3 ? a[k][3] : R(0))));
            }
        } else {
#pragma unroll
            for (int j = 0; j < 4; ++j) wt[(k * 4 + j) * Q27_THREADS] = a[k][j];
        }
    }
    return true;
}

// weight of region row (plane) c for component k of an unpadded axis table
template <typename R>
__device__ __forceinline__ R q27_wt_at(const R *wt, int k, int o, int c)
{
    const int j = c - o;
    return (j >= 0 && j < 4) ? wt[(k * 4 + j) * Q27_THREADS] : R(0);
}

// One population set (27 values at record offset OFF) of a region node carried by the
// per-axis increment maps: t1 = x-increments, t2 = y-increments of h + t1, z = the
// z-increments of h + t1 + t2, and acc_i += w_i (((h_i - ref_i) + t1_i) + t2_i + z_i) with
// the weight w_i = wx[ix] (wy[iy] wz[iz]) (wyz[3 iz + iy] = wy[iy] wz[iz]).
template <typename R, int OFF>
__device__ __forceinline__ void q27_region_pop(const R (&Dx)[3][3], const R (&Dy)[3][3], const R (&Dz)[3][3],
                                               const R *rec, const R (&ref)[Q27], const R (&wx)[3],
                                               const R (&wyz)[9], R (&acc)[Q27])
{
    constexpr int B = OFF & ~3, SH = OFF - B, NL = (SH + Q27 + 3) / 4;   // 16-byte loads covering the set
    R h[Q27];
#pragma unroll
    for (int c = 0; c < NL; ++c) {
        R q[4];
        ld4r(rec + B + 4 * c, q);
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            const int i = 4 * c + e - SH;
            if (i >= 0 && i < Q27) h[i] = q[e];
        }
    }
    R a[Q27], u[Q27];
#pragma unroll
    for (int i = 0; i < Q27; ++i) {
        const int ix = i % 3, r = i - ix;
        const R t1 = Dx[ix][0] * h[r] + Dx[ix][1] * h[r + 1] + Dx[ix][2] * h[r + 2];
        a[i] = (h[i] - ref[i]) + t1;
        u[i] = h[i] + t1;
    }
#pragma unroll
    for (int i = 0; i < Q27; ++i) {
        const int iy = (i / 3) % 3, r = i - 3 * iy;
        // y-increments from h + t1 (held in u before the update below reads it)
        const R t2 = Dy[iy][0] * u[r] + Dy[iy][1] * u[r + 3] + Dy[iy][2] * u[r + 6];
        h[i] = t2;
    }
#pragma unroll
    for (int i = 0; i < Q27; ++i) {
        a[i] += h[i];
        u[i] += h[i];
    }
#pragma unroll
    for (int i = 0; i < Q27; ++i) {
        const int iz = i / 9, r = i - 9 * iz;
        const R z = Dz[iz][0] * u[r] + Dz[iz][1] * u[r + 9] + Dz[iz][2] * u[r + 18];
        acc[i] += (wx[i % 3] * wyz[i / 3]) * (a[i] + z);
    }
}

// The region pass for one population set (record offset OFF: R_F or R_G) over the region
// at (xlo, ylo, zlo) of sides W, H, D, skipping region entry `skip` (-1: none): writes the
// increments of the streamed populations over the node's own (irec) into out.
template <typename R, int OFF>
__device__ __noinline__ void q27_region_pass(const DevParams &p, const Grid3 &g3, const R *__restrict__ in,
                                             const R *irec, int xlo, int ylo, int zlo, int W, int H, int D,
                                             const int (&oy)[3], const int (&oz)[3], int skip, R th,
                                             const R (&u)[3], const R *wt, R *out)
{
    const R s = sqrt_(th), is = R(1) / s;
    R ref[Q27], acc[Q27];
#pragma unroll
    for (int i = 0; i < Q27; ++i) { ref[i] = irec[OFF + i]; acc[i] = R(0); }
    const R *wty = wt + 3 * Q27_REGION_MAX * Q27_THREADS, *wtz = wty + 12 * Q27_THREADS;
    int e = 0;   // region entry index (z-major, then y, then x)
#pragma unroll 1
    for (int cz = 0; cz < D; ++cz) {
        const int zz = bc_wrap(zlo + cz, g3.nz, g3.bcz);
        R wz[3];
#pragma unroll
        for (int k = 0; k < 3; ++k) wz[k] = q27_wt_at(wtz, k, oz[k], cz);
#pragma unroll 1
        for (int cy = 0; cy < H; ++cy) {
            const long long row = ((long long)zz * p.ny + bc_wrap(ylo + cy, p.ny, p.bcy)) * p.nx;
            R wyz[9];   // wy[m] wz[l] at 3 l + m (population i = 9 l + 3 m + k)
#pragma unroll
            for (int m = 0; m < 3; ++m) {
                const R wy = q27_wt_at(wty, m, oy[m], cy);
#pragma unroll
                for (int l = 0; l < 3; ++l) wyz[3 * l + m] = wy * wz[l];
            }
#pragma unroll 1
            for (int cx = 0; cx < W; ++cx, ++e) {
                if (e == skip) continue;
                const R *rec = in + (size_t)(row + bc_wrap(xlo + cx, p.nx, p.bcx)) * SL27;
                R gv[4];
                ld4r(rec + R_TH, gv);   // theta, u_x, u_y, u_z of the region node
                const R ds = (gv[0] - th) / (sqrt_(gv[0]) + s) * is;   // (s' - s)/s
                R Dx[3][3], Dy[3][3], Dz[3][3];
                axis3<R>(ds, (gv[1] - u[0]) * is, Dx);
                axis3<R>(ds, (gv[2] - u[1]) * is, Dy);
                axis3<R>(ds, (gv[3] - u[2]) * is, Dz);
                R wx[3];
#pragma unroll
                for (int k = 0; k < 3; ++k) wx[k] = wt[(k * Q27_REGION_MAX + cx) * Q27_THREADS];
                q27_region_pop<R, OFF>(Dx, Dy, Dz, rec, ref, wx, wyz, acc);
            }
        }
    }
#pragma unroll
    for (int i = 0; i < Q27; ++i) out[i] = acc[i];
}

// Streaming of node (X, Y, Z) into gauge (th, u) by the region stream where the region
// fits, else by q27_stream; skip_own leaves out the node's own region entry (valid when
// the gauge is the node's stored gauge: the map is then the identity and the entry adds
// exactly zero).  Adds the region entries transformed to nreg, or 1 to npair.
template <typename R>
__device__ __forceinline__ void q27_stream_any(const DevParams &p, const Grid3 &g3, const R *__restrict__ in,
                                               int X, int Y, int Z, R th, const R (&u)[3], bool skip_own, R *wt,
                                               R *fi, R *gi, unsigned long long &nreg, unsigned long long &npair)
{
    const R s = sqrt_(th), dt = (R)p.dt;
    int xlo, ylo, zlo, W, H, D, ox[3], oy[3], oz[3];
    R *wty = wt + 3 * Q27_REGION_MAX * Q27_THREADS, *wtz = wty + 12 * Q27_THREADS;
    if (q27_region_axis<R, true>(X, s, u[0], dt, wt, xlo, W, ox) &&
        q27_region_axis<R, false>(Y, s, u[1], dt, wty, ylo, H, oy) &&
        q27_region_axis<R, false>(Z, s, u[2], dt, wtz, zlo, D, oz)) {
        const int cxo = X - xlo, cyo = Y - ylo, czo = Z - zlo;
        const int skip = (skip_own && cxo >= 0 && cxo < W && cyo >= 0 && cyo < H && czo >= 0 && czo < D)
                             ? (czo * H + cyo) * W + cxo : -1;
        const R *irec = in + (size_t)(((long long)Z * p.ny + Y) * p.nx + X) * SL27;
        q27_region_pass<R, R_F>(p, g3, in, irec, xlo, ylo, zlo, W, H, D, oy, oz, skip, th, u, wt, fi);
        q27_region_pass<R, R_G>(p, g3, in, irec, xlo, ylo, zlo, W, H, D, oy, oz, skip, th, u, wt, gi);
        nreg += (unsigned long long)(W * H * D - (skip >= 0 ? 1 : 0));
    } else {
        q27_stream<R>(p, g3, in, X, Y, Z, th, u, fi, gi);
        npair += 1;
    }
}

// ---------------------------------------------------------------------------
// The node step (frame search, then collision), one thread per node.
// FP32: registers capped for three resident blocks per SM (168; the region passes then
// spill 20 bytes; two blocks without spills measured 1.3 % slower); FP64 keeps two.
constexpr int Q27_MIN_BLOCKS = 3;
template <typename R>
__global__ void __launch_bounds__(128, sizeof(R) == 4 ? Q27_MIN_BLOCKS : 2) k_q27_step(DevParams p, Grid3 g3, const R *__restrict__ in,
                                                  const double *__restrict__ nl, R *__restrict__ out,
                                                  DevStats *stats)
{
    const int X = blockIdx.x * blockDim.x + threadIdx.x, Y = blockIdx.y * blockDim.y + threadIdx.y;
    const int Z = blockIdx.z;
    const bool valid = X < p.nx && Y < p.ny;
    const long long N = p.N, n = valid ? ((long long)Z * p.ny + Y) * p.nx + X : 0;
    unsigned long long its = 0, nonconv = 0, clamped = 0, nonfinite = 0, nreg = 0, npair = 0;
    __shared__ Q27Weights<R> qw;
    R *wt = &qw.w[0][threadIdx.y * blockDim.x + threadIdx.x];
    if (valid) {
        const double F[3] = {NL3(nl, N3_F, n, N), NL3(nl, N3_F + 1, n, N), NL3(nl, N3_F + 2, n, N)};
        const double rEl = NL3(nl, N3_REL, n, N), M0 = NL3(nl, N3_M0, n, N);
        const R *irec = in + (size_t)n * SL27;
        R th = irec[R_TH];
        R u[3] = {irec[R_UX], irec[R_UX + 1], irec[R_UX + 2]};
        double own[8];
        q27_own<R>(irec, own);
        R ft[Q27], gt[Q27];
        double mac[13];
        int it = 0;
        bool conv = false;
        for (;;) {
            ++it;
            // the first stream uses the node's stored gauge: its own region entry adds zero
            q27_stream_any<R>(p, g3, in, X, Y, Z, th, u, it == 1, wt, ft, gt, nreg, npair);
            q27_macro<R>(p, th, u, own, ft, gt, F, rEl, mac);
            const double t0 = (double)th, st0 = sqrt(t0);
            double r = fabs(mac[12] - t0) / t0;
            for (int a = 0; a < 3; ++a) r = fmax(r, fabs(mac[1 + a] - (double)u[a]) / st0);
            if (r <= p.tol) { conv = true; break; }
            if (it >= p.max_iter || !(r == r)) break;
            th = (R)mac[12];
            for (int a = 0; a < 3; ++a) u[a] = (R)mac[1 + a];
        }
        its = (unsigned long long)it;
        nonconv = conv ? 0ull : 1ull;
        clamped = mac[10] < p.p_floor ? 1ull : 0ull;
        for (int i = 0; i < Q27; ++i) {
            ft[i] += irec[R_F + i];
            gt[i] += irec[R_G + i];
        }

        // ---- collision in type R, equilibria as increments over their co-moving form
        const TypedParams<R> &q = typed<R>(p);
        const R rho = (R)mac[0], E = (R)mac[7], Pg = (R)mac[11], ths = (R)mac[12];
        const R uu[3] = {(R)mac[1], (R)mac[2], (R)mac[3]}, uh[3] = {(R)mac[4], (R)mac[5], (R)mac[6]};
        const R f3[3] = {(R)F[0], (R)F[1], (R)F[2]}, m0 = (R)M0, dt = q.dt, om = q.omega;
        const double sd = sqrt((double)th), ssd = sqrt(mac[12]);
        const R is = (R)(1.0 / sd), sst = (R)ssd;
        const R ds = (R)((mac[12] - (double)th) / (ssd + sd) / sd);
        R D[3][3][3], Es[3][3][3];
        for (int a = 0; a < 3; ++a) {
            const R du = (R)(mac[1 + a] - (double)u[a]) * is;
            axis3<R>(ds, du, D[a]);
            axis3<R>(ds, du + f3[a] * dt / rho * is, Es[a]);
        }
        R h[Q27], eqi[Q27], shi[Q27];
        for (int i = 0; i < Q27; ++i) h[i] = rho * (R)w27(i);
        apply3_inc<R>(D[0], D[1], D[2], h, eqi);
        apply3_inc<R>(Es[0], Es[1], Es[2], h, shi);
        R fo[Q27];
        double sf = 0.0, sc[3] = {0, 0, 0};
        for (int i = 0; i < Q27; ++i) {
            fo[i] = ft[i] + om * ((h[i] - ft[i]) + eqi[i]) + (shi[i] - eqi[i]);
            const double f = (double)fo[i];
            sf += f;
            sc[0] += f * (i % 3 - 1); sc[1] += f * ((i / 3) % 3 - 1); sc[2] += f * (i / 9 - 1);
        }
        // mass and momentum defects (sum f = rho, sum f v = rho u + F dt exactly), spread by
        // W_i and W_i c_i / (s T_L)
        const double mdef = mac[0] - sf;
        R jd[3];
        for (int a = 0; a < 3; ++a) {
            const double jst = sd * sc[a] + (double)u[a] * sf;
            jd[a] = (R)((mac[0] * mac[1 + a] + F[a] * p.dt - jst - mdef * (double)u[a]) / (sd * POND_TL));
        }
        for (int i = 0; i < Q27; ++i)
            fo[i] += (R)w27(i) * ((R)mdef + jd[0] * R(i % 3 - 1) + jd[1] * R((i / 3) % 3 - 1) + jd[2] * R(i / 9 - 1));
        double mlo = 0.0, jlo[3] = {0, 0, 0};
        if (sizeof(R) == 4) {
            double s0 = 0.0, c0[3] = {0, 0, 0};
            for (int i = 0; i < Q27; ++i) {
                const double f = (double)fo[i];
                s0 += f;
                c0[0] += f * (i % 3 - 1); c0[1] += f * ((i / 3) % 3 - 1); c0[2] += f * (i / 9 - 1);
            }
            mlo = mac[0] - s0;
            for (int a = 0; a < 3; ++a)
                jlo[a] = (mac[0] * mac[1 + a] + F[a] * p.dt) - (sd * c0[a] + (double)u[a] * s0) - mlo * (double)u[a];
        }

        const R H = E + Pg / rho;
        R I[3][3], Mv[3], Nt[3][3];
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
                I[a][b] = uh[a] * f3[b] + f3[a] * uh[b] + dt * f3[a] * f3[b] * E / (R(2) * Pg);
        for (int a = 0; a < 3; ++a) {
            const R sI = I[a][0] * uu[0] + I[a][1] * uu[1] + I[a][2] * uu[2];
            Mv[a] = (dt * rho / Pg) * (f3[a] * H - sI);
            for (int b = 0; b < 3; ++b) Nt[a][b] = (a == b ? rho : R(0)) + (dt * rho / (R(2) * Pg)) * I[a][b];
        }
        const R work = uh[0] * f3[0] + uh[1] * f3[1] + uh[2] * f3[2];
        for (int i = 0; i < Q27; ++i) {
            const R c[3] = {R(i % 3 - 1), R((i / 3) % 3 - 1), R(i / 9 - 1)};
            R v[3];
            for (int a = 0; a < 3; ++a) v[a] = sst * c[a] + uu[a];
            R g = R(2) * rho * E;
            for (int a = 0; a < 3; ++a) {
                g += Mv[a] * (v[a] - uu[a]);
                for (int b = 0; b < 3; ++b) g += Nt[a][b] * (v[a] * v[b] - (a == b ? Pg / rho : R(0)) - uu[a] * uu[b]);
            }
            const R W = (R)w27(i);
            const R uc = uu[0] * c[0] + uu[1] * c[1] + uu[2] * c[2];
            const R v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
            const R gc = m0 * W * (R(1) + rho * uc * uc / (R(2) * Pg * R(POND_TL)) - rho * v2 / (R(2) * Pg) + R(1.5));
            h[i] = om * W * g + dt * (gc + R(2) * W * work);
        }
        R ginc[Q27], go[Q27];
        apply3_inc<R>(D[0], D[1], D[2], h, ginc);
        double sg = 0.0;
        for (int i = 0; i < Q27; ++i) {
            go[i] = gt[i] - om * gt[i] + (h[i] + ginc[i]);
            sg += (double)go[i];
        }
        const double g_tot = 2.0 * mac[0] * mac[7] + p.dt * (M0 + 2.0 * (mac[4] * F[0] + mac[5] * F[1] + mac[6] * F[2]));
        const R gdef = (R)(g_tot - sg);
        for (int i = 0; i < Q27; ++i) go[i] += gdef * (R)w27(i);
        double glo = 0.0;
        if (sizeof(R) == 4) {
            double s1 = 0.0;
            for (int i = 0; i < Q27; ++i) s1 += (double)go[i];
            glo = g_tot - s1;
        }
        R *orec = out + (size_t)n * SL27;
        orec[R_TH] = th;
        for (int a = 0; a < 3; ++a) orec[R_UX + a] = u[a];
        for (int i = 0; i < Q27; ++i) {
            orec[R_F + i] = fo[i];
            orec[R_G + i] = go[i];
        }
        orec[R_RHO] = rho;
        orec[R_T] = (R)mac[9];
        for (int a = 0; a < 3; ++a) {
            orec[R_UHX + a] = uh[a];
            orec[R_JLO + a] = (R)jlo[a];
        }
        orec[R_MLO] = (R)mlo;
        orec[R_GLO] = (R)glo;
        for (int k = R_GLO + 1; k < SL27; ++k) orec[k] = R(0);
        const double chk = mac[0] + mac[9] + (double)ginc[0] + (double)eqi[0];
        nonfinite = (chk - chk == 0.0) ? 0ull : 1ull;
    }
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

// Output fields: rho, uhat (3), T, p in FP64.
template <typename R>
__global__ void k_q27_moments(DevParams p, const R *__restrict__ st, double *rho, double *ux, double *uy,
                              double *uz, double *T, double *pr)
{
    const long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (n >= p.N) return;
    const double r = (double)REC27(st, n, R_RHO), t = (double)REC27(st, n, R_T);
    if (rho) rho[n] = r;
    if (ux) ux[n] = (double)REC27(st, n, R_UHX);
    if (uy) uy[n] = (double)REC27(st, n, R_UHX + 1);
    if (uz) uz[n] = (double)REC27(st, n, R_UHX + 2);
    if (T) T[n] = t;
    if (pr) pr[n] = eos_pressure<double>(p.eos_kind, p.a, p.b, p.R, r, t, p.sp);
}

// Conservation sums, stage 1: {rho, rho uhat_x, rho uhat_y, sum g / 2} per block.
template <typename R>
__global__ void k_q27_conserve1(DevParams p, const R *__restrict__ st, double *part)
{
    const long long N = p.N;
    double s[4] = {0, 0, 0, 0}, c[4] = {0, 0, 0, 0};
    for (long long n = (long long)blockIdx.x * blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const double r = (double)REC27(st, n, R_RHO);
        double eg = (double)REC27(st, n, R_GLO);
        for (int i = 0; i < Q27; ++i) eg += (double)REC27(st, n, R_G + i);
        const double v[4] = {r, r * (double)REC27(st, n, R_UHX), r * (double)REC27(st, n, R_UHX + 1), 0.5 * eg};
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
