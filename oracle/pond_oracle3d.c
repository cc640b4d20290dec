/*
 * pond_oracle3d.c -- plain, slow FP64 CPU oracle for one time step of the
 * two-population "Particles on Demand" (PonD) kinetic model of a van der Waals
 * fluid (Reyhanian, Dorschner & Karlin, arXiv:2002.09217) in three dimensions on the
 * D3Q27 lattice.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA product path (nor with the 2-D oracle).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math).
 *
 * The paper states the model for D dimensions and runs it on D2Q9; this file takes
 * D = 3 and the tensor lattice D3Q27 = C1 x C1 x C1, C1 = {-1, 0, 1}, W = 1/6, 2/3, 1/6
 * per axis, T_L = 1/3, in the paper's order:
 *   - shifted particle velocities v_i = sqrt(p/(rho T_L)) c_i + u   (Eq. particle velocity)
 *   - moments rho = sum f, rho u = sum f v, 2 rho E = sum g
 *   - semi-Lagrangian streaming f_i(x) = f_i(x - v_i) through the transfer matrix
 *     G = M_{lambda'}^{-1} M_{lambda} over the 27 moments M_lmn, l, m, n <= 2 (SM
 *     "Transfer matrix"), an LU solve of that system, and the 4x4x4 cubic Lagrange
 *     stencil (SM "Reconstruction", one factor per axis)
 *   - BGK collision with the Korteweg source S_i, the heat-flux correction and the
 *     forced g equilibrium (Eqs. f/g collision, S-i, gtilde, new geq) with D = 3.
 * Readings beyond the 2-D oracle's: the forced g equilibrium's tensors take their 3-D
 * forms I_ab = uhat_a F_b + F_a uhat_b + dt F_a F_b E/(2P), M_a = (dt rho/P)(F_a H -
 * I_ab u_b), N_ab = rho delta_ab + (dt rho/(2P)) I_ab, A_ab = v_a v_b - delta_ab P/rho
 * - u_a u_b; the non-local terms use the isotropic D3Q27 difference stencils.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define Q3 27
#define NP3 (2 * Q3 + 9)
/* planes: f_0..f_26, g_0..g_26, theta, ux, uy, uz, rho, T, uhat_x, uhat_y, uhat_z */
enum { P3_F = 0, P3_G = 27, P3_TH = 54, P3_UX, P3_UY, P3_UZ, P3_RHO, P3_T, P3_UHX, P3_UHY, P3_UHZ };

static const double TL3 = 1.0 / 3.0;
static const double DIM3 = 3.0;

/* population i = 9*jz + 3*jy + jx, c = j - 1 */
static int c3x(int i) { return i % 3 - 1; }
static int c3y(int i) { return (i / 3) % 3 - 1; }
static int c3z(int i) { return i / 9 - 1; }
static double w1(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
static double w3(int i) { return w1(c3x(i)) * w1(c3y(i)) * w1(c3z(i)); }

typedef struct {
    int32_t nx, ny, nz;
    int32_t bc_x, bc_y, bc_z;  /* 0 periodic, 1 zero-gradient (index clamp) */
    double a, b, R, delta;     /* van der Waals EoS, C_v = R/delta */
    double kappa, tau, k_cond, p_floor, tol;
    int32_t max_iter, pad;
    double dt;
} orc3_params;

static double eos_p3(const orc3_params *P, double rho, double T)
{
    return rho * P->R * T / (1.0 - P->b * rho) - P->a * rho * rho;
}
static double eos_e3(const orc3_params *P, double rho, double T) { return (P->R / P->delta) * T - P->a * rho; }

static double ipow3(double x, int m)
{
    double r = 1.0;
    for (int k = 0; k < m; ++k) r *= x;
    return r;
}

/* moment (l, m, n) of row r = 9 n + 3 m + l: sum_i f_i vx^l vy^m vz^n */
void orc3_moment_matrix(const double lam[4], double M[Q3 * Q3])
{
    double s = sqrt(lam[0]);
    for (int r = 0; r < Q3; ++r)
        for (int i = 0; i < Q3; ++i) {
            double vx = s * c3x(i) + lam[1], vy = s * c3y(i) + lam[2], vz = s * c3z(i) + lam[3];
            M[r * Q3 + i] = ipow3(vx, r % 3) * ipow3(vy, (r / 3) % 3) * ipow3(vz, r / 9);
        }
}

static int lu3(double *A, int *piv)
{
    for (int k = 0; k < Q3; ++k) {
        int p = k;
        double best = fabs(A[k * Q3 + k]);
        for (int r = k + 1; r < Q3; ++r)
            if (fabs(A[r * Q3 + k]) > best) { best = fabs(A[r * Q3 + k]); p = r; }
        piv[k] = p;
        if (best == 0.0) return 1;
        if (p != k)
            for (int c = 0; c < Q3; ++c) {
                double t = A[k * Q3 + c]; A[k * Q3 + c] = A[p * Q3 + c]; A[p * Q3 + c] = t;
            }
        for (int r = k + 1; r < Q3; ++r) {
            double l = A[r * Q3 + k] / A[k * Q3 + k];
            A[r * Q3 + k] = l;
            for (int c = k + 1; c < Q3; ++c) A[r * Q3 + c] -= l * A[k * Q3 + c];
        }
    }
    return 0;
}

static void lu3_solve(const double *LU, const int *piv, const double *b, double *x)
{
    double y[Q3];
    for (int i = 0; i < Q3; ++i) y[i] = b[i];
    for (int k = 0; k < Q3; ++k)
        if (piv[k] != k) { double t = y[k]; y[k] = y[piv[k]]; y[piv[k]] = t; }
    for (int i = 0; i < Q3; ++i)
        for (int c = 0; c < i; ++c) y[i] -= LU[i * Q3 + c] * y[c];
    for (int i = Q3 - 1; i >= 0; --i) {
        for (int c = i + 1; c < Q3; ++c) y[i] -= LU[i * Q3 + c] * y[c];
        y[i] /= LU[i * Q3 + i];
    }
    for (int i = 0; i < Q3; ++i) x[i] = y[i];
}

static void apply3(const double *M, const double *f, double *m)
{
    for (int r = 0; r < Q3; ++r) {
        double s = 0.0;
        for (int i = 0; i < Q3; ++i) s += M[r * Q3 + i] * f[i];
        m[r] = s;
    }
}

/* G_{src}^{dst} = M_dst^{-1} M_src (SM "Transfer matrix"); 0 on success */
int orc3_gauge_matrix(const double src[4], const double dst[4], double G[Q3 * Q3])
{
    double Ms[Q3 * Q3], Md[Q3 * Q3];
    int piv[Q3];
    orc3_moment_matrix(src, Ms);
    orc3_moment_matrix(dst, Md);
    if (lu3(Md, piv)) return 1;
    for (int c = 0; c < Q3; ++c) {
        double col[Q3], x[Q3];
        for (int r = 0; r < Q3; ++r) col[r] = Ms[r * Q3 + c];
        lu3_solve(Md, piv, col, x);
        for (int r = 0; r < Q3; ++r) G[r * Q3 + c] = x[r];
    }
    return 0;
}

static int transform3(const double src[4], const double dst[4], const double *f, double *out)
{
    double Ms[Q3 * Q3], Md[Q3 * Q3], m[Q3];
    int piv[Q3];
    orc3_moment_matrix(src, Ms);
    apply3(Ms, f, m);
    orc3_moment_matrix(dst, Md);
    if (lu3(Md, piv)) return 1;
    lu3_solve(Md, piv, m, out);
    return 0;
}

/* cubic Lagrange basis on the nodes 0..3 (SM "Reconstruction") */
static void lagr4(double xi, double a[4])
{
    for (int n = 0; n < 4; ++n) {
        double r = 1.0;
        for (int k = 0; k < 4; ++k)
            if (k != n) r *= (xi - k) / (double)(n - k);
        a[n] = r;
    }
}

static int bc3(int i, int n, int bc)
{
    if (bc == 0) {
        int r = i % n;
        return r < 0 ? r + n : r;
    }
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

static int64_t node3(const orc3_params *P, int x, int y, int z)
{
    return ((int64_t)bc3(z, P->nz, P->bc_z) * P->ny + bc3(y, P->ny, P->bc_y)) * P->nx + bc3(x, P->nx, P->bc_x);
}

/* isotropic D3Q27 gradient (1/T_L) sum W c phi(x + c) and Laplacian (2/T_L) sum W (phi(x + c) - phi(x)) */
static void grad3(const orc3_params *P, const double *phi, int x, int y, int z, double g[3])
{
    g[0] = g[1] = g[2] = 0.0;
    for (int i = 0; i < Q3; ++i) {
        double v = phi[node3(P, x + c3x(i), y + c3y(i), z + c3z(i))];
        g[0] += w3(i) * c3x(i) * v;
        g[1] += w3(i) * c3y(i) * v;
        g[2] += w3(i) * c3z(i) * v;
    }
    for (int k = 0; k < 3; ++k) g[k] /= TL3;
}

static double lap3(const orc3_params *P, const double *phi, int x, int y, int z)
{
    double c = phi[node3(P, x, y, z)], s = 0.0;
    for (int i = 0; i < Q3; ++i) s += w3(i) * (phi[node3(P, x + c3x(i), y + c3y(i), z + c3z(i))] - c);
    return 2.0 * s / TL3;
}

/* Non-local fields from rho, T (Eq. korteweg, gtilde): nl[6 N]: Fx, Fy, Fz, rho E_lambda, M_0 */
void orc3_nonlocal(const orc3_params *P, const double *rho, const double *T, double *nl)
{
    int64_t N = (int64_t)P->nx * P->ny * P->nz;
    double *K = malloc(sizeof(double) * 9 * N), *q = malloc(sizeof(double) * 3 * N);
    double *h = malloc(sizeof(double) * N), *mu = malloc(sizeof(double) * N), *kc = malloc(sizeof(double) * N);
    double cv = P->R / P->delta;
    for (int64_t n = 0; n < N; ++n) {
        double p = eos_p3(P, rho[n], T[n]);
        double Pg = p > P->p_floor ? p : P->p_floor;
        h[n] = eos_e3(P, rho[n], T[n]) + p / rho[n];
        mu[n] = (P->tau - 0.5) * Pg * P->dt;
        kc[n] = P->k_cond >= 0.0 ? P->k_cond : mu[n] * (cv + P->R);
    }
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                int64_t n = ((int64_t)z * P->ny + y) * P->nx + x;
                double gr[3], gh[3], gT[3];
                grad3(P, rho, x, y, z, gr);
                double lr = lap3(P, rho, x, y, z);
                double g2 = gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2];
                double iso = -P->kappa * (rho[n] * lr + 0.5 * g2);
                for (int a = 0; a < 3; ++a)
                    for (int bb = 0; bb < 3; ++bb)
                        K[(3 * a + bb) * N + n] = (a == bb ? iso : 0.0) + P->kappa * gr[a] * gr[bb];
                grad3(P, h, x, y, z, gh);
                grad3(P, T, x, y, z, gT);
                for (int a = 0; a < 3; ++a) q[a * N + n] = -mu[n] * gh[a] + kc[n] * gT[a];
                nl[3 * N + n] = 0.5 * P->kappa * g2;
            }
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                int64_t n = ((int64_t)z * P->ny + y) * P->nx + x;
                double F[3] = {0.0, 0.0, 0.0}, div_q = 0.0;
                for (int a = 0; a < 3; ++a) {
                    double gK[3];
                    for (int bb = 0; bb < 3; ++bb) {
                        grad3(P, K + (3 * a + bb) * N, x, y, z, gK);
                        F[a] -= gK[bb];          /* F_a = -d_b K_ab (K symmetric) */
                    }
                    double gq[3];
                    grad3(P, q + a * N, x, y, z, gq);
                    div_q += gq[a];
                }
                nl[0 * N + n] = F[0];
                nl[1 * N + n] = F[1];
                nl[2 * N + n] = F[2];
                nl[4 * N + n] = 2.0 * div_q;
            }
    free(K); free(q); free(h); free(mu); free(kc);
}

/* co-moving equilibrium of (rho, u, T) with the interface energy (Eq. geq) */
void orc3_init(const orc3_params *P, const double *rho, const double *ux, const double *uy,
               const double *uz, const double *T, double *st)
{
    int64_t N = (int64_t)P->nx * P->ny * P->nz;
    for (int z = 0; z < P->nz; ++z)
        for (int y = 0; y < P->ny; ++y)
            for (int x = 0; x < P->nx; ++x) {
                int64_t n = ((int64_t)z * P->ny + y) * P->nx + x;
                double gr[3];
                grad3(P, rho, x, y, z, gr);
                double p = eos_p3(P, rho[n], T[n]);
                double Pg = p > P->p_floor ? p : P->p_floor;
                double th = Pg / (rho[n] * TL3), s = sqrt(th), e = eos_e3(P, rho[n], T[n]);
                double lam_e = P->kappa * (gr[0] * gr[0] + gr[1] * gr[1] + gr[2] * gr[2]);
                for (int i = 0; i < Q3; ++i) {
                    double vx = s * c3x(i) + ux[n], vy = s * c3y(i) + uy[n], vz = s * c3z(i) + uz[n];
                    st[(P3_F + i) * N + n] = rho[n] * w3(i);
                    st[(P3_G + i) * N + n] = rho[n] * w3(i) * (2.0 * e - DIM3 * Pg / rho[n] + vx * vx + vy * vy + vz * vz)
                                             + w3(i) * lam_e;
                }
                st[P3_TH * N + n] = th;
                st[P3_UX * N + n] = ux[n]; st[P3_UY * N + n] = uy[n]; st[P3_UZ * N + n] = uz[n];
                st[P3_RHO * N + n] = rho[n]; st[P3_T * N + n] = T[n];
                st[P3_UHX * N + n] = ux[n]; st[P3_UHY * N + n] = uy[n]; st[P3_UHZ * N + n] = uz[n];
            }
}

static void node_moments3(const orc3_params *P, const double *st, double *mf, double *mg)
{
    int64_t N = (int64_t)P->nx * P->ny * P->nz;
    for (int64_t n = 0; n < N; ++n) {
        double lam[4] = {st[P3_TH * N + n], st[P3_UX * N + n], st[P3_UY * N + n], st[P3_UZ * N + n]};
        double M[Q3 * Q3], f[Q3], g[Q3];
        orc3_moment_matrix(lam, M);
        for (int i = 0; i < Q3; ++i) { f[i] = st[(P3_F + i) * N + n]; g[i] = st[(P3_G + i) * N + n]; }
        apply3(M, f, mf + Q3 * n);
        apply3(M, g, mg + Q3 * n);
    }
}

/* streaming into node (X, Y, Z) in gauge lam: departure point x - v_i dt, 4x4x4 stencil */
static int stream3(const orc3_params *P, const double *mf, const double *mg, int X, int Y, int Z,
                   const double lam[4], double *ft, double *gt)
{
    double Md[Q3 * Q3];
    int piv[Q3];
    orc3_moment_matrix(lam, Md);
    if (lu3(Md, piv)) return 1;
    double s = sqrt(lam[0]);
    for (int i = 0; i < Q3; ++i) {
        double v[3] = {s * c3x(i) + lam[1], s * c3y(i) + lam[2], s * c3z(i) + lam[3]};
        double xd = X - v[0] * P->dt, yd = Y - v[1] * P->dt, zd = Z - v[2] * P->dt;
        double x0 = floor(xd) - 1.0, y0 = floor(yd) - 1.0, z0 = floor(zd) - 1.0;
        double ax[4], ay[4], az[4];
        lagr4(xd - x0, ax);
        lagr4(yd - y0, ay);
        lagr4(zd - z0, az);
        double sf = 0.0, sg = 0.0;
        for (int l = 0; l < 4; ++l)
            for (int m = 0; m < 4; ++m)
                for (int k = 0; k < 4; ++k) {
                    int64_t nd = node3(P, (int)x0 + k, (int)y0 + m, (int)z0 + l);
                    double fp[Q3], gp[Q3];
                    lu3_solve(Md, piv, mf + Q3 * nd, fp);
                    lu3_solve(Md, piv, mg + Q3 * nd, gp);
                    double w = ax[k] * ay[m] * az[l];
                    sf += w * fp[i];
                    sg += w * gp[i];
                }
        ft[i] = sf;
        gt[i] = sg;
    }
    return 0;
}

/* out: rho, ux, uy, uz, uhx, uhy, uhz, E, e, T, p, P, theta*   (13 values) */
void orc3_macro(const orc3_params *P, const double lam[4], const double *ft, const double *gt,
                const double F[3], double rEl, double out[13])
{
    double s = sqrt(lam[0]);
    double rho = 0.0, j[3] = {0.0, 0.0, 0.0}, sg = 0.0;
    for (int i = 0; i < Q3; ++i) {
        rho += ft[i];
        j[0] += ft[i] * (s * c3x(i) + lam[1]);
        j[1] += ft[i] * (s * c3y(i) + lam[2]);
        j[2] += ft[i] * (s * c3z(i) + lam[3]);
        sg += gt[i];
    }
    double u[3], uh[3];
    for (int a = 0; a < 3; ++a) {
        u[a] = j[a] / rho;
        uh[a] = u[a] + F[a] * P->dt / (2.0 * rho);
    }
    double E = sg / (2.0 * rho);
    double e = E - 0.5 * (uh[0] * uh[0] + uh[1] * uh[1] + uh[2] * uh[2]) - rEl / rho;
    double T = (e + P->a * rho) / (P->R / P->delta);
    double p = eos_p3(P, rho, T);
    double Pg = p > P->p_floor ? p : P->p_floor;
    out[0] = rho; out[1] = u[0]; out[2] = u[1]; out[3] = u[2];
    out[4] = uh[0]; out[5] = uh[1]; out[6] = uh[2];
    out[7] = E; out[8] = e; out[9] = T; out[10] = p; out[11] = Pg; out[12] = Pg / (rho * TL3);
}

/* BGK collision in the streaming gauge lam (Eqs. f/g collision, S-i, gtilde, new geq) */
int orc3_collide(const orc3_params *P, const double lam[4], const double *ft, const double *gt,
                 const double mac[13], const double F[3], double M0, double *fo, double *go)
{
    double omega = 1.0 / P->tau, dt = P->dt;
    double rho = mac[0], u[3] = {mac[1], mac[2], mac[3]}, uh[3] = {mac[4], mac[5], mac[6]};
    double E = mac[7], Pg = mac[11], ths = mac[12];
    double lst[4] = {ths, u[0], u[1], u[2]};
    double lsh[4] = {ths, u[0] + F[0] * dt / rho, u[1] + F[1] * dt / rho, u[2] + F[2] * dt / rho};
    double feq_s[Q3], feq[Q3], fsh[Q3];
    for (int i = 0; i < Q3; ++i) feq_s[i] = rho * w3(i);
    if (transform3(lst, lam, feq_s, feq)) return 1;
    if (transform3(lsh, lam, feq_s, fsh)) return 1;
    for (int i = 0; i < Q3; ++i) fo[i] = ft[i] + omega * (feq[i] - ft[i]) + (fsh[i] - feq[i]);

    double H = E + Pg / rho;
    double I[3][3], Mv[3], Nt[3][3];
    for (int a = 0; a < 3; ++a)
        for (int bb = 0; bb < 3; ++bb)
            I[a][bb] = uh[a] * F[bb] + F[a] * uh[bb] + dt * F[a] * F[bb] * E / (2.0 * Pg);
    for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int bb = 0; bb < 3; ++bb) s += I[a][bb] * u[bb];
        Mv[a] = (dt * rho / Pg) * (F[a] * H - s);
        for (int bb = 0; bb < 3; ++bb) Nt[a][bb] = (a == bb ? rho : 0.0) + (dt * rho / (2.0 * Pg)) * I[a][bb];
    }
    double sst = sqrt(ths);
    double geq_s[Q3], gc_s[Q3], ph_s[Q3], geq[Q3], gc[Q3], ph[Q3];
    double work = uh[0] * F[0] + uh[1] * F[1] + uh[2] * F[2];
    for (int i = 0; i < Q3; ++i) {
        double c[3] = {c3x(i), c3y(i), c3z(i)}, v[3];
        for (int a = 0; a < 3; ++a) v[a] = sst * c[a] + u[a];
        double g = 2.0 * rho * E;
        for (int a = 0; a < 3; ++a) {
            g += Mv[a] * (v[a] - u[a]);
            for (int bb = 0; bb < 3; ++bb)
                g += Nt[a][bb] * (v[a] * v[bb] - (a == bb ? Pg / rho : 0.0) - u[a] * u[bb]);
        }
        geq_s[i] = w3(i) * g;
        double uc = u[0] * c[0] + u[1] * c[1] + u[2] * c[2];
        double v2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
        gc_s[i] = M0 * w3(i) * (1.0 + rho * uc * uc / (2.0 * Pg * TL3) - rho * v2 / (2.0 * Pg) + DIM3 / 2.0);
        ph_s[i] = 2.0 * w3(i) * work;
    }
    if (transform3(lst, lam, geq_s, geq)) return 1;
    if (transform3(lst, lam, gc_s, gc)) return 1;
    if (transform3(lst, lam, ph_s, ph)) return 1;
    for (int i = 0; i < Q3; ++i) go[i] = gt[i] + omega * (geq[i] - gt[i]) + dt * (gc[i] + ph[i]);
    return 0;
}

static int step_node3(const orc3_params *P, const double *st, const double *mf, const double *mg,
                      const double *nl, int X, int Y, int Z, double *out)
{
    int64_t N = (int64_t)P->nx * P->ny * P->nz;
    int64_t n = ((int64_t)Z * P->ny + Y) * P->nx + X;
    double F[3] = {nl[0 * N + n], nl[1 * N + n], nl[2 * N + n]}, rEl = nl[3 * N + n], M0 = nl[4 * N + n];
    double lam[4] = {st[P3_TH * N + n], st[P3_UX * N + n], st[P3_UY * N + n], st[P3_UZ * N + n]};
    double ft[Q3], gt[Q3], mac[13];
    int it = 0, conv = 0;
    for (;;) {
        ++it;
        if (stream3(P, mf, mg, X, Y, Z, lam, ft, gt)) return 0;
        orc3_macro(P, lam, ft, gt, F, rEl, mac);
        double sl = sqrt(lam[0]);
        double r = fabs(mac[12] - lam[0]) / lam[0];
        for (int a = 0; a < 3; ++a) {
            double ra = fabs(mac[1 + a] - lam[1 + a]) / sl;
            r = r > ra ? r : ra;
        }
        if (r <= P->tol) { conv = 1; break; }
        if (it >= P->max_iter) break;
        lam[0] = mac[12]; lam[1] = mac[1]; lam[2] = mac[2]; lam[3] = mac[3];
    }
    double fo[Q3], go[Q3];
    if (orc3_collide(P, lam, ft, gt, mac, F, M0, fo, go)) return 0;
    for (int i = 0; i < Q3; ++i) { out[P3_F + i] = fo[i]; out[P3_G + i] = go[i]; }
    out[P3_TH] = lam[0]; out[P3_UX] = lam[1]; out[P3_UY] = lam[2]; out[P3_UZ] = lam[3];
    out[P3_RHO] = mac[0]; out[P3_T] = mac[9];
    out[P3_UHX] = mac[4]; out[P3_UHY] = mac[5]; out[P3_UHZ] = mac[6];
    return conv ? it : -it;
}

/* one time step of the whole grid (lagged non-local terms); stats as the 2-D oracle's */
int orc3_step(const orc3_params *P, const double *in, double *out, double stats[4])
{
    int64_t N = (int64_t)P->nx * P->ny * P->nz;
    double *mf = malloc(sizeof(double) * Q3 * N), *mg = malloc(sizeof(double) * Q3 * N);
    double *nl = malloc(sizeof(double) * 5 * N);
    node_moments3(P, in, mf, mg);
    orc3_nonlocal(P, in + P3_RHO * N, in + P3_T * N, nl);
    double its = 0.0, nonconv = 0.0, fail = 0.0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : its, nonconv, fail)
    for (int64_t n = 0; n < N; ++n) {
        int X = (int)(n % P->nx), Y = (int)((n / P->nx) % P->ny), Z = (int)(n / ((int64_t)P->nx * P->ny));
        double o[NP3];
        int r = step_node3(P, in, mf, mg, nl, X, Y, Z, o);
        if (r == 0) { fail += 1.0; continue; }
        its += (double)(r > 0 ? r : -r);
        if (r < 0) nonconv += 1.0;
        for (int p = 0; p < NP3; ++p) out[p * N + n] = o[p];
    }
    free(mf); free(mg); free(nl);
    if (stats) { stats[0] += its; stats[1] += nonconv; stats[3] += fail; }
    return fail > 0.0;
}

/* one step at the listed nodes only; out: count * NP3 values, node-major */
int orc3_step_nodes(const orc3_params *P, const double *in, const int64_t *nodes, int64_t count, double *out)
{
    int64_t N = (int64_t)P->nx * P->ny * P->nz;
    double *mf = malloc(sizeof(double) * Q3 * N), *mg = malloc(sizeof(double) * Q3 * N);
    double *nl = malloc(sizeof(double) * 5 * N);
    node_moments3(P, in, mf, mg);
    orc3_nonlocal(P, in + P3_RHO * N, in + P3_T * N, nl);
    double fail = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : fail)
    for (int64_t k = 0; k < count; ++k) {
        int64_t n = nodes[k];
        int X = (int)(n % P->nx), Y = (int)((n / P->nx) % P->ny), Z = (int)(n / ((int64_t)P->nx * P->ny));
        if (step_node3(P, in, mf, mg, nl, X, Y, Z, out + k * NP3) == 0) fail += 1.0;
    }
    free(mf); free(mg); free(nl);
    return fail > 0.0;
}
