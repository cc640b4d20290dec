/*
 * pond_oracle.c -- plain, slow FP64 CPU oracle for one time step of the
 * two-population "Particles on Demand" (PonD) kinetic model of a van der Waals
 * fluid (Reyhanian, Dorschner & Karlin, arXiv:2002.09217).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test-suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or constant with the CUDA product path.
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -fPIC -shared (no fast-math, no
 * FMA contraction, so x86-64 and aarch64 give bit-identical results).
 *
 * Everything here follows the paper in its own order:
 *   - shifted particle velocities v_i = sqrt(p/(rho T_L)) c_i + u   (Eq. particle velocity)
 *   - vdW EoS and its internal energy e = C_v T - a rho, C_v = R/delta
 *   - moments rho = sum f, rho u = sum f v, 2 rho E = sum g
 *   - semi-Lagrangian streaming f_i(x) = f_i(x - v_i)       (Eqs. f/g streaming)
 *     with neighbours gauge-transformed by the transfer matrix
 *     G = M_{lambda'}^{-1} M_{lambda}  (SM "Transfer matrix", moment-invariance Eq.)
 *     and then combined by the 4x4 Lagrange stencil (SM "Reconstruction")
 *   - BGK collision with the Korteweg source S_i, the heat-flux correction
 *     and the forced g equilibrium (Eqs. f/g collision, S-i, gtilde, new geq)
 *
 * The transfer matrix is deliberately computed from its definition with an LU
 * solve of the 9x9 moment system, not from any closed form.
 *
 * Readings of points the paper leaves open:
 *   - frame search: predictor = previous-step gauge; corrector = re-stream with the
 *     gauge (max(p,p_floor)/(rho T_L), u) from the streamed moments; stop when the
 *     relative change is <= tol or after max_iter streams.  The node keeps the last
 *     gauge it streamed in; equilibria are built in the co-moving frame
 *     lambda* = (max(p,p_floor)/(rho T_L), u) and carried into that gauge by G.
 *   - force F = -div K; g source phi_i = 2 W_i (uhat . F); interface energy
 *     rho E_lambda = kappa |grad rho|^2 / 2 inside the total energy;
 *     H = E + P/rho with P = max(p, p_floor).
 *   - non-local terms (F, E_lambda, M_0) use the previous step's rho and T with the
 *     isotropic D2Q9 stencils grad = (1/T_L) sum W_i c_i phi(x+c_i),
 *     lap = (2/T_L) sum W_i (phi(x+c_i) - phi(x)).
 *   - the explicit dot-product form of the transfer matrix printed in the paper has
 *     the opposite overall sign of the moment-matching definition; the definition is
 *     what is implemented here.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------------------
 * Lattices (SM "Equilibrium": the model holds for any tensor lattice C = C1 x C1
 * with weights W_i = W_jx W_jy and lattice temperature T_L = sum W c^2):
 *   D2Q9:  C1 = {-1, 0, 1}, W = {1/6, 2/3, 1/6}, T_L = 1/3;
 *   D2Q16: C1 = the four roots of the Hermite polynomial He_4(c) = c^4 - 6 c^2 + 3,
 *          c = -+sqrt(3 +- sqrt 6), with the Gauss-Hermite weights
 *          (3 - sqrt 6)/12 (outer) and (3 + sqrt 6)/12 (inner), T_L = 1.
 * Population index i = q1*jy + jx, c_i = (C1[jx], C1[jy]).
 * ------------------------------------------------------------------------- */
#define QMAX 16
#define NPLANES_MAX (2 * QMAX + 7)

static const double DIM = 2.0;

typedef struct {
    int q1, Q;          /* velocities per dimension, populations */
    double c[4], w[4];  /* C1 and its weights */
    double TL;          /* lattice temperature */
} lattice;
typedef struct {
    int32_t nx, ny;
    int32_t bc_x, bc_y;      /* 0 = periodic, 1 = zero-gradient (index clamp) */
    double a, b, R, delta;   /* EoS constants (see eos_kind), C_v = R/delta */
    double kappa;            /* Korteweg coefficient */
    double tau;              /* BGK relaxation time, omega = 1/tau */
    double k_cond;           /* conductivity; < 0 selects k = mu (C_v + R) */
    double p_floor;          /* pressure floor for the gauge temperature */
    double tol;              /* frame-search tolerance */
    int32_t max_iter;        /* maximum number of streams per node and step */
    int32_t eos_kind;        /* 0: van der Waals p = rho R T/(1 - b rho) - a rho^2;
                                1: Dieterici p = rho R T/(1 - b rho) exp(-a rho/(R T)) (SM);
                                2: near-critical double well (SM "Speed of sound"):
                                   p = p0 + rho E0' - E0, E0 = beta (rho - rho_l)^2 (rho - rho_v)^2 */
    double dt;               /* time step delta t (lattice spacing Delta x = 1) */
    int32_t isothermal;      /* 1: T is held at T_iso (the SM's isothermal runs) */
    int32_t pad;
    double T_iso;
    double sp_beta, sp_rho_l, sp_rho_v, sp_p0;   /* constants of eos_kind 2 */
    int32_t lattice;         /* 0: D2Q9, 1: D2Q16 */
    int32_t pad2;
} orc_params;

static lattice lattice_of(int kind)
{
    lattice L;
    if (kind == 1) {
        double ci = sqrt(3.0 - sqrt(6.0)), co = sqrt(3.0 + sqrt(6.0));
        double wi = (3.0 + sqrt(6.0)) / 12.0, wo = (3.0 - sqrt(6.0)) / 12.0;
        L.q1 = 4;
        L.c[0] = -co; L.c[1] = -ci; L.c[2] = ci; L.c[3] = co;
        L.w[0] = wo; L.w[1] = wi; L.w[2] = wi; L.w[3] = wo;
        L.TL = 1.0;
    } else {
        L.q1 = 3;
        L.c[0] = -1.0; L.c[1] = 0.0; L.c[2] = 1.0; L.c[3] = 0.0;
        L.w[0] = 1.0 / 6.0; L.w[1] = 2.0 / 3.0; L.w[2] = 1.0 / 6.0; L.w[3] = 0.0;
        L.TL = 1.0 / 3.0;
    }
    L.Q = L.q1 * L.q1;
    return L;
}
static double lcx(const lattice *L, int i) { return L->c[i % L->q1]; }
static double lcy(const lattice *L, int i) { return L->c[i / L->q1]; }
static double lw(const lattice *L, int i) { return L->w[i % L->q1] * L->w[i / L->q1]; }

/* plane layout of a state: f_0..f_{Q-1}, g_0..g_{Q-1}, theta, ux, uy, rho, T, uhat */
enum { PX_THETA = 0, PX_UX, PX_UY, PX_RHO, PX_T, PX_UHX, PX_UHY };
static int pl_f(const lattice *L, int i) { (void)L; return i; }
static int pl_g(const lattice *L, int i) { return L->Q + i; }
static int pl_x(const lattice *L, int k) { return 2 * L->Q + k; }
static int nplanes(const lattice *L) { return 2 * L->Q + 7; }

/* The finite-difference stencils of the non-local terms are the isotropic D2Q9 ones on
 * the grid, whatever the velocity set: weights 2/3, 1/6 per dimension, T_L = 1/3. */
static const double ST_TL = 1.0 / 3.0;
static int st_cx(int i) { return i % 3 - 1; }
static int st_cy(int i) { return i / 3 - 1; }
static double st_w1(int c) { return c == 0 ? 2.0 / 3.0 : 1.0 / 6.0; }
static double st_w(int i) { return st_w1(st_cx(i)) * st_w1(st_cy(i)); }

/* ------------------------------ EoS ------------------------------------- */
static double eos_p(const orc_params *P, double rho, double T)
{
    if (P->eos_kind == 1)   /* Dieterici (SM "Coexistence curve") */
        return rho * P->R * T / (1.0 - P->b * rho) * exp(-P->a * rho / (P->R * T));
    if (P->eos_kind == 2) { /* double well: E0 = beta (rho - rho_l)^2 (rho - rho_v)^2 */
        double dl = rho - P->sp_rho_l, dv = rho - P->sp_rho_v;
        double E0 = P->sp_beta * dl * dl * dv * dv;
        double dE0 = 2.0 * P->sp_beta * dl * dv * (dl + dv);
        return P->sp_p0 + rho * dE0 - E0;
    }
    return rho * P->R * T / (1.0 - P->b * rho) - P->a * rho * rho;
}
static double eos_e(const orc_params *P, double rho, double T)
{
    return (P->R / P->delta) * T - P->a * rho;
}
static double eos_T_of_e(const orc_params *P, double rho, double e)
{
    return (e + P->a * rho) / (P->R / P->delta);
}

/* --------------------------- small dense algebra ------------------------ */
static double ipow(double x, int m)
{
    double r = 1.0;
    for (int k = 0; k < m; ++k) r *= x;
    return r;
}

/* Moment orders (m, n), m, n < q1, of the rows of the moment matrix (SM Moments).
 * D2Q9 rows: M00, M10, M01, M11, M20, M02, M21, M12, M22; D2Q16 rows: r = 4 n + m. */
static const int MOM_M9[9] = {0, 1, 0, 1, 2, 0, 2, 1, 2};
static const int MOM_N9[9] = {0, 0, 1, 1, 0, 2, 1, 2, 2};
static int mom_m(const lattice *L, int r) { return L->q1 == 3 ? MOM_M9[r] : r % 4; }
static int mom_n(const lattice *L, int r) { return L->q1 == 3 ? MOM_N9[r] : r / 4; }

/* M_lambda: maps populations of gauge lambda = (theta, ux, uy) to the Q moments
 * M_mn = sum_i f_i (sqrt(theta) c_ix + ux)^m (sqrt(theta) c_iy + uy)^n. */
static void moment_matrix(const lattice *L, const double lam[3], double *M)
{
    const int Q = L->Q;
    double s = sqrt(lam[0]);
    for (int r = 0; r < Q; ++r)
        for (int i = 0; i < Q; ++i) {
            double vx = s * lcx(L, i) + lam[1];
            double vy = s * lcy(L, i) + lam[2];
            M[r * Q + i] = ipow(vx, mom_m(L, r)) * ipow(vy, mom_n(L, r));
        }
}

/* LU factorisation with partial pivoting of a Q x Q matrix, in place; 0 on success. */
static int lu_factor(double *A, int *piv, int Q)
{
    for (int k = 0; k < Q; ++k) {
        int p = k;
        double best = fabs(A[k * Q + k]);
        for (int r = k + 1; r < Q; ++r)
            if (fabs(A[r * Q + k]) > best) { best = fabs(A[r * Q + k]); p = r; }
        piv[k] = p;
        if (best == 0.0) return 1;
        if (p != k)
            for (int c = 0; c < Q; ++c) {
                double t = A[k * Q + c]; A[k * Q + c] = A[p * Q + c]; A[p * Q + c] = t;
            }
        for (int r = k + 1; r < Q; ++r) {
            double l = A[r * Q + k] / A[k * Q + k];
            A[r * Q + k] = l;
            for (int c = k + 1; c < Q; ++c) A[r * Q + c] -= l * A[k * Q + c];
        }
    }
    return 0;
}

static void lu_solve(const double *LU, const int *piv, const double *b, double *x, int Q)
{
    double y[QMAX];
    for (int i = 0; i < Q; ++i) y[i] = b[i];
    for (int k = 0; k < Q; ++k)
        if (piv[k] != k) { double t = y[k]; y[k] = y[piv[k]]; y[piv[k]] = t; }
    for (int i = 0; i < Q; ++i)
        for (int c = 0; c < i; ++c) y[i] -= LU[i * Q + c] * y[c];
    for (int i = Q - 1; i >= 0; --i) {
        for (int c = i + 1; c < Q; ++c) y[i] -= LU[i * Q + c] * y[c];
        y[i] /= LU[i * Q + i];
    }
    for (int i = 0; i < Q; ++i) x[i] = y[i];
}

/* moments M_lambda f (gauge invariant, SM moment-invariance Eq.) */
static void apply_moments(const double *M, const double *f, double *m, int Q)
{
    for (int r = 0; r < Q; ++r) {
        double s = 0.0;
        for (int i = 0; i < Q; ++i) s += M[r * Q + i] * f[i];
        m[r] = s;
    }
}

/* Transfer matrix G_{src}^{dst} = M_dst^{-1} M_src (SM "Transfer matrix").
 * Returns 0 on success. */
static int gauge_matrix(const lattice *L, const double src[3], const double dst[3], double *G)
{
    const int Q = L->Q;
    double Ms[QMAX * QMAX], Md[QMAX * QMAX];
    int piv[QMAX];
    moment_matrix(L, src, Ms);
    moment_matrix(L, dst, Md);
    if (lu_factor(Md, piv, Q)) return 1;
    for (int c = 0; c < Q; ++c) {
        double col[QMAX], x[QMAX];
        for (int r = 0; r < Q; ++r) col[r] = Ms[r * Q + c];
        lu_solve(Md, piv, col, x, Q);
        for (int r = 0; r < Q; ++r) G[r * Q + c] = x[r];
    }
    return 0;
}

/* Exported forms: D2Q9 (the paper's lattice) and any lattice kind. */
void orc_moment_matrix(const double lam[3], double M[81])
{
    lattice L = lattice_of(0);
    moment_matrix(&L, lam, M);
}
void orc_moment_matrix_q(int32_t kind, const double lam[3], double *M)
{
    lattice L = lattice_of(kind);
    moment_matrix(&L, lam, M);
}
int orc_gauge_matrix(const double src[3], const double dst[3], double G[81])
{
    lattice L = lattice_of(0);
    return gauge_matrix(&L, src, dst, G);
}
int orc_gauge_matrix_q(int32_t kind, const double src[3], const double dst[3], double *G)
{
    lattice L = lattice_of(kind);
    return gauge_matrix(&L, src, dst, G);
}

/* Transform a population vector from gauge src to gauge dst: f' = M_dst^{-1} M_src f. */
static int transform(const lattice *L, const double src[3], const double dst[3], const double *f,
                     double *out)
{
    const int Q = L->Q;
    double Ms[QMAX * QMAX], Md[QMAX * QMAX], m[QMAX];
    int piv[QMAX];
    moment_matrix(L, src, Ms);
    apply_moments(Ms, f, m, Q);
    moment_matrix(L, dst, Md);
    if (lu_factor(Md, piv, Q)) return 1;
    lu_solve(Md, piv, m, out, Q);
    return 0;
}

/* Cubic Lagrange basis a_n(xi) = prod_{k != n} (xi - k)/(n - k), n = 0..3
 * (SM "Reconstruction"). */
void orc_lagrange4(double xi, double a[4])
{
    for (int n = 0; n < 4; ++n) {
        double r = 1.0;
        for (int k = 0; k < 4; ++k)
            if (k != n) r *= (xi - k) / (double)(n - k);
        a[n] = r;
    }
}

/* ------------------------------ grid helpers ---------------------------- */
static int bc_index(int i, int n, int bc)
{
    if (bc == 0) {
        int r = i % n;
        return r < 0 ? r + n : r;
    }
    return i < 0 ? 0 : (i >= n ? n - 1 : i);
}

static int64_t node_at(const orc_params *P, int x, int y)
{
    int xx = bc_index(x, P->nx, P->bc_x);
    int yy = bc_index(y, P->ny, P->bc_y);
    return (int64_t)yy * P->nx + xx;
}

/* isotropic D2Q9 gradient: d_alpha phi = (1/T_L) sum_i W_i c_i,alpha phi(x + c_i) */
static void grad_at(const orc_params *P, const double *phi, int x, int y, double g[2])
{
    g[0] = 0.0; g[1] = 0.0;
    for (int i = 0; i < 9; ++i) {
        double v = phi[node_at(P, x + st_cx(i), y + st_cy(i))];
        g[0] += st_w(i) * st_cx(i) * v;
        g[1] += st_w(i) * st_cy(i) * v;
    }
    g[0] /= ST_TL; g[1] /= ST_TL;
}

/* isotropic D2Q9 Laplacian: (2/T_L) sum_i W_i (phi(x + c_i) - phi(x)) */
static double lap_at(const orc_params *P, const double *phi, int x, int y)
{
    double c = phi[node_at(P, x, y)], s = 0.0;
    for (int i = 0; i < 9; ++i)
        s += st_w(i) * (phi[node_at(P, x + st_cx(i), y + st_cy(i))] - c);
    return 2.0 * s / ST_TL;
}

/* ----------------------- non-local (interface) terms --------------------
 * From the previous step's rho and T:
 *   K = -kappa (rho lap rho + |grad rho|^2/2) I + kappa grad rho (x) grad rho  (Eq. korteweg)
 *   F = -div K
 *   rho E_lambda = kappa |grad rho|^2 / 2
 *   M_0 = 2 div(-mu grad h + k grad T), mu = (tau - 1/2) P, h = e + p/rho   (Eq. gtilde)
 * Output arrays nl[4*N]: Fx, Fy, rho E_lambda, M_0. */
void orc_nonlocal(const orc_params *P, const double *rho, const double *T, double *nl)
{
    int64_t N = (int64_t)P->nx * P->ny;
    double *Kxx = malloc(sizeof(double) * N), *Kxy = malloc(sizeof(double) * N);
    double *Kyy = malloc(sizeof(double) * N), *qx = malloc(sizeof(double) * N);
    double *qy = malloc(sizeof(double) * N), *h = malloc(sizeof(double) * N);
    double *mu = malloc(sizeof(double) * N), *kc = malloc(sizeof(double) * N);
    double cv = P->R / P->delta;
    for (int64_t n = 0; n < N; ++n) {
        double p = eos_p(P, rho[n], T[n]);
        double Pg = p > P->p_floor ? p : P->p_floor;
        h[n] = eos_e(P, rho[n], T[n]) + p / rho[n];
        mu[n] = (P->tau - 0.5) * Pg * P->dt;
        kc[n] = P->k_cond >= 0.0 ? P->k_cond : mu[n] * (cv + P->R);
    }
    for (int y = 0; y < P->ny; ++y)
        for (int x = 0; x < P->nx; ++x) {
            int64_t n = (int64_t)y * P->nx + x;
            double gr[2], gh[2], gT[2];
            grad_at(P, rho, x, y, gr);
            double lr = lap_at(P, rho, x, y);
            double iso = -P->kappa * (rho[n] * lr + 0.5 * (gr[0] * gr[0] + gr[1] * gr[1]));
            Kxx[n] = iso + P->kappa * gr[0] * gr[0];
            Kxy[n] = P->kappa * gr[0] * gr[1];
            Kyy[n] = iso + P->kappa * gr[1] * gr[1];
            grad_at(P, h, x, y, gh);
            grad_at(P, T, x, y, gT);
            qx[n] = -mu[n] * gh[0] + kc[n] * gT[0];
            qy[n] = -mu[n] * gh[1] + kc[n] * gT[1];
            nl[2 * N + n] = 0.5 * P->kappa * (gr[0] * gr[0] + gr[1] * gr[1]);
        }
    for (int y = 0; y < P->ny; ++y)
        for (int x = 0; x < P->nx; ++x) {
            int64_t n = (int64_t)y * P->nx + x;
            double dKxx[2], dKxy[2], dKyy[2], dqx[2], dqy[2];
            grad_at(P, Kxx, x, y, dKxx);
            grad_at(P, Kxy, x, y, dKxy);
            grad_at(P, Kyy, x, y, dKyy);
            grad_at(P, qx, x, y, dqx);
            grad_at(P, qy, x, y, dqy);
            nl[0 * N + n] = -(dKxx[0] + dKxy[1]);
            nl[1 * N + n] = -(dKxy[0] + dKyy[1]);
            nl[3 * N + n] = 2.0 * (dqx[0] + dqy[1]);
        }
    free(Kxx); free(Kxy); free(Kyy); free(qx); free(qy); free(h); free(mu); free(kc);
}

/* ------------------------------ initial state ---------------------------
 * Co-moving equilibrium of the given (rho, u, T): f_i = rho W_i and
 * g_i = rho W_i (2e - D P/rho + v_i^2) + W_i kappa |grad rho|^2  (Eq. geq with the
 * interface energy included in the total energy). */
void orc_init(const orc_params *P, const double *rho, const double *ux, const double *uy,
              const double *T, double *state)
{
    int64_t N = (int64_t)P->nx * P->ny;
    lattice L = lattice_of(P->lattice);
    for (int y = 0; y < P->ny; ++y)
        for (int x = 0; x < P->nx; ++x) {
            int64_t n = (int64_t)y * P->nx + x;
            double gr[2];
            grad_at(P, rho, x, y, gr);
            double p = eos_p(P, rho[n], T[n]);
            double Pg = p > P->p_floor ? p : P->p_floor;
            double th = Pg / (rho[n] * L.TL);
            double s = sqrt(th), e = eos_e(P, rho[n], T[n]);
            double lam_e = P->kappa * (gr[0] * gr[0] + gr[1] * gr[1]);
            for (int i = 0; i < L.Q; ++i) {
                double vx = s * lcx(&L, i) + ux[n], vy = s * lcy(&L, i) + uy[n];
                state[pl_f(&L, i) * N + n] = rho[n] * lw(&L, i);
                state[pl_g(&L, i) * N + n] =
                    rho[n] * lw(&L, i) * (2.0 * e - DIM * Pg / rho[n] + vx * vx + vy * vy)
                    + lw(&L, i) * lam_e;
            }
            state[pl_x(&L, PX_THETA) * N + n] = th;
            state[pl_x(&L, PX_UX) * N + n] = ux[n];
            state[pl_x(&L, PX_UY) * N + n] = uy[n];
            state[pl_x(&L, PX_RHO) * N + n] = rho[n];
            state[pl_x(&L, PX_T) * N + n] = T[n];
            state[pl_x(&L, PX_UHX) * N + n] = ux[n];
            state[pl_x(&L, PX_UHY) * N + n] = uy[n];
        }
}

/* ---------------------------- per-node pieces --------------------------- */

/* Gauge-invariant moments of every node's f and g (used by streaming: the
 * transformed neighbour populations are M_{lambda'}^{-1} applied to these). */
static void node_moments(const orc_params *P, const lattice *L, const double *state, double *mf,
                         double *mg)
{
    int64_t N = (int64_t)P->nx * P->ny;
    const int Q = L->Q;
    for (int64_t n = 0; n < N; ++n) {
        double lam[3] = {state[pl_x(L, PX_THETA) * N + n], state[pl_x(L, PX_UX) * N + n],
                         state[pl_x(L, PX_UY) * N + n]};
        double M[QMAX * QMAX], f[QMAX], g[QMAX];
        moment_matrix(L, lam, M);
        for (int i = 0; i < Q; ++i) {
            f[i] = state[pl_f(L, i) * N + n];
            g[i] = state[pl_g(L, i) * N + n];
        }
        apply_moments(M, f, mf + Q * n, Q);
        apply_moments(M, g, mg + Q * n, Q);
    }
}

/* Semi-Lagrangian streaming into node (X, Y) in gauge lam (Eqs. f/g streaming):
 * for each direction i, departure point x_d = x - v_i, x_0 = floor(x_d) - 1, and
 * f~_i = sum_{m,n} a_n(x_d - x_0) a_m(y_d - y_0) [G_{lambda(node)}^{lam} f(node)]_i
 * with node = (x_0 + n, y_0 + m).  mf/mg hold M_{lambda(node)} f(node). */
static int stream_node(const orc_params *P, const lattice *L, const double *mf, const double *mg,
                       int X, int Y, const double lam[3], double *ft, double *gt)
{
    const int Q = L->Q;
    double Md[QMAX * QMAX];
    int piv[QMAX];
    moment_matrix(L, lam, Md);
    if (lu_factor(Md, piv, Q)) return 1;
    double s = sqrt(lam[0]);
    for (int i = 0; i < Q; ++i) {
        double vx = s * lcx(L, i) + lam[1];
        double vy = s * lcy(L, i) + lam[2];
        double xd = (double)X - vx * P->dt, yd = (double)Y - vy * P->dt;
        double x0 = floor(xd) - 1.0, y0 = floor(yd) - 1.0;
        double ax[4], ay[4];
        orc_lagrange4(xd - x0, ax);
        orc_lagrange4(yd - y0, ay);
        double sf = 0.0, sg = 0.0;
        for (int m = 0; m < 4; ++m)
            for (int n = 0; n < 4; ++n) {
                int64_t nd = node_at(P, (int)x0 + n, (int)y0 + m);
                double fp[QMAX], gp[QMAX];
                lu_solve(Md, piv, mf + Q * nd, fp, Q);
                lu_solve(Md, piv, mg + Q * nd, gp, Q);
                sf += ax[n] * ay[m] * fp[i];
                sg += ax[n] * ay[m] * gp[i];
            }
        ft[i] = sf;
        gt[i] = sg;
    }
    return 0;
}

/* Macroscopic fields of streamed populations in gauge lam (moments Eq.):
 * rho = sum f, u = sum f v / rho, E = sum g / (2 rho), uhat = u + F/(2 rho),
 * e = E - |uhat|^2/2 - E_lambda, T from e, p from the EoS, P = max(p, p_floor),
 * theta* = P/(rho T_L).
 * out: rho, ux, uy, uhx, uhy, E, e, T, p, P, theta*   (11 values) */
void orc_macro(const orc_params *P, const double lam[3], const double *ft, const double *gt,
               double Fx, double Fy, double rEl, double out[11])
{
    lattice L = lattice_of(P->lattice);
    double s = sqrt(lam[0]);
    double rho = 0.0, jx = 0.0, jy = 0.0, sg = 0.0;
    for (int i = 0; i < L.Q; ++i) {
        double vx = s * lcx(&L, i) + lam[1], vy = s * lcy(&L, i) + lam[2];
        rho += ft[i];
        jx += ft[i] * vx;
        jy += ft[i] * vy;
        sg += gt[i];
    }
    double ux = jx / rho, uy = jy / rho;
    double uhx = ux + Fx * P->dt / (2.0 * rho), uhy = uy + Fy * P->dt / (2.0 * rho);
    double E = sg / (2.0 * rho);
    double e = E - 0.5 * (uhx * uhx + uhy * uhy) - rEl / rho;
    /* isothermal runs hold T; the energy moments then play no part in theta */
    double T = P->isothermal ? P->T_iso : eos_T_of_e(P, rho, e);
    double p = eos_p(P, rho, T);
    double Pg = p > P->p_floor ? p : P->p_floor;
    out[0] = rho; out[1] = ux; out[2] = uy; out[3] = uhx; out[4] = uhy;
    out[5] = E; out[6] = e; out[7] = T; out[8] = p; out[9] = Pg; out[10] = Pg / (rho * L.TL);
}

/* BGK collision (Eqs. f collision with S_i, g collision with gtilde and phi) in the
 * streaming gauge lam, for streamed populations ft, gt with macroscopic fields mac
 * (from orc_macro) and lagged F, M_0.  Equilibria are built in the co-moving frame
 * lambda* = (theta*, u) and transformed into lam with the transfer matrix.
 * Returns 0 on success. */
int orc_collide(const orc_params *P, const double lam[3], const double *ft, const double *gt,
                const double mac[11], double Fx, double Fy, double M0,
                double *fout, double *gout)
{
    lattice L = lattice_of(P->lattice);
    const int Q = L.Q;
    double omega = 1.0 / P->tau;
    double rho = mac[0], ux = mac[1], uy = mac[2], uhx = mac[3], uhy = mac[4], E = mac[5];
    double Pg = mac[9], ths = mac[10];
    double lst[3] = {ths, ux, uy};
    double dt = P->dt;
    double lsh[3] = {ths, ux + Fx * dt / rho, uy + Fy * dt / rho};

    /* f: f^eq = G_{lambda*}^{lam}[rho W], S = G_{lambda*+du}^{lam}[rho W] - f^eq (Eq. S-i) */
    double feq_s[QMAX], feq[QMAX], fsh[QMAX];
    for (int i = 0; i < Q; ++i) feq_s[i] = rho * lw(&L, i);
    if (transform(&L, lst, lam, feq_s, feq)) return 1;
    if (transform(&L, lsh, lam, feq_s, fsh)) return 1;
    for (int i = 0; i < Q; ++i) {
        double S = fsh[i] - feq[i];
        fout[i] = ft[i] + omega * (feq[i] - ft[i]) + S;
    }

    /* g: forced equilibrium (Eq. new geq), heat-flux correction (Eq. gtilde) and
     * force-work source phi, all in lambda*, then carried into lam. */
    double H = E + Pg / rho;
    double Ixx = 2.0 * uhx * Fx + dt * Fx * Fx * E / (2.0 * Pg);
    double Ixy = uhx * Fy + Fx * uhy + dt * Fx * Fy * E / (2.0 * Pg);
    double Iyy = 2.0 * uhy * Fy + dt * Fy * Fy * E / (2.0 * Pg);
    double Mx = (dt * rho / Pg) * (Fx * H - (Ixx * ux + Ixy * uy));
    double My = (dt * rho / Pg) * (Fy * H - (Ixy * ux + Iyy * uy));
    double Nxx = rho + (dt * rho / (2.0 * Pg)) * Ixx;
    double Nxy = (dt * rho / (2.0 * Pg)) * Ixy;
    double Nyy = rho + (dt * rho / (2.0 * Pg)) * Iyy;
    double sst = sqrt(ths);
    double geq_s[QMAX], gc_s[QMAX], ph_s[QMAX], geq[QMAX], gc[QMAX], ph[QMAX];
    for (int i = 0; i < Q; ++i) {
        double cx = lcx(&L, i), cy = lcy(&L, i), W = lw(&L, i);
        double vx = sst * cx + ux, vy = sst * cy + uy;
        double Axx = vx * vx - Pg / rho - ux * ux;
        double Axy = vx * vy - ux * uy;
        double Ayy = vy * vy - Pg / rho - uy * uy;
        geq_s[i] = W * (2.0 * rho * E + Mx * (vx - ux) + My * (vy - uy)
                        + Nxx * Axx + 2.0 * Nxy * Axy + Nyy * Ayy);
        double uc = ux * cx + uy * cy;
        gc_s[i] = M0 * W * (1.0 + rho * uc * uc / (2.0 * Pg * L.TL)
                            - rho * (vx * vx + vy * vy) / (2.0 * Pg) + DIM / 2.0);
        ph_s[i] = 2.0 * W * (uhx * Fx + uhy * Fy);
    }
    if (transform(&L, lst, lam, geq_s, geq)) return 1;
    if (transform(&L, lst, lam, gc_s, gc)) return 1;
    if (transform(&L, lst, lam, ph_s, ph)) return 1;
    for (int i = 0; i < Q; ++i)
        gout[i] = gt[i] + omega * (geq[i] - gt[i]) + dt * (gc[i] + ph[i]);
    return 0;
}

/* One node of one time step.  nl holds the lagged non-local fields.  Writes the
 * node's output values (plane order) to out; returns the number of streams,
 * negated if the frame search did not converge, 0 on a numerical failure. */
static int step_node(const orc_params *P, const lattice *L, const double *state, const double *mf,
                     const double *mg, const double *nl, int X, int Y, double *out, int *clamped)
{
    int64_t N = (int64_t)P->nx * P->ny;
    int64_t n = (int64_t)Y * P->nx + X;
    const int Q = L->Q;
    double Fx = nl[0 * N + n], Fy = nl[1 * N + n], rEl = nl[2 * N + n], M0 = nl[3 * N + n];
    double lam[3] = {state[pl_x(L, PX_THETA) * N + n], state[pl_x(L, PX_UX) * N + n],
                     state[pl_x(L, PX_UY) * N + n]};
    double ft[QMAX], gt[QMAX], mac[11];
    int it = 0, converged = 0;
    for (;;) {
        ++it;
        if (stream_node(P, L, mf, mg, X, Y, lam, ft, gt)) return 0;
        orc_macro(P, lam, ft, gt, Fx, Fy, rEl, mac);
        double r0 = fabs(mac[10] - lam[0]) / lam[0];
        double r1 = fabs(mac[1] - lam[1]) / sqrt(lam[0]);
        double r2 = fabs(mac[2] - lam[2]) / sqrt(lam[0]);
        double r = r0 > r1 ? r0 : r1;
        r = r > r2 ? r : r2;
        if (r <= P->tol) { converged = 1; break; }
        if (it >= P->max_iter) break;
        lam[0] = mac[10]; lam[1] = mac[1]; lam[2] = mac[2];
    }
    double fo[QMAX], go[QMAX];
    if (orc_collide(P, lam, ft, gt, mac, Fx, Fy, M0, fo, go)) return 0;
    for (int i = 0; i < Q; ++i) { out[pl_f(L, i)] = fo[i]; out[pl_g(L, i)] = go[i]; }
    out[pl_x(L, PX_THETA)] = lam[0]; out[pl_x(L, PX_UX)] = lam[1]; out[pl_x(L, PX_UY)] = lam[2];
    out[pl_x(L, PX_RHO)] = mac[0]; out[pl_x(L, PX_T)] = mac[7];
    out[pl_x(L, PX_UHX)] = mac[3]; out[pl_x(L, PX_UHY)] = mac[4];
    *clamped = mac[8] < P->p_floor;
    return converged ? it : -it;
}

/* ------------------------------ public steps ---------------------------- */

/* Stream one node in a given gauge (for unit tests of the streaming stage). */
int orc_stream_node(const orc_params *P, const double *state, int X, int Y, const double lam[3],
                    double *ft, double *gt)
{
    int64_t N = (int64_t)P->nx * P->ny;
    lattice L = lattice_of(P->lattice);
    double *mf = malloc(sizeof(double) * L.Q * N), *mg = malloc(sizeof(double) * L.Q * N);
    node_moments(P, &L, state, mf, mg);
    int rc = stream_node(P, &L, mf, mg, X, Y, lam, ft, gt);
    free(mf); free(mg);
    return rc;
}

/* Full time step of the whole grid from the state `in`, with the non-local terms (F,
 * rho E_lambda, M_0) built from the rho and T planes of the state `nl_src`: `in` itself
 * for the lagged reading, or a first pass's result for the current-time one.
 * stats[0] += streams, stats[1] += non-converged nodes, stats[2] += nodes with
 * p < p_floor, stats[3] += numerical failures.  Returns 0 on success. */
int orc_step_nl(const orc_params *P, const double *in, const double *nl_src, double *out,
                double stats[4])
{
    int64_t N = (int64_t)P->nx * P->ny;
    lattice L = lattice_of(P->lattice);
    const int NP = nplanes(&L);
    double *mf = malloc(sizeof(double) * L.Q * N), *mg = malloc(sizeof(double) * L.Q * N);
    double *nl = malloc(sizeof(double) * 4 * N);
    node_moments(P, &L, in, mf, mg);
    orc_nonlocal(P, nl_src + pl_x(&L, PX_RHO) * N, nl_src + pl_x(&L, PX_T) * N, nl);
    double its = 0.0, nonconv = 0.0, clamp = 0.0, fail = 0.0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : its, nonconv, clamp, fail)
    for (int64_t n = 0; n < N; ++n) {
        int X = (int)(n % P->nx), Y = (int)(n / P->nx);
        double o[NPLANES_MAX];
        int cl = 0;
        int r = step_node(P, &L, in, mf, mg, nl, X, Y, o, &cl);
        if (r == 0) { fail += 1.0; continue; }
        its += (double)(r > 0 ? r : -r);
        if (r < 0) nonconv += 1.0;
        clamp += cl;
        for (int p = 0; p < NP; ++p) out[p * N + n] = o[p];
    }
    free(mf); free(mg); free(nl);
    if (stats) { stats[0] += its; stats[1] += nonconv; stats[2] += clamp; stats[3] += fail; }
    return fail > 0.0;
}

/* Full time step with the lagged non-local terms (reading R10). */
int orc_step(const orc_params *P, const double *in, double *out, double stats[4])
{
    return orc_step_nl(P, in, in, out, stats);
}

/* Step only the listed nodes (flat indices y*nx + x) from the full previous state.
 * out holds count * (2Q + 7) values, node-major.  Returns 0 on success. */
int orc_step_nodes(const orc_params *P, const double *in, const int64_t *nodes, int64_t count,
                   double *out, double stats[4])
{
    int64_t N = (int64_t)P->nx * P->ny;
    lattice L = lattice_of(P->lattice);
    const int NP = nplanes(&L);
    double *mf = malloc(sizeof(double) * L.Q * N), *mg = malloc(sizeof(double) * L.Q * N);
    double *nl = malloc(sizeof(double) * 4 * N);
    node_moments(P, &L, in, mf, mg);
    orc_nonlocal(P, in + pl_x(&L, PX_RHO) * N, in + pl_x(&L, PX_T) * N, nl);
    double its = 0.0, nonconv = 0.0, clamp = 0.0, fail = 0.0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : its, nonconv, clamp, fail)
    for (int64_t k = 0; k < count; ++k) {
        int64_t n = nodes[k];
        int X = (int)(n % P->nx), Y = (int)(n / P->nx);
        int cl = 0;
        int r = step_node(P, &L, in, mf, mg, nl, X, Y, out + k * NP, &cl);
        if (r == 0) { fail += 1.0; continue; }
        its += (double)(r > 0 ? r : -r);
        if (r < 0) nonconv += 1.0;
        clamp += cl;
    }
    free(mf); free(mg); free(nl);
    if (stats) { stats[0] += its; stats[1] += nonconv; stats[2] += clamp; stats[3] += fail; }
    return fail > 0.0;
}

/* Macroscopic output fields: rho, uhat_x, uhat_y, T, p (EoS). */
void orc_moments(const orc_params *P, const double *state, double *rho, double *ux, double *uy,
                 double *T, double *p)
{
    int64_t N = (int64_t)P->nx * P->ny;
    lattice L = lattice_of(P->lattice);
    for (int64_t n = 0; n < N; ++n) {
        rho[n] = state[pl_x(&L, PX_RHO) * N + n];
        ux[n] = state[pl_x(&L, PX_UHX) * N + n];
        uy[n] = state[pl_x(&L, PX_UHY) * N + n];
        T[n] = state[pl_x(&L, PX_T) * N + n];
        p[n] = eos_p(P, rho[n], T[n]);
    }
}

int orc_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
