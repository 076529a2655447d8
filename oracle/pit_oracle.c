/*
 * pit_oracle.c -- plain, slow, FP64 CPU oracle for the all-at-once BDF1 Newton
 * method of Yamaleev & Paudel, "A New Parallel-in-time Direct Inverse Method for
 * Nonlinear Differential Equations" (arXiv 2406.00878).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the independent checker of the CUDA
 * library: only the tests, the smoke check and the benchmark's CPU-baseline leg
 * load it.  It shares no code, header, table or helper with the CUDA path.
 *
 * Everything is IEEE FP64, written as plain loops in the order and notation of
 * the paper. The default build is single-threaded; the timing build (-fopenmp)
 * spreads only loops whose iterations are independent element by element -- the
 * levels of the residual and the Jacobian, the rows of a matrix-vector product,
 * the entries of a vector update -- so both builds return the same bits (dot
 * products, norms and the level chain stay sequential):
 *   - eq. 3  spatial operator F (central convective fluxes, conservative viscous
 *            fluxes with mid-point viscosities) and the BDF1 time difference;
 *   - eq. 4  the all-at-once system over all time levels n = 1..N_t;
 *   - eq. 5  the tau-scaled Newton residual r^n and the blocks
 *            A_n = I + tau dF/du (eq. 6, diagonal blocks; sub-diagonal -I);
 *   - eq. 7  the exact block inverse, applied in its nested (Horner) form
 *            du^n = A_n^{-1} (r^n + du^{n-1}) that the proof of Theorem 1 uses;
 *   - Sec. 8 the per-level linear solver: a banded direct solver without
 *            pivoting; for large levels a Jacobi-preconditioned BiCGStab
 *            (van der Vorst 1992) to a stated tolerance.
 *   - Sec. 2 sequential BDF1 time marching with Newton at every step.
 *
 * Readings of points the paper leaves open (kept identical on the GPU side):
 *   - mid-point viscosity mu_{i+1/2} = mu((u_i + u_{i+1}) / 2), the viscosity
 *     of the mid-point average; with N = grid intervals this reading reproduces
 *     every digit of Table grconv_heat (Sec. 8.1);
 *   - the API counts INTERIOR nodes nx, ny; h_x = (x_R - x_L)/(nx + 1) (the
 *     paper's N_x grid intervals are nx + 1);
 *   - closures: f = g = beta u^2/2 (beta = 1 Burgers, 0 heat),
 *               mu(u) = mu_a + mu_b u^2 (heat mu_0 u^2 is mu_a=0, mu_b=mu_0);
 *   - source q^n and boundary data b are taken at t^n (implicit level).
 *
 * Layouts (shared with the C ABI as an interface, not as code):
 *   level vector   u[j*nx + i], j = y row, i = x (fastest)
 *   space-time     U[(n-1)*Ns + j*nx + i], n = 1..M
 *   boundary level bnd[0..nx)        south row  (j = -1)
 *                  bnd[nx..2nx)      north row  (j = ny)
 *                  bnd[2nx..2nx+ny)  west column (i = -1)
 *                  bnd[2nx+ny..)     east column (i = nx)
 *   coefficients   coef[c][n-1][Ns], c = 0..4 -> C, W, E, S, N of A_n
 */
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Threads of the timing build (no effect in the single-threaded build); returns the
 * number of threads the parallel loops will use. */
int oracle_set_threads(int n) {
#ifdef _OPENMP
    if (n > 0) omp_set_num_threads(n);
    return omp_get_max_threads();
#else
    (void)n;
    return 1;
#endif
}

typedef struct {
    int nx, ny;
    double xl, xr, yl, yr;
} og_grid;

typedef struct {
    int equation; /* 0 = nonlinear heat (f = g = 0), 1 = Burgers (f = g = u^2/2) */
    double mu_a, mu_b;
} og_params;

/* ---------------------------------------------------------------- closures */

static double clo_f(const og_params* p, double u) { return p->equation == 1 ? 0.5 * u * u : 0.0; }
static double clo_fp(const og_params* p, double u) { return p->equation == 1 ? u : 0.0; }
static double clo_mu(const og_params* p, double u) { return p->mu_a + p->mu_b * u * u; }
static double clo_mup(const og_params* p, double u) { return 2.0 * p->mu_b * u; }

static double grid_hx(const og_grid* g) { return (g->xr - g->xl) / (g->nx + 1); }
static double grid_hy(const og_grid* g) { return (g->yr - g->yl) / (g->ny + 1); }

/* Value of u at (j, i) where j in [-1, ny], i in [-1, nx]; off-interior nodes read
 * the Dirichlet data of eq. 2 (zero when bnd is NULL). Corners are never asked for. */
static double node(const og_grid* g, const double* u, const double* bnd, int j, int i) {
    int nx = g->nx, ny = g->ny;
    if (i >= 0 && i < nx && j >= 0 && j < ny) return u[j * nx + i];
    if (!bnd) return 0.0;
    if (j == -1) return bnd[i];
    if (j == ny) return bnd[nx + i];
    if (i == -1) return bnd[2 * nx + j];
    return bnd[2 * nx + ny + j]; /* i == nx */
}

/* ------------------------------------------------------------ eq. 3: F(u) */

/* F at every interior node of one level: the inviscid central differences minus
 * the conservative viscous differences of eq. 3 (everything except the time term). */
void oracle_F(const og_grid* g, const og_params* p, const double* u, const double* bnd, double* F) {
    double hx = grid_hx(g), hy = grid_hy(g);
    for (int j = 0; j < g->ny; ++j) {
        for (int i = 0; i < g->nx; ++i) {
            double uC = node(g, u, bnd, j, i);
            double uW = node(g, u, bnd, j, i - 1);
            double uE = node(g, u, bnd, j, i + 1);
            double uS = node(g, u, bnd, j - 1, i);
            double uN = node(g, u, bnd, j + 1, i);
            double inv_x = (clo_f(p, uE) - clo_f(p, uW)) / (2.0 * hx);
            double inv_y = (clo_f(p, uN) - clo_f(p, uS)) / (2.0 * hy);
            double mu_e = clo_mu(p, 0.5 * (uC + uE));
            double mu_w = clo_mu(p, 0.5 * (uC + uW));
            double mu_n = clo_mu(p, 0.5 * (uC + uN));
            double mu_s = clo_mu(p, 0.5 * (uC + uS));
            double vis_x = (mu_e * (uE - uC) - mu_w * (uC - uW)) / (hx * hx);
            double vis_y = (mu_n * (uN - uC) - mu_s * (uC - uS)) / (hy * hy);
            F[j * g->nx + i] = inv_x + inv_y - vis_x - vis_y;
        }
    }
}

/* --------------------------------------------------- eq. 4/5: the residual */

/* Residual of one level, the right-hand side of eq. 5:
 *   r^n = -tau [ (u^n - u^{n-1})/tau + F(u^n) - q^n ]. */
void oracle_level_residual(const og_grid* g, const og_params* p, double dt, const double* u_prev,
                           const double* u, const double* bnd, const double* q, double* r) {
    int Ns = g->nx * g->ny;
    double* F = (double*)malloc(sizeof(double) * Ns);
    oracle_F(g, p, u, bnd, F);
    for (int k = 0; k < Ns; ++k) {
        double qk = q ? q[k] : 0.0;
        r[k] = -dt * ((u[k] - u_prev[k]) / dt + F[k] - qk);
    }
    free(F);
}

/* All-at-once residual R = [r^1 .. r^M] of eq. 4-5 for the space-time iterate U. */
void oracle_residual(const og_grid* g, const og_params* p, int M, double dt, const double* u0,
                     const double* bc, const double* q, const double* U, double* R) {
    int Ns = g->nx * g->ny, nb = 2 * g->nx + 2 * g->ny;
#pragma omp parallel for schedule(static)
    for (int n = 1; n <= M; ++n) {
        const double* u_prev = (n == 1) ? u0 : U + (size_t)(n - 2) * Ns;
        oracle_level_residual(g, p, dt, u_prev, U + (size_t)(n - 1) * Ns, bc ? bc + (size_t)(n - 1) * nb : NULL,
                              q ? q + (size_t)(n - 1) * Ns : NULL, R + (size_t)(n - 1) * Ns);
    }
}

/* ------------------------------------------- eq. 5/6: the Jacobian blocks */

/* The five nonzeros per row of A_n = I + tau dF/du at u (eq. 5-6), written out
 * from differentiating eq. 3 term by term. Couplings to boundary nodes are zero
 * (they are data, not unknowns). cC,cW,cE,cS,cN each hold Ns values. */
void oracle_level_jacobian(const og_grid* g, const og_params* p, double dt, const double* u, const double* bnd,
                           double* cC, double* cW, double* cE, double* cS, double* cN) {
    double hx = grid_hx(g), hy = grid_hy(g);
    double hx2 = hx * hx, hy2 = hy * hy;
    for (int j = 0; j < g->ny; ++j) {
        for (int i = 0; i < g->nx; ++i) {
            int k = j * g->nx + i;
            double uC = node(g, u, bnd, j, i);
            double uW = node(g, u, bnd, j, i - 1);
            double uE = node(g, u, bnd, j, i + 1);
            double uS = node(g, u, bnd, j - 1, i);
            double uN = node(g, u, bnd, j + 1, i);
            /* mid-point viscosities and their derivatives d mu_e / d u_C = d mu_e / d u_E */
            double mu_e = clo_mu(p, 0.5 * (uC + uE)), dmu_e = 0.5 * clo_mup(p, 0.5 * (uC + uE));
            double mu_w = clo_mu(p, 0.5 * (uC + uW)), dmu_w = 0.5 * clo_mup(p, 0.5 * (uC + uW));
            double mu_n = clo_mu(p, 0.5 * (uC + uN)), dmu_n = 0.5 * clo_mup(p, 0.5 * (uC + uN));
            double mu_s = clo_mu(p, 0.5 * (uC + uS)), dmu_s = 0.5 * clo_mup(p, 0.5 * (uC + uS));
            /* dF_C/du_E, dF_C/du_W and the same in y */
            double dE = clo_fp(p, uE) / (2.0 * hx) - (mu_e + dmu_e * (uE - uC)) / hx2;
            double dW = -clo_fp(p, uW) / (2.0 * hx) - (mu_w - dmu_w * (uC - uW)) / hx2;
            double dN = clo_fp(p, uN) / (2.0 * hy) - (mu_n + dmu_n * (uN - uC)) / hy2;
            double dS = -clo_fp(p, uS) / (2.0 * hy) - (mu_s - dmu_s * (uC - uS)) / hy2;
            /* dF_C/du_C: only the viscous terms depend on u_C */
            double dC = (mu_e + mu_w - dmu_e * (uE - uC) + dmu_w * (uC - uW)) / hx2 +
                        (mu_n + mu_s - dmu_n * (uN - uC) + dmu_s * (uC - uS)) / hy2;
            cC[k] = 1.0 + dt * dC;
            cW[k] = (i > 0) ? dt * dW : 0.0;
            cE[k] = (i < g->nx - 1) ? dt * dE : 0.0;
            cS[k] = (j > 0) ? dt * dS : 0.0;
            cN[k] = (j < g->ny - 1) ? dt * dN : 0.0;
        }
    }
}

/* All blocks A_1..A_M; coef holds 5*M*Ns values laid out coef[c][n-1][k]. */
void oracle_jacobian(const og_grid* g, const og_params* p, int M, double dt, const double* bc, const double* U,
                     double* coef) {
    size_t Ns = (size_t)g->nx * g->ny, plane = (size_t)M * Ns;
    int nb = 2 * g->nx + 2 * g->ny;
#pragma omp parallel for schedule(static)
    for (int n = 1; n <= M; ++n) {
        size_t o = (size_t)(n - 1) * Ns;
        oracle_level_jacobian(g, p, dt, U + o, bc ? bc + (size_t)(n - 1) * nb : NULL, coef + o, coef + plane + o,
                              coef + 2 * plane + o, coef + 3 * plane + o, coef + 4 * plane + o);
    }
}

/* y = A x for one level's 5-point block; coefficient c of the level at cf[c*stride]. */
void oracle_apply_A(int nx, int ny, const double* cf, size_t stride, const double* x, double* y) {
    const double *cC = cf, *cW = cf + stride, *cE = cf + 2 * stride, *cS = cf + 3 * stride, *cN = cf + 4 * stride;
#pragma omp parallel for schedule(static) if (nx * ny >= 16384)
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int k = j * nx + i;
            double s = cC[k] * x[k];
            if (i > 0) s += cW[k] * x[k - 1];
            if (i < nx - 1) s += cE[k] * x[k + 1];
            if (j > 0) s += cS[k] * x[k - nx];
            if (j < ny - 1) s += cN[k] * x[k + nx];
            y[k] = s;
        }
}

/* ------------------------------------ Sec. 8: banded direct solver, no pivoting */

/* Solve A x = b for one level by LU factorisation in band storage without
 * pivoting; bandwidth nx below and above the diagonal (x-fastest ordering).
 * Returns 0 on success, 1 on a zero pivot. */
int oracle_band_lu_solve(int nx, int ny, const double* cf, size_t stride, const double* b, double* x) {
    int N = nx * ny, p = nx, w = 2 * nx + 1;
    double* a = (double*)calloc((size_t)N * w, sizeof(double));
    const double *cC = cf, *cW = cf + stride, *cE = cf + 2 * stride, *cS = cf + 3 * stride, *cN = cf + 4 * stride;
#define BAND(r, c) a[(size_t)(r) * w + ((c) - (r) + p)]
    for (int j = 0; j < ny; ++j)
        for (int i = 0; i < nx; ++i) {
            int k = j * nx + i;
            BAND(k, k) = cC[k];
            if (i > 0) BAND(k, k - 1) = cW[k];
            if (i < nx - 1) BAND(k, k + 1) = cE[k];
            if (j > 0) BAND(k, k - nx) = cS[k];
            if (j < ny - 1) BAND(k, k + nx) = cN[k];
        }
    for (int k = 0; k < N; ++k) {
        double piv = BAND(k, k);
        if (piv == 0.0) { free(a); return 1; }
        int last = (k + p < N - 1) ? k + p : N - 1;
        for (int r = k + 1; r <= last; ++r) {
            double l = BAND(r, k) / piv;
            BAND(r, k) = l;
            if (l != 0.0)
                for (int c = k + 1; c <= last; ++c) BAND(r, c) -= l * BAND(k, c);
        }
    }
    for (int r = 0; r < N; ++r) { /* L y = b (unit lower) */
        double s = b[r];
        int first = (r - p > 0) ? r - p : 0;
        for (int c = first; c < r; ++c) s -= BAND(r, c) * x[c];
        x[r] = s;
    }
    for (int r = N - 1; r >= 0; --r) { /* U x = y */
        double s = x[r];
        int last = (r + p < N - 1) ? r + p : N - 1;
        for (int c = r + 1; c <= last; ++c) s -= BAND(r, c) * x[c];
        x[r] = s / BAND(r, r);
    }
#undef BAND
    free(a);
    return 0;
}

/* ------------------------- BiCGStab with Jacobi preconditioning (large levels) */

static double dot(const double* a, const double* b, int n) {
    double s = 0.0;
    for (int k = 0; k < n; ++k) s += a[k] * b[k];
    return s;
}

/* Right-preconditioned BiCGStab (van der Vorst 1992), M = diag(A). x holds the
 * start vector on entry. Stops when ||b - A x||_2 <= rtol ||b||_2. Returns the
 * iteration count, or -1 on breakdown / no convergence within maxit. */
int oracle_bicgstab(int nx, int ny, const double* cf, size_t stride, const double* b, double* x, double rtol,
                    int maxit) {
    int N = nx * ny;
    double* buf = (double*)calloc((size_t)N * 8, sizeof(double));
    double *r = buf, *rh = buf + N, *pv = buf + 2 * N, *v = buf + 3 * N, *ph = buf + 4 * N, *s = buf + 5 * N,
           *sh = buf + 6 * N, *t = buf + 7 * N;
    const double* diag = cf;
    oracle_apply_A(nx, ny, cf, stride, x, r);
    for (int k = 0; k < N; ++k) r[k] = b[k] - r[k];
    memcpy(rh, r, sizeof(double) * N);
    double bnorm = sqrt(dot(b, b, N));
    if (bnorm == 0.0) {
        for (int k = 0; k < N; ++k) x[k] = 0.0;
        free(buf);
        return 0;
    }
    double rho_old = 1.0, alpha = 1.0, omega = 1.0;
    int it = 0, ok = 0;
    if (sqrt(dot(r, r, N)) <= rtol * bnorm) ok = 1;
    while (!ok && it < maxit) {
        ++it;
        double rho = dot(rh, r, N);
        if (rho == 0.0) break;
        double beta = (rho / rho_old) * (alpha / omega);
#pragma omp parallel for schedule(static) if (N >= 16384)
        for (int k = 0; k < N; ++k) {
            pv[k] = r[k] + beta * (pv[k] - omega * v[k]);
            ph[k] = pv[k] / diag[k];
        }
        oracle_apply_A(nx, ny, cf, stride, ph, v);
        double rv = dot(rh, v, N);
        if (rv == 0.0) break;
        alpha = rho / rv;
#pragma omp parallel for schedule(static) if (N >= 16384)
        for (int k = 0; k < N; ++k) s[k] = r[k] - alpha * v[k];
        if (sqrt(dot(s, s, N)) <= rtol * bnorm) {
            for (int k = 0; k < N; ++k) x[k] += alpha * ph[k];
            ok = 1;
            break;
        }
#pragma omp parallel for schedule(static) if (N >= 16384)
        for (int k = 0; k < N; ++k) sh[k] = s[k] / diag[k];
        oracle_apply_A(nx, ny, cf, stride, sh, t);
        double tt = dot(t, t, N);
        if (tt == 0.0) break;
        omega = dot(t, s, N) / tt;
#pragma omp parallel for schedule(static) if (N >= 16384)
        for (int k = 0; k < N; ++k) {
            x[k] += alpha * ph[k] + omega * sh[k];
            r[k] = s[k] - omega * t[k];
        }
        if (sqrt(dot(r, r, N)) <= rtol * bnorm) ok = 1;
        if (omega == 0.0) break;
        rho_old = rho;
    }
    free(buf);
    return ok ? it : -1;
}

/* One level solve A x = b with the chosen solver: 1 = banded LU (the paper's),
 * 2 = BiCGStab (rtol), 0 = banded LU when nx*ny <= 4096, else BiCGStab.
 * Returns 0 on success. */
int oracle_level_solve(int nx, int ny, const double* cf, size_t stride, const double* b, double* x, int solver,
                       double rtol) {
    int N = nx * ny;
    if (solver == 0) solver = (N <= 4096) ? 1 : 2;
    if (solver == 1) return oracle_band_lu_solve(nx, ny, cf, stride, b, x);
    for (int k = 0; k < N; ++k) x[k] = 0.0;
    return oracle_bicgstab(nx, ny, cf, stride, b, x, rtol, 100000) < 0 ? 1 : 0;
}

/* ------------------------------------------ eq. 7: the exact block inverse */

/* Solve the block-bidiagonal system of eq. 6 (diagonal blocks A_n, sub-diagonal
 * -I) with its exact inverse of eq. 7, evaluated in nested form:
 *   du^1 = A_1^{-1} r^1,   du^n = A_n^{-1} (r^n + du^{n-1}),  n = 2..M.
 * coef as produced by oracle_jacobian; R and dU hold M*Ns values. */
int oracle_block_solve(int nx, int ny, int M, const double* coef, const double* R, double* dU, int solver,
                       double rtol) {
    size_t Ns = (size_t)nx * ny, plane = (size_t)M * Ns;
    double* rhs = (double*)malloc(sizeof(double) * Ns);
    int err = 0;
    for (int n = 1; n <= M && !err; ++n) {
        size_t o = (size_t)(n - 1) * Ns;
        for (size_t k = 0; k < Ns; ++k) rhs[k] = R[o + k] + (n > 1 ? dU[o - Ns + k] : 0.0);
        err = oracle_level_solve(nx, ny, coef + o, plane, rhs, dU + o, solver, rtol);
    }
    free(rhs);
    return err;
}

/* ----------------------------------------- all-at-once Newton (eq. 4 - 7) */

static double max_abs(const double* a, size_t n) {
    double m = 0.0;
    for (size_t k = 0; k < n; ++k) {
        double v = fabs(a[k]);
        if (v > m || v != v) m = v; /* NaN propagates */
    }
    return m;
}

/* Newton for all time levels at once from the iterate in U (overwritten).
 * Each iteration: R = residual (eq. 5), stop if ||R||_inf <= tol, blocks A_n
 * (eq. 6), dU by the exact block inverse (eq. 7), U += dU. res_hist[k] gets
 * ||R_k||_inf and upd_hist[k] the RMS update of Sec. 8 (either may be NULL,
 * else sized maxit+1). Returns the number of Newton updates applied, or -1 when
 * tol was not met within maxit updates (U holds the last iterate). */
int oracle_newton_all_at_once(const og_grid* g, const og_params* p, int M, double dt, const double* u0,
                              const double* bc, const double* q, double* U, double tol, int maxit, int solver,
                              double lin_rtol, double* res_hist, double* upd_hist) {
    size_t Ns = (size_t)g->nx * g->ny, DOF = (size_t)M * Ns;
    double* R = (double*)malloc(sizeof(double) * DOF);
    double* dU = (double*)malloc(sizeof(double) * DOF);
    double* coef = (double*)malloc(sizeof(double) * DOF * 5);
    int k = 0, done = 0;
    for (;;) {
        oracle_residual(g, p, M, dt, u0, bc, q, U, R);
        double rinf = max_abs(R, DOF);
        if (res_hist) res_hist[k] = rinf;
        if (rinf <= tol) { done = 1; break; }
        if (k >= maxit || rinf != rinf) break;
        oracle_jacobian(g, p, M, dt, bc, U, coef);
        if (oracle_block_solve(g->nx, g->ny, M, coef, R, dU, solver, lin_rtol)) break;
        double ss = 0.0;
        for (size_t i = 0; i < DOF; ++i) {
            U[i] += dU[i];
            ss += dU[i] * dU[i];
        }
        if (upd_hist) upd_hist[k] = sqrt(ss / (double)DOF);
        ++k;
    }
    free(R);
    free(dU);
    free(coef);
    return done ? k : -1;
}

/* ---------------------------------------------- sequential BDF1 (Sec. 2) */

/* Classic time marching: for n = 1..M, Newton on eq. 3 at level n alone from the
 * guess u^n = u^{n-1}, until the tau-scaled level residual is <= tol in max norm.
 * Writes all levels to U. iters (may be NULL, sized M) receives the Newton count
 * of every step. Returns 0, or n (1-based) of the first step that failed. */
int oracle_sequential_bdf1(const og_grid* g, const og_params* p, int M, double dt, const double* u0,
                           const double* bc, const double* q, double* U, double tol, int maxit, int solver,
                           double lin_rtol, int* iters) {
    size_t Ns = (size_t)g->nx * g->ny;
    int nb = 2 * g->nx + 2 * g->ny;
    double* r = (double*)malloc(sizeof(double) * Ns);
    double* du = (double*)malloc(sizeof(double) * Ns);
    double* cf = (double*)malloc(sizeof(double) * Ns * 5);
    int fail = 0;
    for (int n = 1; n <= M && !fail; ++n) {
        const double* u_prev = (n == 1) ? u0 : U + (size_t)(n - 2) * Ns;
        double* u = U + (size_t)(n - 1) * Ns;
        const double* bnd = bc ? bc + (size_t)(n - 1) * nb : NULL;
        const double* qn = q ? q + (size_t)(n - 1) * Ns : NULL;
        memcpy(u, u_prev, sizeof(double) * Ns);
        int k = 0;
        for (;;) {
            oracle_level_residual(g, p, dt, u_prev, u, bnd, qn, r);
            double rinf = max_abs(r, Ns);
            if (rinf <= tol) break;
            if (k >= maxit || rinf != rinf) { fail = n; break; }
            oracle_level_jacobian(g, p, dt, u, bnd, cf, cf + Ns, cf + 2 * Ns, cf + 3 * Ns, cf + 4 * Ns);
            if (oracle_level_solve(g->nx, g->ny, cf, Ns, r, du, solver, lin_rtol)) { fail = n; break; }
            for (size_t i = 0; i < Ns; ++i) u[i] += du[i];
            ++k;
        }
        if (iters) iters[n - 1] = k;
    }
    free(r);
    free(du);
    free(cf);
    return fail;
}
