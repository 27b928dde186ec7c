/*
 * psa_oracle.c -- CPU reference for sigma_min(zI - A), A banded.
 *
 * TEST INFRASTRUCTURE. Only the tests, the smoke check and the CPU-baseline
 * leg of the benchmark load this file's library. It shares no code, header,
 * table or helper with the CUDA library; it is plain, slow and written to be
 * read against the mathematics.
 *
 * What it computes. For each complex point z, sigma_min(zI - A), the smallest
 * singular value of zI - A (paper Sec. 2, Definition "Pseudospectrum", third
 * characterisation; Sec. 2.1, sigma_min(z) = sigma_n of the SVD of zI - A).
 * The paper evaluates it with a dense SVD; this file follows the banded
 * reading of the same quantity:
 *
 *   sigma_min(B)^2 = 1 / lambda_max(H),  H = (B B^*)^{-1},  B = zI - A,
 *
 * with lambda_max(H) found by the Lanczos process on H and every product
 * H q = B^{-*} (B^{-1} q) formed from a banded LU factorisation of B:
 *
 *   1. B = P L U by Gaussian elimination with partial pivoting inside the
 *      band: in column j the pivot is the row of largest |Re| + |Im| among
 *      rows j .. j+kl (the first such row on ties); U gets kl + ku
 *      superdiagonals (fill-in).
 *   2. B x = q: forward elimination with the row interchanges and the
 *      multipliers, then back substitution with U.
 *      B^* y = x: forward substitution with U^*, then the transposed
 *      eliminations in reverse order, each followed by its interchange.
 *   3. Lanczos three-term recurrence on the scaled operator H / 2^(2 e1),
 *      where 2^e1 is the binary exponent of |B^{-1} q_1|, so that the
 *      tridiagonal stays of moderate size when sigma_min is tiny. The start
 *      vector q_1 comes from the SplitMix64 generator (Steele, Lea and Flood,
 *      "Fast splittable pseudorandom number generators", OOPSLA 2014).
 *   4. theta_j = largest eigenvalue of the j x j Lanczos tridiagonal T_j by
 *      Sturm-count bisection; the last component s_j of its unit eigenvector
 *      by inverse iteration on T_j - theta_j I (the residual of the Ritz pair
 *      is |beta_j s_j|; Parlett, The Symmetric Eigenvalue Problem, Ch. 13).
 *   5. Stop after step j >= k_min when beta_j = 0, when the residual
 *      estimate beta_j |s_j| <= tol * theta_j, or when the Ritz value stopped
 *      moving, theta_j - theta_{j-1} <= tol * theta_j; or at j = k_max
 *      (status NOT_CONVERGED). sigma = 2^(-e1) / sqrt(theta_j).
 *
 * Per-point status: 0 OK, 1 SINGULAR (an exact zero pivot column: sigma = 0),
 * 2 NOT_CONVERGED (k_max reached), 3 NONFINITE (a band entry of A is not
 * finite: sigma = 0), 5 UNDERFLOW (a value overflowed the double range during
 * the solves although A and z are finite, i.e. |(zI - A)^{-1}| > ~1e308 and
 * sigma_min is below the double range: sigma = 0).
 *
 * Build: gcc -O2 -std=c11 -ffp-contract=off -fopenmp -fPIC -shared.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

enum { OR_OK = 0, OR_SINGULAR = 1, OR_NOT_CONVERGED = 2, OR_NONFINITE = 3, OR_UNDERFLOW = 5 };

static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }

/* |Re a| + |Im a|: the pivot size used by the elimination. */
static double cabs1(cplx a) { return fabs(creal(a)) + fabs(cimag(a)); }

/* Euclidean norm of a complex vector, scaled by its largest component so that
 * the squares neither overflow nor underflow (|v| up to the largest double). */
static double norm2_plain(int n, const cplx *v)
{
    double m = 0.0;
    for (int i = 0; i < n; i++) m = fmax(m, fmax(fabs(creal(v[i])), fabs(cimag(v[i]))));
    if (m == 0.0 || !isfinite(m)) return m;
    double s = 0.0;
    for (int i = 0; i < n; i++) {
        double re = creal(v[i]) / m, im = cimag(v[i]) / m;
        s += re * re + im * im;
    }
    return m * sqrt(s);
}

/* ------------------------------------------------------------------ grid */

/* Grid abscissae (paper Sec. 2.1): x_j = re_min + j * h, h = (re_max - re_min)/(nx - 1),
 * evaluated as one fused multiply-add; nx == 1 gives the single abscissa re_min. */
double oracle_grid_coord(double lo, double hi, int32_t count, int32_t j)
{
    double h = count > 1 ? (hi - lo) / (double)(count - 1) : 0.0;
    return fma((double)j, h, lo);
}

void oracle_grid_points(double re_min, double re_max, double im_min, double im_max,
                        int32_t nx, int32_t ny, double *z /* 2*nx*ny, (re,im) pairs */)
{
    for (int32_t i = 0; i < ny; i++) {
        double y = oracle_grid_coord(im_min, im_max, ny, i);
        for (int32_t j = 0; j < nx; j++) {
            double x = oracle_grid_coord(re_min, re_max, nx, j);
            z[2 * ((int64_t)i * nx + j)] = x;
            z[2 * ((int64_t)i * nx + j) + 1] = y;
        }
    }
}

/* ------------------------------------------------------- start vector */

/* SplitMix64 output number c (c = 0, 1, ...) for the given seed: the state
 * after c + 1 increments by the golden gamma, passed through the mixer. */
uint64_t oracle_splitmix64(uint64_t seed, uint64_t c)
{
    uint64_t z = seed + (c + 1) * 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* Map a 64-bit word to [-1, 1): top 53 bits times 2^-52, minus one (exact). */
static double unit_interval(uint64_t v) { return (double)(v >> 11) * 0x1.0p-52 - 1.0; }

/* Lanczos start vector: h_i = u(2i) + i u(2i+1), q_1 = h / |h|_2. */
void oracle_start_vector(int32_t n, uint64_t seed, double *q /* 2n */)
{
    double s = 0.0;
    for (int32_t i = 0; i < n; i++) {
        double re = unit_interval(oracle_splitmix64(seed, 2 * (uint64_t)i));
        double im = unit_interval(oracle_splitmix64(seed, 2 * (uint64_t)i + 1));
        q[2 * i] = re;
        q[2 * i + 1] = im;
        s += re * re + im * im;
    }
    s = sqrt(s);
    for (int32_t i = 0; i < 2 * n; i++) q[i] /= s;
}

/* --------------------------------------------------------- banded LU */

/* Working storage: row i keeps columns i-kl .. i+ku+kl (width w = 2kl+ku+1). */
typedef struct {
    int n, kl, ku, w;
    cplx *a;
    int *piv;
} band_lu;

static cplx *at(const band_lu *F, int i, int j) { return &F->a[(size_t)i * F->w + (j - i + F->kl)]; }

/* B = zI - A from band storage bands[(d+kl)*n + i] = A[i][i+d]. */
static void lu_load(band_lu *F, const cplx *bands, cplx z)
{
    memset(F->a, 0, sizeof(cplx) * (size_t)F->n * F->w);
    for (int i = 0; i < F->n; i++)
        for (int d = -F->kl; d <= F->ku; d++) {
            int j = i + d;
            if (j < 0 || j >= F->n) continue;
            *at(F, i, j) = -bands[(size_t)(d + F->kl) * F->n + i];
        }
    for (int i = 0; i < F->n; i++) *at(F, i, i) += z;
}

/* Gaussian elimination with partial pivoting inside the band.
 * Returns 0, or j+1 when column j has no nonzero pivot candidate. */
static int lu_factor(band_lu *F)
{
    const int n = F->n, kl = F->kl, ku = F->ku;
    for (int j = 0; j < n; j++) {
        int last = imin(n - 1, j + kl);
        int p = j;
        double best = cabs1(*at(F, j, j));
        for (int i = j + 1; i <= last; i++) {
            double v = cabs1(*at(F, i, j));
            if (v > best) { best = v; p = i; }
        }
        F->piv[j] = p;
        if (best == 0.0) return j + 1;
        int cend = imin(n - 1, j + kl + ku);
        if (p != j)
            for (int c = j; c <= cend; c++) {
                cplx t = *at(F, j, c);
                *at(F, j, c) = *at(F, p, c);
                *at(F, p, c) = t;
            }
        for (int i = j + 1; i <= last; i++) {
            cplx l = *at(F, i, j) / *at(F, j, j);
            *at(F, i, j) = l;
            for (int c = j + 1; c <= cend; c++) *at(F, i, c) -= l * *at(F, j, c);
        }
    }
    return 0;
}

/* U(i, c) for c >= i and the multiplier L(i, j) for j < i <= j + kl. */
static cplx U(const band_lu *F, int i, int c) { return *at(F, i, c); }
static cplx L(const band_lu *F, int i, int j) { return *at(F, i, j); }

/* Solve B x = b (b overwritten by x). */
static void solve_B(const band_lu *F, cplx *b)
{
    const int n = F->n, kl = F->kl, ku = F->ku;
    for (int j = 0; j < n; j++) {
        int p = F->piv[j];
        if (p != j) { cplx t = b[j]; b[j] = b[p]; b[p] = t; }
        for (int i = j + 1; i <= imin(n - 1, j + kl); i++) b[i] -= L(F, i, j) * b[j];
    }
    for (int j = n - 1; j >= 0; j--) {
        cplx s = b[j];
        for (int c = j + 1; c <= imin(n - 1, j + kl + ku); c++) s -= U(F, j, c) * b[c];
        b[j] = s / U(F, j, j);
    }
}

/* Solve B^* y = b (b overwritten by y). */
static void solve_BH(const band_lu *F, cplx *b)
{
    const int n = F->n, kl = F->kl, ku = F->ku;
    for (int i = 0; i < n; i++) {
        cplx s = b[i];
        for (int r = imax(0, i - kl - ku); r < i; r++) s -= conj(U(F, r, i)) * b[r];
        b[i] = s / conj(U(F, i, i));
    }
    for (int j = n - 1; j >= 0; j--) {
        for (int i = j + 1; i <= imin(n - 1, j + kl); i++) b[j] -= conj(L(F, i, j)) * b[i];
        int p = F->piv[j];
        if (p != j) { cplx t = b[j]; b[j] = b[p]; b[p] = t; }
    }
}

/* ------------------------------------------------ tridiagonal top pair */

/* Number of eigenvalues of T (diag a[0..m-1], off-diag b[0..m-2]) below x,
 * from the signs of the pivots of T - xI = L D L^T. */
static int sturm_below(int m, const double *a, const double *b, double x)
{
    int count = 0;
    double d = 1.0;
    for (int i = 0; i < m; i++) {
        double off = i > 0 ? b[i - 1] * b[i - 1] / d : 0.0;
        d = a[i] - x - off;
        if (d == 0.0) d = -0x1.0p-1000;
        if (d < 0.0) count++;
    }
    return count;
}

/* Largest eigenvalue theta of T_m (Sturm bisection to full precision) and the
 * modulus of the last component of its unit eigenvector, by three steps of
 * inverse iteration on T_m - theta I solved with the banded LU above
 * (kl = ku = 1, partial pivoting). */
void oracle_tridiag_top(int32_t m, const double *a, const double *b, double *theta, double *s_last)
{
    if (m == 1) { *theta = a[0]; *s_last = 1.0; return; }
    double lo = a[0], hi = -INFINITY;
    for (int i = 0; i < m; i++) {
        double r = fabs(i > 0 ? b[i - 1] : 0.0) + fabs(i < m - 1 ? b[i] : 0.0);
        if (a[i] > lo) lo = a[i];
        if (a[i] + r > hi) hi = a[i] + r;
    }
    for (int it = 0; it < 2200 && hi - lo > 0x1.0p-52 * fmax(fabs(lo), fabs(hi)); it++) {
        double mid = lo + 0.5 * (hi - lo);
        if (mid <= lo || mid >= hi) break;
        if (sturm_below(m, a, b, mid) < m) lo = mid; else hi = mid;
    }
    *theta = hi;

    /* T - x I in band storage (kl = ku = 1): bands[0] = sub, [1] = diag, [2] = super */
    cplx *tb = malloc(sizeof(cplx) * 3 * (size_t)m);
    cplx *v = malloc(sizeof(cplx) * (size_t)m);
    band_lu F = { m, 1, 1, 4, malloc(sizeof(cplx) * 4 * (size_t)m), malloc(sizeof(int) * (size_t)m) };
    for (int i = 0; i < m; i++) {
        tb[i] = i > 0 ? b[i - 1] : 0.0;
        tb[m + i] = a[i];
        tb[2 * m + i] = i < m - 1 ? b[i] : 0.0;
    }
    double x = hi;
    int singular = 1;
    for (int tries = 0; tries < 8 && singular; tries++) {
        lu_load(&F, tb, x);                    /* x I - T */
        singular = lu_factor(&F) != 0;
        if (singular) x = x + fmax(fabs(x), 1e-300) * 0x1.0p-50 * (double)(1 << tries);
    }
    if (singular) {
        *s_last = 0.0;
    } else {
        for (int i = 0; i < m; i++) v[i] = 1.0;
        for (int it = 0; it < 3; it++) {
            solve_B(&F, v);
            double nv = norm2_plain(m, v);
            for (int i = 0; i < m; i++) v[i] /= nv;
        }
        *s_last = cabs(v[m - 1]);
    }
    free(tb); free(v); free(F.a); free(F.piv);
}

/* ------------------------------------------------------------- Lanczos */

typedef struct {
    band_lu F;
    cplx *q, *qprev, *x, *w;
    double *alpha, *beta;
} point_work;

static int work_alloc(point_work *W, int n, int kl, int ku, int k_max)
{
    W->F.n = n; W->F.kl = kl; W->F.ku = ku; W->F.w = 2 * kl + ku + 1;
    W->F.a = malloc(sizeof(cplx) * (size_t)n * W->F.w);
    W->F.piv = malloc(sizeof(int) * (size_t)n);
    W->q = malloc(sizeof(cplx) * (size_t)n);
    W->qprev = malloc(sizeof(cplx) * (size_t)n);
    W->x = malloc(sizeof(cplx) * (size_t)n);
    W->w = malloc(sizeof(cplx) * (size_t)n);
    W->alpha = malloc(sizeof(double) * (size_t)k_max);
    W->beta = malloc(sizeof(double) * (size_t)k_max);
    return W->F.a && W->F.piv && W->q && W->qprev && W->x && W->w && W->alpha && W->beta;
}

static void work_free(point_work *W)
{
    free(W->F.a); free(W->F.piv); free(W->q); free(W->qprev); free(W->x); free(W->w);
    free(W->alpha); free(W->beta);
}

/* sigma_min(zI - A) at one point; returns the status, writes sigma and steps. */
static int sigma_point(point_work *W, const cplx *bands, cplx z, const double *q1,
                       int k_min, int k_max, double tol, double *sigma, int *steps)
{
    const int n = W->F.n, kl = W->F.kl, ku = W->F.ku;
    *steps = 0;
    for (int d = -kl; d <= ku; d++)
        for (int i = 0; i < n; i++)
            if (i + d >= 0 && i + d < n && !isfinite(cabs(bands[(size_t)(d + kl) * n + i]))) {
                *sigma = 0.0;
                return OR_NONFINITE;
            }
    lu_load(&W->F, bands, z);
    if (lu_factor(&W->F) != 0) { *sigma = 0.0; return OR_SINGULAR; }

    for (int i = 0; i < n; i++) { W->q[i] = CMPLX(q1[2 * i], q1[2 * i + 1]); W->qprev[i] = 0.0; }
    double beta_prev = 0.0, theta = 0.0, theta_prev = 0.0;
    int e1 = 0;
    for (int j = 1; j <= k_max; j++) {
        memcpy(W->x, W->q, sizeof(cplx) * (size_t)n);
        solve_B(&W->F, W->x);                       /* x = B^{-1} q   */
        double s = norm2_plain(n, W->x);
        if (!isfinite(s) || s == 0.0) { *steps = j; *sigma = 0.0; return OR_UNDERFLOW; }
        if (j == 1) (void)frexp(s, &e1);
        for (int i = 0; i < n; i++) W->x[i] /= s;
        solve_BH(&W->F, W->x);                      /* y = B^{-*} x/|x| ; H q = s y */
        double f = ldexp(s, -2 * e1);               /* scaled operator H / 2^(2 e1) */
        for (int i = 0; i < n; i++) W->w[i] = f * W->x[i] - beta_prev * W->qprev[i];
        double alpha = 0.0;
        for (int i = 0; i < n; i++) alpha += creal(conj(W->q[i]) * W->w[i]);
        for (int i = 0; i < n; i++) W->w[i] -= alpha * W->q[i];
        double beta = norm2_plain(n, W->w);
        W->alpha[j - 1] = alpha;
        W->beta[j - 1] = beta;
        double s_last;
        theta_prev = theta;
        oracle_tridiag_top(j, W->alpha, W->beta, &theta, &s_last);
        *steps = j;
        if (!isfinite(theta) || !isfinite(beta) || !(theta > 0.0)) { *sigma = 0.0; return OR_UNDERFLOW; }
        int done = 0;
        if (j >= k_min) {
            if (beta == 0.0) done = 1;
            else if (beta * fabs(s_last) <= tol * theta) done = 1;
            else if (j >= 2 && theta - theta_prev <= tol * theta) done = 1;
        } else if (beta == 0.0) {
            done = 1;
        }
        if (done || j == k_max) {
            *sigma = ldexp(1.0 / sqrt(theta), -e1);
            return done ? OR_OK : OR_NOT_CONVERGED;
        }
        for (int i = 0; i < n; i++) { W->qprev[i] = W->q[i]; W->q[i] = W->w[i] / beta; }
        beta_prev = beta;
    }
    return OR_NOT_CONVERGED; /* not reached: k_max >= 1 */
}

/* sigma_min(z_p I - A) for npts points z (pairs re, im). nthreads <= 0: OpenMP default.
 * Returns 0, or -1 on bad arguments / allocation failure. */
int oracle_sigma_min_points(int32_t n, int32_t kl, int32_t ku, const double *bands_ri,
                            int64_t npts, const double *z_ri,
                            int32_t k_min, int32_t k_max, double tol, uint64_t seed,
                            double *sigma, int8_t *status, int32_t *steps, int32_t nthreads)
{
    if (n < 1 || kl < 0 || ku < 0 || k_max < 1 || k_min < 0)
        return -1;
    const cplx *bands = (const cplx *)bands_ri;
    double *q1 = malloc(sizeof(double) * 2 * (size_t)n);
    if (!q1) return -1;
    oracle_start_vector(n, seed, q1);
    int failed = 0;
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
#pragma omp parallel
    {
        point_work W;
        int ok = work_alloc(&W, n, kl, ku, k_max);
        if (!ok) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t p = 0; p < npts; p++) {
            if (!ok) continue;
            int st, k;
            cplx z = CMPLX(z_ri[2 * p], z_ri[2 * p + 1]);
            st = sigma_point(&W, bands, z, q1, k_min, k_max, tol, &sigma[p], &k);
            status[p] = (int8_t)st;
            if (steps) steps[p] = k;
        }
        work_free(&W);
    }
    free(q1);
    return failed ? -1 : 0;
}

/* ------------------------------------------- step-level entry points
 * (for the checks that pin each step on its own) */

/* Factor B = zI - A. factor: n*(2kl+ku+1) complex (row i: columns i-kl..i+ku+kl),
 * piv: n ints (absolute pivot row of column j). Returns 0 or (singular column + 1). */
int oracle_band_lu(int32_t n, int32_t kl, int32_t ku, const double *bands_ri, double zr, double zi,
                   double *factor_ri, int32_t *piv)
{
    band_lu F = { n, kl, ku, 2 * kl + ku + 1, (cplx *)factor_ri, malloc(sizeof(int) * (size_t)n) };
    lu_load(&F, (const cplx *)bands_ri, CMPLX(zr, zi));
    int r = lu_factor(&F);
    for (int i = 0; i < n; i++) piv[i] = F.piv[i];
    free(F.piv);
    return r;
}

/* Solve B x = b (adjoint = 0) or B^* x = b (adjoint = 1) with a factor from oracle_band_lu. */
void oracle_band_solve(int32_t n, int32_t kl, int32_t ku, const double *factor_ri, const int32_t *piv,
                       int32_t adjoint, double *b_ri)
{
    band_lu F = { n, kl, ku, 2 * kl + ku + 1, (cplx *)factor_ri, malloc(sizeof(int) * (size_t)n) };
    for (int i = 0; i < n; i++) F.piv[i] = piv[i];
    if (adjoint) solve_BH(&F, (cplx *)b_ri); else solve_B(&F, (cplx *)b_ri);
    free(F.piv);
}

/* Lanczos coefficients alpha_1..alpha_k, beta_1..beta_k (no stopping test)
 * of H / 2^(2 e1) at one point, for the checks on the recurrence itself.
 * Returns the number of steps done (< k on breakdown or a singular pivot). */
int32_t oracle_lanczos_coeffs(int32_t n, int32_t kl, int32_t ku, const double *bands_ri,
                              double zr, double zi, int32_t k, uint64_t seed,
                              double *alpha, double *beta, int32_t *e1_out)
{
    point_work W;
    if (!work_alloc(&W, n, kl, ku, k)) return -1;
    double *q1 = malloc(sizeof(double) * 2 * (size_t)n);
    oracle_start_vector(n, seed, q1);
    lu_load(&W.F, (const cplx *)bands_ri, CMPLX(zr, zi));
    int done = 0;
    if (lu_factor(&W.F) == 0) {
        for (int i = 0; i < n; i++) { W.q[i] = CMPLX(q1[2 * i], q1[2 * i + 1]); W.qprev[i] = 0.0; }
        double beta_prev = 0.0;
        int e1 = 0;
        for (int j = 1; j <= k; j++) {
            memcpy(W.x, W.q, sizeof(cplx) * (size_t)n);
            solve_B(&W.F, W.x);
            double s = norm2_plain(n, W.x);
            if (j == 1) (void)frexp(s, &e1);
            for (int i = 0; i < n; i++) W.x[i] /= s;
            solve_BH(&W.F, W.x);
            double f = ldexp(s, -2 * e1);
            for (int i = 0; i < n; i++) W.w[i] = f * W.x[i] - beta_prev * W.qprev[i];
            double a = 0.0;
            for (int i = 0; i < n; i++) a += creal(conj(W.q[i]) * W.w[i]);
            for (int i = 0; i < n; i++) W.w[i] -= a * W.q[i];
            double b = norm2_plain(n, W.w);
            alpha[j - 1] = a; beta[j - 1] = b;
            done = j;
            if (b == 0.0) break;
            for (int i = 0; i < n; i++) { W.qprev[i] = W.q[i]; W.q[i] = W.w[i] / b; }
            beta_prev = b;
        }
        *e1_out = e1;
    }
    free(q1);
    work_free(&W);
    return done;
}
