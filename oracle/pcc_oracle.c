/*
 * pcc_oracle.c -- plain FP64 CPU oracle for all-pairs Pearson correlation.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  It shares no code,
 * header, table or helper with the CUDA library: it is the plain
 * definition of what that library computes, written out slowly and
 * obviously, in double precision, in k order, with no blocking, fusion or
 * reordering.
 *
 * What each function follows (LightPCC, Liu/Pan/Aluru, arXiv 1605.01584):
 *   oracle_pcc_pair      -- Eq. (1): r(u,v) = sum (u-ubar)(v-vbar) /
 *                           sqrt( sum (u-ubar)^2 * sum (v-vbar)^2 ).
 *   oracle_row_stats     -- the two per-variable quantities of Eq. (1) that
 *                           depend on one row only (Section III-A says they
 *                           can be computed once per variable).
 *   oracle_pcc_*         -- Eq. (1) per pair i<j; zero-variance rows give
 *                           0/0 = NaN (the paper is silent; NaN is the
 *                           value Eq. (1) itself produces).
 *   oracle_standardize   -- Eq. (5) with the square restored under the root
 *                           (Algorithm 3: mean, centred sum of squares,
 *                           scale by 1/sqrt).
 *   oracle_pair_index    -- Eq. (9)-(10) adapted to the strict upper
 *                           triangle (i<j), the adaptation Section III-B
 *                           allows: pairs numbered left to right, top to
 *                           bottom, row i holding n-1-i pairs.
 *   oracle_pair_coords   -- inverse of the numbering by searching the row
 *                           whose first index is <= J (the definition, not
 *                           the closed form of Eq. (14)-(15)).
 *   oracle_job_*_diag    -- Eq. (9)-(10) as printed (diagonal counted in),
 *                           the numbering the paper applies to tiles in
 *                           Eq. (16)-(19); inverse again by search.
 *   oracle_edges         -- pairs with |r| >= tau (co-expression network
 *                           edges, Section I).
 *   oracle_cross_*       -- non-symmetric all-pairs (Section III-B, the
 *                           job matrix of Eq. (7)-(8)) between the rows of
 *                           two matrices X (nx x l) and Y (ny x l): Eq. (1)
 *                           for every (x_i, y_j); jobs numbered row-major,
 *                           J = i*ny + j (Eq. (7)), inverse by search.
 *   oracle_perm_counts   -- permutation test (Section IV-A): for each of P
 *                           sample permutations pi_k, Eq. (1) on
 *                           (x_i, x_j o pi_k) with (x_j o pi_k)[s] =
 *                           x_j[pi_k[s]]; count k with |r_k| >= |r_obs|.
 *
 * Parity status: every function here is pinned by the "not gpu" tests
 * (closed forms, invariants, exact rational brute force, numpy.corrcoef,
 * exhaustive numbering round trips, complete permutation tests).
 *
 * Build: gcc -O2 -fopenmp -ffp-contract=off -shared -fPIC (no fast-math, no
 * FMA contraction, so results are the same on x86-64 and aarch64).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Eq. (1) building blocks                                             */
/* ------------------------------------------------------------------ */

/* mean and centred sum of squares of one l-vector (Eq. (1) denominator
 * terms; two passes, as Algorithm 3 does). */
static void row_mean_ssq(const double *x, int64_t l, double *mean, double *ssq)
{
    double s = 0.0;
    for (int64_t k = 0; k < l; ++k)
        s += x[k];
    double m = s / (double)l;
    double q = 0.0;
    for (int64_t k = 0; k < l; ++k) {
        double d = x[k] - m;
        q += d * d;
    }
    *mean = m;
    *ssq = q;
}

/* Eq. (1) numerator for u and v, with v read through an optional sample
 * permutation (perm == NULL means the identity). */
static double centred_dot(const double *u, double mu, const double *v,
                          double mv, const int32_t *perm, int64_t l)
{
    double s = 0.0;
    if (perm) {
        for (int64_t k = 0; k < l; ++k)
            s += (u[k] - mu) * (v[perm[k]] - mv);
    } else {
        for (int64_t k = 0; k < l; ++k)
            s += (u[k] - mu) * (v[k] - mv);
    }
    return s;
}

/* Eq. (1) from the numerator and the two centred sums of squares. */
static double eq1(double num, double ssq_u, double ssq_v)
{
    return num / sqrt(ssq_u * ssq_v);
}

/* Eq. (1) for two l-vectors, from scratch. */
double oracle_pcc_pair(const double *u, const double *v, int64_t l)
{
    double mu, su, mv, sv;
    row_mean_ssq(u, l, &mu, &su);
    row_mean_ssq(v, l, &mv, &sv);
    return eq1(centred_dot(u, mu, v, mv, NULL, l), su, sv);
}

void oracle_row_stats(const double *X, int64_t n, int64_t l, int64_t ldx,
                      double *mean, double *ssq)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i)
        row_mean_ssq(X + i * ldx, l, &mean[i], &ssq[i]);
}

/* ------------------------------------------------------------------ */
/* Strict-upper pair numbering (Eq. (9)-(10), diagonal excluded)       */
/* ------------------------------------------------------------------ */

/* number of pairs before row i: (n-1) + (n-2) + ... + (n-i) */
static int64_t pairs_before_row(int64_t n, int64_t i)
{
    return i * (2 * n - i - 1) / 2;
}

int64_t oracle_num_pairs(int64_t n)
{
    return n < 2 ? 0 : n * (n - 1) / 2;
}

/* -1 when (i,j) is not a strict-upper pair of an n-variable problem */
int64_t oracle_pair_index(int64_t n, int64_t i, int64_t j)
{
    if (i < 0 || j <= i || j >= n)
        return -1;
    return pairs_before_row(n, i) + (j - i - 1);
}

/* row i is the largest i with pairs_before_row(i) <= J (binary search) */
int oracle_pair_coords(int64_t n, int64_t J, int64_t *i, int64_t *j)
{
    if (n < 2 || J < 0 || J >= oracle_num_pairs(n))
        return -1;
    int64_t lo = 0, hi = n - 2; /* answer in [lo, hi] */
    while (lo < hi) {
        int64_t mid = lo + (hi - lo + 1) / 2;
        if (pairs_before_row(n, mid) <= J)
            lo = mid;
        else
            hi = mid - 1;
    }
    *i = lo;
    *j = J - pairs_before_row(n, lo) + lo + 1;
    return 0;
}

/* Eq. (9)-(10) as printed, major diagonal counted in (used for tile
 * numbering): J_n(y,x) = F_n(y) + x - y, F_n(y) = y(2n-y+1)/2, y <= x. */
static int64_t cells_before_row_diag(int64_t n, int64_t y)
{
    return y * (2 * n - y + 1) / 2;
}

int64_t oracle_job_index_diag(int64_t n, int64_t y, int64_t x)
{
    if (y < 0 || x < y || x >= n)
        return -1;
    return cells_before_row_diag(n, y) + x - y;
}

/* inverse by search: y is the largest row with F_n(y) <= J */
int oracle_job_coords_diag(int64_t n, int64_t J, int64_t *y, int64_t *x)
{
    if (n < 1 || J < 0 || J >= n * (n + 1) / 2)
        return -1;
    int64_t lo = 0, hi = n - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo + 1) / 2;
        if (cells_before_row_diag(n, mid) <= J)
            lo = mid;
        else
            hi = mid - 1;
    }
    *y = lo;
    *x = J - cells_before_row_diag(n, lo) + lo;
    return 0;
}

/* ------------------------------------------------------------------ */
/* All-pairs outputs                                                   */
/* ------------------------------------------------------------------ */

/* r for a list of pairs (I[p], Jc[p]); any order, i == j allowed */
void oracle_pcc_pairs(const double *X, int64_t n, int64_t l, int64_t ldx,
                      int64_t npairs, const int64_t *I, const int64_t *Jc,
                      double *r)
{
    double *mean = (double *)malloc(sizeof(double) * (size_t)n);
    double *ssq = (double *)malloc(sizeof(double) * (size_t)n);
    oracle_row_stats(X, n, l, ldx, mean, ssq);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t p = 0; p < npairs; ++p) {
        int64_t i = I[p], j = Jc[p];
        double num = centred_dot(X + i * ldx, mean[i], X + j * ldx, mean[j],
                                 NULL, l);
        r[p] = eq1(num, ssq[i], ssq[j]);
    }
    free(mean);
    free(ssq);
}

/* packed strict-upper r for rows [i0, i1): out[pair_index(i,j) - first]
 * where first = pair_index(i0, i0+1); i1 == n gives the whole triangle
 * when i0 == 0. */
void oracle_pcc_rows(const double *X, int64_t n, int64_t l, int64_t ldx,
                     int64_t i0, int64_t i1, double *out)
{
    double *mean = (double *)malloc(sizeof(double) * (size_t)n);
    double *ssq = (double *)malloc(sizeof(double) * (size_t)n);
    oracle_row_stats(X, n, l, ldx, mean, ssq);
    int64_t first = pairs_before_row(n, i0);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = i0; i < i1; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double num = centred_dot(X + i * ldx, mean[i], X + j * ldx,
                                     mean[j], NULL, l);
            out[oracle_pair_index(n, i, j) - first] = eq1(num, ssq[i], ssq[j]);
        }
    }
    free(mean);
    free(ssq);
}

/* Eq. (5)/Algorithm 3: Z[i] = (X_i - mean_i) / sqrt(sum (X_i - mean_i)^2);
 * flag[i] = 1 when that sum is zero or not finite (Z row set to 0). */
void oracle_standardize(const double *X, int64_t n, int64_t l, int64_t ldx,
                        double *Z, int64_t ldz, uint8_t *flag)
{
#pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < n; ++i) {
        double m, q;
        row_mean_ssq(X + i * ldx, l, &m, &q);
        int bad = !(q > 0.0) || !isfinite(q);
        flag[i] = (uint8_t)bad;
        for (int64_t k = 0; k < l; ++k)
            Z[i * ldz + k] = bad ? 0.0 : (X[i * ldx + k] - m) / sqrt(q);
    }
}

/* pairs with |r| >= tau among rows i in [i0, i1), all j > i.  Returns the
 * total count; stores at most cap of them (in row-major pair order). */
int64_t oracle_edges(const double *X, int64_t n, int64_t l, int64_t ldx,
                     double tau, int64_t i0, int64_t i1, int64_t cap,
                     int64_t *ei, int64_t *ej, double *er)
{
    double *mean = (double *)malloc(sizeof(double) * (size_t)n);
    double *ssq = (double *)malloc(sizeof(double) * (size_t)n);
    oracle_row_stats(X, n, l, ldx, mean, ssq);
    int64_t count = 0;
    /* rows in parallel, each appending to a private list, merged in order */
    int64_t nrows = i1 > i0 ? i1 - i0 : 0;
    int64_t *rowcnt = (int64_t *)calloc((size_t)nrows + 1, sizeof(int64_t));
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = i0; i < i1; ++i) {
        int64_t c = 0;
        for (int64_t j = i + 1; j < n; ++j) {
            double num = centred_dot(X + i * ldx, mean[i], X + j * ldx,
                                     mean[j], NULL, l);
            double r = eq1(num, ssq[i], ssq[j]);
            if (fabs(r) >= tau) /* NaN compares false: never an edge */
                ++c;
        }
        rowcnt[i - i0] = c;
    }
    int64_t *start = (int64_t *)malloc(sizeof(int64_t) * ((size_t)nrows + 1));
    for (int64_t r = 0; r < nrows; ++r) {
        start[r] = count;
        count += rowcnt[r];
    }
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = i0; i < i1; ++i) {
        int64_t pos = start[i - i0];
        if (rowcnt[i - i0] == 0 || pos >= cap)
            continue;
        for (int64_t j = i + 1; j < n; ++j) {
            double num = centred_dot(X + i * ldx, mean[i], X + j * ldx,
                                     mean[j], NULL, l);
            double r = eq1(num, ssq[i], ssq[j]);
            if (fabs(r) >= tau) {
                if (pos < cap) {
                    ei[pos] = i;
                    ej[pos] = j;
                    er[pos] = r;
                }
                ++pos;
            }
        }
    }
    free(start);
    free(rowcnt);
    free(mean);
    free(ssq);
    return count;
}

/* Permutation exceedance counts for a list of pairs.
 *   r_obs = Eq. (1)(x_i, x_j);  r_k = Eq. (1)(x_i, x_j o pi_k)
 *   cnt[p]    = #{k : |r_k| >= |r_obs|}
 *   cnt_lo[p] = #{k : |r_k| >= |r_obs| + delta}   (may be NULL)
 *   cnt_hi[p] = #{k : |r_k| >= |r_obs| - delta}   (may be NULL)
 * perms is P x l (row k = pi_k).  The mean and centred sum of squares of a
 * vector do not change under a permutation of its samples, so the cached
 * row statistics serve every k. */
void oracle_perm_counts(const double *X, int64_t n, int64_t l, int64_t ldx,
                        int64_t P, const int32_t *perms, int64_t npairs,
                        const int64_t *I, const int64_t *Jc, double delta,
                        uint32_t *cnt, uint32_t *cnt_lo, uint32_t *cnt_hi)
{
    double *mean = (double *)malloc(sizeof(double) * (size_t)n);
    double *ssq = (double *)malloc(sizeof(double) * (size_t)n);
    oracle_row_stats(X, n, l, ldx, mean, ssq);
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t p = 0; p < npairs; ++p) {
        int64_t i = I[p], j = Jc[p];
        const double *u = X + i * ldx, *v = X + j * ldx;
        double robs = fabs(eq1(centred_dot(u, mean[i], v, mean[j], NULL, l),
                               ssq[i], ssq[j]));
        uint32_t c = 0, clo = 0, chi = 0;
        for (int64_t k = 0; k < P; ++k) {
            double rk = fabs(eq1(centred_dot(u, mean[i], v, mean[j],
                                             perms + k * l, l),
                                 ssq[i], ssq[j]));
            c += (rk >= robs);
            clo += (rk >= robs + delta);
            chi += (rk >= robs - delta);
        }
        cnt[p] = c;
        if (cnt_lo)
            cnt_lo[p] = clo;
        if (cnt_hi)
            cnt_hi[p] = chi;
    }
    free(mean);
    free(ssq);
}

/* ------------------------------------------------------------------ */
/* Non-symmetric all-pairs between two matrices (Eq. (7)-(8))          */
/* ------------------------------------------------------------------ */

/* Eq. (7) on an nrow x ncol job matrix: J = y*ncol + x; -1 outside it */
int64_t oracle_cross_job_index(int64_t nrow, int64_t ncol, int64_t y,
                               int64_t x)
{
    if (y < 0 || y >= nrow || x < 0 || x >= ncol)
        return -1;
    return y * ncol + x;
}

/* inverse of Eq. (7) by search: y is the largest row with y*ncol <= J */
int oracle_cross_job_coords(int64_t nrow, int64_t ncol, int64_t J, int64_t *y,
                            int64_t *x)
{
    if (nrow < 1 || ncol < 1 || J < 0 || J >= nrow * ncol)
        return -1;
    int64_t lo = 0, hi = nrow - 1;
    while (lo < hi) {
        int64_t mid = lo + (hi - lo + 1) / 2;
        if (mid * ncol <= J)
            lo = mid;
        else
            hi = mid - 1;
    }
    *y = lo;
    *x = J - lo * ncol;
    return 0;
}

/* Eq. (1) for every (x_i, y_j), i in [i0, i1), 0 <= j < ny:
 * out[(i - i0) * ny + j] (row-major job order of Eq. (7)). */
void oracle_cross_rows(const double *X, int64_t nx, int64_t ldx,
                       const double *Y, int64_t ny, int64_t ldy, int64_t l,
                       int64_t i0, int64_t i1, double *out)
{
    double *mx = (double *)malloc(sizeof(double) * (size_t)nx);
    double *sx = (double *)malloc(sizeof(double) * (size_t)nx);
    double *my = (double *)malloc(sizeof(double) * (size_t)ny);
    double *sy = (double *)malloc(sizeof(double) * (size_t)ny);
    oracle_row_stats(X, nx, l, ldx, mx, sx);
    oracle_row_stats(Y, ny, l, ldy, my, sy);
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t i = i0; i < i1; ++i) {
        for (int64_t j = 0; j < ny; ++j) {
            double num = centred_dot(X + i * ldx, mx[i], Y + j * ldy, my[j],
                                     NULL, l);
            out[oracle_cross_job_index(nx, ny, i, j) - i0 * ny] =
                eq1(num, sx[i], sy[j]);
        }
    }
    free(mx);
    free(sx);
    free(my);
    free(sy);
}

/* Eq. (1) for a list of (x_{I[p]}, y_{Jc[p]}) */
void oracle_cross_pairs(const double *X, int64_t nx, int64_t ldx,
                        const double *Y, int64_t ny, int64_t ldy, int64_t l,
                        int64_t npairs, const int64_t *I, const int64_t *Jc,
                        double *r)
{
    double *mx = (double *)malloc(sizeof(double) * (size_t)nx);
    double *sx = (double *)malloc(sizeof(double) * (size_t)nx);
    double *my = (double *)malloc(sizeof(double) * (size_t)ny);
    double *sy = (double *)malloc(sizeof(double) * (size_t)ny);
    oracle_row_stats(X, nx, l, ldx, mx, sx);
    oracle_row_stats(Y, ny, l, ldy, my, sy);
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t p = 0; p < npairs; ++p) {
        int64_t i = I[p], j = Jc[p];
        double num = centred_dot(X + i * ldx, mx[i], Y + j * ldy, my[j],
                                 NULL, l);
        r[p] = eq1(num, sx[i], sy[j]);
    }
    free(mx);
    free(sx);
    free(my);
    free(sy);
}

int oracle_num_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
