/*
 * mlt_oracle.c -- plain CPU oracle for the multilevel Chebyshev-Hutchinson
 * trace estimator of Hallman & Troester (arXiv 2103.10516).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously correct CPU
 * restatement of the method that the CUDA path is checked against.  Only the
 * test suite, the package smoke check and the benchmark's CPU-baseline arm may
 * load it.  It shares no source with the CUDA library.
 *
 * Everything is straight loops in the order the paper states them:
 *   - Rademacher probes (Section 2.1): entries +-1 with equal probability, drawn
 *     from a counter-based generator (SplitMix64 finaliser, Steele/Lea/Flood 2014,
 *     the "mix64variant13" constants), keyed by (seed, probe id, row).
 *   - Chebyshev moments mu_j = z^T T_j(At) z by the three-term recurrence
 *     T_{j+1} = 2x T_j - T_{j-1} (Section 2.2, Eq. recurrence), with the affine
 *     map At = alpha*A + beta*I sending [a, b] to [-1, 1].  No doubling trick: the
 *     oracle evaluates every moment directly as z . w_j.
 *   - Triangle moments (Section 2.1 Example, Section 5.4): x1 = z^T A z,
 *     x2 = z^T A^2 z, x3 = z^T A^3 z in exact 64-bit integers, and a brute-force
 *     triangle count.
 * Dot products are accumulated in long double in row order.
 */
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---- Rademacher probes (Section 2.1) ------------------------------------ */

/* SplitMix64 output finaliser (Steele, Lea, Flood, "Fast splittable
 * pseudorandom number generators", OOPSLA 2014; variant-13 constants). */
uint64_t orc_mix64(uint64_t x)
{
    x = (x ^ (x >> 30)) * 0xbf58476d1ce4e5b9ULL;
    x = (x ^ (x >> 27)) * 0x94d049bb133111ebULL;
    return x ^ (x >> 31);
}

/* Probe entry z_i of probe p: one hash serves the 64 probes 64q .. 64q+63 at
 * row i.  key = (q << 32) | i with q = p / 64, mixed with the seed's
 * golden-ratio multiple; z_i = -1 when bit (p mod 64) of the hash is set. */
int orc_rademacher(uint64_t seed, uint64_t p, uint64_t i)
{
    uint64_t q = p / 64;
    uint64_t key = (q << 32) | (i & 0xffffffffULL);
    uint64_t h = orc_mix64(key ^ (seed * 0x9e3779b97f4a7c15ULL));
    return ((h >> (p % 64)) & 1) ? -1 : 1;
}

void orc_probe(uint64_t seed, uint64_t p, int64_t d, int8_t *z)
{
    for (int64_t i = 0; i < d; ++i)
        z[i] = (int8_t)orc_rademacher(seed, p, (uint64_t)i);
}

/* ---- Chebyshev moments (Section 2.2) ------------------------------------- */

/* y = A x for a CSR matrix; val == NULL means a 0/1 pattern scaled by `scale`.
 * Each row is summed on its own in entry order, so spreading the rows over
 * threads (rowpar) changes no result. */
static void csr_apply(int64_t nrows, const int64_t *rowptr, const int32_t *col,
                      const double *val, double scale, const double *x, double *y, int rowpar)
{
#pragma omp parallel for schedule(static) if (rowpar)
    for (int64_t i = 0; i < nrows; ++i) {
        long double s = 0.0L;
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            double a = val ? val[k] * scale : scale;
            s += (long double)a * (long double)x[col[k]];
        }
        y[i] = (double)s;
    }
}

/* y = A^T x for a CSR matrix with nrows rows (so y has ncols entries). */
static void csr_apply_t(int64_t nrows, int64_t ncols, const int64_t *rowptr, const int32_t *col,
                        const double *val, double scale, const double *x, double *y)
{
    long double *acc = (long double *)calloc((size_t)ncols, sizeof(long double));
    for (int64_t i = 0; i < nrows; ++i)
        for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) {
            double a = val ? val[k] * scale : scale;
            acc[col[k]] += (long double)a * (long double)x[i];
        }
    for (int64_t j = 0; j < ncols; ++j)
        y[j] = (double)acc[j];
    free(acc);
}

/* The operator whose trace function is estimated: A itself (gram == 0), or
 * A = X^T X for the nuclear norm (gram != 0, X has nrows x ncols). */
typedef struct {
    int64_t nrows, ncols;
    const int64_t *rowptr;
    const int32_t *col;
    const double *val;
    double scale;
    int gram;
    double *tmp; /* nrows scratch for the Gram case */
    int rowpar;  /* spread the rows of each product over threads */
} orc_op;

static int64_t op_dim(const orc_op *A) { return A->gram ? A->ncols : A->nrows; }

static void op_apply(const orc_op *A, const double *x, double *y)
{
    if (!A->gram) {
        csr_apply(A->nrows, A->rowptr, A->col, A->val, A->scale, x, y, A->rowpar);
    } else {
        csr_apply(A->nrows, A->rowptr, A->col, A->val, A->scale, x, A->tmp, A->rowpar);
        csr_apply_t(A->nrows, A->ncols, A->rowptr, A->col, A->val, A->scale, A->tmp, y);
    }
}

static long double dotl(int64_t d, const double *x, const double *y)
{
    long double s = 0.0L;
    for (int64_t i = 0; i < d; ++i)
        s += (long double)x[i] * (long double)y[i];
    return s;
}

/* Moments mu[0..deg] of one explicit probe z (entries +-1 or any reals).
 * At = alpha*A + beta*I with alpha = 2/(b-a), beta = -(a+b)/(b-a).
 * w_0 = z, w_1 = At z, w_{j+1} = 2 At w_j - w_{j-1}; mu_j = z . w_j. */
static int moments_one(const orc_op *A, double a, double b, const double *z, int deg, double *mu)
{
    int64_t d = op_dim(A);
    double alpha = 2.0 / (b - a);
    double beta = -(a + b) / (b - a);
    double *wprev = (double *)malloc(sizeof(double) * (size_t)d);
    double *wcur = (double *)malloc(sizeof(double) * (size_t)d);
    double *wnext = (double *)malloc(sizeof(double) * (size_t)d);
    double *aw = (double *)malloc(sizeof(double) * (size_t)d);
    if (!wprev || !wcur || !wnext || !aw) {
        free(wprev); free(wcur); free(wnext); free(aw);
        return -2;
    }
    memcpy(wcur, z, sizeof(double) * (size_t)d);
    mu[0] = (double)dotl(d, z, wcur);
    for (int j = 0; j < deg; ++j) {
        op_apply(A, wcur, aw);
#pragma omp parallel for schedule(static) if (A->rowpar)
        for (int64_t i = 0; i < d; ++i) {
            double atw = alpha * aw[i] + beta * wcur[i];
            wnext[i] = (j == 0) ? atw : 2.0 * atw - wprev[i];
        }
        double *t = wprev; wprev = wcur; wcur = wnext; wnext = t;
        mu[j + 1] = (double)dotl(d, z, wcur);
    }
    free(wprev); free(wcur); free(wnext); free(aw);
    return 0;
}

static int op_init(orc_op *A, int64_t nrows, int64_t ncols, const int64_t *rowptr,
                   const int32_t *col, const double *val, double scale, int gram)
{
    A->nrows = nrows; A->ncols = ncols; A->rowptr = rowptr; A->col = col;
    A->val = val; A->scale = scale; A->gram = gram; A->tmp = NULL; A->rowpar = 0;
    if (gram) {
        A->tmp = (double *)malloc(sizeof(double) * (size_t)(nrows > 0 ? nrows : 1));
        if (!A->tmp) return -2;
    }
    return 0;
}

/* Moments of explicitly given probes: z is nprobes x dim (row-major, doubles),
 * mu is nprobes x ld with mu[p*ld + j] for j <= deg[p]. */
int orc_moments_z(int64_t nrows, int64_t ncols, const int64_t *rowptr, const int32_t *col,
                  const double *val, double scale, int gram, double a, double b,
                  int nprobes, const double *z, const int32_t *deg, double *mu, int64_t ld)
{
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : rc)
    for (int p = 0; p < nprobes; ++p) {
        orc_op A;
        if (op_init(&A, nrows, ncols, rowptr, col, val, scale, gram)) { rc = -2; continue; }
        int64_t d = op_dim(&A);
        int r = moments_one(&A, a, b, z + (int64_t)p * d, deg[p], mu + (int64_t)p * ld);
        if (r < rc) rc = r;
        free(A.tmp);
    }
    return rc;
}

/* Moments of Rademacher probes with global ids probe_offset + p.  With fewer
 * probes than threads (and a plain operator, whose rows are independent
 * sums) the probes run one after another with each product's rows spread
 * over the threads; otherwise the probes are spread.  Either way every
 * number is computed by the same operations in the same order. */
int orc_moments(int64_t nrows, int64_t ncols, const int64_t *rowptr, const int32_t *col,
                const double *val, double scale, int gram, double a, double b, uint64_t seed,
                int64_t probe_offset, int nprobes, const int32_t *deg, double *mu, int64_t ld)
{
    int rc = 0;
    const int rowpar = !gram && nprobes < omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) reduction(min : rc) if (!rowpar)
    for (int p = 0; p < nprobes; ++p) {
        orc_op A;
        if (op_init(&A, nrows, ncols, rowptr, col, val, scale, gram)) { rc = -2; continue; }
        A.rowpar = rowpar;
        int64_t d = op_dim(&A);
        double *z = (double *)malloc(sizeof(double) * (size_t)d);
        if (!z) { free(A.tmp); rc = -2; continue; }
        for (int64_t i = 0; i < d; ++i)
            z[i] = (double)orc_rademacher(seed, (uint64_t)(probe_offset + p), (uint64_t)i);
        int r = moments_one(&A, a, b, z, deg[p], mu + (int64_t)p * ld);
        if (r < rc) rc = r;
        free(z);
        free(A.tmp);
    }
    return rc;
}

/* ---- Triangle moments (Section 2.1 Example; Section 5.4) ----------------- */

/* x[3p+0] = z^T A z, x[3p+1] = z^T A^2 z = |Az|^2, x[3p+2] = z^T A^3 z,
 * exactly in int64, for a 0/1 pattern matrix A and explicit probes
 * z (nprobes x d, +-1 as int8). */
int orc_triangle_moments_z(int64_t d, const int64_t *rowptr, const int32_t *col,
                           int nprobes, const int8_t *z, int64_t *x)
{
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : rc)
    for (int p = 0; p < nprobes; ++p) {
        const int8_t *zp = z + (int64_t)p * d;
        int64_t *y = (int64_t *)malloc(sizeof(int64_t) * (size_t)d);
        int64_t *w = (int64_t *)malloc(sizeof(int64_t) * (size_t)d);
        if (!y || !w) { free(y); free(w); rc = -2; continue; }
        for (int64_t i = 0; i < d; ++i) {        /* y = A z */
            int64_t s = 0;
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += zp[col[k]];
            y[i] = s;
        }
        for (int64_t i = 0; i < d; ++i) {        /* w = A y */
            int64_t s = 0;
            for (int64_t k = rowptr[i]; k < rowptr[i + 1]; ++k) s += y[col[k]];
            w[i] = s;
        }
        int64_t x1 = 0, x2 = 0, x3 = 0;
        for (int64_t i = 0; i < d; ++i) {
            x1 += (int64_t)zp[i] * y[i];
            x2 += y[i] * y[i];
            x3 += y[i] * w[i];
        }
        x[3 * (int64_t)p + 0] = x1;
        x[3 * (int64_t)p + 1] = x2;
        x[3 * (int64_t)p + 2] = x3;
        free(y); free(w);
    }
    return rc;
}

int orc_triangle_moments(int64_t d, const int64_t *rowptr, const int32_t *col, uint64_t seed,
                         int64_t probe_offset, int nprobes, int64_t *x)
{
    int rc = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(min : rc)
    for (int p = 0; p < nprobes; ++p) {
        int8_t *z = (int8_t *)malloc((size_t)(d > 0 ? d : 1));
        if (!z) { rc = -2; continue; }
        orc_probe(seed, (uint64_t)(probe_offset + p), d, z);
        int r = orc_triangle_moments_z(d, rowptr, col, 1, z, x + 3 * (int64_t)p);
        if (r < rc) rc = r;
        free(z);
    }
    return rc;
}

/* Exact triangle count by brute force: for every edge (u, v) with u < v, count
 * the common neighbours w > v by merging the two sorted adjacency lists. */
int64_t orc_triangle_count(int64_t d, const int64_t *rowptr, const int32_t *col)
{
    int64_t total = 0;
#pragma omp parallel for schedule(dynamic, 1024) reduction(+ : total)
    for (int64_t u = 0; u < d; ++u) {
        for (int64_t k = rowptr[u]; k < rowptr[u + 1]; ++k) {
            int64_t v = col[k];
            if (v <= u) continue;
            int64_t i = rowptr[u], j = rowptr[v];
            while (i < rowptr[u + 1] && j < rowptr[v + 1]) {
                int64_t a = col[i], b = col[j];
                if (a < b) ++i;
                else if (b < a) ++j;
                else { if (a > v) ++total; ++i; ++j; }
            }
        }
    }
    return total;
}
