// Host-side arithmetic of the multilevel method: Chebyshev coefficients,
// band variances from a pilot sample, optimal level selection, sample
// allocation, and the triangle control-variate estimate.  All of it is
// O(n^2 m_pilot) or less (Section 3.2), negligible beside the moment kernels.
// Built with -ffp-contract=off so that the rounding of every expression is the
// one written here.
#include <cmath>
#include <cstdint>
#include <limits>
#include <vector>

#include "mlt_internal.h"

namespace mlt {

// Chebyshev interpolant at the extrema nodes x_j = cos(j pi / n) (Section 2.2):
// c_k = (2/n) * sum_j w_j f~(x_j) cos(pi j k / n), w_0 = w_n = 1/2, else 1, and
// c_0, c_n halved.  The cosine argument is reduced exactly (j k mod 2n) before
// the long-double cosine; the FFT of the paper only accelerates this sum.
int cheb_coeffs_host(int fn, double p, double a, double b, int n, double* c)
{
    if (!c) return fail(MLT_EINVAL, "mlt_cheb_coeffs: null output");
    if (n < 1 || n > MLT_MAX_DEGREE) return fail(MLT_EINVAL, "mlt_cheb_coeffs: n out of range");
    if (!(a < b) || !std::isfinite(a) || !std::isfinite(b))
        return fail(MLT_EINVAL, "mlt_cheb_coeffs: need finite a < b");
    switch (fn) {
    case MLT_FN_LOG:
        if (!(a > 0.0)) return fail(MLT_EINVAL, "mlt_cheb_coeffs: log needs a > 0");
        break;
    case MLT_FN_SQRT:
        if (!(a >= 0.0)) return fail(MLT_EINVAL, "mlt_cheb_coeffs: sqrt needs a >= 0");
        break;
    case MLT_FN_INV:
        if (a <= 0.0 && b >= 0.0) return fail(MLT_EINVAL, "mlt_cheb_coeffs: 1/x needs 0 outside [a, b]");
        break;
    case MLT_FN_POW:
        if (!(a >= 0.0) && std::floor(p) != p)
            return fail(MLT_EINVAL, "mlt_cheb_coeffs: x^p with fractional p needs a >= 0");
        if (a <= 0.0 && p < 0.0) return fail(MLT_EINVAL, "mlt_cheb_coeffs: x^p with p < 0 needs a > 0");
        break;
    case MLT_FN_EXP:
    case MLT_FN_CUBE:
        break;
    default:
        return fail(MLT_EINVAL, "mlt_cheb_coeffs: unknown function");
    }
    const long double pi = 3.141592653589793238462643383279502884L;
    std::vector<long double> fx(n + 1);
    for (int j = 0; j <= n; ++j) {
        const long double x = cosl(pi * (long double)j / (long double)n);
        const long double t = 0.5L * ((long double)(b - a) * x + (long double)(a + b));
        long double v;
        switch (fn) {
        case MLT_FN_LOG: v = logl(t); break;
        case MLT_FN_SQRT: v = sqrtl(t > 0 ? t : 0); break;
        case MLT_FN_EXP: v = expl(t); break;
        case MLT_FN_INV: v = 1.0L / t; break;
        case MLT_FN_POW: v = powl(t > 0 ? t : (std::floor(p) == p ? t : 0), (long double)p); break;
        default: v = t * t * t; break;
        }
        fx[j] = v;
    }
    const int two_n = 2 * n;
    std::vector<long double> cosv(two_n);
    for (int r = 0; r < two_n; ++r) cosv[r] = cosl(pi * (long double)r / (long double)n);
    for (int k = 0; k <= n; ++k) {
        long double s = 0.5L * (fx[0] + fx[n] * cosv[(int64_t)n * k % two_n]);
        for (int j = 1; j < n; ++j) s += fx[j] * cosv[(int64_t)j * k % two_n];
        long double ck = 2.0L * s / (long double)n;
        if (k == 0 || k == n) ck *= 0.5L;
        c[k] = (double)ck;
    }
    return MLT_OK;
}

// Section 3.1: a sample of Q_{l'l} costs l matvecs, or ceil(l/2) with the
// symmetric (doubling) evaluation.
double cost_of(int l, int model)
{
    return model == MLT_COST_LINEAR ? (double)l : (double)((l + 1) / 2);
}

// V[lo][hi], 0 <= lo < hi <= n: sample variance over the m pilot probes of
// Q_{lo,hi} = sum_{j=lo+1..hi} c_j mu_j (Section 3.2.1, Eq. def:qlevels).
// For each lo the bands are grown one term at a time, so every band is summed
// left to right from its own first term (no prefix-sum cancellation).
void band_variances(const double* c, int n, const double* mu, int64_t ld, int m, double* V)
{
    const int n1 = n + 1;
    for (int i = 0; i < n1 * n1; ++i) V[i] = 0.0;
    if (m < 2) return;
    std::vector<double> q(m);
    for (int lo = 0; lo < n; ++lo) {
        for (int p = 0; p < m; ++p) q[p] = 0.0;
        for (int hi = lo + 1; hi <= n; ++hi) {
            double mean = 0.0;
            for (int p = 0; p < m; ++p) {
                q[p] += c[hi] * mu[(int64_t)p * ld + hi];
                mean += q[p];
            }
            mean /= m;
            double ss = 0.0;
            for (int p = 0; p < m; ++p) {
                const double e = q[p] - mean;
                ss += e * e;
            }
            V[lo * n1 + hi] = ss / (m - 1);
        }
    }
}

static double mu_factor(double S, int mode, double target)
{
    if (S <= 0.0) return 0.0;
    return mode == MLT_MODE_VARIANCE ? S / target : target / S;
}

static bool top_ok(double S, double Vtop, double Ctop, int mode, double target, int m_pilot)
{
    return mu_factor(S, mode, target) * std::sqrt(Vtop / Ctop) >= (double)m_pilot;
}

// Theorem levels, Eq. costrecurrence: C_0 = 0 and
// C_l = min_{0 <= l' < l} C_{l'} + sqrt(V_{l'l} C_{l'l}); at l = n only
// predecessors whose complete path recommends m_L >= m_pilot are admitted
// (Section 3.2.1).  With max_levels > 0 the programme also counts levels.
// Ties go to the smaller l'.  If no predecessor is admitted: one level, l_1 = n.
int select_levels(const double* V, int n, int cost_model, int m_pilot, int mode, double target,
                  int max_levels, int* levels_out, int* nlevels_out)
{
    const int n1 = n + 1;
    const double INF = std::numeric_limits<double>::infinity();
    const double cn = cost_of(n, cost_model);
    std::vector<int> path;
    if (max_levels <= 0) {
        std::vector<double> C(n1, INF);
        std::vector<int> pred(n1, -1);
        C[0] = 0.0;
        for (int l = 1; l < n; ++l) {
            const double cl = cost_of(l, cost_model);
            for (int lp = 0; lp < l; ++lp) {
                const double v = C[lp] + std::sqrt(V[lp * n1 + l] * cl);
                if (v < C[l]) { C[l] = v; pred[l] = lp; }
            }
        }
        int best = -1;
        double bestS = INF;
        for (int lp = 0; lp < n; ++lp) {
            const double S = C[lp] + std::sqrt(V[lp * n1 + n] * cn);
            if (m_pilot > 0 && !top_ok(S, V[lp * n1 + n], cn, mode, target, m_pilot)) continue;
            if (S < bestS) { bestS = S; best = lp; }
        }
        path.push_back(n);
        for (int l = best; l > 0; l = pred[l]) path.push_back(l);
    } else {
        const int T = max_levels;
        std::vector<double> C((size_t)(T + 1) * n1, INF);
        std::vector<int> pred((size_t)(T + 1) * n1, -1);
        C[0] = 0.0;
        for (int t = 1; t <= T; ++t)
            for (int l = 1; l < n; ++l) {
                const double cl = cost_of(l, cost_model);
                for (int lp = 0; lp < l; ++lp) {
                    const double prev = C[(size_t)(t - 1) * n1 + lp];
                    if (prev == INF) continue;
                    const double v = prev + std::sqrt(V[lp * n1 + l] * cl);
                    if (v < C[(size_t)t * n1 + l]) { C[(size_t)t * n1 + l] = v; pred[(size_t)t * n1 + l] = lp; }
                }
            }
        int best = -1, bestT = -1;
        double bestS = INF;
        for (int t = 1; t <= T; ++t)
            for (int lp = 0; lp < n; ++lp) {
                const double prev = C[(size_t)(t - 1) * n1 + lp];
                if (prev == INF) continue;
                const double S = prev + std::sqrt(V[lp * n1 + n] * cn);
                if (m_pilot > 0 && !top_ok(S, V[lp * n1 + n], cn, mode, target, m_pilot)) continue;
                if (S < bestS) { bestS = S; best = lp; bestT = t; }
            }
        path.push_back(n);
        int l = best, t = bestT - 1;
        while (l > 0) {
            path.push_back(l);
            l = pred[(size_t)t * n1 + l];
            --t;
        }
    }
    const int L = (int)path.size();
    if (L > MLT_MAX_LEVELS) return fail(MLT_ERANGE, "level selection produced too many levels");
    for (int k = 0; k < L; ++k) levels_out[k] = path[L - 1 - k];
    *nlevels_out = L;
    return MLT_OK;
}

// Eqs. optSamples / optMu: m_k = mu sqrt(V_k / C_k) with mu = S / eps^2
// (variance mode) or C / S (budget mode), S = sum_k sqrt(V_k C_k); rounded up,
// at least 1, and at least m_pilot on the top level when the pilot is reused.
void allocate_samples(const int* levels, int L, const double* V, int n, int cost_model, int mode,
                      double target, int m_pilot, int64_t* m_out)
{
    const int n1 = n + 1;
    std::vector<double> Vk(L), Ck(L);
    double S = 0.0;
    for (int k = 0; k < L; ++k) {
        const int lp = k == 0 ? 0 : levels[k - 1];
        Vk[k] = V[lp * n1 + levels[k]];
        Ck[k] = cost_of(levels[k], cost_model);
        S += std::sqrt(Vk[k] * Ck[k]);
    }
    const double mu = mu_factor(S, mode, target);
    for (int k = 0; k < L; ++k) {
        const double want = std::ceil(mu * std::sqrt(Vk[k] / Ck[k]));
        int64_t mk = want >= 1.0 ? (int64_t)want : 1;
        m_out[k] = mk;
    }
    if (m_pilot > 0 && m_out[L - 1] < m_pilot) m_out[L - 1] = m_pilot;
}

// Q_{lo,hi} = sum_{j=lo+1..hi} c_j mu_j for each of nprobes moment rows
// (Eq. def:qlevels), summed left to right from the band's first term.
void band_samples(const double* c, int lo, int hi, const double* mu, int64_t ld, int64_t nprobes, double* q)
{
    for (int64_t p = 0; p < nprobes; ++p) {
        const double* row = mu + p * ld;
        double s = 0.0;
        for (int j = lo + 1; j <= hi; ++j) s += c[j] * row[j];
        q[p] = s;
    }
}

// Mean and sample variance (divisor m - 1, NaN for m < 2) of one level's
// samples, in sample order: the per-level terms of Eq. multiEstimator.
void level_stats(const double* v, int64_t m, double* mean, double* var)
{
    double s = 0.0;
    for (int64_t i = 0; i < m; ++i) s += v[i];
    const double mu = s / (double)m;
    double ss = 0.0;
    for (int64_t i = 0; i < m; ++i) ss += (v[i] - mu) * (v[i] - mu);
    *mean = mu;
    *var = m > 1 ? ss / (double)(m - 1) : std::nan("");
}

// Section 5.4's a-priori coefficients from the Chebyshev expansion
// x^3 = (3 T_1(x) + T_3(x)) / 4 on the map of [a, b] onto [-1, 1]: with
// A = r At + c I, A^3 - a2 A^2 - a1 A = (r^3/4) T_3(At) + (c^3 - 3 c r^2/4) I
// for a2 = 3c and a1 = 3r^2/4 - 3c^2.
void triangle_cv_cheb(double a, double b, double* a1, double* a2)
{
    const double c = 0.5 * (a + b);
    const double r = 0.5 * (b - a);
    *a1 = 0.75 * r * r - 3.0 * c * c;
    *a2 = 3.0 * c;
}

// Section 5.4 with given coefficients: T = [mean x3 - a2 (mean x2 - nnz) -
// a1 mean x1] / 6; the residuals x3 - a2 x2 - a1 x1 have sample variance
// (divisor m - 1) [C33 + a2^2 C22 + a1^2 C11 - 2 a2 C23 - 2 a1 C13 +
// 2 a1 a2 C12] / (m (m - 1)), C_ij = m S_ij - S_i S_j from exact integer sums;
// the double-precision steps run in the order written.
void triangle_estimate_fixed_host(const int64_t* x, int64_t m, int64_t nnz, double a1, double a2, double* est,
                                  double* se)
{
    typedef __int128 i128;
    i128 S1 = 0, S2 = 0, S3 = 0, S11 = 0, S22 = 0, S33 = 0, S12 = 0, S13 = 0, S23 = 0;
    for (int64_t p = 0; p < m; ++p) {
        const i128 u = x[3 * p], v = x[3 * p + 1], w = x[3 * p + 2];
        S1 += u; S2 += v; S3 += w;
        S11 += u * u; S22 += v * v; S33 += w * w;
        S12 += u * v; S13 += u * w; S23 += v * w;
    }
    const i128 mm = m;
    const double C11 = (double)(mm * S11 - S1 * S1);
    const double C22 = (double)(mm * S22 - S2 * S2);
    const double C33 = (double)(mm * S33 - S3 * S3);
    const double C12 = (double)(mm * S12 - S1 * S2);
    const double C13 = (double)(mm * S13 - S1 * S3);
    const double C23 = (double)(mm * S23 - S2 * S3);
    const double fm = (double)m;
    const double mean1 = (double)S1 / fm;
    const double mean2 = (double)S2 / fm;
    const double mean3 = (double)S3 / fm;
    *est = (mean3 - a2 * (mean2 - (double)nnz) - a1 * mean1) / 6.0;
    const double q = C33 + a2 * a2 * C22 + a1 * a1 * C11 - 2.0 * a2 * C23 - 2.0 * a1 * C13 + 2.0 * a1 * a2 * C12;
    const double var = m > 1 ? q / (fm * (fm - 1.0)) : std::nan("");
    *se = std::sqrt((var > 0.0 ? var : (var == var ? 0.0 : var)) / fm) / 6.0;
}

// Section 5.4 estimate from exact integer sums: ordinary least squares of x3
// on (1, x1, x2), then T = [mean x3 - a2 (mean x2 - nnz) - a1 mean x1] / 6
// (tr A = 0, tr A^2 = nnz for a 0/1 symmetric matrix without self-loops).
// Without control variates T = mean x3 / 6.  The double-precision steps run in
// exactly the order written.
void triangle_estimate_host(const int64_t* x, int64_t m, int64_t nnz, int use_cv, double* est,
                            double* se, double* a1_out, double* a2_out)
{
    typedef __int128 i128;
    i128 S1 = 0, S2 = 0, S3 = 0, S11 = 0, S22 = 0, S33 = 0, S12 = 0, S13 = 0, S23 = 0;
    for (int64_t p = 0; p < m; ++p) {
        const i128 a = x[3 * p], b = x[3 * p + 1], c = x[3 * p + 2];
        S1 += a; S2 += b; S3 += c;
        S11 += a * a; S22 += b * b; S33 += c * c;
        S12 += a * b; S13 += a * c; S23 += b * c;
    }
    const i128 mm = m;
    const double fm = (double)m;
    const double C33 = (double)(mm * S33 - S3 * S3);
    if (!use_cv) {
        *est = ((double)S3 / fm) / 6.0;
        const double var = m > 1 ? C33 / (fm * (fm - 1.0)) : std::nan("");
        *se = std::sqrt(var / fm) / 6.0;
        return;
    }
    const double C11 = (double)(mm * S11 - S1 * S1);
    const double C22 = (double)(mm * S22 - S2 * S2);
    const double C12 = (double)(mm * S12 - S1 * S2);
    const double C13 = (double)(mm * S13 - S1 * S3);
    const double C23 = (double)(mm * S23 - S2 * S3);
    const double det = C11 * C22 - C12 * C12;
    double a1 = 0.0, a2 = 0.0;
    if (det != 0.0) {
        a1 = (C13 * C22 - C23 * C12) / det;
        a2 = (C23 * C11 - C13 * C12) / det;
    }
    if (a1_out) *a1_out = a1;
    if (a2_out) *a2_out = a2;
    const double mean1 = (double)S1 / fm;
    const double mean2 = (double)S2 / fm;
    const double mean3 = (double)S3 / fm;
    *est = (mean3 - a2 * (mean2 - (double)nnz) - a1 * mean1) / 6.0;
    const double rss = C33 - a1 * C13 - a2 * C23;
    const double dof = fm - 3.0;
    const double var = m > 3 ? rss / (fm * dof) : std::nan("");
    *se = std::sqrt((var > 0.0 ? var : (var == var ? 0.0 : var)) / fm) / 6.0;
}

}  // namespace mlt
