// Spectrum interval by Lanczos.  The affine map of Section 2.2 needs an
// interval containing the spectrum, and the paper only asks for a rough
// estimate of the extreme eigenvalues.  k steps of the Lanczos recurrence
//   w = A q_j - alpha_j q_j - beta_{j-1} q_{j-1},  beta_j = |w|,  q_{j+1} = w / beta_j
// give a tridiagonal T_k whose extreme eigenvalues (Ritz values) theta approach
// those of A from inside; each Ritz pair's residual |A y - theta y| equals
// beta_k |s_k| (s the eigenvector of T_k, s_k its last entry), and an interval
// of half-width |residual| around theta holds an eigenvalue of A.  The bounds
// returned are theta_min - r_min and theta_max + r_max, widened by 1% of their
// magnitude.  The T_k eigenvalues come from Sturm-sequence bisection and their
// eigenvectors from inverse iteration, both on the host (k is small).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <vector>

#include "mlt_internal.h"
#include "rng.cuh"

namespace mlt {
namespace {

// Vectors live with stride 2 (entry i at v[2 i]; the odd slots stay zero) so
// the product kernel can read them as 16-byte pairs.
__global__ void start_vector_kernel(double* q, int64_t d, uint64_t seedmix, double inv_norm)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
        q[2 * i] = probe_negative(seedmix, 0, (uint64_t)i) ? -inv_norm : inv_norm;
        q[2 * i + 1] = 0.0;
    }
}

// part[block] = partial sum of x[2i] y[2i] over this block's indices
__global__ void dot2_kernel(const double* __restrict__ x, const double* __restrict__ y, int64_t d,
                            double* __restrict__ part)
{
    __shared__ double sh[32];
    double s = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
        s += x[2 * i] * y[2 * i];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        double t = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) t += sh[w];
        part[blockIdx.x] = t;
    }
}

// w = w - alpha q - beta p
__global__ void axpy2_kernel(double* __restrict__ w, const double* __restrict__ q, const double* __restrict__ p,
                             int64_t d, double alpha, double beta)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x)
        w[2 * i] = w[2 * i] - alpha * q[2 * i] - beta * p[2 * i];
}

__global__ void scale2_kernel(double* __restrict__ dst, const double* __restrict__ src, int64_t d, double f)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < d; i += (int64_t)gridDim.x * blockDim.x) {
        dst[2 * i] = src[2 * i] * f;
        dst[2 * i + 1] = 0.0;
    }
}

// Number of eigenvalues of the tridiagonal (dg, e) below x (Sturm sequence).
int count_below(const std::vector<double>& dg, const std::vector<double>& e, double x)
{
    const int n = (int)dg.size();
    int cnt = 0;
    double q = dg[0] - x;
    if (q < 0) ++cnt;
    for (int i = 1; i < n; ++i) {
        if (q == 0.0) q = 1e-300;
        q = (dg[i] - x) - e[i - 1] * e[i - 1] / q;
        if (q < 0) ++cnt;
    }
    return cnt;
}

// The j-th smallest eigenvalue (0-based) by bisection on the Gershgorin interval.
double bisect_eigenvalue(const std::vector<double>& dg, const std::vector<double>& e, int j)
{
    const int n = (int)dg.size();
    double lo = 1e300, hi = -1e300;
    for (int i = 0; i < n; ++i) {
        const double r = (i > 0 ? std::fabs(e[i - 1]) : 0.0) + (i < n - 1 ? std::fabs(e[i]) : 0.0);
        lo = std::min(lo, dg[i] - r);
        hi = std::max(hi, dg[i] + r);
    }
    for (int it = 0; it < 200 && hi - lo > 1e-15 * std::max(std::fabs(lo), std::fabs(hi)) + 1e-300; ++it) {
        const double mid = 0.5 * (lo + hi);
        if (count_below(dg, e, mid) > j) hi = mid;
        else lo = mid;
    }
    return 0.5 * (lo + hi);
}

// Last entry of the unit eigenvector for eigenvalue theta (inverse iteration
// with a tridiagonal solve of (T - theta I) v = b, three sweeps).
double eigvec_last(const std::vector<double>& dg, const std::vector<double>& e, double theta)
{
    const int n = (int)dg.size();
    std::vector<double> v(n, 1.0), c(n), dd(n);
    const double shift = theta + 1e-12 * (std::fabs(theta) + 1.0);
    for (int sweep = 0; sweep < 3; ++sweep) {
        // forward elimination (Thomas), tiny pivots replaced by a small number
        for (int i = 0; i < n; ++i) {
            double piv = dg[i] - shift - (i > 0 ? e[i - 1] * c[i - 1] : 0.0);
            if (std::fabs(piv) < 1e-300) piv = 1e-300;
            c[i] = i < n - 1 ? e[i] / piv : 0.0;
            dd[i] = (v[i] - (i > 0 ? e[i - 1] * dd[i - 1] : 0.0)) / piv;
        }
        for (int i = n - 1; i >= 0; --i) v[i] = dd[i] - (i < n - 1 ? c[i] * v[i + 1] : 0.0);
        double nrm = 0.0;
        for (double x : v) nrm += x * x;
        nrm = std::sqrt(nrm);
        if (!(nrm > 0.0) || !std::isfinite(nrm)) return 1.0;
        for (double& x : v) x /= nrm;
    }
    return v[n - 1];
}

double dot_sync(const double* x, const double* y, int64_t d, double* part, int nblk, std::vector<double>& h,
                cudaStream_t s, int* rc)
{
    dot2_kernel<<<nblk, 256, 0, s>>>(x, y, d, part);
    cudaError_t e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaMemcpyAsync(h.data(), part, nblk * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
        *rc = cuda_fail(e, "lanczos dot");
        return 0.0;
    }
    double t = 0.0;
    for (int b = 0; b < nblk; ++b) t += h[b];
    return t;
}

}  // namespace

int lanczos_bounds(mlt_matrix* M, int steps, uint64_t seed, double* lo, double* hi, cudaStream_t s)
{
    const bool gram = (M->flags & MLT_GRAM) != 0;
    const int64_t d = M->dim();
    if (d < 1) return fail(MLT_EINVAL, "mlt_spectrum_bounds: empty operator");
    const int k = (int)std::min<int64_t>(std::max(steps, 2), d);
    int rc;
    const size_t vb = (size_t)d * 2 * sizeof(double);
    const size_t tb = gram ? (size_t)M->A.nrows * 2 * sizeof(double) : 0;
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((d + 255) / 256, 4LL * M->num_sms));
    if ((rc = M->ws_v[0].ensure(3 * vb + tb + nblk * sizeof(double) + 64, s))) return rc;
    double* q_prev = M->ws_v[0].as<double>();
    double* q = q_prev + 2 * d;
    double* w = q + 2 * d;
    double* t = w + 2 * d;
    double* part = t + (gram ? 2 * M->A.nrows : 0);
    MLT_CUDA_TRY(cudaMemsetAsync(q_prev, 0, vb, s));
    const int g = (int)std::min<int64_t>((d + 255) / 256, 16LL * M->num_sms);
    {
        ProfScope ps("lanczos_vectors", s);
        start_vector_kernel<<<g, 256, 0, s>>>(q, d, seed * kGolden, 1.0 / std::sqrt((double)d));
    }
    MLT_CUDA_TRY(cudaGetLastError());
    if (gram) MLT_CUDA_TRY(cudaMemsetAsync(t, 0, tb, s));
    std::vector<double> alpha, beta, h(nblk);
    double bprev = 0.0;
    for (int j = 0; j < k; ++j) {
        if (gram) {
            if ((rc = spmv_f64(M, M->A, M->plan_A, q, t, s))) return rc;
            if ((rc = spmv_f64(M, M->AT, M->plan_AT, t, w, s))) return rc;
        } else {
            if ((rc = spmv_f64(M, M->A, M->plan_A, q, w, s))) return rc;
        }
        rc = MLT_OK;
        const double a = dot_sync(q, w, d, part, nblk, h, s, &rc);
        if (rc) return rc;
        {
            ProfScope ps("lanczos_vectors", s);
            axpy2_kernel<<<g, 256, 0, s>>>(w, q, q_prev, d, a, bprev);
        }
        MLT_CUDA_TRY(cudaGetLastError());
        const double b2 = dot_sync(w, w, d, part, nblk, h, s, &rc);
        if (rc) return rc;
        alpha.push_back(a);
        const double b = std::sqrt(std::max(b2, 0.0));
        beta.push_back(b);
        if (!(b > 1e-12 * (std::fabs(a) + bprev + 1e-300))) break;   // invariant subspace found
        {
            ProfScope ps("lanczos_vectors", s);
            scale2_kernel<<<g, 256, 0, s>>>(q_prev, q, d, 1.0);       // q_prev <- q
            scale2_kernel<<<g, 256, 0, s>>>(q, w, d, 1.0 / b);        // q <- w / beta
        }
        MLT_CUDA_TRY(cudaGetLastError());
        bprev = b;
    }
    const int n = (int)alpha.size();
    std::vector<double> e(beta.begin(), beta.begin() + (n - 1));
    const double tmin = bisect_eigenvalue(alpha, e, 0);
    const double tmax = bisect_eigenvalue(alpha, e, n - 1);
    const double blast = beta[n - 1];
    const double rmin = std::fabs(blast * eigvec_last(alpha, e, tmin));
    const double rmax = std::fabs(blast * eigvec_last(alpha, e, tmax));
    const double sc = gram ? M->scale * M->scale : M->scale;
    double a0 = (tmin - rmin) * sc, b0 = (tmax + rmax) * sc;
    if (sc < 0) std::swap(a0, b0);
    a0 -= 0.01 * std::fabs(a0);
    b0 += 0.01 * std::fabs(b0);
    if (gram) a0 = std::max(a0, 1e-6 * b0);
    *lo = a0;
    *hi = b0;
    return MLT_OK;
}

}  // namespace mlt
