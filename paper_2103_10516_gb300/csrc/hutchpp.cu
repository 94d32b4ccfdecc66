// Hutch++ on the Chebyshev interpolant, and the block polynomial application
// behind it.  Section 5.3 observes that the Estrada index is dominated by the
// largest eigenvalues and proposes the variance reduction of Hutch++ (Meyer,
// Musco, Musco and Woodruff, 2021): with S and G blocks of Rademacher probes,
//   Q         an orthonormal basis of p(At) S,
//   estimate  tr(Q^T p(At) Q) + (1/g) sum_i g_i'^T p(At) g_i',  g_i' = (I - QQ^T) g_i,
// which is unbiased for any Q built independently of G, exact in the first
// term, and leaves Hutchinson's estimator only the spectrum outside span(Q).
//
// Data layout (device, FP64, row-major like the moment engine's V blocks):
// block[i * ld + c] is entry i of vector c; ld is even (16-byte pairs for the
// step kernel) and columns past the block's width are zero.
//
// Q comes from Cholesky QR applied twice (W = Y^T Y = R^T R, Y <- Y R^{-1})
// when the sketch fits one 64-column tile and W factors: two Gram blocks and
// two tile updates, bound by FP64 arithmetic.  Otherwise (wider sketches, or
// nearly dependent columns) it is classical Gram-Schmidt with one
// reorthogonalisation, column by column: per-CTA partial dot products (a warp
// per row, lanes over columns) added in CTA order by a one-block kernel, then
// the column's update, which also sums its new squared norm; a column left
// with at most kDropTol of its norm is dependent and zeroed.  The remainder
// probes are deflated by one block projection G - Q (Q^T G) against the
// orthonormal Q.  All sums are in a fixed order, so every result is
// reproducible.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <limits>
#include <vector>

#include "mlt_internal.h"
#include "rng.cuh"

namespace mlt {
namespace {

constexpr int kOrthoThreads = 256;
constexpr int kOrthoWarps = kOrthoThreads / 32;
constexpr int kMaxCols = 128;          // columns one dot-product pass covers (four per lane)
constexpr int kMaxSketch = 128;        // s
constexpr int kMaxRemainder = 1024;    // g
constexpr double kDropTol = 1e-10;     // a column keeping at most this fraction of its norm is dependent
constexpr unsigned kFull = 0xFFFFFFFFu;

// block[i * ld + c] = z_c(i) for the Rademacher probe with id id0 + c (c < cols), 0 beyond.
template <typename T>
__global__ void rademacher_block_kernel(T* __restrict__ block, int64_t d, int ld, int cols, uint64_t seedmix,
                                        int64_t id0)
{
    const int64_t total = d * (int64_t)ld;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ld;
        const int c = (int)(e % ld);
        T z = T(0);
        if (c < cols) z = probe_negative(seedmix, (uint64_t)(id0 + c), (uint64_t)i) ? T(-1) : T(1);
        block[e] = z;
    }
}

__global__ void widen_block_kernel(const float* __restrict__ in, double* __restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

// Rows of CTA blockIdx.x: a contiguous range.
__device__ __forceinline__ void cta_rows(int64_t d, int64_t& r0, int64_t& r1)
{
    const int64_t per = (d + gridDim.x - 1) / gridDim.x;
    r0 = min(d, (int64_t)blockIdx.x * per);
    r1 = min(d, r0 + per);
}

// part[blockIdx.x * nq + c] = sum over the CTA's rows r of Q[r, c] * X[r, j]
// for c < nq <= kMaxCols; with X null, Q[r, c]^2 (squared column norms).
__global__ void __launch_bounds__(kOrthoThreads) col_dots_kernel(const double* __restrict__ Q, int ldq, int nq,
                                                                 const double* __restrict__ X, int ldx, int j,
                                                                 int64_t d, double* __restrict__ part)
{
    __shared__ double red[kOrthoWarps][kMaxCols];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t r0, r1;
    cta_rows(d, r0, r1);
    double acc[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll 2
    for (int64_t r = r0 + wid; r < r1; r += kOrthoWarps) {
        const double* q = Q + (size_t)r * ldq;
        const double x = X ? __ldg(X + (size_t)r * ldx + j) : 0.0;
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int c = lane + 32 * t;
            if (c < nq) {
                const double v = __ldg(q + c);
                acc[t] = fma(v, X ? x : v, acc[t]);
            }
        }
    }
#pragma unroll
    for (int t = 0; t < 4; ++t) red[wid][lane + 32 * t] = acc[t];
    __syncthreads();
    for (int c = threadIdx.x; c < nq; c += blockDim.x) {
        double s = 0.0;
        for (int w = 0; w < kOrthoWarps; ++w) s += red[w][c];
        part[(size_t)blockIdx.x * nq + c] = s;
    }
}

// out[c] = sum over b < nparts of part[b * n + c], in b order.
__global__ void sum_parts_kernel(const double* __restrict__ part, int nparts, int n, double* __restrict__ out)
{
    for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < n; c += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nparts; ++b) s += part[(size_t)b * n + c];
        out[c] = s;
    }
}

// X[r, j] -= sum_{c < nq} Q[r, c] coef[c] for every row (Q's columns and X's
// column j never overlap); part[blockIdx.x] = the CTA's sum of the new X[r, j]^2.
__global__ void __launch_bounds__(kOrthoThreads) col_update_kernel(const double* __restrict__ Q, int ldq, int nq,
                                                                   double* __restrict__ X, int ldx, int j,
                                                                   int64_t d, const double* __restrict__ coef,
                                                                   double* __restrict__ part)
{
    __shared__ double red[kOrthoWarps];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t r0, r1;
    cta_rows(d, r0, r1);
    double cf[4];
#pragma unroll
    for (int t = 0; t < 4; ++t) cf[t] = lane + 32 * t < nq ? coef[lane + 32 * t] : 0.0;
    double nrm = 0.0;
    for (int64_t r = r0 + wid; r < r1; r += kOrthoWarps) {
        const double* q = Q + (size_t)r * ldq;
        double v = 0.0;
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (lane + 32 * t < nq) v = fma(__ldg(q + lane + 32 * t), cf[t], v);
#pragma unroll
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
        if (lane == 0) {
            double* xp = X + (size_t)r * ldx + j;
            const double xn = *xp - v;
            *xp = xn;
            nrm = fma(xn, xn, nrm);
        }
    }
    if (lane == 0) red[wid] = nrm;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        for (int w = 0; w < kOrthoWarps; ++w) s += red[w];
        part[blockIdx.x] = s;
    }
}

// Column j of X to unit norm, or to zero when its squared norm *nrm2 is at
// most kDropTol^2 times *orig2 (its squared norm before projection); kept[j]
// records which.
__global__ void col_normalize_kernel(double* __restrict__ X, int ldx, int j, int64_t d, const double* nrm2,
                                     const double* orig2, int* kept)
{
    const double n2 = *nrm2, o2 = *orig2;
    const bool keep = n2 > 0.0 && n2 > kDropTol * kDropTol * o2;
    const double inv = keep ? 1.0 / sqrt(n2) : 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d; r += (int64_t)gridDim.x * blockDim.x) {
        double* xp = X + (size_t)r * ldx + j;
        *xp = keep ? *xp * inv : 0.0;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) kept[j] = keep ? 1 : 0;
}

// ---- 64-column tiles: Gram blocks A^T B and updates X -= Q C ---------------

constexpr int kTile = 64;         // columns per tile
constexpr int kTileRows = 16;     // rows staged in shared memory per iteration

// part[blockIdx.x * kTile^2 + i * kTile + j] = sum over the CTA's rows r of
// A[r, i] * B[r, j] for i < na, j < nb (<= kTile; 0 beyond).  Thread t owns
// i = t / 4 and j = t % 4 + 4k (k < 16), so a warp's shared-memory reads hit
// distinct banks.
__global__ void __launch_bounds__(kOrthoThreads) tile_gram_kernel(const double* __restrict__ A, int lda, int na,
                                                                  const double* __restrict__ B, int ldb, int nb,
                                                                  int64_t d, double* __restrict__ part)
{
    __shared__ double sA[kTileRows][kTile], sB[kTileRows][kTile];
    const int t = threadIdx.x, i = t >> 2, jb = t & 3;
    int64_t r0, r1;
    cta_rows(d, r0, r1);
    double acc[16];
#pragma unroll
    for (int k = 0; k < 16; ++k) acc[k] = 0.0;
    for (int64_t base = r0; base < r1; base += kTileRows) {
        for (int e = t; e < kTileRows * kTile; e += kOrthoThreads) {
            const int rr = e / kTile, cc = e % kTile;
            const int64_t r = base + rr;
            sA[rr][cc] = (r < r1 && cc < na) ? __ldg(A + (size_t)r * lda + cc) : 0.0;
            sB[rr][cc] = (r < r1 && cc < nb) ? __ldg(B + (size_t)r * ldb + cc) : 0.0;
        }
        __syncthreads();
#pragma unroll 4
        for (int rr = 0; rr < kTileRows; ++rr) {
            const double av = sA[rr][i];
#pragma unroll
            for (int k = 0; k < 16; ++k) acc[k] = fma(av, sB[rr][jb + 4 * k], acc[k]);
        }
        __syncthreads();
    }
    double* out = part + (size_t)blockIdx.x * kTile * kTile + i * kTile + jb;
#pragma unroll
    for (int k = 0; k < 16; ++k) out[4 * k] = acc[k];
}

// X[r, j] = sum_{i < nq} Q[r, i] C[i * kTile + j] (assign), or X[r, j] -= that
// sum, for j < nx (<= kTile) and every row.  Each tile of kTileRows rows of Q
// is staged in shared memory before any of those rows of X is written, so Q
// may be X itself for the assignment.
__global__ void __launch_bounds__(kOrthoThreads) tile_update_kernel(const double* Q, int ldq, int nq,
                                                                    const double* __restrict__ C, double* X, int ldx,
                                                                    int nx, int64_t d, int assign)
{
    __shared__ double sC[kTile][kTile];
    __shared__ double sQ[kTileRows][kTile];
    const int t = threadIdx.x, j = t & (kTile - 1), rsub = t >> 6;
    for (int e = t; e < kTile * kTile; e += kOrthoThreads) sC[e / kTile][e % kTile] = C[e];
    int64_t r0, r1;
    cta_rows(d, r0, r1);
    for (int64_t base = r0; base < r1; base += kTileRows) {
        __syncthreads();   // C staged, or the previous tile's reads of sQ done
        for (int e = t; e < kTileRows * kTile; e += kOrthoThreads) {
            const int rr = e / kTile, cc = e % kTile;
            const int64_t r = base + rr;
            sQ[rr][cc] = (r < r1 && cc < nq) ? Q[(size_t)r * ldq + cc] : 0.0;
        }
        __syncthreads();
        for (int rr = rsub; rr < kTileRows; rr += kOrthoThreads / kTile) {
            const int64_t r = base + rr;
            if (r >= r1 || j >= nx) continue;
            double v = 0.0;
#pragma unroll 16
            for (int i = 0; i < kTile; ++i) v = fma(sQ[rr][i], sC[i][j], v);
            double* xp = X + (size_t)r * ldx + j;
            *xp = assign ? v : *xp - v;
        }
    }
}

// Device scratch of the orthonormalisation: CTA partials and small vectors.
struct OrthoScratch {
    double* tpart;   // [nparts][kTile * kTile]: tile Gram partials
    double* tc;      // [kMaxSketch / kTile][kTile * kTile]: tile coefficients
    double* part;    // [nparts][kMaxCols]
    double* r;       // kMaxCols + 1: first-pass coefficients, then the column's squared norm
    double* r2;      // kMaxCols: second-pass coefficients
    double* nrm2;    // 1
    double* norms;   // kMaxRemainder: squared column norms
    int* kept;       // kMaxSketch
    int nparts;
};

int ortho_grid(const mlt_matrix* M, int64_t d)
{
    return (int)std::max<int64_t>(1, std::min<int64_t>(4LL * M->num_sms, (d + 63) / 64));
}

// One projection pass of column j of X against the nq columns of Q:
// coefficients into coef, then the update (its new squared norm's CTA partials in part).
int project_pass(const OrthoScratch& w, const double* Q, int ldq, int nq, double* X, int ldx, int j, int64_t d,
                 double* coef, cudaStream_t s)
{
    col_dots_kernel<<<w.nparts, kOrthoThreads, 0, s>>>(Q, ldq, nq, X, ldx, j, d, w.part);
    sum_parts_kernel<<<1, kMaxCols, 0, s>>>(w.part, w.nparts, nq, coef);
    col_update_kernel<<<w.nparts, kOrthoThreads, 0, s>>>(Q, ldq, nq, X, ldx, j, d, coef, w.part);
    MLT_CUDA_TRY(cudaGetLastError());
    return MLT_OK;
}

// Columns 0 .. cols-1 of Y orthonormal in place (classical Gram-Schmidt, two
// passes per column); dependent columns become zero and kept[] says which.
int orthonormalize(const OrthoScratch& w, double* Y, int ld, int cols, int64_t d, cudaStream_t s)
{
    ProfScope ps("hutchpp_orthonormalize", s);
    const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((d + 255) / 256, 1024));
    int rc;
    for (int j = 0; j < cols; ++j) {
        // pass 1's coefficients with the column's own squared norm as entry j
        col_dots_kernel<<<w.nparts, kOrthoThreads, 0, s>>>(Y, ld, j + 1, Y, ld, j, d, w.part);
        sum_parts_kernel<<<1, kMaxCols, 0, s>>>(w.part, w.nparts, j + 1, w.r);
        MLT_CUDA_TRY(cudaGetLastError());
        const double* n2 = w.r + j;
        if (j > 0) {
            col_update_kernel<<<w.nparts, kOrthoThreads, 0, s>>>(Y, ld, j, Y, ld, j, d, w.r, w.part);
            MLT_CUDA_TRY(cudaGetLastError());
            if ((rc = project_pass(w, Y, ld, j, Y, ld, j, d, w.r2, s))) return rc;
            sum_parts_kernel<<<1, 32, 0, s>>>(w.part, w.nparts, 1, w.nrm2);
            n2 = w.nrm2;
        }
        col_normalize_kernel<<<nb, 256, 0, s>>>(Y, ld, j, d, n2, w.r + j, w.kept);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    return MLT_OK;
}

// Squared norms of the cols columns of X into w.norms (device).
int column_norms(const OrthoScratch& w, const double* X, int ld, int cols, int64_t d, cudaStream_t s)
{
    for (int c0 = 0; c0 < cols; c0 += kMaxCols) {
        const int nq = std::min(kMaxCols, cols - c0);
        col_dots_kernel<<<w.nparts, kOrthoThreads, 0, s>>>(X + c0, ld, nq, nullptr, 0, 0, d, w.part);
        sum_parts_kernel<<<1, kMaxCols, 0, s>>>(w.part, w.nparts, nq, w.norms + c0);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    return MLT_OK;
}

// v_c^T p(At) v_c for the cols columns of V (overwritten; scratch of the same
// shape), from the doubling moments: mu_0 = v.v, mu_1 = v.V_1,
// mu_{2k+2} = 2 V_{k+1}.V_{k+1} - mu_0, mu_{2k+1} = 2 V_{k+1}.V_k - mu_1.
int quad_forms(mlt_matrix* M, const OrthoScratch& w, double a, double b, const double* c, int n, double* V,
               double* scratch, int ld, int cols, int64_t d, bool df, std::vector<double>& out, cudaStream_t s)
{
    out.assign(cols, 0.0);
    if (cols == 0) return MLT_OK;
    int rc;
    if ((rc = column_norms(w, V, ld, cols, d, s))) return rc;
    std::vector<double> mu0(cols);
    MLT_CUDA_TRY(cudaMemcpyAsync(mu0.data(), w.norms, cols * sizeof(double), cudaMemcpyDeviceToHost, s));
    const int K = (n + 1) / 2;
    const double* dots_dev = nullptr;
    if ((rc = moments_block(M, a, b, V, scratch, ld, cols, K, &dots_dev, df, s))) return rc;
    std::vector<double> dots((size_t)K * 2 * cols);
    MLT_CUDA_TRY(cudaMemcpyAsync(dots.data(), dots_dev, dots.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaStreamSynchronize(s));
    for (int col = 0; col < cols; ++col) {
        const double m0 = mu0[col];
        const double m1 = dots[(size_t)cols + col];
        double acc = c[0] * m0 + c[1] * m1;
        for (int j = 2; j <= n; ++j) {
            const double mj = (j & 1) ? 2.0 * dots[(size_t)((j - 1) / 2) * 2 * cols + cols + col] - m1
                                      : 2.0 * dots[(size_t)(j / 2 - 1) * 2 * cols + col] - m0;
            acc += c[j] * mj;
        }
        out[col] = acc;
    }
    return MLT_OK;
}

// C (tile-stride kTile) = A^T B for the na <= kTile columns of A and nb <= kTile of B.
int tile_gram(const OrthoScratch& w, const double* A, int lda, int na, const double* B, int ldb, int nb, int64_t d,
              double* C, cudaStream_t s)
{
    tile_gram_kernel<<<w.nparts, kOrthoThreads, 0, s>>>(A, lda, na, B, ldb, nb, d, w.tpart);
    sum_parts_kernel<<<kTile * kTile / 256, 256, 0, s>>>(w.tpart, w.nparts, kTile * kTile, C);
    MLT_CUDA_TRY(cudaGetLastError());
    return MLT_OK;
}

// Upper Cholesky factor of the s x s Gram matrix W (row stride kTile), then its
// inverse into Rinv (same layout).  False when W is not numerically positive
// definite: a pivot at most 1e-13 of its diagonal entry (the columns are close
// to dependent, beyond what two Cholesky QR passes restore).
bool cholesky_inverse(const std::vector<double>& W, int s, std::vector<double>& Rinv)
{
    std::vector<double> R((size_t)kTile * kTile, 0.0);
    for (int i = 0; i < s; ++i) {
        double piv = W[(size_t)i * kTile + i];
        for (int k = 0; k < i; ++k) piv -= R[(size_t)k * kTile + i] * R[(size_t)k * kTile + i];
        if (!(piv > 1e-13 * W[(size_t)i * kTile + i])) return false;
        const double rii = std::sqrt(piv);
        R[(size_t)i * kTile + i] = rii;
        for (int j = i + 1; j < s; ++j) {
            double v = W[(size_t)i * kTile + j];
            for (int k = 0; k < i; ++k) v -= R[(size_t)k * kTile + i] * R[(size_t)k * kTile + j];
            R[(size_t)i * kTile + j] = v / rii;
        }
    }
    Rinv.assign((size_t)kTile * kTile, 0.0);
    for (int j = 0; j < s; ++j) {   // column j of R^{-1} by back substitution
        Rinv[(size_t)j * kTile + j] = 1.0 / R[(size_t)j * kTile + j];
        for (int i = j - 1; i >= 0; --i) {
            double v = 0.0;
            for (int k = i + 1; k <= j; ++k) v += R[(size_t)i * kTile + k] * Rinv[(size_t)k * kTile + j];
            Rinv[(size_t)i * kTile + j] = -v / R[(size_t)i * kTile + i];
        }
    }
    return true;
}

// Cholesky QR, twice, of the s <= kTile columns of Y in place: W = Y^T Y =
// R^T R, Y <- Y R^{-1}.  *ok stays false when a factorisation breaks down (Y
// then still spans the sketch's range); the caller then uses Gram-Schmidt.
int cholqr2(const OrthoScratch& w, double* Y, int ld, int s_cols, int64_t d, bool* ok, cudaStream_t s)
{
    ProfScope ps("hutchpp_orthonormalize", s);
    *ok = false;
    std::vector<double> W((size_t)kTile * kTile), Rinv;
    int rc;
    for (int pass = 0; pass < 2; ++pass) {
        if ((rc = tile_gram(w, Y, ld, s_cols, Y, ld, s_cols, d, w.tc, s))) return rc;
        MLT_CUDA_TRY(cudaMemcpyAsync(W.data(), w.tc, W.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        MLT_CUDA_TRY(cudaStreamSynchronize(s));
        if (!cholesky_inverse(W, s_cols, Rinv)) return MLT_OK;   // Y still spans the same space
        MLT_CUDA_TRY(cudaMemcpyAsync(w.tc, Rinv.data(), Rinv.size() * sizeof(double), cudaMemcpyHostToDevice, s));
        tile_update_kernel<<<w.nparts, kOrthoThreads, 0, s>>>(Y, ld, s_cols, w.tc, Y, ld, s_cols, d, 1);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    MLT_CUDA_TRY(cudaStreamSynchronize(s));   // Rinv's host buffer goes out of scope
    *ok = true;
    return MLT_OK;
}

// G <- (I - Q Q^T) G for the s columns of Q (orthonormal, or zero where
// dropped) and the g columns of G, 64 at a time: all of C = Q^T G_j first,
// then G_j -= Q C.
int deflate_blocked(const OrthoScratch& w, const double* Q, int ldq, int s_cols, double* G, int ldg, int g_cols,
                    int64_t d, cudaStream_t s)
{
    ProfScope ps("hutchpp_deflate", s);
    int rc;
    const int ti = (s_cols + kTile - 1) / kTile;
    for (int j0 = 0; j0 < g_cols; j0 += kTile) {
        const int nx = std::min(kTile, g_cols - j0);
        for (int it = 0; it < ti; ++it) {
            const int nq = std::min(kTile, s_cols - it * kTile);
            if ((rc = tile_gram(w, Q + it * kTile, ldq, nq, G + j0, ldg, nx, d, w.tc + (size_t)it * kTile * kTile,
                                s)))
                return rc;
        }
        for (int it = 0; it < ti; ++it) {
            const int nq = std::min(kTile, s_cols - it * kTile);
            tile_update_kernel<<<w.nparts, kOrthoThreads, 0, s>>>(Q + it * kTile, ldq, nq,
                                                                 w.tc + (size_t)it * kTile * kTile, G + j0, ldg, nx,
                                                                 d, 0);
        }
        MLT_CUDA_TRY(cudaGetLastError());
    }
    return MLT_OK;
}

int check_poly_args(mlt_matrix* m, double a, double b, const double* c, int n, const char* who)
{
    if (!m) return fail(MLT_EINVAL, std::string(who) + ": null matrix");
    if (int rcb = handle_busy(m, who)) return rcb;
    if (!c) return fail(MLT_EINVAL, std::string(who) + ": null coefficients");
    if (n < 1 || n > MLT_MAX_DEGREE) return fail(MLT_EINVAL, std::string(who) + ": n out of range");
    if (!(a < b) || !std::isfinite(a) || !std::isfinite(b))
        return fail(MLT_EINVAL, std::string(who) + ": need finite a < b");
    if (!m->A.val64 && m->val_type != MLT_PATTERN) return fail(MLT_EINVAL, std::string(who) + ": no FP64 values");
    return MLT_OK;
}

int64_t op_dim(const mlt_matrix* m)
{
    return (m->flags & MLT_GRAM) ? m->A.ncols : m->A.nrows;
}

int alloc_scratch(mlt_matrix* M, int64_t d, OrthoScratch& w, cudaStream_t s)
{
    w.nparts = ortho_grid(M, d);
    const size_t tiles = (size_t)w.nparts * kTile * kTile + (size_t)(kMaxSketch / kTile) * kTile * kTile;
    const size_t bytes = (tiles + (size_t)w.nparts * kMaxCols + 2 * kMaxCols + 8 + kMaxRemainder) * sizeof(double) +
                         kMaxSketch * sizeof(int);
    int rc;
    if ((rc = M->ws_misc.ensure(bytes, s))) return rc;
    double* p = M->ws_misc.as<double>();
    w.tpart = p;
    w.tc = p + (size_t)w.nparts * kTile * kTile;
    p += tiles;
    w.part = p;
    w.r = p + (size_t)w.nparts * kMaxCols;
    w.r2 = w.r + kMaxCols + 1;
    w.nrm2 = w.r2 + kMaxCols;
    w.norms = w.nrm2 + 7;
    w.kept = reinterpret_cast<int*>(w.norms + kMaxRemainder);
    return MLT_OK;
}

}  // namespace
}  // namespace mlt

using namespace mlt;

int mlt_poly_apply(mlt_matrix* m, double a, double b, const double* c, int n, const double* X, int64_t ldx,
                   double* Y, int64_t ldy, int ncols, unsigned flags, void* stream)
{
    try {
        int rc;
        if ((rc = check_poly_args(m, a, b, c, n, "mlt_poly_apply"))) return rc;
        if (!X || !Y) return fail(MLT_EINVAL, "mlt_poly_apply: null block");
        if (ncols < 1 || ncols > 4096) return fail(MLT_EINVAL, "mlt_poly_apply: ncols must be in [1, 4096]");
        if (ldx < ncols || ldy < ncols) return fail(MLT_EINVAL, "mlt_poly_apply: row strides must be >= ncols");
        if (flags & ~MLT_DEVICE_PTRS) return fail(MLT_EINVAL, "mlt_poly_apply: unknown flags");
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t d = op_dim(m);
        const int ld = (ncols + 1) & ~1;
        const size_t bytes = (size_t)std::max<int64_t>(d, 1) * ld * sizeof(double);
        for (int i = 0; i < 3; ++i)
            if ((rc = m->ws_blk[i].ensure(bytes, s))) return rc;
        double* Xb = m->ws_blk[0].as<double>();
        double* P[2] = {m->ws_blk[1].as<double>(), m->ws_blk[2].as<double>()};
        const cudaMemcpyKind in = (flags & MLT_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        const cudaMemcpyKind outk = (flags & MLT_DEVICE_PTRS) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        if (d > 0) {
            MLT_CUDA_TRY(cudaMemsetAsync(Xb, 0, bytes, s));
            MLT_CUDA_TRY(cudaMemcpy2DAsync(Xb, ld * sizeof(double), X, ldx * sizeof(double), ncols * sizeof(double),
                                           d, in, s));
            double* res = P[(n + 1) & 1];
            if ((rc = poly_apply_block(m, a, b, c, n, Xb, res, ld, ncols, P[0], P[1], s))) return rc;
            MLT_CUDA_TRY(cudaMemcpy2DAsync(Y, ldy * sizeof(double), res, ld * sizeof(double), ncols * sizeof(double),
                                           d, outk, s));
        }
        MLT_CUDA_TRY(cudaStreamSynchronize(s));
        return MLT_OK;
    } catch (const std::bad_alloc&) {
        return fail(MLT_ENOMEM, "mlt_poly_apply: host allocation failed");
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_poly_apply: exception");
    }
}

int mlt_hutchpp_estimate(mlt_matrix* m, double a, double b, const double* c, int n, uint64_t seed,
                         int64_t probe_offset, int s_cols, int g_cols, int precision, double* samples,
                         mlt_hutchpp_result* out, void* stream)
{
    try {
        int rc;
        if ((rc = check_poly_args(m, a, b, c, n, "mlt_hutchpp_estimate"))) return rc;
        if (!out) return fail(MLT_EINVAL, "mlt_hutchpp_estimate: null result");
        if (s_cols < 0 || s_cols > kMaxSketch) return fail(MLT_EINVAL, "mlt_hutchpp_estimate: s must be in [0, 128]");
        if (g_cols < 0 || g_cols > kMaxRemainder)
            return fail(MLT_EINVAL, "mlt_hutchpp_estimate: g must be in [0, 1024]");
        if (s_cols + g_cols < 1) return fail(MLT_EINVAL, "mlt_hutchpp_estimate: s + g must be at least 1");
        if (probe_offset < 0 || probe_offset + s_cols + g_cols > (int64_t)1 << 32)
            return fail(MLT_EINVAL, "mlt_hutchpp_estimate: probe ids must lie in [0, 2^32)");
        if (precision != MLT_PREC_FP64 && precision != MLT_PREC_FP32 && precision != MLT_PREC_DF64)
            return fail(MLT_EINVAL, "mlt_hutchpp_estimate: precision must be MLT_PREC_FP64, _FP32 or _DF64");
        const bool f32 = precision != MLT_PREC_FP64;   // the sketch in FP32
        const bool dfm = precision == MLT_PREC_DF64;   // the moments in double-float pairs
        cudaStream_t s = (cudaStream_t)stream;
        const int64_t d = op_dim(m);
        if (d < 1) return fail(MLT_EINVAL, "mlt_hutchpp_estimate: empty operator");
        // row strides: even for FP64 pairs, a multiple of 4 when the sketch runs in FP32
        const int ls = f32 ? std::max(4, (s_cols + 3) & ~3) : std::max(2, (s_cols + 1) & ~1);
        const int lg = std::max(2, (g_cols + 1) & ~1);
        const size_t dd = (size_t)d;
        // blk[0]: S, later the moments' scratch; blk[1], blk[2]: Clenshaw pair (Q ends in one); blk[3]: G.
        // FP32 sketch: S and one Clenshaw buffer share blk[0], the other is blk[1]; Q is blk[2].
        if ((rc = m->ws_blk[0].ensure(dd * std::max(ls, lg) * sizeof(double), s))) return rc;
        if ((rc = m->ws_blk[1].ensure(dd * ls * sizeof(double), s))) return rc;
        if ((rc = m->ws_blk[2].ensure(dd * ls * sizeof(double), s))) return rc;
        if ((rc = m->ws_blk[3].ensure(dd * lg * sizeof(double), s))) return rc;
        OrthoScratch w;
        if ((rc = alloc_scratch(m, d, w, s))) return rc;
        double* Sb = m->ws_blk[0].as<double>();
        double* P[2] = {m->ws_blk[1].as<double>(), m->ws_blk[2].as<double>()};
        double* Gb = m->ws_blk[3].as<double>();
        double* Q = f32 ? P[1] : P[(n + 1) & 1];
        float* S32 = reinterpret_cast<float*>(Sb);
        float* P32[2] = {S32 + dd * ls, reinterpret_cast<float*>(P[0])};
        const uint64_t seedmix = seed * kGolden;
        const int nbk = (int)std::max<int64_t>(1, std::min<int64_t>((d * 2 + 255) / 256, 16LL * m->num_sms));
        {
            ProfScope ps("hutchpp_probes", s);
            if (f32) rademacher_block_kernel<float><<<nbk, 256, 0, s>>>(S32, d, ls, s_cols, seedmix, probe_offset);
            else rademacher_block_kernel<double><<<nbk, 256, 0, s>>>(Sb, d, ls, s_cols, seedmix, probe_offset);
            rademacher_block_kernel<double><<<nbk, 256, 0, s>>>(Gb, d, lg, g_cols, seedmix, probe_offset + s_cols);
        }
        MLT_CUDA_TRY(cudaGetLastError());
        int rank = 0;
        if (s_cols > 0) {
            if (f32) {
                float* Y32 = P32[(n + 1) & 1];
                if ((rc = poly_apply_block_f32(m, a, b, c, n, S32, Y32, ls, s_cols, P32[0], P32[1], s))) return rc;
                ProfScope ps("hutchpp_widen", s);
                widen_block_kernel<<<nbk, 256, 0, s>>>(Y32, Q, (int64_t)dd * ls);
                MLT_CUDA_TRY(cudaGetLastError());
            } else if ((rc = poly_apply_block(m, a, b, c, n, Sb, Q, ls, s_cols, P[0], P[1], s))) {
                return rc;
            }
            // Q: Cholesky QR twice when the sketch fits one tile and is well conditioned,
            // else Gram-Schmidt (which also drops dependent columns)
            bool done = false;
            if (s_cols <= kTile && (rc = cholqr2(w, Q, ls, s_cols, d, &done, s))) return rc;
            std::vector<int> kept(s_cols, 1);
            if (!done) {
                if ((rc = orthonormalize(w, Q, ls, s_cols, d, s))) return rc;
                MLT_CUDA_TRY(cudaMemcpyAsync(kept.data(), w.kept, s_cols * sizeof(int), cudaMemcpyDeviceToHost, s));
            }
            // G' = (I - QQ^T) G: one block projection against the orthonormal Q
            if ((rc = deflate_blocked(w, Q, ls, s_cols, Gb, lg, g_cols, d, s))) return rc;
            MLT_CUDA_TRY(cudaStreamSynchronize(s));
            for (int k : kept) rank += k;
        }
        std::vector<double> tq, tg;
        if ((rc = quad_forms(m, w, a, b, c, n, Q, Sb, ls, s_cols, d, dfm, tq, s))) return rc;
        if ((rc = quad_forms(m, w, a, b, c, n, Gb, Sb, lg, g_cols, d, dfm, tg, s))) return rc;
        double t1 = 0.0, t2 = 0.0;
        for (double v : tq) t1 += v;
        for (double v : tg) t2 += v;
        t2 = g_cols > 0 ? t2 / g_cols : 0.0;
        double var = std::numeric_limits<double>::quiet_NaN();
        if (g_cols > 1) {
            double ss = 0.0;
            for (double v : tg) ss += (v - t2) * (v - t2);
            var = ss / (g_cols - 1);
        }
        if (samples)
            for (int i = 0; i < g_cols; ++i) samples[i] = tg[i];
        out->estimate = t1 + t2;
        out->std_error = g_cols > 1 ? std::sqrt(var / g_cols) : std::numeric_limits<double>::quiet_NaN();
        out->t_sketch = t1;
        out->t_rest = t2;
        out->rank = rank;
        out->matvecs = (int64_t)s_cols * n + (int64_t)(s_cols + g_cols) * ((n + 1) / 2);
        return MLT_OK;
    } catch (const std::bad_alloc&) {
        return fail(MLT_ENOMEM, "mlt_hutchpp_estimate: host allocation failed");
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_hutchpp_estimate: exception");
    }
}
