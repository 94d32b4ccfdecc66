// Exact integer triangle moments (Section 2.1 Example; Section 5.4).
//
// For a block of 128 Rademacher probes and a symmetric 0/1 adjacency matrix A
// with no self-loops, per probe:
//   y  = A z                      (pass 1; |y_i| <= deg_i, int32)
//   x1 = z . y = z^T A z,  x2 = y . y = z^T A^2 z
//   x3 = y^T A y = z^T A^3 z = 2 sum_i y_i sum_{j in N(i), j > i} y_j   (pass 2)
// Pass 2 walks only the upper triangle: the quadratic form is symmetric, so the
// two products of the paper's footnote suffice and half the gathers are saved.
//
// Layout: probe signs are bit-packed, 4 words (128 bits) per row; y is int32,
// 128 per row (512 B), so a warp owns one row with 4 probes per lane.
// All sums are integers, accumulated with integer atomics: exact and
// independent of order.
#include <cuda_runtime.h>

#include <algorithm>

#include "mlt_internal.h"
#include "rng.cuh"

namespace mlt {
namespace {

constexpr int kTriThreads = 256;
constexpr int kProbes = 128;

// zb[i * 4 + w] bit t = 1 when z_i of probe (id0 + 32 w + t) is -1.
__global__ void zbits_kernel(int64_t d, uint64_t seedmix, int64_t id0, int nb, uint32_t* __restrict__ zb)
{
    const int64_t total = d * 4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e >> 2;
        const int w = (int)(e & 3);
        uint32_t bits = 0;
        for (int t = 0; t < 32; ++t) {
            const int p = w * 32 + t;
            if (p < nb && probe_negative(seedmix, (uint64_t)(id0 + p), (uint64_t)i)) bits |= 1u << t;
        }
        zb[e] = bits;
    }
}

// Per row: first index with col > row, self-loop detection and the bound
// sum_j deg_i deg_j used to certify that x3 fits in int64.
__global__ void tri_prepare_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                   int64_t d, int64_t* __restrict__ upper, double* bound, int* selfloop)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    double wsum = 0.0;
    for (int64_t r = warp; r < d; r += nwarps) {
        const int64_t beg = rowptr[r], end = rowptr[r + 1];
        int64_t first = end;
        double dsum = 0.0;
        for (int64_t base = beg; base < end; base += 32) {
            const int64_t k = base + lane;
            int c = -1;
            if (k < end) {
                c = col[k];
                dsum += (double)(rowptr[c + 1] - rowptr[c]);
                if (c == r) atomicOr(selfloop, 1);
            }
            const unsigned above = __ballot_sync(0xFFFFFFFFu, k < end && c > r);
            if (above && first == end) first = base + __ffs(above) - 1;
        }
        for (int o = 16; o; o >>= 1) dsum += __shfl_xor_sync(0xFFFFFFFFu, dsum, o);
        if (lane == 0) {
            upper[r] = first;
            wsum += dsum * (double)(end - beg);
        }
    }
    if (lane == 0 && wsum != 0.0) atomicAdd(bound, wsum);
}

// Pass 1: y = A z for 128 probes, plus x1 = z.y and x2 = y.y.
__global__ void __launch_bounds__(kTriThreads) tri_pass1_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t d,
    const uint32_t* __restrict__ zb, int32_t* __restrict__ y, unsigned long long* __restrict__ xacc)
{
    __shared__ long long sx[2][kProbes];
    for (int t = threadIdx.x; t < 2 * kProbes; t += blockDim.x) (&sx[0][0])[t] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    const int wl = lane >> 3;              // word holding this lane's 4 probes
    const int sh = (lane & 7) * 4;         // bit offset of probe 4*lane
    long long x1[4] = {0, 0, 0, 0}, x2[4] = {0, 0, 0, 0};
    for (int64_t r = warp; r < d; r += nwarps) {
        const int64_t beg = rowptr[r], end = rowptr[r + 1];
        int cnt[4] = {0, 0, 0, 0};
        for (int64_t base = beg; base < end; base += 32) {
            const int64_t k = base + lane;
            const int cj = k < end ? __ldg(col + k) : 0;
            const int n = (int)min((int64_t)32, end - base);
#pragma unroll 4
            for (int t = 0; t < n; ++t) {
                const int j = __shfl_sync(0xFFFFFFFFu, cj, t);
                const uint32_t nib = (__ldg(zb + (size_t)j * 4 + wl) >> sh) & 0xFu;
                cnt[0] += nib & 1u;
                cnt[1] += (nib >> 1) & 1u;
                cnt[2] += (nib >> 2) & 1u;
                cnt[3] += (nib >> 3) & 1u;
            }
        }
        const int deg = (int)(end - beg);
        const uint32_t own = (__ldg(zb + (size_t)r * 4 + wl) >> sh) & 0xFu;
        int4 yv;
        yv.x = deg - 2 * cnt[0];
        yv.y = deg - 2 * cnt[1];
        yv.z = deg - 2 * cnt[2];
        yv.w = deg - 2 * cnt[3];
        *reinterpret_cast<int4*>(y + (size_t)r * kProbes + 4 * lane) = yv;
        const int yy[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const long long yq = yy[q];
            x1[q] += ((own >> q) & 1u) ? -yq : yq;
            x2[q] += yq * yq;
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        atomicAdd((unsigned long long*)&sx[0][4 * lane + q], (unsigned long long)x1[q]);
        atomicAdd((unsigned long long*)&sx[1][4 * lane + q], (unsigned long long)x2[q]);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kProbes; t += blockDim.x) {
        atomicAdd(xacc + 3 * t + 0, (unsigned long long)sx[0][t]);
        atomicAdd(xacc + 3 * t + 1, (unsigned long long)sx[1][t]);
    }
}

// Pass 2: x3 = 2 sum_i y_i sum_{j in N(i), j > i} y_j.
__global__ void __launch_bounds__(kTriThreads) tri_pass2_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const int64_t* __restrict__ upper, int64_t d, const int32_t* __restrict__ y,
    unsigned long long* __restrict__ xacc)
{
    __shared__ long long sx[kProbes];
    for (int t = threadIdx.x; t < kProbes; t += blockDim.x) sx[t] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    long long x3[4] = {0, 0, 0, 0};
    for (int64_t r = warp; r < d; r += nwarps) {
        const int64_t beg = upper[r], end = rowptr[r + 1];
        if (beg >= end) continue;
        int s[4] = {0, 0, 0, 0};
        for (int64_t base = beg; base < end; base += 32) {
            const int64_t k = base + lane;
            const int cj = k < end ? __ldg(col + k) : 0;
            const int n = (int)min((int64_t)32, end - base);
#pragma unroll 4
            for (int t = 0; t < n; ++t) {
                const int j = __shfl_sync(0xFFFFFFFFu, cj, t);
                const int4 yj = __ldg(reinterpret_cast<const int4*>(y + (size_t)j * kProbes) + lane);
                s[0] += yj.x;
                s[1] += yj.y;
                s[2] += yj.z;
                s[3] += yj.w;
            }
        }
        const int4 yi = __ldg(reinterpret_cast<const int4*>(y + (size_t)r * kProbes) + lane);
        x3[0] += (long long)yi.x * s[0];
        x3[1] += (long long)yi.y * s[1];
        x3[2] += (long long)yi.z * s[2];
        x3[3] += (long long)yi.w * s[3];
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        atomicAdd((unsigned long long*)&sx[4 * lane + q], (unsigned long long)(2 * x3[q]));
    __syncthreads();
    for (int t = threadIdx.x; t < kProbes; t += blockDim.x)
        atomicAdd(xacc + 3 * t + 2, (unsigned long long)sx[t]);
}

int grid_for(int num_sms, int64_t warps_needed)
{
    const int64_t blocks = (warps_needed * 32 + kTriThreads - 1) / kTriThreads;
    return (int)std::max<int64_t>(1, std::min<int64_t>(blocks, 8LL * num_sms));
}

}  // namespace

int tri_prepare(mlt_matrix* M, cudaStream_t s)
{
    if (M->tri_state == 1) return MLT_OK;
    if (M->tri_state < 0) return fail(M->tri_state, "matrix is not a valid triangle-counting input");
    const int64_t d = M->A.nrows;
    int rc;
    if ((rc = M->ws_misc.ensure(64, s))) return rc;
    double* bound = M->ws_misc.as<double>();
    int* selfloop = reinterpret_cast<int*>(bound + 1);
    MLT_CUDA_TRY(cudaMemsetAsync(bound, 0, 16, s));
    int64_t* upper = nullptr;
    if (cudaMallocAsync((void**)&upper, (size_t)std::max<int64_t>(d, 1) * sizeof(int64_t), s) != cudaSuccess)
        return fail(MLT_ENOMEM, "cudaMallocAsync (triangle row split) failed");
    M->upper = upper;
    {
    ProfScope ps("tri_prepare", s);
    tri_prepare_kernel<<<grid_for(M->num_sms, d), kTriThreads, 0, s>>>(M->A.rowptr, M->A.col, d, upper,
                                                                      bound, selfloop);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    double hb = 0.0;
    int hs = 0;
    MLT_CUDA_TRY(cudaMemcpyAsync(&hb, bound, sizeof(double), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaMemcpyAsync(&hs, selfloop, sizeof(int), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaStreamSynchronize(s));
    M->tri_bound = hb;
    if (hs) {
        M->tri_state = MLT_EINVAL;
        return fail(MLT_EINVAL, "triangle counting needs an adjacency matrix without self-loops");
    }
    if (!(hb < 4611686018427387904.0)) {   // 2^62
        M->tri_state = MLT_ERANGE;
        return fail(MLT_ERANGE, "sum of deg_i*deg_j over edges reaches 2^62: x3 may overflow int64");
    }
    M->tri_state = 1;
    return MLT_OK;
}

int tri_block(mlt_matrix* M, uint64_t seed, int64_t id0, int nb, int64_t* x_dev, cudaStream_t s)
{
    const int64_t d = M->A.nrows;
    int rc;
    if ((rc = M->ws_z.ensure((size_t)std::max<int64_t>(d, 1) * 4 * sizeof(uint32_t), s))) return rc;
    if ((rc = M->ws_y.ensure((size_t)std::max<int64_t>(d, 1) * kProbes * sizeof(int32_t), s))) return rc;
    if ((rc = M->ws_x.ensure((size_t)kProbes * 3 * sizeof(unsigned long long), s))) return rc;
    uint32_t* zb = M->ws_z.as<uint32_t>();
    int32_t* y = M->ws_y.as<int32_t>();
    unsigned long long* xacc = M->ws_x.as<unsigned long long>();
    MLT_CUDA_TRY(cudaMemsetAsync(xacc, 0, (size_t)kProbes * 3 * sizeof(unsigned long long), s));
    {
        const int64_t total = d * 4;
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 16LL * M->num_sms));
        ProfScope ps("tri_zbits", s);
        zbits_kernel<<<g, 256, 0, s>>>(d, seed * kGolden, id0, nb, zb);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    const int g = grid_for(M->num_sms, d);
    {
        ProfScope ps("tri_pass1", s);
        tri_pass1_kernel<<<g, kTriThreads, 0, s>>>(M->A.rowptr, M->A.col, d, zb, y, xacc);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    {
        ProfScope ps("tri_pass2", s);
        tri_pass2_kernel<<<g, kTriThreads, 0, s>>>(M->A.rowptr, M->A.col, M->upper, d, y, xacc);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    MLT_CUDA_TRY(cudaMemcpyAsync(x_dev, xacc, (size_t)nb * 3 * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    return MLT_OK;
}

}  // namespace mlt
