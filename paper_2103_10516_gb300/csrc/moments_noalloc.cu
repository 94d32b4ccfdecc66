// Chebyshev moments without any device allocation.
//
// Some callers cannot call cudaMalloc: code that runs inside a stream capture
// it does not own (an allocation there is illegal or breaks the capture), loops
// with latency limits that cannot absorb the device-wide synchronisation an
// allocation may cause, and hosts whose memory pool has already claimed the
// device memory.  mlt_moments_noalloc serves them: it computes what
// mlt_moments computes (FP64, doubling identities) for a device CSR matrix the
// caller owns, writing into a device array the caller owns, and keeps all of
// its working memory in one fixed array below.
//
// That array is a file-scope __device__ variable of kScratchBytes (32 MiB).
// Every GPU that loads the library holds it until the process exits.  All
// calls share it and it keeps the last call's contents, so calls that overlap
// on the GPU (different streams, or another host thread) race; callers must
// order them (a captured graph that holds a call races the same way with any
// other call while it replays).  In host code the array's name is only a
// host-side stand-in, so the device address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the first
// call there.  That lookup is not a stream operation and may load the module,
// so make the first call on each device before any stream capture: a call
// made during capture on a device not yet looked up fails with MLT_EINVAL.
//
// Inside a capture the call issues only capturable work: the per-probe tables
// travel by value as a kernel parameter (no host-to-device copy of host
// memory), the CSR range check runs on the device and sets a flag in the
// array that makes every later kernel of the call skip its work and the
// output rows NaN (a host cannot read it back before the graph runs), and the
// call does not synchronise.  Outside a capture the flag is read back and
// bad input fails with MLT_EINVAL, and the call returns after mu is written.
//
// The kernels are simpler than the main engine's (warp groups walk rows in
// grid-stride order, no splitting of long rows), which suits the small
// problems that fit in the fixed array.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <mutex>

#include "mlt_internal.h"
#include "rng.cuh"

namespace mlt {
namespace {

constexpr size_t kScratchBytes = (size_t)32 << 20;              // 32 MiB
constexpr int64_t kScratchDoubles = (int64_t)(kScratchBytes / sizeof(double));
constexpr int kMaxProbes = 512;
constexpr int kThreadsNa = 256;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_scratch[kScratchDoubles];

std::mutex g_na_mu;
double* g_na_ptr[kMaxDevices] = {};

// Probe tables, passed by value (3 KB of kernel parameters): probe slot c
// (degree-descending order) holds caller row row[c] and degree deg[c].
struct NaProbes {
    int32_t deg[kMaxProbes];
    int16_t row[kMaxProbes];
};

// bad |= 1 if some rowptr step leaves [0, nnz] or goes down, 2 if a column is
// outside [0, d): checked before any kernel indexes with the caller's arrays.
__global__ void na_check_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t d,
                                int64_t nnz, int* bad)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d; r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t a = rowptr[r], b = rowptr[r + 1];
        if (a < 0 || b < a || b > nnz) atomicOr(bad, 1);
    }
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz; k += (int64_t)gridDim.x * blockDim.x)
        if (col[k] < 0 || col[k] >= d) atomicOr(bad, 2);
}

// V_0 = z (probe signs) for the first B columns, zero padding after.
__global__ void na_init_kernel(double* v0, int64_t d, int ldv, int B, int64_t probe_offset, const NaProbes pr,
                               uint64_t seedmix, const int* __restrict__ bad)
{
    if (*bad) return;
    const int64_t total = d * (int64_t)ldv;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ldv;
        const int c = (int)(e % ldv);
        v0[e] = c < B ? (probe_negative(seedmix, (uint64_t)(probe_offset + pr.row[c]), (uint64_t)i) ? -1.0 : 1.0)
                      : 0.0;
    }
}

// One recurrence step for the first `act` columns: a warp per row, lane l
// holding columns l, l + 32, ... (act / 32 rounded up passes, at most
// kMaxPasses), so each row's bounds and entries are read once per step.
// out = first ? alpha A v + beta v : 2 (alpha A v + beta v) - prev, with
// per-CTA partial dots out.out and out.cur written in a fixed order: each
// lane sums its rows in row order, then the CTA sums its warps in warp order.
constexpr int kMaxPasses = kMaxProbes / 32;
__global__ void __launch_bounds__(kThreadsNa) na_step_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const double* __restrict__ val,
    int64_t d, int ldv, int act, const double* __restrict__ cur, double* prev_out, double alpha, double beta,
    int first, double* __restrict__ partials, const int* __restrict__ bad)
{
    if (*bad) return;  // uniform across the grid: no CTA reaches a barrier
    __shared__ double red[2][kThreadsNa / 32][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t gw = (int64_t)blockIdx.x * (kThreadsNa / 32) + warp;
    const int64_t nw = (int64_t)gridDim.x * (kThreadsNa / 32);
    const int passes = (act + 31) / 32;
    double s_self[kMaxPasses], s_cross[kMaxPasses];
#pragma unroll
    for (int ps = 0; ps < kMaxPasses; ++ps) s_self[ps] = s_cross[ps] = 0.0;
    for (int64_t r = gw; r < d; r += nw) {
        const int64_t k0 = rowptr[r], k1 = rowptr[r + 1];
        double acc[kMaxPasses];
#pragma unroll
        for (int ps = 0; ps < kMaxPasses; ++ps) acc[ps] = 0.0;
        for (int64_t k = k0; k < k1; ++k) {
            const double a = val ? val[k] : 1.0;
            const double* row = cur + (size_t)col[k] * ldv;
#pragma unroll
            for (int ps = 0; ps < kMaxPasses; ++ps) {
                const int c = ps * 32 + lane;
                if (ps < passes && c < act) acc[ps] = fma(a, row[c], acc[ps]);
            }
        }
#pragma unroll
        for (int ps = 0; ps < kMaxPasses; ++ps) {
            const int c = ps * 32 + lane;
            if (ps < passes && c < act) {
                const size_t off = (size_t)r * ldv + c;
                const double xc = cur[off];
                const double o = first ? alpha * acc[ps] + beta * xc : 2.0 * (alpha * acc[ps] + beta * xc) - prev_out[off];
                prev_out[off] = o;
                s_self[ps] = fma(o, o, s_self[ps]);
                s_cross[ps] = fma(o, xc, s_cross[ps]);
            }
        }
    }
#pragma unroll
    for (int ps = 0; ps < kMaxPasses; ++ps) {
        if (ps >= passes) break;   // uniform: passes is a kernel argument
        const int c = ps * 32 + lane;
        red[0][warp][lane] = s_self[ps];
        red[1][warp][lane] = s_cross[ps];
        __syncthreads();
        if (warp == 0) {
            double a0 = 0.0, a1 = 0.0;
            for (int w = 0; w < kThreadsNa / 32; ++w) {
                a0 += red[0][w][lane];
                a1 += red[1][w][lane];
            }
            if (c < act) {
                partials[(size_t)blockIdx.x * 2 * ldv + c] = a0;
                partials[(size_t)blockIdx.x * 2 * ldv + ldv + c] = a1;
            }
        }
        __syncthreads();
    }
}

// dots[step][kind][c] = sum over CTAs, in CTA order.
__global__ void na_reduce_kernel(const double* __restrict__ partials, int nblk, int ldv, int act, int step,
                                 double* __restrict__ dots, int B, const int* __restrict__ bad)
{
    if (*bad) return;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * act) return;
    const int kind = idx / act, c = idx % act;
    double s = 0.0;
    for (int b = 0; b < nblk; ++b) s += partials[(size_t)b * 2 * ldv + (size_t)kind * ldv + c];
    dots[(size_t)step * 2 * B + (size_t)kind * B + c] = s;
}

// mu rows from the dots (doubling identities), entries past a probe's degree
// 0; every entry NaN when the range check failed.
__global__ void na_finalize_kernel(const double* __restrict__ dots, int B, const NaProbes pr, double* mu, int64_t ld,
                                   double d, const int* __restrict__ bad)
{
    const int c = blockIdx.y;
    const int dg = pr.deg[c];
    const bool failed = *bad != 0;
    const double x0 = dg >= 1 && !failed ? dots[B + c] : 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ld; j += (int64_t)gridDim.x * blockDim.x) {
        double v;
        if (failed) v = __longlong_as_double(0x7ff8000000000000LL);
        else if (j > dg) v = 0.0;
        else if (j == 0) v = d;
        else if (j == 1) v = x0;
        else if ((j & 1) == 0) v = 2.0 * dots[(size_t)(j / 2 - 1) * 2 * B + c] - d;
        else v = 2.0 * dots[(size_t)((j - 1) / 2) * 2 * B + B + c] - x0;
        mu[(int64_t)pr.row[c] * ld + j] = v;
    }
}

}  // namespace
}  // namespace mlt

using namespace mlt;

extern "C" int mlt_moments_noalloc(int64_t d, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                                   const double* vals, double scale, double a, double b, uint64_t seed,
                                   int64_t probe_offset, int nprobes, const int32_t* degree, double* mu,
                                   int64_t ld_mu, void* stream)
{
    if (d < 1 || nnz < 0 || !rowptr || (nnz > 0 && !col)) return fail(MLT_EINVAL, "mlt_moments_noalloc: bad matrix");
    if (!(a < b) || !std::isfinite(a) || !std::isfinite(b) || !std::isfinite(scale))
        return fail(MLT_EINVAL, "mlt_moments_noalloc: need finite a < b and scale");
    if (nprobes < 0 || nprobes > kMaxProbes)
        return fail(MLT_EINVAL, "mlt_moments_noalloc: nprobes must be 0..512");
    if (nprobes == 0) return MLT_OK;
    if (!degree || !mu) return fail(MLT_EINVAL, "mlt_moments_noalloc: null degree or mu");
    if (probe_offset < 0 || probe_offset + nprobes > (1LL << 32))
        return fail(MLT_EINVAL, "mlt_moments_noalloc: probe ids must lie in [0, 2^32)");
    // probe order by degree, descending (stable insertion sort in fixed arrays)
    NaProbes pr;
    int32_t* degs = pr.deg;
    int16_t* rows = pr.row;
    int maxdeg = 0;
    for (int p = 0; p < nprobes; ++p) {
        if (degree[p] < 0 || degree[p] > MLT_MAX_DEGREE) return fail(MLT_EINVAL, "mlt_moments_noalloc: degree out of range");
        maxdeg = std::max(maxdeg, (int)degree[p]);
        int q = p;
        while (q > 0 && degs[q - 1] < degree[p]) {
            degs[q] = degs[q - 1];
            rows[q] = rows[q - 1];
            --q;
        }
        degs[q] = degree[p];
        rows[q] = (int16_t)p;
    }
    if (ld_mu < maxdeg + 1) return fail(MLT_EINVAL, "mlt_moments_noalloc: ld_mu below max degree + 1");
    const int B = nprobes;
    const int ldv = (B + 31) & ~31;
    const int K = (maxdeg + 1) / 2;
    int dev = 0;
    MLT_CUDA_TRY(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices) return fail(MLT_EINVAL, "mlt_moments_noalloc: device index too large");
    int num_sms = 0;
    MLT_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
    // the two vector blocks alone must fit before anything is sized from d
    if (d > kScratchDoubles / (2 * (int64_t)ldv))
        return fail(MLT_ERANGE, "mlt_moments_noalloc: d * round_up(nprobes, 32) too large for the 32 MiB scratch "
                                "array (need 2 d ldv + partials + dots <= 4,194,304 doubles)");
    const int nblk = (int)std::max<int64_t>(1, std::min<int64_t>((d + 7) / 8, 2 * (int64_t)num_sms));
    // layout inside the fixed array (in doubles): V0, V1, partials, dots, metadata
    const int64_t n_v = d * (int64_t)ldv;
    const int64_t n_part = (int64_t)nblk * 2 * ldv;
    const int64_t n_dots = (int64_t)std::max(K, 1) * 2 * B;
    const int64_t n_meta = 8;
    if (2 * n_v + n_part + n_dots + n_meta > kScratchDoubles)
        return fail(MLT_ERANGE, "mlt_moments_noalloc: d * round_up(nprobes, 32) too large for the 32 MiB scratch "
                                "array (need 2 d ldv + partials + dots <= 4,194,304 doubles)");
    cudaStream_t s = (cudaStream_t)stream;
    cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
    MLT_CUDA_TRY(cudaStreamIsCapturing(s, &cap));
    const bool capturing = cap != cudaStreamCaptureStatusNone;
    double* base = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_na_mu);
        if (!g_na_ptr[dev] && capturing)
            return fail(MLT_EINVAL, "mlt_moments_noalloc: first call on a device must come before stream capture");
        if (!g_na_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
            if (e != cudaSuccess || !p) return cuda_fail(e != cudaSuccess ? e : cudaErrorInvalidSymbol, "cudaGetSymbolAddress");
            g_na_ptr[dev] = static_cast<double*>(p);
        }
        base = g_na_ptr[dev];
    }
    double* V[2] = {base, base + n_v};
    double* part = base + 2 * n_v;
    double* dots = part + n_part;
    int* bad = reinterpret_cast<int*>(dots + n_dots);  // cleared at the start of every call
    {
        MLT_CUDA_TRY(cudaMemsetAsync(bad, 0, sizeof(int), s));
        const int g = (int)std::min<int64_t>((std::max(d, nnz) + 255) / 256, 16LL * num_sms);
        na_check_kernel<<<std::max(g, 1), 256, 0, s>>>(rowptr, col, d, nnz, bad);
        MLT_CUDA_TRY(cudaGetLastError());
        if (!capturing) {
            int hbad = 0;
            MLT_CUDA_TRY(cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s));
            MLT_CUDA_TRY(cudaStreamSynchronize(s));
            if (hbad) return fail(MLT_EINVAL, "mlt_moments_noalloc: rowptr or column index out of range");
        }
    }
    const uint64_t seedmix = seed * kGolden;
    {
        const int g = (int)std::min<int64_t>((n_v + 255) / 256, 16LL * num_sms);
        na_init_kernel<<<std::max(g, 1), 256, 0, s>>>(V[0], d, ldv, B, probe_offset, pr, seedmix, bad);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    const double alpha = 2.0 / (b - a) * scale;
    const double beta = -(a + b) / (b - a);
    for (int k = 0; k < K; ++k) {
        int act = 0;
        while (act < B && (degs[act] + 1) / 2 > k) ++act;
        na_step_kernel<<<nblk, kThreadsNa, 0, s>>>(rowptr, col, vals, d, ldv, act, V[k & 1], V[(k + 1) & 1], alpha,
                                                   beta, k == 0 ? 1 : 0, part, bad);
        na_reduce_kernel<<<(2 * act + 127) / 128, 128, 0, s>>>(part, nblk, ldv, act, k, dots, B, bad);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    {
        dim3 grid((unsigned)std::min<int64_t>((ld_mu + 127) / 128, 64), B);
        na_finalize_kernel<<<grid, 128, 0, s>>>(dots, B, pr, mu, ld_mu, (double)d, bad);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    if (!capturing) MLT_CUDA_TRY(cudaStreamSynchronize(s));
    return MLT_OK;
}
