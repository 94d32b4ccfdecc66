// Chebyshev moment engine: a block of Rademacher probes pushed through the
// three-term recurrence V_{k+1} = 2 At V_k - V_{k-1} (Section 2.2,
// Eq. recurrence), At = alpha A + beta I, with the per-probe dot products that
// give the moments fused into the same pass over the matrix.
//
// Data layout (device, row-major): V[i * ldv + c] is entry i of probe c, so a
// gathered row of V is ldv contiguous values and each probe's column is strided.
// Probes are sorted by degree, descending; at step k only the first act_k
// columns are live, so retired probes cost nothing.
//
// Doubling mode (the symmetric quadratic-form trick the paper cites in
// Section 2.2): with T_{2k} = 2 T_k^2 - 1 and T_{2k+1} = 2 T_{k+1} T_k - T_1,
//   mu_{2k+2} = 2 V_{k+1}.V_{k+1} - mu_0,   mu_{2k+1} = 2 V_{k+1}.V_k - mu_1,
// so degree n needs ceil(n/2) operator applications.  Direct mode keeps
// mu_{k+1} = z . V_{k+1} (n applications).
//
// Reductions are deterministic: each CTA writes per-column partial sums in a
// fixed order, and a separate kernel adds the CTA partials in CTA order.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "mlt_internal.h"
#include "rng.cuh"

namespace mlt {
namespace {

constexpr int kThreads = 256;
constexpr int kSlots = 16;          // steps whose partials are buffered before a reduction

template <typename T> struct Lanes;
template <> struct Lanes<double> { static constexpr int N = 2; };   // 16-byte vectors
template <> struct Lanes<float> { static constexpr int N = 4; };

template <typename T, int N> struct alignas(sizeof(T) * N) Pack { T v[N]; };

template <typename T>
struct StepArgs {
    const int64_t* rowptr;
    const int32_t* col;
    const T* val;          // null: pattern (all ones)
    int64_t nrows;         // rows handled by this launch
    int ldv;               // row stride of every vector buffer
    int nvec;              // live vectors per row: ceil(act / N)
    int nchunks;           // vector chunks of width G per row
    const T* vgather;      // gathered operand (V_k, or W = X V_k for a Gram step)
    const T* vcur;         // V_k at the row itself
    T* vprev_out;          // in: V_{k-1} (unless first); out: V_{k+1}
    T alpha, beta;         // At = alpha A + beta I
    int mode;              // 0 first step, 1 recurrence step, 2 plain product
    int direct;            // dots are z . V_{k+1} instead of V.V and V.V_k
    int B;                 // probes in the group (columns >= B are padding)
    uint64_t seedmix;
    const int64_t* ids;    // global id of each column's probe (direct mode)
    double* partials;      // [gridDim.x][2][ldv]
};

template <typename T, int G>
__global__ void __launch_bounds__(kThreads) cheb_step_kernel(StepArgs<T> a)
{
    constexpr int N = Lanes<T>::N;
    using P = Pack<T, N>;
    __shared__ double red[2][kThreads * N];

    const int tid = threadIdx.x;
    const int lane = tid & 31;
    const int glane = lane & (G - 1);
    const unsigned gmask = (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << (lane & ~(G - 1)));
    const int gpb = kThreads / G;
    const int gib = tid / G;
    const long long gg = (long long)blockIdx.x * gpb + gib;
    const long long total = (long long)gridDim.x * gpb;
    const long long rstride = total / a.nchunks;
    const int chunk = (int)(gg % a.nchunks);
    const int vidx = chunk * G + glane;
    const bool vok = vidx < a.nvec;
    const int c0 = vidx * N;

    double s_self[N], s_cross[N];
#pragma unroll
    for (int q = 0; q < N; ++q) { s_self[q] = 0.0; s_cross[q] = 0.0; }

    if (gg < rstride * a.nchunks) {
        for (long long r = gg / a.nchunks; r < a.nrows; r += rstride) {
            const int64_t beg = a.rowptr[r];
            const int64_t end = a.rowptr[r + 1];
            T acc[N];
#pragma unroll
            for (int q = 0; q < N; ++q) acc[q] = T(0);
            for (int64_t base = beg; base < end; base += G) {
                const int64_t k = base + glane;
                int cj = 0;
                T vj = T(0);
                if (k < end) {
                    cj = __ldg(a.col + k);
                    vj = a.val ? __ldg(a.val + k) : T(1);
                }
                const int cnt = (int)min((int64_t)G, end - base);
#pragma unroll 4
                for (int t = 0; t < cnt; ++t) {
                    const int c = __shfl_sync(gmask, cj, t, G);
                    const T v = __shfl_sync(gmask, vj, t, G);
                    if (vok) {
                        const P x = *reinterpret_cast<const P*>(a.vgather + (size_t)c * a.ldv + c0);
#pragma unroll
                        for (int q = 0; q < N; ++q) acc[q] = fma(v, x.v[q], acc[q]);
                    }
                }
            }
            if (!vok) continue;
            const size_t off = (size_t)r * a.ldv + c0;
            P out;
            if (a.mode == 2) {
#pragma unroll
                for (int q = 0; q < N; ++q) out.v[q] = acc[q];
                *reinterpret_cast<P*>(a.vprev_out + off) = out;
                continue;
            }
            const P xc = *reinterpret_cast<const P*>(a.vcur + off);
            if (a.mode == 0) {
#pragma unroll
                for (int q = 0; q < N; ++q) out.v[q] = a.alpha * acc[q] + a.beta * xc.v[q];
            } else {
                const P xp = *reinterpret_cast<const P*>(a.vprev_out + off);
#pragma unroll
                for (int q = 0; q < N; ++q)
                    out.v[q] = T(2) * (a.alpha * acc[q] + a.beta * xc.v[q]) - xp.v[q];
            }
            *reinterpret_cast<P*>(a.vprev_out + off) = out;
            if (!a.direct) {
#pragma unroll
                for (int q = 0; q < N; ++q) {
                    const double o = (double)out.v[q];
                    s_self[q] = fma(o, o, s_self[q]);
                    s_cross[q] = fma(o, (double)xc.v[q], s_cross[q]);
                }
            } else {
#pragma unroll
                for (int q = 0; q < N; ++q) {
                    if (c0 + q >= a.B) break;
                    const bool neg = probe_negative(a.seedmix, (uint64_t)a.ids[c0 + q], (uint64_t)r);
                    const double o = (double)out.v[q];
                    s_cross[q] += neg ? -o : o;
                }
            }
        }
    }
    if (a.mode == 2) return;

    // CTA reduction in a fixed order: column c collects the groups of this CTA
    // whose chunk holds it, in group order.
#pragma unroll
    for (int q = 0; q < N; ++q) {
        red[0][tid * N + q] = s_self[q];
        red[1][tid * N + q] = s_cross[q];
    }
    __syncthreads();
    const int ncols = a.nvec * N;
    double* part = a.partials + (size_t)blockIdx.x * 2 * a.ldv;
    const long long g0 = (long long)blockIdx.x * gpb;
    for (int c = tid; c < ncols; c += kThreads) {
        const int v = c / N, q = c % N;
        const int ch = v / G, gl = v % G;
        double s0 = 0.0, s1 = 0.0;
        for (int g = 0; g < gpb; ++g) {
            const long long gglob = g0 + g;
            if (gglob >= rstride * a.nchunks || (int)(gglob % a.nchunks) != ch) continue;
            const int t = g * G + gl;
            s0 += red[0][t * N + q];
            s1 += red[1][t * N + q];
        }
        part[c] = s0;
        part[a.ldv + c] = s1;
    }
}

struct ReduceArgs {
    int nslots;
    int step0;
    int nblocks[kSlots];
    int act[kSlots];
};

__global__ void reduce_partials_kernel(const double* __restrict__ part, int max_blocks, int ldv,
                                       ReduceArgs ra, double* __restrict__ dots, int B)
{
    const int slot = blockIdx.y;
    const int act = ra.act[slot];
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= 2 * act) return;
    const int kind = idx / act, c = idx % act;
    const double* p = part + (size_t)slot * max_blocks * 2 * ldv + (size_t)kind * ldv + c;
    double s = 0.0;
    const int nb = ra.nblocks[slot];
    for (int b = 0; b < nb; ++b) s += p[(size_t)b * 2 * ldv];
    dots[(size_t)(ra.step0 + slot) * 2 * B + (size_t)kind * B + c] = s;
}

template <typename T>
__global__ void init_probes_kernel(T* v0, int64_t d, int ldv, int B, const int64_t* __restrict__ ids,
                                   uint64_t seedmix)
{
    const int64_t total = d * (int64_t)ldv;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ldv;
        const int c = (int)(e % ldv);
        T z = T(0);
        if (c < B) z = probe_negative(seedmix, (uint64_t)ids[c], (uint64_t)i) ? T(-1) : T(1);
        v0[e] = z;
    }
}

__global__ void finalize_moments_kernel(const double* __restrict__ dots, int B,
                                        const int32_t* __restrict__ deg,
                                        const int64_t* __restrict__ row, double* mu, int64_t ld,
                                        double d, int direct, int* err)
{
    const int c = blockIdx.y;
    const int dg = deg[c];
    double* out = mu + row[c] * ld;
    const double x0 = dg >= 1 ? dots[B + c] : 0.0;
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < ld;
         j += (int64_t)gridDim.x * blockDim.x) {
        double v;
        if (j > dg) {
            v = 0.0;
        } else if (j == 0) {
            v = d;
        } else if (direct) {
            v = dots[(size_t)(j - 1) * 2 * B + B + c];
        } else if (j == 1) {
            v = x0;
        } else if ((j & 1) == 0) {
            v = 2.0 * dots[(size_t)(j / 2 - 1) * 2 * B + c] - d;
        } else {
            v = 2.0 * dots[(size_t)((j - 1) / 2) * 2 * B + B + c] - x0;
        }
        if (!(fabs(v) <= d * (1.0 + 1e-6))) atomicOr(err, 1);
        out[j] = v;
    }
}

__global__ void to_float_kernel(const double* __restrict__ in, float* __restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (float)in[i];
}

int pow2_at_least(int v)
{
    int g = 1;
    while (g < v && g < 32) g <<= 1;
    return g;
}

template <typename T, int G>
int launch_step_g(const StepArgs<T>& a, int max_blocks, int* nblocks_out, cudaStream_t s)
{
    const long long items = a.nrows * (long long)a.nchunks;
    const int gpb = kThreads / G;
    long long want = (items + gpb - 1) / gpb;
    int nb = (int)std::max<long long>(1, std::min<long long>(want, max_blocks));
    // every CTA must own at least one group per chunk so rstride > 0
    const long long min_groups = a.nchunks;
    if ((long long)nb * gpb < min_groups) nb = (int)((min_groups + gpb - 1) / gpb);
    {
        ProfScope ps(a.mode == 2 ? "gram_spmm" : "cheb_step", s);
        cheb_step_kernel<T, G><<<nb, kThreads, 0, s>>>(a);
    }
    *nblocks_out = nb;
    return cuda_fail(cudaGetLastError(), "cheb_step_kernel launch");
}

template <typename T>
int launch_step(int G, const StepArgs<T>& a, int max_blocks, int* nb, cudaStream_t s)
{
    switch (G) {
    case 1: return launch_step_g<T, 1>(a, max_blocks, nb, s);
    case 2: return launch_step_g<T, 2>(a, max_blocks, nb, s);
    case 4: return launch_step_g<T, 4>(a, max_blocks, nb, s);
    case 8: return launch_step_g<T, 8>(a, max_blocks, nb, s);
    case 16: return launch_step_g<T, 16>(a, max_blocks, nb, s);
    default: return launch_step_g<T, 32>(a, max_blocks, nb, s);
    }
}

template <typename T>
int run_group(mlt_matrix* M, const MomentPlan& plan, double a, double b, uint64_t seed,
              double* mu_dev, int64_t ld_mu, int* err_flag, cudaStream_t s)
{
    constexpr int N = Lanes<T>::N;
    const bool gram = (M->flags & MLT_GRAM) != 0;
    const int64_t d = plan.dim;
    const int ldv = plan.ldv;
    const size_t vbytes = (size_t)d * ldv * sizeof(T);
    int rc;
    if ((rc = M->ws_v[0].ensure(vbytes, s)) || (rc = M->ws_v[1].ensure(vbytes, s))) return rc;
    T* V[2] = {M->ws_v[0].as<T>(), M->ws_v[1].as<T>()};
    T* W = nullptr;
    if (gram) {
        if ((rc = M->ws_w.ensure((size_t)M->A.nrows * ldv * sizeof(T), s))) return rc;
        W = M->ws_w.as<T>();
    }
    const int max_blocks = 8 * M->num_sms;
    if ((rc = M->ws_part.ensure((size_t)kSlots * max_blocks * 2 * ldv * sizeof(double), s))) return rc;
    if ((rc = M->ws_dots.ensure((size_t)std::max(plan.K, 1) * 2 * plan.B * sizeof(double), s))) return rc;
    double* part = M->ws_part.as<double>();
    double* dots = M->ws_dots.as<double>();
    const uint64_t seedmix = seed * kGolden;

    {
        const int64_t total = d * (int64_t)ldv;
        const int nb = (int)std::min<int64_t>((total + 255) / 256, 16LL * M->num_sms);
        ProfScope ps("init_probes", s);
        init_probes_kernel<T><<<std::max(nb, 1), 256, 0, s>>>(V[0], d, ldv, plan.B, plan.ids_dev, seedmix);
        MLT_CUDA_TRY(cudaGetLastError());
    }

    // At = alpha A + beta I; the stored entries carry `scale` (squared for X^T X).
    const double sc = gram ? M->scale * M->scale : M->scale;
    const double alpha = 2.0 / (b - a) * sc;
    const double beta = -(a + b) / (b - a);

    const DevCSR& A = M->A;
    const DevCSR& AT = M->AT;
    const T* valA = std::is_same<T, double>::value ? (const T*)A.val64 : (const T*)A.val32;
    const T* valAT = std::is_same<T, double>::value ? (const T*)AT.val64 : (const T*)AT.val32;

    ReduceArgs ra{};
    ra.step0 = 0;
    ra.nslots = 0;
    for (int k = 0; k < plan.K; ++k) {
        const int act = plan.act[k];
        const int nvec = (act + N - 1) / N;
        const int G = pow2_at_least(std::min(nvec, 32));
        const int nchunks = (nvec + G - 1) / G;
        T* cur = V[k & 1];
        T* out = V[(k + 1) & 1];
        StepArgs<T> sa{};
        sa.ldv = ldv;
        sa.nvec = nvec;
        sa.nchunks = nchunks;
        sa.alpha = (T)alpha;
        sa.beta = (T)beta;
        sa.direct = plan.direct;
        sa.B = plan.B;
        sa.seedmix = seedmix;
        sa.ids = plan.ids_dev;
        int nb = 0;
        if (gram) {
            StepArgs<T> pa = sa;
            pa.rowptr = A.rowptr; pa.col = A.col; pa.val = valA; pa.nrows = A.nrows;
            pa.vgather = cur; pa.vcur = nullptr; pa.vprev_out = W; pa.mode = 2;
            pa.partials = nullptr;
            if ((rc = launch_step<T>(G, pa, max_blocks, &nb, s))) return rc;
            sa.rowptr = AT.rowptr; sa.col = AT.col; sa.val = valAT; sa.nrows = AT.nrows;
            sa.vgather = W;
        } else {
            sa.rowptr = A.rowptr; sa.col = A.col; sa.val = valA; sa.nrows = A.nrows;
            sa.vgather = cur;
        }
        sa.vcur = cur;
        sa.vprev_out = out;
        sa.mode = (k == 0) ? 0 : 1;
        const int slot = k - ra.step0;
        sa.partials = part + (size_t)slot * max_blocks * 2 * ldv;
        if ((rc = launch_step<T>(G, sa, max_blocks, &nb, s))) return rc;
        ra.nblocks[slot] = nb;
        ra.act[slot] = act;
        ra.nslots = slot + 1;
        if (ra.nslots == kSlots || k == plan.K - 1) {
            int amax = 0;
            for (int i = 0; i < ra.nslots; ++i) amax = std::max(amax, ra.act[i]);
            dim3 grid((2 * amax + 127) / 128, ra.nslots);
            ProfScope ps("reduce_partials", s);
            reduce_partials_kernel<<<grid, 128, 0, s>>>(part, max_blocks, ldv, ra, dots, plan.B);
            MLT_CUDA_TRY(cudaGetLastError());
            ra.step0 = k + 1;
            ra.nslots = 0;
        }
    }
    {
        dim3 grid((unsigned)std::min<int64_t>((ld_mu + 127) / 128, 64), plan.B);
        ProfScope ps("finalize_moments", s);
        finalize_moments_kernel<<<grid, 128, 0, s>>>(dots, plan.B, plan.deg_dev, plan.row_dev, mu_dev,
                                                     ld_mu, (double)d, plan.direct, err_flag);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    return MLT_OK;
}

}  // namespace

int ensure_fp32_values(mlt_matrix* M, cudaStream_t s)
{
    auto conv = [&](DevCSR& C, void*& own) -> int {
        if (C.val32 || !C.val64 || C.nnz == 0) return MLT_OK;
        float* p = nullptr;
        cudaError_t e = cudaMallocAsync((void**)&p, (size_t)C.nnz * sizeof(float), s);
        if (e != cudaSuccess) return fail(MLT_ENOMEM, "cudaMallocAsync (fp32 values) failed");
        const int nb = (int)std::min<int64_t>((C.nnz + 255) / 256, 16LL * M->num_sms);
        ProfScope ps("to_float", s);
        to_float_kernel<<<std::max(nb, 1), 256, 0, s>>>(C.val64, p, C.nnz);
        MLT_CUDA_TRY(cudaGetLastError());
        own = p;
        C.val32 = p;
        return MLT_OK;
    };
    int rc = conv(M->A, M->own_val32);
    if (rc) return rc;
    if (M->flags & MLT_GRAM) rc = conv(M->AT, M->own_t_val32);
    return rc;
}

int run_moments_group(mlt_matrix* M, int precision, const MomentPlan& plan, double a, double b,
                      uint64_t seed, double* mu_dev, int64_t ld_mu, int* err_flag, cudaStream_t s)
{
    if (precision == MLT_PREC_FP32) {
        int rc = ensure_fp32_values(M, s);
        if (rc) return rc;
        return run_group<float>(M, plan, a, b, seed, mu_dev, ld_mu, err_flag, s);
    }
    return run_group<double>(M, plan, a, b, seed, mu_dev, ld_mu, err_flag, s);
}

}  // namespace mlt
