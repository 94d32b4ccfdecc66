// Learned coarse level: a 16 -> 128 -> 128 -> 1 ReLU network in BF16 with FP32
// accumulation, trained by mean squared error on (low-degree moments ->
// degree-n quadratic form) pairs the method itself produces.  It is a project
// addition; its nearest relative in the paper is the regression control
// variate of Section 5.4.  The multilevel estimator stays unbiased for any
// network, because the network's level is corrected by an exact level above it.
//
// One CTA of 128 threads handles a tile of 128 samples, forward and backward.
// The GEMM-shaped steps run on the 5th-generation tensor cores: operands are
// staged in shared memory in the canonical no-swizzle K-major layout (core
// matrices of 8 rows x 16 bytes; 128 bytes to the next 8 columns, K/8 * 128
// bytes to the next 8 rows), one elected thread issues tcgen05.mma with an
// FP32 accumulator in tensor memory, tcgen05.commit arrives on an mbarrier,
// and each thread reads its accumulator row back with tcgen05.ld:
//   layer 1   D1 = X  W1^T     (M 128 samples, N 128, K 16)
//   layer 2   D2 = H1 W2^T     (M 128, N 128, K 128)
//   backward  D3 = dH2 W2      (M 128, N 128, K 128)
//             D4 = dH2^T H1    (M 128 outputs, N 128 inputs, K 128 samples)  -> dW2
//             D5 = dH1^T X     (M 128, N 16, K 128 samples)                  -> dW1
// Every mbarrier wait is bounded; a wait that runs out sets the error flag and
// the CTA stops issuing work.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <algorithm>

#include "mlt_internal.h"

namespace mlt {

namespace {

constexpr int kIn = MLP_IN;
constexpr int kHid = MLP_HID;
constexpr int kTile = 128;
constexpr int kThreadsMlp = 128;
constexpr uint32_t kTmemCols = 512;

// shared-memory tiles (bytes); 1024-byte aligned offsets
constexpr uint32_t kW1s = 0;                       // 128 x 16  (W1, rows = outputs)
constexpr uint32_t kW2s = kW1s + 128 * 16 * 2;     // 128 x 128 (W2, rows = outputs)
constexpr uint32_t kW2Ts = kW2s + 128 * 128 * 2;   // 128 x 128 (W2^T, rows = inputs)
constexpr uint32_t kXs = kW2Ts + 128 * 128 * 2;    // 128 x 16  (X, rows = samples)
constexpr uint32_t kXTs = kXs + 128 * 16 * 2;      // 16 x 128  (X^T, rows = features)
constexpr uint32_t kH1s = kXTs + 16 * 128 * 2;     // 128 x 128 (H1, rows = samples)
constexpr uint32_t kH1Ts = kH1s + 128 * 128 * 2;   // 128 x 128 (H1^T, rows = units)
constexpr uint32_t kG2s = kH1Ts + 128 * 128 * 2;   // 128 x 128 (dH2, later dH1^T)
constexpr uint32_t kG2Ts = kG2s + 128 * 128 * 2;   // 128 x 128 (dH2^T, rows = units)
constexpr uint32_t kRed = kG2Ts + 128 * 128 * 2;   // 4 warps x 3 x 128 floats of column sums
constexpr uint32_t kSmemBytes = kRed + 4 * 3 * 128 * 4;

// byte offset of element (r, k) in a canonical K-major tile with K columns
__device__ __forceinline__ uint32_t cofs(int r, int k, int K)
{
    return (uint32_t)((((r >> 3) * (K >> 3)) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor: start, leading-dimension byte offset (next
// 8 columns), stride byte offset (next 8 rows), descriptor version 1, no swizzle
__device__ __forceinline__ uint64_t mdesc(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = 0;
    d |= (uint64_t)((addr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((lbo & 0x3FFFFu) >> 4) << 16;
    d |= (uint64_t)((sbo & 0x3FFFFu) >> 4) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// instruction descriptor of kind::f16: FP32 accumulator, BF16 A and B, both
// K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(idesc), "r"(acc));
}

__device__ __forceinline__ void mma_commit(uint64_t* mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(mbar))
                 : "memory");
}

__device__ __forceinline__ void fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_smem_async() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

__device__ __forceinline__ bool mbar_try_wait(uint64_t* mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the mbarrier phase with an iteration limit; false if it ran out.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* mbar, uint32_t parity)
{
    for (uint32_t it = 0; it < (1u << 20); ++it)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void st_bf16(uint8_t* base, uint32_t off, float v)
{
    *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

// Sum of v over the 128 threads for each of 16 columns c0..c0+15 (fixed order:
// butterfly inside each warp, then warps 0..3); written to out[c0 + j].
__device__ __forceinline__ void column_sums16(const float (&v)[16], float* red_w, float* out, int c0)
{
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        float s = v[j];
#pragma unroll
        for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
        if (lane == 0) red_w[warp * 384 + c0 + j] = s;
    }
    (void)out;
}

struct MlpArgs {
    const float* X;        // n x 16 features
    const float* T;        // n targets (training)
    int64_t n;
    float inv_n;           // 1 / (number of samples in the loss mean)
    const __nv_bfloat16* W1b;   // 128 x 16
    const __nv_bfloat16* W2b;   // 128 x 128
    const __nv_bfloat16* W2Tb;  // 128 x 128 (transpose)
    const float* P;        // fp32 parameters (biases and w3 are read from here)
    int train;             // 0: predict y; 1: loss and gradient partials
    float* y;              // predictions (predict mode)
    float* part;           // per-CTA partials [gridDim.x][MLP_NPARAMS + 1]
    int* err;
};

__global__ void __launch_bounds__(kThreadsMlp, 1) mlp_tile_kernel(MlpArgs a)
{
    extern __shared__ __align__(1024) uint8_t sm[];
    __shared__ uint64_t mbar;
    __shared__ uint32_t tmem_base;
    __shared__ int failed;
    const int t = threadIdx.x, warp = t >> 5;
    const int64_t row = (int64_t)blockIdx.x * kTile + t;
    const bool valid = row < a.n;
    float* red = reinterpret_cast<float*>(sm + kRed);

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (t == 0) {
        failed = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(&mbar)), "r"(1));
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    // weights and features into the canonical layouts
    for (int e = t; e < kHid * kIn; e += kThreadsMlp)
        *reinterpret_cast<__nv_bfloat16*>(sm + kW1s + cofs(e / kIn, e % kIn, kIn)) = a.W1b[e];
    for (int e = t; e < kHid * kHid; e += kThreadsMlp) {
        *reinterpret_cast<__nv_bfloat16*>(sm + kW2s + cofs(e >> 7, e & 127, kHid)) = a.W2b[e];
        *reinterpret_cast<__nv_bfloat16*>(sm + kW2Ts + cofs(e >> 7, e & 127, kHid)) = a.W2Tb[e];
    }
    {
        float x[kIn];
#pragma unroll
        for (int k = 0; k < kIn; ++k) x[k] = valid ? a.X[row * kIn + k] : 0.0f;
#pragma unroll
        for (int k = 0; k < kIn; ++k) {
            st_bf16(sm, kXs + cofs(t, k, kIn), x[k]);
            st_bf16(sm, kXTs + cofs(k, t, kTile), x[k]);
        }
    }
    fence_smem_async();
    fence_before();
    __syncthreads();
    fence_after();
    const uint32_t tm = tmem_base;
    const uint32_t tl = tm + ((uint32_t)(warp * 32) << 16);   // this warp's 32 TMEM lanes
    const uint32_t sbase = smem_u32(sm);
    uint32_t phase = 0;
    const float* b1 = a.P + MLP_OFF_B1;
    const float* b2 = a.P + MLP_OFF_B2;
    const float* w3 = a.P + MLP_OFF_W3;

    auto issue_wait = [&](auto&& issue) -> bool {
        if (t == 0) {
            issue();
            mma_commit(&mbar);
        }
        const bool ok = mbar_wait_bounded(&mbar, phase);
        phase ^= 1u;
        if (!ok) {
            atomicOr(a.err, 1);
            failed = 1;
        }
        fence_after();
        return ok;
    };

    // ---- layer 1: D1[b][o] = sum_k X[b][k] W1[o][k]
    bool ok = issue_wait([&] {
        mma_bf16(tm + 0, mdesc(sbase + kXs, 128, 256), mdesc(sbase + kW1s, 128, 256), idesc_bf16(128, 128), 0);
    });
    if (ok) {
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float v[16];
            tmem_ld16(tl + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const float h = fmaxf(v[j] + b1[c0 + j], 0.0f);
                st_bf16(sm, kH1s + cofs(t, c0 + j, kHid), h);
                st_bf16(sm, kH1Ts + cofs(c0 + j, t, kTile), h);
            }
        }
    }
    fence_smem_async();
    fence_before();
    __syncthreads();
    fence_after();
    // ---- layer 2: D2[b][o] = sum_k H1[b][k] W2[o][k]
    if (!failed)
        ok = issue_wait([&] {
            for (int s = 0; s < kHid / 16; ++s)
                mma_bf16(tm + 128, mdesc(sbase + kH1s + 256 * s, 128, 2048), mdesc(sbase + kW2s + 256 * s, 128, 2048),
                         idesc_bf16(128, 128), s > 0);
        });
    float y = a.P[MLP_OFF_B3];
    if (!failed) {
        for (int c0 = 0; c0 < kHid; c0 += 16) {
            float v[16];
            tmem_ld16(tl + 128 + c0, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) y = fmaf(w3[c0 + j], fmaxf(v[j] + b2[c0 + j], 0.0f), y);
        }
    }
    float* part = a.part + (size_t)blockIdx.x * (MLP_NPARAMS + 1);
    if (!a.train) {
        if (valid && !failed) a.y[row] = y;
    } else {
        const float r = valid ? (y - a.T[row]) : 0.0f;
        const float dy = 2.0f * r * a.inv_n;
        // dH2 = dy w3 (.) [pre2 > 0]; column sums dw3 = sum dy h2, db2 = sum dH2
        if (!failed) {
            for (int c0 = 0; c0 < kHid; c0 += 16) {
                float v[16], g[16], hw[16];
                tmem_ld16(tl + 128 + c0, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const float pre = v[j] + b2[c0 + j];
                    g[j] = pre > 0.0f ? dy * w3[c0 + j] : 0.0f;
                    hw[j] = dy * fmaxf(pre, 0.0f);
                    st_bf16(sm, kG2s + cofs(t, c0 + j, kHid), g[j]);
                    st_bf16(sm, kG2Ts + cofs(c0 + j, t, kTile), g[j]);
                }
                column_sums16(g, red, nullptr, c0);          // db2 -> red[w][0..127]
                float* r2 = red + 128;
                const int lane = t & 31;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    float s = hw[j];
#pragma unroll
                    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xFFFFFFFFu, s, o);
                    if (lane == 0) r2[warp * 384 + c0 + j] = s;   // dw3 -> red[w][128..255]
                }
            }
        }
        fence_smem_async();
        fence_before();
        __syncthreads();
        fence_after();
        for (int c = t; c < kHid; c += kThreadsMlp) {
            float s2 = 0.0f, s3 = 0.0f;
            for (int w = 0; w < 4; ++w) {
                s2 += red[w * 384 + c];
                s3 += red[w * 384 + 128 + c];
            }
            part[MLP_OFF_B2 + c] = s2;
            part[MLP_OFF_W3 + c] = s3;
        }
        // ---- D3 = dH2 W2 (dH1 before the ReLU mask) and D4 = dH2^T H1 (dW2)
        if (!failed)
            ok = issue_wait([&] {
                for (int s = 0; s < kHid / 16; ++s)
                    mma_bf16(tm + 0, mdesc(sbase + kG2s + 256 * s, 128, 2048),
                             mdesc(sbase + kW2Ts + 256 * s, 128, 2048), idesc_bf16(128, 128), s > 0);
                for (int s = 0; s < kTile / 16; ++s)
                    mma_bf16(tm + 256, mdesc(sbase + kG2Ts + 256 * s, 128, 2048),
                             mdesc(sbase + kH1Ts + 256 * s, 128, 2048), idesc_bf16(128, 128), s > 0);
            });
        __syncthreads();   // every thread has read red before it is reused
        if (!failed) {
            for (int c0 = 0; c0 < kHid; c0 += 16) {
                float v[16], g[16];
                tmem_ld16(tl + c0, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const __nv_bfloat16 hb =
                        *reinterpret_cast<const __nv_bfloat16*>(sm + kH1s + cofs(t, c0 + j, kHid));
                    g[j] = __bfloat162float(hb) > 0.0f ? v[j] : 0.0f;
                    st_bf16(sm, kG2s + cofs(c0 + j, t, kTile), g[j]);   // dH1^T over the old dH2 tile
                }
                column_sums16(g, red, nullptr, c0);          // db1 -> red[w][0..127]
            }
            // dW2 row t of this tile's partial
            for (int c0 = 0; c0 < kHid; c0 += 16) {
                float v[16];
                tmem_ld16(tl + 256 + c0, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) part[MLP_OFF_W2 + t * kHid + c0 + j] = v[j];
            }
        }
        fence_smem_async();
        fence_before();
        __syncthreads();
        fence_after();
        for (int c = t; c < kHid; c += kThreadsMlp) {
            float s1 = 0.0f;
            for (int w = 0; w < 4; ++w) s1 += red[w * 384 + c];
            part[MLP_OFF_B1 + c] = s1;
        }
        // ---- D5 = dH1^T X (dW1), N = 16
        if (!failed)
            ok = issue_wait([&] {
                for (int s = 0; s < kTile / 16; ++s)
                    mma_bf16(tm + 384, mdesc(sbase + kG2s + 256 * s, 128, 2048),
                             mdesc(sbase + kXTs + 256 * s, 128, 2048), idesc_bf16(128, 16), s > 0);
            });
        if (!failed) {
            float v[16];
            tmem_ld16(tl + 384, v);
#pragma unroll
            for (int j = 0; j < 16; ++j) part[MLP_OFF_W1 + t * kIn + j] = v[j];
        }
        // loss and db3 (= sum dy): warp butterflies, then warps in order
        __syncthreads();
        {
            float l = r * r, g3 = dy;
#pragma unroll
            for (int o = 16; o; o >>= 1) {
                l += __shfl_xor_sync(0xFFFFFFFFu, l, o);
                g3 += __shfl_xor_sync(0xFFFFFFFFu, g3, o);
            }
            if ((t & 31) == 0) {
                red[warp * 2] = l;
                red[warp * 2 + 1] = g3;
            }
        }
        __syncthreads();
        if (t == 0) {
            float l = 0.0f, g3 = 0.0f;
            for (int w = 0; w < 4; ++w) {
                l += red[w * 2];
                g3 += red[w * 2 + 1];
            }
            part[MLP_OFF_B3] = g3;
            part[MLP_NPARAMS] = l;
        }
    }
    fence_before();
    __syncthreads();
    fence_after();
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tm), "r"(kTmemCols));
}

// grads[p] = sum over CTAs (in CTA order) of the partials; also the loss sum.
__global__ void mlp_reduce_kernel(const float* __restrict__ part, int nblk, float* __restrict__ grads,
                                  double* __restrict__ loss)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p <= MLP_NPARAMS; p += gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int b = 0; b < nblk; ++b) s += part[(size_t)b * (MLP_NPARAMS + 1) + p];
        if (p < MLP_NPARAMS) grads[p] = (float)s;
        else *loss = s;
    }
}

// Adam step on the FP32 master parameters, then the BF16 copies the tiles read.
__global__ void mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ g, float* __restrict__ m,
                                float* __restrict__ v, float lr, float b1, float b2, float eps, float c1,
                                float c2, __nv_bfloat16* __restrict__ W1b, __nv_bfloat16* __restrict__ W2b,
                                __nv_bfloat16* __restrict__ W2Tb, int update)
{
    for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < MLP_NPARAMS; p += gridDim.x * blockDim.x) {
        float w = P[p];
        if (update) {
            const float gp = g[p];
            const float mp = b1 * m[p] + (1.0f - b1) * gp;
            const float vp = b2 * v[p] + (1.0f - b2) * gp * gp;
            m[p] = mp;
            v[p] = vp;
            w -= lr * (mp / c1) / (sqrtf(vp / c2) + eps);
            P[p] = w;
        }
        if (p >= MLP_OFF_W1 && p < MLP_OFF_W1 + kHid * kIn) {
            W1b[p - MLP_OFF_W1] = __float2bfloat16_rn(w);
        } else if (p >= MLP_OFF_W2 && p < MLP_OFF_W2 + kHid * kHid) {
            const int e = p - MLP_OFF_W2;
            const __nv_bfloat16 wb = __float2bfloat16_rn(w);
            W2b[e] = wb;
            W2Tb[(e & 127) * kHid + (e >> 7)] = wb;
        }
    }
}

}  // namespace

size_t mlp_smem_bytes() { return kSmemBytes; }

int mlp_launch_tiles(const MlpDev& D, const float* X, const float* T, int64_t n, float inv_n, int train,
                     float* y, int* err, cudaStream_t s)
{
    if (n <= 0) return MLT_OK;
    static bool attr_set = false;
    if (!attr_set) {
        MLT_CUDA_TRY(cudaFuncSetAttribute(mlp_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                          (int)kSmemBytes));
        attr_set = true;
    }
    MlpArgs a;
    a.X = X;
    a.T = T;
    a.n = n;
    a.inv_n = inv_n;
    a.W1b = D.W1b;
    a.W2b = D.W2b;
    a.W2Tb = D.W2Tb;
    a.P = D.P;
    a.train = train;
    a.y = y;
    a.part = D.part;
    a.err = err;
    const int nblk = (int)((n + kTile - 1) / kTile);
    {
        ProfScope ps(train ? "mlp_fwd_bwd" : "mlp_forward", s);
        mlp_tile_kernel<<<nblk, kThreadsMlp, kSmemBytes, s>>>(a);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    if (train) {
        ProfScope ps("mlp_reduce", s);
        mlp_reduce_kernel<<<(MLP_NPARAMS + 256) / 256, 256, 0, s>>>(D.part, nblk, D.G, D.loss);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    return MLT_OK;
}

int mlp_adam(const MlpDev& D, float lr, int64_t step, int update, cudaStream_t s)
{
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    const float c1 = update ? 1.0f - powf(b1, (float)step) : 1.0f;
    const float c2 = update ? 1.0f - powf(b2, (float)step) : 1.0f;
    ProfScope ps("mlp_adam", s);
    mlp_adam_kernel<<<(MLP_NPARAMS + 255) / 256, 256, 0, s>>>(D.P, D.G, D.M, D.V, lr, b1, b2, eps, c1, c2, D.W1b,
                                                              D.W2b, D.W2Tb, update);
    return cuda_fail(cudaGetLastError(), "mlp_adam_kernel");
}

}  // namespace mlt
