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
// Work split (fixed per matrix, so every result is reproducible): rows cost
// kRowCost units plus one per entry; the unit axis is cut into chunks of Uc
// units.  A row of degree <= Ul (>= Uc) belongs to the chunk holding its first
// unit.  Longer rows are cut into fixed segments of Ul entries whose partial
// products go to a scratch table; a second kernel adds each row's segments in
// order and applies the recurrence there.  Work items (chunks, then segments)
// are dealt round-robin to groups of G lanes on a grid no larger than the
// resident one; a group always owns the same columns.  Chunks are small (about
// a thousand per SM), so at any moment the groups work on one narrow band of
// rows and the rows of V gathered by neighbouring rows are still in L2.
//
// Reductions are deterministic: each CTA writes per-column partial sums in a
// fixed order, and a separate kernel adds the CTA partials in CTA order.
// Each thread's running dot products are FP64 for FP64 vectors.  For FP32
// vectors they are compensated (Kahan) FP32 sums, whose error is at most
// 2^-23 times the sum of |terms| (below the rounding already in the FP32
// vectors), because FP64 arithmetic on GB300 runs at 1/64 of the FP32 rate
// and a per-row FP64 update would cost more than streaming the vectors; the
// sums leave each thread as FP64 and everything after that is FP64.
#include <cuda_runtime.h>

#include <algorithm>
#include <type_traits>
#include <vector>

#include "df64.cuh"
#include "mlt_internal.h"
#include "rng.cuh"


namespace mlt {
namespace {

constexpr int kThreads = 256;
constexpr int kSlots = 16;          // steps whose partials are buffered before a reduction
constexpr int64_t kRowCost = 4;     // units charged per row (the epilogue) on top of its entries
constexpr int64_t kChunksPerSm = 1024;  // work chunks per SM in the split of an operand
constexpr int64_t kLongRow = 128;   // rows above max(Uc, this) are cut into segments
constexpr int32_t kSegWindow = 16384;    // column window of the segment dealing order

template <typename T> struct Lanes;
template <> struct Lanes<double> { static constexpr int N = 2; };   // 16-byte vectors
template <> struct Lanes<float> { static constexpr int N = 4; };
template <> struct Lanes<df64> { static constexpr int N = 2; };     // 16-byte vectors of pairs

// A lane's 16-byte slice of a vector row.  Double-float slices hold the high
// parts of their two entries, then the two low parts, so that a slice loads as
// two packed FP32 pairs (see the f32x2 operations below).
template <typename T, int N> struct alignas(sizeof(T) * N) Pack {
    T v[N];
    __device__ __forceinline__ T get(int q) const { return v[q]; }
    __device__ __forceinline__ void set(int q, T x) { v[q] = x; }
};
template <> struct alignas(16) Pack<df64, 2> {
    float h[2], l[2];
    __device__ __forceinline__ df64 get(int q) const { return df64(h[q], l[q]); }
    __device__ __forceinline__ void set(int q, df64 x) { h[q] = x.hi; l[q] = x.lo; }
};

// Entry c of the vector row at v + row_off (row_off = row * ldv, ldv even).
template <typename T>
__device__ __forceinline__ void put_entry(T* v, size_t row_off, int c, T x) { v[row_off + c] = x; }
template <>
__device__ __forceinline__ void put_entry<df64>(df64* v, size_t row_off, int c, df64 x)
{
    float* f = reinterpret_cast<float*>(v + row_off + (c & ~1));
    f[c & 1] = x.hi;
    f[2 + (c & 1)] = x.lo;
}


// Per vector type: the resident CTAs per SM the step kernel is compiled for
// (C), the unroll depth of its gather loop (U), whether its gathers carry an
// L2 evict-last policy (E), whether long-row segments are dealt out in
// column-window order (W, see ensure_spmm_plan), predicated gather blocks (PR)
// and the column-index prefetch on pattern matrices (PF).  More unrolled gathers keep more row
// reads outstanding but need registers, which lowers the resident CTAs; the
// evict-last policy keeps the gathered V_k rows in L2 against the streams of
// V_{k-1}, V_{k+1} and the column indices.  Measured on the scale-22 R-MAT
// graph (gather-bound) and the 100^3 diffusion operator (streaming): FP32 and
// FP64 gain from the deeper unroll (FP32 9.5 -> 8.1 ms a step on the graph)
// and FP32 from the policy (8.1 -> 7.5 ms).  The double-float step on packed
// pairs (row_sum_df2, epilogue_df2) needs few enough registers for eight
// unrolled gathers at five CTAs: 8.4 -> 7.2 ms on the graph, against 8.3 at
// six CTAs and unroll 8 and 8.1 at five and unroll 12 (3% slower on the
// streaming operator).  The column-window order takes FP32 and double-float
// steps on the graph 3-4% lower and the FP64 step, bound by FP64 arithmetic,
// 2% higher.
//
// PR shapes the gather loop for rows whose length is not a multiple of the
// unroll depth: predicated gathers go in blocks of
// unroll-depth slots, each slot switched off past the row's end, so that a
// short row's gathers are all in flight together; without PR the compiler's
// remainder loop takes them one at a time.  Predicated blocks took the FP32
// step on the 100^3 diffusion operator (7 entries a row) from 0.569 to
// 0.516 ms and the Gram operator's X^T step from 0.201 to 0.182 ms, left FP32
// on the graph unchanged (6.18 -> 6.14 ms), and slowed the double-float and
// FP64 steps by 2-9%.  They apply to groups of at least unroll-depth lanes:
// a narrower group (few live probes) takes at most G entries a batch, and a
// block of mostly idle slots cost the learned estimator's FP32 moments, whose
// last steps run 1-2 live probes, 16% of their time.
//
// PF: on pattern matrices, a batch's column indices are loaded one batch
// ahead, so that their latency overlaps the previous batch's gathers.  That
// took the FP32 step on the graph from 6.12 to 5.87 ms; the double-float step
// went from 7.17 to 7.60 ms and FP64 1% slower, and on valued FP32 matrices
// (stencil, Gram) it lost 1-5%, so it is on for FP32 patterns only.
template <int C, int U, bool E, bool W, bool PR, bool PF> struct TuneOf {
    static constexpr int kCtas = C, kUnroll = U;
    static constexpr bool kEvictLast = E, kWindowSegs = W, kPredicated = PR, kPrefetchPattern = PF;
};
template <typename T> struct StepTuning;
template <> struct StepTuning<float> : TuneOf<5, 8, true, true, true, true> {};
template <> struct StepTuning<double> : TuneOf<4, 8, false, false, false, false> {};
template <> struct StepTuning<df64> : TuneOf<5, 8, false, true, false, false> {};

// An L2 access policy that marks lines evict-last (createpolicy, PTX ISA).
__device__ __forceinline__ uint64_t evict_last_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// A gathered 16-byte row slice, under the L2 policy `pol` when E.
template <bool E, typename P>
__device__ __forceinline__ P ld_gather(const P* p, uint64_t pol)
{
    static_assert(sizeof(P) == 16, "16-byte packs");
    if constexpr (E) {
        uint4 u;
        asm volatile("ld.global.L2::cache_hint.v4.u32 {%0,%1,%2,%3}, [%4], %5;"
                     : "=r"(u.x), "=r"(u.y), "=r"(u.z), "=r"(u.w)
                     : "l"(p), "l"(pol));
        P r;
        memcpy(&r, &u, 16);
        return r;
    } else {
        (void)pol;
        return *p;
    }
}

// The same 16-byte load as two 64-bit words (the operands of packed pair
// arithmetic).
template <bool E>
__device__ __forceinline__ ulonglong2 ld_gather2(const void* p, uint64_t pol)
{
    if constexpr (E) {
        ulonglong2 u;
        asm volatile("ld.global.L2::cache_hint.v2.u64 {%0,%1}, [%2], %3;"
                     : "=l"(u.x), "=l"(u.y)
                     : "l"(p), "l"(pol));
        return u;
    } else {
        (void)pol;
        return *reinterpret_cast<const ulonglong2*>(p);
    }
}

// A thread's running dot product.  The kernels keep these in shared memory
// (one slot per thread, see DotSlots): held in registers beside a row's
// gathers they pushed the step kernel past the six-CTA register budget, and
// the spilled copies went through L1 to L2.
template <typename T> struct DotAcc;
template <> struct DotAcc<double> {
    double s;
    __device__ __forceinline__ void clear() { s = 0.0; }
    __device__ __forceinline__ void add_prod(double a, double b) { s = fma(a, b, s); }
    __device__ __forceinline__ void add(double x) { s += x; }
    __device__ __forceinline__ double value() const { return s; }
};
template <> struct DotAcc<float> {
    float s, c;   // Kahan: s - c is the running sum
    __device__ __forceinline__ void clear() { s = c = 0.0f; }
    __device__ __forceinline__ void add(float x)
    {
        const float y = x - c;
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ void add_prod(float a, float b)
    {
        const float y = fmaf(a, b, -c);   // the product enters unrounded
        const float t = s + y;
        c = (t - s) - y;
        s = t;
    }
    __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <> struct DotAcc<df64> {
    df64 s;
    __device__ __forceinline__ void clear() { s = df64(0); }
    __device__ __forceinline__ void add_prod(df64 a, df64 b) { s = a * b + s; }
    __device__ __forceinline__ void add(df64 x) { s = s + x; }
    __device__ __forceinline__ double value() const { return df_to_double(s); }
};

// The CTA's running dots: kind [0] V_{k+1}.V_{k+1} (unused in direct mode),
// [1] V_{k+1}.V_k or z.V_{k+1}, for the thread's columns c0 + q.  Each thread
// only touches its own slots, and a warp's accesses are consecutive.
template <typename T>
struct DotSlots {
    DotAcc<T> d[2][Lanes<T>::N][kThreads];
    __device__ __forceinline__ DotAcc<T> load(int kind, int q, int t) const { return d[kind][q][t]; }
    __device__ __forceinline__ void store(int kind, int q, int t, DotAcc<T> x) { d[kind][q][t] = x; }
};
// FP32: the Kahan sums of columns (c0, c0 + 1) and (c0 + 2, c0 + 3) as packed
// pairs, (sums, compensations), so that epilogue_f2 updates two columns with
// each packed instruction.
template <>
struct DotSlots<float> {
    ulonglong2 d[2][2][kThreads];
    __device__ __forceinline__ DotAcc<float> load(int kind, int q, int t) const
    {
        const ulonglong2 v = d[kind][q >> 1][t];
        DotAcc<float> x;
        x.s = (q & 1) ? hi_half(v.x) : lo_half(v.x);
        x.c = (q & 1) ? hi_half(v.y) : lo_half(v.y);
        return x;
    }
    __device__ __forceinline__ void store(int kind, int q, int t, DotAcc<float> x)
    {
        ulonglong2 v = d[kind][q >> 1][t];
        if (q & 1) {
            v.x = pack2(lo_half(v.x), x.s);
            v.y = pack2(lo_half(v.y), x.c);
        } else {
            v.x = pack2(x.s, hi_half(v.x));
            v.y = pack2(x.c, hi_half(v.y));
        }
        d[kind][q >> 1][t] = v;
    }
};

// A matrix value through the read-only cache.
template <typename T>
__device__ __forceinline__ T ldg_val(const T* p) { return __ldg(p); }
template <>
__device__ __forceinline__ df64 ldg_val<df64>(const df64* p)
{
    const float2 v = __ldg(reinterpret_cast<const float2*>(p));
    return df64(v.x, v.y);
}

// A register value from lane src of the group.
template <typename T>
__device__ __forceinline__ T shfl_val(unsigned mask, T v, int src, int width)
{
    return __shfl_sync(mask, v, src, width);
}
template <>
__device__ __forceinline__ df64 shfl_val<df64>(unsigned mask, df64 v, int src, int width)
{
    return df64(__shfl_sync(mask, v.hi, src, width), __shfl_sync(mask, v.lo, src, width));
}

// The operand's values in precision T (null for a pattern matrix).
template <typename T>
const T* vals_of(const DevCSR& C)
{
    if (std::is_same<T, double>::value) return reinterpret_cast<const T*>(C.val64);
    if (std::is_same<T, float>::value) return reinterpret_cast<const T*>(C.val32);
    return reinterpret_cast<const T*>(C.valdf);
}

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
    int mode;              // 0 first step, 1 recurrence step, 2 plain product, 3 Clenshaw step
    const T* addv;         // mode 3: out = m1 * At V_k - V_{k-1} + coef * addv (no dots)
    T coef, m1;
    int direct;            // dots are z . V_{k+1} instead of V.V and V.V_k
    int B;                 // probes in the group (columns >= B are padding)
    uint64_t seedmix;
    const int64_t* ids;    // global id of each column's probe (direct mode)
    const int32_t* orig;   // original id of each row (relabelled operator), or null
    double* partials;      // [gridDim.x][2][ldv] for this launch
    // work split of this operand
    int64_t nch, Uc, Ul, nseg;
    int nlong;
    const int64_t* crow;
    const int32_t* seg_row;
    const int64_t* seg_k0;
    const int32_t* long_rows;
    const int64_t* long_seg0;
    const int32_t* seg_order;   // dealing order of the segments, or null (segment order)
    T* segpart;            // [nseg][ldv] partial products of long-row segments
};

template <typename T, int G>
struct Lane {
    static constexpr int N = Lanes<T>::N;
    int glane;
    unsigned gmask;
    bool vok;
    int c0;
    long long gcls, ncls;   // group index within its column class, groups per class
    bool active;

    __device__ Lane(const StepArgs<T>& a)
    {
        const int tid = threadIdx.x;
        const int lane = tid & 31;
        glane = lane & (G - 1);
        gmask = (G == 32) ? 0xFFFFFFFFu : (((1u << G) - 1u) << (lane & ~(G - 1)));
        const int gpb = kThreads / G;
        const long long gg = (long long)blockIdx.x * gpb + tid / G;
        const long long total = (long long)gridDim.x * gpb;
        ncls = total / a.nchunks;
        gcls = gg / a.nchunks;
        const int chunk = (int)(gg % a.nchunks);
        const int vidx = chunk * G + glane;
        vok = vidx < a.nvec;
        c0 = vidx * N;
        active = gg < ncls * a.nchunks;
    }
};


// Running sums of one row over the lane's N columns: add() takes one gathered
// row slice (and the entry's value, for valued matrices), close() ends a batch
// of at most G entries, out() gives the N sums.  Three forms:
//  - SumScalar: any vector type, acc = fma(a_ij, x, acc) for valued matrices
//    and acc + x for patterns (every a_ij = 1; for FP32 and FP64 that equals
//    fma(1, x, acc) bit for bit);
//  - SumF2, FP32 patterns: the four sums as two packed pairs, each packed add
//    the scalar add on both halves, so the sums are the same bit for bit (on
//    valued matrices the packed form, with a_ij broadcast into a pair,
//    measured slower);
//  - SumDf2, double-float patterns: the two sums as packed pairs of high and
//    low parts, added as df_add_lazy does (the rounding error of the high
//    parts into the low parts, left unnormalised) and renormalised as df_norm
//    does at the end of each batch.  That cuts the arithmetic from 11 to 8
//    FP32 operations per value, each packed instruction doing two, and the
//    deferred error stays below 2^-38 of the sum.  A double-float slice loads
//    as (high parts, low parts), the two packed operands.
template <typename T, bool PAT>
struct SumScalar {
    static constexpr int N = Lanes<T>::N;
    using P = Pack<T, N>;
    T s[N];
    __device__ __forceinline__ void init()
    {
#pragma unroll
        for (int q = 0; q < N; ++q) s[q] = T(0);
    }
    template <bool E>
    __device__ __forceinline__ void add(const T* p, T v, uint64_t pol)
    {
        const P x = ld_gather<E>(reinterpret_cast<const P*>(p), pol);
#pragma unroll
        for (int q = 0; q < N; ++q) {
            if constexpr (PAT) s[q] = s[q] + x.get(q);
            else s[q] = fma(v, x.get(q), s[q]);
        }
    }
    __device__ __forceinline__ void close() {}
    __device__ __forceinline__ void out(T (&acc)[N]) const
    {
#pragma unroll
        for (int q = 0; q < N; ++q) acc[q] = s[q];
    }
};

struct SumF2 {
    uint64_t A0, A1;
    __device__ __forceinline__ void init() { A0 = A1 = 0; }
    template <bool E>
    __device__ __forceinline__ void add(const float* p, float, uint64_t pol)
    {
        const ulonglong2 x = ld_gather2<E>(p, pol);
        A0 = add2(A0, x.x);
        A1 = add2(A1, x.y);
    }
    __device__ __forceinline__ void close() {}
    __device__ __forceinline__ void out(float (&acc)[4]) const
    {
        acc[0] = lo_half(A0);
        acc[1] = hi_half(A0);
        acc[2] = lo_half(A1);
        acc[3] = hi_half(A1);
    }
};

struct SumDf2 {
    uint64_t H, Lo;
    __device__ __forceinline__ void init() { H = Lo = 0; }
    template <bool E>
    __device__ __forceinline__ void add(const df64* p, df64, uint64_t pol)
    {
        const ulonglong2 x = ld_gather2<E>(p, pol);
        const uint64_t s = add2(H, x.x);
        const uint64_t bb = sub2(s, H);
        const uint64_t e = add2(sub2(H, sub2(s, bb)), sub2(x.x, bb));
        Lo = add2(Lo, add2(e, x.y));
        H = s;
    }
    __device__ __forceinline__ void close()
    {
        const uint64_t s = add2(H, Lo);
        Lo = sub2(Lo, sub2(s, H));
        H = s;
    }
    __device__ __forceinline__ void out(df64 (&acc)[2]) const
    {
        acc[0] = df64(lo_half(H), lo_half(Lo));
        acc[1] = df64(hi_half(H), hi_half(Lo));
    }
};

template <typename T, bool PAT> struct SumOf { using type = SumScalar<T, PAT>; };
template <> struct SumOf<float, true> { using type = SumF2; };
template <> struct SumOf<df64, true> { using type = SumDf2; };

// acc = sum over entries [k0, k1) of a_ij * V[j, c0 .. c0+N), the column
// indices (and values) loaded G at a time from the row's first entry.  Row
// and entry indices fit in 32 bits (nnz < 2^31 is checked when the handle is
// made).
template <typename T, int G, bool PAT>
__device__ __forceinline__ void row_product_t(const StepArgs<T>& a, const Lane<T, G>& L, int k0, int k1,
                                              T (&acc)[Lanes<T>::N], uint64_t pol)
{
    constexpr int kGatherUnroll = StepTuning<T>::kUnroll;
    constexpr bool E = StepTuning<T>::kEvictLast;
    typename SumOf<T, PAT>::type S;
    S.init();
    // the batch's column indices (and values); with PF the next batch's are
    // loaded while this batch's gathers are in flight
    constexpr bool PF = PAT && StepTuning<T>::kPrefetchPattern;
    int cj = 0;
    T vj = T(0);
    if (PF && k0 + L.glane < k1) cj = __ldg(a.col + k0 + L.glane);
    for (int base = k0; base < k1; base += G) {
        int cn = 0;
        T vn = T(0);
        if constexpr (PF) {
            if (base + G + L.glane < k1) cn = __ldg(a.col + base + G + L.glane);
        } else {
            const int k = base + L.glane;
            if (k < k1) {
                cj = __ldg(a.col + k);
                if constexpr (!PAT) vj = ldg_val(a.val + k);
            }
        }
        const int cnt = min(G, k1 - base);
        if constexpr (StepTuning<T>::kPredicated && G >= kGatherUnroll) {
            // blocks of kGatherUnroll predicated slots: every gather of a block
            // is issued before the first of them is consumed, also in the
            // last, partial block (groups narrower than a block, which take
            // at most G entries a batch, keep the plain loop)
            for (int t0 = 0; t0 < cnt; t0 += kGatherUnroll) {
#pragma unroll
                for (int u = 0; u < kGatherUnroll; ++u) {
                    const int t = t0 + u;
                    const int c = __shfl_sync(L.gmask, cj, t, G);
                    T v = T(1);
                    if constexpr (!PAT) v = shfl_val(L.gmask, vj, t, G);
                    if (t < cnt && L.vok) S.template add<E>(a.vgather + (size_t)c * a.ldv + L.c0, v, pol);
                }
            }
        } else {
#pragma unroll kGatherUnroll
            for (int t = 0; t < cnt; ++t) {
                const int c = __shfl_sync(L.gmask, cj, t, G);
                T v = T(1);
                if constexpr (!PAT) v = shfl_val(L.gmask, vj, t, G);
                if (L.vok) S.template add<E>(a.vgather + (size_t)c * a.ldv + L.c0, v, pol);
            }
        }
        S.close();
        if constexpr (PF) cj = cn;
        (void)vn;
    }
    S.out(acc);
}

template <typename T, int G>
__device__ __forceinline__ void row_product(const StepArgs<T>& a, const Lane<T, G>& L, int k0, int k1,
                                            T (&acc)[Lanes<T>::N], uint64_t pol)
{
    if (a.val) row_product_t<T, G, false>(a, L, k0, k1, acc, pol);
    else row_product_t<T, G, true>(a, L, k0, k1, acc, pol);
}

// The row's operands of the epilogue, loaded before its gathers (they do not
// depend on them): V_k at the row and, in a recurrence step, V_{k-1}.
template <typename T>
struct RowOperands {
    Pack<T, Lanes<T>::N> xc, xp;
};

template <typename T>
__device__ __forceinline__ RowOperands<T> load_operands(const StepArgs<T>& a, int64_t r, int c0)
{
    using P = Pack<T, Lanes<T>::N>;
    RowOperands<T> o;
    const size_t off = (size_t)r * a.ldv + c0;
    if (a.mode != 2) o.xc = *reinterpret_cast<const P*>(a.vcur + off);
    if (a.mode == 1 || a.mode == 3) o.xp = *reinterpret_cast<const P*>(a.vprev_out + off);
    return o;
}

// The recurrence update and the V.V, V.V_k dot products of epilogue (below)
// for double-float vectors, on packed pairs: the lane's two entries go through
// the df64 operations of the generic code side by side.  A recurrence step
// folds its factor 2 into alpha and beta (doubling is exact), so
// out = (2 alpha) acc + (2 beta) xc - xp equals 2 (alpha acc + beta xc) - xp.
__device__ __forceinline__ void epilogue_df2(const StepArgs<df64>& a, size_t off, const df64 (&acc)[2],
                                             const RowOperands<df64>& ops, DotSlots<df64>& dots)
{
    df2 xc;
    memcpy(&xc, &ops.xc, sizeof(df2));
    df2 al = df2_of(a.alpha, a.alpha), be = df2_of(a.beta, a.beta);
    if (a.mode != 0) {
        al = df2_twice(al);
        be = df2_twice(be);
    }
    df2 out = al * df2_of(acc[0], acc[1]) + be * xc;
    if (a.mode != 0) {
        df2 xp;
        memcpy(&xp, &ops.xp, sizeof(df2));
        out = out + (-xp);
    }
    *reinterpret_cast<ulonglong2*>(a.vprev_out + off) = make_ulonglong2(out.h, out.l);
    const int tid = threadIdx.x;
    const df2 s0 = out * out + df2_of(dots.d[0][0][tid].s, dots.d[0][1][tid].s);
    dots.d[0][0][tid].s = df2_first(s0);
    dots.d[0][1][tid].s = df2_second(s0);
    const df2 s1 = out * xc + df2_of(dots.d[1][0][tid].s, dots.d[1][1][tid].s);
    dots.d[1][0][tid].s = df2_first(s1);
    dots.d[1][1][tid].s = df2_second(s1);
}

// A packed Kahan step on two columns: sc = (sums, compensations) takes the
// products a * b, each as DotAcc<float>::add_prod does.
__device__ __forceinline__ void kahan_prod2(ulonglong2& sc, uint64_t a, uint64_t b)
{
    ulonglong2 v = sc;
    const uint64_t y = fma2(a, b, neg2(v.y));
    const uint64_t t = add2(v.x, y);
    v.y = sub2(sub2(t, v.x), y);
    v.x = t;
    sc = v;
}

// The recurrence update and the V.V, V.V_k dot products of epilogue (below)
// for FP32 vectors, on packed pairs: out = alpha' acc + beta' xc (- xp), the
// product beta' xc rounded and alpha' acc fused into the sum, with the factor
// 2 of a recurrence step folded into alpha' and beta' (doubling is exact).
__device__ __forceinline__ void epilogue_f2(const StepArgs<float>& a, size_t off, const float (&acc)[4],
                                            const RowOperands<float>& ops, DotSlots<float>& dots)
{
    ulonglong2 xc;
    memcpy(&xc, &ops.xc, sizeof(xc));
    const float al = a.mode != 0 ? 2.0f * a.alpha : a.alpha;
    const float be = a.mode != 0 ? 2.0f * a.beta : a.beta;
    const uint64_t al2 = pack2(al, al), be2 = pack2(be, be);
    uint64_t o0 = fma2(al2, pack2(acc[0], acc[1]), mul2(be2, xc.x));
    uint64_t o1 = fma2(al2, pack2(acc[2], acc[3]), mul2(be2, xc.y));
    if (a.mode != 0) {
        ulonglong2 xp;
        memcpy(&xp, &ops.xp, sizeof(xp));
        o0 = sub2(o0, xp.x);
        o1 = sub2(o1, xp.y);
    }
    *reinterpret_cast<ulonglong2*>(a.vprev_out + off) = make_ulonglong2(o0, o1);
    const int tid = threadIdx.x;
    kahan_prod2(dots.d[0][0][tid], o0, o0);
    kahan_prod2(dots.d[0][1][tid], o1, o1);
    kahan_prod2(dots.d[1][0][tid], o0, xc.x);
    kahan_prod2(dots.d[1][1][tid], o1, xc.y);
}

// V_{k+1}[r] from acc = (A V_k)[r], and the fused dot products.
template <typename T, bool CL>
__device__ __forceinline__ void epilogue(const StepArgs<T>& a, int64_t r, int c0, const T (&acc)[Lanes<T>::N],
                                         const RowOperands<T>& ops, DotSlots<T>& dots)
{
    constexpr int N = Lanes<T>::N;
    using P = Pack<T, N>;
    const size_t off = (size_t)r * a.ldv + c0;
    P out;
    if (a.mode == 2) {
#pragma unroll
        for (int q = 0; q < N; ++q) out.set(q, acc[q]);
        *reinterpret_cast<P*>(a.vprev_out + off) = out;
        return;
    }
    const P& xc = ops.xc;
    if constexpr (CL) {   // Clenshaw step (mode 3): compiled into its own kernels only
        const P& xp = ops.xp;
        const P xa = *reinterpret_cast<const P*>(a.addv + off);
#pragma unroll
        for (int q = 0; q < N; ++q)
            out.set(q, a.m1 * (a.alpha * acc[q] + a.beta * xc.get(q)) - xp.get(q) + a.coef * xa.get(q));
        *reinterpret_cast<P*>(a.vprev_out + off) = out;
        return;
    }
    if constexpr (std::is_same<T, df64>::value) {
        if (!a.direct) {
            epilogue_df2(a, off, acc, ops, dots);
            return;
        }
    }
    if constexpr (std::is_same<T, float>::value) {
        if (!a.direct) {
            epilogue_f2(a, off, acc, ops, dots);
            return;
        }
    }
    if (a.mode == 0) {
#pragma unroll
        for (int q = 0; q < N; ++q) out.set(q, a.alpha * acc[q] + a.beta * xc.get(q));
    } else {
        const P& xp = ops.xp;
#pragma unroll
        for (int q = 0; q < N; ++q) out.set(q, T(2) * (a.alpha * acc[q] + a.beta * xc.get(q)) - xp.get(q));
    }
    *reinterpret_cast<P*>(a.vprev_out + off) = out;
    const int tid = threadIdx.x;
    if (!a.direct) {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            DotAcc<T> s0 = dots.load(0, q, tid), s1 = dots.load(1, q, tid);
            const T o = out.get(q);
            s0.add_prod(o, o);
            s1.add_prod(o, xc.get(q));
            dots.store(0, q, tid, s0);
            dots.store(1, q, tid, s1);
        }
    } else {
#pragma unroll
        for (int q = 0; q < N; ++q) {
            if (c0 + q >= a.B) break;
            const bool neg = probe_negative(a.seedmix, (uint64_t)a.ids[c0 + q], (uint64_t)(a.orig ? a.orig[r] : r));
            DotAcc<T> s1 = dots.load(1, q, tid);
            s1.add(neg ? -out.get(q) : out.get(q));
            dots.store(1, q, tid, s1);
        }
    }
}

// Zero the thread's dot slots (each thread only ever touches its own).
template <typename T>
__device__ __forceinline__ void clear_dots(DotSlots<T>& dots)
{
#pragma unroll
    for (int q = 0; q < Lanes<T>::N; ++q) {
        DotAcc<T> z;
        z.clear();
        dots.store(0, q, threadIdx.x, z);
        dots.store(1, q, threadIdx.x, z);
    }
}

// CTA reduction in a fixed order: column c collects the groups of this CTA
// whose column chunk holds it, in group order.
template <typename T, int G>
__device__ __forceinline__ void cta_partials(const StepArgs<T>& a, const Lane<T, G>& L, const DotSlots<T>& dots)
{
    constexpr int N = Lanes<T>::N;
    __syncthreads();
    const int gpb = kThreads / G;
    const int ncols = a.nvec * N;
    double* part = a.partials + (size_t)blockIdx.x * 2 * a.ldv;
    const long long g0 = (long long)blockIdx.x * gpb;
    for (int c = threadIdx.x; c < ncols; c += kThreads) {
        const int v = c / N, q = c % N;
        const int ch = v / G, gl = v % G;
        double s0 = 0.0, s1 = 0.0;
        for (int g = 0; g < gpb; ++g) {
            const long long gglob = g0 + g;
            if (gglob >= L.ncls * a.nchunks || (int)(gglob % a.nchunks) != ch) continue;
            const int t = g * G + gl;
            s0 += dots.load(0, q, t).value();
            s1 += dots.load(1, q, t).value();
        }
        part[c] = s0;
        part[a.ldv + c] = s1;
    }
}

template <typename T, int G, bool CL>
__global__ void __launch_bounds__(kThreads, StepTuning<T>::kCtas) cheb_step_kernel(StepArgs<T> a)
{
    constexpr int N = Lanes<T>::N;
    const Lane<T, G> L(a);
    __shared__ DotSlots<T> dots;
    if constexpr (!CL) clear_dots<T>(dots);
    const uint64_t pol = StepTuning<T>::kEvictLast ? evict_last_policy() : 0;

    if (L.active) {
        const int64_t nitems = a.nch + a.nseg;
        for (int64_t it = L.gcls; it < nitems; it += L.ncls) {
            T acc[N];
            if (it < a.nch) {
                // row and entry indices fit in 32 bits (nnz < 2^31); units may not
                const int64_t u0 = it * a.Uc, u1 = u0 + a.Uc;
                const int nrows = (int)a.nrows;
                int r = (int)__ldg(a.crow + it);
                int beg = r < nrows ? (int)__ldg(a.rowptr + r) : 0;
                int end = r < nrows ? (int)__ldg(a.rowptr + r + 1) : 0;
                for (; r < nrows; ++r) {
                    const int64_t pr = (int64_t)beg + kRowCost * r;
                    if (pr >= u1) break;
                    // the row after next's end, one row ahead of its use
                    const int nxt = r + 2 <= nrows ? (int)__ldg(a.rowptr + r + 2) : end;
                    // rows before u0 belong to the previous chunk; long rows are done by segments
                    if (pr >= u0 && end - beg <= a.Ul) {
                        RowOperands<T> ops;
                        if (L.vok) ops = load_operands(a, r, L.c0);
                        row_product<T, G>(a, L, beg, end, acc, pol);
                        if (L.vok) epilogue<T, CL>(a, r, L.c0, acc, ops, dots);
                    }
                    beg = end;
                    end = nxt;
                }
            } else {
                const int64_t sidx = a.seg_order ? (int64_t)__ldg(a.seg_order + (it - a.nch)) : it - a.nch;
                const int64_t r = __ldg(a.seg_row + sidx);
                const int k0 = (int)__ldg(a.seg_k0 + sidx);
                const int k1 = (int)min((int64_t)k0 + a.Ul, __ldg(a.rowptr + r + 1));
                row_product<T, G>(a, L, k0, k1, acc, pol);
                if (L.vok) {
                    Pack<T, N> p;
#pragma unroll
                    for (int q = 0; q < N; ++q) p.set(q, acc[q]);
                    *reinterpret_cast<Pack<T, N>*>(a.segpart + (size_t)sidx * a.ldv + L.c0) = p;
                }
            }
        }
    }
    if (CL || a.mode >= 2) return;
    cta_partials<T, G>(a, L, dots);
}

// Long rows: add the segment products in segment order, then the recurrence.
template <typename T, int G, bool CL>
__global__ void __launch_bounds__(kThreads) cheb_long_kernel(StepArgs<T> a)
{
    constexpr int N = Lanes<T>::N;
    using P = Pack<T, N>;
    const Lane<T, G> L(a);
    __shared__ DotSlots<T> dots;
    if constexpr (!CL) clear_dots<T>(dots);
    if (L.active) {
        for (int64_t i = L.gcls; i < a.nlong; i += L.ncls) {
            if (!L.vok) continue;
            T acc[N];
#pragma unroll
            for (int q = 0; q < N; ++q) acc[q] = T(0);
            const int64_t r = a.long_rows[i];
            const RowOperands<T> ops = load_operands(a, r, L.c0);
            for (int64_t sidx = a.long_seg0[i]; sidx < a.long_seg0[i + 1]; ++sidx) {
                const P p = *reinterpret_cast<const P*>(a.segpart + (size_t)sidx * a.ldv + L.c0);
#pragma unroll
                for (int q = 0; q < N; ++q) acc[q] += p.get(q);
            }
            epilogue<T, CL>(a, r, L.c0, acc, ops, dots);
        }
    }
    if (CL || a.mode >= 2) return;
    cta_partials<T, G>(a, L, dots);
}

struct ReduceArgs {
    int nslots;
    int step0;
    int nblocks[kSlots];
    int act[kSlots];
};

// One warp per (slot, kind, column): lane l adds CTAs l, l+32, ... in order, then
// a fixed shuffle tree; the summation order never depends on timing.
__global__ void reduce_partials_kernel(const double* __restrict__ part, int max_blocks, int ldv,
                                       ReduceArgs ra, double* __restrict__ dots, int B)
{
    const int slot = blockIdx.y;
    const int act = ra.act[slot];
    const int lane = threadIdx.x & 31;
    const int idx = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    if (idx >= 2 * act) return;
    const int kind = idx / act, c = idx % act;
    const double* p = part + (size_t)slot * max_blocks * 2 * ldv + (size_t)kind * ldv + c;
    double s = 0.0;
    const int nb = ra.nblocks[slot];
    for (int b = lane; b < nb; b += 32) s += p[(size_t)b * 2 * ldv];
#pragma unroll
    for (int o = 16; o; o >>= 1) s += __shfl_down_sync(0xFFFFFFFFu, s, o);
    if (lane == 0) dots[(size_t)(ra.step0 + slot) * 2 * B + (size_t)kind * B + c] = s;
}

// V_0 = z: row i of a relabelled operator holds the probe entry of original
// row orig[i].
template <typename T>
__global__ void init_probes_kernel(T* v0, int64_t d, int ldv, int B, const int64_t* __restrict__ ids,
                                   uint64_t seedmix, const int32_t* __restrict__ orig)
{
    const int64_t total = d * (int64_t)ldv;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t i = e / ldv;
        const int c = (int)(e % ldv);
        T z = T(0);
        if (c < B) z = probe_negative(seedmix, (uint64_t)ids[c], (uint64_t)(orig ? orig[i] : i)) ? T(-1) : T(1);
        put_entry(v0, (size_t)(e - c), c, z);
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

// Launch the step (and, with long rows, the segment kernel after it).  The
// CTA partials of the two kernels sit next to each other in `part`.
// Resident CTAs per SM of one instance of the step kernel.
template <typename T, int G>
int resident_ctas()
{
    static const int occ = [] {
        int o = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&o, cheb_step_kernel<T, G, false>, kThreads, 0) !=
            cudaSuccess) {
            cudaGetLastError();
            o = 0;
        }
        return o;
    }();
    return occ;
}

template <typename T, int G>
int launch_step_g(StepArgs<T> a, int max_main, int max_long, int num_sms, int* nblocks_out, cudaStream_t s)
{
    const int gpb = kThreads / G;
    const long long items = (a.nch + a.nseg) * (long long)a.nchunks;
    const int occ = resident_ctas<T, G>();
    if (occ > 0) max_main = std::min(max_main, occ * num_sms);   // one resident wave
    int nb = (int)std::max<long long>(1, std::min<long long>((items + gpb - 1) / gpb, max_main));
    if ((long long)nb * gpb < a.nchunks) nb = (a.nchunks + gpb - 1) / gpb;
    {
        ProfScope ps(a.mode == 2 ? "gram_spmm" : (a.mode == 3 ? "clenshaw_step" : "cheb_step"), s);
        if (a.mode == 3) cheb_step_kernel<T, G, true><<<nb, kThreads, 0, s>>>(a);
        else cheb_step_kernel<T, G, false><<<nb, kThreads, 0, s>>>(a);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    int nl = 0;
    if (a.nlong > 0) {
        const long long litems = (long long)a.nlong * a.nchunks;
        nl = (int)std::max<long long>(1, std::min<long long>((litems + gpb - 1) / gpb, max_long));
        if ((long long)nl * gpb < a.nchunks) nl = (a.nchunks + gpb - 1) / gpb;
        StepArgs<T> b = a;
        if (b.partials) b.partials += (size_t)nb * 2 * a.ldv;
        ProfScope ps(a.mode == 2 ? "gram_spmm_long" : (a.mode == 3 ? "clenshaw_step_long" : "cheb_step_long"), s);
        if (a.mode == 3) cheb_long_kernel<T, G, true><<<nl, kThreads, 0, s>>>(b);
        else cheb_long_kernel<T, G, false><<<nl, kThreads, 0, s>>>(b);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    *nblocks_out = nb + nl;
    return MLT_OK;
}

template <typename T>
int launch_step(int G, const StepArgs<T>& a, int max_main, int max_long, int num_sms, int* nb, cudaStream_t s)
{
    switch (G) {
    case 1: return launch_step_g<T, 1>(a, max_main, max_long, num_sms, nb, s);
    case 2: return launch_step_g<T, 2>(a, max_main, max_long, num_sms, nb, s);
    case 4: return launch_step_g<T, 4>(a, max_main, max_long, num_sms, nb, s);
    case 8: return launch_step_g<T, 8>(a, max_main, max_long, num_sms, nb, s);
    case 16: return launch_step_g<T, 16>(a, max_main, max_long, num_sms, nb, s);
    default: return launch_step_g<T, 32>(a, max_main, max_long, num_sms, nb, s);
    }
}

template <typename T>
void set_split(StepArgs<T>& a, const SpmmPlan& P, T* segpart)
{
    a.nch = P.nch;
    a.Uc = P.Uc;
    a.Ul = P.Ul;
    a.nseg = P.nseg;
    a.nlong = P.nlong;
    a.crow = P.crow;
    a.seg_row = P.seg_row;
    a.seg_k0 = P.seg_k0;
    a.long_rows = P.long_rows;
    a.long_seg0 = P.long_seg0;
    a.seg_order = StepTuning<T>::kWindowSegs ? P.seg_order : nullptr;
    a.segpart = segpart;
}

// State shared by the recurrence steps of one probe group.
struct GroupCtx {
    bool gram;
    const int32_t* orig;    // relabelled operator (MLT_REORDER): original row ids, else null
    int64_t d;
    int ldv;
    double alpha, beta;
    uint64_t seedmix;
    double* part;
    double* dots;
    int max_main, max_long, max_blocks;
    ReduceArgs ra;
};

// Recurrence steps k0 <= k < k1 in precision T: V[k & 1] holds V_k and
// V[(k + 1) & 1] holds V_{k-1} on entry to step k.
template <typename T>
int run_steps(mlt_matrix* M, const MomentPlan& plan, GroupCtx& g, int k0, int k1, T* const* V, T* W,
              T* segpart, cudaStream_t s)
{
    constexpr int N = Lanes<T>::N;
    const DevCSR& A = g.orig ? M->P : M->A;
    const DevCSR& AT = M->AT;
    SpmmPlan& planA = g.orig ? M->plan_P : M->plan_A;
    const T* valA = vals_of<T>(A);
    const T* valAT = vals_of<T>(AT);
    int rc;
    for (int k = k0; k < k1; ++k) {
        const int act = plan.act[k];
        const int nvec = (act + N - 1) / N;
        const int G = pow2_at_least(std::min(nvec, 32));
        const int nchunks = (nvec + G - 1) / G;
        T* cur = V[k & 1];
        T* out = V[(k + 1) & 1];
        StepArgs<T> sa{};
        sa.ldv = g.ldv;
        sa.nvec = nvec;
        sa.nchunks = nchunks;
        sa.alpha = (T)g.alpha;
        sa.beta = (T)g.beta;
        sa.direct = plan.direct;
        sa.B = plan.B;
        sa.seedmix = g.seedmix;
        sa.ids = plan.ids_dev;
        sa.orig = g.orig;
        int nb = 0;
        if (g.gram) {
            StepArgs<T> pa = sa;
            pa.rowptr = A.rowptr; pa.col = A.col; pa.val = valA; pa.nrows = A.nrows;
            pa.vgather = cur; pa.vcur = nullptr; pa.vprev_out = W; pa.mode = 2;
            pa.partials = nullptr;
            set_split(pa, M->plan_A, segpart);
            if ((rc = launch_step<T>(G, pa, g.max_main, g.max_long, M->num_sms, &nb, s))) return rc;
            sa.rowptr = AT.rowptr; sa.col = AT.col; sa.val = valAT; sa.nrows = AT.nrows;
            sa.vgather = W;
            set_split(sa, M->plan_AT, segpart);
        } else {
            sa.rowptr = A.rowptr; sa.col = A.col; sa.val = valA; sa.nrows = A.nrows;
            sa.vgather = cur;
            set_split(sa, planA, segpart);
        }
        sa.vcur = cur;
        sa.vprev_out = out;
        sa.mode = (k == 0) ? 0 : 1;
        ReduceArgs& ra = g.ra;
        const int slot = k - ra.step0;
        sa.partials = g.part + (size_t)slot * g.max_blocks * 2 * g.ldv;
        if ((rc = launch_step<T>(G, sa, g.max_main, g.max_long, M->num_sms, &nb, s))) return rc;
        ra.nblocks[slot] = nb;
        ra.act[slot] = act;
        ra.nslots = slot + 1;
        if (ra.nslots == kSlots || k == plan.K - 1) {
            int amax = 0;
            for (int i = 0; i < ra.nslots; ++i) amax = std::max(amax, ra.act[i]);
            dim3 grid((2 * amax + 3) / 4, ra.nslots);
            ProfScope ps("reduce_partials", s);
            reduce_partials_kernel<<<grid, 128, 0, s>>>(g.part, g.max_blocks, g.ldv, ra, g.dots, plan.B);
            MLT_CUDA_TRY(cudaGetLastError());
            ra.step0 = k + 1;
            ra.nslots = 0;
        }
    }
    return MLT_OK;
}

__global__ void widen_kernel(const float* __restrict__ in, double* __restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

// One probe group: steps [0, ks) in FP32 (when the group starts in FP32) and
// [ks, K) in FP64; ks = 0 is all FP64, ks >= K all FP32.  At the switch the
// two live vectors V_k, V_{k-1} are widened to FP64 and the recurrence goes on.
int run_group(mlt_matrix* M, const MomentPlan& plan, int ks, double a, double b, uint64_t seed,
              double* mu_dev, int64_t ld_mu, int* err_flag, cudaStream_t s, bool alloc_only)
{
    GroupCtx g;
    g.gram = (M->flags & MLT_GRAM) != 0;
    g.orig = M->perm;
    g.d = plan.dim;
    g.ldv = plan.ldv;
    ks = std::max(0, std::min(ks, plan.K));
    const bool f32 = ks > 0;
    const bool f64 = ks < plan.K || !f32;
    const size_t n = (size_t)g.d * g.ldv;
    const size_t wrows = g.gram ? (size_t)M->A.nrows * g.ldv : 0;
    int rc;
    if ((rc = ensure_spmm_plan(M, g.orig ? M->P : M->A, g.orig ? M->plan_P : M->plan_A, s))) return rc;
    if (g.gram && (rc = ensure_spmm_plan(M, M->AT, M->plan_AT, s))) return rc;
    if (f32 && (rc = ensure_fp32_values(M, s))) return rc;
    // V buffers: FP32 pair in ws_v (when used), FP64 pair in ws_v (all-FP64) or ws_v2 (mixed)
    float* Vf[2] = {nullptr, nullptr};
    double* Vd[2] = {nullptr, nullptr};
    if (f32) {
        if ((rc = M->ws_v[0].ensure(n * sizeof(float), s)) || (rc = M->ws_v[1].ensure(n * sizeof(float), s))) return rc;
        Vf[0] = M->ws_v[0].as<float>();
        Vf[1] = M->ws_v[1].as<float>();
    }
    if (f64) {
        DevBuf* vb = f32 ? M->ws_v2 : M->ws_v;
        if ((rc = vb[0].ensure(n * sizeof(double), s)) || (rc = vb[1].ensure(n * sizeof(double), s))) return rc;
        Vd[0] = vb[0].as<double>();
        Vd[1] = vb[1].as<double>();
    }
    const size_t tsz = f64 ? sizeof(double) : sizeof(float);
    if (g.gram && (rc = M->ws_w.ensure(wrows * tsz, s))) return rc;
    const int64_t nseg = std::max((g.orig ? M->plan_P : M->plan_A).nseg, g.gram ? M->plan_AT.nseg : (int64_t)0);
    if ((rc = M->ws_seg.ensure((size_t)std::max<int64_t>(nseg, 1) * g.ldv * tsz, s))) return rc;
    g.max_main = 8 * M->num_sms;
    g.max_long = 2 * M->num_sms;
    g.max_blocks = g.max_main + g.max_long;
    if ((rc = M->ws_part.ensure((size_t)kSlots * g.max_blocks * 2 * g.ldv * sizeof(double), s))) return rc;
    if ((rc = M->ws_dots.ensure((size_t)std::max(plan.K, 1) * 2 * plan.B * sizeof(double), s))) return rc;
    g.part = M->ws_part.as<double>();
    g.dots = M->ws_dots.as<double>();
    g.seedmix = seed * kGolden;
    g.ra = ReduceArgs{};
    // At = alpha A + beta I; the stored entries carry `scale` (squared for X^T X).
    const double sc = g.gram ? M->scale * M->scale : M->scale;
    g.alpha = 2.0 / (b - a) * sc;
    g.beta = -(a + b) / (b - a);
    if (alloc_only) return MLT_OK;
    {
        const int nb = (int)std::min<int64_t>(((int64_t)n + 255) / 256, 16LL * M->num_sms);
        ProfScope ps("init_probes", s);
        if (f32) init_probes_kernel<float><<<std::max(nb, 1), 256, 0, s>>>(Vf[0], g.d, g.ldv, plan.B, plan.ids_dev, g.seedmix, g.orig);
        else init_probes_kernel<double><<<std::max(nb, 1), 256, 0, s>>>(Vd[0], g.d, g.ldv, plan.B, plan.ids_dev, g.seedmix, g.orig);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    if (f32) {
        if ((rc = run_steps<float>(M, plan, g, 0, ks, Vf, M->ws_w.as<float>(), M->ws_seg.as<float>(), s))) return rc;
    }
    if (f32 && f64 && ks < plan.K) {
        const int nb = (int)std::min<int64_t>(((int64_t)n + 255) / 256, 16LL * M->num_sms);
        ProfScope ps("widen_vectors", s);
        widen_kernel<<<std::max(nb, 1), 256, 0, s>>>(Vf[0], Vd[0], (int64_t)n);
        widen_kernel<<<std::max(nb, 1), 256, 0, s>>>(Vf[1], Vd[1], (int64_t)n);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    if (f64) {
        if ((rc = run_steps<double>(M, plan, g, f32 ? ks : 0, plan.K, Vd, M->ws_w.as<double>(),
                                    M->ws_seg.as<double>(), s))) return rc;
    }
    {
        dim3 grid((unsigned)std::min<int64_t>((ld_mu + 127) / 128, 64), plan.B);
        ProfScope ps("finalize_moments", s);
        finalize_moments_kernel<<<grid, 128, 0, s>>>(g.dots, plan.B, plan.deg_dev, plan.row_dev, mu_dev,
                                                     ld_mu, (double)g.d, plan.direct, err_flag);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    return MLT_OK;
}

// One probe group in double-float arithmetic throughout (MLT_PREC_DF64): the
// steps of run_group with df64 vectors, SpMM and per-thread dot products, the
// CTA partials and everything after them in FP64.
int run_group_df(mlt_matrix* M, const MomentPlan& plan, double a, double b, uint64_t seed, double* mu_dev,
                 int64_t ld_mu, int* err_flag, cudaStream_t s, bool alloc_only)
{
    GroupCtx g;
    g.gram = (M->flags & MLT_GRAM) != 0;
    g.orig = M->perm;
    g.d = plan.dim;
    g.ldv = plan.ldv;
    const size_t n = (size_t)g.d * g.ldv;
    const size_t wrows = g.gram ? (size_t)M->A.nrows * g.ldv : 0;
    int rc;
    if ((rc = ensure_spmm_plan(M, g.orig ? M->P : M->A, g.orig ? M->plan_P : M->plan_A, s))) return rc;
    if (g.gram && (rc = ensure_spmm_plan(M, M->AT, M->plan_AT, s))) return rc;
    if ((rc = ensure_df_values(M, s))) return rc;
    if ((rc = M->ws_v[0].ensure(n * sizeof(df64), s)) || (rc = M->ws_v[1].ensure(n * sizeof(df64), s))) return rc;
    df64* V[2] = {M->ws_v[0].as<df64>(), M->ws_v[1].as<df64>()};
    if (g.gram && (rc = M->ws_w.ensure(wrows * sizeof(df64), s))) return rc;
    const int64_t nseg = std::max((g.orig ? M->plan_P : M->plan_A).nseg, g.gram ? M->plan_AT.nseg : (int64_t)0);
    if ((rc = M->ws_seg.ensure((size_t)std::max<int64_t>(nseg, 1) * g.ldv * sizeof(df64), s))) return rc;
    g.max_main = 8 * M->num_sms;
    g.max_long = 2 * M->num_sms;
    g.max_blocks = g.max_main + g.max_long;
    if ((rc = M->ws_part.ensure((size_t)kSlots * g.max_blocks * 2 * g.ldv * sizeof(double), s))) return rc;
    if ((rc = M->ws_dots.ensure((size_t)std::max(plan.K, 1) * 2 * plan.B * sizeof(double), s))) return rc;
    g.part = M->ws_part.as<double>();
    g.dots = M->ws_dots.as<double>();
    g.seedmix = seed * kGolden;
    g.ra = ReduceArgs{};
    const double sc = g.gram ? M->scale * M->scale : M->scale;
    g.alpha = 2.0 / (b - a) * sc;
    g.beta = -(a + b) / (b - a);
    if (alloc_only) return MLT_OK;
    {
        const int nb = (int)std::min<int64_t>(((int64_t)n + 255) / 256, 16LL * M->num_sms);
        ProfScope ps("init_probes", s);
        init_probes_kernel<df64><<<std::max(nb, 1), 256, 0, s>>>(V[0], g.d, g.ldv, plan.B, plan.ids_dev, g.seedmix, g.orig);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    if ((rc = run_steps<df64>(M, plan, g, 0, plan.K, V, M->ws_w.as<df64>(), M->ws_seg.as<df64>(), s))) return rc;
    {
        dim3 grid((unsigned)std::min<int64_t>((ld_mu + 127) / 128, 64), plan.B);
        ProfScope ps("finalize_moments", s);
        finalize_moments_kernel<<<grid, 128, 0, s>>>(g.dots, plan.B, plan.deg_dev, plan.row_dev, mu_dev, ld_mu,
                                                     (double)g.d, plan.direct, err_flag);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    return MLT_OK;
}

// Matrix values as double-float pairs, entry by entry (values are read one
// entry at a time, not as vector slices).
__global__ void to_df_values_kernel(const double* __restrict__ in, df64* __restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = df64(in[i]);
}

// In place: the n (even) doubles at v become n double-float entries in the
// slice layout of Pack<df64, 2>; one thread per pair reads both before writing.
__global__ void to_df_kernel(double* v, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n / 2;
         i += (int64_t)gridDim.x * blockDim.x) {
        const double2 x = reinterpret_cast<const double2*>(v)[i];
        const df64 p(x.x), q(x.y);
        reinterpret_cast<float4*>(v)[i] = make_float4(p.hi, q.hi, p.lo, q.lo);
    }
}

// out[i] = coef * x[i] over n elements (x null: zeros).
template <typename T>
__global__ void scaled_copy_kernel(T* __restrict__ out, const T* __restrict__ x, T coef, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = x ? coef * x[i] : T(0);
}

// The context of FP64 steps over an explicit block of `cols` vectors with row
// stride ldv (buffers sized, map At = alpha A + beta I set).
int block_ctx(mlt_matrix* M, int ldv, int cols, int K, double a, double b, GroupCtx& g, cudaStream_t s)
{
    g.gram = (M->flags & MLT_GRAM) != 0;
    g.orig = nullptr;   // explicit vector blocks are in original row order
    g.d = g.gram ? M->A.ncols : M->A.nrows;
    g.ldv = ldv;
    int rc;
    if ((rc = ensure_spmm_plan(M, M->A, M->plan_A, s))) return rc;
    if (g.gram && (rc = ensure_spmm_plan(M, M->AT, M->plan_AT, s))) return rc;
    if (g.gram && (rc = M->ws_w.ensure((size_t)M->A.nrows * ldv * sizeof(double), s))) return rc;
    const int64_t nseg = std::max(M->plan_A.nseg, g.gram ? M->plan_AT.nseg : (int64_t)0);
    if ((rc = M->ws_seg.ensure((size_t)std::max<int64_t>(nseg, 1) * ldv * sizeof(double), s))) return rc;
    g.max_main = 8 * M->num_sms;
    g.max_long = 2 * M->num_sms;
    g.max_blocks = g.max_main + g.max_long;
    if ((rc = M->ws_part.ensure((size_t)kSlots * g.max_blocks * 2 * ldv * sizeof(double), s))) return rc;
    if ((rc = M->ws_dots.ensure((size_t)std::max(K, 1) * 2 * cols * sizeof(double), s))) return rc;
    g.part = M->ws_part.as<double>();
    g.dots = M->ws_dots.as<double>();
    g.seedmix = 0;
    g.ra = ReduceArgs{};
    const double sc = g.gram ? M->scale * M->scale : M->scale;
    g.alpha = 2.0 / (b - a) * sc;
    g.beta = -(a + b) / (b - a);
    return MLT_OK;
}

}  // namespace

// Y = p(At) X by Clenshaw's recurrence for p = sum_k c_k T_k (in FP64, or in
// FP32 with the handle's FP32 values): b_{n+1} = 0,
// b_n = c_n X, b_k = 2 At b_{k+1} - b_{k+2} + c_k X (k = n-1 .. 1), and
// p(At) X = At b_1 - b_2 + c_0 X: n operator applications.  b_j lives in
// P[(n + 1 - j) & 1], so each step overwrites b_{k+2} in place.
template <typename T>
int poly_apply_block_t(mlt_matrix* M, double a, double b, const double* c, int n, const T* X, T* Y, int ldv,
                       int ncols, T* P0, T* P1, cudaStream_t s)
{
    GroupCtx g;
    int rc;
    if ((rc = block_ctx(M, ldv, ncols, 1, a, b, g, s))) return rc;
    if (std::is_same<T, float>::value && (rc = ensure_fp32_values(M, s))) return rc;
    if (std::is_same<T, df64>::value && (rc = ensure_df_values(M, s))) return rc;
    const T* valA = vals_of<T>(M->A);
    const T* valAT = vals_of<T>(M->AT);
    const int64_t total = g.d * (int64_t)ldv;
    const int nbk = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 16LL * M->num_sms));
    T* P[2] = {P0, P1};
    {
        ProfScope ps("clenshaw_init", s);
        scaled_copy_kernel<T><<<nbk, 256, 0, s>>>(P[0], nullptr, T(0), total);
        scaled_copy_kernel<T><<<nbk, 256, 0, s>>>(P[1], X, (T)c[n], total);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    const int nvec = (ncols + Lanes<T>::N - 1) / Lanes<T>::N;
    const int G = pow2_at_least(std::min(nvec, 32));
    const DevCSR& A = M->A;
    const DevCSR& AT = M->AT;
    for (int k = n - 1; k >= 0; --k) {
        T* cur = P[(n - k) & 1];               // b_{k+1}
        T* out = P[(n + 1 - k) & 1];           // in: b_{k+2}; out: b_k (or the result at k = 0)
        StepArgs<T> sa{};
        sa.ldv = ldv;
        sa.nvec = nvec;
        sa.nchunks = (nvec + G - 1) / G;
        sa.alpha = (T)g.alpha;
        sa.beta = (T)g.beta;
        sa.B = ncols;
        int nb = 0;
        if (g.gram) {
            StepArgs<T> pa = sa;
            pa.rowptr = A.rowptr; pa.col = A.col; pa.val = valA; pa.nrows = A.nrows;
            pa.vgather = cur; pa.vcur = nullptr; pa.vprev_out = M->ws_w.as<T>(); pa.mode = 2;
            set_split(pa, M->plan_A, M->ws_seg.as<T>());
            if ((rc = launch_step<T>(G, pa, g.max_main, g.max_long, M->num_sms, &nb, s))) return rc;
            sa.rowptr = AT.rowptr; sa.col = AT.col; sa.val = valAT; sa.nrows = AT.nrows;
            sa.vgather = M->ws_w.as<T>();
            set_split(sa, M->plan_AT, M->ws_seg.as<T>());
        } else {
            sa.rowptr = A.rowptr; sa.col = A.col; sa.val = valA; sa.nrows = A.nrows;
            sa.vgather = cur;
            set_split(sa, M->plan_A, M->ws_seg.as<T>());
        }
        sa.vcur = cur;
        sa.vprev_out = out;
        sa.mode = 3;
        sa.addv = X;
        sa.coef = (T)c[k];
        sa.m1 = k > 0 ? T(2) : T(1);
        if ((rc = launch_step<T>(G, sa, g.max_main, g.max_long, M->num_sms, &nb, s))) return rc;
    }
    T* res = P[(n + 1) & 1];
    if (res != Y) MLT_CUDA_TRY(cudaMemcpyAsync(Y, res, (size_t)total * sizeof(T), cudaMemcpyDeviceToDevice, s));
    return MLT_OK;
}

int poly_apply_block(mlt_matrix* M, double a, double b, const double* c, int n, const double* X, double* Y, int ldv,
                     int ncols, double* P0, double* P1, cudaStream_t s)
{
    return poly_apply_block_t<double>(M, a, b, c, n, X, Y, ldv, ncols, P0, P1, s);
}

int poly_apply_block_f32(mlt_matrix* M, double a, double b, const double* c, int n, const float* X, float* Y,
                         int ldv, int ncols, float* P0, float* P1, cudaStream_t s)
{
    return poly_apply_block_t<float>(M, a, b, c, n, X, Y, ldv, ncols, P0, P1, s);
}

// Doubling moments of an explicit FP64 block: V0 holds the start vectors (row
// stride ldv, columns >= cols zero) and V1 is scratch of the same size, both
// overwritten; with df the steps run in double-float pairs.  After K steps dots[k][0][c] = V_{k+1}.V_{k+1} and
// dots[k][1][c] = V_{k+1}.V_k for column c (device, in the handle's scratch).
int moments_block(mlt_matrix* M, double a, double b, double* V0, double* V1, int ldv, int cols, int K,
                  const double** dots_dev, bool df, cudaStream_t s)
{
    GroupCtx g;
    int rc;
    if ((rc = block_ctx(M, ldv, cols, K, a, b, g, s))) return rc;
    std::vector<int> act(std::max(K, 1), cols);
    MomentPlan plan{};
    plan.dim = g.d;
    plan.B = cols;
    plan.ldv = ldv;
    plan.K = K;
    plan.act = act.data();
    plan.direct = 0;
    if (df) {
        // the start block becomes double-float pairs in place (both 8 bytes an entry)
        if ((rc = ensure_df_values(M, s))) return rc;
        const int64_t n = g.d * (int64_t)ldv;
        const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16LL * M->num_sms));
        if (ldv & 1) return MLT_EINVAL;
        df64* W0 = reinterpret_cast<df64*>(V0);
        {
            ProfScope ps("to_df", s);
            to_df_kernel<<<nb, 256, 0, s>>>(V0, n);
        }
        MLT_CUDA_TRY(cudaGetLastError());
        df64* V[2] = {W0, reinterpret_cast<df64*>(V1)};
        if ((rc = run_steps<df64>(M, plan, g, 0, K, V, M->ws_w.as<df64>(), M->ws_seg.as<df64>(), s))) return rc;
    } else {
        double* V[2] = {V0, V1};
        if ((rc = run_steps<double>(M, plan, g, 0, K, V, M->ws_w.as<double>(), M->ws_seg.as<double>(), s)))
            return rc;
    }
    *dots_dev = g.dots;
    return MLT_OK;
}

// The first column of each segment.
__global__ void seg_first_col_kernel(const int32_t* __restrict__ col, const int64_t* __restrict__ k0, int64_t n,
                                     int32_t* __restrict__ out)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        out[i] = col[k0[i]];
}

// Build the fixed work split of one CSR operand (once per matrix): chunk size
// Uc from the unit count so that there are a few dozen chunks per SM, the row
// holding the first unit of every chunk, and the segment table of rows longer
// than Uc.  Computed on the host from a copy of rowptr.
//
// Segments are dealt out in the order of their first column, in windows of
// kSegWindow columns (row order within a window).  Where a row's columns are
// sorted, the segments in flight at any moment gather from one narrow band of
// columns, and a vector row that several long rows share is read from L2
// rather than DRAM by all but the first.  (The relabelled operator keeps each
// row's entries in their original order, so there the bands are wider; the
// order still measured 3-4% faster for FP32 and double-float steps on the
// scale-22 graph.)  The order only decides when a segment runs; its partial
// product, and the order in which a row's segments are added, do not change.
int ensure_spmm_plan(mlt_matrix* M, const DevCSR& C, SpmmPlan& P, cudaStream_t s)
{
    if (P.ready) return MLT_OK;
    const int64_t n = C.nrows;
    std::vector<int64_t> rp(n + 1);
    MLT_CUDA_TRY(cudaMemcpyAsync(rp.data(), C.rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaStreamSynchronize(s));
    // about kChunksPerSm chunks per SM (at least 8 units each, at most 4096):
    // with the resident grid dealing them round-robin, the rows being worked
    // on at any moment form a band of about 1/(kChunksPerSm/32) of the matrix
    const int64_t units = C.nnz + kRowCost * n;
    int64_t Uc = units / (kChunksPerSm * M->num_sms);
    Uc = std::max<int64_t>(8, std::min<int64_t>(4096, Uc));
    const int64_t Ul = std::max<int64_t>(Uc, kLongRow);
    const int64_t nch = std::max<int64_t>(1, (units + Uc - 1) / Uc);
    std::vector<int64_t> crow(nch);
    {
        int64_t r = 0;
        for (int64_t c = 0; c < nch; ++c) {
            const int64_t u = c * Uc;
            while (r + 1 < n && rp[r + 1] + kRowCost * (r + 1) <= u) ++r;
            crow[c] = r;
        }
    }
    std::vector<int32_t> seg_row, long_rows;
    std::vector<int64_t> seg_k0, long_seg0;
    for (int64_t r = 0; r < n; ++r) {
        const int64_t deg = rp[r + 1] - rp[r];
        if (deg <= Ul) continue;
        long_rows.push_back((int32_t)r);
        long_seg0.push_back((int64_t)seg_row.size());
        for (int64_t k0 = rp[r]; k0 < rp[r + 1]; k0 += Ul) {
            seg_row.push_back((int32_t)r);
            seg_k0.push_back(k0);
        }
    }
    long_seg0.push_back((int64_t)seg_row.size());
    const int64_t nseg = (int64_t)seg_row.size();
    const int nlong = (int)long_rows.size();
    const size_t bytes = nch * sizeof(int64_t) + nseg * (sizeof(int64_t) + 2 * sizeof(int32_t)) +
                         (nlong + 1) * sizeof(int64_t) + nlong * sizeof(int32_t) + 64;
    char* mem = nullptr;
    if (pool_malloc((void**)&mem, bytes, s) != cudaSuccess) {
        cudaGetLastError();
        return fail(MLT_ENOMEM, "device allocation (work split) failed");
    }
    P.mem = mem;
    P.crow = reinterpret_cast<int64_t*>(mem);
    P.seg_k0 = P.crow + nch;
    P.long_seg0 = P.seg_k0 + nseg;
    P.seg_row = reinterpret_cast<int32_t*>(P.long_seg0 + nlong + 1);
    P.long_rows = P.seg_row + nseg;
    P.seg_order = P.long_rows + nlong;
    MLT_CUDA_TRY(cudaMemcpyAsync(P.crow, crow.data(), nch * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    if (nseg) {
        MLT_CUDA_TRY(cudaMemcpyAsync(P.seg_k0, seg_k0.data(), nseg * sizeof(int64_t), cudaMemcpyHostToDevice, s));
        MLT_CUDA_TRY(cudaMemcpyAsync(P.seg_row, seg_row.data(), nseg * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    MLT_CUDA_TRY(cudaMemcpyAsync(P.long_seg0, long_seg0.data(), (nlong + 1) * sizeof(int64_t),
                                 cudaMemcpyHostToDevice, s));
    if (nlong)
        MLT_CUDA_TRY(cudaMemcpyAsync(P.long_rows, long_rows.data(), nlong * sizeof(int32_t),
                                     cudaMemcpyHostToDevice, s));
    if (nseg) {
        std::vector<int32_t> first(nseg), order(nseg);
        const int nb = (int)std::min<int64_t>((nseg + 255) / 256, 16LL * M->num_sms);
        seg_first_col_kernel<<<nb, 256, 0, s>>>(C.col, P.seg_k0, nseg, P.seg_order);
        MLT_CUDA_TRY(cudaGetLastError());
        MLT_CUDA_TRY(cudaMemcpyAsync(first.data(), P.seg_order, nseg * sizeof(int32_t), cudaMemcpyDeviceToHost, s));
        MLT_CUDA_TRY(cudaStreamSynchronize(s));
        for (int64_t i = 0; i < nseg; ++i) order[i] = (int32_t)i;
        std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
            return first[x] / kSegWindow < first[y] / kSegWindow;
        });
        MLT_CUDA_TRY(cudaMemcpyAsync(P.seg_order, order.data(), nseg * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    }
    MLT_CUDA_TRY(cudaStreamSynchronize(s));
    P.nch = nch;
    P.Uc = Uc;
    P.Ul = Ul;
    P.nseg = nseg;
    P.nlong = nlong;
    P.ready = true;
    return MLT_OK;
}

// y = C x for one FP64 vector stored with stride 2 (entry i at x[2 i], the
// other slot zero), through the balanced product kernel; the stored values
// are used as they are (the handle's scale is not applied).
int spmv_f64(mlt_matrix* M, const DevCSR& C, SpmmPlan& P, const double* x, double* y, cudaStream_t s)
{
    int rc;
    if ((rc = ensure_spmm_plan(M, C, P, s))) return rc;
    if ((rc = M->ws_seg.ensure((size_t)std::max<int64_t>(P.nseg, 1) * 2 * sizeof(double), s))) return rc;
    StepArgs<double> a{};
    a.rowptr = C.rowptr;
    a.col = C.col;
    a.val = C.val64;
    a.nrows = C.nrows;
    a.ldv = 2;
    a.nvec = 1;
    a.nchunks = 1;
    a.vgather = x;
    a.vcur = nullptr;
    a.vprev_out = y;
    a.mode = 2;
    a.B = 1;
    a.partials = nullptr;
    set_split(a, P, M->ws_seg.as<double>());
    int nb = 0;
    return launch_step<double>(1, a, 8 * M->num_sms, 2 * M->num_sms, M->num_sms, &nb, s);
}

int ensure_df_values(mlt_matrix* M, cudaStream_t s)
{
    auto conv = [&](DevCSR& C, void*& own) -> int {
        if (C.valdf || !C.val64 || C.nnz == 0) return MLT_OK;
        df64* p = nullptr;
        cudaError_t e = pool_malloc((void**)&p, (size_t)C.nnz * sizeof(df64), s);
        if (e != cudaSuccess) return fail(MLT_ENOMEM, "device allocation (double-float values) failed");
        const int nb = (int)std::min<int64_t>((C.nnz + 255) / 256, 16LL * M->num_sms);
        ProfScope ps("to_df", s);
        to_df_values_kernel<<<std::max(nb, 1), 256, 0, s>>>(C.val64, p, C.nnz);
        MLT_CUDA_TRY(cudaGetLastError());
        own = p;
        C.valdf = p;
        return MLT_OK;
    };
    int rc = conv(M->A, M->own_val_df);
    if (rc) return rc;
    if (M->perm && (rc = conv(M->P, M->own_p_val_df))) return rc;
    if (M->flags & MLT_GRAM) rc = conv(M->AT, M->own_t_val_df);
    return rc;
}

int ensure_fp32_values(mlt_matrix* M, cudaStream_t s)
{
    auto conv = [&](DevCSR& C, void*& own) -> int {
        if (C.val32 || !C.val64 || C.nnz == 0) return MLT_OK;
        float* p = nullptr;
        cudaError_t e = pool_malloc((void**)&p, (size_t)C.nnz * sizeof(float), s);
        if (e != cudaSuccess) return fail(MLT_ENOMEM, "device allocation (fp32 values) failed");
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
    if (M->perm && (rc = conv(M->P, M->own_p_val32))) return rc;
    if (M->flags & MLT_GRAM) rc = conv(M->AT, M->own_t_val32);
    return rc;
}

int run_moments_group(mlt_matrix* M, int precision, const MomentPlan& plan, double a, double b,
                      uint64_t seed, double* mu_dev, int64_t ld_mu, int* err_flag, cudaStream_t s,
                      bool alloc_only)
{
    if (precision == MLT_PREC_DF64)
        return run_group_df(M, plan, a, b, seed, mu_dev, ld_mu, err_flag, s, alloc_only);
    // FP64: no FP32 steps; FP32: all steps FP32; mixed: FP32 for the first k steps
    int ks = 0;
    if (precision == MLT_PREC_FP32) ks = plan.K;
    else if ((precision & 0xFF) == MLT_PREC_MIXED) ks = precision >> 8;
    return run_group(M, plan, ks, a, b, seed, mu_dev, ld_mu, err_flag, s, alloc_only);
}

}  // namespace mlt
