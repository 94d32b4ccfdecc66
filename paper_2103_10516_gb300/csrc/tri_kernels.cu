// Exact integer triangle moments (Section 2.1 Example; Section 5.4).
//
// For a block of 128 Rademacher probes and a symmetric 0/1 adjacency matrix A
// with no self-loops, per probe:
//   y  = A z                      (pass 1; |y_i| <= deg_i)
//   x1 = z . y = z^T A z,  x2 = y . y = z^T A^2 z
//   x3 = y^T A y = z^T A^3 z = 2 sum_i y_i sum_{j in N(i), j > i} y_j   (pass 2)
// Pass 2 walks only the upper triangle: the quadratic form is symmetric, so the
// two products of the paper's footnote suffice and half the gathers are saved.
//
// Layout (device):
//   zb     : 4 x uint32 per row, bit t of word w = 1 when z_i of probe 32w+t is -1
//   y8     : 128 x int8 per row (one 128-byte line); the byte -128 is an escape
//            meaning "look in y32", used only where |y_i| > 127
//   y32    : 128 x int32 per "big" row (degree > 127), slot bslot[i]
//   up_ptr : row pointer of the strictly upper triangle, its columns in up_col
// Work split: every row costs kRowCost "units" plus one per entry (all entries
// in pass 1, upper entries in pass 2); the unit axis is cut into chunks of
// kChunk units that warps of a persistent grid take from an atomic counter.
// A row of degree <= kChunk is handled whole by the chunk holding its first
// unit; consecutive such rows are walked as one stream of entries, with the
// row ends of 32 rows at a time held in lanes.  Longer rows are cut at chunk
// edges: pass-1 counts are merged with integer atomics in y32 and finished by
// a per-row kernel; pass 2 is linear in the row sums, so a cut needs no merge.
// All sums are integers (exact, independent of order).
#include <cuda_runtime.h>

#include <algorithm>

#include "mlt_internal.h"
#include "rng.cuh"

namespace mlt {
namespace {

constexpr int kTriThreads = 256;
constexpr int kProbes = 128;
constexpr int kBigDeg = 127;          // rows above this degree get an int32 slot
constexpr int64_t kRowCost = 4;       // units charged per row on top of its entries
constexpr int64_t kChunk = 1024;      // units per dynamically scheduled chunk
constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kScanBlock = 1024;      // elements per CTA of the prefix scan

// zb[i * 4 + w] bit t = 1 when z_i of probe (id0 + 32 w + t) is -1 (0 for
// t >= nb - 32 w).  The 32 bits come from one or two 64-probe hash words.
__global__ void zbits_kernel(int64_t d, uint64_t seedmix, int64_t id0, int nb, uint32_t* __restrict__ zb)
{
    const int64_t total = d * 4;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < total;
         e += (int64_t)gridDim.x * blockDim.x) {
        const uint64_t i = (uint64_t)(e >> 2);
        const int w = (int)(e & 3);
        const int valid = min(32, max(0, nb - 32 * w));
        uint32_t bits = 0;
        if (valid > 0) {
            const uint64_t p0 = (uint64_t)(id0 + 32 * w);
            const int o = (int)(p0 & 63);
            uint64_t v = probe_word(seedmix, p0 >> 6, i) >> o;
            if (o > 32) v |= probe_word(seedmix, (p0 >> 6) + 1, i) << (64 - o);
            bits = (uint32_t)v;
            if (valid < 32) bits &= (1u << valid) - 1u;
        }
        zb[e] = bits;
    }
}

// Per row: first index with col > row, its count of upper entries (into
// upcnt, scanned later into up_ptr), self-loop detection, the bound
// sum_j deg_i deg_j certifying that x3 fits in int64, and slots for big rows
// and long rows (slot order is irrelevant to every result).
__global__ void tri_prepare_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                   int64_t d, int64_t* __restrict__ upper, int64_t* __restrict__ upcnt,
                                   int32_t* __restrict__ bslot, int32_t* __restrict__ longlist,
                                   int* counters /* [0] nbig, [1] nlong, [2] selfloop */, double* bound)
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
                if (c == r) atomicOr(counters + 2, 1);
            }
            const unsigned above = __ballot_sync(kFull, k < end && c > r);
            if (above && first == end) first = base + __ffs(above) - 1;
        }
        for (int o = 16; o; o >>= 1) dsum += __shfl_xor_sync(kFull, dsum, o);
        if (lane == 0) {
            const int64_t deg = end - beg;
            upper[r] = first;
            upcnt[r] = end - first;
            wsum += dsum * (double)deg;
            int32_t s = -1;
            if (deg > kBigDeg) s = atomicAdd(counters + 0, 1);
            bslot[r] = s;
            if (deg > kChunk) longlist[atomicAdd(counters + 1, 1)] = (int32_t)r;
        }
    }
    if (lane == 0 && wsum != 0.0) atomicAdd(bound, wsum);
}

// ---- exclusive prefix scan of int64 counts, in place (three passes) --------

__device__ __forceinline__ int64_t block_inclusive_scan(int64_t v, int64_t* warp_tot)
{
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    for (int o = 1; o < 32; o <<= 1) {
        const int64_t t = __shfl_up_sync(kFull, v, o);
        if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
        int64_t w = lane < (int)(blockDim.x >> 5) ? warp_tot[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            const int64_t t = __shfl_up_sync(kFull, w, o);
            if (lane >= o) w += t;
        }
        warp_tot[lane] = w;
    }
    __syncthreads();
    if (wid > 0) v += warp_tot[wid - 1];
    return v;
}

__global__ void scan_sums_kernel(const int64_t* __restrict__ x, int64_t n, int64_t* __restrict__ bsum)
{
    __shared__ int64_t wt[32];
    const int64_t b0 = (int64_t)blockIdx.x * kScanBlock;
    int64_t s = 0;
    for (int i = 0; i < 4; ++i) {
        const int64_t k = b0 + threadIdx.x * 4 + i;
        if (k < n) s += x[k];
    }
    s = block_inclusive_scan(s, wt);
    if (threadIdx.x == blockDim.x - 1) bsum[blockIdx.x] = s;
}

// bsum[b] -> exclusive prefix over the blocks; total written to *out_total.
__global__ void scan_offsets_kernel(int64_t* __restrict__ bsum, int64_t nb, int64_t* __restrict__ out_total)
{
    __shared__ int64_t wt[32];
    __shared__ int64_t carry;
    if (threadIdx.x == 0) carry = 0;
    __syncthreads();
    for (int64_t base = 0; base < nb; base += blockDim.x) {
        const int64_t k = base + threadIdx.x;
        const int64_t v = k < nb ? bsum[k] : 0;
        const int64_t inc = block_inclusive_scan(v, wt);
        const int64_t c = carry;
        if (k < nb) bsum[k] = c + inc - v;
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) carry = c + inc;
        __syncthreads();
    }
    if (threadIdx.x == 0) *out_total = carry;
}

__global__ void scan_apply_kernel(int64_t* __restrict__ x, int64_t n, const int64_t* __restrict__ boff)
{
    __shared__ int64_t wt[32];
    const int64_t b0 = (int64_t)blockIdx.x * kScanBlock;
    int64_t v[4], s = 0;
    for (int i = 0; i < 4; ++i) {
        const int64_t k = b0 + threadIdx.x * 4 + i;
        v[i] = k < n ? x[k] : 0;
        s += v[i];
    }
    int64_t run = block_inclusive_scan(s, wt) - s + boff[blockIdx.x];
    for (int i = 0; i < 4; ++i) {
        const int64_t k = b0 + threadIdx.x * 4 + i;
        if (k < n) x[k] = run;
        run += v[i];
    }
}

// up_col[up_ptr[r] ...] = the columns of row r above the diagonal.
__global__ void fill_upper_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const int64_t* __restrict__ upper, const int64_t* __restrict__ up_ptr,
                                  int64_t d, int32_t* __restrict__ up_col)
{
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t r = warp; r < d; r += nwarps) {
        const int64_t a = upper[r], b = rowptr[r + 1], o = up_ptr[r];
        for (int64_t k = a + lane; k < b; k += 32) up_col[o + (k - a)] = col[k];
    }
}

// crow[c] = the row whose units hold unit c*kChunk: the largest r with
// ptr[r] + kRowCost*r <= c*kChunk.
__global__ void chunk_rows_kernel(const int64_t* __restrict__ ptr, int64_t d, int64_t nch,
                                  int64_t* __restrict__ crow)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nch;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = c * kChunk;
        int64_t lo = 0, hi = d;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (ptr[mid] + kRowCost * mid <= u) lo = mid;
            else hi = mid;
        }
        crow[c] = lo;
    }
}

// Next chunk for this warp (lane 0 takes it, the warp shares it).
__device__ __forceinline__ int64_t next_chunk(unsigned long long* counter, int lane)
{
    unsigned long long c = 0;
    if (lane == 0) c = atomicAdd(counter, 1ull);
    return (int64_t)__shfl_sync(kFull, c, 0);
}

__global__ void zero_long_rows_kernel(const int32_t* __restrict__ longlist, int nlong,
                                      const int32_t* __restrict__ bslot, int32_t* __restrict__ y32)
{
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < (int64_t)nlong * kProbes;
         e += (int64_t)gridDim.x * blockDim.x) {
        const int r = longlist[e / kProbes];
        y32[(size_t)bslot[r] * kProbes + (e % kProbes)] = 0;
    }
}

// The 4 sign bits of probes 4*lane .. 4*lane+3 at row j.
__device__ __forceinline__ uint32_t sign_nibble(const uint32_t* __restrict__ zb, int64_t j, int lane)
{
    return (__ldg(zb + (size_t)j * 4 + (lane >> 3)) >> ((lane & 7) * 4)) & 0xFu;
}

// Byte q of `packed` counts sign bit q; folded into int counters before it can wrap.
__device__ __forceinline__ void fold(uint32_t& packed, int cnt[4])
{
    cnt[0] += packed & 0xFF;
    cnt[1] += (packed >> 8) & 0xFF;
    cnt[2] += (packed >> 16) & 0xFF;
    cnt[3] += packed >> 24;
    packed = 0;
}

// Negative-sign counts over entries [a, b) of one row, for this lane's 4 probes.
__device__ __forceinline__ void count_negatives(const int32_t* __restrict__ col, int64_t a, int64_t b,
                                                const uint32_t* __restrict__ zb, int lane, int cnt[4])
{
    uint32_t packed = 0;
    for (int64_t base = a; base < b; base += 32) {
        const int64_t k = base + lane;
        const int cj = k < b ? __ldg(col + k) : 0;
        const int n = (int)min((int64_t)32, b - base);
#pragma unroll 8
        for (int t = 0; t < n; ++t)
            packed += (sign_nibble(zb, __shfl_sync(kFull, cj, t), lane) * 0x00204081u) & 0x01010101u;
        fold(packed, cnt);
    }
}

// Store y for probes 4*lane .. 4*lane+3 of row r and add its x1, x2 terms.
__device__ __forceinline__ void store_row(int64_t r, const int yv[4], uint32_t own, int32_t slot,
                                          uint32_t* __restrict__ y8, int32_t* __restrict__ y32, int lane,
                                          long long x1[4], long long x2[4])
{
    uint32_t packed = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        const int v = yv[q];
        const uint32_t byte = (v >= -127 && v <= 127) ? (uint32_t)(v & 0xFF) : 0x80u;
        packed |= byte << (8 * q);
        const long long yq = v;
        x1[q] += ((own >> q) & 1u) ? -yq : yq;
        x2[q] += yq * yq;
    }
    y8[(size_t)r * 32 + lane] = packed;
    if (slot >= 0) *reinterpret_cast<int4*>(y32 + (size_t)slot * kProbes + 4 * lane) =
        make_int4(yv[0], yv[1], yv[2], yv[3]);
}

__device__ __forceinline__ void finish_pass1_row(int64_t r, int deg, int cnt[4], uint32_t own,
                                                 const int32_t* __restrict__ bslot, uint32_t* __restrict__ y8,
                                                 int32_t* __restrict__ y32, int lane, long long x1[4],
                                                 long long x2[4])
{
    if (deg > 0) {
        const int yv[4] = {deg - 2 * cnt[0], deg - 2 * cnt[1], deg - 2 * cnt[2], deg - 2 * cnt[3]};
        store_row(r, yv, own, deg > kBigDeg ? __ldg(bslot + r) : -1, y8, y32, lane, x1, x2);
    }
    cnt[0] = cnt[1] = cnt[2] = cnt[3] = 0;
}

__device__ __forceinline__ void flush_x(long long (*sx)[kProbes], int which, const long long v[4], int lane)
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (v[q]) atomicAdd((unsigned long long*)&sx[which][4 * lane + q], (unsigned long long)v[q]);
}

// Pass 1: y = A z for 128 probes, plus x1 = z.y and x2 = y.y (rows of degree
// <= kChunk; longer rows only accumulate their counts here).
__global__ void __launch_bounds__(kTriThreads) tri_pass1_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t d, int64_t nch,
    const int64_t* __restrict__ crow, const int32_t* __restrict__ bslot,
    const uint32_t* __restrict__ zb, uint32_t* __restrict__ y8, int32_t* __restrict__ y32,
    unsigned long long* __restrict__ xacc, unsigned long long* __restrict__ counter)
{
    __shared__ long long sx[2][kProbes];
    for (int t = threadIdx.x; t < 2 * kProbes; t += blockDim.x) (&sx[0][0])[t] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    long long x1[4] = {0, 0, 0, 0}, x2[4] = {0, 0, 0, 0};
    for (int64_t c = next_chunk(counter, lane); c < nch; c = next_chunk(counter, lane)) {
        const int64_t u0 = c * kChunk, u1 = u0 + kChunk;
        int64_t r = crow[c];
        while (r < d) {
            const int64_t beg = __ldg(rowptr + r);
            const int64_t pr = beg + kRowCost * r;          // first unit of row r
            if (pr >= u1) break;
            const int64_t end = __ldg(rowptr + r + 1);
            const int64_t deg = end - beg;
            if (deg > kChunk) {                             // long row: this chunk's part
                const int64_t e0 = pr + kRowCost;
                const int64_t a = beg + max((int64_t)0, u0 - e0);
                const int64_t b = beg + min(deg, u1 - e0);
                if (a < b) {
                    int cnt[4] = {0, 0, 0, 0};
                    count_negatives(col, a, b, zb, lane, cnt);
                    int32_t* acc = y32 + (size_t)__ldg(bslot + r) * kProbes + 4 * lane;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        if (cnt[q]) atomicAdd(acc + q, cnt[q]);
                }
                ++r;
                continue;
            }
            if (pr < u0) {                                  // belongs to the previous chunk
                ++r;
                continue;
            }
            // rows owned by this chunk: row ends of 32 rows at a time in lanes,
            // then each row's entries with an unrolled loop (no boundary tests)
            for (;;) {
                const int64_t rr = r + lane;
                int a0 = 0, a1 = 0;
                bool ok = false;
                if (rr < d) {
                    const int64_t s0 = __ldg(rowptr + rr), e0 = __ldg(rowptr + rr + 1);
                    a0 = (int)s0;
                    a1 = (int)e0;
                    ok = (s0 + kRowCost * rr < u1) && (e0 - s0 <= kChunk);
                }
                const unsigned okm = __ballot_sync(kFull, ok);
                const int f = (okm == kFull) ? 32 : (__ffs(~okm) - 1);
                for (int cur = 0; cur < f; ++cur) {
                    const int a = __shfl_sync(kFull, a0, cur);
                    const int b = __shfl_sync(kFull, a1, cur);
                    if (a == b) continue;
                    const int64_t row = r + cur;
                    const uint32_t own = sign_nibble(zb, row, lane);   // fetched before the entries
                    int cnt[4] = {0, 0, 0, 0};
                    uint32_t packed = 0;
                    for (int base = a; base < b; base += 32) {
                        const int k = base + lane;
                        const int cj = k < b ? __ldg(col + k) : 0;
                        const int n = min(32, b - base);
#pragma unroll 8
                        for (int t = 0; t < n; ++t)
                            packed += (sign_nibble(zb, __shfl_sync(kFull, cj, t), lane) * 0x00204081u) & 0x01010101u;
                        fold(packed, cnt);
                    }
                    finish_pass1_row(row, b - a, cnt, own, bslot, y8, y32, lane, x1, x2);
                }
                r += f;
                if (f < 32) break;
            }
        }
    }
    flush_x(sx, 0, x1, lane);
    flush_x(sx, 1, x2, lane);
    __syncthreads();
    for (int t = threadIdx.x; t < kProbes; t += blockDim.x) {
        if (sx[0][t]) atomicAdd(xacc + 3 * t + 0, (unsigned long long)sx[0][t]);
        if (sx[1][t]) atomicAdd(xacc + 3 * t + 1, (unsigned long long)sx[1][t]);
    }
}

// Finish long rows: counts -> y, the int8 escapes, and their x1, x2 terms.
__global__ void __launch_bounds__(kTriThreads) tri_long_rows_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ longlist, int nlong,
    const int32_t* __restrict__ bslot, const uint32_t* __restrict__ zb, uint32_t* __restrict__ y8,
    int32_t* __restrict__ y32, unsigned long long* __restrict__ xacc)
{
    __shared__ long long sx[2][kProbes];
    for (int t = threadIdx.x; t < 2 * kProbes; t += blockDim.x) (&sx[0][0])[t] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    long long x1[4] = {0, 0, 0, 0}, x2[4] = {0, 0, 0, 0};
    for (int64_t i = warp; i < nlong; i += nwarps) {
        const int64_t r = longlist[i];
        const int deg = (int)(rowptr[r + 1] - rowptr[r]);
        const int32_t slot = bslot[r];
        const int4 c = *reinterpret_cast<const int4*>(y32 + (size_t)slot * kProbes + 4 * lane);
        const int yv[4] = {deg - 2 * c.x, deg - 2 * c.y, deg - 2 * c.z, deg - 2 * c.w};
        store_row(r, yv, sign_nibble(zb, r, lane), slot, y8, y32, lane, x1, x2);
    }
    flush_x(sx, 0, x1, lane);
    flush_x(sx, 1, x2, lane);
    __syncthreads();
    for (int t = threadIdx.x; t < kProbes; t += blockDim.x) {
        if (sx[0][t]) atomicAdd(xacc + 3 * t + 0, (unsigned long long)sx[0][t]);
        if (sx[1][t]) atomicAdd(xacc + 3 * t + 1, (unsigned long long)sx[1][t]);
    }
}

// Add y of row j (this lane's 4 probes) into s: the int8 bytes are summed
// with dp4a against unit vectors; an escape byte sends the lane to y32.
__device__ __forceinline__ void add_y(int64_t j, const uint32_t* __restrict__ y8,
                                      const int32_t* __restrict__ y32, const int32_t* __restrict__ bslot,
                                      int lane, int s[4])
{
    const uint32_t w = __ldg(y8 + (size_t)j * 32 + lane);
    const uint32_t v = w ^ 0x80808080u;
    if ((v - 0x01010101u) & ~v & 0x80808080u) {
        const int4 t = __ldg(reinterpret_cast<const int4*>(y32 + (size_t)__ldg(bslot + j) * kProbes) + lane);
        s[0] += t.x;
        s[1] += t.y;
        s[2] += t.z;
        s[3] += t.w;
        return;
    }
    s[0] = __dp4a((int)w, 0x00000001, s[0]);
    s[1] = __dp4a((int)w, 0x00000100, s[1]);
    s[2] = __dp4a((int)w, 0x00010000, s[2]);
    s[3] = __dp4a((int)w, 0x01000000, s[3]);
}

// Add an already loaded y8 word of row j into s (escape bytes go to y32).
__device__ __forceinline__ void acc_y(uint32_t w, int64_t j, const int32_t* __restrict__ y32,
                                      const int32_t* __restrict__ bslot, int lane, int s[4])
{
    const uint32_t v = w ^ 0x80808080u;
    if ((v - 0x01010101u) & ~v & 0x80808080u) {
        const int4 t = __ldg(reinterpret_cast<const int4*>(y32 + (size_t)__ldg(bslot + j) * kProbes) + lane);
        s[0] += t.x;
        s[1] += t.y;
        s[2] += t.z;
        s[3] += t.w;
        return;
    }
    s[0] = __dp4a((int)w, 0x00000001, s[0]);
    s[1] = __dp4a((int)w, 0x00000100, s[1]);
    s[2] = __dp4a((int)w, 0x00010000, s[2]);
    s[3] = __dp4a((int)w, 0x01000000, s[3]);
}

// x3 += y_r * s for row r (own = its y8 word), then s = 0.
__device__ __forceinline__ void finish_pass2_row(int64_t r, uint32_t own, int s[4],
                                                 const int32_t* __restrict__ y32,
                                                 const int32_t* __restrict__ bslot, int lane, long long x3[4])
{
    int yi[4] = {0, 0, 0, 0};
    acc_y(own, r, y32, bslot, lane, yi);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        x3[q] += (long long)yi[q] * s[q];
        s[q] = 0;
    }
}

// Pass 2: x3 = 2 sum_i y_i sum_{j in N(i), j > i} y_j over the upper CSR.
__global__ void __launch_bounds__(kTriThreads) tri_pass2_kernel(
    const int64_t* __restrict__ up_ptr, const int32_t* __restrict__ up_col, int64_t d, int64_t nch,
    const int64_t* __restrict__ crow, const int32_t* __restrict__ bslot,
    const uint32_t* __restrict__ y8, const int32_t* __restrict__ y32,
    unsigned long long* __restrict__ xacc, unsigned long long* __restrict__ counter)
{
    __shared__ long long sx[kProbes];
    for (int t = threadIdx.x; t < kProbes; t += blockDim.x) sx[t] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    long long x3[4] = {0, 0, 0, 0};
    for (int64_t c = next_chunk(counter, lane); c < nch; c = next_chunk(counter, lane)) {
        const int64_t u0 = c * kChunk, u1 = u0 + kChunk;
        int64_t r = crow[c];
        while (r < d) {
            const int64_t beg = __ldg(up_ptr + r);
            const int64_t pr = beg + kRowCost * r;
            if (pr >= u1) break;
            const int64_t end = __ldg(up_ptr + r + 1);
            const int64_t deg = end - beg;
            if (deg > kChunk) {                             // long row: this chunk's part
                const int64_t e0 = pr + kRowCost;
                const int64_t a = beg + max((int64_t)0, u0 - e0);
                const int64_t b = beg + min(deg, u1 - e0);
                if (a < b) {
                    int s[4] = {0, 0, 0, 0};
                    for (int64_t base = a; base < b; base += 32) {
                        const int64_t k = base + lane;
                        const int cj = k < b ? __ldg(up_col + k) : 0;
                        const int n = (int)min((int64_t)32, b - base);
#pragma unroll 8
                        for (int t = 0; t < n; ++t) add_y(__shfl_sync(kFull, cj, t), y8, y32, bslot, lane, s);
                    }
                    finish_pass2_row(r, __ldg(y8 + (size_t)r * 32 + lane), s, y32, bslot, lane, x3);
                }
                ++r;
                continue;
            }
            if (pr < u0) {
                ++r;
                continue;
            }
            // rows owned by this chunk: row ends of 32 rows at a time in lanes,
            // then each row's entries with an unrolled loop (no boundary tests)
            for (;;) {
                const int64_t rr = r + lane;
                int a0 = 0, a1 = 0;
                bool ok = false;
                if (rr < d) {
                    const int64_t s0 = __ldg(up_ptr + rr), e0 = __ldg(up_ptr + rr + 1);
                    a0 = (int)s0;
                    a1 = (int)e0;
                    ok = (s0 + kRowCost * rr < u1) && (e0 - s0 <= kChunk);
                }
                const unsigned okm = __ballot_sync(kFull, ok);
                const int f = (okm == kFull) ? 32 : (__ffs(~okm) - 1);
                for (int cur = 0; cur < f; ++cur) {
                    const int a = __shfl_sync(kFull, a0, cur);
                    const int b = __shfl_sync(kFull, a1, cur);
                    if (a == b) continue;
                    const int64_t row = r + cur;
                    const uint32_t own = __ldg(y8 + (size_t)row * 32 + lane);   // fetched before the entries
                    int s[4] = {0, 0, 0, 0};
                    for (int base = a; base < b; base += 32) {
                        const int k = base + lane;
                        const int cj = k < b ? __ldg(up_col + k) : 0;
                        const int n = min(32, b - base);
                        for (int t0 = 0; t0 < n; t0 += 8) {
                            // 8 gathers issued before any is used: the escape branch in
                            // acc_y would otherwise keep one load in flight per warp
                            // (lanes past n read row 0, whose line is harmless to load)
                            int jj[8];
                            uint32_t w[8];
#pragma unroll
                            for (int u = 0; u < 8; ++u) {
                                jj[u] = __shfl_sync(kFull, cj, t0 + u);
                                w[u] = __ldg(y8 + (size_t)jj[u] * 32 + lane);
                            }
#pragma unroll
                            for (int u = 0; u < 8; ++u)
                                if (t0 + u < n) acc_y(w[u], jj[u], y32, bslot, lane, s);
                        }
                    }
                    finish_pass2_row(row, own, s, y32, bslot, lane, x3);
                }
                r += f;
                if (f < 32) break;
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (x3[q]) atomicAdd((unsigned long long*)&sx[4 * lane + q], (unsigned long long)(2 * x3[q]));
    __syncthreads();
    for (int t = threadIdx.x; t < kProbes; t += blockDim.x)
        if (sx[t]) atomicAdd(xacc + 3 * t + 2, (unsigned long long)sx[t]);
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
    const int64_t nnz = M->A.nnz;
    const int64_t nch1 = std::max<int64_t>(1, (nnz + kRowCost * d + kChunk - 1) / kChunk);
    int occ1 = 0, occ2 = 0;
    MLT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, tri_pass1_kernel, kTriThreads, 0));
    MLT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, tri_pass2_kernel, kTriThreads, 0));
    const size_t dd = (size_t)std::max<int64_t>(d, 1);
    const int64_t nsb = (d + kScanBlock - 1) / kScanBlock;
    int rc;
    // upper[d], up_ptr[d+1], crow1[nch1], crow2[nch1], scan sums[nsb], bslot[d], longlist[d], counters
    if ((rc = M->ws_tri.ensure(dd * 8 + (dd + 1) * 8 + 2 * (size_t)nch1 * 8 + (size_t)(nsb + 1) * 8 +
                               dd * 4 * 2 + 1024, s))) return rc;
    char* base = M->ws_tri.as<char>();
    int64_t* upper = reinterpret_cast<int64_t*>(base);
    int64_t* up_ptr = upper + dd;
    int64_t* crow1 = up_ptr + dd + 1;
    int64_t* crow2 = crow1 + nch1;
    int64_t* bsum = crow2 + nch1;
    int32_t* bslot = reinterpret_cast<int32_t*>(bsum + nsb + 1);
    int32_t* longlist = bslot + dd;
    int* counters = reinterpret_cast<int*>(longlist + dd);
    double* bound = reinterpret_cast<double*>(counters + 4);
    unsigned long long* chunk_ctr = reinterpret_cast<unsigned long long*>(bound + 1);
    MLT_CUDA_TRY(cudaMemsetAsync(counters, 0, 4 * sizeof(int) + sizeof(double), s));
    {
        ProfScope ps("tri_prepare", s);
        tri_prepare_kernel<<<grid_for(M->num_sms, d), kTriThreads, 0, s>>>(
            M->A.rowptr, M->A.col, d, upper, up_ptr, bslot, longlist, counters, bound);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    if (d > 0) {
        ProfScope ps("tri_scan", s);
        scan_sums_kernel<<<(unsigned)nsb, 256, 0, s>>>(up_ptr, d, bsum);
        scan_offsets_kernel<<<1, 1024, 0, s>>>(bsum, nsb, up_ptr + d);
        scan_apply_kernel<<<(unsigned)nsb, 256, 0, s>>>(up_ptr, d, bsum);
    } else {
        MLT_CUDA_TRY(cudaMemsetAsync(up_ptr, 0, sizeof(int64_t), s));
    }
    MLT_CUDA_TRY(cudaGetLastError());
    int hc[4] = {0, 0, 0, 0};
    double hb = 0.0;
    int64_t nnz_up = 0;
    MLT_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaMemcpyAsync(&hb, bound, sizeof(double), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaMemcpyAsync(&nnz_up, up_ptr + d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaStreamSynchronize(s));
    M->tri_bound = hb;
    if (hc[2]) {
        M->tri_state = MLT_EINVAL;
        return fail(MLT_EINVAL, "triangle counting needs an adjacency matrix without self-loops");
    }
    if (!(hb < 4611686018427387904.0)) {   // 2^62
        M->tri_state = MLT_ERANGE;
        return fail(MLT_ERANGE, "sum of deg_i*deg_j over edges reaches 2^62: x3 may overflow int64");
    }
    if ((rc = M->ws_upcol.ensure((size_t)std::max<int64_t>(nnz_up, 1) * sizeof(int32_t), s))) return rc;
    int32_t* up_col = M->ws_upcol.as<int32_t>();
    const int64_t nch2 = std::max<int64_t>(1, (nnz_up + kRowCost * d + kChunk - 1) / kChunk);
    {
        ProfScope ps("tri_fill_upper", s);
        fill_upper_kernel<<<grid_for(M->num_sms, d), kTriThreads, 0, s>>>(M->A.rowptr, M->A.col, upper,
                                                                          up_ptr, d, up_col);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    {
        ProfScope ps("tri_chunk_rows", s);
        const int g1 = (int)std::min<int64_t>((nch1 + 255) / 256, 16LL * M->num_sms);
        chunk_rows_kernel<<<std::max(g1, 1), 256, 0, s>>>(M->A.rowptr, d, nch1, crow1);
        const int g2 = (int)std::min<int64_t>((nch2 + 255) / 256, 16LL * M->num_sms);
        chunk_rows_kernel<<<std::max(g2, 1), 256, 0, s>>>(up_ptr, d, nch2, crow2);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    M->upper = upper;
    M->tri.up_ptr = up_ptr;
    M->tri.up_col = up_col;
    M->tri.crow1 = crow1;
    M->tri.crow2 = crow2;
    M->tri.bslot = bslot;
    M->tri.longlist = longlist;
    M->tri.counters = chunk_ctr;
    M->tri.nbig = hc[0];
    M->tri.nlong = hc[1];
    M->tri.nch1 = nch1;
    M->tri.nch2 = nch2;
    M->tri.grid1 = std::max(1, occ1) * M->num_sms;
    M->tri.grid2 = std::max(1, occ2) * M->num_sms;
    M->tri_state = 1;
    return MLT_OK;
}

int tri_block(mlt_matrix* M, uint64_t seed, int64_t id0, int nb, int64_t* x_dev, cudaStream_t s)
{
    const int64_t d = M->A.nrows;
    const auto& T = M->tri;
    int rc;
    const size_t dd = (size_t)std::max<int64_t>(d, 1);
    if ((rc = M->ws_z.ensure(dd * 4 * sizeof(uint32_t), s))) return rc;
    if ((rc = M->ws_y.ensure(dd * kProbes, s))) return rc;
    if ((rc = M->ws_y32.ensure((size_t)std::max(T.nbig, 1) * kProbes * sizeof(int32_t), s))) return rc;
    if ((rc = M->ws_x.ensure((size_t)kProbes * 3 * sizeof(unsigned long long), s))) return rc;
    uint32_t* zb = M->ws_z.as<uint32_t>();
    uint32_t* y8 = M->ws_y.as<uint32_t>();
    int32_t* y32 = M->ws_y32.as<int32_t>();
    unsigned long long* xacc = M->ws_x.as<unsigned long long>();
    MLT_CUDA_TRY(cudaMemsetAsync(xacc, 0, (size_t)kProbes * 3 * sizeof(unsigned long long), s));
    MLT_CUDA_TRY(cudaMemsetAsync(T.counters, 0, 2 * sizeof(unsigned long long), s));
    {
        const int64_t total = d * 4;
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 16LL * M->num_sms));
        ProfScope ps("tri_zbits", s);
        zbits_kernel<<<g, 256, 0, s>>>(d, seed * kGolden, id0, nb, zb);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    if (T.nlong > 0) {
        const int g = (int)std::min<int64_t>(((int64_t)T.nlong * kProbes + 255) / 256, 4LL * M->num_sms);
        ProfScope ps("tri_zero_long", s);
        zero_long_rows_kernel<<<std::max(g, 1), 256, 0, s>>>(T.longlist, T.nlong, T.bslot, y32);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    {
        ProfScope ps("tri_pass1", s);
        tri_pass1_kernel<<<T.grid1, kTriThreads, 0, s>>>(M->A.rowptr, M->A.col, d, T.nch1, T.crow1, T.bslot,
                                                         zb, y8, y32, xacc, T.counters);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    if (T.nlong > 0) {
        const int g = (int)std::min<int64_t>(((int64_t)T.nlong * 32 + kTriThreads - 1) / kTriThreads,
                                             4LL * M->num_sms);
        ProfScope ps("tri_long_rows", s);
        tri_long_rows_kernel<<<std::max(g, 1), kTriThreads, 0, s>>>(M->A.rowptr, T.longlist, T.nlong,
                                                                    T.bslot, zb, y8, y32, xacc);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    {
        ProfScope ps("tri_pass2", s);
        tri_pass2_kernel<<<T.grid2, kTriThreads, 0, s>>>(T.up_ptr, T.up_col, d, T.nch2, T.crow2, T.bslot,
                                                         y8, y32, xacc, T.counters + 1);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    MLT_CUDA_TRY(cudaMemcpyAsync(x_dev, xacc, (size_t)nb * 3 * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    return MLT_OK;
}

}  // namespace mlt
