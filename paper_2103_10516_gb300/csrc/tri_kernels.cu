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
//   zb  : 4 x uint32 per row, bit t of word w = 1 when z_i of probe 32w+t is -1
//   y8  : 128 x int8 per row (one 128-byte line); the byte -128 is an escape
//         meaning "look in y32", used only where |y_i| > 127
//   y32 : 128 x int32 per "big" row (degree > 127), slot bslot[i]
// Work split: every row costs kRowCost "units" plus one per entry; row r
// starts at unit P(r) = rowptr[r] + kRowCost * r.  The unit axis is cut into
// chunks of kChunk units that warps of a persistent grid take from an atomic
// counter, so rows with few entries and rows with many balance alike.  A row
// of degree <= long_deg is handled whole by the chunk holding its first unit;
// longer rows are cut at chunk edges, their pass-1 counts merged with integer
// atomics in y32 and finished by a per-row kernel.  Pass 2 is linear in the
// row sums, so a cut row needs no merge there.
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
constexpr int64_t kRowCost = 8;       // units charged per row on top of its entries
constexpr int64_t kChunk = 1024;      // units per dynamically scheduled chunk
constexpr unsigned kFull = 0xFFFFFFFFu;

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

// Per row: first index with col > row, self-loop detection, the bound
// sum_j deg_i deg_j certifying that x3 fits in int64, and slots for big rows
// and long rows (slot order is irrelevant to every result).
__global__ void tri_prepare_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                   int64_t d, int64_t long_deg, int64_t* __restrict__ upper,
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
            wsum += dsum * (double)deg;
            int32_t s = -1;
            if (deg > kBigDeg) s = atomicAdd(counters + 0, 1);
            bslot[r] = s;
            if (deg > long_deg) longlist[atomicAdd(counters + 1, 1)] = (int32_t)r;
        }
    }
    if (lane == 0 && wsum != 0.0) atomicAdd(bound, wsum);
}

// crow[c] = the row whose units hold unit c*kChunk: the largest r with
// P(r) = rowptr[r] + kRowCost*r <= c*kChunk.
__global__ void chunk_rows_kernel(const int64_t* __restrict__ rowptr, int64_t d, int64_t nch,
                                  int64_t* __restrict__ crow)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nch;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = c * kChunk;
        int64_t lo = 0, hi = d;
        while (hi - lo > 1) {
            const int64_t mid = (lo + hi) >> 1;
            if (rowptr[mid] + kRowCost * mid <= u) lo = mid;
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
    return (int64_t)__shfl_sync(0xFFFFFFFFu, c, 0);
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

// Count, over entries [a, b) of one row, the neighbours whose sign is -1, for
// the 4 probes of this lane: byte q of the packed counter holds probe 4*lane+q.
// Bytes are flushed into int counters every 224 entries, before they can wrap.
__device__ __forceinline__ void count_negatives(const int32_t* __restrict__ col, int64_t a, int64_t b,
                                                const uint32_t* __restrict__ zb, int lane, int cnt[4])
{
    const int wl = lane >> 3;
    const int sh = (lane & 7) * 4;
    uint32_t packed = 0;
    int chunks = 0;
    for (int64_t base = a; base < b; base += 32) {
        const int64_t k = base + lane;
        const int cj = k < b ? __ldg(col + k) : 0;
        const int n = (int)min((int64_t)32, b - base);
#pragma unroll 8
        for (int t = 0; t < n; ++t) {
            const int j = __shfl_sync(kFull, cj, t);
            const uint32_t nib = (__ldg(zb + (size_t)j * 4 + wl) >> sh) & 0xFu;
            packed += (nib * 0x00204081u) & 0x01010101u;
        }
        if (++chunks == 7) {
            cnt[0] += packed & 0xFF;
            cnt[1] += (packed >> 8) & 0xFF;
            cnt[2] += (packed >> 16) & 0xFF;
            cnt[3] += packed >> 24;
            packed = 0;
            chunks = 0;
        }
    }
    cnt[0] += packed & 0xFF;
    cnt[1] += (packed >> 8) & 0xFF;
    cnt[2] += (packed >> 16) & 0xFF;
    cnt[3] += packed >> 24;
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

__device__ __forceinline__ void flush_x(long long (*sx)[kProbes], int which, const long long v[4], int lane)
{
#pragma unroll
    for (int q = 0; q < 4; ++q)
        if (v[q]) atomicAdd((unsigned long long*)&sx[which][4 * lane + q], (unsigned long long)v[q]);
}

// Pass 1: y = A z for 128 probes, plus x1 = z.y and x2 = y.y (short rows).
__global__ void __launch_bounds__(kTriThreads) tri_pass1_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t d, int64_t nch,
    int64_t long_deg, const int64_t* __restrict__ crow, const int32_t* __restrict__ bslot,
    const uint32_t* __restrict__ zb, uint32_t* __restrict__ y8, int32_t* __restrict__ y32,
    unsigned long long* __restrict__ xacc, unsigned long long* __restrict__ counter)
{
    __shared__ long long sx[2][kProbes];
    for (int t = threadIdx.x; t < 2 * kProbes; t += blockDim.x) (&sx[0][0])[t] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const int wl = lane >> 3;
    const int sh = (lane & 7) * 4;
    long long x1[4] = {0, 0, 0, 0}, x2[4] = {0, 0, 0, 0};
    for (int64_t c = next_chunk(counter, lane); c < nch; c = next_chunk(counter, lane)) {
        const int64_t u0 = c * kChunk, u1 = u0 + kChunk;
        for (int64_t r = crow[c]; r < d; ++r) {
            const int64_t beg = __ldg(rowptr + r), end = __ldg(rowptr + r + 1);
            const int64_t pr = beg + kRowCost * r;          // first unit of row r
            if (pr >= u1) break;
            const int64_t deg = end - beg;
            if (deg == 0) continue;
            int cnt[4] = {0, 0, 0, 0};
            if (deg > long_deg) {
                const int64_t e0 = pr + kRowCost;          // unit of entry beg
                const int64_t a = beg + max((int64_t)0, u0 - e0);
                const int64_t b = beg + min(deg, u1 - e0);
                if (a >= b) continue;
                count_negatives(col, a, b, zb, lane, cnt);
                int32_t* acc = y32 + (size_t)__ldg(bslot + r) * kProbes + 4 * lane;
#pragma unroll
                for (int q = 0; q < 4; ++q)
                    if (cnt[q]) atomicAdd(acc + q, cnt[q]);
                continue;
            }
            if (pr < u0) continue;                  // belongs to the previous chunk
            count_negatives(col, beg, end, zb, lane, cnt);
            const uint32_t own = (__ldg(zb + (size_t)r * 4 + wl) >> sh) & 0xFu;
            const int yv[4] = {(int)deg - 2 * cnt[0], (int)deg - 2 * cnt[1], (int)deg - 2 * cnt[2],
                               (int)deg - 2 * cnt[3]};
            store_row(r, yv, own, __ldg(bslot + r), y8, y32, lane, x1, x2);
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
        const uint32_t own = (zb[(size_t)r * 4 + (lane >> 3)] >> ((lane & 7) * 4)) & 0xFu;
        const int yv[4] = {deg - 2 * c.x, deg - 2 * c.y, deg - 2 * c.z, deg - 2 * c.w};
        store_row(r, yv, own, slot, y8, y32, lane, x1, x2);
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

// Pass 2: x3 = 2 sum_i y_i sum_{j in N(i), j > i} y_j, chunks as in pass 1.
__global__ void __launch_bounds__(kTriThreads) tri_pass2_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
    const int64_t* __restrict__ upper, int64_t d, int64_t nch, int64_t long_deg,
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
        for (int64_t r = crow[c]; r < d; ++r) {
            const int64_t beg = __ldg(rowptr + r);
            const int64_t pr = beg + kRowCost * r;
            if (pr >= u1) break;
            const int64_t end = __ldg(rowptr + r + 1);
            const int64_t deg = end - beg;
            int64_t a = __ldg(upper + r), b = end;
            if (deg > long_deg) {
                const int64_t e0 = pr + kRowCost;
                a = max(a, beg + max((int64_t)0, u0 - e0));
                b = beg + min(deg, u1 - e0);
            } else if (pr < u0) {
                continue;
            }
            if (a >= b) continue;
            int s[4] = {0, 0, 0, 0};
            for (int64_t base = a; base < b; base += 32) {
                const int64_t k = base + lane;
                const int cj = k < b ? __ldg(col + k) : 0;
                const int n = (int)min((int64_t)32, b - base);
#pragma unroll 8
                for (int t = 0; t < n; ++t) add_y(__shfl_sync(kFull, cj, t), y8, y32, bslot, lane, s);
            }
            int yi[4] = {0, 0, 0, 0};
            add_y(r, y8, y32, bslot, lane, yi);
            x3[0] += (long long)yi[0] * s[0];
            x3[1] += (long long)yi[1] * s[1];
            x3[2] += (long long)yi[2] * s[2];
            x3[3] += (long long)yi[3] * s[3];
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
    // the unit axis (entries + kRowCost per row) in chunks of kChunk units
    const int64_t nch = std::max<int64_t>(1, (nnz + kRowCost * d + kChunk - 1) / kChunk);
    const int64_t long_deg = std::max<int64_t>(kChunk, 2 * kBigDeg);
    int occ1 = 0, occ2 = 0;
    MLT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, tri_pass1_kernel, kTriThreads, 0));
    MLT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, tri_pass2_kernel, kTriThreads, 0));
    const int nw = (int)nch;   // sizing of the chunk-row table below
    int rc;
    const size_t dd = (size_t)std::max<int64_t>(d, 1);
    if ((rc = M->ws_tri.ensure(dd * (sizeof(int64_t) + 2 * sizeof(int32_t)) +
                               (size_t)(nw + 1) * sizeof(int64_t) + 1024, s))) return rc;
    char* base = M->ws_tri.as<char>();
    int64_t* upper = reinterpret_cast<int64_t*>(base);
    int64_t* crow = upper + dd;
    int32_t* bslot = reinterpret_cast<int32_t*>(crow + nw + 1);
    int32_t* longlist = bslot + dd;
    int* counters = reinterpret_cast<int*>(longlist + dd);
    double* bound = reinterpret_cast<double*>(counters + 4);
    MLT_CUDA_TRY(cudaMemsetAsync(counters, 0, 4 * sizeof(int) + sizeof(double), s));
    {
        ProfScope ps("tri_prepare", s);
        tri_prepare_kernel<<<grid_for(M->num_sms, d), kTriThreads, 0, s>>>(
            M->A.rowptr, M->A.col, d, long_deg, upper, bslot, longlist, counters, bound);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    {
        ProfScope ps("tri_chunk_rows", s);
        const int g = (int)std::min<int64_t>((nch + 255) / 256, 16LL * M->num_sms);
        chunk_rows_kernel<<<std::max(g, 1), 256, 0, s>>>(M->A.rowptr, d, nch, crow);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    int hc[4] = {0, 0, 0, 0};
    double hb = 0.0;
    MLT_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaMemcpyAsync(&hb, bound, sizeof(double), cudaMemcpyDeviceToHost, s));
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
    M->upper = upper;
    M->tri.crow = crow;
    M->tri.bslot = bslot;
    M->tri.longlist = longlist;
    M->tri.counters = reinterpret_cast<unsigned long long*>(counters + 4) + 1;
    M->tri.nbig = hc[0];
    M->tri.nlong = hc[1];
    M->tri.nch = nch;
    M->tri.long_deg = long_deg;
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
        tri_pass1_kernel<<<T.grid1, kTriThreads, 0, s>>>(M->A.rowptr, M->A.col, d, T.nch, T.long_deg,
                                                         T.crow, T.bslot, zb, y8, y32, xacc, T.counters);
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
        tri_pass2_kernel<<<T.grid2, kTriThreads, 0, s>>>(M->A.rowptr, M->A.col, M->upper, d, T.nch,
                                                         T.long_deg, T.crow, T.bslot, y8, y32, xacc,
                                                         T.counters + 1);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    MLT_CUDA_TRY(cudaMemcpyAsync(x_dev, xacc, (size_t)nb * 3 * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    return MLT_OK;
}

}  // namespace mlt
