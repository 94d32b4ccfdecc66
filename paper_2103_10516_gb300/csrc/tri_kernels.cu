// Exact integer triangle moments (Section 2.1 Example; Section 5.4).
//
// For a block of 256 Rademacher probes and a symmetric 0/1 adjacency matrix A
// with no self-loops, per probe:
//   y  = A z                      (pass 1; |y_i| <= deg_i)
//   x1 = z . y = z^T A z,  x2 = y . y = z^T A^2 z
//   x3 = y^T A y = z^T A^3 z = 2 sum over edges {i,j} of y_i y_j      (pass 2)
// Pass 2 visits every undirected edge once, so the two products of the
// paper's footnote suffice and half the gathers are saved.  Each edge is
// oriented from the endpoint of lower (degree, index) to the higher one: a
// row's out-list then holds at most sqrt(2 nnz) entries, and the gathered
// rows y_j concentrate on the high-degree vertices, a set small enough to stay
// in L2.
//
// Row classes by degree (|y_i| <= deg_i makes each storage exact):
//   small  deg <= 127    : y in y8, 256 x int8 per row (two 128-byte lines)
//   mid    deg <= 32767  : y in y16, 256 x int16 per row, slot bslot[i]
//   huge   deg >  32767  : y in y32, 256 x int32 per row, slot bslot[i]
// Each out-list is stored as [small targets (column index) | mid targets (y16
// slot)], so the inner loops need no escape test.  Edges into huge rows (a
// handful of vertices) go to a separate pair list with its own kernel.
//
// Lanes and probes: the block is two halves of 128 probes, and lane l owns
// probes 4l..4l+3 of each (block probes 4l + q and 128 + 4l + q), so every
// gathered row serves 256 probes while each lane keeps the 4-probe byte
// arithmetic per half.
// Layout (device):
//   zb      : 8 x uint32 (one 32-byte sector) per row; word 2w + h holds the
//             signs of probes 128h + 32w .. +31, bit t + 8q set when z_i of
//             probe 128h + 32w + 4t + q is -1.  Lane l loads words 2(l/8) and
//             2(l/8) + 1 as one uint2 and shifts both right by l%8: its four
//             signs of each half, one byte apart
//   y8, y16 : per row, lane l's uint2 (int8) or uint4 (int16) holds its four
//             values of half 0, then of half 1
//   y32     : 256 x int32 per slot in block-probe order; also the pass-1
//             accumulator of rows longer than a chunk
//   out_ptr : row pointer of the oriented out-lists, out_col their entries,
//             nsmall the length of each list's small section
//   pairs   : (class of i, row or slot of i, y32 slot of the huge target)
// Work split: every row costs kRowCost "units" plus one per entry (all entries
// in pass 1, out-entries in pass 2); the unit axis is cut into chunks of
// kChunk1 (pass 1) or kChunk2 (pass 2) units that warps of a persistent grid
// take from an atomic counter
// (small chunks, so the last ones to finish leave little idle time).  A row of
// degree <= kLongRow is handled whole by the chunk holding its first unit;
// consecutive such rows are walked with the row ends of 32 rows at a time held
// in lanes.  Longer rows are cut at chunk edges: pass-1 counts are
// merged with integer atomics in y32 and finished by a per-row kernel; pass 2
// is linear in the row sums, so a cut needs no merge.
// All sums are integers (exact, independent of order).
#include <cuda_runtime.h>

#include <algorithm>

#include "mlt_internal.h"
#include "rng.cuh"

namespace mlt {
namespace {

constexpr int kTriThreads = 256;
constexpr int kProbes = 256;       // probes per block: two halves of 128
constexpr int kHalf = 128;
constexpr int kZWords = kProbes / 32;   // sign words per row
constexpr int kSmallDeg = 127;        // y of rows up to this degree fits int8
constexpr int kMidDeg = 32767;        // ... int16; rows above it keep int32
constexpr int64_t kRowCost = 4;       // units charged per row on top of its entries
constexpr int64_t kChunk1 = 512;      // units per dynamically scheduled chunk: pass 1 (and preparation)
constexpr int64_t kChunk2 = 256;      // ... and pass 2
constexpr int64_t kLongRow = 1024;    // rows above this degree are cut at chunk edges
constexpr int kGather = 4;            // pass-1 short rows: gathers in flight per batch (divides 32);
                                      // most such rows have a few entries, so wider batches idle
constexpr unsigned kFull = 0xFFFFFFFFu;
static_assert(32 % kGather == 0, "a gather batch never crosses a 32-entry column block");
constexpr int kScanBlock = 1024;      // elements per CTA of the prefix scan
constexpr int kPass2CtasPerSm = 4;    // pass 2 compiled for four resident CTAs (64 registers)
static_assert(kLongRow <= kMidDeg && kChunk1 <= kLongRow && kChunk2 <= kLongRow,
              "rows handled whole by the passes must be small or mid");

enum RowClass { kClassSmall = 0, kClassMid = 1, kClassHuge = 2 };

__host__ __device__ __forceinline__ int row_class(int64_t deg)
{
    return deg <= kSmallDeg ? kClassSmall : (deg <= kMidDeg ? kClassMid : kClassHuge);
}

// Bit 4t + q of x moved to bit t + 8q (an 8 x 4 bit transpose).
__device__ __forceinline__ uint32_t interleave_bytes(uint32_t x)
{
    uint32_t out = 0;
#pragma unroll
    for (int q = 0; q < 4; ++q) {
        uint32_t m = (x >> q) & 0x11111111u;   // bits 4t
        m = (m | (m >> 3)) & 0x03030303u;      // pairs of t
        m = (m | (m >> 6)) & 0x000F000Fu;      // quads of t
        m = (m | (m >> 12)) & 0xFFu;           // t = 0..7 in bits 0..7
        out |= m << (8 * q);
    }
    return out;
}

// zb[i * 8 + 2w + h]: the signs of block probes 128h + 32w .. + 31 at row i
// in the byte-interleaved order above (0 for probes past nb).  The 32 bits
// come from one or two 64-probe hash words; when id0 is a multiple of 64 (a
// run of blocks that starts aligned), words 4m + h and 4m + 2 + h share one
// hash word (probes 128h + 64m .. +63), computed once.  The same launch zeroes
// the y32 accumulators of the nlong rows longer than a chunk.
__global__ void zbits_kernel(int64_t d, uint64_t seedmix, int64_t id0, int nb, uint32_t* __restrict__ zb,
                             const int32_t* __restrict__ longlist, int nlong, const int32_t* __restrict__ bslot,
                             int32_t* __restrict__ y32)
{
    const int64_t t0 = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    if ((id0 & 63) == 0) {
        for (int64_t e = t0; e < d * 4; e += stride) {
            const uint64_t i = (uint64_t)(e >> 2);
            const int h = (int)(e & 1), m = (int)((e >> 1) & 1);
            const int pb = kHalf * h + 64 * m;            // first block probe of the hash word
            const int valid = min(64, max(0, nb - pb));
            uint64_t v = 0;
            if (valid > 0) {
                v = probe_word(seedmix, (uint64_t)(id0 + pb) >> 6, i);
                if (valid < 64) v &= (1ull << valid) - 1ull;
            }
            zb[i * kZWords + 4 * m + h] = interleave_bytes((uint32_t)v);
            zb[i * kZWords + 4 * m + 2 + h] = interleave_bytes((uint32_t)(v >> 32));
        }
    } else {
        for (int64_t e = t0; e < d * kZWords; e += stride) {
            const uint64_t i = (uint64_t)(e >> 3);
            const int w8 = (int)(e & 7);
            const int pb = kHalf * (w8 & 1) + 32 * (w8 >> 1);   // first block probe of the word
            const int valid = min(32, max(0, nb - pb));
            uint32_t bits = 0;
            if (valid > 0) {
                const uint64_t p0 = (uint64_t)(id0 + pb);
                const int o = (int)(p0 & 63);
                uint64_t v = probe_word(seedmix, p0 >> 6, i) >> o;
                if (o > 32) v |= probe_word(seedmix, (p0 >> 6) + 1, i) << (64 - o);
                bits = (uint32_t)v;
                if (valid < 32) bits &= (1u << valid) - 1u;
            }
            zb[e] = interleave_bytes(bits);
        }
    }
    for (int64_t e = t0; e < (int64_t)nlong * kProbes; e += stride) {
        const int r = longlist[e / kProbes];
        y32[(size_t)bslot[r] * kProbes + (e % kProbes)] = 0;
    }
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

// crow[c] = the row whose units hold unit c*chunk: the largest r with
// ptr[r] + kRowCost*r <= c*chunk.
__global__ void chunk_rows_kernel(const int64_t* __restrict__ ptr, int64_t d, int64_t nch, int64_t chunk,
                                  int64_t* __restrict__ crow)
{
    for (int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; c < nch;
         c += (int64_t)gridDim.x * blockDim.x) {
        const int64_t u = c * chunk;
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

// ---- preparation: orientation, classes, slots, out-lists ---------------------

// Neighbour c (degree dc) of row r (degree deg) is an out-target of r when its
// (degree, index) key is larger.
__device__ __forceinline__ bool is_target(int64_t r, int deg, int c, int dc)
{
    return dc > deg || (dc == deg && c > r);
}

// A thread per row: its degree as int32 (nnz < 2^31), a y16 / y32 slot for
// rows above kSmallDeg, and the list of rows above kLongRow, whose out-list
// counts and fill cursors start at zero here (the entry passes add to them).
// Slots and list positions come from warp-aggregated atomics: their order is
// irrelevant to every result.
__global__ void tri_degrees_kernel(const int64_t* __restrict__ rowptr, int64_t d, int32_t* __restrict__ deg32,
                                   int32_t* __restrict__ bslot, int32_t* __restrict__ longlist,
                                   int64_t* __restrict__ outcnt, int32_t* __restrict__ nsmall,
                                   int32_t* __restrict__ cur, int* counters /* [0] nbig, [1] nlong */)
{
    const int lane = threadIdx.x & 31;
    const unsigned below = (1u << lane) - 1u;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t r0 = blockIdx.x * (int64_t)blockDim.x + (threadIdx.x & ~31); r0 < d; r0 += stride) {
        const int64_t r = r0 + lane;
        const bool valid = r < d;
        const int deg = valid ? (int)(rowptr[r + 1] - rowptr[r]) : 0;
        const bool big = valid && deg > kSmallDeg, lng = valid && deg > kLongRow;
        const unsigned mb = __ballot_sync(kFull, big), ml = __ballot_sync(kFull, lng);
        int sb = 0, sl = 0;
        if (lane == 0) {
            if (mb) sb = atomicAdd(counters + 0, __popc(mb));
            if (ml) sl = atomicAdd(counters + 1, __popc(ml));
        }
        sb = __shfl_sync(kFull, sb, 0);
        sl = __shfl_sync(kFull, sl, 0);
        if (!valid) continue;
        deg32[r] = deg;
        const int slot = big ? sb + __popc(mb & below) : -1;
        bslot[r] = slot;
        if (big) {
            cur[2 * (size_t)slot] = 0;
            cur[2 * (size_t)slot + 1] = 0;
        }
        if (lng) {
            longlist[sl + __popc(ml & below)] = (int32_t)r;
            outcnt[r] = 0;
            nsmall[r] = 0;
        }
    }
}

// Walk the rows of unit chunk c exactly as pass 1 does: a row above kLongRow
// is cut at the chunk's edges (long_part(r, deg, a, b) for its entries
// [a, b)); every shorter row belongs to the chunk holding its first unit,
// and runs of 1 to 32 of them are handed to group(r, f, s0, e0) with row
// r + lane's entry range [s0, e0) in lane `lane` (meaningful for lanes below f).
template <typename Group, typename LongPart>
__device__ __forceinline__ void walk_chunk(const int64_t* __restrict__ rowptr, int64_t d, int64_t c,
                                           const int64_t* __restrict__ crow, int lane, Group group,
                                           LongPart long_part)
{
    const int64_t u0 = c * kChunk1, u1 = u0 + kChunk1;
    int64_t r = crow[c];
    while (r < d) {
        const int64_t beg = __ldg(rowptr + r);
        const int64_t pr = beg + kRowCost * r;
        if (pr >= u1) break;
        const int64_t deg = __ldg(rowptr + r + 1) - beg;
        if (deg > kLongRow) {
            const int64_t e0 = pr + kRowCost;
            const int64_t a = beg + max((int64_t)0, u0 - e0);
            const int64_t b = beg + min(deg, u1 - e0);
            if (a < b) long_part(r, (int)deg, a, b);
            ++r;
            continue;
        }
        if (pr < u0) {
            ++r;
            continue;
        }
        for (;;) {
            const int64_t rr = r + lane;
            int s0 = 0, e0 = 0;
            bool ok = false;
            if (rr < d) {
                const int64_t x0 = __ldg(rowptr + rr), x1 = __ldg(rowptr + rr + 1);
                s0 = (int)x0;
                e0 = (int)x1;
                ok = (x0 + kRowCost * rr < u1) && (x1 - x0 <= kLongRow);
            }
            const unsigned okm = __ballot_sync(kFull, ok);
            const int f = (okm == kFull) ? 32 : (__ffs(~okm) - 1);
            if (f > 0) group(r, f, s0, e0);
            r += f;
            if (f < 32) break;
        }
    }
}

// One batch of up to 32 consecutive entries [base, B) of a run of f short
// rows (row r + i starts at s0 of lane i): this lane's entry, its row's
// position i in the run, the row's degree, and whether this lane is the first
// of its row in the batch (row segments are contiguous in lane order).
struct RunEntry {
    int k, idx, deg;
    bool valid;
};

__device__ __forceinline__ RunEntry run_entry(int base, int B, int f, int s0, int dg, int lane)
{
    RunEntry e;
    e.k = base + lane;
    e.valid = e.k < B;
    int idx = 0;   // the last row of the run starting at or before k
#pragma unroll
    for (int st = 16; st; st >>= 1) {
        const int cand = idx + st;
        const int sv = __shfl_sync(kFull, s0, min(cand, 31));
        if (cand < f && sv <= e.k) idx = cand;
    }
    e.idx = idx;
    e.deg = __shfl_sync(kFull, dg, idx);
    return e;
}

// Lanes [l, next head) hold the row segment that starts at head lane l.
__device__ __forceinline__ unsigned segment_from(unsigned heads, int l)
{
    const unsigned above = heads & ~((2u << l) - 1u);
    const unsigned upto = above ? (1u << (__ffs(above) - 1)) - 1u : kFull;
    return upto & ~((1u << l) - 1u);
}

// Class of entry k's target as seen from its row (-1: not an out-target).
__device__ __forceinline__ int target_class(int64_t row, int deg, int c, int dc)
{
    return is_target(row, deg, c, dc) ? row_class(dc) : -1;
}

// Counting pass over the chunks of pass 1: per row the out-list length
// (outcnt, scanned into out_ptr next) and its small section (nsmall); the
// number of edges into huge rows; self-loops; and the bound sum over entries
// of deg_i deg_j certifying that x3 fits in int64.  Short rows are written
// whole by their chunk; long rows add their parts.
__global__ void __launch_bounds__(kTriThreads) tri_classify_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int32_t* __restrict__ deg32,
    int64_t d, int64_t nch, const int64_t* __restrict__ crow, int64_t* __restrict__ outcnt,
    int32_t* __restrict__ nsmall, int* counters /* [2] selfloop, [3] npairs */, double* bound,
    unsigned long long* __restrict__ chunk_ctr)
{
    __shared__ int sc[kTriThreads / 32][32], mc[kTriThreads / 32][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    sc[wid][lane] = 0;
    mc[wid][lane] = 0;
    __syncwarp();
    double wsum = 0.0;
    int nh = 0;
    bool loop = false;
    auto group = [&](int64_t r, int f, int s0, int e0) {
        const int A = __shfl_sync(kFull, s0, 0), B = __shfl_sync(kFull, e0, f - 1);
        const int dg = e0 - s0;
        for (int base = A; base < B; base += 32) {
            const RunEntry e = run_entry(base, B, f, s0, dg, lane);
            const int64_t row = r + e.idx;
            int cl = -1;
            if (e.valid) {
                const int c = __ldg(col + e.k);
                const int dc = __ldg(deg32 + c);
                loop |= c == row;
                wsum += (double)dc * (double)e.deg;
                cl = target_class(row, e.deg, c, dc);
            }
            const unsigned ms = __ballot_sync(kFull, cl == kClassSmall);
            const unsigned mm = __ballot_sync(kFull, cl == kClassMid);
            nh += __popc(__ballot_sync(kFull, cl == kClassHuge));
            const int prev = __shfl_up_sync(kFull, e.idx, 1);
            const bool head = e.valid && (lane == 0 || prev != e.idx);
            const unsigned heads = __ballot_sync(kFull, head);
            if (head) {
                const unsigned seg = segment_from(heads, lane);
                sc[wid][e.idx] += __popc(ms & seg);
                mc[wid][e.idx] += __popc(mm & seg);
            }
            __syncwarp();
        }
        if (lane < f) {
            outcnt[r + lane] = sc[wid][lane] + mc[wid][lane];
            nsmall[r + lane] = sc[wid][lane];
        }
        sc[wid][lane] = 0;
        mc[wid][lane] = 0;
        __syncwarp();
    };
    auto long_part = [&](int64_t r, int deg, int64_t a, int64_t b) {
        int ns = 0, nm = 0;
        for (int64_t base = a; base < b; base += 32) {
            const int64_t k = base + lane;
            int cl = -1;
            if (k < b) {
                const int c = __ldg(col + k);
                const int dc = __ldg(deg32 + c);
                loop |= c == r;
                wsum += (double)dc * (double)deg;
                cl = target_class(r, deg, c, dc);
            }
            ns += __popc(__ballot_sync(kFull, cl == kClassSmall));
            nm += __popc(__ballot_sync(kFull, cl == kClassMid));
            nh += __popc(__ballot_sync(kFull, cl == kClassHuge));
        }
        if (lane == 0) {
            if (ns + nm) atomicAdd(reinterpret_cast<unsigned long long*>(outcnt + r), (unsigned long long)(ns + nm));
            if (ns) atomicAdd(nsmall + r, ns);
        }
    };
    for (int64_t c = next_chunk(chunk_ctr, lane); c < nch; c = next_chunk(chunk_ctr, lane))
        walk_chunk(rowptr, d, c, crow, lane, group, long_part);
    for (int o = 16; o; o >>= 1) wsum += __shfl_xor_sync(kFull, wsum, o);
    if (__any_sync(kFull, loop) && lane == 0) atomicOr(counters + 2, 1);
    if (lane == 0) {
        if (nh) atomicAdd(counters + 3, nh);
        if (wsum != 0.0) atomicAdd(bound, wsum);
    }
}

// One pair of the huge-target list: how to read y_i, and the target's slot.
__device__ __forceinline__ int4 make_pair(int64_t r, int deg, const int32_t* __restrict__ bslot, int target_slot)
{
    const int cl = row_class(deg);
    return make_int4(cl, cl == kClassSmall ? (int)r : __ldg(bslot + r), target_slot, 0);
}

// Fill pass, the same walk: each out-list gets its small targets (their row)
// before its mid targets (their slot); edges into huge rows go to the pair
// list.  A short row's entries keep neighbour order (running offsets per row
// of the run in shared memory); a long row's parts take their places from
// per-row cursors, so their order within a section is arbitrary, which pass 2
// (integer sums) does not see.
__global__ void __launch_bounds__(kTriThreads) tri_fill_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, const int32_t* __restrict__ deg32,
    int64_t d, int64_t nch, const int64_t* __restrict__ crow, const int64_t* __restrict__ out_ptr,
    const int32_t* __restrict__ nsmall, const int32_t* __restrict__ bslot, int32_t* __restrict__ cur,
    int32_t* __restrict__ out_col, int4* __restrict__ pairs, int npairs, int* pair_ctr,
    unsigned long long* __restrict__ chunk_ctr)
{
    __shared__ int sc[kTriThreads / 32][32], mc[kTriThreads / 32][32];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    sc[wid][lane] = 0;
    mc[wid][lane] = 0;
    __syncwarp();
    // edges into huge rows: places for this batch's pairs, in lane order
    auto add_pairs = [&](int cl, int64_t row, int deg, int c) {
        const unsigned mh = __ballot_sync(kFull, cl == kClassHuge);
        if (!mh) return;
        int p0 = 0;
        if (lane == 0) p0 = atomicAdd(pair_ctr, __popc(mh));
        p0 = __shfl_sync(kFull, p0, 0);
        const int at = p0 + __popc(mh & below);
        if (cl == kClassHuge && at < npairs)   // at < npairs by construction
            pairs[at] = make_pair(row, deg, bslot, __ldg(bslot + c));
    };
    auto group = [&](int64_t r, int f, int s0, int e0) {
        const int A = __shfl_sync(kFull, s0, 0), B = __shfl_sync(kFull, e0, f - 1);
        const int dg = e0 - s0;
        int64_t op = 0;
        int ns = 0;
        if (lane < f && e0 > s0) {
            op = __ldg(out_ptr + r + lane);
            ns = __ldg(nsmall + r + lane);
        }
        for (int base = A; base < B; base += 32) {
            const RunEntry e = run_entry(base, B, f, s0, dg, lane);
            const int64_t row = r + e.idx;
            int c = 0, cl = -1;
            if (e.valid) {
                c = __ldg(col + e.k);
                cl = target_class(row, e.deg, c, __ldg(deg32 + c));
            }
            const unsigned ms = __ballot_sync(kFull, cl == kClassSmall);
            const unsigned mm = __ballot_sync(kFull, cl == kClassMid);
            const int prev = __shfl_up_sync(kFull, e.idx, 1);
            const bool head = e.valid && (lane == 0 || prev != e.idx);
            const unsigned heads = __ballot_sync(kFull, head);
            const int64_t rop = __shfl_sync(kFull, op, e.idx);
            const int rns = __shfl_sync(kFull, ns, e.idx);
            if (cl >= 0) {
                const int h = 31 - __clz(heads & ((2u << lane) - 1u));   // head of this lane's segment
                const unsigned before = below & ~((1u << h) - 1u);
                if (cl == kClassSmall)
                    out_col[rop + sc[wid][e.idx] + __popc(ms & before)] = c;
                else if (cl == kClassMid)
                    out_col[rop + rns + mc[wid][e.idx] + __popc(mm & before)] = __ldg(bslot + c);
            }
            add_pairs(cl, row, e.deg, c);
            __syncwarp();
            if (head) {
                const unsigned seg = segment_from(heads, lane);
                sc[wid][e.idx] += __popc(ms & seg);
                mc[wid][e.idx] += __popc(mm & seg);
            }
            __syncwarp();
        }
        sc[wid][lane] = 0;
        mc[wid][lane] = 0;
        __syncwarp();
    };
    auto long_part = [&](int64_t r, int deg, int64_t a, int64_t b) {
        const int64_t op = __ldg(out_ptr + r);
        const int rns = __ldg(nsmall + r);
        int32_t* rc = cur + 2 * (size_t)__ldg(bslot + r);
        for (int64_t base = a; base < b; base += 32) {
            const int64_t k = base + lane;
            int c = 0, cl = -1;
            if (k < b) {
                c = __ldg(col + k);
                cl = target_class(r, deg, c, __ldg(deg32 + c));
            }
            const unsigned ms = __ballot_sync(kFull, cl == kClassSmall);
            const unsigned mm = __ballot_sync(kFull, cl == kClassMid);
            int bs = 0, bm = 0;
            if (lane == 0) {
                if (ms) bs = atomicAdd(rc, __popc(ms));
                if (mm) bm = atomicAdd(rc + 1, __popc(mm));
            }
            bs = __shfl_sync(kFull, bs, 0);
            bm = __shfl_sync(kFull, bm, 0);
            if (cl == kClassSmall) out_col[op + bs + __popc(ms & below)] = c;
            else if (cl == kClassMid) out_col[op + rns + bm + __popc(mm & below)] = __ldg(bslot + c);
            add_pairs(cl, r, deg, c);
        }
    };
    for (int64_t c = next_chunk(chunk_ctr, lane); c < nch; c = next_chunk(chunk_ctr, lane))
        walk_chunk(rowptr, d, c, crow, lane, group, long_part);
}

// Entries t0 .. t0+D-1 of the current block of 32 (their row or slot in lane
// t0+u's cj): D gathers are issued before the first is used.
template <int D, typename Load, typename Use>
__device__ __forceinline__ void gather_batch(int cj, int t0, Load load, Use use)
{
    decltype(load(0)) w[D];
#pragma unroll
    for (int u = 0; u < D; ++u) w[u] = load(__shfl_sync(kFull, cj, t0 + u));
#pragma unroll
    for (int u = 0; u < D; ++u) use(w[u]);
}

// The n (<= 32, warp-uniform) entries of a block: batches of D while that
// many remain, then one of 4 (D = 8), then one at a time, so a short out-list
// wastes no gather slot and no slot needs a bounds test (pass 2; pass 1's
// short rows keep predicated batches, which measured faster there).  D
// bounds the registers the batch holds: 8 x uint2 or 4 x uint4 keep the same
// bytes in flight per lane.
template <int D, typename Load, typename Use>
__device__ __forceinline__ void gather_block(int cj, int n, Load load, Use use)
{
    static_assert(D == 8 || D == 4, "batches of 8 then 4, or of 4");
    int t0 = 0;
    for (; t0 + D <= n; t0 += D) gather_batch<D>(cj, t0, load, use);
    if (D > 4 && t0 + 4 <= n) {
        gather_batch<4>(cj, t0, load, use);
        t0 += 4;
    }
    for (; t0 < n; ++t0) gather_batch<1>(cj, t0, load, use);
}

// ---- pass 1 ------------------------------------------------------------------

// This lane's sign bits of row j: .x for half 0 (probes 4*lane + q), .y for
// half 1 (128 + 4*lane + q), probe q in bit 8q.
__device__ __forceinline__ uint2 sign_pair(const uint2* __restrict__ zb2, int64_t j, int lane)
{
    const uint2 w = __ldg(zb2 + (size_t)j * 4 + (lane >> 3));
    const int sh = lane & 7;
    return make_uint2((w.x >> sh) & 0x01010101u, (w.y >> sh) & 0x01010101u);
}

// Byte q of `packed` counts sign bit q; folded into int counters before it can wrap.
__device__ __forceinline__ void fold(uint32_t& packed, int* cnt)
{
    cnt[0] += packed & 0xFF;
    cnt[1] += (packed >> 8) & 0xFF;
    cnt[2] += (packed >> 16) & 0xFF;
    cnt[3] += packed >> 24;
    packed = 0;
}

// Negative-sign counts over entries [a, b) of one row, for this lane's 8
// probes (cnt[0..3] half 0, cnt[4..7] half 1).  kGather gathers are in flight
// before the first is used; lanes past the end load nothing and add zero.
__device__ __forceinline__ void count_negatives(const int32_t* __restrict__ col, int64_t a, int64_t b,
                                                const uint2* __restrict__ zb2, int lane, int cnt[8])
{
    const uint2* zbl = zb2 + (lane >> 3);
    const int sh = lane & 7;
    uint32_t pa = 0, pb = 0;
    for (int64_t base = a; base < b; base += 32) {
        const int64_t k = base + lane;
        const int cj = k < b ? __ldg(col + k) : 0;
        const int n = (int)min((int64_t)32, b - base);
        for (int t0 = 0; t0 < n; t0 += kGather) {
            uint2 w[kGather];
#pragma unroll
            for (int u = 0; u < kGather; ++u) {
                const int j = __shfl_sync(kFull, cj, t0 + u);
                w[u] = t0 + u < n ? __ldg(zbl + (size_t)j * 4) : make_uint2(0u, 0u);
            }
#pragma unroll
            for (int u = 0; u < kGather; ++u) {
                pa += (w[u].x >> sh) & 0x01010101u;
                pb += (w[u].y >> sh) & 0x01010101u;
            }
        }
        fold(pa, cnt);
        fold(pb, cnt + 4);
    }
}

// The same counts, bit-sliced, for spans of at least kSliceMin entries (and
// at most kLongRow).  Lane l takes entry l/8 of every batch of 4 entries and
// sign word l%8 of it (32 probes of one half), and counts each of the 32 bit
// positions in P bit planes: bit t of c[p] is bit p of position t's count.
// Blocks of 32 (P >= 4) and then 16 entries give each lane eight or four
// words at once (that many gathers in flight), added with carry-save adders:
// for four words, c0 + x0 + x1 = c0' + 2 t0 and c0' + x2 + x3 = c0'' + 2 t1,
// then c1 + t0 + t1 = c1' + 2 f, and f ripples into planes 2 .. P-1 (15 +
// 2(P-2) bitwise operations, where a ripple-carry increment takes 3P per
// word); eight words add two such groups and c2 + f0 + f1 = c2' + 2 e.  The
// rest of the span adds one word per batch of 4 by ripple.  The four entry
// slots are then summed lane against lane with a bit-sliced adder whose sums
// gain one plane per level, and each lane reads its own probes out of the
// planes of words 2(l/8) (half 0) and 2(l/8) + 1 (half 1).  P planes must hold
// the words one lane sees, ceil(n / 4) for a span of n entries (the planes
// always hold a lane's exact count).
constexpr int kSliceMin = 16;   // long rows' parts below it use count_negatives
static_assert(kLongRow <= 1024, "nine planes hold a lane's count of at most 256 words");

// a + b + c = s + 2 carry, bitwise (a full adder per bit position); s replaces a.
__device__ __forceinline__ void carry_save(uint32_t& a, uint32_t b, uint32_t c, uint32_t& carry)
{
    const uint32_t u = a ^ b;
    carry = (a & b) | (u & c);
    a = u ^ c;
}

// This lane's four counts of the word held (after the adder) by lane src.
template <int Q>
__device__ __forceinline__ void read_counts(const uint32_t (&c)[Q], int src, int sh, int* cnt)
{
    uint32_t lo = 0u, hi = 0u;   // 16-bit lanes: probes q = 0, 2 and q = 1, 3
#pragma unroll
    for (int p = 0; p < Q; ++p) {
        const uint32_t t = (__shfl_sync(kFull, c[p], src) >> sh) & 0x01010101u;
        lo += (t & 0x00010001u) << p;
        hi += ((t >> 8) & 0x00010001u) << p;
    }
    cnt[0] += (int)(lo & 0xFFFFu);
    cnt[1] += (int)(hi & 0xFFFFu);
    cnt[2] += (int)(lo >> 16);
    cnt[3] += (int)(hi >> 16);
}

template <int P>
__device__ __forceinline__ void count_negatives_sliced_p(const int32_t* __restrict__ col, int64_t a, int64_t b,
                                                         const uint32_t* __restrict__ zb, int lane, int cnt[8])
{
    constexpr int Q = P + 2;   // planes of the sum of four slots
    static_assert(P >= 3, "the carry-save blocks use planes 0, 1 and 2");
    uint32_t c[Q];
#pragma unroll
    for (int p = 0; p < Q; ++p) c[p] = 0u;
    const int slot = lane >> 3, w8 = lane & 7;
    int64_t base = a;
    if constexpr (P >= 4) {
        for (; base + 32 <= b; base += 32) {
            const int cj = __ldg(col + base + lane);
            uint32_t x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = __ldg(zb + (size_t)__shfl_sync(kFull, cj, 4 * u + slot) * 8 + w8);
            uint32_t t0, t1, t2, t3, f0, f1, e;
            carry_save(c[0], x[0], x[1], t0);
            carry_save(c[0], x[2], x[3], t1);
            carry_save(c[1], t0, t1, f0);
            carry_save(c[0], x[4], x[5], t2);
            carry_save(c[0], x[6], x[7], t3);
            carry_save(c[1], t2, t3, f1);
            carry_save(c[2], f0, f1, e);
#pragma unroll
            for (int p = 3; p < P; ++p) {
                const uint32_t t = c[p] & e;
                c[p] ^= e;
                e = t;
            }
        }
    }
    for (; base + 16 <= b; base += 16) {
        const int cj = base + lane < b ? __ldg(col + base + lane) : 0;
        uint32_t x[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) x[u] = __ldg(zb + (size_t)__shfl_sync(kFull, cj, 4 * u + slot) * 8 + w8);
        uint32_t t0, t1, f;
        carry_save(c[0], x[0], x[1], t0);
        carry_save(c[0], x[2], x[3], t1);
        carry_save(c[1], t0, t1, f);
#pragma unroll
        for (int p = 2; p < P; ++p) {
            const uint32_t t = c[p] & f;
            c[p] ^= f;
            f = t;
        }
    }
    for (; base < b; base += 4) {
        const int64_t k = base + slot;
        uint32_t x = 0u;
        if (k < b) x = __ldg(zb + (size_t)__ldg(col + k) * 8 + w8);
#pragma unroll
        for (int p = 0; p < P; ++p) {
            const uint32_t t = c[p] & x;
            c[p] ^= x;
            x = t;
        }
    }
#pragma unroll
    for (int lv = 0; lv < 2; ++lv) {
        const int m = 8 << lv;
        uint32_t carry = 0u;
#pragma unroll
        for (int p = 0; p < P + lv; ++p) {
            const uint32_t o = __shfl_xor_sync(kFull, c[p], m);
            const uint32_t sum = c[p] ^ o ^ carry;
            carry = (c[p] & o) | (carry & (c[p] ^ o));
            c[p] = sum;
        }
        c[P + lv] = carry;
    }
    const int src = 2 * (lane >> 3), sh = lane & 7;
    read_counts<Q>(c, src, sh, cnt);
    read_counts<Q>(c, src + 1, sh, cnt + 4);
}

// A span of n = b - a entries, kSliceMin <= n <= kLongRow: a lane sees at
// most ceil(n / 4) <= 256 words, which nine planes hold.  One instantiation
// serves every span: the few bitwise operations that fewer planes would save
// on short spans cost less than the instruction-cache misses of several
// unrolled copies of the counter (measured: 0.47 ms per pass-1 launch on the
// R-MAT 20 block with one copy, 0.60 ms with seven).
__device__ __forceinline__ void count_negatives_sliced(const int32_t* __restrict__ col, int64_t a, int64_t b,
                                                       const uint32_t* __restrict__ zb, int lane, int cnt[8])
{
    count_negatives_sliced_p<9>(col, a, b, zb, lane, cnt);
}

__device__ __forceinline__ uint32_t pack_bytes(const int* v)
{
    return (uint32_t)(v[0] & 0xFF) | ((uint32_t)(v[1] & 0xFF) << 8) | ((uint32_t)(v[2] & 0xFF) << 16) |
           ((uint32_t)(v[3] & 0xFF) << 24);
}

__device__ __forceinline__ uint32_t pack_halves(int lo, int hi)
{
    return (uint32_t)(lo & 0xFFFF) | ((uint32_t)hi << 16);
}

// Store y for this lane's 8 probes of row r (degree deg, slot if deg >
// kSmallDeg) in its class's array, and add its x1, x2 terms (Acc: int for
// the sums of one pass-1 chunk, long long otherwise).
template <typename Acc>
__device__ __forceinline__ void store_row(int64_t r, int64_t deg, const int yv[8], uint2 own, int32_t slot,
                                          uint2* __restrict__ y8, uint4* __restrict__ y16,
                                          int32_t* __restrict__ y32, int lane, Acc x1[8], Acc x2[8])
{
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        const Acc yq = yv[q];
        const uint32_t ob = q < 4 ? own.x >> (8 * q) : own.y >> (8 * (q - 4));
        x1[q] += (ob & 1u) ? -yq : yq;
        x2[q] += yq * yq;
    }
    const int cl = row_class(deg);
    if (cl == kClassSmall) {
        y8[(size_t)r * 32 + lane] = make_uint2(pack_bytes(yv), pack_bytes(yv + 4));
    } else if (cl == kClassMid) {
        y16[(size_t)slot * 32 + lane] = make_uint4(pack_halves(yv[0], yv[1]), pack_halves(yv[2], yv[3]),
                                                   pack_halves(yv[4], yv[5]), pack_halves(yv[6], yv[7]));
    } else {
        int32_t* yr = y32 + (size_t)slot * kProbes + 4 * lane;
        *reinterpret_cast<int4*>(yr) = make_int4(yv[0], yv[1], yv[2], yv[3]);
        *reinterpret_cast<int4*>(yr + kHalf) = make_int4(yv[4], yv[5], yv[6], yv[7]);
    }
}

// y of a row handled whole by one chunk, from its negative-sign counts.  x1
// and x2 take int sums: the rows a chunk owns hold at most kChunk1 + kLongRow
// entries, so their sum of y^2 <= kLongRow * (kChunk1 + kLongRow) < 2^31.
static_assert((int64_t)kLongRow * (kChunk1 + kLongRow) < (1LL << 31), "int sums of x2 over one chunk");
__device__ __forceinline__ void finish_pass1_row(int64_t r, int deg, int cnt[8], uint2 own,
                                                 const int32_t* __restrict__ bslot, uint2* __restrict__ y8,
                                                 uint4* __restrict__ y16, int32_t* __restrict__ y32, int lane,
                                                 int x1[8], int x2[8])
{
    if (deg > 0) {
        int yv[8];
#pragma unroll
        for (int q = 0; q < 8; ++q) yv[q] = deg - 2 * cnt[q];
        store_row(r, deg, yv, own, deg > kSmallDeg ? __ldg(bslot + r) : -1, y8, y16, y32, lane, x1, x2);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) cnt[q] = 0;
}

// sx[which][block probe] += this lane's 8 values.
template <typename Acc>
__device__ __forceinline__ void flush_x(long long (*sx)[kProbes], int which, const Acc v[8], int lane)
{
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (v[q]) atomicAdd((unsigned long long*)&sx[which][(q < 4 ? 0 : kHalf) + 4 * lane + (q & 3)],
                            (unsigned long long)(long long)v[q]);
}

// Pass 1: y = A z for 256 probes, plus x1 = z.y and x2 = y.y (rows of degree
// <= kLongRow; longer rows only accumulate their counts here).
__global__ void __launch_bounds__(kTriThreads) tri_pass1_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col, int64_t d, int64_t nch,
    const int64_t* __restrict__ crow, const int32_t* __restrict__ bslot,
    const uint32_t* __restrict__ zb, uint2* __restrict__ y8, uint4* __restrict__ y16,
    int32_t* __restrict__ y32, unsigned long long* __restrict__ xacc, unsigned long long* __restrict__ counter)
{
    __shared__ long long sx[2][kProbes];
    for (int t = threadIdx.x; t < 2 * kProbes; t += blockDim.x) (&sx[0][0])[t] = 0;
    __syncthreads();

    const uint2* zb2 = reinterpret_cast<const uint2*>(zb);
    const int lane = threadIdx.x & 31;
    for (int64_t c = next_chunk(counter, lane); c < nch; c = next_chunk(counter, lane)) {
        const int64_t u0 = c * kChunk1, u1 = u0 + kChunk1;
        int64_t r = crow[c];
        int cx1[8] = {0, 0, 0, 0, 0, 0, 0, 0}, cx2[8] = {0, 0, 0, 0, 0, 0, 0, 0};   // this chunk's rows
        while (r < d) {
            const int64_t beg = __ldg(rowptr + r);
            const int64_t pr = beg + kRowCost * r;          // first unit of row r
            if (pr >= u1) break;
            const int64_t end = __ldg(rowptr + r + 1);
            const int64_t deg = end - beg;
            if (deg > kLongRow) {                           // long row: this chunk's part
                const int64_t e0 = pr + kRowCost;
                const int64_t a = beg + max((int64_t)0, u0 - e0);
                const int64_t b = beg + min(deg, u1 - e0);
                if (a < b) {
                    int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    if (b - a >= kSliceMin) count_negatives_sliced(col, a, b, zb, lane, cnt);
                    else count_negatives(col, a, b, zb2, lane, cnt);
                    int32_t* acc = y32 + (size_t)__ldg(bslot + r) * kProbes + 4 * lane;
#pragma unroll
                    for (int q = 0; q < 8; ++q)
                        if (cnt[q]) atomicAdd(acc + (q < 4 ? 0 : kHalf) + (q & 3), cnt[q]);
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
                    ok = (s0 + kRowCost * rr < u1) && (e0 - s0 <= kLongRow);
                }
                const unsigned okm = __ballot_sync(kFull, ok);
                const int f = (okm == kFull) ? 32 : (__ffs(~okm) - 1);
                for (int cur = 0; cur < f; ++cur) {
                    const int a = __shfl_sync(kFull, a0, cur);
                    const int b = __shfl_sync(kFull, a1, cur);
                    if (a == b) continue;
                    const int64_t row = r + cur;
                    const uint2 own = sign_pair(zb2, row, lane);   // fetched before the entries
                    int cnt[8] = {0, 0, 0, 0, 0, 0, 0, 0};
                    if (b - a >= kSliceMin) count_negatives_sliced(col, a, b, zb, lane, cnt);
                    else count_negatives(col, a, b, zb2, lane, cnt);
                    finish_pass1_row(row, b - a, cnt, own, bslot, y8, y16, y32, lane, cx1, cx2);
                }
                r += f;
                if (f < 32) break;
            }
        }
        flush_x(sx, 0, cx1, lane);   // the chunk's sums, into the CTA's 64-bit totals
        flush_x(sx, 1, cx2, lane);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < kProbes; t += blockDim.x) {
        if (sx[0][t]) atomicAdd(xacc + 3 * t + 0, (unsigned long long)sx[0][t]);
        if (sx[1][t]) atomicAdd(xacc + 3 * t + 1, (unsigned long long)sx[1][t]);
    }
}

// Finish long rows: counts -> y in the row's class array, and their x1, x2
// terms (a huge row's y replaces its counts in y32, lane by lane).
__global__ void __launch_bounds__(kTriThreads) tri_long_rows_kernel(
    const int64_t* __restrict__ rowptr, const int32_t* __restrict__ longlist, int nlong,
    const int32_t* __restrict__ bslot, const uint32_t* __restrict__ zb, uint2* __restrict__ y8,
    uint4* __restrict__ y16, int32_t* __restrict__ y32, unsigned long long* __restrict__ xacc)
{
    __shared__ long long sx[2][kProbes];
    for (int t = threadIdx.x; t < 2 * kProbes; t += blockDim.x) (&sx[0][0])[t] = 0;
    __syncthreads();
    const uint2* zb2 = reinterpret_cast<const uint2*>(zb);
    const int lane = threadIdx.x & 31;
    const int64_t warp = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
    long long x1[8] = {0, 0, 0, 0, 0, 0, 0, 0}, x2[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t i = warp; i < nlong; i += nwarps) {
        const int64_t r = longlist[i];
        const int dg = (int)(rowptr[r + 1] - rowptr[r]);
        const int32_t slot = bslot[r];
        const int32_t* cr = y32 + (size_t)slot * kProbes + 4 * lane;
        const int4 ca = *reinterpret_cast<const int4*>(cr);
        const int4 cb = *reinterpret_cast<const int4*>(cr + kHalf);
        const int yv[8] = {dg - 2 * ca.x, dg - 2 * ca.y, dg - 2 * ca.z, dg - 2 * ca.w,
                           dg - 2 * cb.x, dg - 2 * cb.y, dg - 2 * cb.z, dg - 2 * cb.w};
        store_row(r, dg, yv, sign_pair(zb2, r, lane), slot, y8, y16, y32, lane, x1, x2);
    }
    flush_x(sx, 0, x1, lane);
    flush_x(sx, 1, x2, lane);
    __syncthreads();
    for (int t = threadIdx.x; t < kProbes; t += blockDim.x) {
        if (sx[0][t]) atomicAdd(xacc + 3 * t + 0, (unsigned long long)sx[0][t]);
        if (sx[1][t]) atomicAdd(xacc + 3 * t + 1, (unsigned long long)sx[1][t]);
    }
}

// ---- pass 2 ------------------------------------------------------------------

// s += y of the small targets (rows) listed in col[a, b), this lane's 8
// probes; y8l = y8 + lane; the gathers batched by gather_block.
__device__ __forceinline__ void sum_small(const int32_t* __restrict__ col, int64_t a, int64_t b,
                                          const uint2* __restrict__ y8l, int lane, int s[8])
{
    for (int64_t base = a; base < b; base += 32) {
        const int64_t k = base + lane;
        const int cj = k < b ? __ldg(col + k) : 0;
        const int n = (int)min((int64_t)32, b - base);
        gather_block<8>(cj, n, [&](int j) { return __ldg(y8l + (size_t)j * 32); },
                     [&](uint2 w) {
                         s[0] = __dp4a((int)w.x, 0x00000001, s[0]);
                         s[1] = __dp4a((int)w.x, 0x00000100, s[1]);
                         s[2] = __dp4a((int)w.x, 0x00010000, s[2]);
                         s[3] = __dp4a((int)w.x, 0x01000000, s[3]);
                         s[4] = __dp4a((int)w.y, 0x00000001, s[4]);
                         s[5] = __dp4a((int)w.y, 0x00000100, s[5]);
                         s[6] = __dp4a((int)w.y, 0x00010000, s[6]);
                         s[7] = __dp4a((int)w.y, 0x01000000, s[7]);
                     });
    }
}

// s += y of the mid targets (y16 slots) listed in col[a, b); y16l = y16 + lane.
__device__ __forceinline__ void sum_mid(const int32_t* __restrict__ col, int64_t a, int64_t b,
                                        const uint4* __restrict__ y16l, int lane, int s[8])
{
    for (int64_t base = a; base < b; base += 32) {
        const int64_t k = base + lane;
        const int cj = k < b ? __ldg(col + k) : 0;
        const int n = (int)min((int64_t)32, b - base);
        gather_block<4>(cj, n, [&](int j) { return __ldg(y16l + (size_t)j * 32); },
                     [&](uint4 w) {
                         s[0] = __dp2a_lo((int)w.x, 0x0001, s[0]);
                         s[1] = __dp2a_lo((int)w.x, 0x0100, s[1]);
                         s[2] = __dp2a_lo((int)w.y, 0x0001, s[2]);
                         s[3] = __dp2a_lo((int)w.y, 0x0100, s[3]);
                         s[4] = __dp2a_lo((int)w.z, 0x0001, s[4]);
                         s[5] = __dp2a_lo((int)w.z, 0x0100, s[5]);
                         s[6] = __dp2a_lo((int)w.w, 0x0001, s[6]);
                         s[7] = __dp2a_lo((int)w.w, 0x0100, s[7]);
                     });
    }
}

// y of a small or mid row, this lane's 8 probes, as raw words (a huge row has
// no out-entries: every neighbour above it is huge too).
__device__ __forceinline__ uint4 load_own(int64_t row, int32_t slot, const uint2* __restrict__ y8l,
                                          const uint4* __restrict__ y16l)
{
    if (slot < 0) {
        const uint2 w = __ldg(y8l + (size_t)row * 32);
        return make_uint4(w.x, w.y, 0u, 0u);
    }
    return __ldg(y16l + (size_t)slot * 32);
}

__device__ __forceinline__ void unpack_own(uint4 w, int32_t slot, int yi[8])
{
    if (slot < 0) {
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            yi[q] = (int)(int8_t)(w.x >> (8 * q));
            yi[4 + q] = (int)(int8_t)(w.y >> (8 * q));
        }
    } else {
        const uint32_t v[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
        for (int h = 0; h < 4; ++h) {
            yi[2 * h] = (int)(int16_t)(v[h] & 0xFFFF);
            yi[2 * h + 1] = (int)v[h] >> 16;
        }
    }
}

// x3 += y_i * s, then s = 0.
__device__ __forceinline__ void finish_pass2_row(uint4 own, int32_t slot, int s[8], long long x3[8])
{
    int yi[8];
    unpack_own(own, slot, yi);
#pragma unroll
    for (int q = 0; q < 8; ++q) {
        x3[q] += (long long)yi[q] * s[q];
        s[q] = 0;
    }
}

// sx[block probe] += 2 * x3 of this lane's 8 probes.
__device__ __forceinline__ void flush_x3(long long* sx, const long long x3[8], int lane)
{
#pragma unroll
    for (int q = 0; q < 8; ++q)
        if (x3[q])
            atomicAdd((unsigned long long*)&sx[(q < 4 ? 0 : kHalf) + 4 * lane + (q & 3)],
                      (unsigned long long)(2 * x3[q]));
}

// One edge into a huge row, a warp per pair: x3 += y_i y_h for this lane's 8 probes.
constexpr int64_t kPairBatch = 16;
__device__ __forceinline__ void pair_product(const int4 pr, const uint2* __restrict__ y8, const uint4* __restrict__ y16,
                                             const int32_t* __restrict__ y32, int lane, long long x3[8])
{
    int yi[8];
    if (pr.x == kClassHuge) {
        const int32_t* yr = y32 + (size_t)pr.y * kProbes + 4 * lane;
        const int4 ta = *reinterpret_cast<const int4*>(yr);
        const int4 tb = *reinterpret_cast<const int4*>(yr + kHalf);
        yi[0] = ta.x; yi[1] = ta.y; yi[2] = ta.z; yi[3] = ta.w;
        yi[4] = tb.x; yi[5] = tb.y; yi[6] = tb.z; yi[7] = tb.w;
    } else {
        const int32_t slot = pr.x == kClassSmall ? -1 : pr.y;
        unpack_own(load_own(pr.y, slot, y8 + lane, y16 + lane), slot, yi);
    }
    const int32_t* hr = y32 + (size_t)pr.z * kProbes + 4 * lane;
    const int4 ha = *reinterpret_cast<const int4*>(hr);
    const int4 hb = *reinterpret_cast<const int4*>(hr + kHalf);
    const int h[8] = {ha.x, ha.y, ha.z, ha.w, hb.x, hb.y, hb.z, hb.w};
#pragma unroll
    for (int q = 0; q < 8; ++q) x3[q] += (long long)yi[q] * h[q];
}

// Pass 2: x3 = 2 sum_i y_i sum_{j in out(i)} y_j over the oriented out-lists
// (|s| <= kLongRow * kMidDeg < 2^31: a row part never holds more than
// kLongRow entries and every main target is small or mid), then the pairs of
// edges into huge rows, which fill the warps that the chunks leave idle.
__global__ void __launch_bounds__(kTriThreads, kPass2CtasPerSm) tri_pass2_kernel(
    const int64_t* __restrict__ out_ptr, const int32_t* __restrict__ out_col, const int32_t* __restrict__ nsmall,
    const int32_t* __restrict__ bslot, int64_t d, int64_t nch, const int64_t* __restrict__ crow,
    const uint2* __restrict__ y8, const uint4* __restrict__ y16, const int32_t* __restrict__ y32,
    const int4* __restrict__ pairs, int64_t npairs, unsigned long long* __restrict__ xacc,
    unsigned long long* __restrict__ counter, unsigned long long* __restrict__ pair_counter)
{
    __shared__ long long sx[kProbes];
    for (int t = threadIdx.x; t < kProbes; t += blockDim.x) sx[t] = 0;
    __syncthreads();

    const int lane = threadIdx.x & 31;
    const uint2* y8l = y8 + lane;
    const uint4* y16l = y16 + lane;
    long long x3[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    int s[8] = {0, 0, 0, 0, 0, 0, 0, 0};
    for (int64_t c = next_chunk(counter, lane); c < nch; c = next_chunk(counter, lane)) {
        const int64_t u0 = c * kChunk2, u1 = u0 + kChunk2;
        int64_t r = crow[c];
        while (r < d) {
            const int64_t beg = __ldg(out_ptr + r);
            const int64_t pr = beg + kRowCost * r;
            if (pr >= u1) break;
            const int64_t end = __ldg(out_ptr + r + 1);
            const int64_t deg = end - beg;
            if (deg > kLongRow) {                           // long out-list: this chunk's part
                const int64_t e0 = pr + kRowCost;
                const int64_t a = beg + max((int64_t)0, u0 - e0);
                const int64_t b = beg + min(deg, u1 - e0);
                if (a < b) {
                    const int64_t mid = beg + __ldg(nsmall + r);
                    const int32_t slot = __ldg(bslot + r);
                    const uint4 own = load_own(r, slot, y8l, y16l);
                    sum_small(out_col, a, min(b, mid), y8l, lane, s);
                    sum_mid(out_col, max(a, mid), b, y16l, lane, s);
                    finish_pass2_row(own, slot, s, x3);
                }
                ++r;
                continue;
            }
            if (pr < u0) {
                ++r;
                continue;
            }
            // rows owned by this chunk: row ends, small-section lengths and
            // slots of 32 rows at a time in lanes
            for (;;) {
                const int64_t rr = r + lane;
                int a0 = 0, a1 = 0, ns = 0, sl = -1;
                bool ok = false;
                if (rr < d) {
                    const int64_t s0 = __ldg(out_ptr + rr), e0 = __ldg(out_ptr + rr + 1);
                    a0 = (int)s0;
                    a1 = (int)e0;
                    ok = (s0 + kRowCost * rr < u1) && (e0 - s0 <= kLongRow);
                    if (ok && e0 > s0) {
                        ns = __ldg(nsmall + rr);
                        sl = __ldg(bslot + rr);
                    }
                }
                const unsigned okm = __ballot_sync(kFull, ok);
                const int f = (okm == kFull) ? 32 : (__ffs(~okm) - 1);
                for (int cur = 0; cur < f; ++cur) {
                    const int a = __shfl_sync(kFull, a0, cur);
                    const int b = __shfl_sync(kFull, a1, cur);
                    if (a == b) continue;
                    const int m = a + __shfl_sync(kFull, ns, cur);
                    const int32_t slot = __shfl_sync(kFull, sl, cur);
                    const uint4 own = load_own(r + cur, slot, y8l, y16l);   // fetched before the entries
                    sum_small(out_col, a, m, y8l, lane, s);
                    sum_mid(out_col, m, b, y16l, lane, s);
                    finish_pass2_row(own, slot, s, x3);
                }
                r += f;
                if (f < 32) break;
            }
        }
    }
    // the edges into huge rows, kPairBatch at a time once the chunks are gone
    for (int64_t p0 = next_chunk(pair_counter, lane) * kPairBatch; p0 < npairs;
         p0 = next_chunk(pair_counter, lane) * kPairBatch)
        for (int64_t p = p0; p < min(p0 + kPairBatch, npairs); ++p) pair_product(pairs[p], y8, y16, y32, lane, x3);
    flush_x3(sx, x3, lane);
    __syncthreads();
    for (int t = threadIdx.x; t < kProbes; t += blockDim.x)
        if (sx[t]) atomicAdd(xacc + 3 * t + 2, (unsigned long long)sx[t]);
}

}  // namespace

int tri_prepare(mlt_matrix* M, cudaStream_t s)
{
    if (M->tri_state == 1) return MLT_OK;
    if (M->tri_state < 0) return fail(M->tri_state, "matrix is not a valid triangle-counting input");
    const int64_t d = M->A.nrows;
    const int64_t nnz = M->A.nnz;
    const int64_t nch1 = std::max<int64_t>(1, (nnz + kRowCost * d + kChunk1 - 1) / kChunk1);
    // pass 2's chunks cover the out-lists, at most nnz entries
    const int64_t nch2max = std::max<int64_t>(1, (nnz + kRowCost * d + kChunk2 - 1) / kChunk2);
    int occ1 = 0, occ2 = 0, occc = 0, occf = 0;
    MLT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ1, tri_pass1_kernel, kTriThreads, 0));
    MLT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ2, tri_pass2_kernel, kTriThreads, 0));
    MLT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occc, tri_classify_kernel, kTriThreads, 0));
    MLT_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occf, tri_fill_kernel, kTriThreads, 0));
    const size_t dd = (size_t)std::max<int64_t>(d, 1);
    const int64_t nsb = (d + kScanBlock - 1) / kScanBlock;
    int rc;
    // out_ptr[d+1], crow1[nch1], crow2[nch2max], scan sums[nsb+1]; nsmall,
    // bslot, longlist, deg32 [d] and the fill cursors [2d]; counters
    if ((rc = M->ws_tri.ensure((dd + 1) * 8 + (size_t)(nch1 + nch2max) * 8 + (size_t)(nsb + 1) * 8 + dd * 4 * 6 +
                                   1024,
                               s)))
        return rc;
    char* base = M->ws_tri.as<char>();
    int64_t* out_ptr = reinterpret_cast<int64_t*>(base);
    int64_t* crow1 = out_ptr + dd + 1;
    int64_t* crow2 = crow1 + nch1;
    int64_t* bsum = crow2 + nch2max;
    int32_t* nsmall = reinterpret_cast<int32_t*>(bsum + nsb + 1);
    int32_t* bslot = nsmall + dd;
    int32_t* longlist = bslot + dd;
    int32_t* deg32 = longlist + dd;
    int32_t* cur = deg32 + dd;
    // nbig, nlong, selfloop, npairs, pair cursor, then the bound and four
    // chunk counters (pass 1, pass 2, counting, filling); 16-byte aligned: the
    // int32 arrays before it may end anywhere
    int* counters = reinterpret_cast<int*>((reinterpret_cast<uintptr_t>(cur + 2 * dd) + 15) & ~(uintptr_t)15);
    double* bound = reinterpret_cast<double*>(counters + 6);
    unsigned long long* chunk_ctr = reinterpret_cast<unsigned long long*>(bound + 1);
    MLT_CUDA_TRY(cudaMemsetAsync(counters, 0, 6 * sizeof(int) + sizeof(double) + 4 * sizeof(unsigned long long), s));
    const int gridc = std::max(1, occc) * M->num_sms, gridf = std::max(1, occf) * M->num_sms;
    {
        ProfScope ps("tri_prepare", s);
        const int gd = (int)std::max<int64_t>(1, std::min<int64_t>((d + 255) / 256, 16LL * M->num_sms));
        tri_degrees_kernel<<<gd, 256, 0, s>>>(M->A.rowptr, d, deg32, bslot, longlist, out_ptr, nsmall, cur,
                                              counters);
        const int g1 = (int)std::min<int64_t>((nch1 + 255) / 256, 16LL * M->num_sms);
        chunk_rows_kernel<<<std::max(g1, 1), 256, 0, s>>>(M->A.rowptr, d, nch1, kChunk1, crow1);
        tri_classify_kernel<<<gridc, kTriThreads, 0, s>>>(M->A.rowptr, M->A.col, deg32, d, nch1, crow1, out_ptr,
                                                          nsmall, counters, bound, chunk_ctr + 2);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    if (d > 0) {
        ProfScope ps("tri_scan", s);
        scan_sums_kernel<<<(unsigned)nsb, 256, 0, s>>>(out_ptr, d, bsum);
        scan_offsets_kernel<<<1, 1024, 0, s>>>(bsum, nsb, out_ptr + d);
        scan_apply_kernel<<<(unsigned)nsb, 256, 0, s>>>(out_ptr, d, bsum);
    } else {
        MLT_CUDA_TRY(cudaMemsetAsync(out_ptr, 0, sizeof(int64_t), s));
    }
    MLT_CUDA_TRY(cudaGetLastError());
    int hc[4] = {0, 0, 0, 0};
    double hb = 0.0;
    int64_t nnz_out = 0;
    MLT_CUDA_TRY(cudaMemcpyAsync(hc, counters, sizeof(hc), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaMemcpyAsync(&hb, bound, sizeof(double), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaMemcpyAsync(&nnz_out, out_ptr + d, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
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
    const int64_t npairs = hc[3];
    // out_col (16-byte aligned end) then the pair list
    const size_t col_bytes = ((size_t)std::max<int64_t>(nnz_out, 1) * sizeof(int32_t) + 15) & ~(size_t)15;
    if ((rc = M->ws_upcol.ensure(col_bytes + (size_t)std::max<int64_t>(npairs, 1) * sizeof(int4), s))) return rc;
    int32_t* out_col = M->ws_upcol.as<int32_t>();
    int4* pairs = reinterpret_cast<int4*>(M->ws_upcol.as<char>() + col_bytes);
    const int64_t nch2 = std::max<int64_t>(1, (nnz_out + kRowCost * d + kChunk2 - 1) / kChunk2);
    {
        ProfScope ps("tri_fill_out", s);
        tri_fill_kernel<<<gridf, kTriThreads, 0, s>>>(M->A.rowptr, M->A.col, deg32, d, nch1, crow1, out_ptr, nsmall,
                                                      bslot, cur, out_col, pairs, (int)npairs, counters + 4,
                                                      chunk_ctr + 3);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    {
        ProfScope ps("tri_chunk_rows", s);
        const int g2 = (int)std::min<int64_t>((nch2 + 255) / 256, 16LL * M->num_sms);
        chunk_rows_kernel<<<std::max(g2, 1), 256, 0, s>>>(out_ptr, d, nch2, kChunk2, crow2);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    M->tri.out_ptr = out_ptr;
    M->tri.out_col = out_col;
    M->tri.nsmall = nsmall;
    M->tri.pairs = pairs;
    M->tri.npairs = npairs;
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
    const size_t nbig = (size_t)std::max(T.nbig, 1);
    if ((rc = M->ws_z.ensure(dd * kZWords * sizeof(uint32_t), s))) return rc;
    if ((rc = M->ws_y.ensure(dd * kProbes, s))) return rc;
    if ((rc = M->ws_y16.ensure(nbig * kProbes * sizeof(int16_t), s))) return rc;
    if ((rc = M->ws_y32.ensure(nbig * kProbes * sizeof(int32_t), s))) return rc;
    if ((rc = M->ws_x.ensure((size_t)kProbes * 3 * sizeof(unsigned long long), s))) return rc;
    uint32_t* zb = M->ws_z.as<uint32_t>();
    uint2* y8 = M->ws_y.as<uint2>();
    uint4* y16 = M->ws_y16.as<uint4>();
    int32_t* y32 = M->ws_y32.as<int32_t>();
    unsigned long long* xacc = M->ws_x.as<unsigned long long>();
    MLT_CUDA_TRY(cudaMemsetAsync(xacc, 0, (size_t)kProbes * 3 * sizeof(unsigned long long), s));
    // chunk counters of pass 1 and pass 2 and pass 2's pair counter (the third
    // slot served the preparation's counting pass before any block ran)
    MLT_CUDA_TRY(cudaMemsetAsync(T.counters, 0, 3 * sizeof(unsigned long long), s));
    {
        const int64_t total = d * kZWords;
        const int g = (int)std::max<int64_t>(1, std::min<int64_t>((total + 255) / 256, 16LL * M->num_sms));
        ProfScope ps("tri_zbits", s);
        zbits_kernel<<<g, 256, 0, s>>>(d, seed * kGolden, id0, nb, zb, T.longlist, T.nlong, T.bslot, y32);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    {
        ProfScope ps("tri_pass1", s);
        tri_pass1_kernel<<<T.grid1, kTriThreads, 0, s>>>(M->A.rowptr, M->A.col, d, T.nch1, T.crow1, T.bslot,
                                                         zb, y8, y16, y32, xacc, T.counters);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    if (T.nlong > 0) {
        const int g = (int)std::min<int64_t>(((int64_t)T.nlong * 32 + kTriThreads - 1) / kTriThreads,
                                             4LL * M->num_sms);
        ProfScope ps("tri_long_rows", s);
        tri_long_rows_kernel<<<std::max(g, 1), kTriThreads, 0, s>>>(M->A.rowptr, T.longlist, T.nlong,
                                                                    T.bslot, zb, y8, y16, y32, xacc);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    {
        ProfScope ps("tri_pass2", s);
        tri_pass2_kernel<<<T.grid2, kTriThreads, 0, s>>>(T.out_ptr, T.out_col, T.nsmall, T.bslot, d, T.nch2,
                                                         T.crow2, y8, y16, y32, T.pairs, T.npairs, xacc,
                                                         T.counters + 1, T.counters + 2);
    }
    MLT_CUDA_TRY(cudaGetLastError());
    MLT_CUDA_TRY(cudaMemcpyAsync(x_dev, xacc, (size_t)nb * 3 * sizeof(int64_t), cudaMemcpyDeviceToDevice, s));
    return MLT_OK;
}

}  // namespace mlt
