// The C ABI declared in include/mlt.h: argument checking, device memory of the
// matrix handles, probe ordering and grouping for the moment engine, and the
// multilevel and triangle drivers that tie kernels and host arithmetic together.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <mutex>
#include <new>
#include <numeric>
#include <string>
#include <vector>

#include "mlt_internal.h"

namespace mlt {

static thread_local std::string g_error;

void set_error(const std::string& msg) { g_error = msg; }

int fail(int code, const std::string& msg)
{
    g_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char* what)
{
    if (e == cudaSuccess) return MLT_OK;
    g_error = std::string(what) + ": " + cudaGetErrorString(e);
    if (e == cudaErrorMemoryAllocation) return MLT_ENOMEM;
    return MLT_ECUDA;
}

// ---- kernel timing ---------------------------------------------------------
namespace {
struct ProfRec {
    const char* name;
    cudaEvent_t e0, e1;
};
std::mutex g_prof_mu;
bool g_prof_on = false;
std::vector<ProfRec> g_prof;
std::vector<cudaEvent_t> g_event_pool;

cudaEvent_t take_event()
{
    if (!g_event_pool.empty()) {
        cudaEvent_t e = g_event_pool.back();
        g_event_pool.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}
}  // namespace

static thread_local int g_prof_paused = 0;
ProfPause::ProfPause() { ++g_prof_paused; }
ProfPause::~ProfPause() { --g_prof_paused; }

ProfScope::ProfScope(const char* name, cudaStream_t stream) : idx(-1), s(stream)
{
    if (!g_prof_on || g_prof_paused) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    ProfRec r{name, take_event(), take_event()};
    if (!r.e0 || !r.e1) return;
    cudaEventRecord(r.e0, s);
    g_prof.push_back(r);
    idx = (int)g_prof.size() - 1;
}

ProfScope::~ProfScope()
{
    if (idx < 0) return;
    std::lock_guard<std::mutex> lk(g_prof_mu);
    cudaEventRecord(g_prof[idx].e1, s);
}

namespace {
constexpr int kMaxDevices = 64;
std::mutex g_pool_mu;
cudaMemPool_t g_pools[kMaxDevices] = {};
}  // namespace

cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return e;
    if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
    cudaMemPool_t pool;
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g_pools[dev]) {
            cudaMemPoolProps props = {};
            props.allocType = cudaMemAllocationTypePinned;
            props.handleTypes = cudaMemHandleTypeNone;
            props.location.type = cudaMemLocationTypeDevice;
            props.location.id = dev;
            if ((e = cudaMemPoolCreate(&g_pools[dev], &props)) != cudaSuccess) {
                g_pools[dev] = nullptr;
                return e;
            }
            uint64_t keep = ~(uint64_t)0;   // never trim at synchronisation
            if ((e = cudaMemPoolSetAttribute(g_pools[dev], cudaMemPoolAttrReleaseThreshold, &keep)) != cudaSuccess)
                return e;
        }
        pool = g_pools[dev];
    }
    return cudaMallocFromPoolAsync(p, bytes, pool, s);
}

// Every pool's cached blocks back to the driver (blocks in use stay).
cudaError_t trim_pools()
{
    std::lock_guard<std::mutex> lk(g_pool_mu);
    for (cudaMemPool_t pool : g_pools) {
        if (!pool) continue;
        cudaError_t e = cudaMemPoolTrimTo(pool, 0);
        if (e != cudaSuccess) return e;
    }
    return cudaSuccess;
}

int DevBuf::ensure(size_t want, cudaStream_t s)
{
    if (want <= bytes) return MLT_OK;
    if (p) {
        cudaFreeAsync(p, s);
        p = nullptr;
        bytes = 0;
    }
    size_t sz = want + want / 8;
    sz = (sz + (1u << 21) - 1) & ~((size_t)(1u << 21) - 1);
    cudaError_t e = pool_malloc(&p, sz, s);
    if (e != cudaSuccess) {
        p = nullptr;
        cudaGetLastError();
        return fail(MLT_ENOMEM, "device scratch allocation of " + std::to_string(sz) + " bytes failed");
    }
    bytes = sz;
    return MLT_OK;
}

// The device is idle for this buffer (a handle is released after a
// synchronisation), so the block returns to the pool at once.
void DevBuf::release()
{
    if (p) cudaFreeAsync(p, 0);
    p = nullptr;
    bytes = 0;
}

static bool is_device_ptr(const void* ptr)
{
    if (!ptr) return false;
    cudaPointerAttributes at;
    cudaError_t e = cudaPointerGetAttributes(&at, ptr);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
static int dev_alloc_copy(T** dst, const void* src, size_t count, bool src_dev, cudaStream_t s)
{
    *dst = nullptr;
    if (count == 0) count = 1;
    if (pool_malloc((void**)dst, count * sizeof(T), s) != cudaSuccess) {
        cudaGetLastError();
        return fail(MLT_ENOMEM, "device allocation for the matrix failed");
    }
    if (src) {
        MLT_CUDA_TRY(cudaMemcpyAsync(*dst, src, count * sizeof(T),
                                     src_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, s));
    }
    return MLT_OK;
}

// Eight independent FP64 FMA chains per thread, `iters` steps, all in
// registers: the FP64 pipe's rate with no memory traffic (the denominator of
// FP64-bound rooflines).  The result is stored so that nothing is elided.
__global__ void fp64_fma_kernel(double* sink, int64_t iters)
{
    double x[8];
    const double m = 1.0 + 1e-12 * threadIdx.x, c = 1e-9;
#pragma unroll
    for (int i = 0; i < 8; ++i) x[i] = (double)(i + 1);
    for (int64_t k = 0; k < iters; ++k) {
#pragma unroll
        for (int i = 0; i < 8; ++i) x[i] = fma(x[i], m, c);
    }
    double t = 0.0;
#pragma unroll
    for (int i = 0; i < 8; ++i) t += x[i];
    sink[blockIdx.x * (int64_t)blockDim.x + threadIdx.x] = t;
}

__global__ void f32_to_f64_kernel(const float* __restrict__ in, double* __restrict__ out, int64_t n)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n;
         i += (int64_t)gridDim.x * blockDim.x)
        out[i] = (double)in[i];
}

// CSR sanity in two fully parallel passes (no thread walks a whole row):
// per row, rowptr must be non-decreasing within [0, nnz] and each non-empty
// row marks its first entry in a bitmap; per entry, the column must lie in
// [0, ncols) and exceed the previous entry's unless a row starts there.
// bad[0] |= 1 (rowptr), 2 (column range), 4 (order or duplicate).
__global__ void validate_rows_kernel(const int64_t* __restrict__ rowptr, int64_t nrows, int64_t nnz,
                                     unsigned* __restrict__ starts, int* bad)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows;
         r += (int64_t)gridDim.x * blockDim.x) {
        const int64_t beg = rowptr[r], end = rowptr[r + 1];
        if (beg < 0 || end > nnz || end < beg) {
            atomicOr(bad, 1);
            continue;
        }
        if (end > beg) atomicOr(starts + (beg >> 5), 1u << (beg & 31));
    }
}

__global__ void validate_cols_kernel(const int32_t* __restrict__ col, int64_t nnz, int64_t ncols,
                                     const unsigned* __restrict__ starts, int* bad)
{
    for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < nnz;
         k += (int64_t)gridDim.x * blockDim.x) {
        const int64_t c = col[k];
        if (c < 0 || c >= ncols) {
            atomicOr(bad, 2);
            continue;
        }
        const bool first = (starts[k >> 5] >> (k & 31)) & 1u;
        if (!first && (k == 0 || c <= (int64_t)col[k - 1])) atomicOr(bad, 4);
    }
}

// Gershgorin discs: lo_i = a_ii - r_i, hi_i = a_ii + r_i (scaled entries).
__global__ void gershgorin_kernel(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                  const double* __restrict__ val, double scale, int64_t d,
                                  double* lo_out, double* hi_out)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < d;
         r += (int64_t)gridDim.x * blockDim.x) {
        double dg = 0.0, off = 0.0;
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
            const double v = (val ? val[k] : 1.0) * scale;
            if (col[k] == r) dg += v;
            else off += fabs(v);
        }
        lo_out[r] = dg - off;
        hi_out[r] = dg + off;
    }
}

// ||X||_1 (max column sum) and ||X||_inf (max row sum) for a Gram bound.
__global__ void absrow_kernel(const int64_t* __restrict__ rowptr, const double* __restrict__ val,
                              double scale, int64_t nrows, double* out)
{
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows;
         r += (int64_t)gridDim.x * blockDim.x) {
        double s = 0.0;
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) s += fabs((val ? val[k] : 1.0) * scale);
        out[r] = s;
    }
}

// Per CTA: the sum of the diagonal and the sum of squared values of rows
// blockIdx.x*256 + threadIdx.x (+ grid stride), reduced in a fixed tree.
__global__ void __launch_bounds__(256) low_sums_kernel(const int64_t* __restrict__ rowptr,
                                                       const int32_t* __restrict__ col,
                                                       const double* __restrict__ val, int64_t nrows,
                                                       double* __restrict__ part)
{
    __shared__ double sd[256], ss[256];
    double dg = 0.0, sq = 0.0;
    for (int64_t r = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; r < nrows;
         r += (int64_t)gridDim.x * blockDim.x) {
        for (int64_t k = rowptr[r]; k < rowptr[r + 1]; ++k) {
            const double v = val ? val[k] : 1.0;
            if (col[k] == r) dg += v;
            sq += v * v;
        }
    }
    sd[threadIdx.x] = dg;
    ss[threadIdx.x] = sq;
    __syncthreads();
    for (int o = 128; o; o >>= 1) {
        if ((int)threadIdx.x < o) {
            sd[threadIdx.x] += sd[threadIdx.x + o];
            ss[threadIdx.x] += ss[threadIdx.x + o];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        part[2 * blockIdx.x] = sd[0];
        part[2 * blockIdx.x + 1] = ss[0];
    }
}

// tr T_j(At) for j = 0, 1, 2 (j <= 1 for a Gram handle) from d, tr A and
// ||A||_F^2 (closing remark of Section 5.4); the two sums are reduced on the
// device once per handle, in a fixed order.
int low_traces(mlt_matrix* M, double a, double b, double* t, int* count, cudaStream_t s)
{
    if (!M->low_ready) {
        const int64_t nr = M->A.nrows;
        const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((nr + 255) / 256, 16LL * M->num_sms));
        int rc;
        if ((rc = M->ws_out.ensure((size_t)2 * nb * sizeof(double), s))) return rc;
        double* part = M->ws_out.as<double>();
        {
            ProfScope ps("low_sums", s);
            low_sums_kernel<<<nb, 256, 0, s>>>(M->A.rowptr, M->A.col, M->A.val64, nr, part);
        }
        MLT_CUDA_TRY(cudaGetLastError());
        std::vector<double> h(2 * (size_t)nb);
        MLT_CUDA_TRY(cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        MLT_CUDA_TRY(cudaStreamSynchronize(s));
        double dg = 0.0, sq = 0.0;
        for (int i = 0; i < nb; ++i) {
            dg += h[2 * (size_t)i];
            sq += h[2 * (size_t)i + 1];
        }
        M->low_diag = dg;
        M->low_sq = sq;
        M->low_ready = true;
    }
    const double alpha = 2.0 / (b - a), beta = -(a + b) / (b - a);
    const double sc = M->scale;
    const double d = (double)M->dim();
    if (M->flags & MLT_GRAM) {
        t[0] = d;
        t[1] = alpha * (sc * sc * M->low_sq) + beta * d;
        t[2] = 0.0;
        if (count) *count = 2;
        return MLT_OK;
    }
    const double tr_a = sc * M->low_diag, tr_a2 = sc * sc * M->low_sq;
    t[0] = d;
    t[1] = alpha * tr_a + beta * d;
    t[2] = 2.0 * (alpha * alpha * tr_a2 + 2.0 * alpha * beta * tr_a + beta * beta * d) - d;
    if (count) *count = 3;
    return MLT_OK;
}

int gershgorin_device(mlt_matrix* M, double* lo, double* hi, cudaStream_t s)
{
    int rc;
    const bool gram = (M->flags & MLT_GRAM) != 0;
    if (!gram) {
        const int64_t d = M->A.nrows;
        if ((rc = M->ws_out.ensure((size_t)2 * std::max<int64_t>(d, 1) * sizeof(double), s))) return rc;
        double* buf = M->ws_out.as<double>();
        const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((d + 255) / 256, 16LL * M->num_sms));
        ProfScope ps("gershgorin", s);
        gershgorin_kernel<<<nb, 256, 0, s>>>(M->A.rowptr, M->A.col, M->A.val64, M->scale, d, buf, buf + d);
        MLT_CUDA_TRY(cudaGetLastError());
        std::vector<double> h(2 * d);
        MLT_CUDA_TRY(cudaMemcpyAsync(h.data(), buf, 2 * d * sizeof(double), cudaMemcpyDeviceToHost, s));
        MLT_CUDA_TRY(cudaStreamSynchronize(s));
        double l = INFINITY, u = -INFINITY;
        for (int64_t i = 0; i < d; ++i) { l = std::min(l, h[i]); u = std::max(u, h[d + i]); }
        *lo = l;
        *hi = u;
        return MLT_OK;
    }
    const int64_t nr = M->A.nrows, nc = M->A.ncols;
    const int64_t tot = nr + nc;
    if ((rc = M->ws_out.ensure((size_t)std::max<int64_t>(tot, 1) * sizeof(double), s))) return rc;
    double* buf = M->ws_out.as<double>();
    int nb = (int)std::max<int64_t>(1, std::min<int64_t>((nr + 255) / 256, 16LL * M->num_sms));
    ProfScope ps("abs_row_sums", s);
    absrow_kernel<<<nb, 256, 0, s>>>(M->A.rowptr, M->A.val64, M->scale, nr, buf);
    nb = (int)std::max<int64_t>(1, std::min<int64_t>((nc + 255) / 256, 16LL * M->num_sms));
    absrow_kernel<<<nb, 256, 0, s>>>(M->AT.rowptr, M->AT.val64, M->scale, nc, buf + nr);
    MLT_CUDA_TRY(cudaGetLastError());
    std::vector<double> h(tot);
    MLT_CUDA_TRY(cudaMemcpyAsync(h.data(), buf, tot * sizeof(double), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaStreamSynchronize(s));
    double rmax = 0.0, cmax = 0.0;
    for (int64_t i = 0; i < nr; ++i) rmax = std::max(rmax, h[i]);
    for (int64_t i = 0; i < nc; ++i) cmax = std::max(cmax, h[nr + i]);
    *lo = 0.0;
    *hi = rmax * cmax;
    return MLT_OK;
}

static void free_matrix(mlt_matrix* M)
{
    void* owned[] = {M->own_rowptr, M->own_col, M->own_val, M->own_val32, M->own_t_rowptr,
                     M->own_t_col, M->own_t_val, M->own_t_val32, M->own_val_df, M->own_t_val_df,
                     M->own_p_rowptr, M->own_p_col, M->own_p_val, M->own_p_val32, M->own_p_val_df,
                     M->perm, M->plan_A.mem, M->plan_AT.mem, M->plan_P.mem};
    for (void* p : owned)
        if (p) cudaFreeAsync(p, 0);   // called with the handle's work finished
    mlt::DevBuf* bufs[] = {&M->ws_v[0], &M->ws_v[1], &M->ws_v2[0], &M->ws_v2[1], &M->ws_w, &M->ws_part, &M->ws_dots,
                           &M->ws_misc, &M->ws_out, &M->ws_y, &M->ws_y16, &M->ws_y32, &M->ws_z, &M->ws_x,
                           &M->ws_tri, &M->ws_seg, &M->ws_upcol, &M->ws_blk[0], &M->ws_blk[1], &M->ws_blk[2],
                           &M->ws_blk[3]};
    for (auto* b : bufs) b->release();
}

// Transpose a host CSR (counting sort by column; rows stay ascending).
static void host_transpose(int64_t nrows, int64_t ncols, const int64_t* rp, const int32_t* ci,
                           const double* v, std::vector<int64_t>& trp, std::vector<int32_t>& tci,
                           std::vector<double>& tv)
{
    const int64_t nnz = rp[nrows];
    trp.assign(ncols + 1, 0);
    for (int64_t k = 0; k < nnz; ++k) ++trp[ci[k] + 1];
    for (int64_t j = 0; j < ncols; ++j) trp[j + 1] += trp[j];
    std::vector<int64_t> pos(trp.begin(), trp.end() - 1);
    tci.resize(std::max<int64_t>(nnz, 1));
    if (v) tv.resize(std::max<int64_t>(nnz, 1));
    for (int64_t i = 0; i < nrows; ++i)
        for (int64_t k = rp[i]; k < rp[i + 1]; ++k) {
            const int64_t q = pos[ci[k]]++;
            tci[q] = (int32_t)i;
            if (v) tv[q] = v[k];
        }
}


// ---- moment jobs: prepare (validation, probe order, groups, device metadata,
// every allocation), enqueue (kernels only: no host sync, no allocation, so a
// job can be captured in a graph), finish (results to the caller, checks) ----

int prepare_moment_job(mlt_matrix* m, double a, double b, uint64_t seed, int64_t probe_offset, int64_t nprobes,
                       const int32_t* degree, int precision, unsigned flags, double* mu, int64_t ld_mu,
                       int group_width, MomentJob& J, cudaStream_t s)
{
    if (!m) return fail(MLT_EINVAL, "mlt_moments: null handle");
    if (int rcb = handle_busy(m, "mlt_moments")) return rcb;
    if (nprobes < 0) return fail(MLT_EINVAL, "mlt_moments: negative probe count");
    if (nprobes > 0 && (!degree || !mu)) return fail(MLT_EINVAL, "mlt_moments: null degree or mu");
    if (!(a < b) || !std::isfinite(a) || !std::isfinite(b))
        return fail(MLT_EINVAL, "mlt_moments: need finite a < b");
    if (precision != MLT_PREC_FP64 && precision != MLT_PREC_FP32 && precision != MLT_PREC_DF64 &&
        !((precision & 0xFF) == MLT_PREC_MIXED && precision >= 0))
        return fail(MLT_EINVAL, "mlt_moments: unknown precision");
    if (flags & ~MLT_DIRECT) return fail(MLT_EINVAL, "mlt_moments: unknown flags");
    if (probe_offset < 0 || probe_offset + nprobes > (1LL << 32))
        return fail(MLT_EINVAL, "mlt_moments: probe ids must lie in [0, 2^32)");
    if (group_width < 0) return fail(MLT_EINVAL, "mlt_moments: negative group width");
    int maxdeg = 0;
    for (int64_t p = 0; p < nprobes; ++p) {
        if (degree[p] < 0 || degree[p] > MLT_MAX_DEGREE) return fail(MLT_EINVAL, "mlt_moments: degree out of range");
        maxdeg = std::max(maxdeg, (int)degree[p]);
    }
    if (nprobes > 0 && ld_mu < maxdeg + 1) return fail(MLT_EINVAL, "mlt_moments: ld_mu below max degree + 1");
    J = MomentJob();
    J.m = m;
    J.a = a;
    J.b = b;
    J.seed = seed;
    J.precision = precision;
    J.direct = (flags & MLT_DIRECT) ? 1 : 0;
    J.mu_user = mu;
    J.ld_mu = ld_mu;
    J.nprobes = nprobes;
    if (nprobes == 0) return MLT_OK;
    const int64_t d = m->dim();
    int rc;
    J.out_dev = is_device_ptr(mu);
    J.out_bytes = (size_t)nprobes * ld_mu * sizeof(double);
    J.mu_dev = mu;
    if (!J.out_dev) {
        if ((rc = m->ws_out.ensure(J.out_bytes, s))) return rc;
        J.mu_dev = m->ws_out.as<double>();
    }
    // probe order: by degree, descending (stable), so live probes are a prefix
    std::vector<int64_t> order(nprobes);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int64_t x, int64_t y) { return degree[x] > degree[y]; });
    // group width: the caller's, else m->group_width (autotuned), else from memory
    int64_t gmax = group_width > 0 ? group_width : m->group_width;
    if (gmax <= 0) {
        const size_t sv = precision == MLT_PREC_FP32 ? sizeof(float) : sizeof(double);
        const bool gram = (m->flags & MLT_GRAM) != 0;
        const size_t per_probe = sv * ((size_t)2 * std::max<int64_t>(d, 1) + (gram ? (size_t)m->A.nrows : 0));
        size_t free_b = 0, total_b = 0;
        MLT_CUDA_TRY(cudaMemGetInfo(&free_b, &total_b));
        const size_t budget = std::min<size_t>((size_t)16 << 30, free_b / 3);
        gmax = (int64_t)std::max<size_t>(8, budget / per_probe);
        // large operators gather more than they stream: at 8-byte vectors the
        // 512-byte row slices of 64 probes measured fastest (R-MAT scale 22:
        // 9.2 ms a step at 64 against 19.8 ms at 128, for twice the probes)
        if (sv == sizeof(double) && d >= (int64_t(1) << 20)) gmax = std::min<int64_t>(gmax, 64);
    }
    gmax = std::min<int64_t>(gmax, 1024);
    const int64_t ngroups = (nprobes + gmax - 1) / gmax;
    const int64_t gsz = (nprobes + ngroups - 1) / ngroups;
    // device metadata for every group at once: error flag, then ids, rows, degrees
    const size_t meta = 256 + (size_t)nprobes * (2 * sizeof(int64_t) + sizeof(int32_t)) + 256;
    if ((rc = m->ws_misc.ensure(meta, s))) return rc;
    char* base = m->ws_misc.as<char>();
    J.err = reinterpret_cast<int*>(base);
    int64_t* ids_dev = reinterpret_cast<int64_t*>(base + 256);
    int64_t* row_dev = ids_dev + nprobes;
    int32_t* deg_dev = reinterpret_cast<int32_t*>(row_dev + nprobes);
    std::vector<int64_t> hid(nprobes), hrow(nprobes);
    std::vector<int32_t> hdeg(nprobes);
    for (int64_t c = 0; c < nprobes; ++c) {
        hid[c] = probe_offset + order[c];
        hrow[c] = order[c];
        hdeg[c] = degree[order[c]];
    }
    MLT_CUDA_TRY(cudaMemsetAsync(J.err, 0, sizeof(int), s));
    MLT_CUDA_TRY(cudaMemcpyAsync(ids_dev, hid.data(), nprobes * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    MLT_CUDA_TRY(cudaMemcpyAsync(row_dev, hrow.data(), nprobes * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    MLT_CUDA_TRY(cudaMemcpyAsync(deg_dev, hdeg.data(), nprobes * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    for (int64_t g0 = 0; g0 < nprobes; g0 += gsz) {
        const int B = (int)std::min<int64_t>(gsz, nprobes - g0);
        int K = 0;
        for (int c = 0; c < B; ++c) K = std::max(K, J.direct ? hdeg[g0 + c] : (hdeg[g0 + c] + 1) / 2);
        std::vector<int> act(std::max(K, 1));
        for (int k = 0; k < K; ++k) {
            int n = 0;
            while (n < B && (J.direct ? hdeg[g0 + n] : (hdeg[g0 + n] + 1) / 2) > k) ++n;
            act[k] = n;
        }
        J.acts.push_back(std::move(act));
        MomentPlan plan;
        plan.dim = d;
        plan.B = B;
        plan.ldv = (B + 7) & ~7;
        plan.K = K;
        plan.act = nullptr;
        plan.ids_dev = ids_dev + g0;
        plan.deg_dev = deg_dev + g0;
        plan.row_dev = row_dev + g0;
        plan.direct = J.direct;
        J.groups.push_back(plan);
    }
    for (size_t i = 0; i < J.groups.size(); ++i) J.groups[i].act = J.acts[i].data();
    // every device buffer the kernels will use, sized now
    for (auto& plan : J.groups)
        if ((rc = run_moments_group(m, precision, plan, a, b, seed, J.mu_dev, ld_mu, J.err, s, true))) return rc;
    return MLT_OK;
}

int enqueue_moment_job(MomentJob& J, cudaStream_t s)
{
    for (auto& plan : J.groups) {
        int rc = run_moments_group(J.m, J.precision, plan, J.a, J.b, J.seed, J.mu_dev, J.ld_mu, J.err, s, false);
        if (rc) return rc;
    }
    return MLT_OK;
}

int finish_moment_job(MomentJob& J, cudaStream_t s)
{
    if (J.nprobes == 0) return MLT_OK;
    if (!J.out_dev) MLT_CUDA_TRY(cudaMemcpyAsync(J.mu_user, J.mu_dev, J.out_bytes, cudaMemcpyDeviceToHost, s));
    int herr = 0;
    MLT_CUDA_TRY(cudaMemcpyAsync(&herr, J.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaStreamSynchronize(s));
    if (herr) return fail(MLT_ERANGE, "mlt_moments: |mu_j| > d; the spectrum is not inside [a, b]");
    return MLT_OK;
}

}  // namespace mlt

using namespace mlt;

extern "C" {

const char* mlt_last_error(void) { return g_error.c_str(); }

int mlt_profile_start(void)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    for (auto& r : g_prof) {
        g_event_pool.push_back(r.e0);
        g_event_pool.push_back(r.e1);
    }
    g_prof.clear();
    g_prof_on = true;
    return MLT_OK;
}

int mlt_profile_stop(mlt_kernel_stat* stats, int max_stats, int* nstats)
{
    std::lock_guard<std::mutex> lk(g_prof_mu);
    g_prof_on = false;
    std::map<std::string, std::pair<int64_t, double>> agg;
    int rc = MLT_OK;
    for (auto& r : g_prof) {
        float ms = 0.0f;
        cudaError_t e = cudaEventSynchronize(r.e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, r.e0, r.e1);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "mlt_profile_stop");
            continue;
        }
        auto& a = agg[r.name];
        a.first += 1;
        a.second += ms;
        g_event_pool.push_back(r.e0);
        g_event_pool.push_back(r.e1);
    }
    g_prof.clear();
    int n = 0;
    for (auto& kv : agg) {
        if (stats && n < max_stats) {
            std::memset(stats[n].name, 0, sizeof(stats[n].name));
            std::strncpy(stats[n].name, kv.first.c_str(), sizeof(stats[n].name) - 1);
            stats[n].launches = kv.second.first;
            stats[n].total_ms = kv.second.second;
        }
        ++n;
    }
    if (nstats) *nstats = std::min(n, max_stats);
    return rc;
}

int mlt_create_csr(int64_t nrows, int64_t ncols, int64_t nnz, const int64_t* rowptr,
                   const int32_t* col, const void* vals, int val_type, double scale, unsigned flags,
                   void* stream, mlt_matrix** out)
{
    try {
        if (!out) return fail(MLT_EINVAL, "mlt_create_csr: null output handle");
        *out = nullptr;
        if (nrows < 0 || ncols < 0 || nnz < 0) return fail(MLT_EINVAL, "mlt_create_csr: negative size");
        if (nnz > 2147483647LL) return fail(MLT_EINVAL, "mlt_create_csr: nnz must be below 2^31");
        if (nrows > 2147483647LL || ncols > 2147483647LL)
            return fail(MLT_EINVAL, "mlt_create_csr: dimensions must be below 2^31");
        if (!rowptr) return fail(MLT_EINVAL, "mlt_create_csr: null rowptr");
        if (nnz > 0 && !col) return fail(MLT_EINVAL, "mlt_create_csr: null col");
        if (val_type != MLT_F64 && val_type != MLT_F32 && val_type != MLT_PATTERN)
            return fail(MLT_EINVAL, "mlt_create_csr: unknown value type");
        if (val_type != MLT_PATTERN && nnz > 0 && !vals)
            return fail(MLT_EINVAL, "mlt_create_csr: null values");
        if (!std::isfinite(scale)) return fail(MLT_EINVAL, "mlt_create_csr: scale must be finite");
        const bool gram = (flags & MLT_GRAM) != 0;
        if (!gram && nrows != ncols) return fail(MLT_EINVAL, "mlt_create_csr: matrix must be square");
        if (flags & ~(MLT_GRAM | MLT_DEVICE_PTRS | MLT_REORDER)) return fail(MLT_EINVAL, "mlt_create_csr: unknown flags");
        if ((flags & MLT_REORDER) && gram) return fail(MLT_EINVAL, "mlt_create_csr: MLT_REORDER needs a square operator, not X^T X");
        const bool dev = (flags & MLT_DEVICE_PTRS) != 0;
        cudaStream_t s = (cudaStream_t)stream;

        int64_t r0 = 0, rn = 0;
        if (dev) {
            MLT_CUDA_TRY(cudaMemcpy(&r0, rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost));
            MLT_CUDA_TRY(cudaMemcpy(&rn, rowptr + nrows, sizeof(int64_t), cudaMemcpyDeviceToHost));
        } else {
            r0 = rowptr[0];
            rn = rowptr[nrows];
        }
        if (r0 != 0 || rn != nnz) return fail(MLT_EINVAL, "mlt_create_csr: rowptr[0] must be 0 and rowptr[nrows] nnz");

        int device = 0, num_sms = 0;
        MLT_CUDA_TRY(cudaGetDevice(&device));
        MLT_CUDA_TRY(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, device));
        mlt_matrix* M = new (std::nothrow) mlt_matrix();
        if (!M) return fail(MLT_ENOMEM, "mlt_create_csr: host allocation failed");
        int rc = MLT_OK;
        auto bail = [&](int code) {
            cudaStreamSynchronize(s);
            free_matrix(M);
            delete M;
            return code;
        };
        M->device = device;
        M->num_sms = num_sms;
        M->val_type = val_type;
        M->flags = flags;
        M->scale = scale;
        M->A.nrows = nrows;
        M->A.ncols = ncols;
        M->A.nnz = nnz;

        // rowptr / col
        if (dev) {
            M->A.rowptr = rowptr;
            M->A.col = col;
        } else {
            int64_t* rp = nullptr;
            int32_t* ci = nullptr;
            if ((rc = dev_alloc_copy(&rp, rowptr, nrows + 1, false, s))) return bail(rc);
            M->own_rowptr = rp;
            M->A.rowptr = rp;
            if ((rc = dev_alloc_copy(&ci, col, nnz, false, s))) return bail(rc);
            M->own_col = ci;
            M->A.col = ci;
        }
        // reject malformed CSR arrays before any kernel indexes with them
        {
            const size_t words = (size_t)(nnz / 32 + 1);
            char* scratch = nullptr;
            if (pool_malloc((void**)&scratch, 256 + words * sizeof(unsigned), s) != cudaSuccess) {
                cudaGetLastError();
                return bail(fail(MLT_ENOMEM, "device allocation for CSR validation failed"));
            }
            int* bad = reinterpret_cast<int*>(scratch);
            unsigned* starts = reinterpret_cast<unsigned*>(scratch + 256);
            int hbad = 0;
            cudaError_t e = cudaMemsetAsync(scratch, 0, 256 + words * sizeof(unsigned), s);
            const int nbr = (int)std::max<int64_t>(1, std::min<int64_t>((nrows + 255) / 256, 16LL * num_sms));
            const int nbc = (int)std::max<int64_t>(1, std::min<int64_t>((nnz + 255) / 256, 16LL * num_sms));
            if (e == cudaSuccess) {
                ProfScope ps("validate_csr", s);
                validate_rows_kernel<<<nbr, 256, 0, s>>>(M->A.rowptr, nrows, nnz, starts, bad);
                e = cudaGetLastError();
            }
            if (e == cudaSuccess) {
                e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            }
            if (e == cudaSuccess && hbad == 0 && nnz > 0) {
                {
                    ProfScope ps("validate_csr", s);
                    validate_cols_kernel<<<nbc, 256, 0, s>>>(M->A.col, nnz, ncols, starts, bad);
                }
                e = cudaGetLastError();
                if (e == cudaSuccess) e = cudaMemcpyAsync(&hbad, bad, sizeof(int), cudaMemcpyDeviceToHost, s);
                if (e == cudaSuccess) e = cudaStreamSynchronize(s);
            }
            cudaFreeAsync(scratch, s);
            if (e != cudaSuccess) return bail(cuda_fail(e, "CSR validation"));
            if (hbad & 1) return bail(fail(MLT_EINVAL, "mlt_create_csr: rowptr must be non-decreasing within [0, nnz]"));
            if (hbad & 2) return bail(fail(MLT_EINVAL, "mlt_create_csr: column index out of range"));
            if (hbad & 4) return bail(fail(MLT_EINVAL, "mlt_create_csr: columns must increase strictly within each row"));
        }
        // values: always keep an FP64 copy; an FP32 copy is made when needed
        if (val_type == MLT_F64) {
            if (dev) {
                M->A.val64 = (const double*)vals;
            } else {
                double* v = nullptr;
                if ((rc = dev_alloc_copy(&v, vals, nnz, false, s))) return bail(rc);
                M->own_val = v;
                M->A.val64 = v;
            }
        } else if (val_type == MLT_F32) {
            float* v32 = nullptr;
            if (dev) {
                M->A.val32 = (const float*)vals;
            } else {
                if ((rc = dev_alloc_copy(&v32, vals, nnz, false, s))) return bail(rc);
                M->own_val32 = v32;
                M->A.val32 = v32;
            }
            double* v = nullptr;
            if ((rc = dev_alloc_copy(&v, nullptr, nnz, false, s))) return bail(rc);
            M->own_val = v;
            M->A.val64 = v;
            if (nnz > 0) {
                const int nb = (int)std::min<int64_t>((nnz + 255) / 256, 4096);
                ProfScope ps("f32_to_f64", s);
                f32_to_f64_kernel<<<nb, 256, 0, s>>>(M->A.val32, v, nnz);
                if ((rc = cuda_fail(cudaGetLastError(), "f32_to_f64_kernel"))) return bail(rc);
            }
        }
        if (gram) {
            // X^T as its own CSR, built on the host from the (host) arrays
            std::vector<int64_t> hrp;
            std::vector<int32_t> hci;
            std::vector<double> hv;
            const int64_t* rp = rowptr;
            const int32_t* ci = col;
            const double* vv = nullptr;
            if (dev || val_type != MLT_F64) {
                hrp.resize(nrows + 1);
                hci.resize(std::max<int64_t>(nnz, 1));
                if ((rc = cuda_fail(cudaMemcpyAsync(hrp.data(), M->A.rowptr, (nrows + 1) * sizeof(int64_t),
                                                    cudaMemcpyDeviceToHost, s), "copy rowptr"))) return bail(rc);
                if (nnz && (rc = cuda_fail(cudaMemcpyAsync(hci.data(), M->A.col, nnz * sizeof(int32_t),
                                                           cudaMemcpyDeviceToHost, s), "copy col"))) return bail(rc);
                if (M->A.val64) {
                    hv.resize(std::max<int64_t>(nnz, 1));
                    if (nnz && (rc = cuda_fail(cudaMemcpyAsync(hv.data(), M->A.val64, nnz * sizeof(double),
                                                               cudaMemcpyDeviceToHost, s), "copy vals"))) return bail(rc);
                    vv = hv.data();
                }
                if ((rc = cuda_fail(cudaStreamSynchronize(s), "sync"))) return bail(rc);
                rp = hrp.data();
                ci = hci.data();
            } else {
                vv = (const double*)vals;
            }
            std::vector<int64_t> trp;
            std::vector<int32_t> tci;
            std::vector<double> tv;
            host_transpose(nrows, ncols, rp, ci, vv, trp, tci, tv);
            int64_t* drp = nullptr;
            int32_t* dci = nullptr;
            if ((rc = dev_alloc_copy(&drp, trp.data(), ncols + 1, false, s))) return bail(rc);
            M->own_t_rowptr = drp;
            if ((rc = dev_alloc_copy(&dci, tci.data(), nnz, false, s))) return bail(rc);
            M->own_t_col = dci;
            M->AT.nrows = ncols;
            M->AT.ncols = nrows;
            M->AT.nnz = nnz;
            M->AT.rowptr = drp;
            M->AT.col = dci;
            if (vv) {
                double* dv = nullptr;
                if ((rc = dev_alloc_copy(&dv, tv.data(), nnz, false, s))) return bail(rc);
                M->own_t_val = dv;
                M->AT.val64 = dv;
            }
            if ((rc = cuda_fail(cudaStreamSynchronize(s), "sync"))) return bail(rc);
        }
        if ((flags & MLT_REORDER) && (rc = build_reorder(M, s))) return bail(rc);
        if ((rc = cuda_fail(cudaStreamSynchronize(s), "mlt_create_csr sync"))) return bail(rc);
        *out = M;
        return MLT_OK;
    } catch (...) {
        return fail(MLT_ENOMEM, "mlt_create_csr: exception");
    }
}

int mlt_destroy(mlt_matrix* m)
{
    if (!m) return MLT_OK;
    if (int rcb = handle_busy(m, "mlt_destroy")) return rcb;
    int cur = 0;
    cudaGetDevice(&cur);
    const int dev = m->device;
    if (cur != dev) cudaSetDevice(dev);
    cudaDeviceSynchronize();
    free_matrix(m);
    delete m;
    if (cur != dev) cudaSetDevice(cur);
    return MLT_OK;
}

int mlt_release_cached(void)
{
    return cuda_fail(mlt::trim_pools(), "mlt_release_cached");
}

int mlt_matrix_info(const mlt_matrix* m, int64_t* dim, int64_t* nnz)
{
    if (!m) return fail(MLT_EINVAL, "mlt_matrix_info: null handle");
    if (dim) *dim = m->dim();
    if (nnz) *nnz = m->A.nnz;
    return MLT_OK;
}

int mlt_spectrum_bounds(mlt_matrix* m, int method, int steps, uint64_t seed, double* a, double* b)
{
    (void)steps;
    (void)seed;
    if (!m || !a || !b) return fail(MLT_EINVAL, "mlt_spectrum_bounds: null argument");
    if (int rcb = handle_busy(m, "mlt_spectrum_bounds")) return rcb;
    if (method != MLT_BOUNDS_GERSHGORIN && method != MLT_BOUNDS_LANCZOS)
        return fail(MLT_EINVAL, "mlt_spectrum_bounds: unknown method");
    try {
        if (method == MLT_BOUNDS_LANCZOS) {
            if (steps < 2) return fail(MLT_EINVAL, "mlt_spectrum_bounds: Lanczos needs steps >= 2");
            return lanczos_bounds(m, steps, seed, a, b, (cudaStream_t)0);
        }
        return gershgorin_device(m, a, b, (cudaStream_t)0);
    } catch (...) {
        return fail(MLT_ENOMEM, "mlt_spectrum_bounds: exception");
    }
}

int mlt_cheb_coeffs(int fn, double p, double a, double b, int n, double* c)
{
    try {
        return cheb_coeffs_host(fn, p, a, b, n, c);
    } catch (...) {
        return fail(MLT_ENOMEM, "mlt_cheb_coeffs: exception");
    }
}

int mlt_moments(mlt_matrix* m, double a, double b, uint64_t seed, int64_t probe_offset,
                int64_t nprobes, const int32_t* degree, int precision, unsigned flags, double* mu,
                int64_t ld_mu, void* stream)
{
    try {
        if (nprobes == 0 && m) return MLT_OK;
        cudaStream_t s = (cudaStream_t)stream;
        MomentJob J;
        int rc = prepare_moment_job(m, a, b, seed, probe_offset, nprobes, degree, precision, flags, mu, ld_mu,
                                    0, J, s);
        if (rc) return rc;
        if ((rc = enqueue_moment_job(J, s))) return rc;
        return finish_moment_job(J, s);
    } catch (const std::bad_alloc&) {
        return fail(MLT_ENOMEM, "mlt_moments: host allocation failed");
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_moments: exception");
    }
}

int mlt_moments_batched(const mlt_moments_job* jobs, int njobs, int precision, unsigned flags, void* stream)
{
    try {
        if (njobs < 0 || (njobs > 0 && !jobs)) return fail(MLT_EINVAL, "mlt_moments_batched: bad job list");
        if (njobs == 0) return MLT_OK;
        for (int i = 0; i < njobs; ++i)
            for (int k = 0; k < i; ++k)
                if (jobs[i].matrix == jobs[k].matrix)
                    return fail(MLT_EINVAL, "mlt_moments_batched: each job needs its own matrix handle");
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<MomentJob> J(njobs);
        int rc;
        for (int i = 0; i < njobs; ++i) {
            const mlt_moments_job& q = jobs[i];
            if ((rc = prepare_moment_job(q.matrix, q.a, q.b, q.seed, q.probe_offset, q.nprobes, q.degree, precision,
                                         flags, q.mu, q.ld_mu, q.group_width, J[i], s)))
                return rc;
        }
        MLT_CUDA_TRY(cudaStreamSynchronize(s));
        // one graph: a branch per job on its own stream, forked from and joined to cs
        cudaStream_t cs = nullptr;
        MLT_CUDA_TRY(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
        std::vector<cudaStream_t> br(std::min(njobs, 64), nullptr);
        std::vector<cudaEvent_t> ev(njobs + 1, nullptr);
        auto cleanup = [&]() {
            for (auto& x : br) if (x) cudaStreamDestroy(x);
            for (auto& e : ev) if (e) cudaEventDestroy(e);
            if (cs) cudaStreamDestroy(cs);
        };
        for (auto& x : br)
            if (cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking) != cudaSuccess) { cleanup(); return cuda_fail(cudaGetLastError(), "stream"); }
        for (auto& e : ev)
            if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess) { cleanup(); return cuda_fail(cudaGetLastError(), "event"); }
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        ProfPause pause;
        cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) e = cudaEventRecord(ev[njobs], cs);
        for (int i = 0; i < njobs && e == cudaSuccess; ++i) {
            cudaStream_t si = br[i % br.size()];
            e = cudaStreamWaitEvent(si, ev[njobs], 0);
            if (e == cudaSuccess && (rc = enqueue_moment_job(J[i], si))) e = cudaErrorUnknown;
            if (e == cudaSuccess) e = cudaEventRecord(ev[i], si);
            if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[i], 0);
        }
        cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
        if (e == cudaSuccess) e = e2;
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (e == cudaSuccess) {
            ProfScope ps("moments_graph", s);
            e = cudaGraphLaunch(exec, s);
        }
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        cleanup();
        if (e != cudaSuccess) return rc ? rc : cuda_fail(e, "mlt_moments_batched graph");
        for (int i = 0; i < njobs; ++i)
            if ((rc = finish_moment_job(J[i], s))) return rc;
        return MLT_OK;
    } catch (const std::bad_alloc&) {
        return fail(MLT_ENOMEM, "mlt_moments_batched: host allocation failed");
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_moments_batched: exception");
    }
}

}  // extern "C"

// A persistent batch: every job prepared once, one CUDA graph captured and
// instantiated once, replayed by mlt_batch_run with new probe ids written
// into the id tables the graph reads.
struct mlt_batch {
    std::vector<mlt::MomentJob> jobs;
    std::vector<std::vector<int64_t>> ids;     // per job: probe ids in group order, before the shift
    std::vector<int64_t*> ids_dev;             // per job: the device id table its kernels read
    std::vector<int64_t> first, count;         // per job: first probe id and probe count
    cudaGraphExec_t exec = nullptr;
    int device = 0;
};

extern "C" {

int mlt_batch_destroy(mlt_batch* b)
{
    if (!b) return MLT_OK;
    cudaDeviceSynchronize();
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (auto& J : b->jobs)
        if (J.m) --J.m->batch_refs;
    delete b;
    return MLT_OK;
}

int mlt_batch_create(const mlt_moments_job* jobs, int njobs, int precision, unsigned flags, void* stream,
                     mlt_batch** out)
{
    try {
        if (!out) return fail(MLT_EINVAL, "mlt_batch_create: null output");
        *out = nullptr;
        if (njobs < 1 || !jobs) return fail(MLT_EINVAL, "mlt_batch_create: need at least one job");
        for (int i = 0; i < njobs; ++i) {
            if (!jobs[i].matrix) return fail(MLT_EINVAL, "mlt_batch_create: null matrix");
            if (jobs[i].nprobes < 1) return fail(MLT_EINVAL, "mlt_batch_create: every job needs a probe");
            for (int k = 0; k < i; ++k)
                if (jobs[i].matrix == jobs[k].matrix)
                    return fail(MLT_EINVAL, "mlt_batch_create: each job needs its own matrix handle");
        }
        cudaStream_t s = (cudaStream_t)stream;
        mlt_batch* B = new mlt_batch();
        B->jobs.resize(njobs);
        int rc;
        for (int i = 0; i < njobs; ++i) {
            const mlt_moments_job& q = jobs[i];
            if ((rc = prepare_moment_job(q.matrix, q.a, q.b, q.seed, q.probe_offset, q.nprobes, q.degree, precision,
                                         flags, q.mu, q.ld_mu, q.group_width, B->jobs[i], s))) {
                delete B;
                return rc;
            }
        }
        // the handles are locked from here on: the graph points into their workspaces
        for (auto& J : B->jobs) ++J.m->batch_refs;
        for (int i = 0; i < njobs; ++i) {
            const MomentJob& J = B->jobs[i];
            const int64_t n = J.nprobes;
            B->first.push_back(jobs[i].probe_offset);
            B->count.push_back(n);
            B->ids_dev.push_back(const_cast<int64_t*>(J.groups.front().ids_dev));
            std::vector<int64_t> h(n);
            MLT_CUDA_TRY(cudaMemcpyAsync(h.data(), J.groups.front().ids_dev, n * sizeof(int64_t),
                                         cudaMemcpyDeviceToHost, s));
            MLT_CUDA_TRY(cudaStreamSynchronize(s));
            B->ids.push_back(std::move(h));
        }
        MLT_CUDA_TRY(cudaGetDevice(&B->device));
        cudaStream_t cs = nullptr;
        std::vector<cudaStream_t> br(std::min(njobs, 64), nullptr);
        std::vector<cudaEvent_t> ev(njobs + 1, nullptr);
        auto cleanup = [&]() {
            for (auto& x : br) if (x) cudaStreamDestroy(x);
            for (auto& e : ev) if (e) cudaEventDestroy(e);
            if (cs) cudaStreamDestroy(cs);
        };
        cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
        for (auto& x : br)
            if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&x, cudaStreamNonBlocking);
        for (auto& ev1 : ev)
            if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev1, cudaEventDisableTiming);
        cudaGraph_t graph = nullptr;
        rc = MLT_OK;
        {
            ProfPause pause;
            if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
            const bool capturing = e == cudaSuccess;
            if (e == cudaSuccess) e = cudaEventRecord(ev[njobs], cs);
            for (int i = 0; i < njobs && e == cudaSuccess; ++i) {
                cudaStream_t si = br[i % br.size()];
                e = cudaStreamWaitEvent(si, ev[njobs], 0);
                if (e == cudaSuccess && (rc = enqueue_moment_job(B->jobs[i], si))) e = cudaErrorUnknown;
                if (e == cudaSuccess) e = cudaEventRecord(ev[i], si);
                if (e == cudaSuccess) e = cudaStreamWaitEvent(cs, ev[i], 0);
            }
            if (capturing) {
                cudaError_t e2 = cudaStreamEndCapture(cs, &graph);
                if (e == cudaSuccess) e = e2;
            }
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&B->exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        cleanup();
        if (e != cudaSuccess) {
            mlt_batch_destroy(B);
            return rc ? rc : cuda_fail(e, "mlt_batch_create graph");
        }
        *out = B;
        return MLT_OK;
    } catch (const std::bad_alloc&) {
        return fail(MLT_ENOMEM, "mlt_batch_create: host allocation failed");
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_batch_create: exception");
    }
}

int mlt_batch_run(mlt_batch* B, int64_t id_shift, void* stream)
{
    try {
        if (!B || !B->exec) return fail(MLT_EINVAL, "mlt_batch_run: null batch");
        const size_t njobs = B->jobs.size();
        for (size_t i = 0; i < njobs; ++i) {
            const int64_t lo = B->first[i] + id_shift;
            if (lo < 0 || lo + B->count[i] > (1LL << 32))
                return fail(MLT_EINVAL, "mlt_batch_run: shifted probe ids must lie in [0, 2^32)");
        }
        cudaStream_t s = (cudaStream_t)stream;
        std::vector<int64_t> h;
        for (size_t i = 0; i < njobs; ++i) {
            MomentJob& J = B->jobs[i];
            h.resize(B->ids[i].size());
            for (size_t p = 0; p < h.size(); ++p) h[p] = B->ids[i][p] + id_shift;
            // pageable source: the copy has left h when the call returns
            MLT_CUDA_TRY(cudaMemcpyAsync(B->ids_dev[i], h.data(), h.size() * sizeof(int64_t), cudaMemcpyHostToDevice, s));
            MLT_CUDA_TRY(cudaMemsetAsync(J.err, 0, sizeof(int), s));
        }
        {
            ProfScope ps("moments_graph", s);
            MLT_CUDA_TRY(cudaGraphLaunch(B->exec, s));
        }
        int rc;
        for (size_t i = 0; i < njobs; ++i)
            if ((rc = finish_moment_job(B->jobs[i], s))) return rc;
        return MLT_OK;
    } catch (const std::bad_alloc&) {
        return fail(MLT_ENOMEM, "mlt_batch_run: host allocation failed");
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_batch_run: exception");
    }
}

int mlt_autotune(mlt_matrix* m, int precision, int trial_steps, int* best, void* stream)
{
    try {
        if (!m) return fail(MLT_EINVAL, "mlt_autotune: null handle");
        if (int rcb = handle_busy(m, "mlt_autotune")) return rcb;
        if (trial_steps < 1 || trial_steps > MLT_MAX_DEGREE / 2) return fail(MLT_EINVAL, "mlt_autotune: bad trial length");
        cudaStream_t s = (cudaStream_t)stream;
        double a = 0.0, b = 0.0;
        int rc = gershgorin_device(m, &a, &b, s);
        if (rc) return rc;
        if (!(a < b)) b = a + 1.0;
        const int widths[] = {8, 16, 32, 64, 128};
        cudaEvent_t e0 = nullptr, e1 = nullptr;
        MLT_CUDA_TRY(cudaEventCreate(&e0));
        MLT_CUDA_TRY(cudaEventCreate(&e1));
        int bestw = 0;
        double bestt = 0.0;
        const int deg = 2 * trial_steps;
        const int saved = m->group_width;
        for (int w : widths) {
            const int np = 2 * w;
            std::vector<int32_t> dg(np, deg);
            // output to a device scratch buffer; nothing is copied back
            if ((rc = m->ws_out.ensure((size_t)np * (deg + 1) * sizeof(double), s))) break;
            MomentJob J;
            rc = prepare_moment_job(m, a, b, 0, 0, np, dg.data(), precision, 0, m->ws_out.as<double>(), deg + 1,
                                    w, J, s);
            if (rc) break;
            if ((rc = enqueue_moment_job(J, s))) break;            // warm-up
            MLT_CUDA_TRY(cudaEventRecord(e0, s));
            if ((rc = enqueue_moment_job(J, s))) break;
            MLT_CUDA_TRY(cudaEventRecord(e1, s));
            MLT_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.0f;
            MLT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
            const double per = ms / ((double)np * trial_steps);
            if (bestw == 0 || per < bestt) {
                bestw = w;
                bestt = per;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        if (rc && bestw == 0) {
            m->group_width = saved;
            return rc;
        }
        m->group_width = bestw;
        if (best) *best = bestw;
        return MLT_OK;
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_autotune: exception");
    }
}

void mlt_mlmc_default_params(mlt_mlmc_params* p)
{
    if (!p) return;
    std::memset(p, 0, sizeof(*p));
    p->fn = MLT_FN_LOG;
    p->n = 64;
    p->m_pilot = 10;
    p->mode = MLT_MODE_BUDGET;
    p->target = 1000.0;
    p->cost_model = MLT_COST_SYMMETRIC;
    p->reuse_pilot = 1;
    p->precision = MLT_PREC_FP64;
}

int mlt_mlmc_estimate(mlt_matrix* m, const mlt_mlmc_params* P, mlt_mlmc_result* R)
{
    try {
        if (!m || !P || !R) return fail(MLT_EINVAL, "mlt_mlmc_estimate: null argument");
        const int n = P->n;
        if (n < 1 || n > MLT_MAX_DEGREE) return fail(MLT_EINVAL, "mlt_mlmc_estimate: n out of range");
        if (P->cost_model != MLT_COST_SYMMETRIC && P->cost_model != MLT_COST_LINEAR)
            return fail(MLT_EINVAL, "mlt_mlmc_estimate: unknown cost model");
        std::vector<double> c(n + 1);
        int rc = cheb_coeffs_host(P->fn, P->fn_p, P->a, P->b, n, c.data());
        if (rc) return rc;
        const int64_t d = m->dim();
        std::vector<int> levels;
        std::vector<int64_t> counts, fresh;
        std::vector<double> pilot;     // m_pilot x (n+1) moments, reused by the top level
        int m_pilot = 0;
        int64_t next_id = 0;
        int64_t matvecs = 0;
        const int dir = (P->flags & MLT_DIRECT) ? 1 : 0;
        auto steps_of = [&](int l) -> int64_t { return dir ? l : (l + 1) / 2; };
        if (P->flags & ~(MLT_DIRECT | MLT_LOW_CV)) return fail(MLT_EINVAL, "mlt_mlmc_estimate: unknown flags");
        const unsigned mflags = P->flags & ~MLT_LOW_CV;     // the moment call's own flags
        // with MLT_LOW_CV, w_j = mu_j - tr T_j(At) (1 <= j < nlow) are the control variates
        double tlow[3] = {0.0, 0.0, 0.0};
        int nlow = 0;
        if (P->flags & MLT_LOW_CV) {
            if (!(P->a < P->b)) return fail(MLT_EINVAL, "mlt_mlmc_estimate: need a < b");
            rc = low_traces(m, P->a, P->b, tlow, &nlow, (cudaStream_t)P->stream);
            if (rc) return rc;
        }
        if (P->nlevels > 0) {
            if (P->nlevels > MLT_MAX_LEVELS) return fail(MLT_EINVAL, "mlt_mlmc_estimate: too many levels");
            for (int k = 0; k < P->nlevels; ++k) {
                const int l = P->levels[k];
                if (l < 0 || l > n || (k > 0 && l <= P->levels[k - 1]))
                    return fail(MLT_EINVAL, "mlt_mlmc_estimate: levels must rise strictly within [0, n]");
                if (P->m[k] < 1) return fail(MLT_EINVAL, "mlt_mlmc_estimate: every level needs m >= 1");
                levels.push_back(l);
                counts.push_back(P->m[k]);
            }
            if (levels.back() != n) return fail(MLT_EINVAL, "mlt_mlmc_estimate: the last level must be n");
            fresh = counts;
        } else {
            m_pilot = P->m_pilot;
            if (m_pilot < 2) return fail(MLT_EINVAL, "mlt_mlmc_estimate: automatic mode needs m_pilot >= 2");
            if (!(P->target > 0.0) || !std::isfinite(P->target))
                return fail(MLT_EINVAL, "mlt_mlmc_estimate: target must be positive");
            if (P->mode != MLT_MODE_BUDGET && P->mode != MLT_MODE_VARIANCE)
                return fail(MLT_EINVAL, "mlt_mlmc_estimate: unknown mode");
            pilot.assign((size_t)m_pilot * (n + 1), 0.0);
            std::vector<int32_t> pdeg(m_pilot, n);
            rc = mlt_moments(m, P->a, P->b, P->seed, 0, m_pilot, pdeg.data(), P->precision, mflags,
                             pilot.data(), n + 1, P->stream);
            if (rc) return rc;
            matvecs += (int64_t)m_pilot * steps_of(n);
            next_id = m_pilot;
            std::vector<double> V((size_t)(n + 1) * (n + 1));
            band_variances(c.data(), n, pilot.data(), n + 1, m_pilot, V.data());
            std::vector<int> lv(n + 1);
            int L = 0;
            const int mp = P->reuse_pilot ? m_pilot : 0;
            rc = select_levels(V.data(), n, P->cost_model, mp, P->mode, P->target, P->max_levels, lv.data(), &L);
            if (rc) return rc;
            levels.assign(lv.begin(), lv.begin() + L);
            counts.resize(L);
            allocate_samples(levels.data(), L, V.data(), n, P->cost_model, P->mode, P->target, mp, counts.data());
            fresh = counts;
            if (P->reuse_pilot) fresh[L - 1] = counts[L - 1] - m_pilot;
        }
        const int L = (int)levels.size();
        // one ragged moment call for all levels' fresh probes
        int64_t total = 0;
        for (int k = 0; k < L; ++k) total += fresh[k];
        std::vector<int32_t> deg(total);
        {
            int64_t q = 0;
            for (int k = 0; k < L; ++k)
                for (int64_t i = 0; i < fresh[k]; ++i) deg[q++] = levels[k];
        }
        std::vector<double> mu((size_t)std::max<int64_t>(total, 1) * (n + 1));
        if (total > 0) {
            rc = mlt_moments(m, P->a, P->b, P->seed, next_id, total, deg.data(), P->precision, mflags,
                             mu.data(), n + 1, P->stream);
            if (rc) return rc;
        }
        for (int k = 0; k < L; ++k) matvecs += fresh[k] * steps_of(levels[k]);
        // combination (Eq. multiEstimator)
        std::memset(R, 0, sizeof(*R));
        double est = 0.0, var_sum = 0.0;
        int64_t q = 0;
        int lo = -1;
        for (int k = 0; k < L; ++k) {
            const int hi = levels[k];
            std::vector<double> samples, w1, w2;
            samples.reserve(counts[k]);
            const int J = std::min(nlow - 1, hi);        // control variates this level has (0: none)
            auto band = [&](const double* row) {
                double s = 0.0;
                band_samples(c.data(), lo, hi, row, n + 1, 1, &s);
                samples.push_back(s);
                if (J >= 1) w1.push_back(row[1] - tlow[1]);
                if (J >= 2) w2.push_back(row[2] - tlow[2]);
            };
            if (k == L - 1 && m_pilot > 0 && P->reuse_pilot)
                for (int p = 0; p < m_pilot; ++p) band(&pilot[(size_t)p * (n + 1)]);
            for (int64_t i = 0; i < fresh[k]; ++i, ++q) band(&mu[(size_t)q * (n + 1)]);
            const int64_t mk = (int64_t)samples.size();
            double mean = 0.0, var = 0.0;
            level_stats(samples.data(), mk, &mean, &var);
            // the low-degree control variates (Section 5.4): least squares of the
            // band on (1, w); the level's estimate is the intercept, its variance
            // the residual one (divisor m - 1 - J); skipped when m <= J + 1 or the
            // centred covariates are degenerate
            if (J >= 1 && mk > J + 1) {
                double m1 = 0.0, m2 = 0.0;
                for (int64_t i = 0; i < mk; ++i) {
                    m1 += w1[i];
                    if (J >= 2) m2 += w2[i];
                }
                m1 /= (double)mk;
                m2 /= (double)mk;
                double g11 = 0.0, g12 = 0.0, g22 = 0.0, r1 = 0.0, r2 = 0.0;
                for (int64_t i = 0; i < mk; ++i) {
                    const double e = samples[i] - mean, u = w1[i] - m1, v = J >= 2 ? w2[i] - m2 : 0.0;
                    g11 += u * u;
                    g12 += u * v;
                    g22 += v * v;
                    r1 += u * e;
                    r2 += v * e;
                }
                double a1 = 0.0, a2 = 0.0;
                bool ok = false;
                if (J >= 2) {
                    const double det = g11 * g22 - g12 * g12;
                    if (det > 1e-12 * g11 * g22) {
                        a1 = (g22 * r1 - g12 * r2) / det;
                        a2 = (g11 * r2 - g12 * r1) / det;
                        ok = true;
                    }
                } else if (g11 > 0.0) {
                    a1 = r1 / g11;
                    ok = true;
                }
                if (ok) {
                    double rs = 0.0;
                    for (int64_t i = 0; i < mk; ++i) {
                        const double e = (samples[i] - mean) - a1 * (w1[i] - m1) - (J >= 2 ? a2 * (w2[i] - m2) : 0.0);
                        rs += e * e;
                    }
                    mean = mean - a1 * m1 - a2 * m2;
                    var = rs / (double)(mk - 1 - J);
                }
            }
            R->levels[k] = hi;
            R->m[k] = mk;
            R->level_mean[k] = mean;
            R->level_var[k] = var;
            est += mean;
            var_sum += var / (double)mk;
            lo = hi;
        }
        R->nlevels = L;
        R->estimate = est;
        R->std_error = std::sqrt(var_sum);
        R->probes = next_id + total;
        R->matvecs = matvecs;
        (void)d;
        return MLT_OK;
    } catch (const std::bad_alloc&) {
        return fail(MLT_ENOMEM, "mlt_mlmc_estimate: host allocation failed");
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_mlmc_estimate: exception");
    }
}

int mlt_low_traces(mlt_matrix* m, double a, double b, double* t, int* count, void* stream)
{
    try {
        if (!m || !t) return fail(MLT_EINVAL, "mlt_low_traces: null argument");
        if (int rcb = handle_busy(m, "mlt_low_traces")) return rcb;
        if (!(a < b) || !std::isfinite(a) || !std::isfinite(b)) return fail(MLT_EINVAL, "mlt_low_traces: need finite a < b");
        return low_traces(m, a, b, t, count, (cudaStream_t)stream);
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_low_traces: exception");
    }
}

int mlt_fp64_rate(int64_t iters, double* tflops, void* stream)
{
    try {
        if (!tflops || iters < 1 || iters > (1LL << 30)) return fail(MLT_EINVAL, "mlt_fp64_rate: need tflops and 1 <= iters <= 2^30");
        int dev = 0, sms = 0;
        MLT_CUDA_TRY(cudaGetDevice(&dev));
        MLT_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        cudaStream_t s = (cudaStream_t)stream;
        double* sink = nullptr;
        const int blocks = 8 * sms;
        if (pool_malloc((void**)&sink, (size_t)blocks * 256 * sizeof(double), s) != cudaSuccess) {
            cudaGetLastError();
            return fail(MLT_ENOMEM, "mlt_fp64_rate: device allocation failed");
        }
        cudaEvent_t e0, e1;
        MLT_CUDA_TRY(cudaEventCreate(&e0));
        MLT_CUDA_TRY(cudaEventCreate(&e1));
        fp64_fma_kernel<<<blocks, 256, 0, s>>>(sink, 16);     // warm-up
        MLT_CUDA_TRY(cudaEventRecord(e0, s));
        fp64_fma_kernel<<<blocks, 256, 0, s>>>(sink, iters);
        MLT_CUDA_TRY(cudaEventRecord(e1, s));
        MLT_CUDA_TRY(cudaGetLastError());
        MLT_CUDA_TRY(cudaEventSynchronize(e1));
        float ms = 0.0f;
        MLT_CUDA_TRY(cudaEventElapsedTime(&ms, e0, e1));
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFreeAsync(sink, s);
        MLT_CUDA_TRY(cudaStreamSynchronize(s));
        // 8 chains, one FMA (2 flops) each per iteration
        *tflops = 2.0 * 8.0 * (double)iters * (double)blocks * 256.0 / ((double)ms * 1e-3) / 1e12;
        return MLT_OK;
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_fp64_rate: exception");
    }
}

int mlt_pilot_variances(const double* c, int n, const double* mu, int64_t ld_mu, int64_t m_pilot, double* V)
{
    try {
        if (!c || !V || (m_pilot > 0 && !mu)) return fail(MLT_EINVAL, "mlt_pilot_variances: null argument");
        if (n < 1 || n > MLT_MAX_DEGREE) return fail(MLT_EINVAL, "mlt_pilot_variances: n out of range");
        if (m_pilot < 0 || m_pilot > INT32_MAX) return fail(MLT_EINVAL, "mlt_pilot_variances: bad pilot count");
        if (m_pilot > 0 && ld_mu < n + 1) return fail(MLT_EINVAL, "mlt_pilot_variances: ld_mu below n + 1");
        band_variances(c, n, mu, ld_mu, (int)m_pilot, V);
        return MLT_OK;
    } catch (...) {
        return fail(MLT_ENOMEM, "mlt_pilot_variances: host allocation failed");
    }
}

int mlt_select_levels(const double* V, int n, int cost_model, int m_pilot, int mode, double target,
                      int max_levels, int32_t* levels, int64_t* m, int* nlevels)
{
    try {
        if (!V || !levels || !m || !nlevels) return fail(MLT_EINVAL, "mlt_select_levels: null argument");
        if (n < 1 || n > MLT_MAX_DEGREE) return fail(MLT_EINVAL, "mlt_select_levels: n out of range");
        if (cost_model != MLT_COST_SYMMETRIC && cost_model != MLT_COST_LINEAR)
            return fail(MLT_EINVAL, "mlt_select_levels: unknown cost model");
        if (mode != MLT_MODE_BUDGET && mode != MLT_MODE_VARIANCE) return fail(MLT_EINVAL, "mlt_select_levels: unknown mode");
        if (!(target > 0.0) || !std::isfinite(target)) return fail(MLT_EINVAL, "mlt_select_levels: target must be positive");
        if (m_pilot < 0 || max_levels < 0) return fail(MLT_EINVAL, "mlt_select_levels: negative m_pilot or max_levels");
        for (int64_t i = 0; i < (int64_t)(n + 1) * (n + 1); ++i)
            if (!(V[i] >= 0.0) || !std::isfinite(V[i])) return fail(MLT_EINVAL, "mlt_select_levels: V must be finite and >= 0");
        std::vector<int> lv(n + 1);
        int L = 0;
        int rc = select_levels(V, n, cost_model, m_pilot, mode, target, max_levels, lv.data(), &L);
        if (rc) return rc;
        allocate_samples(lv.data(), L, V, n, cost_model, mode, target, m_pilot, m);
        for (int k = 0; k < L; ++k) levels[k] = lv[k];
        *nlevels = L;
        return MLT_OK;
    } catch (const std::bad_alloc&) {
        return fail(MLT_ENOMEM, "mlt_select_levels: host allocation failed");
    } catch (...) {
        return fail(MLT_EINVAL, "mlt_select_levels: exception");
    }
}

int mlt_band_samples(const double* c, int lo, int hi, const double* mu, int64_t ld_mu, int64_t nprobes, double* q)
{
    if (nprobes < 0) return fail(MLT_EINVAL, "mlt_band_samples: negative probe count");
    if (nprobes == 0) return MLT_OK;
    if (!c || !mu || !q) return fail(MLT_EINVAL, "mlt_band_samples: null argument");
    if (lo < -1 || hi <= lo || hi > MLT_MAX_DEGREE) return fail(MLT_EINVAL, "mlt_band_samples: need -1 <= lo < hi <= MLT_MAX_DEGREE");
    if (ld_mu < hi + 1) return fail(MLT_EINVAL, "mlt_band_samples: ld_mu below hi + 1");
    band_samples(c, lo, hi, mu, ld_mu, nprobes, q);
    return MLT_OK;
}

int mlt_mlmc_combine(int nlevels, const int32_t* levels, const int64_t* m, const double* samples, mlt_mlmc_result* R)
{
    if (!levels || !m || !samples || !R) return fail(MLT_EINVAL, "mlt_mlmc_combine: null argument");
    if (nlevels < 1 || nlevels > MLT_MAX_LEVELS) return fail(MLT_EINVAL, "mlt_mlmc_combine: nlevels out of range");
    for (int k = 0; k < nlevels; ++k)
        if (m[k] < 1) return fail(MLT_EINVAL, "mlt_mlmc_combine: every level needs m >= 1");
    std::memset(R, 0, sizeof(*R));
    double est = 0.0, var_sum = 0.0;
    const double* v = samples;
    for (int k = 0; k < nlevels; ++k) {
        double mean = 0.0, var = 0.0;
        level_stats(v, m[k], &mean, &var);
        R->levels[k] = levels[k];
        R->m[k] = m[k];
        R->level_mean[k] = mean;
        R->level_var[k] = var;
        est += mean;
        var_sum += var / (double)m[k];
        v += m[k];
    }
    R->nlevels = nlevels;
    R->estimate = est;
    R->std_error = std::sqrt(var_sum);
    return MLT_OK;
}

int mlt_triangle_estimate(const int64_t* x, int64_t nprobes, int64_t nnz, int cv, double a, double b,
                          double* estimate, double* std_error, double* a1_out, double* a2_out)
{
    try {
        if (!x || nprobes < 1) return fail(MLT_EINVAL, "mlt_triangle_estimate: need x and nprobes >= 1");
        if (nnz < 0) return fail(MLT_EINVAL, "mlt_triangle_estimate: negative nnz");
        double mx = 0.0;
        for (int64_t i = 0; i < 3 * nprobes; ++i) mx = std::max(mx, std::fabs((double)x[i]));
        if ((double)nprobes * (double)nprobes * mx * mx >= 4.2e37)
            return fail(MLT_ERANGE, "mlt_triangle_estimate: moment sums would overflow 128-bit integers");
        double est = 0.0, se = 0.0, a1 = 0.0, a2 = 0.0;
        if (cv == MLT_TRI_CV_NONE || cv == MLT_TRI_CV_FIT) {
            triangle_estimate_host(x, nprobes, nnz, cv == MLT_TRI_CV_FIT, &est, &se, &a1, &a2);
        } else if (cv == MLT_TRI_CV_CHEB) {
            if (!(a < b) || !std::isfinite(a) || !std::isfinite(b))
                return fail(MLT_EINVAL, "mlt_triangle_estimate: need finite a < b");
            triangle_cv_cheb(a, b, &a1, &a2);
            triangle_estimate_fixed_host(x, nprobes, nnz, a1, a2, &est, &se);
        } else {
            return fail(MLT_EINVAL, "mlt_triangle_estimate: unknown control-variate mode");
        }
        if (estimate) *estimate = est;
        if (std_error) *std_error = se;
        if (a1_out) *a1_out = a1;
        if (a2_out) *a2_out = a2;
        return MLT_OK;
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_triangle_estimate: exception");
    }
}

int mlt_triangle_trace(mlt_matrix* m, uint64_t seed, int64_t probe_offset, int64_t nprobes, int block,
                       int use_cv, int64_t* x, double* estimate, double* std_error, void* stream)
{
    try {
        if (!m) return fail(MLT_EINVAL, "mlt_triangle_trace: null handle");
        if (int rcb = handle_busy(m, "mlt_triangle_trace")) return rcb;
        if (m->val_type != MLT_PATTERN || (m->flags & MLT_GRAM) || m->A.nrows != m->A.ncols)
            return fail(MLT_EINVAL, "mlt_triangle_trace: needs a square 0/1 pattern matrix");
        if (nprobes < 1) return fail(MLT_EINVAL, "mlt_triangle_trace: need at least one probe");
        if (block != 128 && block != 256) return fail(MLT_EINVAL, "mlt_triangle_trace: block must be 128 or 256");
        if (probe_offset < 0 || probe_offset + nprobes > (1LL << 32))
            return fail(MLT_EINVAL, "mlt_triangle_trace: probe ids must lie in [0, 2^32)");
        cudaStream_t s = (cudaStream_t)stream;
        int rc = tri_prepare(m, s);
        if (rc) return rc;
        const bool out_dev = x && is_device_ptr(x);
        int64_t* x_dev = x;
        const size_t xbytes = (size_t)nprobes * 3 * sizeof(int64_t);
        if (!out_dev) {
            if ((rc = m->ws_out.ensure(xbytes, s))) return rc;
            x_dev = m->ws_out.as<int64_t>();
        }
        // Blocks of 128 probes run two per launch: a launch serves 256
        // consecutive probe ids, and every probe's (x1, x2, x3) is an exact
        // integer sum that does not depend on which probes share its launch.
        constexpr int kLaunchProbes = 256;
        for (int64_t b0 = 0; b0 < nprobes; b0 += kLaunchProbes) {
            const int nb = (int)std::min<int64_t>(kLaunchProbes, nprobes - b0);
            if ((rc = tri_block(m, seed, probe_offset + b0, nb, x_dev + 3 * b0, s))) return rc;
        }
        std::vector<int64_t> hx(nprobes * 3);
        MLT_CUDA_TRY(cudaMemcpyAsync(hx.data(), x_dev, xbytes, cudaMemcpyDeviceToHost, s));
        MLT_CUDA_TRY(cudaStreamSynchronize(s));
        if (x && !out_dev) std::memcpy(x, hx.data(), xbytes);
        double mx = 0.0;
        for (int64_t v : hx) mx = std::max(mx, std::fabs((double)v));
        if ((double)nprobes * (double)nprobes * mx * mx >= 4.2e37)
            return fail(MLT_ERANGE, "mlt_triangle_trace: moment sums would overflow 128-bit integers");
        double est = 0.0, se = 0.0;
        triangle_estimate_host(hx.data(), nprobes, m->A.nnz, use_cv, &est, &se);
        if (estimate) *estimate = est;
        if (std_error) *std_error = se;
        return MLT_OK;
    } catch (const std::bad_alloc&) {
        return fail(MLT_ENOMEM, "mlt_triangle_trace: host allocation failed");
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_triangle_trace: exception");
    }
}

}  // extern "C"
