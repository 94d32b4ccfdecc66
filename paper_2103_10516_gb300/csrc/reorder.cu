// The operator relabelled by decreasing degree, for the moment engine.
//
// On a power-law graph (the R-MAT adjacency of the Estrada workload) most
// gathered rows of V_k belong to a few hub vertices, and the generator spreads
// those hubs over the whole id range.  Relabelling rows and columns in order
// of decreasing degree (ties by increasing original id, so the order is fixed)
// puts the most-gathered rows of V_k into one contiguous prefix: fewer DRAM
// pages and L2 lines hold the rows that most gathers hit, and the work
// chunks, which follow row order, start with the hub rows.
//
// The relabelled operator is P A P^T for the permutation P.  The moment
// engine applies it to probes written in relabelled order, z'_j = z_{perm[j]}
// with perm[j] the original id of row j, so z'^T T_k(P At P^T) z' = z^T T_k(At) z:
// the moments are those of the original operator and its original probes, up
// to the order of the floating-point sums.  Only the moment engine uses the
// copy; everything else keeps the original arrays.
#include <cuda_runtime.h>

#include <cub/cub.cuh>

#include <algorithm>
#include <vector>

#include "mlt_internal.h"

namespace mlt {
namespace {

// key[i] = ~deg_i, so that an ascending sort puts larger degrees first; id[i] = i.
__global__ void degree_keys_kernel(const int64_t* __restrict__ rp, int64_t n, uint32_t* __restrict__ key,
                                   int32_t* __restrict__ id)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        key[i] = ~(uint32_t)(rp[i + 1] - rp[i]);
        id[i] = (int32_t)i;
    }
}

// pdeg[j] = degree of row perm[j]; inv[perm[j]] = j.
__global__ void permuted_degrees_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ perm, int64_t n,
                                        int64_t* __restrict__ pdeg, int32_t* __restrict__ inv)
{
    for (int64_t j = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; j < n; j += (int64_t)gridDim.x * blockDim.x) {
        const int64_t o = perm[j];
        pdeg[j] = rp[o + 1] - rp[o];
        inv[o] = (int32_t)j;
    }
}

// Row j of the relabelled matrix is row perm[j] of the original, with every
// column c renamed inv[c].  One warp per row (entries in their original order).
__global__ void relabel_rows_kernel(const int64_t* __restrict__ rp, const int32_t* __restrict__ col,
                                    const double* __restrict__ val, const int64_t* __restrict__ prp,
                                    const int32_t* __restrict__ perm, const int32_t* __restrict__ inv,
                                    int32_t* __restrict__ pcol, double* __restrict__ pval, int64_t n)
{
    const int lane = threadIdx.x & 31;
    const int64_t w0 = (blockIdx.x * (int64_t)blockDim.x + threadIdx.x) >> 5;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t j = w0; j < n; j += nw) {
        const int64_t o = perm[j];
        const int64_t src = rp[o], dst = prp[j], len = rp[o + 1] - src;
        for (int64_t k = lane; k < len; k += 32) {
            pcol[dst + k] = inv[col[src + k]];
            if (val) pval[dst + k] = val[src + k];
        }
    }
}

}  // namespace

// All on the device, in stream order: the stable radix sort of the keys ~deg
// gives perm (decreasing degree, equal degrees in increasing id), a prefix
// sum of the permuted degrees gives the relabelled row pointers, and one
// warp per row copies and renames the entries.
int build_reorder(mlt_matrix* M, cudaStream_t s)
{
    const DevCSR& A = M->A;
    const int64_t n = A.nrows, nnz = A.nnz;
    if (n >= (int64_t(1) << 31)) return fail(MLT_EINVAL, "relabelling needs fewer than 2^31 rows");
    const int nn = (int)n;
    std::vector<void*> scratch;
    auto alloc = [&](void** p, size_t bytes) -> int {
        if (pool_malloc(p, std::max<size_t>(bytes, 16), s) != cudaSuccess) {
            cudaGetLastError();
            return fail(MLT_ENOMEM, "device allocation (relabelled operator) failed");
        }
        return MLT_OK;
    };
    auto release = [&]() {
        for (void* p : scratch) cudaFreeAsync(p, s);
        scratch.clear();
    };
    int rc = MLT_OK;
    void *d_prp = nullptr, *d_pcol = nullptr, *d_pval = nullptr, *d_perm = nullptr;
    void *d_inv = nullptr, *d_key = nullptr, *d_key2 = nullptr, *d_id = nullptr, *d_pdeg = nullptr, *d_tmp = nullptr;
    if ((rc = alloc(&d_prp, (n + 1) * sizeof(int64_t)))) return rc;
    M->own_p_rowptr = d_prp;
    if ((rc = alloc(&d_pcol, nnz * sizeof(int32_t)))) return rc;
    M->own_p_col = d_pcol;
    if (A.val64) {
        if ((rc = alloc(&d_pval, nnz * sizeof(double)))) return rc;
        M->own_p_val = d_pval;
    }
    if ((rc = alloc(&d_perm, n * sizeof(int32_t)))) return rc;
    M->perm = static_cast<int32_t*>(d_perm);
    // scratch, freed (stream-ordered) before returning
    auto alloc_scratch = [&](void** p, size_t bytes) -> int {
        const int r = alloc(p, bytes);
        if (r == MLT_OK) scratch.push_back(*p);
        return r;
    };
    if ((rc = alloc_scratch(&d_inv, n * sizeof(int32_t))) || (rc = alloc_scratch(&d_key, n * sizeof(uint32_t))) ||
        (rc = alloc_scratch(&d_key2, n * sizeof(uint32_t))) || (rc = alloc_scratch(&d_id, n * sizeof(int32_t))) ||
        (rc = alloc_scratch(&d_pdeg, n * sizeof(int64_t)))) {
        release();
        return rc;
    }
    size_t sort_bytes = 0, scan_bytes = 0;
    cudaError_t e = cub::DeviceRadixSort::SortPairs(nullptr, sort_bytes, static_cast<uint32_t*>(d_key),
                                                    static_cast<uint32_t*>(d_key2), static_cast<int32_t*>(d_id),
                                                    static_cast<int32_t*>(d_perm), nn, 0, 32, s);
    if (e == cudaSuccess)
        e = cub::DeviceScan::InclusiveSum(nullptr, scan_bytes, static_cast<int64_t*>(d_pdeg),
                                          static_cast<int64_t*>(d_prp) + 1, nn, s);
    if (e != cudaSuccess) {
        release();
        return fail(MLT_ECUDA, "relabelling: cub sizing failed");
    }
    const size_t tmp_bytes = std::max(sort_bytes, scan_bytes);
    if ((rc = alloc_scratch(&d_tmp, tmp_bytes))) {
        release();
        return rc;
    }
    if (n > 0) {
        const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n + 255) / 256, 16LL * M->num_sms));
        ProfScope ps("relabel", s);
        degree_keys_kernel<<<nb, 256, 0, s>>>(A.rowptr, n, static_cast<uint32_t*>(d_key), static_cast<int32_t*>(d_id));
        size_t b = tmp_bytes;
        e = cub::DeviceRadixSort::SortPairs(d_tmp, b, static_cast<uint32_t*>(d_key), static_cast<uint32_t*>(d_key2),
                                            static_cast<int32_t*>(d_id), static_cast<int32_t*>(d_perm), nn, 0, 32, s);
        if (e == cudaSuccess) {
            permuted_degrees_kernel<<<nb, 256, 0, s>>>(A.rowptr, static_cast<int32_t*>(d_perm), n,
                                                       static_cast<int64_t*>(d_pdeg), static_cast<int32_t*>(d_inv));
            e = cudaMemsetAsync(d_prp, 0, sizeof(int64_t), s);
        }
        if (e == cudaSuccess) {
            b = tmp_bytes;
            e = cub::DeviceScan::InclusiveSum(d_tmp, b, static_cast<int64_t*>(d_pdeg), static_cast<int64_t*>(d_prp) + 1,
                                              nn, s);
        }
        if (e == cudaSuccess) {
            const int nbr = (int)std::max<int64_t>(1, std::min<int64_t>((n * 32 + 255) / 256, 16LL * M->num_sms));
            relabel_rows_kernel<<<nbr, 256, 0, s>>>(A.rowptr, A.col, A.val64, static_cast<int64_t*>(d_prp), M->perm,
                                                    static_cast<int32_t*>(d_inv), static_cast<int32_t*>(d_pcol),
                                                    static_cast<double*>(d_pval), n);
            e = cudaGetLastError();
        }
        if (e != cudaSuccess) {
            release();
            return fail(MLT_ECUDA, "relabelling kernels failed");
        }
    } else {
        MLT_CUDA_TRY(cudaMemsetAsync(d_prp, 0, sizeof(int64_t), s));
    }
    release();
    M->P.nrows = n;
    M->P.ncols = n;
    M->P.nnz = nnz;
    M->P.rowptr = static_cast<int64_t*>(d_prp);
    M->P.col = static_cast<int32_t*>(d_pcol);
    M->P.val64 = static_cast<double*>(d_pval);
    MLT_CUDA_TRY(cudaStreamSynchronize(s));
    return MLT_OK;
}

}  // namespace mlt
