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

#include <algorithm>
#include <vector>

#include "mlt_internal.h"

namespace mlt {
namespace {

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

int build_reorder(mlt_matrix* M, cudaStream_t s)
{
    const DevCSR& A = M->A;
    const int64_t n = A.nrows, nnz = A.nnz;
    std::vector<int64_t> rp(n + 1);
    MLT_CUDA_TRY(cudaMemcpyAsync(rp.data(), A.rowptr, (n + 1) * sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaStreamSynchronize(s));
    // counting sort by degree, descending; equal degrees keep increasing ids
    int64_t maxdeg = 0;
    for (int64_t i = 0; i < n; ++i) maxdeg = std::max(maxdeg, rp[i + 1] - rp[i]);
    std::vector<int64_t> start(maxdeg + 2, 0);
    for (int64_t i = 0; i < n; ++i) ++start[maxdeg - (rp[i + 1] - rp[i]) + 1];
    for (int64_t b = 0; b <= maxdeg; ++b) start[b + 1] += start[b];
    std::vector<int32_t> perm(std::max<int64_t>(n, 1)), inv(std::max<int64_t>(n, 1));
    for (int64_t i = 0; i < n; ++i) perm[start[maxdeg - (rp[i + 1] - rp[i])]++] = (int32_t)i;
    std::vector<int64_t> prp(n + 1);
    prp[0] = 0;
    for (int64_t j = 0; j < n; ++j) {
        inv[perm[j]] = (int32_t)j;
        prp[j + 1] = prp[j] + (rp[perm[j] + 1] - rp[perm[j]]);
    }
    auto alloc = [&](void** p, size_t bytes) -> int {
        if (pool_malloc(p, std::max<size_t>(bytes, 16), s) != cudaSuccess) {
            cudaGetLastError();
            return fail(MLT_ENOMEM, "device allocation (relabelled operator) failed");
        }
        return MLT_OK;
    };
    int rc;
    void *d_prp = nullptr, *d_pcol = nullptr, *d_pval = nullptr, *d_perm = nullptr, *d_inv = nullptr;
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
    if ((rc = alloc(&d_inv, n * sizeof(int32_t)))) return rc;
    MLT_CUDA_TRY(cudaMemcpyAsync(d_prp, prp.data(), (n + 1) * sizeof(int64_t), cudaMemcpyHostToDevice, s));
    MLT_CUDA_TRY(cudaMemcpyAsync(d_perm, perm.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    MLT_CUDA_TRY(cudaMemcpyAsync(d_inv, inv.data(), n * sizeof(int32_t), cudaMemcpyHostToDevice, s));
    if (n > 0) {
        const int nb = (int)std::max<int64_t>(1, std::min<int64_t>((n * 32 + 255) / 256, 16LL * M->num_sms));
        ProfScope ps("relabel_rows", s);
        relabel_rows_kernel<<<nb, 256, 0, s>>>(A.rowptr, A.col, A.val64, static_cast<int64_t*>(d_prp),
                                               M->perm, static_cast<int32_t*>(d_inv), static_cast<int32_t*>(d_pcol),
                                               static_cast<double*>(d_pval), n);
        MLT_CUDA_TRY(cudaGetLastError());
    }
    cudaFreeAsync(d_inv, s);
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
