// Internal declarations shared by the translation units of libmlt.
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <string>
#include <vector>

#include "mlt.h"

namespace mlt {

// Thread-local error message behind mlt_last_error().
void set_error(const std::string& msg);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t e, const char* what);

#define MLT_CUDA_TRY(expr)                                   \
    do {                                                     \
        cudaError_t e_ = (expr);                             \
        if (e_ != cudaSuccess) return ::mlt::cuda_fail(e_, #expr); \
    } while (0)

// Kernel timing: while mlt_profile_start() is in effect, every library kernel
// launch is bracketed by CUDA events recorded on its own stream.
struct ProfScope {
    int idx;
    cudaStream_t s;
    ProfScope(const char* name, cudaStream_t stream);
    ~ProfScope();
};

// No kernel timing on this thread while alive (used around graph capture).
struct ProfPause {
    ProfPause();
    ~ProfPause();
};

// Stream-ordered device allocation from the library's pool on the current
// device: freed blocks stay cached there for later handles instead of going
// back to the driver at each synchronisation (mlt_release_cached trims it).
cudaError_t pool_malloc(void** p, size_t bytes, cudaStream_t s);

// A grow-only device buffer owned by a matrix handle.
struct DevBuf {
    void* p = nullptr;
    size_t bytes = 0;
    int ensure(size_t want, cudaStream_t s);
    void release();
    template <typename T> T* as() const { return static_cast<T*>(p); }
};

// One CSR operand on the device.
struct DevCSR {
    int64_t nrows = 0, ncols = 0, nnz = 0;
    const int64_t* rowptr = nullptr;
    const int32_t* col = nullptr;
    const double* val64 = nullptr;   // null for a pattern matrix
    const float* val32 = nullptr;    // FP32 copy of the values (lazily made)
    const void* valdf = nullptr;     // double-float copy (df64 pairs, lazily made)
};

// Fixed work split of one CSR operand for the moment engine (see
// cheb_kernels.cu): chunks of Uc units and segments of rows longer than Uc.
struct SpmmPlan {
    bool ready = false;
    int64_t nch = 0, Uc = 0, Ul = 0, nseg = 0;   // chunks, chunk units, long-row threshold, segments
    int nlong = 0;
    int64_t* crow = nullptr;       // row holding the first unit of each chunk
    int64_t* seg_k0 = nullptr;     // first entry of each segment
    int64_t* long_seg0 = nullptr;  // first segment of each long row (nlong + 1)
    int32_t* seg_row = nullptr;    // row of each segment
    int32_t* long_rows = nullptr;  // the long rows
    int32_t* seg_order = nullptr;  // segments in the order they are dealt out (see ensure_spmm_plan)
    void* mem = nullptr;           // one device allocation holding all of the above
};

}  // namespace mlt

struct mlt_matrix {
    int device = 0;
    int num_sms = 0;
    int val_type = MLT_PATTERN;
    unsigned flags = 0;
    double scale = 1.0;
    mlt::DevCSR A;     // A itself, or X for a Gram handle
    mlt::DevCSR AT;    // X^T for a Gram handle
    mlt::DevCSR P;     // MLT_REORDER: A relabelled by decreasing degree (the moment engine's operand)
    int32_t* perm = nullptr;   // MLT_REORDER: original id of each relabelled row (device), else null
    bool owns = true;
    // owned device allocations (null when referencing caller memory)
    void* own_rowptr = nullptr; void* own_col = nullptr; void* own_val = nullptr;
    void* own_val32 = nullptr;
    void* own_t_rowptr = nullptr; void* own_t_col = nullptr; void* own_t_val = nullptr;
    void* own_t_val32 = nullptr;
    void* own_val_df = nullptr;
    void* own_t_val_df = nullptr;
    void* own_p_rowptr = nullptr; void* own_p_col = nullptr; void* own_p_val = nullptr;
    void* own_p_val32 = nullptr; void* own_p_val_df = nullptr;
    // triangle preparation (inside ws_tri; out_col and pairs inside ws_upcol)
    struct {
        int64_t* out_ptr = nullptr;  // row pointer of the degree-oriented out-lists
        int32_t* out_col = nullptr;  // per row: small targets (rows), then mid targets (y16 slots)
        int32_t* nsmall = nullptr;   // length of each out-list's small section
        int4* pairs = nullptr;       // edges into rows of degree > 32767
        int64_t npairs = 0;
        int64_t* crow1 = nullptr;    // row holding the first unit of each pass-1 chunk
        int64_t* crow2 = nullptr;    // same over the out-lists (pass 2)
        int32_t* bslot = nullptr;    // y16 / y32 slot of rows with degree > 127, else -1
        int32_t* longlist = nullptr; // rows cut across pass-1 chunks
        unsigned long long* counters = nullptr;  // chunk counters of pass 1 and pass 2
        int nbig = 0, nlong = 0, grid1 = 0, grid2 = 0;
        int64_t nch1 = 0, nch2 = 0;
    } tri;
    int tri_state = 0;          // 0 unprepared, 1 ready, <0 error code
    bool low_ready = false;     // sum of the diagonal and of squared values, unscaled
    double low_diag = 0.0, low_sq = 0.0;
    double tri_bound = 0.0;     // sum_(i,j) deg_i deg_j
    int group_width = 0;        // probes per group chosen by mlt_autotune (0: from memory)
    int batch_refs = 0;         // persistent batches (mlt_batch) whose graph uses this handle
    // scratch
    mlt::SpmmPlan plan_A, plan_AT, plan_P;
    mlt::DevBuf ws_v[2], ws_v2[2], ws_w, ws_part, ws_dots, ws_misc, ws_out, ws_y, ws_y16, ws_y32, ws_z, ws_x, ws_tri,
        ws_seg, ws_upcol;
    mlt::DevBuf ws_blk[4];      // explicit FP64 vector blocks (polynomial application, Hutch++)
    int64_t dim() const { return (flags & MLT_GRAM) ? A.ncols : A.nrows; }
};

namespace mlt {

// ---- Chebyshev moment kernels (cheb_kernels.cu) -----------------------------
struct MomentPlan {
    int64_t dim;            // operator dimension d
    int B;                  // probes in this group (sorted by degree, descending)
    int ldv;                // row stride of the V buffers (>= B, multiple of 8)
    int K;                  // steps of the longest probe
    const int* act;         // host: active probes at step k (k < K)
    const int64_t* ids_dev; // device: global probe id of each sorted probe
    const int32_t* deg_dev; // device: degree of each sorted probe
    const int64_t* row_dev; // device: output row of each sorted probe
    int direct;
};

// With alloc_only, every device buffer of the group is sized and nothing is
// launched; without it, only kernels are enqueued (buffers already sized).
int run_moments_group(mlt_matrix* M, int precision, const MomentPlan& plan, double a, double b,
                      uint64_t seed, double* mu_dev, int64_t ld_mu, int* err_flag_dev,
                      cudaStream_t s, bool alloc_only);

// One mlt_moments call split into its phases (see mlt_api.cu).
struct MomentJob {
    mlt_matrix* m = nullptr;
    double a = 0, b = 0;
    uint64_t seed = 0;
    int precision = 0, direct = 0;
    double* mu_user = nullptr;
    double* mu_dev = nullptr;
    bool out_dev = false;
    int64_t ld_mu = 0, nprobes = 0;
    size_t out_bytes = 0;
    int* err = nullptr;
    std::vector<MomentPlan> groups;
    std::vector<std::vector<int>> acts;
};
// A persistent batch's CUDA graph points into the workspaces of its handles,
// so no other call may use (and perhaps regrow) them while the batch lives.
inline int handle_busy(const mlt_matrix* m, const char* who)
{
    if (m && m->batch_refs > 0)
        return fail(MLT_EINVAL, std::string(who) + ": the handle belongs to a live mlt_batch (destroy it first)");
    return MLT_OK;
}
int prepare_moment_job(mlt_matrix* m, double a, double b, uint64_t seed, int64_t probe_offset, int64_t nprobes,
                       const int32_t* degree, int precision, unsigned flags, double* mu, int64_t ld_mu,
                       int group_width, MomentJob& J, cudaStream_t s);
int enqueue_moment_job(MomentJob& J, cudaStream_t s);
int finish_moment_job(MomentJob& J, cudaStream_t s);

int ensure_fp32_values(mlt_matrix* M, cudaStream_t s);
int ensure_df_values(mlt_matrix* M, cudaStream_t s);
// FP64 blocks of explicit vectors (row-major, row stride ldv even, columns
// >= cols zero): Y = p(At) X with P0, P1 as scratch (cheb_kernels.cu), and
// the doubling moments of a start block V0 (V1 scratch; dots stay on the device).
int poly_apply_block(mlt_matrix* M, double a, double b, const double* c, int n, const double* X, double* Y, int ldv,
                     int ncols, double* P0, double* P1, cudaStream_t s);
int poly_apply_block_f32(mlt_matrix* M, double a, double b, const double* c, int n, const float* X, float* Y,
                         int ldv, int ncols, float* P0, float* P1, cudaStream_t s);
int moments_block(mlt_matrix* M, double a, double b, double* V0, double* V1, int ldv, int cols, int K,
                  const double** dots_dev, bool df, cudaStream_t s);
int ensure_spmm_plan(mlt_matrix* M, const DevCSR& C, SpmmPlan& P, cudaStream_t s);
// MLT_REORDER: build M->P and M->perm (reorder.cu).
int build_reorder(mlt_matrix* M, cudaStream_t s);
int spmv_f64(mlt_matrix* M, const DevCSR& C, SpmmPlan& P, const double* x, double* y, cudaStream_t s);
int lanczos_bounds(mlt_matrix* M, int steps, uint64_t seed, double* lo, double* hi, cudaStream_t s);

// ---- triangle kernels (tri_kernels.cu) ---------------------------------------
int tri_prepare(mlt_matrix* M, cudaStream_t s);
int tri_block(mlt_matrix* M, uint64_t seed, int64_t id0, int nb, int64_t* x_dev, cudaStream_t s);

// ---- learned level network (mlp_kernels.cu) ---------------------------------
// FP32 parameter vector: W1[128][16], b1[128], W2[128][128], b2[128], w3[128], b3.
constexpr int MLP_IN = 16;
constexpr int MLP_HID = 128;
constexpr int MLP_OFF_W1 = 0;
constexpr int MLP_OFF_B1 = MLP_OFF_W1 + MLP_HID * MLP_IN;
constexpr int MLP_OFF_W2 = MLP_OFF_B1 + MLP_HID;
constexpr int MLP_OFF_B2 = MLP_OFF_W2 + MLP_HID * MLP_HID;
constexpr int MLP_OFF_W3 = MLP_OFF_B2 + MLP_HID;
constexpr int MLP_OFF_B3 = MLP_OFF_W3 + MLP_HID;
constexpr int MLP_NPARAMS = MLP_OFF_B3 + 1;

struct MlpDev {
    float* P = nullptr;            // FP32 master parameters
    float* G = nullptr;            // gradient
    float* M = nullptr;            // Adam first moment
    float* V = nullptr;            // Adam second moment
    __nv_bfloat16* W1b = nullptr;  // BF16 copies read by the tiles
    __nv_bfloat16* W2b = nullptr;
    __nv_bfloat16* W2Tb = nullptr;
    float* part = nullptr;         // per-tile partial gradients
    int64_t part_tiles = 0;
    double* loss = nullptr;        // summed squared error of the last pass
    int* err = nullptr;
};

size_t mlp_smem_bytes();
int mlp_launch_tiles(const MlpDev& D, const float* X, const float* T, int64_t n, float inv_n, int train,
                     float* y, int* err, cudaStream_t s);
int mlp_adam(const MlpDev& D, float lr, int64_t step, int update, cudaStream_t s);

// ---- misc kernels -----------------------------------------------------------
int gershgorin_device(mlt_matrix* M, double* lo, double* hi, cudaStream_t s);

// ---- host-side method (mlt_host.cpp) -----------------------------------------
int cheb_coeffs_host(int fn, double p, double a, double b, int n, double* c);
double cost_of(int l, int model);
// V is (n+1) x (n+1) row-major: V[lo*(n+1)+hi], sample variance of Q_{lo,hi}.
void band_variances(const double* c, int n, const double* mu, int64_t ld, int m, double* V);
int select_levels(const double* V, int n, int cost_model, int m_pilot, int mode, double target,
                  int max_levels, int* levels_out, int* nlevels_out);
void allocate_samples(const int* levels, int L, const double* V, int n, int cost_model, int mode,
                      double target, int m_pilot, int64_t* m_out);
void triangle_estimate_host(const int64_t* x, int64_t m, int64_t nnz, int use_cv, double* est,
                            double* se, double* a1_out = nullptr, double* a2_out = nullptr);
void band_samples(const double* c, int lo, int hi, const double* mu, int64_t ld, int64_t nprobes, double* q);
void level_stats(const double* v, int64_t m, double* mean, double* var);
void triangle_cv_cheb(double a, double b, double* a1, double* a2);
void triangle_estimate_fixed_host(const int64_t* x, int64_t m, int64_t nnz, double a1, double a2, double* est,
                                  double* se);

}  // namespace mlt
