/*
 * mlt.h -- C ABI of the GB300 multilevel Chebyshev-Hutchinson trace engine.
 *
 * Estimates tr f(A) = sum_i f(lambda_i) for a large sparse symmetric A
 * (Hallman & Troester, "A Multilevel Approach to Stochastic Trace Estimation",
 * Section 1, Eq. def:trace) by Hutchinson's estimator with Rademacher probes
 * (Section 2.1, Eq. def:mcEstimate), a degree-n Chebyshev interpolant of f
 * (Section 2.2, Eq. chebSeries) and multilevel Monte Carlo over bands of its
 * coefficients (Section 3, Eqs. def:qlevels, decomposition; Section 4,
 * Eq. multiEstimator).  Triangle counting uses tr(A^3)/6 with control variates
 * (Section 5.4).
 *
 * Conventions shared by every entry point
 *   - Return value: MLT_OK (0) on success, a negative MLT_E* code otherwise.
 *     No call aborts the process or throws; mlt_last_error() returns a message
 *     for the calling thread's most recent failure.
 *   - Arrays passed in are owned by the caller.  A pointer documented as
 *     "host or device" may be either: the library asks the CUDA driver which
 *     one it is.  Device pointers must be on the current device.
 *   - `stream` is a cudaStream_t (NULL = legacy default stream).  Calls return
 *     after their results are in the caller's arrays (host outputs) or after
 *     the work producing them has been queued on `stream` (device outputs of
 *     mlt_moments); scratch buffers belong to the matrix handle, so calls on
 *     one handle must not overlap.
 *   - CSR layout: rowptr int64[nrows+1], col int32[nnz] (each row's columns
 *     ascending, no duplicates), values per val_type.
 *   - Probes: probe id p (a global counter, p < 2^32) has entries
 *       h   = mix64((((p / 64) << 32) | i) ^ (seed * 0x9E3779B97F4A7C15)),
 *       z_i = -1 if bit (p mod 64) of h is set, +1 otherwise,
 *     mix64 the SplitMix64 output finaliser (Steele, Lea, Flood 2014), so one
 *     hash gives the signs of 64 consecutive probes at one row.  The paper
 *     only asks for Rademacher entries (Section 2.1); fixing the generator
 *     makes every result reproducible under any blocking.
 */
#ifndef MLT_H
#define MLT_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---- status codes -------------------------------------------------------- */
#define MLT_OK        0
#define MLT_EINVAL   (-1)  /* bad argument (null pointer, size, interval, ...) */
#define MLT_ENOMEM   (-2)  /* device or host allocation failed                 */
#define MLT_ECUDA    (-3)  /* a CUDA call failed                               */
#define MLT_ERANGE   (-4)  /* result bound exceeded (int64 triangle bound, ...) */
#define MLT_ETIMEOUT (-5)  /* a bounded device wait gave up                    */

/* ---- value types of mlt_create_csr --------------------------------------- */
#define MLT_F64      0     /* vals is double[nnz]                            */
#define MLT_F32      1     /* vals is float[nnz]                             */
#define MLT_PATTERN  2     /* vals ignored: every stored entry equals 1      */

/* ---- flags of mlt_create_csr --------------------------------------------- */
#define MLT_GRAM        1u /* the operator is A = X^T X of the given X        */
#define MLT_DEVICE_PTRS 2u /* rowptr/col/vals are device pointers; they are
                              referenced, not copied, and must outlive the
                              handle                                         */
#define MLT_REORDER     4u /* the moment engine (mlt_moments and the calls
                              built on it) runs on a copy of the operator
                              relabelled by decreasing degree (ties by
                              increasing id), with each probe entry taken
                              at its original row id: the moments are those
                              of the original operator and probes, up to
                              the order of the floating-point sums.  Pays
                              on power-law graphs, whose hub rows take most
                              gathers; square (non-Gram) handles only; the
                              copy doubles the handle's CSR memory        */

/* ---- functions f of mlt_cheb_coeffs -------------------------------------- */
#define MLT_FN_LOG   0     /* log x      (log-determinant)                   */
#define MLT_FN_SQRT  1     /* sqrt x     (nuclear norm with A = X^T X)       */
#define MLT_FN_EXP   2     /* exp x      (Estrada index)                     */
#define MLT_FN_INV   3     /* 1/x        (trace of the inverse)              */
#define MLT_FN_POW   4     /* x^p        (Schatten p-norms use p/2)          */
#define MLT_FN_CUBE  5     /* x^3        (triangle counting, tr A^3)         */

/* ---- precision of mlt_moments -------------------------------------------- */
#define MLT_PREC_FP64 0    /* vectors, SpMM and dots in FP64                 */
#define MLT_PREC_FP32 1    /* vectors and SpMM in FP32, dots summed in FP64  */
#define MLT_PREC_MIXED 2   /* FP32 steps first, FP64 after: see below       */
#define MLT_PREC_DF64 3    /* vectors, SpMM and per-thread dots as double-
                              float pairs (hi + lo, about 48 significant
                              bits) on the FP32 pipes, FP64 from the CTA
                              sums on: FP64-class moments at FP32 speed     */
/* MLT_PREC_MIXED_AT(k): the first k recurrence steps (degrees up to 2k with
 * the doubling identities, up to k in direct mode) run with FP32 vectors, the
 * rest with FP64 vectors (the two live vectors are widened at the switch);
 * FP32 drift grows with the degree, FP64 steps stop it from growing further. */
#define MLT_PREC_MIXED_AT(k) (MLT_PREC_MIXED | ((k) << 8))

/* ---- flags of mlt_moments ------------------------------------------------ */
#define MLT_DIRECT   1u    /* mu_j = z . V_j at every step (n matvecs for
                              degree n) instead of the doubling identities
                              mu_2k = 2 V_k.V_k - mu_0,
                              mu_2k+1 = 2 V_k+1.V_k - mu_1 (ceil(n/2) matvecs) */

/* ---- flags of mlt_mlmc_estimate (with those of mlt_moments) -------------- */
#define MLT_LOW_CV 4u      /* the low-degree terms as control variates (Section
                              5.4, applied to the bands as its closing remark
                              suggests): per level, w_j = mu_j - tr T_j(At)
                              (j = 1, 2; j = 1 for X^T X; j <= the level's
                              degree) have mean zero; the band samples are
                              fitted by least squares on (1, w) and the level
                              reports the intercept and the residual variance
                              (divisor m - 1 - J).  The fit reuses the samples
                              (an O(1/m) bias, as in the triangle estimator)
                              and is skipped when m <= J + 1 or the centred
                              covariates are degenerate (det <= 1e-12 x the
                              product of their sums of squares).  Levels and
                              sample counts still come from the plain pilot
                              variances. */

/* ---- spectrum interval methods ------------------------------------------- */
#define MLT_BOUNDS_GERSHGORIN 0
#define MLT_BOUNDS_LANCZOS    1

/* ---- multilevel parameters ------------------------------------------------ */
#define MLT_MAX_LEVELS 1024
#define MLT_MAX_DEGREE 4096
#define MLT_MODE_BUDGET    0   /* target = total cost C in cost-model units   */
#define MLT_MODE_VARIANCE  1   /* target = estimator variance eps^2           */
#define MLT_COST_SYMMETRIC 0   /* C_{l'l} = ceil(l/2)  (Section 3.1)          */
#define MLT_COST_LINEAR    1   /* C_{l'l} = l          (Section 3.1)          */

typedef struct mlt_matrix mlt_matrix;   /* opaque; owns device copies */

/*
 * Create a matrix handle from a CSR matrix (nrows x ncols, nnz entries).
 * The stored entries are multiplied by `scale` (use 1.0 for none; a 0/1
 * adjacency scaled to a chosen spectral radius uses scale != 1).  Without
 * MLT_GRAM the matrix must be square and symmetric (symmetry is the caller's
 * promise, not checked) and the operator is A itself; with MLT_GRAM the
 * operator is A = X^T X (dimension ncols), applied as X^T (X v) (Section 1,
 * footnote on Schatten norms).  Host arrays are copied to the device (on
 * `stream`, finished before return); with MLT_DEVICE_PTRS they are used in
 * place.  Errors: MLT_EINVAL on negative sizes, null arrays with nnz > 0,
 * nnz > 2^31-1, rowptr[0] != 0 or rowptr[nrows] != nnz, MLT_REORDER with
 * MLT_GRAM; MLT_ENOMEM; MLT_ECUDA.
 */
int mlt_create_csr(int64_t nrows, int64_t ncols, int64_t nnz,
                   const int64_t* rowptr, const int32_t* col, const void* vals,
                   int val_type, double scale, unsigned flags, void* stream,
                   mlt_matrix** out);

/* Release a handle and every device buffer it owns (NULL is a no-op).  The
 * call waits for the device to finish its work first; it fails with
 * MLT_EINVAL while a live mlt_batch holds the handle.  The buffers go back to
 * the library's memory pool (see mlt_release_cached), not to the driver. */
int mlt_destroy(mlt_matrix* m);

/* Return to the driver the device memory that destroyed handles left cached.
 * Handles take their device memory from one stream-ordered pool per device
 * that keeps freed blocks for later handles (a handle created after another
 * was destroyed maps no new memory); memory of live handles is untouched.
 * No counterpart in the paper: memory management only.  Errors: MLT_ECUDA. */
int mlt_release_cached(void);

/* Operator dimension d (nrows, or ncols for a Gram handle) and stored nnz. */
int mlt_matrix_info(const mlt_matrix* m, int64_t* dim, int64_t* nnz);

/*
 * Interval [a, b] containing the spectrum of the operator.  The map
 * g(x) = (2x - a - b)/(b - a) needs one (Section 2.2).  MLT_BOUNDS_GERSHGORIN:
 * Gershgorin discs (min_i a_ii - r_i, max_i a_ii + r_i) for A; for a Gram
 * handle [0, ||X||_1 ||X||_inf].  MLT_BOUNDS_LANCZOS: `steps` Lanczos steps
 * (at least 2) from the Rademacher start vector of probe id 0 under `seed`;
 * the interval is [theta_min - r_min, theta_max + r_max] (extreme Ritz values
 * and their residual norms), widened by 1%, with the lower end at least
 * 1e-6 b for a Gram handle.  A Lanczos interval is an estimate, not a proof.
 */
int mlt_spectrum_bounds(mlt_matrix* m, int method, int steps, uint64_t seed,
                        double* a, double* b);

/*
 * Chebyshev coefficients c[0..n] of the degree-n interpolant of
 * f~ = f o g^{-1} on [-1, 1] at the nodes x_j = cos(j pi / n), 0 <= j <= n
 * (Section 2.2, Eq. chebSeries and the node formula), so that
 * f(x) ~= sum_j c_j T_j(g(x)) on [a, b].  `p` is the exponent for MLT_FN_POW.
 * c: host array of n+1 doubles.  Errors: MLT_EINVAL for n < 1 or n > MLT_MAX_DEGREE,
 * a >= b, an unknown fn, or f undefined somewhere on [a, b] (log/sqrt/pow of a
 * negative number, 1/x across 0).
 */
int mlt_cheb_coeffs(int fn, double p, double a, double b, int n, double* c);

/*
 * Chebyshev moments mu[p][j] = z_p^T T_j(At) z_p, j = 0..degree[p], with
 * At = (2A - (a+b) I)/(b-a) and z_p the probe with id probe_offset + p
 * (Section 2.2: the three-term recurrence Eq. recurrence applied to a block of
 * probes; the doubling identities unless MLT_DIRECT).  Each probe stops at its
 * own degree, so one call serves all levels of a multilevel run.
 *   degree : host int32[nprobes], each 0..MLT_MAX_DEGREE.
 *   mu     : host or device double[nprobes * ld_mu], row p = probe p;
 *            entries j > degree[p] are set to 0.  ld_mu >= max degree + 1.
 *   precision: MLT_PREC_FP64, MLT_PREC_FP32, MLT_PREC_MIXED_AT(k) or
 *              MLT_PREC_DF64 (see their definitions above); flags: 0 or
 *              MLT_DIRECT.
 * Errors: MLT_EINVAL (a >= b, bad sizes, ld_mu too small), MLT_ENOMEM,
 * MLT_ECUDA.  Moments with |mu_j| > d (1 + 1e-6), impossible when the spectrum
 * lies in [a, b], give MLT_ERANGE after the results are written.
 */
int mlt_moments(mlt_matrix* m, double a, double b, uint64_t seed,
                int64_t probe_offset, int64_t nprobes, const int32_t* degree,
                int precision, unsigned flags, double* mu, int64_t ld_mu,
                void* stream);

/*
 * Many moment computations (each as one mlt_moments call would do it) run as
 * a single CUDA-graph launch, one graph branch per job, so that small
 * matrices with ragged probe blocks share the GPU instead of queueing launch
 * after launch.  Every job must use its own matrix handle.  All device memory
 * is reserved and all inputs are on the device before the graph is captured;
 * the call returns when every job's results are in its mu.  group_width is the
 * number of probes per group (0: the handle's, see mlt_autotune; without one,
 * as many as fit a third of the free device memory, at most 1024, and at most
 * 64 for operators of 2^20 rows or more with 8-byte vectors).  Errors as
 * mlt_moments, plus MLT_EINVAL for a repeated handle.
 */
typedef struct {
    mlt_matrix* matrix;
    double a, b;
    uint64_t seed;
    int64_t probe_offset;
    int64_t nprobes;
    const int32_t* degree;   /* host int32[nprobes]                       */
    double* mu;              /* host or device double[nprobes * ld_mu]    */
    int64_t ld_mu;
    int group_width;
} mlt_moments_job;

int mlt_moments_batched(const mlt_moments_job* jobs, int njobs, int precision, unsigned flags,
                        void* stream);

/*
 * The same job set as a persistent batch: mlt_batch_create prepares every job
 * (validation, probe order, groups, every device buffer) and captures and
 * instantiates one CUDA graph with a branch per job, once; mlt_batch_run
 * replays that graph, each job's probes taking ids probe_offset + id_shift + p
 * (the shift is written into the id tables the graph reads, so one graph
 * serves any number of fresh probe sets), and returns when every job's moments
 * are in its mu (host outputs are copied there after the replay).  The seeds,
 * degrees, intervals, outputs and precision stay those of the create call.
 * While a batch lives, its graph points into the workspaces of its handles:
 * every other call on those handles, mlt_destroy included, fails with
 * MLT_EINVAL until mlt_batch_destroy.  Calls of one batch must not overlap.
 * Errors: as mlt_moments_batched; mlt_batch_run also MLT_EINVAL when shifted
 * ids leave [0, 2^32).
 */
typedef struct mlt_batch mlt_batch;   /* opaque */

int mlt_batch_create(const mlt_moments_job* jobs, int njobs, int precision, unsigned flags, void* stream,
                     mlt_batch** out);
int mlt_batch_run(mlt_batch* b, int64_t id_shift, void* stream);
int mlt_batch_destroy(mlt_batch* b);   /* NULL is a no-op; waits for the device */

/*
 * Choose the probe-group width (probes sharing one pass over the matrix) for
 * this handle: each width in {8, 16, 32, 64, 128} is timed on a short trial
 * (two groups of that width, trial_steps recurrence steps, CUDA events) and
 * the one with the least time per probe-matvec is kept on the handle for later
 * mlt_moments calls.  *best (may be NULL) receives it.
 */
int mlt_autotune(mlt_matrix* m, int precision, int trial_steps, int* best, void* stream);

typedef struct {
    int fn;                          /* MLT_FN_*                                  */
    double fn_p;                     /* exponent for MLT_FN_POW                   */
    double a, b;                     /* spectrum interval, a < b                  */
    int n;                           /* interpolant degree, 1..MLT_MAX_DEGREE     */
    uint64_t seed;                   /* probe seed; probe ids start at 0          */
    int nlevels;                     /* > 0: fixed levels/m below; 0: automatic   */
    int32_t levels[MLT_MAX_LEVELS];  /* fixed: 0 <= l_1 < ... < l_L = n           */
    int64_t m[MLT_MAX_LEVELS];       /* fixed: samples per level (>= 1)           */
    int m_pilot;                     /* automatic: pilot probes at degree n (>= 2) */
    int mode;                        /* automatic: MLT_MODE_BUDGET / _VARIANCE    */
    double target;                   /* automatic: budget C or variance eps^2     */
    int cost_model;                  /* MLT_COST_SYMMETRIC / MLT_COST_LINEAR      */
    int max_levels;                  /* automatic: at most this many levels, 0 = any */
    int reuse_pilot;                 /* automatic: pilot rows count as top-level samples */
    int precision;                   /* MLT_PREC_*                                */
    unsigned flags;                  /* mlt_moments flags                         */
    void* stream;                    /* cudaStream_t                              */
} mlt_mlmc_params;

typedef struct {
    double estimate;                 /* Gamma_m of Eq. multiEstimator             */
    double std_error;                /* sqrt(sum_k s_k^2 / m_k)                   */
    int nlevels;
    int32_t levels[MLT_MAX_LEVELS];
    int64_t m[MLT_MAX_LEVELS];       /* samples used per level                    */
    double level_mean[MLT_MAX_LEVELS];
    double level_var[MLT_MAX_LEVELS];/* sample variance of each level's Q         */
    int64_t probes;                  /* probe ids consumed (pilot included)       */
    int64_t matvecs;                 /* operator applications, pilot included     */
} mlt_mlmc_result;

/* Default parameters: automatic levels, budget mode, symmetric cost model,
 * reuse of the pilot, FP64. */
void mlt_mlmc_default_params(mlt_mlmc_params* p);

/*
 * Multilevel estimate of tr p_n(At) ~= tr f(A) (Section 3; Section 4,
 * Eq. multiEstimator).  Fixed mode (nlevels > 0): level k uses m[k] fresh
 * probes, ids following those of level k-1 (level 1 starts at id 0), each run
 * to degree levels[k]; its samples are Q_{l_{k-1} l_k} = sum of c_j mu_j over
 * j = l_{k-1}+1 .. l_k (l_0 = -1).  Automatic mode (nlevels == 0): m_pilot
 * probes (ids 0..m_pilot-1) at degree n give the variance of every band
 * (Section 3.2.1); levels come from the dynamic programme of Theorem levels,
 * where at l = n only predecessors whose path recommends at least m_pilot
 * top-level samples are allowed; sample counts are
 * m_k = max(1, ceil(mu sqrt(V_k/C_k))) (Eqs. optSamples, optMu); fresh probes
 * follow the pilot's ids level by level.  All levels' probes run in one
 * ragged mlt_moments call.  Errors as mlt_moments, plus MLT_EINVAL for bad
 * parameters.
 */
int mlt_mlmc_estimate(mlt_matrix* m, const mlt_mlmc_params* p, mlt_mlmc_result* r);

/*
 * The host-side steps of mlt_mlmc_estimate, one by one, for callers that
 * spread a multilevel estimate over several processes or GPUs (the probes are
 * independent samples, Section 4, Eq. multiEstimator): one process runs the
 * pilot and the level selection, every process computes moments and band
 * samples for its own probe ids, and the samples, gathered in probe-id order,
 * are combined.  mlt_mlmc_estimate calls the same routines, so with the same
 * moments the combination is the same to the last bit.  None of these calls
 * touches a GPU; all arrays are host memory.
 *
 * mlt_pilot_variances (Section 3.2.1): V[lo * (n+1) + hi], 0 <= lo < hi <= n,
 *   is the sample variance (divisor m_pilot - 1) over the m_pilot moment rows
 *   of Q_{lo,hi} = sum_{j=lo+1..hi} c_j mu_j (Eq. def:qlevels); every other
 *   entry is 0, and all entries are 0 when m_pilot < 2.  mu: m_pilot rows of
 *   ld_mu >= n+1 doubles (mu_0..mu_n first); V: (n+1)^2 doubles.  Errors:
 *   MLT_EINVAL (null pointers, n outside [1, MLT_MAX_DEGREE], ld_mu < n+1).
 */
int mlt_pilot_variances(const double* c, int n, const double* mu, int64_t ld_mu, int64_t m_pilot, double* V);

/*
 * mlt_select_levels: the levels l_1 < ... < l_L = n of the dynamic programme
 *   of Theorem levels (Eq. costrecurrence) on the variance table V of
 *   mlt_pilot_variances, and their sample counts
 *   m_k = max(1, ceil(mu sqrt(V_k / C_k))) (Eqs. optSamples, optMu; budget
 *   or variance mode, cost model as in mlt_mlmc_params).  With m_pilot > 0 the
 *   top level must be recommended at least m_pilot samples and gets at least
 *   that many (the pilot rows are reused there, Section 3.2.1); max_levels > 0
 *   caps the number of levels.  levels, m: arrays of at least n+1 entries
 *   (L <= n+1); *nlevels receives L.  Errors: MLT_EINVAL (bad sizes, mode,
 *   cost model, a non-positive target, a negative or non-finite V entry).
 */
int mlt_select_levels(const double* V, int n, int cost_model, int m_pilot, int mode, double target,
                      int max_levels, int32_t* levels, int64_t* m, int* nlevels);

/*
 * mlt_band_samples: q[p] = sum_{j=lo+1..hi} c_j mu[p * ld_mu + j] for
 *   p < nprobes (Eq. def:qlevels; lo = -1 starts the first band at c_0 mu_0),
 *   summed left to right.  Errors: MLT_EINVAL (null pointers with
 *   nprobes > 0, not -1 <= lo < hi <= MLT_MAX_DEGREE, ld_mu < hi + 1).
 */
int mlt_band_samples(const double* c, int lo, int hi, const double* mu, int64_t ld_mu, int64_t nprobes,
                     double* q);

/*
 * mlt_mlmc_combine: Eq. multiEstimator from the samples of each level,
 *   concatenated level by level (m[0] samples of level 0 first), each level's
 *   samples in probe-id order (pilot rows first on a level that reuses them):
 *   estimate = sum_k mean_k, std_error = sqrt(sum_k var_k / m_k), var_k with
 *   divisor m_k - 1 (NaN when m_k = 1).  Fills estimate, std_error, nlevels,
 *   levels, m, level_mean and level_var of r; probes and matvecs are set to 0
 *   (they depend on how the samples were drawn).  Errors: MLT_EINVAL (null
 *   pointers, nlevels outside [1, MLT_MAX_LEVELS], some m[k] < 1).
 */
int mlt_mlmc_combine(int nlevels, const int32_t* levels, const int64_t* m, const double* samples,
                     mlt_mlmc_result* r);

/*
 * Exact traces of the low-degree Chebyshev terms (closing remark of Section
 * 5.4), At = alpha A + beta I on [a, b] (Section 2.2): t[0] = tr I = d,
 * t[1] = tr At = alpha tr A + beta d, t[2] = tr T_2(At) = 2 tr At^2 - d with
 * tr A^2 = ||A||_F^2 (A symmetric).  For a Gram handle only t[0], t[1]
 * (tr X^T X = ||X||_F^2).  Values count scale times (a pattern entry is 1;
 * X^T X scales by scale^2).  tr A and ||A||_F^2 are reduced on the device
 * once per handle in a fixed order.  t: host double[3]; *count (may be NULL)
 * receives 3, or 2 for a Gram handle.  Errors: MLT_EINVAL (null handle or
 * t, a >= b), MLT_ECUDA.
 */
int mlt_low_traces(mlt_matrix* m, double a, double b, double* t, int* count, void* stream);

/*
 * Y = p(At) X for a block of ncols vectors, p = sum_{k=0..n} c[k] T_k with the
 * coefficients of mlt_cheb_coeffs (Section 2.2, Eq. chebSeries), At the map of
 * [a, b] onto [-1, 1] applied to the handle's operator (A scaled, or X^T X).
 * Evaluated by Clenshaw's recurrence for Chebyshev sums: n operator
 * applications per vector, FP64 throughout.
 * X, Y: d x ncols, row-major with row strides ldx, ldy >= ncols (entry i of
 * vector j at X[i * ldx + j]); host memory, or device memory with
 * MLT_DEVICE_PTRS in flags; they must not overlap.  Y is complete on return
 * (the call synchronises `stream`).
 * Errors: MLT_EINVAL (null pointers, n outside [1, MLT_MAX_DEGREE], a >= b,
 * ncols outside [1, 4096], strides below ncols, unknown flags), MLT_ENOMEM,
 * MLT_ECUDA.
 */
int mlt_poly_apply(mlt_matrix* m, double a, double b, const double* c, int n,
                   const double* X, int64_t ldx, double* Y, int64_t ldy, int ncols,
                   unsigned flags, void* stream);

/*
 * Hutch++ on tr p(At), the variance reduction Section 5.3 proposes for the
 * Estrada index (the method of Meyer, Musco, Musco and Woodruff, 2021).
 * p = sum_{k=0..n} c[k] T_k as in mlt_poly_apply.  With S the s Rademacher
 * probes of ids probe_offset .. probe_offset + s - 1 and G the g probes that
 * follow (the generator of mlt_moments):
 *   Q         orthonormal basis of p(At) S: Cholesky QR applied twice when
 *             s <= 64 and both Gram matrices factor (every pivot above 1e-13
 *             of its diagonal entry); otherwise classical Gram-Schmidt with
 *             every column projected twice, where a column left with at most
 *             1e-10 of its norm is dependent and dropped (rank counts the
 *             columns kept);
 *   t_sketch  tr(Q^T p(At) Q), from the doubling moments of Q's columns;
 *   samples   q_i = g_i'^T p(At) g_i' with g_i' = (I - Q Q^T) g_i;
 *   estimate  t_sketch + t_rest, t_rest the mean of the q_i, and std_error
 *             sqrt(var(q) / g) (divisor g - 1; NaN when g < 2).
 * Unbiased for tr p(At) whatever Q is, since Q does not depend on G; exact
 * when Q spans the whole space.  Cost: s*n + (s + g)*ceil(n/2) operator
 * applications (matvecs).
 * precision: MLT_PREC_FP64 (all FP64); MLT_PREC_FP32 to evaluate the sketch
 * p(At) S in FP32 (the handle's FP32 values), Q, its trace, the deflation and
 * the remainder staying FP64; or MLT_PREC_DF64, the FP32 sketch with the
 * moments of Q and of the remainder probes in double-float pairs.  Rounding
 * in the sketch only moves span(Q), which changes the variance but not the
 * expectation.
 * samples: g doubles (host) or NULL.  0 <= s <= 128, 0 <= g <= 1024, s + g >= 1.
 * Errors: MLT_EINVAL (null m, c or out; n outside [1, MLT_MAX_DEGREE]; a >= b;
 * s, g out of range; probe ids beyond 2^32; other precisions), MLT_ENOMEM,
 * MLT_ECUDA.
 */
typedef struct {
    double estimate;
    double std_error;
    double t_sketch;
    double t_rest;
    int rank;
    int64_t matvecs;
} mlt_hutchpp_result;

int mlt_hutchpp_estimate(mlt_matrix* m, double a, double b, const double* c, int n,
                         uint64_t seed, int64_t probe_offset, int s, int g, int precision,
                         double* samples, mlt_hutchpp_result* out, void* stream);

/*
 * Triangle-count estimate tr(A^3)/6 for a symmetric 0/1 adjacency matrix with
 * no self-loops (Section 2.1 Example; Section 5.4).  For probes
 * probe_offset .. probe_offset+nprobes-1 it computes, exactly in int64,
 * x1 = z^T A z, x2 = z^T A^2 z, x3 = z^T A^3 z (two sparse products per probe
 * block, using the symmetry of the quadratic form), in blocks of `block`
 * probes, 128 or 256.  Blocks of 128 (the block of Section 5.4's workload)
 * run two per launch, so both sizes cost the same and every probe's moments
 * are the same integers under either; a last, partial launch costs a full
 * one.  With
 * use_cv the estimate is
 * [mean x3 - a2 (mean x2 - nnz) - a1 mean x1] / 6 with a1, a2 the least-squares
 * slopes of x3 on (x1, x2) (Section 5.4; tr A = 0, tr A^2 = nnz); without it,
 * mean x3 / 6.  x (host or device int64[nprobes*3], may be NULL) receives the
 * per-probe moments.  Errors: MLT_EINVAL (not a square pattern matrix, a
 * self-loop, nprobes < 1, block not 128 or 256); MLT_ERANGE when the bound
 * sum_(i,j) deg_i deg_j on |x3| reaches 2^62.
 */
int mlt_triangle_trace(mlt_matrix* m, uint64_t seed, int64_t probe_offset,
                       int64_t nprobes, int block, int use_cv, int64_t* x,
                       double* estimate, double* std_error, void* stream);

/* ---- control variates of mlt_triangle_estimate ---------------------------- */
#define MLT_TRI_CV_NONE 0  /* mean x3 / 6                                        */
#define MLT_TRI_CV_FIT  1  /* a1, a2 by least squares over the samples (as
                              mlt_triangle_trace with use_cv)                    */
#define MLT_TRI_CV_CHEB 2  /* a1, a2 chosen a priori from the Chebyshev
                              expansion of x^3 on [a, b] (Section 5.4)           */

/*
 * The estimate of mlt_triangle_trace from per-probe moments x (host
 * int64[nprobes * 3]: x1, x2, x3 of each probe), with the control variates of
 * Section 5.4: T = [mean x3 - a2 (mean x2 - nnz) - a1 mean x1] / 6
 * (tr A = 0, tr A^2 = nnz).  MLT_TRI_CV_NONE: a1 = a2 = 0, variance divisor
 * m - 1.  MLT_TRI_CV_FIT: the least-squares slopes of x3 on (1, x1, x2),
 * residual variance divisor m - 3 (an O(1/m) bias from fitting on the same
 * samples).  MLT_TRI_CV_CHEB: with [a, b] holding the spectrum of A,
 * c = (a+b)/2, r = (b-a)/2 and x^3 = (3 T_1(x) + T_3(x))/4 on [-1, 1],
 * A^3 - a2 A^2 - a1 A = (r^3/4) T_3(At) + (c^3 - 3 c r^2/4) I for
 * a2 = 3c, a1 = 3r^2/4 - 3c^2; fixed in advance, these leave the estimate
 * unbiased, and the residual variance has divisor m - 1.  Sums are exact
 * 128-bit integers; the double-precision steps follow a fixed order.
 * a1, a2 (may be NULL) receive the coefficients used.  Errors: MLT_EINVAL
 * (null x, nprobes < 1, nnz < 0, unknown cv, a >= b for MLT_TRI_CV_CHEB),
 * MLT_ERANGE (sums beyond 128 bits).
 */
int mlt_triangle_estimate(const int64_t* x, int64_t nprobes, int64_t nnz, int cv, double a, double b,
                          double* estimate, double* std_error, double* a1, double* a2);

/*
 * Learned coarse level.  The paper has no network; this is a project addition
 * whose nearest relative is the regression control variate of Section 5.4.  A
 * 16 -> 128 -> 128 -> 1 ReLU network S (BF16 weights and activations, FP32
 * accumulation on the tensor cores) maps the scaled low-degree moments
 * (mu_0 .. mu_15) / d of a probe to an estimate of its degree-l1 quadratic
 * form P_l1 / d.  Used as the lowest level of a multilevel estimator,
 *   E[P_n] = E[d S] + E[P_l1 - d S] + E[P_n - P_l1],
 * it keeps the estimate unbiased for any S; a good S only lowers the variance.
 * Parameters (FP32, MLT_NET_NPARAMS values): W1[128][16], b1[128],
 * W2[128][128], b2[128], w3[128], b3; y = w3 . relu(W2 relu(W1 x + b1) + b2) + b3.
 * Feature and target arrays (x: n x 16 floats row-major, t: n floats) may be
 * host or device memory.  Errors: MLT_EINVAL, MLT_ENOMEM, MLT_ECUDA, and
 * MLT_ETIMEOUT if a bounded tensor-core wait gave up.
 */
#define MLT_NET_IN       16
#define MLT_NET_HID      128
#define MLT_NET_NPARAMS  18817

typedef struct mlt_surrogate mlt_surrogate;   /* opaque; owns device parameters */

/* New network on the current device, weights drawn from N(0, 2/fan_in) with a
 * generator seeded by `seed` (biases 0). */
int mlt_surrogate_create(uint64_t seed, mlt_surrogate** out);
int mlt_surrogate_destroy(mlt_surrogate* s);
/* Copy the FP32 parameter vector in or out (host arrays of MLT_NET_NPARAMS). */
int mlt_surrogate_set_params(mlt_surrogate* s, const float* params);
int mlt_surrogate_get_params(mlt_surrogate* s, float* params);
/* The standardisation mlt_learned_train set (host array of 34 doubles): the
 * 16 feature means, the 16 feature standard deviations, then the target's
 * mean and standard deviation; feature k enters the network as
 * (mu_k/d - mean_k)/std_k and the network's estimate of P_l1 is
 * d (mean_t + std_t y).  *has_norm is 0 (and the array all zeros) before any
 * training, when features and target enter unscaled. */
int mlt_surrogate_get_norm(mlt_surrogate* s, double* norm, int* has_norm);
/* Mean squared error over n samples and its gradient (host array of
 * MLT_NET_NPARAMS, may be NULL); the parameters are not changed. */
int mlt_surrogate_loss_grad(mlt_surrogate* s, const float* x, const float* t, int64_t n,
                            double* loss, float* grad, void* stream);
/* `epochs` passes of Adam (lr, beta1 0.9, beta2 0.999) over consecutive
 * minibatches of `batch` samples (the samples are independent probes, so no
 * shuffling); *final_loss (may be NULL) is the mean squared error of the last
 * epoch. */
int mlt_surrogate_train(mlt_surrogate* s, const float* x, const float* t, int64_t n, int epochs,
                        int64_t batch, double lr, double* final_loss, void* stream);
/* y[i] = S(x_i), n outputs (host or device). */
int mlt_surrogate_predict(mlt_surrogate* s, const float* x, int64_t n, float* y, void* stream);

typedef struct {
    int fn;             /* MLT_FN_*                                            */
    double fn_p;        /* exponent for MLT_FN_POW                             */
    double a, b;        /* spectrum interval                                   */
    int n;              /* interpolant degree                                  */
    int l1;             /* degree of the exact level above the network (>= 15) */
    int64_t m_net;      /* samples of d S                                      */
    int64_t m_1;        /* samples of P_l1 - d S                               */
    int64_t m_2;        /* samples of P_n - P_l1 (0 when l1 == n)              */
    uint64_t seed;
    int64_t probe_offset;  /* first probe id; ids run level by level           */
    int precision;      /* MLT_PREC_*                                           */
    void* stream;
} mlt_learned_params;

/*
 * Train s on n_train probes (ids train_offset ..): features (mu_0..mu_15)/d,
 * target P_l1/d with the Chebyshev coefficients of f (Section 2.2).  The
 * moments come from mlt_moments at degree l1.  Features and target are
 * standardised with their training mean and standard deviation (kept in s),
 * so the network models the probe-to-probe fluctuation, which is far below
 * the mean and would otherwise be lost to BF16 rounding; mlt_learned_estimate
 * then uses d (mean_t + std_t S(x)) as the network's estimate of P_l1.
 */
int mlt_learned_train(mlt_matrix* m, mlt_surrogate* s, const mlt_learned_params* p,
                      int64_t n_train, int64_t train_offset, int epochs, int64_t batch, double lr,
                      double* final_loss);

/*
 * Three-level estimate of tr p_n(At) with the network as the lowest level:
 * levels (S, P_l1 - S, P_n - P_l1) with m_net, m_1, m_2 fresh probes; the
 * result's levels[] are {15, l1, n}.  Each level is an independent sample
 * mean, as in Eq. multiEstimator.
 */
int mlt_learned_estimate(mlt_matrix* m, mlt_surrogate* s, const mlt_learned_params* p,
                         mlt_mlmc_result* r);

/*
 * Chebyshev moments with no device allocation at all (the paper has no
 * counterpart).  For callers that cannot call cudaMalloc: code running inside
 * a stream capture it does not own, loops that cannot absorb the device-wide
 * synchronisation an allocation may cause, and hosts whose memory pool has
 * claimed the device memory.  It computes what mlt_moments computes with
 * MLT_PREC_FP64 and the doubling identities, for a CSR matrix given directly
 * by device arrays (d x d, symmetric: rowptr int64[d+1], col int32[nnz],
 * vals double[nnz] or NULL for a 0/1 pattern, every entry times `scale`), and
 * writes mu (device double[nprobes * ld_mu]).  degree is a host array of
 * nprobes (at most 512) degrees.  Working memory is one fixed 32 MiB device
 * array inside the library, held by every GPU that loads it until the process
 * exits: the call fails with MLT_ERANGE when 2 d ldv plus its small tables
 * exceed 4,194,304 doubles (ldv = nprobes rounded up to 32).  All calls share
 * that array and it keeps the last call's contents, so calls that overlap on
 * the GPU race (a captured graph holding a call included); order them.  The
 * first call on each device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; make it before any stream
 * capture (during capture that first call fails with MLT_EINVAL).  Later
 * calls may be captured: they then copy nothing from host memory and do not
 * synchronise, and CSR entries out of range turn the probes' mu rows into NaN
 * when the graph runs.  Outside a capture the call returns after mu is
 * written.  Errors: MLT_EINVAL (bad sizes, pointers, interval, CSR entries out
 * of range outside a capture), MLT_ERANGE, MLT_ECUDA.
 */
int mlt_moments_noalloc(int64_t d, int64_t nnz, const int64_t* rowptr, const int32_t* col,
                        const double* vals, double scale, double a, double b, uint64_t seed,
                        int64_t probe_offset, int nprobes, const int32_t* degree, double* mu,
                        int64_t ld_mu, void* stream);

/*
 * The FP64 arithmetic rate of the current device, in TFLOP/s, measured (the
 * paper has no counterpart: it is the denominator of the roofline of FP64
 * moment steps, which this part bounds by FP64 arithmetic, not memory).  One
 * launch of 8 CTAs per SM x 256 threads, each thread running eight independent
 * register-resident FMA chains for `iters` steps, timed with CUDA events on
 * `stream` after a short warm-up launch; 2 flops per FMA.  Allocates (and
 * frees) a small device array.  Errors: MLT_EINVAL (null tflops, iters
 * outside [1, 2^30]), MLT_ENOMEM, MLT_ECUDA.
 */
int mlt_fp64_rate(int64_t iters, double* tflops, void* stream);

/*
 * Kernel timing (instrumentation; the paper has no counterpart).  Between
 * mlt_profile_start() and mlt_profile_stop() every kernel the library launches
 * is bracketed by a pair of CUDA events recorded on the stream it runs on.
 * mlt_profile_stop waits for those events, disables timing and writes up to
 * max_stats per-kernel totals (launch count, summed event time in ms) into
 * stats (host array), the number written to *nstats.  Not thread-safe with
 * respect to concurrent library calls on other threads.
 */
typedef struct {
    char name[40];
    int64_t launches;
    double total_ms;
} mlt_kernel_stat;

int mlt_profile_start(void);
int mlt_profile_stop(mlt_kernel_stat* stats, int max_stats, int* nstats);

/* Message describing the calling thread's most recent failure ("" if none). */
const char* mlt_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* MLT_H */
