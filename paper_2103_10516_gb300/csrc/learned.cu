// C ABI of the learned coarse level: the network handle, its training and
// inference, and the three-level estimator E[d S] + E[P_l1 - d S] + E[P_n - P_l1]
// (each term an independent sample mean, as in Eq. multiEstimator).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "mlt_internal.h"
#include "rng.cuh"

struct mlt_surrogate {
    int device = 0;
    mlt::MlpDev D;
    void* mem = nullptr;
    mlt::DevBuf ws_x, ws_t, ws_y, ws_part, ws_mu, ws_c, ws_loss, ws_norm;
    int64_t step = 0;
    // standardisation of the learned level (set by mlt_learned_train): feature k
    // enters as (mu_k/d - mean_k)/std_k, the network predicts (P_l1/d - tmean)/tstd
    bool has_norm = false;
    double norm[2 * mlt::MLP_IN + 2] = {};
};

namespace mlt {
namespace {

// X[i][k] = mu[i][k] / d (k < 16); T[i] = sum_{j <= l1} c_j mu[i][j] / d; with
// `norm` (means, then standard deviations of the 16 features, then of the
// target) both are standardised, in double precision, before the rounding.
__global__ void features_kernel(const double* __restrict__ mu, int64_t ld, int64_t n, double inv_d,
                                const double* __restrict__ c, int l1, const double* __restrict__ norm,
                                float* __restrict__ X, float* __restrict__ T)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const double* row = mu + i * ld;
        for (int k = 0; k < MLP_IN; ++k) {
            double v = row[k] * inv_d;
            if (norm) v = (v - norm[k]) / norm[MLP_IN + k];
            X[i * MLP_IN + k] = (float)v;
        }
        if (T) {
            double s = 0.0;
            for (int j = 0; j <= l1; ++j) s += c[j] * row[j];
            double v = s * inv_d;
            if (norm) v = (v - norm[2 * MLP_IN]) / norm[2 * MLP_IN + 1];
            T[i] = (float)v;
        }
    }
}

bool is_dev(const void* p)
{
    if (!p) return false;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// Device copy of a caller array (host or device) in a scratch buffer.
int stage(DevBuf& buf, const void* src, size_t bytes, cudaStream_t s, const void** out)
{
    if (is_dev(src)) {
        *out = src;
        return MLT_OK;
    }
    int rc = buf.ensure(bytes, s);
    if (rc) return rc;
    MLT_CUDA_TRY(cudaMemcpyAsync(buf.p, src, bytes, cudaMemcpyHostToDevice, s));
    *out = buf.p;
    return MLT_OK;
}

int ensure_part(mlt_surrogate* S, int64_t n, cudaStream_t s)
{
    const int64_t tiles = (n + 127) / 128;
    int rc = S->ws_part.ensure((size_t)tiles * (MLP_NPARAMS + 1) * sizeof(float), s);
    if (rc) return rc;
    S->D.part = S->ws_part.as<float>();
    S->D.part_tiles = tiles;
    return MLT_OK;
}

int check_err(mlt_surrogate* S, cudaStream_t s)
{
    int h = 0;
    MLT_CUDA_TRY(cudaMemcpyAsync(&h, S->D.err, sizeof(int), cudaMemcpyDeviceToHost, s));
    MLT_CUDA_TRY(cudaStreamSynchronize(s));
    if (h) {
        MLT_CUDA_TRY(cudaMemsetAsync(S->D.err, 0, sizeof(int), s));
        return fail(MLT_ETIMEOUT, "a tensor-core wait in the network kernel gave up");
    }
    return MLT_OK;
}

// N(0, 1) draws by Box-Muller on the SplitMix64 finaliser of a counter.
double normal_draw(uint64_t seed, uint64_t k)
{
    const double two_pi = 6.283185307179586476925286766559;
    const uint64_t a = splitmix_finalise(seed * kGolden + 2 * k + 1);
    const uint64_t b = splitmix_finalise(seed * kGolden + 2 * k + 2);
    const double u1 = ((double)(a >> 11) + 1.0) * (1.0 / 9007199254740992.0);
    const double u2 = (double)(b >> 11) * (1.0 / 9007199254740992.0);
    return std::sqrt(-2.0 * std::log(u1)) * std::cos(two_pi * u2);
}

}  // namespace
}  // namespace mlt

using namespace mlt;

extern "C" {

int mlt_surrogate_create(uint64_t seed, mlt_surrogate** out)
{
    try {
        if (!out) return fail(MLT_EINVAL, "mlt_surrogate_create: null output");
        *out = nullptr;
        mlt_surrogate* S = new (std::nothrow) mlt_surrogate();
        if (!S) return fail(MLT_ENOMEM, "mlt_surrogate_create: host allocation failed");
        MLT_CUDA_TRY(cudaGetDevice(&S->device));
        const size_t nf = (size_t)MLP_NPARAMS;
        const size_t bytes = 4 * nf * sizeof(float) + 3 * (size_t)MLP_HID * MLP_HID * sizeof(__nv_bfloat16) +
                             2 * sizeof(double) + 256;
        char* mem = nullptr;
        if (cudaMalloc((void**)&mem, bytes) != cudaSuccess) {
            cudaGetLastError();
            delete S;
            return fail(MLT_ENOMEM, "mlt_surrogate_create: cudaMalloc failed");
        }
        S->mem = mem;
        cudaMemset(mem, 0, bytes);
        S->D.P = reinterpret_cast<float*>(mem);
        S->D.G = S->D.P + nf;
        S->D.M = S->D.G + nf;
        S->D.V = S->D.M + nf;
        S->D.W1b = reinterpret_cast<__nv_bfloat16*>(S->D.V + nf);
        S->D.W2b = S->D.W1b + MLP_HID * MLP_HID;   // W1b uses 128*16 of its 128*128 slot
        S->D.W2Tb = S->D.W2b + MLP_HID * MLP_HID;
        S->D.loss = reinterpret_cast<double*>(reinterpret_cast<char*>(mem) + ((4 * nf * sizeof(float) +
                        3 * (size_t)MLP_HID * MLP_HID * sizeof(__nv_bfloat16) + 15) & ~(size_t)15));
        S->D.err = reinterpret_cast<int*>(S->D.loss + 1);
        std::vector<float> P(nf, 0.0f);
        uint64_t k = 0;
        for (int i = 0; i < MLP_HID * MLP_IN; ++i)
            P[MLP_OFF_W1 + i] = (float)(normal_draw(seed, k++) * std::sqrt(2.0 / MLP_IN));
        for (int i = 0; i < MLP_HID * MLP_HID; ++i)
            P[MLP_OFF_W2 + i] = (float)(normal_draw(seed, k++) * std::sqrt(2.0 / MLP_HID));
        for (int i = 0; i < MLP_HID; ++i) P[MLP_OFF_W3 + i] = (float)(normal_draw(seed, k++) * std::sqrt(1.0 / MLP_HID));
        *out = S;
        return mlt_surrogate_set_params(S, P.data());
    } catch (...) {
        return fail(MLT_ENOMEM, "mlt_surrogate_create: exception");
    }
}

int mlt_surrogate_destroy(mlt_surrogate* S)
{
    if (!S) return MLT_OK;
    cudaDeviceSynchronize();
    DevBuf* bufs[] = {&S->ws_x, &S->ws_t, &S->ws_y, &S->ws_part, &S->ws_mu, &S->ws_c, &S->ws_loss, &S->ws_norm};
    for (auto* b : bufs) b->release();
    if (S->mem) cudaFree(S->mem);
    delete S;
    return MLT_OK;
}

int mlt_surrogate_set_params(mlt_surrogate* S, const float* params)
{
    if (!S || !params) return fail(MLT_EINVAL, "mlt_surrogate_set_params: null argument");
    MLT_CUDA_TRY(cudaMemcpy(S->D.P, params, MLP_NPARAMS * sizeof(float), cudaMemcpyHostToDevice));
    MLT_CUDA_TRY(cudaMemset(S->D.M, 0, 2 * MLP_NPARAMS * sizeof(float)));
    S->step = 0;
    int rc = mlp_adam(S->D, 0.0f, 0, 0, (cudaStream_t)0);   // refresh the BF16 copies
    if (rc) return rc;
    MLT_CUDA_TRY(cudaDeviceSynchronize());
    return MLT_OK;
}

int mlt_surrogate_get_params(mlt_surrogate* S, float* params)
{
    if (!S || !params) return fail(MLT_EINVAL, "mlt_surrogate_get_params: null argument");
    MLT_CUDA_TRY(cudaMemcpy(params, S->D.P, MLP_NPARAMS * sizeof(float), cudaMemcpyDeviceToHost));
    return MLT_OK;
}

int mlt_surrogate_get_norm(mlt_surrogate* S, double* norm, int* has_norm)
{
    if (!S || !norm || !has_norm) return fail(MLT_EINVAL, "mlt_surrogate_get_norm: null argument");
    std::memcpy(norm, S->norm, sizeof(S->norm));
    *has_norm = S->has_norm ? 1 : 0;
    return MLT_OK;
}

int mlt_surrogate_loss_grad(mlt_surrogate* S, const float* x, const float* t, int64_t n, double* loss,
                            float* grad, void* stream)
{
    try {
        if (!S || !x || !t || n < 1) return fail(MLT_EINVAL, "mlt_surrogate_loss_grad: bad argument");
        cudaStream_t s = (cudaStream_t)stream;
        const void *dx, *dt;
        int rc;
        if ((rc = stage(S->ws_x, x, (size_t)n * MLP_IN * sizeof(float), s, &dx))) return rc;
        if ((rc = stage(S->ws_t, t, (size_t)n * sizeof(float), s, &dt))) return rc;
        if ((rc = ensure_part(S, n, s))) return rc;
        if ((rc = mlp_launch_tiles(S->D, (const float*)dx, (const float*)dt, n, (float)(1.0 / (double)n), 1,
                                   nullptr, S->D.err, s))) return rc;
        if ((rc = check_err(S, s))) return rc;
        double hl = 0.0;
        MLT_CUDA_TRY(cudaMemcpyAsync(&hl, S->D.loss, sizeof(double), cudaMemcpyDeviceToHost, s));
        if (grad) MLT_CUDA_TRY(cudaMemcpyAsync(grad, S->D.G, MLP_NPARAMS * sizeof(float), cudaMemcpyDeviceToHost, s));
        MLT_CUDA_TRY(cudaStreamSynchronize(s));
        if (loss) *loss = hl / (double)n;
        return MLT_OK;
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_surrogate_loss_grad: exception");
    }
}

int mlt_surrogate_train(mlt_surrogate* S, const float* x, const float* t, int64_t n, int epochs, int64_t batch,
                        double lr, double* final_loss, void* stream)
{
    try {
        if (!S || !x || !t || n < 1 || epochs < 0 || batch < 1 || !(lr >= 0.0))
            return fail(MLT_EINVAL, "mlt_surrogate_train: bad argument");
        cudaStream_t s = (cudaStream_t)stream;
        const void *dx, *dt;
        int rc;
        if ((rc = stage(S->ws_x, x, (size_t)n * MLP_IN * sizeof(float), s, &dx))) return rc;
        if ((rc = stage(S->ws_t, t, (size_t)n * sizeof(float), s, &dt))) return rc;
        const int64_t bs = std::min(batch, n);
        if ((rc = ensure_part(S, bs, s))) return rc;
        const int64_t nb = (n + bs - 1) / bs;
        if ((rc = S->ws_loss.ensure((size_t)nb * sizeof(double), s))) return rc;
        double* losses = S->ws_loss.as<double>();
        for (int e = 0; e < epochs; ++e) {
            for (int64_t b = 0; b < nb; ++b) {
                const int64_t off = b * bs;
                const int64_t cnt = std::min(bs, n - off);
                MlpDev D = S->D;
                D.loss = losses + b;
                if ((rc = mlp_launch_tiles(D, (const float*)dx + off * MLP_IN, (const float*)dt + off, cnt,
                                           (float)(1.0 / (double)cnt), 1, nullptr, S->D.err, s))) return rc;
                if ((rc = mlp_adam(S->D, (float)lr, ++S->step, 1, s))) return rc;
            }
        }
        if ((rc = check_err(S, s))) return rc;
        if (final_loss) {
            std::vector<double> hl(nb);
            MLT_CUDA_TRY(cudaMemcpyAsync(hl.data(), losses, nb * sizeof(double), cudaMemcpyDeviceToHost, s));
            MLT_CUDA_TRY(cudaStreamSynchronize(s));
            double sum = 0.0;
            for (double v : hl) sum += v;
            *final_loss = epochs > 0 ? sum / (double)n : std::nan("");
        }
        return MLT_OK;
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_surrogate_train: exception");
    }
}

int mlt_surrogate_predict(mlt_surrogate* S, const float* x, int64_t n, float* y, void* stream)
{
    try {
        if (!S || !x || !y || n < 0) return fail(MLT_EINVAL, "mlt_surrogate_predict: bad argument");
        if (n == 0) return MLT_OK;
        cudaStream_t s = (cudaStream_t)stream;
        const void* dx;
        int rc;
        if ((rc = stage(S->ws_x, x, (size_t)n * MLP_IN * sizeof(float), s, &dx))) return rc;
        float* dy = y;
        const bool ydev = is_dev(y);
        if (!ydev) {
            if ((rc = S->ws_y.ensure((size_t)n * sizeof(float), s))) return rc;
            dy = S->ws_y.as<float>();
        }
        if ((rc = ensure_part(S, 128, s))) return rc;
        if ((rc = mlp_launch_tiles(S->D, (const float*)dx, nullptr, n, 1.0f, 0, dy, S->D.err, s))) return rc;
        if ((rc = check_err(S, s))) return rc;
        if (!ydev) {
            MLT_CUDA_TRY(cudaMemcpyAsync(y, dy, (size_t)n * sizeof(float), cudaMemcpyDeviceToHost, s));
            MLT_CUDA_TRY(cudaStreamSynchronize(s));
        }
        return MLT_OK;
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_surrogate_predict: exception");
    }
}

int mlt_learned_train(mlt_matrix* m, mlt_surrogate* S, const mlt_learned_params* P, int64_t n_train,
                      int64_t train_offset, int epochs, int64_t batch, double lr, double* final_loss)
{
    try {
        if (!m || !S || !P || n_train < 1) return fail(MLT_EINVAL, "mlt_learned_train: bad argument");
        if (P->l1 < MLP_IN - 1 || P->l1 > P->n) return fail(MLT_EINVAL, "mlt_learned_train: need 15 <= l1 <= n");
        cudaStream_t s = (cudaStream_t)P->stream;
        std::vector<double> c(P->n + 1);
        int rc = cheb_coeffs_host(P->fn, P->fn_p, P->a, P->b, P->n, c.data());
        if (rc) return rc;
        const int64_t ld = P->l1 + 1;
        if ((rc = S->ws_mu.ensure((size_t)n_train * ld * sizeof(double), s))) return rc;
        if ((rc = S->ws_c.ensure((size_t)(P->n + 1) * sizeof(double), s))) return rc;
        if ((rc = S->ws_x.ensure((size_t)n_train * MLP_IN * sizeof(float), s))) return rc;
        if ((rc = S->ws_t.ensure((size_t)n_train * sizeof(float), s))) return rc;
        std::vector<int32_t> deg(n_train, P->l1);
        rc = mlt_moments(m, P->a, P->b, P->seed, train_offset, n_train, deg.data(), P->precision, 0,
                         S->ws_mu.as<double>(), ld, P->stream);
        if (rc) return rc;
        MLT_CUDA_TRY(cudaMemcpyAsync(S->ws_c.p, c.data(), (P->n + 1) * sizeof(double), cudaMemcpyHostToDevice, s));
        const int64_t d = m->dim();
        // standardisation from the training moments (host, double precision)
        {
            std::vector<double> hm((size_t)n_train * ld);
            MLT_CUDA_TRY(cudaMemcpyAsync(hm.data(), S->ws_mu.p, hm.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
            MLT_CUDA_TRY(cudaStreamSynchronize(s));
            const int nf = MLP_IN + 1;
            std::vector<double> sum(nf, 0.0), sq(nf, 0.0);
            for (int64_t i = 0; i < n_train; ++i) {
                const double* row = &hm[(size_t)i * ld];
                double t = 0.0;
                for (int j = 0; j <= P->l1; ++j) t += c[j] * row[j];
                for (int k = 0; k < nf; ++k) {
                    const double v = (k < MLP_IN ? row[k] : t) / (double)d;
                    sum[k] += v;
                }
            }
            for (int k = 0; k < nf; ++k) sum[k] /= (double)n_train;
            for (int64_t i = 0; i < n_train; ++i) {
                const double* row = &hm[(size_t)i * ld];
                double t = 0.0;
                for (int j = 0; j <= P->l1; ++j) t += c[j] * row[j];
                for (int k = 0; k < nf; ++k) {
                    const double v = (k < MLP_IN ? row[k] : t) / (double)d - sum[k];
                    sq[k] += v * v;
                }
            }
            for (int k = 0; k < nf; ++k) {
                const double sd = n_train > 1 ? std::sqrt(sq[k] / (double)(n_train - 1)) : 0.0;
                const double safe = sd > 1e-300 ? sd : 1.0;
                if (k < MLP_IN) {
                    S->norm[k] = sum[k];
                    S->norm[MLP_IN + k] = safe;
                } else {
                    S->norm[2 * MLP_IN] = sum[k];
                    S->norm[2 * MLP_IN + 1] = safe;
                }
            }
            S->has_norm = true;
            if ((rc = S->ws_norm.ensure(sizeof(S->norm), s))) return rc;
            MLT_CUDA_TRY(cudaMemcpyAsync(S->ws_norm.p, S->norm, sizeof(S->norm), cudaMemcpyHostToDevice, s));
        }
        {
            ProfScope ps("learned_features", s);
            features_kernel<<<(unsigned)std::min<int64_t>((n_train + 255) / 256, 4096), 256, 0, s>>>(
                S->ws_mu.as<double>(), ld, n_train, 1.0 / (double)d, S->ws_c.as<double>(), P->l1,
                S->ws_norm.as<double>(), S->ws_x.as<float>(), S->ws_t.as<float>());
        }
        return mlt_surrogate_train(S, S->ws_x.as<float>(), S->ws_t.as<float>(), n_train, epochs, batch, lr,
                                   final_loss, P->stream);
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_learned_train: exception");
    }
}

int mlt_learned_estimate(mlt_matrix* m, mlt_surrogate* S, const mlt_learned_params* P, mlt_mlmc_result* R)
{
    try {
        if (!m || !S || !P || !R) return fail(MLT_EINVAL, "mlt_learned_estimate: null argument");
        if (P->l1 < MLP_IN - 1 || P->l1 > P->n) return fail(MLT_EINVAL, "mlt_learned_estimate: need 15 <= l1 <= n");
        if (P->m_net < 2 || P->m_1 < 2 || P->m_2 < 0 || (P->l1 < P->n && P->m_2 < 2))
            return fail(MLT_EINVAL, "mlt_learned_estimate: every level needs at least 2 samples");
        cudaStream_t s = (cudaStream_t)P->stream;
        const int n = P->n;
        std::vector<double> c(n + 1);
        int rc = cheb_coeffs_host(P->fn, P->fn_p, P->a, P->b, n, c.data());
        if (rc) return rc;
        const int64_t m2 = P->l1 < n ? P->m_2 : 0;
        const int64_t total = P->m_net + P->m_1 + m2;
        std::vector<int32_t> deg(total);
        for (int64_t i = 0; i < total; ++i)
            deg[i] = i < P->m_net ? MLP_IN - 1 : (i < P->m_net + P->m_1 ? P->l1 : n);
        const int64_t ld = n + 1;
        if ((rc = S->ws_mu.ensure((size_t)total * ld * sizeof(double), s))) return rc;
        rc = mlt_moments(m, P->a, P->b, P->seed, P->probe_offset, total, deg.data(), P->precision, 0,
                         S->ws_mu.as<double>(), ld, P->stream);
        if (rc) return rc;
        // network on the probes of the first two levels
        const int64_t nn = P->m_net + P->m_1;
        if ((rc = S->ws_x.ensure((size_t)nn * MLP_IN * sizeof(float), s))) return rc;
        if ((rc = S->ws_y.ensure((size_t)nn * sizeof(float), s))) return rc;
        const int64_t d = m->dim();
        {
            ProfScope ps("learned_features", s);
            features_kernel<<<(unsigned)std::min<int64_t>((nn + 255) / 256, 4096), 256, 0, s>>>(
                S->ws_mu.as<double>(), ld, nn, 1.0 / (double)d, nullptr, 0,
                S->has_norm ? S->ws_norm.as<double>() : nullptr, S->ws_x.as<float>(), nullptr);
        }
        MLT_CUDA_TRY(cudaGetLastError());
        if ((rc = ensure_part(S, 128, s))) return rc;
        if ((rc = mlp_launch_tiles(S->D, S->ws_x.as<float>(), nullptr, nn, 1.0f, 0, S->ws_y.as<float>(),
                                   S->D.err, s))) return rc;
        if ((rc = check_err(S, s))) return rc;
        std::vector<double> mu((size_t)total * ld);
        std::vector<float> y(nn);
        MLT_CUDA_TRY(cudaMemcpyAsync(mu.data(), S->ws_mu.p, mu.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        MLT_CUDA_TRY(cudaMemcpyAsync(y.data(), S->ws_y.p, nn * sizeof(float), cudaMemcpyDeviceToHost, s));
        MLT_CUDA_TRY(cudaStreamSynchronize(s));
        auto band = [&](const double* row, int lo, int hi) {
            double acc = 0.0;
            for (int j = lo + 1; j <= hi; ++j) acc += c[j] * row[j];
            return acc;
        };
        // the network's estimate of P_l1: d (tmean + tstd y), or d y without standardisation
        auto net = [&](int64_t i) {
            const double v = S->has_norm ? S->norm[2 * MLP_IN] + S->norm[2 * MLP_IN + 1] * (double)y[i] : (double)y[i];
            return (double)d * v;
        };
        std::vector<std::vector<double>> lv(3);
        for (int64_t i = 0; i < total; ++i) {
            const double* row = &mu[(size_t)i * ld];
            if (i < P->m_net) {
                lv[0].push_back(net(i));
            } else if (i < nn) {
                lv[1].push_back(band(row, -1, P->l1) - net(i));
            } else {
                lv[2].push_back(band(row, P->l1, n));
            }
        }
        std::memset(R, 0, sizeof(*R));
        const int L = m2 > 0 ? 3 : 2;
        const int lab[3] = {MLP_IN - 1, P->l1, n};
        double est = 0.0, var_sum = 0.0;
        for (int k = 0; k < L; ++k) {
            const auto& v = lv[k];
            double mean = 0.0;
            for (double x : v) mean += x;
            mean /= (double)v.size();
            double ss = 0.0;
            for (double x : v) ss += (x - mean) * (x - mean);
            const double var = ss / (double)(v.size() - 1);
            R->levels[k] = lab[k];
            R->m[k] = (int64_t)v.size();
            R->level_mean[k] = mean;
            R->level_var[k] = var;
            est += mean;
            var_sum += var / (double)v.size();
        }
        R->nlevels = L;
        R->estimate = est;
        R->std_error = std::sqrt(var_sum);
        R->probes = total;
        R->matvecs = P->m_net * (MLP_IN / 2) + P->m_1 * ((P->l1 + 1) / 2) + m2 * ((n + 1) / 2);
        return MLT_OK;
    } catch (...) {
        return fail(MLT_ECUDA, "mlt_learned_estimate: exception");
    }
}

}  // extern "C"
