// The learned score inside the rare-event algorithms.
//   - a CNN attached to an ensemble is evaluated on every stepped clone at each
//     checkpoint, giving a score series at checkpoint resolution (the AMS score
//     of App. B.1 replaced by the surrogate; the event stays judged on the drag);
//   - the same evaluation at the GKTL cloning times gives a potential V that
//     is added to the exponent as k A + kappa (V(t_i) - V(t_{i-1})) and removed
//     from the estimator weight, which leaves the estimator's target unchanged;
//   - a data set of (network input, future time-averaged drag) pairs is
//     recorded from an ensemble run.
#include <cmath>
#include <limits>
#include <vector>

#include "internal.h"
#include "lbm_device.cuh"

namespace lbm {

__global__ void scatter_score_kernel(const float* pred, const int32_t* list, int32_t n, double* out, int32_t stride,
                                     int32_t k)
{
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j < n) out[(int64_t)list[j] * stride + k] = (double)pred[j];
}

__global__ void fill_kernel(double* p, int64_t n, double v)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        p[i] = v;
}

// label of snapshot i of clone c: mean drag over (t_i, t_i + horizon]
__global__ void labels_kernel(const double* drag, int32_t max_steps, int32_t n, int32_t n_snaps, int32_t t0,
                              int32_t every, int32_t horizon, float* y)
{
    const int64_t idx = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (idx >= (int64_t)n * n_snaps) return;
    const int i = (int)(idx / n), c = (int)(idx - (int64_t)i * n);
    const int ti = t0 + i * every;
    double acc = 0.0;
    for (int t = ti + 1; t <= ti + horizon; ++t) acc += drag[(int64_t)c * max_steps + t - 1];
    y[idx] = (float)(acc / horizon);
}

int score_clones(lbm_ensemble* e, const int32_t* clones, int32_t n, double* out, int32_t stride, int32_t k)
{
    int32_t H = 0, W = 0, mb = 0;
    int rc = cnn_shape(e->cnn, &H, &W, &mb);
    if (rc) return rc;
    for (int32_t j0 = 0; j0 < n; j0 += mb) {
        const int32_t chunk = n - j0 < mb ? n - j0 : mb;
        LBM_CUDA(cudaMemcpyAsync(e->fields_list_dev, clones + j0, sizeof(int32_t) * chunk, cudaMemcpyHostToDevice,
                                 e->stream));
        if ((rc = fields_launch(e, e->fields_list_dev, chunk, e->cnn_factor, e->cnn_rho_scale, e->cnn_u_scale,
                                e->cnn_x)))
            return rc;
        if ((rc = cnn_forward(e->cnn, e->cnn_x, chunk, e->cnn_pred, e->stream))) return rc;
        scatter_score_kernel<<<(chunk + 127) / 128, 128, 0, e->stream>>>(e->cnn_pred, e->fields_list_dev, chunk, out,
                                                                         stride, k);
        LBM_CUDA(cudaGetLastError());
        count_launches(1);
        LBM_CUDA(cudaStreamSynchronize(e->stream));  // the host list chunk and the staging buffers are reused
    }
    return LBM_OK;
}

}  // namespace lbm

using namespace lbm;

extern "C" {

int lbm_ensemble_attach_score(lbm_ensemble* e, cnn_model* m, int32_t factor, float rho_scale, float u_scale)
{
    if (!e) return fail(LBM_ERR_ARG, "lbm_ensemble_attach_score: null ensemble");
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    void* old[] = {e->cnn_x, e->cnn_pred, e->cnn_score, e->pot[0], e->pot[1], e->pot[2], e->pot_tmp[0], e->pot_tmp[1]};
    for (void* p : old)
        if (p) cudaFree(p);
    e->cnn_x = nullptr;
    e->cnn_pred = nullptr;
    e->cnn_score = nullptr;
    for (auto& p : e->pot) p = nullptr;
    for (auto& p : e->pot_tmp) p = nullptr;
    e->cnn = nullptr;
    if (!m) return LBM_OK;
    int32_t H = 0, W = 0, mb = 0;
    int rc = cnn_shape(m, &H, &W, &mb);
    if (rc) return rc;
    if (factor < 1 || factor > e->cfg.nx || factor > e->cfg.ny || e->cfg.ny / factor != H || e->cfg.nx / factor != W)
        return fail(LBM_ERR_ARG, "lbm_ensemble_attach_score: the model's input size is not the downsampled channel");
    if (!std::isfinite(rho_scale) || !std::isfinite(u_scale)) return fail(LBM_ERR_ARG, "scales must be finite");
    cudaError_t err;
    if ((err = cudaMalloc(&e->cnn_x, sizeof(__nv_bfloat16) * (size_t)mb * H * W * 8)) != cudaSuccess)
        return cuda_fail(err, "cudaMalloc score input");
    if ((err = cudaMalloc((void**)&e->cnn_pred, sizeof(float) * mb)) != cudaSuccess)
        return cuda_fail(err, "cudaMalloc score output");
    const int64_t nk = e->n_ckpt > 0 ? (int64_t)e->n * e->n_ckpt : 1;
    if ((err = cudaMalloc((void**)&e->cnn_score, sizeof(double) * nk)) != cudaSuccess)
        return cuda_fail(err, "cudaMalloc score history");
    for (auto& p : e->pot)
        if ((err = cudaMalloc((void**)&p, sizeof(double) * e->n)) != cudaSuccess) return cuda_fail(err, "cudaMalloc potential");
    for (auto& p : e->pot_tmp)
        if ((err = cudaMalloc((void**)&p, sizeof(double) * e->n)) != cudaSuccess) return cuda_fail(err, "cudaMalloc potential");
    fill_kernel<<<64, 256, 0, e->stream>>>(e->cnn_score, nk, std::numeric_limits<double>::quiet_NaN());
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    e->cnn = m;
    e->cnn_factor = factor;
    e->cnn_rho_scale = rho_scale;
    e->cnn_u_scale = u_scale;
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    return LBM_OK;
}

int lbm_ensemble_score_history(lbm_ensemble* e, double* host)
{
    if (!e || !host) return fail(LBM_ERR_ARG, "lbm_ensemble_score_history: null argument");
    if (!e->cnn || e->n_ckpt < 1) return fail(LBM_ERR_STATE, "no learned score attached or no checkpoints");
    LBM_CUDA(cudaMemcpyAsync(host, e->cnn_score, sizeof(double) * (size_t)e->n * e->n_ckpt, cudaMemcpyDeviceToHost,
                             e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    return LBM_OK;
}

int lbm_ensemble_evaluate_score(lbm_ensemble* e, double* out_dev)
{
    if (!e || !out_dev) return fail(LBM_ERR_ARG, "lbm_ensemble_evaluate_score: null argument");
    if (!e->cnn) return fail(LBM_ERR_STATE, "no learned score attached");
    std::vector<int32_t> all(e->n);
    for (int i = 0; i < e->n; ++i) all[i] = i;
    return score_clones(e, all.data(), e->n, out_dev, 1, 0);
}

int lbm_surrogate_dataset(lbm_ensemble* e, int32_t n_snaps, int32_t every, int32_t horizon, int32_t factor,
                          float rho_scale, float u_scale, void* x_dev, float* y_dev, double* label_mean,
                          double* label_std)
{
    if (!e || !x_dev || !y_dev) return fail(LBM_ERR_ARG, "lbm_surrogate_dataset: null argument");
    if (n_snaps < 1 || every < 1 || horizon < 1) return fail(LBM_ERR_ARG, "lbm_surrogate_dataset: counts");
    if (factor < 1 || factor > e->cfg.nx || factor > e->cfg.ny)
        return fail(LBM_ERR_ARG, "lbm_surrogate_dataset: factor must be in [1, min(nx, ny)]");
    const int32_t t0 = e->t_host[0];
    for (int i = 1; i < e->n; ++i)
        if (e->t_host[i] != t0) return fail(LBM_ERR_STATE, "clones at different times");
    const int64_t total = (int64_t)t0 + (int64_t)(n_snaps - 1) * every + horizon;
    if (total > e->cfg.max_steps) return fail(LBM_ERR_ARG, "lbm_surrogate_dataset: exceeds max_steps");
    const int64_t per = (int64_t)(e->cfg.ny / factor) * (e->cfg.nx / factor) * 8;
    auto* x = static_cast<__nv_bfloat16*>(x_dev);
    int rc;
    for (int32_t i = 0; i < n_snaps; ++i) {
        if ((rc = fields_launch(e, e->all_dev, e->n, factor, rho_scale, u_scale, x + (int64_t)i * e->n * per))) return rc;
        if (i + 1 < n_snaps && (rc = lbm_ensemble_step(e, every))) return rc;
    }
    if ((rc = lbm_ensemble_step(e, horizon))) return rc;
    const int64_t ny = (int64_t)n_snaps * e->n;
    labels_kernel<<<(int)((ny + 255) / 256), 256, 0, e->stream>>>(e->drag, e->cfg.max_steps, e->n, n_snaps, t0, every,
                                                                   horizon, y_dev);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    // normalise the labels to zero mean and unit variance (FP64 on the host)
    std::vector<float> y(ny);
    LBM_CUDA(cudaMemcpyAsync(y.data(), y_dev, sizeof(float) * ny, cudaMemcpyDeviceToHost, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    double s = 0.0, s2 = 0.0;
    for (float v : y) {
        if (!std::isfinite(v)) return fail(LBM_ERR_NONFINITE, "lbm_surrogate_dataset: drag not finite");
        s += v;
    }
    const double mean = s / ny;
    for (float v : y) s2 += (v - mean) * (v - mean);
    const double sd = std::sqrt(s2 / ny);
    const double inv = sd > 0 ? 1.0 / sd : 1.0;
    for (auto& v : y) v = (float)((v - mean) * inv);
    LBM_CUDA(cudaMemcpyAsync(y_dev, y.data(), sizeof(float) * ny, cudaMemcpyHostToDevice, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    if (label_mean) *label_mean = mean;
    if (label_std) *label_std = sd;
    return LBM_OK;
}

}  // extern "C"
