// Direct-sampling statistics of the drag (Sec. 3): the autocorrelation of the
// drag fluctuations and its correlation time (caption of Fig. pdf_drag), and
// the waiting-time return time r(a) of a level.  The ensemble's clones are
// independent trajectories; their drag series over [t0, t1) are pooled.  FP64
// throughout, every sum in a fixed order (results do not depend on timing).
#include <cmath>
#include <limits>
#include <vector>

#include "internal.h"

namespace lbm {
namespace {

constexpr int kStatThreads = 256;

// fixed-order block sum of per-thread FP64 partials
__device__ double block_sum(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kStatThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// mean and variance of the pooled series (one block)
__global__ void drag_moments_kernel(const double* drag, int32_t max_steps, int32_t n, int32_t t0, int32_t len,
                                    double* mv)
{
    __shared__ double sh[kStatThreads];
    const int64_t total = (int64_t)n * len;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < total; i += kStatThreads) {
        const int64_t c = i / len, t = i - c * len;
        s += drag[c * max_steps + t0 + t];
    }
    const double mean = block_sum(s, sh) / (double)total;
    double q = 0.0;
    for (int64_t i = threadIdx.x; i < total; i += kStatThreads) {
        const int64_t c = i / len, t = i - c * len;
        const double x = drag[c * max_steps + t0 + t] - mean;
        q += x * x;
    }
    const double var = block_sum(q, sh) / (double)total;
    if (threadIdx.x == 0) {
        mv[0] = mean;
        mv[1] = var;
    }
}

// C(tau) for tau = blockIdx.x: mean over clones and t of x(t) x(t + tau) / var
__global__ void autocorr_kernel(const double* drag, int32_t max_steps, int32_t n, int32_t t0, int32_t len,
                                const double* mv, double* c)
{
    __shared__ double sh[kStatThreads];
    const int tau = blockIdx.x;
    const int m = len - tau;
    const double mean = mv[0];
    const int64_t total = (int64_t)n * m;
    double s = 0.0;
    for (int64_t i = threadIdx.x; i < total; i += kStatThreads) {
        const int64_t cl = i / m, t = i - cl * m;
        const double* row = drag + cl * max_steps + t0;
        s += (row[t] - mean) * (row[t + tau] - mean);
    }
    const double sum = block_sum(s, sh);
    if (threadIdx.x == 0) c[tau] = sum / (double)total / mv[1];
}

// events of level j in clone c: up-crossings to >= a, merged with an earlier
// one when the series was >= a within the last `gap` steps
__global__ void upcross_kernel(const double* drag, int32_t max_steps, int32_t n, int32_t t0, int32_t len,
                               const double* levels, int32_t n_levels, int32_t gap, long long* ev)
{
    const int id = blockIdx.x * blockDim.x + threadIdx.x;
    if (id >= n * n_levels) return;
    const int j = id / n, c = id - j * n;
    const double a = levels[j];
    const double* row = drag + (int64_t)c * max_steps + t0;
    long long count = 0;
    int last_above = -1;
    bool above_prev = false;
    for (int t = 0; t < len; ++t) {
        const bool above = row[t] >= a;
        if (above) {
            if (t > 0 && !above_prev && (last_above < 0 || t - last_above > gap)) ++count;
            last_above = t;
        }
        above_prev = above;
    }
    ev[id] = count;
}

int check_window(lbm_ensemble* e, int32_t t0, int32_t t1)
{
    if (t0 < 0 || t1 <= t0 || t1 > e->cfg.max_steps) return fail(LBM_ERR_ARG, "drag statistics: need 0 <= t0 < t1 <= max_steps");
    for (int i = 0; i < e->n; ++i)
        if (e->t_host[i] < t1) return fail(LBM_ERR_STATE, "drag statistics: a clone has not reached t1");
    return LBM_OK;
}

}  // namespace
}  // namespace lbm

using namespace lbm;

extern "C" {

int lbm_drag_autocorrelation(lbm_ensemble* e, int32_t t0, int32_t t1, int32_t max_lag, double* c_dev, int32_t* tau_c)
{
    if (!e || !c_dev) return fail(LBM_ERR_ARG, "lbm_drag_autocorrelation: null argument");
    if (int rc = check_window(e, t0, t1)) return rc;
    if (max_lag < 0 || max_lag >= t1 - t0) return fail(LBM_ERR_ARG, "lbm_drag_autocorrelation: need 0 <= max_lag < t1 - t0");
    double* mv = e->mass_dev;  // [N] x 3 doubles of scratch: two are enough
    drag_moments_kernel<<<1, kStatThreads, 0, e->stream>>>(e->drag, e->cfg.max_steps, e->n, t0, t1 - t0, mv);
    autocorr_kernel<<<max_lag + 1, kStatThreads, 0, e->stream>>>(e->drag, e->cfg.max_steps, e->n, t0, t1 - t0, mv,
                                                                  c_dev);
    LBM_CUDA(cudaGetLastError());
    count_launches(2);
    if (tau_c) {
        std::vector<double> c(max_lag + 1);
        LBM_CUDA(cudaMemcpyAsync(c.data(), c_dev, sizeof(double) * c.size(), cudaMemcpyDeviceToHost, e->stream));
        LBM_CUDA(cudaStreamSynchronize(e->stream));
        *tau_c = -1;
        for (int i = 0; i <= max_lag; ++i)
            if (c[i] <= 0.0) {
                *tau_c = i;
                break;
            }
    }
    return LBM_OK;
}

int lbm_drag_return_times(lbm_ensemble* e, int32_t t0, int32_t t1, int32_t n_levels, const double* levels_dev,
                          int32_t gap, int64_t* events, double* r)
{
    if (!e || !levels_dev || !events || !r) return fail(LBM_ERR_ARG, "lbm_drag_return_times: null argument");
    if (int rc = check_window(e, t0, t1)) return rc;
    if (n_levels < 1 || n_levels > 4096 || gap < 0) return fail(LBM_ERR_ARG, "lbm_drag_return_times: levels or gap");
    const int64_t m = (int64_t)e->n * n_levels;
    long long* ev = nullptr;
    LBM_CUDA(cudaMallocAsync((void**)&ev, sizeof(long long) * m, e->stream));
    upcross_kernel<<<(int)((m + 127) / 128), 128, 0, e->stream>>>(e->drag, e->cfg.max_steps, e->n, t0, t1 - t0,
                                                                   levels_dev, n_levels, gap, ev);
    cudaError_t err = cudaGetLastError();
    std::vector<long long> h(m);
    if (err == cudaSuccess)
        err = cudaMemcpyAsync(h.data(), ev, sizeof(long long) * m, cudaMemcpyDeviceToHost, e->stream);
    cudaFreeAsync(ev, e->stream);
    if (err == cudaSuccess) err = cudaStreamSynchronize(e->stream);
    if (err != cudaSuccess) return cuda_fail(err, "lbm_drag_return_times");
    count_launches(1);
    const double observed = (double)e->n * (double)(t1 - t0);
    for (int j = 0; j < n_levels; ++j) {
        long long s = 0;
        for (int c = 0; c < e->n; ++c) s += h[(int64_t)j * e->n + c];
        events[j] = s;
        r[j] = s > 0 ? observed / (double)s : std::numeric_limits<double>::infinity();
    }
    return LBM_OK;
}

}  // extern "C"
