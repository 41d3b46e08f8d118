// Selection steps of the two rare-event algorithms on the device: GKTL
// weights and resampling (App. C.1) and AMS kill/branch choice (App. B.1).
// One block each; the integer decisions are taken in one thread in a fixed
// order, so given the same weights or scores and the same seed they are the
// same on every run (and match any implementation of the same definition).
#include <cmath>

#include "internal.h"
#include "lbm_device.cuh"

namespace lbm {

constexpr int kSelThreads = 256;
constexpr int kMaxSel = 4096;

__global__ void gktl_weights_kernel(int32_t n, const double* s, double* W, double* logR)
{
    __shared__ double sh[kSelThreads];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    double m = -INFINITY;
    for (int i = threadIdx.x; i < n; i += kSelThreads) {
        const double v = s[i];
        if (!isfinite(v)) bad = 1;
        m = fmax(m, v);
    }
    sh[threadIdx.x] = m;
    __syncthreads();
    for (int off = kSelThreads / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + off]);
        __syncthreads();
    }
    m = sh[0];
    __syncthreads();
    if (bad) {
        for (int i = threadIdx.x; i < n; i += kSelThreads) W[i] = NAN;
        if (threadIdx.x == 0) *logR = NAN;
        return;
    }
    // S = sum_n e^{s_n - m}: strided partial sums, then a fixed tree
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += kSelThreads) acc += exp(s[i] - m);
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int off = kSelThreads / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    const double S = sh[0];
    for (int i = threadIdx.x; i < n; i += kSelThreads) W[i] = (double)n * exp(s[i] - m) / S;
    if (threadIdx.x == 0) *logR = m + log(S / (double)n);
}

// residual resampling with a systematic draw of the residuals
__global__ void gktl_select_kernel(int32_t n, const double* W, uint64_t seed, uint64_t iter, int32_t* parent,
                                   int32_t* status)
{
    __shared__ double sh[kSelThreads];
    __shared__ int cnt[kMaxSel];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    double acc = 0.0;
    for (int i = threadIdx.x; i < n; i += kSelThreads) {
        const double w = W[i];
        if (!isfinite(w) || w < 0.0) bad = 1;
        acc += w;
    }
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int off = kSelThreads / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    int code = 0;
    if (bad) code = LBM_ERR_NONFINITE;
    else if (fabs(sh[0] - (double)n) > 1e-9 * (double)n) code = LBM_ERR_ARG;
    if (code) {
        for (int i = threadIdx.x; i < n; i += kSelThreads) parent[i] = -1;
        if (threadIdx.x == 0 && status) *status = code;
        return;
    }
    if (threadIdx.x != 0) return;
    long long whole = 0;
    double csum = 0.0;
    for (int i = 0; i < n; ++i) {
        const double fl = floor(W[i]);
        cnt[i] = (int)fl;
        whole += cnt[i];
        csum += W[i] - fl;
    }
    const long long R = (long long)n - whole;
    if (R < 0 || (R > 0 && !(csum > 0.0))) {
        for (int i = 0; i < n; ++i) parent[i] = -1;
        if (status) *status = LBM_ERR_ARG;
        return;
    }
    if (R > 0) {
        const double U = unit_double(philox(kStreamGktl, iter, 0u, 0u, seed, 0u).v[0]);
        const double spacing = csum / (double)R;
        int i = 0;
        double edge = W[0] - floor(W[0]);
        for (long long k = 0; k < R; ++k) {
            const double point = (U + (double)k) * spacing;
            while (point >= edge && i < n - 1) {
                ++i;
                edge += W[i] - floor(W[i]);
            }
            cnt[i] += 1;
        }
    }
    for (int i = 0; i < n; ++i) parent[i] = cnt[i] >= 1 ? i : -1;
    int next_empty = 0;
    for (int i = 0; i < n; ++i)
        for (int c = 1; c < cnt[i]; ++c) {
            while (next_empty < n - 1 && parent[next_empty] != -1) ++next_empty;
            parent[next_empty] = i;
        }
    if (status) *status = 0;
}

__global__ void ams_select_kernel(int32_t n, const double* Q, uint64_t seed, uint64_t iter, int32_t* killed,
                                  int32_t* n_killed, int32_t* survivor, double* level)
{
    __shared__ double sh[kSelThreads];
    __shared__ int bad;
    if (threadIdx.x == 0) bad = 0;
    __syncthreads();
    double z = INFINITY;
    for (int i = threadIdx.x; i < n; i += kSelThreads) {
        const double q = Q[i];
        if (isnan(q)) bad = 1;
        z = fmin(z, q);
    }
    sh[threadIdx.x] = z;
    __syncthreads();
    for (int off = kSelThreads / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] = fmin(sh[threadIdx.x], sh[threadIdx.x + off]);
        __syncthreads();
    }
    if (threadIdx.x != 0) return;
    if (bad) {
        *n_killed = -1;
        *level = NAN;
        return;
    }
    z = sh[0];
    int nk = 0;
    for (int i = 0; i < n; ++i)
        if (Q[i] == z) killed[nk++] = i;
    *n_killed = nk;
    *level = z;
    if (nk == n) return;
    for (int k = 0; k < nk; ++k) {
        const uint64_t x = philox(kStreamAms, iter, (uint64_t)killed[k], 0u, seed, 0u).v[0];
        const long long r = (long long)index_below(x, (uint64_t)(n - nk));
        long long seen = 0;
        for (int i = 0; i < n; ++i) {
            if (Q[i] == z) continue;
            if (seen == r) {
                survivor[k] = i;
                break;
            }
            ++seen;
        }
    }
}

}  // namespace lbm

using namespace lbm;

extern "C" {

int gktl_weights(int32_t n, const double* s_dev, double* W_dev, double* logR_dev, void* stream)
{
    if (n < 1 || n > kMaxSel) return fail(LBM_ERR_ARG, "gktl_weights: n must be in [1, 4096]");
    if (!s_dev || !W_dev || !logR_dev) return fail(LBM_ERR_ARG, "gktl_weights: null pointer");
    gktl_weights_kernel<<<1, kSelThreads, 0, static_cast<cudaStream_t>(stream)>>>(n, s_dev, W_dev, logR_dev);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    return LBM_OK;
}

int gktl_select(int32_t n, const double* W_dev, uint64_t seed, uint64_t iter, int32_t* parent_dev, int32_t* status_dev,
                void* stream)
{
    if (n < 1 || n > kMaxSel) return fail(LBM_ERR_ARG, "gktl_select: n must be in [1, 4096]");
    if (!W_dev || !parent_dev) return fail(LBM_ERR_ARG, "gktl_select: null pointer");
    gktl_select_kernel<<<1, kSelThreads, 0, static_cast<cudaStream_t>(stream)>>>(n, W_dev, seed, iter, parent_dev,
                                                                                status_dev);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    return LBM_OK;
}

int ams_select(int32_t n, const double* Q_dev, uint64_t seed, uint64_t iter, int32_t* killed_dev, int32_t* n_killed_dev,
               int32_t* survivor_dev, double* level_dev, void* stream)
{
    if (n < 1 || n > kMaxSel) return fail(LBM_ERR_ARG, "ams_select: n must be in [1, 4096]");
    if (!Q_dev || !killed_dev || !n_killed_dev || !survivor_dev || !level_dev)
        return fail(LBM_ERR_ARG, "ams_select: null pointer");
    ams_select_kernel<<<1, kSelThreads, 0, static_cast<cudaStream_t>(stream)>>>(n, Q_dev, seed, iter, killed_dev,
                                                                               n_killed_dev, survivor_dev, level_dev);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    return LBM_OK;
}

}  // extern "C"
