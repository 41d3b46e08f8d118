// Observables of the square, recorded after every step when enabled (Sec. 2.1
// and Sec. 3.2): the pressures integrated over its upstream face (forebody)
// and downstream face (base), whose difference approximates the drag (eq.
// drag_approx), and the mean wall shear d u_x / d y along its top and bottom
// faces (eq. avg_shear_def).  On the lattice, from the post-collision state
// of the step:
//   p_fb   = cs2 * sum over rows [oy0, oy1) of rho(ox0 - 1, y),
//   p_base = cs2 * sum over rows [oy0, oy1) of rho(ox1, y),
//   gamma_top    = mean over x in [ox0, ox1) of (9 u(x, oy1) - u(x, oy1 + 1)) / 3,
//   gamma_bottom = mean over x in [ox0, ox1) of -(9 u(x, oy0 - 1) - u(x, oy0 - 2)) / 3,
// the one-sided second-order slope at the halfway wall from the fluid rows at
// distances 1/2 and 3/2, with rho u = sum c f - F/2 (the post-collision
// momentum carries the step's whole force).  FP64 sums in a fixed order.
#include <cmath>

#include "internal.h"
#include "lbm_device.cuh"

namespace lbm {
namespace {

constexpr int kObsThreads = 128;

__device__ double obs_block_sum(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
    for (int s = kObsThreads / 2; s > 0; s >>= 1) {
        if ((int)threadIdx.x < s) sh[threadIdx.x] += sh[threadIdx.x + s];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

// density and velocity of node (x, y) of a post-collision state
template <int S>
__device__ void node_macro(const typename Codec<S>::T* st, int64_t plane, int32_t pitch, int x, int y, float inv_scale,
                           double hgx, double& rho, double& ux)
{
    const typename Codec<S>::T* cell = st + (int64_t)y * pitch + x;
    double drho = 0.0, jx = 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const double g = (double)Codec<S>::dec(cell[q * plane], wf(q), inv_scale);
        drho += g;
        jx += cx(q) * g;
    }
    rho = 1.0 + drho;
    ux = (jx - hgx) / rho;
}

template <int S>
__global__ void __launch_bounds__(kObsThreads)
observables_kernel(const void* buf0, const void* buf1, const int32_t* parity, const int32_t* list, int32_t step,
                   int64_t clone_stride, int64_t plane, int32_t pitch, int32_t ox0, int32_t ox1, int32_t oy0,
                   int32_t oy1, double hgx, float inv_scale, const int32_t* t, double* obs, int32_t max_steps)
{
    using T = typename Codec<S>::T;
    __shared__ double sh[kObsThreads];
    const int c = list[blockIdx.x];
    const int cur = parity[c] ^ (step & 1);
    const T* st = static_cast<const T*>(cur ? buf0 : buf1) + (int64_t)c * clone_stride;  // this step's state
    constexpr double kCs2 = 1.0 / 3.0;
    double pfb = 0.0, pbase = 0.0, gt = 0.0, gb = 0.0;
    double rho, u1, u2;
    for (int y = oy0 + threadIdx.x; y < oy1; y += kObsThreads) {
        node_macro<S>(st, plane, pitch, ox0 - 1, y, inv_scale, hgx, rho, u1);
        pfb += kCs2 * rho;
        node_macro<S>(st, plane, pitch, ox1, y, inv_scale, hgx, rho, u1);
        pbase += kCs2 * rho;
    }
    for (int x = ox0 + threadIdx.x; x < ox1; x += kObsThreads) {
        node_macro<S>(st, plane, pitch, x, oy1, inv_scale, hgx, rho, u1);
        node_macro<S>(st, plane, pitch, x, oy1 + 1, inv_scale, hgx, rho, u2);
        gt += (9.0 * u1 - u2) / 3.0;
        node_macro<S>(st, plane, pitch, x, oy0 - 1, inv_scale, hgx, rho, u1);
        node_macro<S>(st, plane, pitch, x, oy0 - 2, inv_scale, hgx, rho, u2);
        gb -= (9.0 * u1 - u2) / 3.0;
    }
    pfb = obs_block_sum(pfb, sh);
    pbase = obs_block_sum(pbase, sh);
    gt = obs_block_sum(gt, sh);
    gb = obs_block_sum(gb, sh);
    if (threadIdx.x == 0) {
        double* o = obs + ((int64_t)c * max_steps + t[c] + step) * 4;
        o[0] = pfb;
        o[1] = pbase;
        o[2] = gt / (ox1 - ox0);
        o[3] = gb / (ox1 - ox0);
    }
}

}  // namespace

int observables_launch(lbm_ensemble* e, const int32_t* list_dev, int32_t n_list, int32_t step, cudaStream_t s)
{
    const lbm_config& c = e->cfg;
    const int ox0 = c.obs_x0, ox1 = c.obs_x0 + c.obs_w, oy0 = c.obs_y0, oy1 = c.obs_y0 + c.obs_h;
    const double hgx = 0.5 * c.gx;
    switch (c.storage) {
    case kFP32:
        observables_kernel<kFP32><<<n_list, kObsThreads, 0, s>>>(e->buf[0], e->buf[1], e->parity_dev, list_dev, step,
                                                                 e->clone_stride, e->plane, e->pitch, ox0, ox1, oy0,
                                                                 oy1, hgx, e->inv_scale, e->t_dev, e->obs,
                                                                 c.max_steps);
        break;
    case kFP16:
        observables_kernel<kFP16><<<n_list, kObsThreads, 0, s>>>(e->buf[0], e->buf[1], e->parity_dev, list_dev, step,
                                                                 e->clone_stride, e->plane, e->pitch, ox0, ox1, oy0,
                                                                 oy1, hgx, e->inv_scale, e->t_dev, e->obs,
                                                                 c.max_steps);
        break;
    default:
        observables_kernel<kBF16><<<n_list, kObsThreads, 0, s>>>(e->buf[0], e->buf[1], e->parity_dev, list_dev, step,
                                                                 e->clone_stride, e->plane, e->pitch, ox0, ox1, oy0,
                                                                 oy1, hgx, e->inv_scale, e->t_dev, e->obs,
                                                                 c.max_steps);
    }
    return cudaGetLastError() == cudaSuccess ? LBM_OK : LBM_ERR_CUDA;
}

}  // namespace lbm

using namespace lbm;

extern "C" {

int lbm_ensemble_set_observables(lbm_ensemble* e, int32_t enable)
{
    if (!e) return fail(LBM_ERR_ARG, "null ensemble");
    const lbm_config& c = e->cfg;
    if (enable) {
        if (c.obs_w <= 0 || c.obs_x0 < 1 || c.obs_x0 + c.obs_w > c.nx - 1 || c.obs_y0 < 2 ||
            c.obs_y0 + c.obs_h > c.ny - 2)
            return fail(LBM_ERR_ARG, "observables need a square with two fluid rows above and below it and a "
                                     "fluid column on either side");
        if (!e->obs) {
            const size_t bytes = sizeof(double) * 4 * (size_t)e->n * c.max_steps;
            LBM_CUDA(cudaMalloc((void**)&e->obs, bytes));
            LBM_CUDA(cudaMemsetAsync(e->obs, 0, bytes, e->stream));
        }
    }
    if ((enable != 0) != e->observe) {  // the captured step chunks change
        for (auto& g : e->graphs) cudaGraphExecDestroy(g.exec);
        e->graphs.clear();
    }
    e->observe = enable != 0;
    return LBM_OK;
}

int lbm_ensemble_observables(lbm_ensemble* e, int32_t t0, int32_t t1, double* dst, int32_t dst_on_device)
{
    if (!e || !dst) return fail(LBM_ERR_ARG, "null argument");
    if (!e->obs) return fail(LBM_ERR_STATE, "observables were never enabled");
    if (t0 < 0 || t1 < t0 || t1 > e->cfg.max_steps) return fail(LBM_ERR_ARG, "need 0 <= t0 <= t1 <= max_steps");
    const size_t row = sizeof(double) * 4 * (size_t)(t1 - t0);
    if (row == 0) return LBM_OK;
    const cudaMemcpyKind kind = dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
    LBM_CUDA(cudaMemcpy2DAsync(dst, row, e->obs + (size_t)t0 * 4, sizeof(double) * 4 * (size_t)e->cfg.max_steps, row,
                               e->n, kind, e->stream));
    if (!dst_on_device) LBM_CUDA(cudaStreamSynchronize(e->stream));
    return LBM_OK;
}

}  // extern "C"
