// lbm_step_noalloc: one fused lattice-Boltzmann step over caller-owned
// population buffers, for callers that cannot allocate device memory.
//
// The ensemble API owns its buffers and allocates them with cudaMalloc when an
// ensemble is created.  Some callers cannot do that: a host program whose
// device memory is owned by another allocator (a framework's memory pool, a
// fixed arena sized at start-up), or a real-time loop where an allocation's
// implicit device synchronisation is not acceptable.  This entry point takes
// the populations in and out as plain device pointers and keeps the only
// scratch the step needs - the per-warp drag partials and two small index
// tables - in a fixed device array that is part of the library image.
#include <cmath>
#include <cstdint>
#include <mutex>

#include "internal.h"
#include "lbm_device.cuh"

namespace lbm {

// Scratch of every lbm_step_noalloc call: clone index table, parity table and
// drag partials.  1 MiB, allocated once per device when the library's module
// is loaded there, held until the process exits.
constexpr size_t kNoAllocScratchBytes = size_t(1) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

static std::mutex g_noalloc_mutex;
static void* g_noalloc_ptr[64];  // device address of the scratch, per device id

__global__ void noalloc_tables_kernel(int32_t* list, int32_t* parity, int32_t n)
{
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        list[i] = i;
        parity[i] = 0;
    }
}

// drag of each clone: the warp partials of the obstacle ring summed in slot
// order in FP64, as the ensemble's own bookkeeping does
__global__ void noalloc_drag_kernel(const float* partials, int32_t n, int32_t n_slots, double* drag)
{
    const int c = blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= n) return;
    double acc = 0.0;
    for (int k = 0; k < n_slots; ++k) acc += (double)partials[(int64_t)c * n_slots + k];
    drag[c] = acc;
}

}  // namespace lbm

using namespace lbm;

extern "C" int lbm_step_noalloc(const lbm_config* cfg, int32_t n_clones, const void* f_in_dev, void* f_out_dev,
                                double* drag_dev, void* stream)
{
    if (!cfg || !f_in_dev || !f_out_dev || !drag_dev) return fail(LBM_ERR_ARG, "lbm_step_noalloc: null argument");
    // the step moves populations in 16-byte vectors and writes the drag as doubles
    if (reinterpret_cast<uintptr_t>(f_in_dev) % 16 != 0 || reinterpret_cast<uintptr_t>(f_out_dev) % 16 != 0)
        return fail(LBM_ERR_ARG, "lbm_step_noalloc: population buffers must be 16-byte aligned");
    if (reinterpret_cast<uintptr_t>(drag_dev) % 8 != 0)
        return fail(LBM_ERR_ARG, "lbm_step_noalloc: drag_dev must be 8-byte aligned");
    const lbm_config c = *cfg;
    if (c.nx < 8 || c.nx % 8 != 0) return fail(LBM_ERR_ARG, "lbm_step_noalloc: nx must be a positive multiple of 8");
    if (c.ny < 2) return fail(LBM_ERR_ARG, "lbm_step_noalloc: ny must be at least 2");
    if (n_clones < 1 || n_clones > 65535) return fail(LBM_ERR_ARG, "lbm_step_noalloc: clone count must be in [1, 65535]");
    if (!(c.tau > 0.5) || !std::isfinite(c.tau)) return fail(LBM_ERR_ARG, "lbm_step_noalloc: tau must exceed 1/2");
    if (!std::isfinite(c.gx) || !std::isfinite(c.gy)) return fail(LBM_ERR_ARG, "lbm_step_noalloc: force must be finite");
    if (c.storage < 0 || c.storage > 2) return fail(LBM_ERR_ARG, "lbm_step_noalloc: unknown storage");
    if (c.shift_exp < -20 || c.shift_exp > 20) return fail(LBM_ERR_ARG, "lbm_step_noalloc: shift_exp out of range");
    if (c.obs_w < 0 || c.obs_h < 0 || (c.obs_w > 0) != (c.obs_h > 0))
        return fail(LBM_ERR_ARG, "lbm_step_noalloc: obstacle size");
    if (c.obs_w > 0 && (c.obs_x0 < 1 || c.obs_x0 + c.obs_w > c.nx - 1 || c.obs_y0 < 0 || c.obs_y0 + c.obs_h > c.ny))
        return fail(LBM_ERR_ARG, "lbm_step_noalloc: obstacle outside the allowed region");
    if (f_in_dev == f_out_dev) return fail(LBM_ERR_ARG, "lbm_step_noalloc: input and output must differ");
    if (int rc = check_collision(c)) return rc;
    if (c.open_x != 0) return fail(LBM_ERR_ARG, "lbm_step_noalloc: open channels step through an ensemble only");
    if (int rc = check_open(c)) return rc;  // a periodic channel carries no grid or sponge
    const int32_t pitch = ((c.nx + 255) / 256) * 256;
    if ((int64_t)9 * pitch * c.ny >= ((int64_t)1 << 31))
        return fail(LBM_ERR_ARG, "lbm_step_noalloc: one clone must hold fewer than 2^31 population values");

    // the default variant of the fused step for this storage format
    const auto& vars = step_variants();
    const int want_vec = c.storage == kFP32 ? 4 : 8;
    int vi = -1;
    for (size_t i = 0; i < vars.size(); ++i)
        if (vars[i].storage == c.storage && vars[i].vec == want_vec && vars[i].warps == 4) vi = (int)i;
    if (vi < 0) return fail(LBM_ERR_STATE, "lbm_step_noalloc: no compiled step variant for this storage");
    const StepVariant& v = vars[vi];

    // drag ring of the obstacle in units of this variant's row segments
    int ry0 = 0, ry1 = -1, rs0 = 0, rs1 = -1, n_slots = 0;
    if (c.obs_w > 0) {
        const int seg_w = 32 * v.vec;
        ry0 = c.obs_y0 - 1 < 0 ? 0 : c.obs_y0 - 1;
        ry1 = c.obs_y0 + c.obs_h > c.ny - 1 ? c.ny - 1 : c.obs_y0 + c.obs_h;
        rs0 = (c.obs_x0 - 1) / seg_w;
        rs1 = (c.obs_x0 + c.obs_w) / seg_w;
        n_slots = (ry1 - ry0 + 1) * (rs1 - rs0 + 1);
    }
    const size_t table_bytes = ((size_t)n_clones * sizeof(int32_t) + 255) / 256 * 256;
    const size_t partial_bytes = (size_t)n_clones * (size_t)(n_slots > 0 ? n_slots : 1) * sizeof(float);
    if (2 * table_bytes + partial_bytes > kNoAllocScratchBytes)
        return fail(LBM_ERR_ARG, "lbm_step_noalloc: clones x drag slots need " +
                                     std::to_string(2 * table_bytes + partial_bytes) +
                                     " bytes of scratch; the fixed scratch holds 1048576");

    // once per device, with that device current: the scratch's device address
    int dev = 0;
    LBM_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(LBM_ERR_STATE, "lbm_step_noalloc: device index beyond 63");
    void* base = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_noalloc_mutex);
        if (!g_noalloc_ptr[dev]) {
            void* ptr = nullptr;
            cudaError_t err = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
            if (err != cudaSuccess) return cuda_fail(err, "cudaGetSymbolAddress(g_noalloc_scratch)");
            g_noalloc_ptr[dev] = ptr;
        }
        base = g_noalloc_ptr[dev];
    }
    int32_t* list = static_cast<int32_t*>(base);
    int32_t* parity = reinterpret_cast<int32_t*>(static_cast<char*>(base) + table_bytes);
    float* partials = reinterpret_cast<float*>(static_cast<char*>(base) + 2 * table_bytes);
    cudaStream_t s = static_cast<cudaStream_t>(stream);

    noalloc_tables_kernel<<<(n_clones + 255) / 256, 256, 0, s>>>(list, parity, n_clones);
    LBM_CUDA(cudaGetLastError());
    LBM_CUDA(cudaMemsetAsync(partials, 0, partial_bytes, s));

    StepParams p{};
    p.buf0 = const_cast<void*>(f_in_dev);
    p.buf1 = f_out_dev;
    p.parity = parity;
    p.clone_list = list;
    p.n_list = n_clones;
    p.nx = c.nx;
    p.ny = c.ny;
    p.pitch = pitch;
    p.plane = (int64_t)pitch * c.ny;
    p.clone_stride = 9 * p.plane;
    p.nseg = (c.nx + 32 * v.vec - 1) / (32 * v.vec);
    p.ox0 = c.obs_x0;
    p.ox1 = c.obs_w > 0 ? c.obs_x0 + c.obs_w : c.obs_x0;
    p.oy0 = c.obs_y0;
    p.oy1 = c.obs_w > 0 ? c.obs_y0 + c.obs_h : c.obs_y0;
    p.ry0 = ry0;
    p.ry1 = ry1;
    p.rs0 = rs0;
    p.rs1 = rs1;
    p.n_slots = n_slots > 0 ? n_slots : 1;
    p.batch_cap = 1;
    p.partials = partials;
    p.omega = (float)(1.0 / c.tau);
    p.gx = (float)c.gx;
    p.gy = (float)c.gy;
    p.bgk = bgk_consts(p.omega, p.gx, p.gy);
    p.coll = c.collision;
    p.cm = cm_consts(p.omega, (float)c.omega_bulk, (float)c.omega_3, (float)c.omega_4, p.gx, p.gy);
    const int sexp = c.storage == kFP32 ? 0 : c.shift_exp;
    p.scale = (float)std::ldexp(1.0, sexp);
    p.inv_scale = (float)std::ldexp(1.0, -sexp);
    p.step_in_batch = 0;
    LBM_CUDA(v.launch(p, s));
    noalloc_drag_kernel<<<(n_clones + 127) / 128, 128, 0, s>>>(partials, n_clones, n_slots, drag_dev);
    LBM_CUDA(cudaGetLastError());
    count_launches(3);
    return LBM_OK;
}
