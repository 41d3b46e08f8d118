// Ensemble runtime of liblbmrare: device memory, initial state, drag
// bookkeeping, deterministic reductions, GKTL cloning and AMS branching with
// the App. D perturbation, checkpoints, and the C ABI around them.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "internal.h"
#include "lbm_device.cuh"

namespace lbm {

static thread_local std::string g_error;
static std::atomic<int64_t> g_launches{0};

void count_launches(int64_t n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

void set_error(const std::string& msg) { g_error = msg; }
int fail(int code, const std::string& msg)
{
    g_error = msg;
    return code;
}
int cuda_fail(cudaError_t err, const char* what)
{
    g_error = std::string(what) + ": " + cudaGetErrorName(err) + " (" + cudaGetErrorString(err) + ")";
    return err == cudaErrorMemoryAllocation ? LBM_ERR_OOM : LBM_ERR_CUDA;
}

void register_step_fp32(std::vector<StepVariant>&);
void register_step_fp16(std::vector<StepVariant>&);
void register_step_bf16(std::vector<StepVariant>&);
void register_open_fp32(std::vector<StepVariant>&);
void register_open_fp16(std::vector<StepVariant>&);
void register_open_bf16(std::vector<StepVariant>&);

const std::vector<StepVariant>& step_variants()
{
    static const std::vector<StepVariant> table = [] {
        std::vector<StepVariant> v;
        register_step_fp32(v);
        register_step_fp16(v);
        register_step_bf16(v);
        register_open_fp32(v);
        register_open_fp16(v);
        register_open_bf16(v);
        return v;
    }();
    return table;
}

constexpr int kBatchCap = 512;     // steps per drag-finalisation batch
constexpr int kGraphCache = 24;    // cached step-chunk graphs per ensemble
// step calls over at most this many sites (n clones x nx x ny) use the
// small-list variant: one wave of the wide variants would leave most SMs idle
constexpr int64_t kSmallSites = int64_t(1) << 18;
constexpr int kRedBlocks = 152;    // blocks of a per-clone reduction (one wave)
constexpr int kRedThreads = 256;

static int elem_size(int storage) { return storage == kFP32 ? 4 : 2; }

// ---------------------------------------------------------------- kernels
template <int S>
__global__ void init_kernel(void* buf, int64_t clone_stride, int64_t plane, int32_t pitch, int32_t nx,
                            int32_t ny, int32_t n, Solids sol, uint64_t seed, double amp, double u_in, float scale)
{
    using T = typename Codec<S>::T;
    T* base = static_cast<T*>(buf);
    const int64_t sites = (int64_t)nx * ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sites * n; i += (int64_t)gridDim.x * blockDim.x) {
        const int c = (int)(i / sites);
        const int64_t site = i - (int64_t)c * sites;
        const int y = (int)(site / nx), x = (int)(site - (int64_t)y * nx);
        double ux = 0.0, uy = 0.0;
        if (!sol.at(x, y)) {
            const u64x4 r = philox(kStreamInit, (uint64_t)c, (uint64_t)site, 0u, seed, 0u);
            ux = amp * (2.0 * unit_double(r.v[0]) - 1.0);
            uy = amp * (2.0 * unit_double(r.v[1]) - 1.0);
            if (u_in != 0.0) {  // open channel: the inlet profile everywhere
                const double h = ny, yy = y + 0.5;
                ux += u_in * 4.0 * yy * (h - yy) / (h * h);
            }
        }
        const double usq = ux * ux + uy * uy;
        T* cell = base + (int64_t)c * clone_stride + (int64_t)y * pitch + x;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const double cu = cx(q) * ux + cy(q) * uy;
            // f^eq(rho = 1, u) - w_q (App. A); zero on solid nodes
            const double g = wd(q) * (3.0 * cu + 4.5 * cu * cu - 1.5 * usq);
            T v;
            if constexpr (S == kFP32)
                v = (float)(wd(q) + g);
            else
                v = Codec<S>::enc((float)g, 0.f, scale);
            cell[q * plane] = v;
        }
    }
}

// Sum the per-warp drag partials of each step in slot order (FP64), append to
// the drag history, then advance the clone's time and buffer parity.
__global__ void finalize_kernel(const float* partials, int32_t batch_cap, int32_t n_slots, int32_t used_slots,
                                const int32_t* list, int32_t n_steps, double* drag, int32_t max_steps,
                                int32_t* t, int32_t* parity, int32_t* flag)
{
    const int c = list[blockIdx.x];
    const int t0 = t[c];
    for (int s = threadIdx.x; s < n_steps; s += blockDim.x) {
        const float* pp = partials + ((int64_t)c * batch_cap + s) * n_slots;
        double acc = 0.0;
        for (int k = 0; k < used_slots; ++k) acc += (double)pp[k];
        if (!isfinite(acc)) *flag = 1;
        drag[(int64_t)c * max_steps + t0 + s] = acc;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        t[c] = t0 + n_steps;
        parity[c] ^= (n_steps & 1);
    }
}

// block-wide FP64 sum in a fixed order (tree over the shared array)
template <int THREADS>
__device__ double block_sum(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
#pragma unroll
    for (int off = THREADS / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

template <int THREADS>
__device__ double block_max(double v, double* sh)
{
    sh[threadIdx.x] = v;
    __syncthreads();
#pragma unroll
    for (int off = THREADS / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] = fmax(sh[threadIdx.x], sh[threadIdx.x + off]);
        __syncthreads();
    }
    const double r = sh[0];
    __syncthreads();
    return r;
}

__global__ void window_sum_kernel(const double* drag, int32_t max_steps, int32_t t0, int32_t t1, double k,
                                  double* out)
{
    __shared__ double sh[kRedThreads];
    const int c = blockIdx.x;
    double acc = 0.0;
    for (int t = t0 + (int)threadIdx.x; t < t1; t += kRedThreads) acc += drag[(int64_t)c * max_steps + t];
    const double s = block_sum<kRedThreads>(acc, sh);
    if (threadIdx.x == 0) out[c] = k * s;
}

// F(t) = (1/W) sum_{s=t-W+1}^{t} D(s); thread i owns a contiguous range of t,
// opens it with a direct sum and slides the window across it.
__global__ void scores_kernel(const double* drag, int32_t max_steps, int32_t window, int32_t t_begin, int32_t t_end,
                              double* scores, double* out_max)
{
    __shared__ double sh[kRedThreads];
    const int c = blockIdx.x;
    const double* d = drag + (int64_t)c * max_steps;  // d[t-1] = D(t)
    double* F = scores + (int64_t)c * max_steps;      // F[t-1] = F(t)
    const int first = t_begin + window, count = t_end - first + 1;
    double best = -INFINITY;
    if (count > 0) {
        const int chunk = (count + kRedThreads - 1) / kRedThreads;
        const int ta = first + (int)threadIdx.x * chunk;
        const int tb = min(ta + chunk - 1, t_end);
        if (ta <= tb) {
            double acc = 0.0;
            for (int s = ta - window + 1; s <= ta; ++s) acc += d[s - 1];
            for (int t = ta; t <= tb; ++t) {
                if (t > ta) acc += d[t - 1] - d[t - window - 1];
                const double m = acc / (double)window;
                F[t - 1] = m;
                best = fmax(best, m);
            }
        }
    }
    for (int t = t_begin + 1 + (int)threadIdx.x; t < min(first, t_end + 1); t += kRedThreads) F[t - 1] = -INFINITY;
    const double mx = block_max<kRedThreads>(best, sh);
    if (threadIdx.x == 0 && out_max) out_max[c] = mx;
}

__global__ void first_crossing_kernel(const double* F, int32_t t_lo, int32_t t_hi, double level, int32_t* out)
{
    __shared__ int sh[kRedThreads];
    int best = INT32_MAX;
    for (int t = t_lo + (int)threadIdx.x; t <= t_hi; t += kRedThreads)
        if (F[t - 1] > level) { best = t; break; }
    sh[threadIdx.x] = best;
    __syncthreads();
    for (int off = kRedThreads / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] = min(sh[threadIdx.x], sh[threadIdx.x + off]);
        __syncthreads();
    }
    if (threadIdx.x == 0) *out = sh[0] == INT32_MAX ? -1 : sh[0];
}

// Per-block FP64 partial sums of mass and momentum over the fluid nodes of
// each listed clone (the blocks of one clone cover its sites in a fixed way).
template <int S>
__global__ void moments_partial_kernel(const void* buf0, const void* buf1, const int32_t* parity, const int32_t* list,
                                       int64_t clone_stride, int64_t plane, int32_t pitch, int32_t nx, int32_t ny,
                                       Solids sol, float inv_scale, double* partial)
{
    using T = typename Codec<S>::T;
    __shared__ double sh[kRedThreads];
    const int li = blockIdx.y;
    const int c = list[li];
    const T* base = static_cast<const T*>(parity[c] ? buf1 : buf0) + (int64_t)c * clone_stride;
    const int64_t sites = (int64_t)nx * ny;
    double m = 0.0, px = 0.0, py = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < sites; i += (int64_t)gridDim.x * kRedThreads) {
        const int y = (int)(i / nx), x = (int)(i - (int64_t)y * nx);
        if (sol.at(x, y)) continue;
        const T* cell = base + (int64_t)y * pitch + x;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const double f = (double)wf(q) + (double)Codec<S>::dec(cell[q * plane], wf(q), inv_scale);
            m += f;
            px += cx(q) * f;
            py += cy(q) * f;
        }
    }
    const double sm = block_sum<kRedThreads>(m, sh);
    const double sx = block_sum<kRedThreads>(px, sh);
    const double sy = block_sum<kRedThreads>(py, sh);
    if (threadIdx.x == 0) {
        double* o = partial + ((int64_t)c * gridDim.x + blockIdx.x) * 3;
        o[0] = sm; o[1] = sx; o[2] = sy;
    }
}

__global__ void moments_final_kernel(const double* partial, int32_t nblocks, const int32_t* list, double* mass,
                                     double* px, double* py)
{
    const int c = list[blockIdx.x];
    if (threadIdx.x != 0) return;
    double m = 0, x = 0, y = 0;
    for (int b = 0; b < nblocks; ++b) {
        const double* o = partial + ((int64_t)c * nblocks + b) * 3;
        m += o[0]; x += o[1]; y += o[2];
    }
    mass[c] = m;
    if (px) px[c] = x;
    if (py) py[c] = y;
}

// fluid mass of every state in the snapshot bank (fixed-order FP64 partials)
template <int S>
__global__ void bank_mass_partial_kernel(const void* snaps, int64_t clone_stride, int64_t plane, int32_t pitch,
                                         int32_t nx, int32_t ny, Solids sol, float inv_scale, double* partial)
{
    using T = typename Codec<S>::T;
    __shared__ double sh[kRedThreads];
    const int k = blockIdx.y;
    const T* base = static_cast<const T*>(snaps) + (int64_t)k * clone_stride;
    const int64_t sites = (int64_t)nx * ny;
    double m = 0.0;
    for (int64_t i = blockIdx.x * (int64_t)kRedThreads + threadIdx.x; i < sites; i += (int64_t)gridDim.x * kRedThreads) {
        const int y = (int)(i / nx), x = (int)(i - (int64_t)y * nx);
        if (sol.at(x, y)) continue;
        const T* cell = base + (int64_t)y * pitch + x;
#pragma unroll
        for (int q = 0; q < 9; ++q) m += (double)wf(q) + (double)Codec<S>::dec(cell[q * plane], wf(q), inv_scale);
    }
    const double sm = block_sum<kRedThreads>(m, sh);
    if (threadIdx.x == 0) partial[(int64_t)k * gridDim.x + blockIdx.x] = sm;
}

__global__ void bank_mass_final_kernel(const double* partial, int32_t nblocks, double* snap_mass)
{
    if (threadIdx.x != 0) return;
    double m = 0.0;
    for (int b = 0; b < nblocks; ++b) m += partial[(int64_t)blockIdx.x * nblocks + b];
    snap_mass[blockIdx.x] = m;
}

// perturb_kernel's `inplace` value that perturbs every listed slot in place
constexpr int32_t kAllInPlace = -2;

// App. D: slot s with parent p != s (or s == inplace, or every listed slot
// with inplace == kAllInPlace) becomes
//   f_s = (f_p + eps sum_n alpha_n f^(n)) * M_p / (M_p + eps sum_n alpha_n M^(n))
// on fluid nodes, written in the shifted variable g = f - w.  alpha_n is the
// counter-based uniform in [0, 1) minus alpha_shift: 0 for the printed form,
// 1/2 for the centred coefficients (lbm_ensemble_set_perturbation).
template <int S>
__global__ void perturb_kernel(void* buf0, void* buf1, const int32_t* parity, const int32_t* parent, int32_t n_clones,
                               int32_t* flag, int32_t inplace, const int32_t* slots,
                               int64_t clone_stride, int64_t plane, int32_t pitch, int32_t nx, int32_t ny,
                               Solids sol, const void* snaps, int32_t n_s,
                               const double* snap_mass, const double* mass, double eps, uint64_t seed, uint64_t iter,
                               double alpha_shift, float scale, float inv_scale)
{
    using T = typename Codec<S>::T;
    const int s = slots ? slots[blockIdx.y] : (int)blockIdx.y;
    const int p = parent[s];
    if (p < 0 || p >= n_clones) {  // rejected selection: leave the slot alone
        if (threadIdx.x == 0) flag[0] = 1;
        return;
    }
    if (p == s && s != inplace && inplace != kAllInPlace) return;  // block-uniform
    __shared__ float alpha_eps[16];
    __shared__ float sc_m1[2];
    if (threadIdx.x == 0) {
        double lin = 0.0;
        for (int k = 0; k < n_s; ++k) {
            const u64x4 r = philox(kStreamPerturb, iter, (uint64_t)s, (uint64_t)k, seed, 0u);
            const double a = unit_double(r.v[0]) - alpha_shift;
            alpha_eps[k] = (float)(eps * a);
            lin += eps * a * snap_mass[k];
        }
        const double Mp = mass[p];
        const double scale_m = eps == 0.0 ? 1.0 : Mp / (Mp + lin);
        sc_m1[0] = (float)scale_m;
        sc_m1[1] = (float)(scale_m - 1.0);
    }
    __syncthreads();
    const float sm = sc_m1[0], sm1 = sc_m1[1];
    const T* from = static_cast<const T*>(parity[p] ? buf1 : buf0) + (int64_t)p * clone_stride;
    T* to = static_cast<T*>(parity[s] ? buf1 : buf0) + (int64_t)s * clone_stride;
    const T* sn = static_cast<const T*>(snaps);
    const int64_t sites = (int64_t)nx * ny;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < sites; i += (int64_t)gridDim.x * blockDim.x) {
        const int y = (int)(i / nx), x = (int)(i - (int64_t)y * nx);
        if (sol.at(x, y)) continue;  // solid: stays at rest
        const int64_t off = (int64_t)y * pitch + x;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float w = wf(q);
            const float g = Codec<S>::dec(from[q * plane + off], w, inv_scale);
            float add = 0.f;
            for (int k = 0; k < n_s; ++k)
                add += alpha_eps[k] * (w + Codec<S>::dec(sn[(int64_t)k * clone_stride + q * plane + off], w, inv_scale));
            // f_new - w = (g + add) * sm + w * (sm - 1)
            const float gn = (g + add) * sm + w * sm1;
            to[q * plane + off] = Codec<S>::enc(gn, w, scale);
        }
    }
}

__global__ void copy_history_kernel(double* drag, int32_t max_steps, const int32_t* parent, int32_t n_clones,
                                    int32_t n_hist)
{
    const int s = blockIdx.y;
    const int p = parent[s];
    if (p == s || p < 0 || p >= n_clones) return;
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < n_hist; t += gridDim.x * blockDim.x)
        drag[(int64_t)s * max_steps + t] = drag[(int64_t)p * max_steps + t];
}

}  // namespace lbm

using namespace lbm;

// ---------------------------------------------------------------- host helpers
namespace {

struct Ring {
    int ry0, ry1, rs0, rs1, n_slots;
};

}  // namespace

int lbm::check_collision(const lbm_config& c)
{
    if (c.collision != 0 && c.collision != 1) return fail(LBM_ERR_ARG, "collision must be 0 (BGK) or 1 (central moments)");
    if (c.collision == 1) {
        const double r[3] = {c.omega_bulk, c.omega_3, c.omega_4};
        for (double w : r)
            if (!(w > 0.0 && w < 2.0)) return fail(LBM_ERR_ARG, "central-moment rates must lie in (0, 2)");
    }
    return LBM_OK;
}

int lbm::check_open(const lbm_config& c)
{
    if (c.open_x == 0) {
        if (c.grid_w != 0 || c.sponge_len != 0)
            return fail(LBM_ERR_ARG, "the entrance grid and the sponge belong to an open channel (open_x = 1)");
        return LBM_OK;
    }
    if (c.open_x != 1) return fail(LBM_ERR_ARG, "open_x must be 0 or 1");
    if (c.gx != 0.0 || c.gy != 0.0) return fail(LBM_ERR_ARG, "an open channel has no body force (gx = gy = 0)");
    if (c.ny < 3) return fail(LBM_ERR_ARG, "an open channel needs ny >= 3");
    if (!(std::fabs(c.u_in) < 0.3)) return fail(LBM_ERR_ARG, "u_in must satisfy |u_in| < 0.3");
    if (c.obs_w > 0 && c.obs_x0 + c.obs_w > c.nx - 3)
        return fail(LBM_ERR_ARG, "an open channel's obstacle must end before column nx-3");
    if (c.grid_w < 0) return fail(LBM_ERR_ARG, "grid_w must be >= 0");
    if (c.grid_w > 0 && (c.grid_x0 < 1 || c.grid_x0 + c.grid_w > c.nx - 3 || c.grid_bar < 1 || c.grid_gap < 1))
        return fail(LBM_ERR_ARG, "grid: need 1 <= grid_x0, grid_x0 + grid_w <= nx - 3, grid_bar >= 1, grid_gap >= 1");
    if (c.sponge_len < 0 || c.sponge_len > c.nx) return fail(LBM_ERR_ARG, "sponge_len must be in [0, nx]");
    if (c.sponge_len > 0 && !(c.sponge_tau > 0.5)) return fail(LBM_ERR_ARG, "sponge_tau must exceed 1/2");
    const double tau_out = c.sponge_len > 0 ? c.sponge_tau : c.tau;
    if (!(tau_out <= 1.0)) return fail(LBM_ERR_ARG, "the relaxation time at the outlet must be at most 1");
    return LBM_OK;
}

namespace {

// relaxation time of column x of an open channel (the sponge profile)
double open_tau(const lbm_config& c, int x)
{
    if (c.sponge_len <= 0 || x < c.nx - c.sponge_len) return c.tau;
    const double s = (double)(x - (c.nx - c.sponge_len) + 1) / c.sponge_len;
    return c.tau + (c.sponge_tau - c.tau) * s * s;
}

Solids solids_of(const lbm_config& c)
{
    Solids s{};
    s.ox0 = c.obs_x0;
    s.oy0 = c.obs_y0;
    s.ox1 = c.obs_w > 0 ? c.obs_x0 + c.obs_w : c.obs_x0;
    s.oy1 = c.obs_w > 0 ? c.obs_y0 + c.obs_h : c.obs_y0;
    if (c.open_x && c.grid_w > 0) {
        s.gx0 = c.grid_x0;
        s.gx1 = c.grid_x0 + c.grid_w;
        s.gap = c.grid_gap;
        s.period = c.grid_bar + c.grid_gap;
    } else {
        s.gx0 = s.gx1 = 0;
        s.gap = s.period = 1;
    }
    return s;
}

// the launcher of variant v for this ensemble's channel
StepVariant::Launch launcher(const lbm_ensemble* e, const StepVariant& v)
{
    return e->cfg.open_x ? v.launch_open : v.launch;
}

// drag slots of a variant: kind 0, one per warp segment of vec sites in each
// ring row; kind 1 (row-staged), one per consumer warp in each ring row; kind 2
// (tiles), one per tile that holds part of the ring (rs0, rs1: tile columns)
Ring ring_for(const lbm_config& c, int vec, int kind)
{
    Ring r{0, -1, 0, -1, 0};
    if (c.obs_w <= 0) return r;
    r.ry0 = std::max(c.obs_y0 - 1, 0);
    r.ry1 = std::min(c.obs_y0 + c.obs_h, c.ny - 1);
    if (kind == 2) {
        r.rs0 = (c.obs_x0 - 1) / kTbTx;
        r.rs1 = (c.obs_x0 + c.obs_w) / kTbTx;
        r.n_slots = (r.ry1 / kTbTy - r.ry0 / kTbTy + 1) * (r.rs1 - r.rs0 + 1);
        return r;
    }
    if (kind == 0) {
        const int seg_w = 32 * vec;
        r.rs0 = (c.obs_x0 - 1) / seg_w;
        r.rs1 = (c.obs_x0 + c.obs_w) / seg_w;
    } else {
        r.rs0 = 0;
        r.rs1 = kRowWarps - 1;
    }
    r.n_slots = (r.ry1 - r.ry0 + 1) * (r.rs1 - r.rs0 + 1);
    return r;
}

int default_variant(int storage)
{
    const auto& v = step_variants();
    const int want_vec = storage == kFP32 ? 4 : 8;
    for (size_t i = 0; i < v.size(); ++i)
        if (v[i].storage == storage && v[i].kind == 0 && v[i].vec == want_vec && v[i].warps == 4) return (int)i;
    return -1;
}

// the variant of small step calls (one AMS branch): on a periodic channel the
// temporally blocked one (measured fastest for one 512 x 128 clone: 1.8
// against 2.7 us per step); on an open channel the narrowest register-staged
// variant with 8 warps per block, the most threads for a small call
int default_variant_small(int storage, bool open)
{
    const auto& v = step_variants();
    if (!open)
        for (size_t i = 0; i < v.size(); ++i)
            if (v[i].storage == storage && v[i].kind == 2) return (int)i;
    int best = -1;
    for (size_t i = 0; i < v.size(); ++i)
        if (v[i].storage == storage && v[i].kind == 0 && v[i].warps == 8 && (best < 0 || v[i].vec < v[best].vec))
            best = (int)i;
    return best >= 0 ? best : default_variant(storage);
}

int variant_for(const lbm_ensemble* e, int n_list)
{
    return (int64_t)n_list * e->cfg.nx * e->cfg.ny <= kSmallSites ? e->variant_small : e->variant;
}

// parameters of step `step` (0-based) of a chunk of `chunk` steps (chunk 0: a
// single step); an open channel's chunk writes its outlet column after the last
// step only, and the steps after the first pull from the outlet of the
// previous step's velocities
StepParams make_params(const lbm_ensemble* e, const int32_t* list, int32_t n_list, int vec, int step, int kind = 0,
                       int chunk = 0)
{
    const lbm_config& c = e->cfg;
    StepParams p{};
    p.buf0 = e->buf[0];
    p.buf1 = e->buf[1];
    p.parity = e->parity_dev;
    p.clone_list = list;
    p.n_list = n_list;
    p.nx = c.nx;
    p.ny = c.ny;
    p.pitch = e->pitch;
    p.plane = e->plane;
    p.clone_stride = e->clone_stride;
    p.nseg = (c.nx + 32 * vec - 1) / (32 * vec);
    p.err_flag = e->flag_dev + 2;
    p.ox0 = c.obs_x0;
    p.ox1 = c.obs_w > 0 ? c.obs_x0 + c.obs_w : c.obs_x0;
    p.oy0 = c.obs_y0;
    p.oy1 = c.obs_w > 0 ? c.obs_y0 + c.obs_h : c.obs_y0;
    const Ring r = ring_for(c, vec, kind);
    p.ry0 = r.ry0;
    p.ry1 = r.ry1;
    p.rs0 = r.rs0;
    p.rs1 = r.rs1;
    p.n_slots = e->n_slots;
    p.batch_cap = e->batch_cap;
    p.partials = e->partials;
    p.omega = (float)(1.0 / c.tau);
    p.gx = (float)c.gx;
    p.gy = (float)c.gy;
    p.bgk = bgk_consts(p.omega, p.gx, p.gy);
    p.coll = c.collision;
    p.cm = cm_consts(p.omega, (float)c.omega_bulk, (float)c.omega_3, (float)c.omega_4, p.gx, p.gy);
    p.scale = e->scale;
    p.inv_scale = e->inv_scale;
    p.step_in_batch = step;
    p.tb_steps = 1;
    const Solids sol = solids_of(c);
    p.open = c.open_x;
    p.gx0 = sol.gx0;
    p.gx1 = sol.gx1;
    p.ggap = sol.gap;
    p.gperiod = sol.period;
    p.gs0 = 1;
    p.gs1 = 0;
    p.sx0 = c.nx;
    if (c.open_x) {
        if (c.grid_w > 0 && vec > 0) {
            p.gs0 = (c.grid_x0 - 1) / (32 * vec);
            p.gs1 = (c.grid_x0 + c.grid_w) / (32 * vec);
        }
        if (c.sponge_len > 0) p.sx0 = c.nx - c.sponge_len;
        p.om_col = e->om_col;
        p.inlet_g = e->inlet_g;
        const int64_t u_buf = (int64_t)4 * c.ny * e->n;  // one velocity buffer per step parity
        p.open_u = e->open_u + (step & 1) * u_buf;
        p.open_u_prev = e->open_u + ((step + 1) & 1) * u_buf;
        p.outlet_from_u = step > 0 ? 1 : 0;
        p.write_outlet = step + 1 >= chunk ? 1 : 0;
        // the outlet column is the boundary kernel's: a row segment that would
        // hold it alone is not launched
        p.nseg = std::max(1, (c.nx - 1 + 32 * vec - 1) / (32 * vec));
        p.bc_pre = (float)(-2.0 / 3.0 * (open_tau(c, c.nx - 1) - 1.0));
    }
    return p;
}

int check_sticky(lbm_ensemble* e)
{
    int32_t flag[3] = {0, 0, 0};
    LBM_CUDA(cudaMemcpyAsync(flag, e->flag_dev, sizeof(int32_t) * 3, cudaMemcpyDeviceToHost, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    if (flag[2]) return fail(LBM_ERR_TIMEOUT, "a bounded device-side wait of the fused step ran out");
    if (flag[0]) return fail(LBM_ERR_NONFINITE, "a drag value of the ensemble is not finite (unstable flow?)");
    return LBM_OK;
}

template <typename F>
int dispatch_storage(int storage, F&& f)
{
    switch (storage) {
    case kFP32: return f(std::integral_constant<int, kFP32>{});
    case kFP16: return f(std::integral_constant<int, kFP16>{});
    case kBF16: return f(std::integral_constant<int, kBF16>{});
    }
    return fail(LBM_ERR_ARG, "unknown storage");
}

// the fused step launches of one chunk: steps 0 .. chunk-1 of a drag batch.
// With graphs on, the chunk is captured once (on a private stream, so that the
// caller's stream may be the legacy default stream) and the cached executable
// is replayed on the ensemble's stream; every kernel argument except the step
// index is fixed for the life of the ensemble, and the clone list is read
// through its device pointer at run time, so a replay is the same work as the
// launches it was captured from.
int launch_chunk(lbm_ensemble* e, int vi, const int32_t* list_dev, int n_list, int chunk)
{
    const StepVariant& v = step_variants()[vi];
    const StepVariant::Launch launch = launcher(e, v);
    if (!launch) return fail(LBM_ERR_ARG, "the step variant has no open-channel instantiation");
    // the steps of each launch: one, or for a multi-step variant an odd number
    // of at most v.multi (observables need the state after every step: one)
    std::vector<int> first, count;
    for (int s = 0; s < chunk;) {
        int k = (v.multi > 1 && !e->observe) ? std::min(v.multi, chunk - s) : 1;
        if (k % 2 == 0) k -= 1;
        first.push_back(s);
        count.push_back(k);
        s += k;
    }
    auto params = [&](size_t i) {
        StepParams p = make_params(e, list_dev, n_list, v.vec, first[i], v.kind, chunk);
        p.tb_steps = count[i];
        return p;
    };
    // an open channel adds the outlet kernel once per chunk, observables their own kernel per step
    const int launches = (int)first.size() + (e->observe ? chunk : 0) + (e->cfg.open_x ? 1 : 0);
    if (!e->use_graphs) {
        for (size_t i = 0; i < first.size(); ++i) {
            cudaError_t err = launch(params(i), e->stream);
            if (err != cudaSuccess) return cuda_fail(err, "step kernel launch");
            if (e->observe && observables_launch(e, list_dev, n_list, first[i], e->stream))
                return cuda_fail(cudaGetLastError(), "observables kernel launch");
        }
        count_launches(launches);
        return LBM_OK;
    }
    lbm_ensemble::StepGraph* hit = nullptr;
    for (auto& g : e->graphs)
        if (g.variant == vi && g.list == list_dev && g.n_list == n_list && g.chunk == chunk) hit = &g;
    if (!hit) {
        if (!e->cap_stream) LBM_CUDA(cudaStreamCreateWithFlags(&e->cap_stream, cudaStreamNonBlocking));
        LBM_CUDA(cudaStreamBeginCapture(e->cap_stream, cudaStreamCaptureModeRelaxed));
        cudaError_t launch_err = cudaSuccess;
        for (size_t i = 0; i < first.size() && launch_err == cudaSuccess; ++i) {
            launch_err = launch(params(i), e->cap_stream);
            if (launch_err == cudaSuccess && e->observe &&
                observables_launch(e, list_dev, n_list, first[i], e->cap_stream))
                launch_err = cudaGetLastError();
        }
        cudaGraph_t graph = nullptr;
        const cudaError_t end_err = cudaStreamEndCapture(e->cap_stream, &graph);
        if (launch_err != cudaSuccess || end_err != cudaSuccess) {
            if (graph) cudaGraphDestroy(graph);
            cudaGetLastError();
            return cuda_fail(launch_err != cudaSuccess ? launch_err : end_err, "capture of the step chunk");
        }
        cudaGraphExec_t exec = nullptr;
        const cudaError_t inst_err = cudaGraphInstantiate(&exec, graph, 0);
        cudaGraphDestroy(graph);
        if (inst_err != cudaSuccess) return cuda_fail(inst_err, "cudaGraphInstantiate of the step chunk");
        if (e->graphs.size() >= (size_t)kGraphCache) {  // drop the least recently used
            auto lru = std::min_element(e->graphs.begin(), e->graphs.end(),
                                        [](const auto& a, const auto& b) { return a.used < b.used; });
            cudaGraphExecDestroy(lru->exec);
            e->graphs.erase(lru);
        }
        e->graphs.push_back({vi, list_dev, n_list, chunk, exec, 0});
        hit = &e->graphs.back();
    }
    hit->used = ++e->graph_clock;
    LBM_CUDA(cudaGraphLaunch(hit->exec, e->stream));
    count_launches(launches);
    return LBM_OK;
}

// run the fused step n times on the listed clones (all at time t), with drag
// finalisation per batch and checkpoints at multiples of ckpt_stride
int step_list(lbm_ensemble* e, const int32_t* list_dev, const std::vector<int32_t>& list, int32_t n_steps)
{
    const auto& vars = step_variants();
    const int n_list = (int)list.size();
    int vi = variant_for(e, n_list);
    if (vars[vi].supports && !vars[vi].supports(make_params(e, list_dev, n_list, vars[vi].vec, 0, vars[vi].kind)))
        vi = (int64_t)n_list * e->cfg.nx * e->cfg.ny <= kSmallSites ? default_variant_small(e->cfg.storage, true)
                                                                     : default_variant(e->cfg.storage);
    const StepVariant& v = vars[vi];
    const Ring r = ring_for(e->cfg, v.vec, v.kind);
    int32_t t = e->t_host[list[0]];
    int32_t left = n_steps;
    while (left > 0) {
        int32_t chunk = std::min(left, e->batch_cap);
        if (e->cfg.ckpt_stride > 0) {
            const int32_t to_ckpt = e->cfg.ckpt_stride - (t % e->cfg.ckpt_stride);
            chunk = std::min(chunk, to_ckpt);
        }
        cudaEvent_t ev0 = nullptr, ev1 = nullptr;
        if (e->timing) {
            LBM_CUDA(cudaEventCreate(&ev0));
            LBM_CUDA(cudaEventCreate(&ev1));
            LBM_CUDA(cudaEventRecord(ev0, e->stream));
        }
        if (int rc = launch_chunk(e, vi, list_dev, n_list, chunk)) return rc;
        if (e->timing) {
            LBM_CUDA(cudaEventRecord(ev1, e->stream));
            e->events.emplace_back(ev0, ev1);
            e->timed_launches += chunk;
        }
        finalize_kernel<<<n_list, 128, 0, e->stream>>>(e->partials, e->batch_cap, e->n_slots, r.n_slots, list_dev,
                                                        chunk, e->drag, e->cfg.max_steps, e->t_dev, e->parity_dev,
                                                        e->flag_dev);
        count_launches(1);
        LBM_CUDA(cudaGetLastError());
        t += chunk;
        left -= chunk;
        for (int32_t c : list) {
            e->t_host[c] = t;
            e->parity_host[c] ^= (chunk & 1);
        }
        if (e->cfg.ckpt_stride > 0 && t % e->cfg.ckpt_stride == 0) {
            const int k = t / e->cfg.ckpt_stride;
            if (k < e->n_ckpt) {
                const size_t bytes = (size_t)e->clone_stride * e->elem_bytes;
                for (int32_t c : list) {
                    const char* from = static_cast<const char*>(e->buf[e->parity_host[c]]) + (size_t)c * bytes;
                    char* to = static_cast<char*>(e->ckpt) + ((size_t)c * e->n_ckpt + k) * bytes;
                    LBM_CUDA(cudaMemcpyAsync(to, from, bytes, cudaMemcpyDeviceToDevice, e->stream));
                }
                if (e->cnn) {  // learned score of every checkpointed state
                    int rc = score_clones(e, list.data(), (int32_t)list.size(), e->cnn_score, e->n_ckpt, k);
                    if (rc) return rc;
                }
            }
        }
    }
    return LBM_OK;
}

int compute_masses(lbm_ensemble* e, const int32_t* list_dev, int n_list)
{
    const Solids sol = solids_of(e->cfg);
    return dispatch_storage(e->cfg.storage, [&](auto tag) -> int {
        constexpr int S = decltype(tag)::value;
        dim3 grid(e->red_blocks, n_list);
        moments_partial_kernel<S><<<grid, kRedThreads, 0, e->stream>>>(
            e->buf[0], e->buf[1], e->parity_dev, list_dev, e->clone_stride, e->plane, e->pitch, e->cfg.nx, e->cfg.ny,
            sol, e->inv_scale, e->red_partials);
        count_launches(1);
        LBM_CUDA(cudaGetLastError());
        moments_final_kernel<<<n_list, 32, 0, e->stream>>>(e->red_partials, e->red_blocks, list_dev, e->mass_dev,
                                                            e->mass_dev + e->n, e->mass_dev + 2 * e->n);
        count_launches(1);
        LBM_CUDA(cudaGetLastError());
        return LBM_OK;
    });
}

int bank_masses(lbm_ensemble* e, int n_s)
{
    const Solids sol = solids_of(e->cfg);
    return dispatch_storage(e->cfg.storage, [&](auto tag) -> int {
        constexpr int S = decltype(tag)::value;
        bank_mass_partial_kernel<S><<<dim3(e->red_blocks, n_s), kRedThreads, 0, e->stream>>>(
            e->snaps, e->clone_stride, e->plane, e->pitch, e->cfg.nx, e->cfg.ny, sol, e->inv_scale,
            e->red_partials);
        LBM_CUDA(cudaGetLastError());
        bank_mass_final_kernel<<<n_s, 32, 0, e->stream>>>(e->red_partials, e->red_blocks, e->snap_mass);
        LBM_CUDA(cudaGetLastError());
        count_launches(2);
        return LBM_OK;
    });
}

int run_perturb(lbm_ensemble* e, const int32_t* parent_dev, int32_t inplace, double eps, uint64_t seed, uint64_t iter,
                const int32_t* slots = nullptr, int32_t n_slots = -1)
{
    const Solids sol = solids_of(e->cfg);
    const int n_s = eps != 0.0 ? e->n_snaps_set : 0;
    return dispatch_storage(e->cfg.storage, [&](auto tag) -> int {
        constexpr int S = decltype(tag)::value;
        const int64_t sites = (int64_t)e->cfg.nx * e->cfg.ny;
        const int bx = (int)std::min<int64_t>((sites + 255) / 256, 1024);
        dim3 grid(bx, slots ? n_slots : e->n);
        perturb_kernel<S><<<grid, 256, 0, e->stream>>>(
            e->buf[0], e->buf[1], e->parity_dev, parent_dev, e->n, e->flag_dev, inplace, slots, e->clone_stride, e->plane, e->pitch, e->cfg.nx,
            e->cfg.ny, sol, e->snaps, n_s, e->snap_mass, e->mass_dev, eps, seed, iter,
            e->perturb_mode ? 0.5 : 0.0, e->scale, e->inv_scale);
        count_launches(1);
        LBM_CUDA(cudaGetLastError());
        return LBM_OK;
    });
}

}  // namespace

// ---------------------------------------------------------------- C ABI
extern "C" {

const char* lbm_last_error(void) { return g_error.c_str(); }

int64_t lbm_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

int32_t lbm_step_variant_count(void) { return (int32_t)step_variants().size(); }

int32_t lbm_step_variant_kind(int32_t variant)
{
    const auto& v = step_variants();
    if (variant < 0 || variant >= (int32_t)v.size()) return fail(LBM_ERR_ARG, "variant index out of range");
    return v[variant].kind;
}

int lbm_step_variant_info(int32_t variant, int32_t* storage, int32_t* vec, int32_t* warps)
{
    const auto& v = step_variants();
    if (variant < 0 || variant >= (int32_t)v.size()) return fail(LBM_ERR_ARG, "variant index out of range");
    if (storage) *storage = v[variant].storage;
    if (vec) *vec = v[variant].vec;
    if (warps) *warps = v[variant].warps;
    return LBM_OK;
}

int lbm_ensemble_create(const lbm_config* cfg, int32_t n_clones, uint64_t seed, void* stream, lbm_ensemble** out)
{
    if (!cfg || !out) return fail(LBM_ERR_ARG, "null config or output pointer");
    *out = nullptr;
    const lbm_config c = *cfg;
    if (c.nx < 8 || (c.open_x == 0 && c.nx % 8 != 0))
        return fail(LBM_ERR_ARG, "nx must be a positive multiple of 8 (any nx >= 8 in an open channel)");
    if (c.ny < 2) return fail(LBM_ERR_ARG, "ny must be at least 2");
    if (n_clones < 1 || n_clones > 65535) return fail(LBM_ERR_ARG, "clone count must be in [1, 65535]");
    if ((int64_t)9 * (((c.nx + 255) / 256) * 256) * c.ny >= ((int64_t)1 << 31))
        return fail(LBM_ERR_ARG, "one clone must hold fewer than 2^31 population values");
    if (!(c.tau > 0.5) || !std::isfinite(c.tau)) return fail(LBM_ERR_ARG, "tau must exceed 1/2");
    if (!std::isfinite(c.gx) || !std::isfinite(c.gy)) return fail(LBM_ERR_ARG, "force must be finite");
    if (c.storage < 0 || c.storage > 2) return fail(LBM_ERR_ARG, "unknown storage");
    if (c.max_steps < 1) return fail(LBM_ERR_ARG, "max_steps must be positive");
    if (c.ckpt_stride < 0) return fail(LBM_ERR_ARG, "ckpt_stride must be >= 0");
    if (c.n_snapshots < 0 || c.n_snapshots > 16) return fail(LBM_ERR_ARG, "n_snapshots must be in [0, 16]");
    if (c.shift_exp < -20 || c.shift_exp > 20) return fail(LBM_ERR_ARG, "shift_exp out of range");
    if (c.obs_w < 0 || c.obs_h < 0 || (c.obs_w > 0) != (c.obs_h > 0)) return fail(LBM_ERR_ARG, "obstacle size");
    if (c.obs_w > 0) {
        if (c.obs_x0 < 1 || c.obs_x0 + c.obs_w > c.nx - 1)
            return fail(LBM_ERR_ARG, "obstacle must leave a fluid column on both sides in x");
        if (c.obs_y0 < 0 || c.obs_y0 + c.obs_h > c.ny) return fail(LBM_ERR_ARG, "obstacle outside the channel");
    }
    if (int rc = check_collision(c)) return rc;
    if (int rc = check_open(c)) return rc;
    int dev = 0;
    LBM_CUDA(cudaGetDevice(&dev));
    auto* e = new lbm_ensemble();
    e->cfg = c;
    e->n = n_clones;
    e->seed = seed;
    e->stream = static_cast<cudaStream_t>(stream);
    e->device = dev;
    e->elem_bytes = elem_size(c.storage);
    e->pitch = ((c.nx + 255) / 256) * 256;
    e->plane = (int64_t)e->pitch * c.ny;
    e->clone_stride = 9 * e->plane;
    e->scale = (float)std::ldexp(1.0, c.storage == kFP32 ? 0 : c.shift_exp);
    e->inv_scale = (float)std::ldexp(1.0, c.storage == kFP32 ? 0 : -c.shift_exp);
    e->variant = default_variant(c.storage);
    e->perturb_mode = 0;
    e->variant_small = default_variant_small(c.storage, c.open_x != 0);
    e->use_graphs = true;
    e->batch_cap = kBatchCap;
    e->red_blocks = kRedBlocks;
    // partial slots: enough for the narrowest segments of any variant
    int max_slots = 1;
    for (const auto& v : step_variants())
        if (v.storage == c.storage) max_slots = std::max(max_slots, ring_for(c, v.vec, v.kind).n_slots);
    e->n_slots = max_slots;
    e->n_ckpt = c.ckpt_stride > 0 ? c.max_steps / c.ckpt_stride + 1 : 0;
    e->parity_host.assign(n_clones, 0);
    e->t_host.assign(n_clones, 0);

    auto cleanup = [&](int code) {
        lbm_ensemble_destroy(e);
        return code;
    };
    const size_t state_bytes = (size_t)e->clone_stride * e->elem_bytes * n_clones;
    cudaError_t err;
#define ALLOC(ptr, bytes)                                                         \
    err = cudaMalloc((void**)&(ptr), (bytes));                                    \
    if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaMalloc " #ptr));
    ALLOC(e->buf[0], state_bytes);
    ALLOC(e->buf[1], state_bytes);
    ALLOC(e->parity_dev, sizeof(int32_t) * n_clones);
    ALLOC(e->t_dev, sizeof(int32_t) * n_clones);
    ALLOC(e->list_dev, sizeof(int32_t) * n_clones);
    ALLOC(e->all_dev, sizeof(int32_t) * n_clones);
    ALLOC(e->fields_list_dev, sizeof(int32_t) * n_clones);
    ALLOC(e->partials, sizeof(float) * (size_t)n_clones * e->batch_cap * e->n_slots);
    ALLOC(e->drag, sizeof(double) * (size_t)n_clones * c.max_steps);
    ALLOC(e->scores, sizeof(double) * (size_t)n_clones * c.max_steps);
    ALLOC(e->flag_dev, sizeof(int32_t) * 4);
    ALLOC(e->red_partials, sizeof(double) * 3 * (size_t)n_clones * e->red_blocks);
    ALLOC(e->mass_dev, sizeof(double) * 3 * n_clones);
    if (c.n_snapshots > 0) {
        ALLOC(e->snaps, (size_t)e->clone_stride * e->elem_bytes * c.n_snapshots);
        ALLOC(e->snap_mass, sizeof(double) * c.n_snapshots);
    }
    if (e->n_ckpt > 0) { ALLOC(e->ckpt, (size_t)e->clone_stride * e->elem_bytes * n_clones * e->n_ckpt); }
    if (c.open_x) {
        ALLOC(e->om_col, sizeof(float) * c.nx);
        ALLOC(e->inlet_g, sizeof(float) * 9 * c.ny);
        ALLOC(e->open_u, sizeof(float) * 2 * 4 * c.ny * (size_t)n_clones);
    }
#undef ALLOC
    std::vector<int32_t> iota(n_clones);
    for (int i = 0; i < n_clones; ++i) iota[i] = i;
    auto chk = [&](cudaError_t er, const char* what) { return er == cudaSuccess ? 0 : cleanup(cuda_fail(er, what)); };
    int rc;
    if ((rc = chk(cudaMemcpyAsync(e->all_dev, iota.data(), sizeof(int32_t) * n_clones, cudaMemcpyHostToDevice, e->stream), "copy clone index"))) return rc;
    if ((rc = chk(cudaMemsetAsync(e->parity_dev, 0, sizeof(int32_t) * n_clones, e->stream), "memset parity"))) return rc;
    if ((rc = chk(cudaMemsetAsync(e->t_dev, 0, sizeof(int32_t) * n_clones, e->stream), "memset time"))) return rc;
    if ((rc = chk(cudaMemsetAsync(e->flag_dev, 0, sizeof(int32_t) * 4, e->stream), "memset flag"))) return rc;
    if ((rc = chk(cudaMemsetAsync(e->buf[0], 0, state_bytes, e->stream), "memset state"))) return rc;
    if ((rc = chk(cudaMemsetAsync(e->buf[1], 0, state_bytes, e->stream), "memset state"))) return rc;
    if ((rc = chk(cudaMemsetAsync(e->partials, 0, sizeof(float) * (size_t)n_clones * e->batch_cap * e->n_slots, e->stream), "memset partials"))) return rc;
    if ((rc = chk(cudaMemsetAsync(e->drag, 0, sizeof(double) * (size_t)n_clones * c.max_steps, e->stream), "memset drag"))) return rc;
    if (c.open_x) {
        // per-column relaxation rate and the inlet populations (FP64, then FP32)
        std::vector<float> om(c.nx), inlet(9 * (size_t)c.ny);
        for (int x = 0; x < c.nx; ++x) om[x] = (float)(1.0 / open_tau(c, x));
        for (int y = 0; y < c.ny; ++y) {
            const double h = c.ny, yy = y + 0.5, u = c.u_in * 4.0 * yy * (h - yy) / (h * h);
            for (int q = 0; q < 9; ++q) {
                const double cu = cx(q) * u;
                inlet[(size_t)q * c.ny + y] = (float)(wd(q) * (3.0 * cu + 4.5 * cu * cu - 1.5 * u * u));
            }
        }
        if ((rc = chk(cudaMemcpyAsync(e->om_col, om.data(), sizeof(float) * c.nx, cudaMemcpyHostToDevice, e->stream), "copy sponge rates"))) return rc;
        if ((rc = chk(cudaMemcpyAsync(e->inlet_g, inlet.data(), sizeof(float) * inlet.size(), cudaMemcpyHostToDevice, e->stream), "copy inlet"))) return rc;
        // the copies read pageable host memory: wait before the vectors go
        if ((rc = chk(cudaStreamSynchronize(e->stream), "open-channel tables"))) return rc;
    }
    const Solids sol = solids_of(c);
    rc = dispatch_storage(c.storage, [&](auto tag) -> int {
        constexpr int S = decltype(tag)::value;
        const int64_t total = (int64_t)c.nx * c.ny * n_clones;
        const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 64);
        init_kernel<S><<<grid, 256, 0, e->stream>>>(e->buf[0], e->clone_stride, e->plane, e->pitch, c.nx, c.ny,
                                                    n_clones, sol, seed, c.init_amp, c.open_x ? c.u_in : 0.0, e->scale);
        count_launches(1);
        return chk(cudaGetLastError(), "init kernel");
    });
    if (rc) return rc;
    if (e->n_ckpt > 0) {
        const size_t bytes = (size_t)e->clone_stride * e->elem_bytes;
        for (int i = 0; i < n_clones; ++i) {
            rc = chk(cudaMemcpyAsync(static_cast<char*>(e->ckpt) + (size_t)i * e->n_ckpt * bytes,
                                     static_cast<char*>(e->buf[0]) + (size_t)i * bytes, bytes,
                                     cudaMemcpyDeviceToDevice, e->stream), "checkpoint 0");
            if (rc) return rc;
        }
    }
    if ((rc = chk(cudaStreamSynchronize(e->stream), "create sync"))) return rc;
    *out = e;
    return LBM_OK;
}

int lbm_ensemble_destroy(lbm_ensemble* e)
{
    if (!e) return LBM_OK;
    cudaStreamSynchronize(e->stream);
    for (auto& pr : e->events) {
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    for (auto& g : e->graphs) cudaGraphExecDestroy(g.exec);
    if (e->cap_stream) cudaStreamDestroy(e->cap_stream);
    void* ptrs[] = {e->buf[0], e->buf[1], e->parity_dev, e->t_dev, e->list_dev, e->all_dev, e->partials,
                    e->drag, e->scores, e->flag_dev, e->red_partials, e->mass_dev, e->snaps, e->snap_mass, e->ckpt,
                    e->fields_list_dev, e->cnn_x, e->cnn_pred, e->cnn_score, e->pot[0], e->pot[1], e->pot[2],
                    e->pot_tmp[0], e->pot_tmp[1], e->om_col, e->inlet_g, e->open_u, e->obs};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    delete e;
    return LBM_OK;
}

int lbm_ensemble_step(lbm_ensemble* e, int32_t n_steps)
{
    if (!e) return fail(LBM_ERR_ARG, "null ensemble");
    if (n_steps < 0) return fail(LBM_ERR_ARG, "n_steps must be >= 0");
    const int32_t t = e->t_host[0];
    for (int i = 1; i < e->n; ++i)
        if (e->t_host[i] != t) return fail(LBM_ERR_STATE, "clones are at different times; use lbm_ensemble_step_clones");
    if ((int64_t)t + n_steps > e->cfg.max_steps) return fail(LBM_ERR_ARG, "drag history capacity (max_steps) exceeded");
    if (n_steps == 0) return LBM_OK;
    std::vector<int32_t> all(e->n);
    for (int i = 0; i < e->n; ++i) all[i] = i;
    return step_list(e, e->all_dev, all, n_steps);
}

int lbm_ensemble_step_clones(lbm_ensemble* e, int32_t n_steps, const int32_t* clones, int32_t n)
{
    if (!e || !clones) return fail(LBM_ERR_ARG, "null argument");
    if (n < 1 || n > e->n || n_steps < 0) return fail(LBM_ERR_ARG, "bad clone count or step count");
    std::vector<int32_t> list(clones, clones + n), sorted(list);
    std::sort(sorted.begin(), sorted.end());
    for (int i = 0; i < n; ++i) {
        if (sorted[i] < 0 || sorted[i] >= e->n) return fail(LBM_ERR_ARG, "clone index out of range");
        if (i > 0 && sorted[i] == sorted[i - 1]) return fail(LBM_ERR_ARG, "repeated clone index");
    }
    const int32_t t = e->t_host[list[0]];
    for (int32_t c : list)
        if (e->t_host[c] != t) return fail(LBM_ERR_STATE, "listed clones are at different times");
    if ((int64_t)t + n_steps > e->cfg.max_steps) return fail(LBM_ERR_ARG, "drag history capacity (max_steps) exceeded");
    if (n_steps == 0) return LBM_OK;
    LBM_CUDA(cudaMemcpyAsync(e->list_dev, list.data(), sizeof(int32_t) * n, cudaMemcpyHostToDevice, e->stream));
    int rc = step_list(e, e->list_dev, list, n_steps);
    if (rc) return rc;
    // the list buffer is reused by the next call: keep the host copy alive
    // until the enqueued copy has been consumed
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    return LBM_OK;
}

int lbm_ensemble_time(lbm_ensemble* e, int32_t* t)
{
    if (!e || !t) return fail(LBM_ERR_ARG, "null argument");
    std::copy(e->t_host.begin(), e->t_host.end(), t);
    return LBM_OK;
}

int lbm_ensemble_drag(lbm_ensemble* e, int32_t t0, int32_t t1, double* dst, int32_t dst_on_device)
{
    if (!e || !dst) return fail(LBM_ERR_ARG, "null argument");
    const int32_t tmax = *std::max_element(e->t_host.begin(), e->t_host.end());
    if (t0 < 0 || t1 < t0 || t1 > tmax) return fail(LBM_ERR_ARG, "drag window outside the recorded history");
    const int32_t w = t1 - t0;
    if (w == 0) return LBM_OK;
    LBM_CUDA(cudaMemcpy2DAsync(dst, sizeof(double) * w, e->drag + t0, sizeof(double) * e->cfg.max_steps,
                               sizeof(double) * w, e->n,
                               dst_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, e->stream));
    if (!dst_on_device) return check_sticky(e);
    return LBM_OK;
}

int lbm_ensemble_set_drag(lbm_ensemble* e, int32_t t0, int32_t t1, const double* src)
{
    if (!e || !src) return fail(LBM_ERR_ARG, "null argument");
    const int32_t tmax = *std::max_element(e->t_host.begin(), e->t_host.end());
    if (t0 < 0 || t1 < t0 || t1 > tmax) return fail(LBM_ERR_ARG, "drag window outside the recorded history");
    const int32_t w = t1 - t0;
    for (int64_t i = 0; i < (int64_t)w * e->n; ++i)
        if (!std::isfinite(src[i])) return fail(LBM_ERR_ARG, "drag values must be finite");
    if (w == 0) return LBM_OK;
    LBM_CUDA(cudaMemcpy2DAsync(e->drag + t0, sizeof(double) * e->cfg.max_steps, src, sizeof(double) * w,
                               sizeof(double) * w, e->n, cudaMemcpyHostToDevice, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    return LBM_OK;
}

int lbm_ensemble_window_sum(lbm_ensemble* e, int32_t t0, int32_t t1, double k, double* out_dev)
{
    if (!e || !out_dev) return fail(LBM_ERR_ARG, "null argument");
    const int32_t tmax = *std::max_element(e->t_host.begin(), e->t_host.end());
    if (t0 < 0 || t1 < t0 || t1 > tmax) return fail(LBM_ERR_ARG, "window outside the recorded history");
    if (!std::isfinite(k)) return fail(LBM_ERR_ARG, "k must be finite");
    window_sum_kernel<<<e->n, kRedThreads, 0, e->stream>>>(e->drag, e->cfg.max_steps, t0, t1, k, out_dev);
    count_launches(1);
    LBM_CUDA(cudaGetLastError());
    return LBM_OK;
}

int lbm_ensemble_scores(lbm_ensemble* e, int32_t window, int32_t t_begin, int32_t t_end, double* out_dev)
{
    if (!e) return fail(LBM_ERR_ARG, "null ensemble");
    const int32_t tmax = *std::max_element(e->t_host.begin(), e->t_host.end());
    if (window < 1 || t_begin < 0 || t_end < t_begin || t_end > tmax) return fail(LBM_ERR_ARG, "bad window or time range");
    scores_kernel<<<e->n, kRedThreads, 0, e->stream>>>(e->drag, e->cfg.max_steps, window, t_begin, t_end, e->scores,
                                                       out_dev);
    count_launches(1);
    LBM_CUDA(cudaGetLastError());
    e->score_window = window;
    e->score_t_begin = t_begin;
    e->score_t_end = t_end;
    return LBM_OK;
}

int lbm_ensemble_first_crossing(lbm_ensemble* e, int32_t clone, double level, int32_t* t)
{
    if (!e || !t) return fail(LBM_ERR_ARG, "null argument");
    if (clone < 0 || clone >= e->n) return fail(LBM_ERR_ARG, "clone index out of range");
    if (e->score_window < 1) return fail(LBM_ERR_STATE, "call lbm_ensemble_scores first");
    first_crossing_kernel<<<1, kRedThreads, 0, e->stream>>>(e->scores + (int64_t)clone * e->cfg.max_steps,
                                                           e->score_t_begin + e->score_window, e->score_t_end, level,
                                                           e->flag_dev + 1);
    count_launches(1);
    LBM_CUDA(cudaGetLastError());
    LBM_CUDA(cudaMemcpyAsync(t, e->flag_dev + 1, sizeof(int32_t), cudaMemcpyDeviceToHost, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    return LBM_OK;
}

int lbm_ensemble_set_snapshots(lbm_ensemble* e, int32_t n_s, const int32_t* clones)
{
    if (!e || (n_s > 0 && !clones)) return fail(LBM_ERR_ARG, "null argument");
    if (n_s < 0 || n_s > e->cfg.n_snapshots) return fail(LBM_ERR_ARG, "more snapshots than the bank holds");
    const size_t bytes = (size_t)e->clone_stride * e->elem_bytes;
    std::vector<int32_t> list(clones, clones + n_s);
    for (int k = 0; k < n_s; ++k) {
        const int c = list[k];
        if (c < 0 || c >= e->n) return fail(LBM_ERR_ARG, "clone index out of range");
        LBM_CUDA(cudaMemcpyAsync(static_cast<char*>(e->snaps) + (size_t)k * bytes,
                                 static_cast<char*>(e->buf[e->parity_host[c]]) + (size_t)c * bytes, bytes,
                                 cudaMemcpyDeviceToDevice, e->stream));
    }
    if (n_s > 0) {
        int rc = bank_masses(e, n_s);
        if (rc) return rc;
    }
    e->n_snaps_set = n_s;
    return LBM_OK;
}

int lbm_ensemble_set_snapshots_from_checkpoint(lbm_ensemble* e, int32_t n_s, const int32_t* clones, int32_t k)
{
    if (!e || (n_s > 0 && !clones)) return fail(LBM_ERR_ARG, "null argument");
    if (n_s < 0 || n_s > e->cfg.n_snapshots) return fail(LBM_ERR_ARG, "more snapshots than the bank holds");
    if (e->n_ckpt < 1 || k < 0 || k >= e->n_ckpt) return fail(LBM_ERR_ARG, "no such checkpoint");
    const size_t bytes = (size_t)e->clone_stride * e->elem_bytes;
    for (int i = 0; i < n_s; ++i) {
        const int c = clones[i];
        if (c < 0 || c >= e->n) return fail(LBM_ERR_ARG, "clone index out of range");
        LBM_CUDA(cudaMemcpyAsync(static_cast<char*>(e->snaps) + (size_t)i * bytes,
                                 static_cast<char*>(e->ckpt) + ((size_t)c * e->n_ckpt + k) * bytes, bytes,
                                 cudaMemcpyDeviceToDevice, e->stream));
    }
    if (n_s > 0) {
        int rc = bank_masses(e, n_s);
        if (rc) return rc;
    }
    e->n_snaps_set = n_s;
    return LBM_OK;
}

int lbm_ensemble_clone(lbm_ensemble* e, const int32_t* parent_dev, double eps, uint64_t seed, uint64_t iter)
{
    if (!e || !parent_dev) return fail(LBM_ERR_ARG, "null argument");
    if (!std::isfinite(eps) || eps < 0.0) return fail(LBM_ERR_ARG, "eps must be finite and >= 0");
    if (eps != 0.0 && e->n_snaps_set < 1) return fail(LBM_ERR_STATE, "perturbation needs the snapshot bank");
    const int32_t t = e->t_host[0];
    for (int i = 1; i < e->n; ++i)
        if (e->t_host[i] != t || e->parity_host[i] != e->parity_host[0])
            return fail(LBM_ERR_STATE, "cloning needs every clone at the same time");
    if (eps != 0.0) {
        int rc = compute_masses(e, e->all_dev, e->n);
        if (rc) return rc;
    }
    int rc = run_perturb(e, parent_dev, -1, eps, seed, iter);
    if (rc) return rc;
    if (t > 0) {
        dim3 grid((unsigned)std::min(64, (t + 255) / 256), e->n);
        copy_history_kernel<<<grid, 256, 0, e->stream>>>(e->drag, e->cfg.max_steps, parent_dev, e->n, t);
        count_launches(1);
        LBM_CUDA(cudaGetLastError());
        if (e->obs) {  // the observables of a copied trajectory are its parent's
            dim3 g4((unsigned)std::min(64, (4 * t + 255) / 256), e->n);
            copy_history_kernel<<<g4, 256, 0, e->stream>>>(e->obs, 4 * e->cfg.max_steps, parent_dev, e->n, 4 * t);
            count_launches(1);
            LBM_CUDA(cudaGetLastError());
        }
    }
    return LBM_OK;
}

int lbm_ensemble_branch(lbm_ensemble* e, int32_t dst, int32_t src, int32_t t_b, double eps, uint64_t seed,
                        uint64_t iter)
{
    if (!e) return fail(LBM_ERR_ARG, "null ensemble");
    if (dst < 0 || dst >= e->n || src < 0 || src >= e->n || dst == src) return fail(LBM_ERR_ARG, "bad clone indices");
    if (e->cfg.ckpt_stride <= 0) return fail(LBM_ERR_STATE, "branching needs checkpoints (ckpt_stride > 0)");
    if (t_b < 0 || t_b > e->t_host[src]) return fail(LBM_ERR_ARG, "branch time beyond the source trajectory");
    if (!std::isfinite(eps) || eps < 0.0) return fail(LBM_ERR_ARG, "eps must be finite and >= 0");
    if (eps != 0.0 && e->n_snaps_set < 1) return fail(LBM_ERR_STATE, "perturbation needs the snapshot bank");
    const int kc = t_b / e->cfg.ckpt_stride;
    const int32_t tc = kc * e->cfg.ckpt_stride;
    if (kc >= e->n_ckpt) return fail(LBM_ERR_ARG, "no checkpoint covers the branch time");
    const size_t bytes = (size_t)e->clone_stride * e->elem_bytes;
    char* ck = static_cast<char*>(e->ckpt);
    // checkpoints 0..kc and the state at tc
    for (int k = 0; k <= kc; ++k)
        LBM_CUDA(cudaMemcpyAsync(ck + ((size_t)dst * e->n_ckpt + k) * bytes, ck + ((size_t)src * e->n_ckpt + k) * bytes,
                                 bytes, cudaMemcpyDeviceToDevice, e->stream));
    LBM_CUDA(cudaMemcpyAsync(static_cast<char*>(e->buf[e->parity_host[dst]]) + (size_t)dst * bytes,
                             ck + ((size_t)src * e->n_ckpt + kc) * bytes, bytes, cudaMemcpyDeviceToDevice, e->stream));
    if (e->cnn_score)  // the learned score of the shared checkpoints
        LBM_CUDA(cudaMemcpyAsync(e->cnn_score + (size_t)dst * e->n_ckpt, e->cnn_score + (size_t)src * e->n_ckpt,
                                 sizeof(double) * (kc + 1), cudaMemcpyDeviceToDevice, e->stream));
    // dst is now the source at time tc; replay to t_b (bitwise the source's path)
    e->t_host[dst] = tc;
    LBM_CUDA(cudaMemcpyAsync(e->t_dev + dst, &e->t_host[dst], sizeof(int32_t), cudaMemcpyHostToDevice, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    if (t_b > tc) {
        int rc = lbm_ensemble_step_clones(e, t_b - tc, &dst, 1);
        if (rc) return rc;
    }
    // the drag history up to t_b is the source's own, copied after the replay:
    // the replay may run another step variant, whose per-warp drag partials
    // are summed in another grouping (the populations are identical bit for bit)
    if (t_b > 0) {
        LBM_CUDA(cudaMemcpyAsync(e->drag + (size_t)dst * e->cfg.max_steps, e->drag + (size_t)src * e->cfg.max_steps,
                                 sizeof(double) * t_b, cudaMemcpyDeviceToDevice, e->stream));
        if (e->obs)
            LBM_CUDA(cudaMemcpyAsync(e->obs + (size_t)dst * 4 * e->cfg.max_steps,
                                     e->obs + (size_t)src * 4 * e->cfg.max_steps, sizeof(double) * 4 * t_b,
                                     cudaMemcpyDeviceToDevice, e->stream));
    }
    if (eps != 0.0) {
        LBM_CUDA(cudaMemcpyAsync(e->list_dev, &dst, sizeof(int32_t), cudaMemcpyHostToDevice, e->stream));
        int rc = compute_masses(e, e->list_dev, 1);
        if (rc) return rc;
        rc = run_perturb(e, e->all_dev, dst, eps, seed, iter);
        if (rc) return rc;
        LBM_CUDA(cudaStreamSynchronize(e->stream));
    }
    return LBM_OK;
}

int lbm_ensemble_perturb(lbm_ensemble* e, int32_t n, const int32_t* clones, double eps, uint64_t seed, uint64_t iter)
{
    if (!e || !clones) return fail(LBM_ERR_ARG, "null argument");
    if (n < 1 || n > e->n) return fail(LBM_ERR_ARG, "clone count out of range");
    std::vector<char> seen(e->n, 0);
    for (int i = 0; i < n; ++i) {
        if (clones[i] < 0 || clones[i] >= e->n || seen[clones[i]]) return fail(LBM_ERR_ARG, "bad or repeated clone index");
        seen[clones[i]] = 1;
    }
    if (!std::isfinite(eps) || eps < 0.0) return fail(LBM_ERR_ARG, "eps must be finite and >= 0");
    if (eps == 0.0) return LBM_OK;  // the identity
    if (e->n_snaps_set < 1) return fail(LBM_ERR_STATE, "perturbation needs the snapshot bank");
    LBM_CUDA(cudaMemcpyAsync(e->list_dev, clones, sizeof(int32_t) * n, cudaMemcpyHostToDevice, e->stream));
    int rc = compute_masses(e, e->list_dev, n);
    if (rc) return rc;
    rc = run_perturb(e, e->all_dev, kAllInPlace, eps, seed, iter, e->list_dev, n);
    if (rc) return rc;
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    return LBM_OK;
}

int lbm_ensemble_set_perturbation(lbm_ensemble* e, int32_t mode)
{
    if (!e) return fail(LBM_ERR_ARG, "null ensemble");
    if (mode != 0 && mode != 1) return fail(LBM_ERR_ARG, "perturbation mode must be 0 (App. D) or 1 (centred)");
    e->perturb_mode = mode;
    return LBM_OK;
}

int lbm_ensemble_moments(lbm_ensemble* e, double* mass, double* px, double* py)
{
    if (!e) return fail(LBM_ERR_ARG, "null ensemble");
    int rc = compute_masses(e, e->all_dev, e->n);
    if (rc) return rc;
    std::vector<double> h(3 * (size_t)e->n);
    LBM_CUDA(cudaMemcpyAsync(h.data(), e->mass_dev, sizeof(double) * 3 * e->n, cudaMemcpyDeviceToHost, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    for (int i = 0; i < e->n; ++i) {
        if (mass) mass[i] = h[i];
        if (px) px[i] = h[e->n + i];
        if (py) py[i] = h[2 * e->n + i];
    }
    return LBM_OK;
}

namespace {
double decode_host(int storage, const void* raw, size_t idx, int q, float inv_scale)
{
    const double w = wd(q);
    if (storage == kFP32) return (double)static_cast<const float*>(raw)[idx];
    if (storage == kFP16) return w + (double)__half2float(static_cast<const __half*>(raw)[idx]) * inv_scale;
    return w + (double)__bfloat162float(static_cast<const __nv_bfloat16*>(raw)[idx]) * inv_scale;
}
}  // namespace

int lbm_ensemble_get_populations(lbm_ensemble* e, int32_t clone, double* host)
{
    if (!e || !host) return fail(LBM_ERR_ARG, "null argument");
    if (clone < 0 || clone >= e->n) return fail(LBM_ERR_ARG, "clone index out of range");
    const size_t bytes = (size_t)e->clone_stride * e->elem_bytes;
    std::vector<char> raw(bytes);
    LBM_CUDA(cudaMemcpyAsync(raw.data(), static_cast<char*>(e->buf[e->parity_host[clone]]) + (size_t)clone * bytes,
                             bytes, cudaMemcpyDeviceToHost, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    const int nx = e->cfg.nx, ny = e->cfg.ny;
    for (int q = 0; q < 9; ++q)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x)
                host[((size_t)q * ny + y) * nx + x] =
                    decode_host(e->cfg.storage, raw.data(), (size_t)q * e->plane + (size_t)y * e->pitch + x, q, e->inv_scale);
    return LBM_OK;
}

int lbm_ensemble_set_populations(lbm_ensemble* e, int32_t clone, const double* host)
{
    if (!e || !host) return fail(LBM_ERR_ARG, "null argument");
    if (clone < 0 || clone >= e->n) return fail(LBM_ERR_ARG, "clone index out of range");
    const size_t bytes = (size_t)e->clone_stride * e->elem_bytes;
    std::vector<char> raw(bytes, 0);
    const int nx = e->cfg.nx, ny = e->cfg.ny;
    for (int q = 0; q < 9; ++q)
        for (int y = 0; y < ny; ++y)
            for (int x = 0; x < nx; ++x) {
                const double f = host[((size_t)q * ny + y) * nx + x];
                if (!std::isfinite(f)) return fail(LBM_ERR_NONFINITE, "population not finite");
                const size_t idx = (size_t)q * e->plane + (size_t)y * e->pitch + x;
                if (e->cfg.storage == kFP32)
                    reinterpret_cast<float*>(raw.data())[idx] = (float)f;
                else if (e->cfg.storage == kFP16)
                    reinterpret_cast<__half*>(raw.data())[idx] = __float2half_rn((float)((f - wd(q)) * e->scale));
                else
                    reinterpret_cast<__nv_bfloat16*>(raw.data())[idx] = __float2bfloat16_rn((float)((f - wd(q)) * e->scale));
            }
    LBM_CUDA(cudaMemcpyAsync(static_cast<char*>(e->buf[e->parity_host[clone]]) + (size_t)clone * bytes, raw.data(),
                             bytes, cudaMemcpyHostToDevice, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    return LBM_OK;
}

int lbm_ensemble_set_variant(lbm_ensemble* e, int32_t variant)
{
    if (!e) return fail(LBM_ERR_ARG, "null ensemble");
    if (variant == -1) {
        e->variant = default_variant(e->cfg.storage);
        e->variant_small = default_variant_small(e->cfg.storage, e->cfg.open_x != 0);
        return LBM_OK;
    }
    const auto& v = step_variants();
    if (variant < 0 || variant >= (int32_t)v.size()) return fail(LBM_ERR_ARG, "variant index out of range");
    if (v[variant].storage != e->cfg.storage) return fail(LBM_ERR_ARG, "variant is for another storage format");
    if (!launcher(e, v[variant])) return fail(LBM_ERR_ARG, "the variant has no open-channel instantiation");
    e->variant = variant;  // a forced variant runs every step call
    e->variant_small = variant;
    return LBM_OK;
}

int lbm_ensemble_autotune(lbm_ensemble* e, int32_t* variant)
{
    if (!e) return fail(LBM_ERR_ARG, "null ensemble");
    const auto& vars = step_variants();
    cudaEvent_t a, b;
    LBM_CUDA(cudaEventCreate(&a));
    LBM_CUDA(cudaEventCreate(&b));
    // Every trial launch reads the current buffer and rewrites the other one
    // at step_in_batch 0: the state does not advance and no drag is recorded.
    auto tune = [&](int n_list, int reps, int best) -> int {
        float best_ms = std::numeric_limits<float>::infinity();
        for (size_t i = 0; i < vars.size(); ++i) {
            const StepVariant& v = vars[i];
            if (v.storage != e->cfg.storage) continue;
            const StepVariant::Launch launch = launcher(e, v);
            if (!launch) continue;
            StepParams p = make_params(e, e->all_dev, n_list, v.vec, 0, v.kind);
            p.tb_steps = v.multi;  // a multi-step trial runs its steps: timed per step below
            if (v.supports && !v.supports(p)) continue;
            for (int r = 0; r < 2; ++r)
                if (launch(p, e->stream) != cudaSuccess) return -1;
            cudaEventRecord(a, e->stream);
            for (int r = 0; r < reps; ++r)
                if (launch(p, e->stream) != cudaSuccess) return -1;
            count_launches((2 + reps) * (e->cfg.open_x ? 2 : 1));
            cudaEventRecord(b, e->stream);
            if (cudaEventSynchronize(b) != cudaSuccess) return -1;
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            ms /= (float)v.multi;
            if (ms < best_ms) {
                best_ms = ms;
                best = (int)i;
            }
        }
        return best;
    };
    // the wide variant on the whole ensemble; the small-list one on a single
    // clone (one AMS branch), with more launches since each is short
    const int wide = tune(e->n, 5, e->variant);
    const int small = wide < 0 ? -1 : tune(1, 40, e->variant_small);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (wide < 0 || small < 0) return cuda_fail(cudaGetLastError(), "lbm_ensemble_autotune trial launch");
    e->variant = wide;
    e->variant_small = small;
    if (variant) *variant = wide;
    return LBM_OK;
}

int lbm_ensemble_set_graphs(lbm_ensemble* e, int32_t enable)
{
    if (!e) return fail(LBM_ERR_ARG, "null ensemble");
    e->use_graphs = enable != 0;
    return LBM_OK;
}

int lbm_ensemble_set_timing(lbm_ensemble* e, int32_t enable)
{
    if (!e) return fail(LBM_ERR_ARG, "null ensemble");
    e->timing = enable != 0;
    return LBM_OK;
}

int lbm_ensemble_kernel_time(lbm_ensemble* e, double* ms, int64_t* launches, int32_t reset)
{
    if (!e) return fail(LBM_ERR_ARG, "null ensemble");
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    for (auto& pr : e->events) {
        float t = 0.f;
        LBM_CUDA(cudaEventElapsedTime(&t, pr.first, pr.second));
        e->timed_ms += t;
        cudaEventDestroy(pr.first);
        cudaEventDestroy(pr.second);
    }
    e->events.clear();
    if (ms) *ms = e->timed_ms;
    if (launches) *launches = e->timed_launches;
    if (reset) {
        e->timed_ms = 0.0;
        e->timed_launches = 0;
    }
    return LBM_OK;
}

}  // extern "C"
