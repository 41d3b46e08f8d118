// Row-staged variant of the fused stream-collide-drag step.
//
// Same arithmetic as lbm_step.cuh (pull streaming with halfway bounce-back,
// BGK with Guo forcing, momentum-exchange drag), different data movement:
// a persistent block walks a list of (clone, row) work items; for each item the
// nine source rows (plane q at row y - c_qy, or at the wall the own row of the
// opposite plane) are brought into a shared-memory stage by nine asynchronous
// bulk copies (cp.async.bulk, completion counted in bytes on an mbarrier),
// several stages ahead of the computation.  The bytes in flight are then held
// by shared memory, not by registers, which is what the 16-bit formats need
// (a register-staged 16-bit kernel keeps only ~74 KB per SM in flight).  The
// +-1 shift in x and the periodic seam become plain shared-memory indexing
// because the whole row is present.
//
// Every wait on an mbarrier is bounded; on timeout the block records an error
// flag (reported as LBM_ERR_TIMEOUT), waits (bounded) for its copies in flight
// and returns.
#pragma once
#include "internal.h"
#include "lbm_device.cuh"
#include "async_copy.cuh"

namespace lbm {

constexpr int kRowConsumers = 32 * kRowWarps;
constexpr int kRowThreads = kRowConsumers + 32;   // + 1 producer warp
constexpr int kRowMaxStages = 8;
constexpr int kRowSmemBudget = 110 * 1024;        // two blocks per SM

// what the consumers of a stage need to know about its work item
struct StageInfo {
    int c, y, cur;
};

// V sites x0 .. x0+V-1 of row y from the staged rows st; returns this
// thread's share of the momentum exchange with the obstacle (GENERAL rows only:
// the walls, and the ring of rows around the obstacle)
template <int S, int V, bool SCALED, bool GENERAL, int COLL>
__device__ __forceinline__ float rows_sites(const StepParams& p, const typename Codec<S>::T* st,
                                            const typename Codec<S>::T* gsrc, typename Codec<S>::T* dst, int y,
                                            int x0, bool ring)
{
    using T = typename Codec<S>::T;
    using K = Carry<S, SCALED>;
    const int nx = p.nx;
    float g[9][V];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const bool wall = GENERAL && ((y - cy(q)) < 0 || (y - cy(q)) >= p.ny);
        const T* r = st + q * nx;
        // V aligned values in one shared-memory load, the one across the +-1
        // shift (periodic at the seam) in a second
        const Vec<T, V> v = *reinterpret_cast<const Vec<T, V>*>(r + x0);
        float d[V];
        if constexpr (V % 2 == 0) {
#pragma unroll
            for (int j = 0; j < V; j += 2) {
                const float2 f = K::in2(&v.e[j], wf(q), p.inv_scale);
                d[j] = f.x;
                d[j + 1] = f.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) d[j] = K::in(v.e[j], wf(q), p.inv_scale);
        }
        if (cx(q) == 0 || wall) {  // the wall returns this node's own population: no shift
#pragma unroll
            for (int j = 0; j < V; ++j) g[q][j] = d[j];
        } else if (cx(q) == 1) {
            g[q][0] = K::in(r[x0 == 0 ? nx - 1 : x0 - 1], wf(q), p.inv_scale);
#pragma unroll
            for (int j = 1; j < V; ++j) g[q][j] = d[j - 1];
        } else {
            g[q][V - 1] = K::in(r[x0 + V >= nx ? 0 : x0 + V], wf(q), p.inv_scale);
#pragma unroll
            for (int j = 0; j < V - 1; ++j) g[q][j] = d[j + 1];
        }
    }
    if (GENERAL && ring) {
        // links whose upstream node is solid bounce back at this node
#pragma unroll
        for (int q = 1; q < 9; ++q) {
            const int ys = y - cy(q);
            if (ys < p.oy0 || ys >= p.oy1) continue;
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int xs = x0 + j - cx(q);
                if (xs >= p.ox0 && xs < p.ox1)
                    g[q][j] = K::in(gsrc[opp(q) * p.plane + (int64_t)y * p.pitch + x0 + j], wf(q), p.inv_scale);
            }
        }
    }
#pragma unroll
    for (int j = 0; j < V; ++j) collide<COLL, V>(g, j, p);
    float acc = 0.f;
    if (GENERAL && ring) {
        const bool row_solid = y >= p.oy0 && y < p.oy1;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const int x = x0 + j;
            if (row_solid && x >= p.ox0 && x < p.ox1) {
#pragma unroll
                for (int q = 0; q < 9; ++q) g[q][j] = 0.f;  // solid node: rest state f = w
            } else {
#pragma unroll
                for (int q = 1; q < 9; ++q) {
                    if (cx(q) == 0) continue;
                    const int xn = x + cx(q), yn = y + cy(q);
                    if (xn >= p.ox0 && xn < p.ox1 && yn >= p.oy0 && yn < p.oy1)
                        acc += 2.0f * (float)cx(q) * (wf(q) + g[q][j]);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        Vec<T, V> o;
        if constexpr (V % 2 == 0) {
#pragma unroll
            for (int j = 0; j < V; j += 2) K::out2(&o.e[j], g[q][j], g[q][j + 1], wf(q), p.scale);
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) o.e[j] = K::out(g[q][j], wf(q), p.scale);
        }
        st_stream<T, V>(dst + q * p.plane + (int64_t)y * p.pitch + x0, o);
    }
    return acc;
}

template <int S, int V, bool SCALED, int COLL>
__global__ void __launch_bounds__(kRowThreads, 2) step_rows_kernel(const StepParams p, int stages)
{
    using T = typename Codec<S>::T;
    using K = Carry<S, SCALED>;
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t full[kRowMaxStages];
    __shared__ __align__(8) uint64_t empty[kRowMaxStages];
    __shared__ StageInfo info[kRowMaxStages];
    __shared__ volatile int abort_flag;
    const int nx = p.nx;
    const int64_t row_bytes = (int64_t)nx * sizeof(T);
    const int64_t stage_bytes = 9 * row_bytes;
    const int items = p.n_list * p.ny;
    const int tid = threadIdx.x;
    if (tid == 0) {
        abort_flag = 0;
        for (int s = 0; s < stages; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), kRowConsumers / 32);
        }
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();

    if (tid >= kRowConsumers) {
        // ---------------- producer warp: one lane issues the copies
        if (tid != kRowConsumers) return;
        int k = 0, issued_last = -1;
        for (int item = blockIdx.x; item < items; item += gridDim.x, ++k) {
            const int s = k % stages;
            if (k >= stages && !mbar_wait_cycles(smem_addr(&empty[s]), (uint32_t)(((k / stages) - 1) & 1), kWaitCycles)) {
                if (p.err_flag) atomicExch(p.err_flag, 1);
                abort_flag = 1;
                break;
            }
            if (abort_flag) break;
            const int li = item / p.ny, y = item - li * p.ny;
            const int c = p.clone_list[li];
            const int cur = p.parity[c] ^ (p.step_in_batch & 1);
            info[s] = StageInfo{c, y, cur};
            const T* src = static_cast<const T*>(cur ? p.buf1 : p.buf0) + (int64_t)c * p.clone_stride;
            const uint32_t bar = smem_addr(&full[s]);
            const uint32_t dst = smem_addr(smem + s * stage_bytes);
            mbar_expect_tx(bar, (uint32_t)(9 * row_bytes));
#pragma unroll
            for (int q = 0; q < 9; ++q) {
                int sy = y - cy(q), plane_q = q;
                if (sy < 0 || sy >= p.ny) {  // the wall returns the population that left this node
                    sy = y;
                    plane_q = opp(q);
                }
                bulk_g2s(dst + (uint32_t)(q * row_bytes), src + plane_q * p.plane + (int64_t)sy * p.pitch,
                         (uint32_t)row_bytes, bar);
            }
            issued_last = k;
        }
        // the block's shared memory must outlive every copy issued into it
        for (int kk = issued_last - stages + 1 > 0 ? issued_last - stages + 1 : 0; kk <= issued_last; ++kk)
            mbar_wait_cycles(smem_addr(&full[kk % stages]), (uint32_t)((kk / stages) & 1), kWaitCycles);
        return;
    }

    // ---------------- consumer warps
    int k = 0;
    for (int item = blockIdx.x; item < items; item += gridDim.x, ++k) {
        const int s = k % stages;
        if (!mbar_wait_cycles(smem_addr(&full[s]), (uint32_t)((k / stages) & 1), kWaitCycles)) {
            if (p.err_flag) atomicExch(p.err_flag, 1);
            abort_flag = 1;
        }
        if (abort_flag) break;
        const StageInfo inf = info[s];
        const int c = inf.c, y = inf.y;
        const T* st = reinterpret_cast<const T*>(smem + s * stage_bytes);
        const T* gsrc = static_cast<const T*>(inf.cur ? p.buf1 : p.buf0) + (int64_t)c * p.clone_stride;
        T* dst = static_cast<T*>(inf.cur ? p.buf0 : p.buf1) + (int64_t)c * p.clone_stride;
        const bool ring = p.ox1 > p.ox0 && y >= p.ry0 && y <= p.ry1;
        if (ring || y == 0 || y == p.ny - 1) {
            float acc = 0.f;
            for (int x0 = tid * V; x0 < nx; x0 += kRowConsumers * V)
                acc += rows_sites<S, V, SCALED, true, COLL>(p, st, gsrc, dst, y, x0, ring);
            if (ring) {  // one drag partial per consumer warp and ring row
#pragma unroll
                for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
                if ((tid & 31) == 0)
                    p.partials[((int64_t)c * p.batch_cap + p.step_in_batch) * p.n_slots + (y - p.ry0) * kRowWarps +
                               (tid >> 5)] = acc;
            }
        } else {
            for (int x0 = tid * V; x0 < nx; x0 += kRowConsumers * V)
                rows_sites<S, V, SCALED, false, COLL>(p, st, gsrc, dst, y, x0, false);
        }
        __syncwarp();
        if ((tid & 31) == 0) mbar_arrive(smem_addr(&empty[s]));  // this warp is done with the stage
    }
}

template <int S, int V>
bool rows_supported(const StepParams& p)
{
    using T = typename Codec<S>::T;
    const int64_t stage = 9 * (int64_t)p.nx * sizeof(T);
    return p.nx % V == 0 && (p.nx * (int64_t)sizeof(T)) % 16 == 0 && 2 * stage <= kRowSmemBudget;
}

// one launch of one instantiation; the opt-in to more than 48 KB of dynamic
// shared memory is made once per instantiation (its own static flag)
template <int S, int V, bool SCALED, int COLL>
cudaError_t launch_rows_kernel(const StepParams& p, cudaStream_t s, int grid, int stages, size_t smem)
{
    static bool attr = false;
    if (!attr) {
        const cudaError_t e = cudaFuncSetAttribute(step_rows_kernel<S, V, SCALED, COLL>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize, kRowSmemBudget);
        if (e != cudaSuccess) return e;
        attr = true;
    }
    step_rows_kernel<S, V, SCALED, COLL><<<grid, kRowThreads, smem, s>>>(p, stages);
    return cudaGetLastError();
}

template <int S, int V>
cudaError_t launch_rows(const StepParams& p, cudaStream_t s)
{
    using T = typename Codec<S>::T;
    if (!rows_supported<S, V>(p)) return cudaErrorInvalidValue;
    const int64_t stage = 9 * (int64_t)p.nx * sizeof(T);
    int stages = (int)(kRowSmemBudget / stage);
    stages = stages > kRowMaxStages ? kRowMaxStages : stages;
    const size_t smem = (size_t)stages * stage;
    const int items = p.n_list * p.ny;
    int sms = 152;
    int dev = 0;
    if (cudaGetDevice(&dev) == cudaSuccess) cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int grid = items < 2 * sms ? items : 2 * sms;
    const bool scaled = S != kFP32 && p.scale != 1.0f;
    if (p.coll == 1)
        return scaled ? launch_rows_kernel<S, V, S != kFP32, 1>(p, s, grid, stages, smem)
                      : launch_rows_kernel<S, V, false, 1>(p, s, grid, stages, smem);
    return scaled ? launch_rows_kernel<S, V, S != kFP32, 0>(p, s, grid, stages, smem)
                  : launch_rows_kernel<S, V, false, 0>(p, s, grid, stages, smem);
}

}  // namespace lbm
