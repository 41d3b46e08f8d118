// Temporally blocked fused step: several steps of App. A per launch, for the
// small step calls of one AMS branch (App. B.1: one trajectory re-simulated
// from a checkpoint), where a single 512 x 128 clone is a few megabytes that
// L2 holds and the step is bound by the boundary between launches rather than
// by memory.
//
// A CTA owns a tile of kTbTx x kTbTy sites.  It loads the tile with a halo of
// kTbHalo sites on every side - a 32 x 16 region, one site per thread
// (periodic in x, rows beyond the walls left unused) - into shared memory
// once, runs up to kTbHalo steps there - step s computes the sites that are
// still exact after it, the tile grown by kTbHalo - 1 - s sites - and writes
// the tile back.  The halo is recomputed by the neighbouring tiles (1.3 times
// the sites of a step for three steps); in exchange the steps of a launch read
// and write shared memory only.  Tiles away from the walls and the obstacle
// take a path without any boundary test.
//
// The per-site work is the register-staged kernels' own: the same pulls (wall
// and obstacle bounce-back from the node's opposite direction), the same
// collision routine, and every value passes through the storage format
// between steps exactly as through global memory, so the populations are
// those of every other variant bit for bit.  The drag of each step is reduced
// per tile in a fixed order (FP32 partial sums grouped otherwise than in the
// other variants).  A launch runs an odd number of steps, so that it ends in
// the buffer the ensemble's parity bookkeeping expects and never overwrites
// the buffer another tile is still loading.  Periodic channels only.
#pragma once
#include "lbm_step.cuh"

namespace lbm {

constexpr int kTbSites = kTbRw * kTbRh;  // 512

template <int S>
constexpr size_t tb_smem_bytes()
{
    return 2 * 9 * (size_t)kTbSites * sizeof(typename Codec<S>::T);
}

template <int S, bool SCALED, int COLL>
__global__ void __launch_bounds__(kTbThreads, 2) step_tb_kernel(const StepParams p)
{
    using T = typename Codec<S>::T;
    using K = Carry<S, SCALED>;
    extern __shared__ __align__(16) unsigned char tb_smem[];
    __shared__ float red[2][kTbThreads / 32];  // per step parity: thread 0 reads one while warps fill the other
    T* const b0 = reinterpret_cast<T*>(tb_smem);
    T* const b1 = b0 + 9 * kTbSites;
    const int c = p.clone_list[blockIdx.z];
    const int cur = p.parity[c] ^ (p.step_in_batch & 1);
    const T* src = static_cast<const T*>(cur ? p.buf1 : p.buf0) + (int64_t)c * p.clone_stride;
    T* dst = static_cast<T*>(cur ? p.buf0 : p.buf1) + (int64_t)c * p.clone_stride;
    const int plane = (int)p.plane;
    // this thread's site of the region: column rx = lane, row ry = warp
    const int rx = threadIdx.x & 31, ry = threadIdx.x >> 5;
    const int o = ry * kTbRw + rx;
    const int gx0 = blockIdx.x * kTbTx - kTbHalo, gy0 = blockIdx.y * kTbTy - kTbHalo;  // the region's origin
    int x = gx0 + rx;
    x = x < 0 ? x + p.nx : (x >= p.nx ? x - p.nx : x);
    const int y = gy0 + ry;
    const bool row_in = y >= 0 && y < p.ny;
    const int ox0 = p.ox0, ox1 = p.ox1, oy0 = p.oy0, oy1 = p.oy1;
    // the boundary tests are needed only where the region meets a wall or the
    // obstacle's neighbourhood (a region that wraps around the periodic seam
    // is taken as general too)
    const bool general = gy0 < 1 || gy0 + kTbRh > p.ny - 1 || gx0 < 0 || gx0 + kTbRw > p.nx ||
                         (ox1 > ox0 && gx0 <= ox1 && gx0 + kTbRw > ox0 - 1 && gy0 <= oy1 && gy0 + kTbRh > oy0 - 1);
    // a tile of the drag ring (one partial per ring tile and step)
    const int ts0 = p.ry0 / kTbTy, ts1 = p.ry1 / kTbTy;
    const bool ring = ox1 > ox0 && (int)blockIdx.x >= p.rs0 && (int)blockIdx.x <= p.rs1 && (int)blockIdx.y >= ts0 &&
                      (int)blockIdx.y <= ts1;
    const bool interior = rx >= kTbHalo && rx < kTbHalo + kTbTx && ry >= kTbHalo && ry < kTbHalo + kTbTy &&
                          gx0 + rx < p.nx && row_in;

    // ---- load the region (rows beyond the walls are never read)
    if (row_in) {
#pragma unroll
        for (int q = 0; q < 9; ++q) b0[q * kTbSites + o] = src[q * plane + y * p.pitch + x];
    }
    __syncthreads();

    const int steps = p.tb_steps;
    for (int s = 0; s < steps; ++s) {
        const T* in = (s & 1) ? b1 : b0;
        T* out = (s & 1) ? b0 : b1;
        // the sites still exact after this step: the tile grown by steps - 1 - s
        const int m = kTbHalo - (steps - 1 - s);
        float acc = 0.f;
        if (row_in && rx >= m && rx < kTbRw - m && ry >= m && ry < kTbRh - m) {
            float g[9][1];
            if (!general) {
#pragma unroll
                for (int q = 0; q < 9; ++q)
                    g[q][0] = K::in(in[q * kTbSites + o - cy(q) * kTbRw - cx(q)], wf(q), p.inv_scale);
            } else {
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const int ex = cx(q), ey = cy(q);
                    const int ys = y - ey;
                    int xs = x - ex;
                    xs = xs < 0 ? xs + p.nx : (xs >= p.nx ? xs - p.nx : xs);
                    const bool back = ys < 0 || ys >= p.ny || (xs >= ox0 && xs < ox1 && ys >= oy0 && ys < oy1);
                    // wall or obstacle upstream: the population that left this node comes back
                    const T v = back ? in[opp(q) * kTbSites + o] : in[q * kTbSites + o - ey * kTbRw - ex];
                    g[q][0] = K::in(v, wf(q), p.inv_scale);
                }
            }
            collide<COLL, 1>(g, 0, p);
            if (general) {
                if (x >= ox0 && x < ox1 && y >= oy0 && y < oy1) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) g[q][0] = 0.f;  // solid node: rest state f = w
                } else if (ring && interior) {
                    // momentum exchange with the obstacle, sites of this tile only
#pragma unroll
                    for (int q = 1; q < 9; ++q) {
                        if (cx(q) == 0) continue;
                        const int xn = x + cx(q), yn = y + cy(q);
                        if (xn >= ox0 && xn < ox1 && yn >= oy0 && yn < oy1)
                            acc += 2.0f * (float)cx(q) * (wf(q) + g[q][0]);
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < 9; ++q) out[q * kTbSites + o] = K::out(g[q][0], wf(q), p.scale);
        }
        if (ring) {  // the tile's drag partial of this step, in a fixed order
#pragma unroll
            for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
            if (rx == 0) red[s & 1][ry] = acc;
        }
        __syncthreads();
        if (ring && threadIdx.x == 0) {
            float sum = 0.f;
            for (int k = 0; k < kTbThreads / 32; ++k) sum += red[s & 1][k];
            const int slot = ((int)blockIdx.y - ts0) * (p.rs1 - p.rs0 + 1) + ((int)blockIdx.x - p.rs0);
            p.partials[((int64_t)c * p.batch_cap + p.step_in_batch + s) * p.n_slots + slot] = sum;
        }
    }

    // ---- write the tile (the last step's buffer)
    if (interior) {
        const T* fin = (steps & 1) ? b1 : b0;
#pragma unroll
        for (int q = 0; q < 9; ++q) dst[q * plane + y * p.pitch + x] = fin[q * kTbSites + o];
    }
}

// periodic channels at least 40 sites wide (one wrap covers every halo)
template <int S>
bool tb_supported(const StepParams& p)
{
    return !p.open && p.nx >= 40;
}

// one launch of p.tb_steps (odd, at most kTbHalo) steps
template <int S, bool SCALED, int COLL>
cudaError_t launch_tb_kernel(const StepParams& p, cudaStream_t s)
{
    const dim3 grid((p.nx + kTbTx - 1) / kTbTx, (p.ny + kTbTy - 1) / kTbTy, p.n_list);
    step_tb_kernel<S, SCALED, COLL><<<grid, kTbThreads, tb_smem_bytes<S>(), s>>>(p);
    return cudaGetLastError();
}

template <int S>
cudaError_t launch_tb(const StepParams& p, cudaStream_t s)
{
    if (!tb_supported<S>(p) || p.tb_steps < 1 || p.tb_steps > kTbHalo || p.tb_steps % 2 == 0)
        return cudaErrorInvalidValue;
    const bool scaled = S != kFP32 && p.scale != 1.0f;
    if (p.coll == 1)
        return scaled ? launch_tb_kernel<S, S != kFP32, 1>(p, s) : launch_tb_kernel<S, false, 1>(p, s);
    return scaled ? launch_tb_kernel<S, S != kFP32, 0>(p, s) : launch_tb_kernel<S, false, 0>(p, s);
}

static_assert(tb_smem_bytes<kFP32>() <= 48 * 1024, "the region fits the default dynamic shared memory");

}  // namespace lbm
