// Fused D2Q9 pull-stream + BGK/Guo collide + momentum-exchange drag kernel.
//
// One step t -> t+1 of App. A for every listed clone:
//   streaming   f_q(x, t+1) = f*_q(x - c_q, t), or f*_{opp q}(x, t) when
//               x - c_q lies beyond a wall or inside the obstacle (halfway
//               bounce-back, Sec. 2); periodic in x;
//   collision   f*_q = f_q + (f_q^eq - f_q)/tau + (1 - 1/(2 tau)) S_q with the
//               Guo source S_q = w_q [3 (c_q - u) + 9 (c_q.u) c_q] . F and
//               rho u = sum f c + F/2;
//   drag        D_x(t+1) = sum over fluid x, q with x + c_q solid of 2 c_qx f*_q:
//               the momentum the next streaming step hands to the obstacle
//               (eq. (drag_definition) for the bounce-back surface).
//
// Memory layout: structure of arrays, plane q of clone c is a ny x pitch
// array.  Thread = V consecutive sites of one row; warp = 32 V sites.  Every
// plane is read with one aligned V-wide vector load per thread (16 bytes when
// V * sizeof(T) = 16); the one-site shift of directions with c_x = +-1 is
// done in registers with a warp shuffle, and only the two warp-edge elements
// are fetched separately (they sit in sectors the neighbouring warp reads, so
// they come from L2).  Each population value is read once and written once:
// there is no reuse for shared memory or TMA staging to exploit, the kernel is
// bound by HBM bandwidth at 2 * 9 * sizeof(T) bytes per site.
#pragma once
#include "internal.h"
#include "lbm_device.cuh"

namespace lbm {

template <int S, int V, int WARPS>
__global__ void __launch_bounds__(WARPS * 32) step_kernel(const StepParams p)
{
    using C = Codec<S>;
    using T = typename C::T;
    const int lane = threadIdx.x & 31;
    const int64_t gwarp = (int64_t)blockIdx.x * WARPS + (threadIdx.x >> 5);
    const int64_t per_clone = (int64_t)p.ny * p.nseg;
    const int li = (int)(gwarp / per_clone);
    if (li >= p.n_list) return;  // warp-uniform
    const int rem = (int)(gwarp - (int64_t)li * per_clone);
    const int y = rem / p.nseg;
    const int seg = rem - y * p.nseg;
    const int c = p.clone_list[li];
    const int cur = p.parity[c] ^ (p.step_in_batch & 1);
    const T* __restrict__ src = static_cast<const T*>(cur ? p.buf1 : p.buf0) + (int64_t)c * p.clone_stride;
    T* __restrict__ dst = static_cast<T*>(cur ? p.buf0 : p.buf1) + (int64_t)c * p.clone_stride;
    const int x0 = seg * 32 * V + lane * V;
    const bool active = x0 < p.nx;
    const int64_t row_off = (int64_t)y * p.pitch;

    const bool obst = p.ox1 > p.ox0;
    float g[9][V];

#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int ex = cx(q), ey = cy(q);
        const float wq = wf(q);
        const int ys = y - ey;
        if (ys < 0 || ys >= p.ny) {
            // the wall sends back the population that left this node
            const Vec<T, V> v = ld_stream<T, V>(src + opp(q) * p.plane + row_off + x0);
#pragma unroll
            for (int j = 0; j < V; ++j) g[q][j] = C::dec(v.e[j], wq, p.inv_scale);
        } else {
            const T* row = src + q * p.plane + (int64_t)ys * p.pitch;
            const Vec<T, V> v = ld_stream<T, V>(row + x0);
            float d[V];
#pragma unroll
            for (int j = 0; j < V; ++j) d[j] = C::dec(v.e[j], wq, p.inv_scale);
            if (ex == 0) {
#pragma unroll
                for (int j = 0; j < V; ++j) g[q][j] = d[j];
            } else if (ex == 1) {
                // site x pulls from x - 1
                float edge = __shfl_up_sync(0xffffffffu, d[V - 1], 1);
                if (lane == 0 || x0 == 0) {
                    const int xs = x0 == 0 ? p.nx - 1 : x0 - 1;
                    edge = C::dec(ld_one(row + xs), wq, p.inv_scale);
                }
                g[q][0] = edge;
#pragma unroll
                for (int j = 1; j < V; ++j) g[q][j] = d[j - 1];
            } else {
                // site x pulls from x + 1
                float edge = __shfl_down_sync(0xffffffffu, d[0], 1);
                if (lane == 31 || x0 + V >= p.nx) {
                    const int xs = x0 + V >= p.nx ? 0 : x0 + V;
                    edge = C::dec(ld_one(row + xs), wq, p.inv_scale);
                }
#pragma unroll
                for (int j = 0; j < V - 1; ++j) g[q][j] = d[j + 1];
                g[q][V - 1] = edge;
            }
            // links whose upstream node is solid bounce back at this node
            if (obst && ys >= p.oy0 && ys < p.oy1) {
                bool any = false;
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const int xs = x0 + j - ex;
                    any |= (xs >= p.ox0 && xs < p.ox1);
                }
                if (any) {
                    const Vec<T, V> o = ld_stream<T, V>(src + opp(q) * p.plane + row_off + x0);
#pragma unroll
                    for (int j = 0; j < V; ++j) {
                        const int xs = x0 + j - ex;
                        if (xs >= p.ox0 && xs < p.ox1) g[q][j] = C::dec(o.e[j], wq, p.inv_scale);
                    }
                }
            }
        }
    }

    // BGK collision with Guo forcing, in the shifted variables g = f - w
    const float om = p.omega;
    const float src_coef = 1.0f - 0.5f * om;
    const float gx = p.gx, gy = p.gy;
    const bool row_has_solid = obst && y >= p.oy0 && y < p.oy1;
#pragma unroll
    for (int j = 0; j < V; ++j) {
        float drho = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            drho += g[q][j];
            if (cx(q) != 0) jx += (float)cx(q) * g[q][j];
            if (cy(q) != 0) jy += (float)cy(q) * g[q][j];
        }
        const float rho = 1.0f + drho;
        const float inv = __frcp_rn(rho);
        const float ux = (jx + 0.5f * gx) * inv;
        const float uy = (jy + 0.5f * gy) * inv;
        const float usq15 = 1.5f * (ux * ux + uy * uy);
        const float uF = ux * gx + uy * gy;
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            const float wq = wf(q);
            const float cu = (float)cx(q) * ux + (float)cy(q) * uy;
            const float cF = (float)cx(q) * gx + (float)cy(q) * gy;
            const float geq = wq * (drho + rho * (cu * (3.0f + 4.5f * cu) - usq15));
            const float Sq = wq * (3.0f * (cF - uF) + 9.0f * cu * cF);
            g[q][j] = g[q][j] + om * (geq - g[q][j]) + src_coef * Sq;
        }
        if (row_has_solid) {
            const int x = x0 + j;
            if (x >= p.ox0 && x < p.ox1) {
#pragma unroll
                for (int q = 0; q < 9; ++q) g[q][j] = 0.f;  // solid node: rest state
            }
        }
    }

    // momentum exchange with the obstacle, one partial per warp of the ring
    if (obst && y >= p.ry0 && y <= p.ry1 && seg >= p.rs0 && seg <= p.rs1) {
        float acc = 0.f;
        if (active) {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int x = x0 + j;
                const bool solid_here = y >= p.oy0 && y < p.oy1 && x >= p.ox0 && x < p.ox1;
                if (solid_here) continue;
#pragma unroll
                for (int q = 1; q < 9; ++q) {
                    if (cx(q) == 0) continue;
                    const int xn = x + cx(q), yn = y + cy(q);
                    if (xn >= p.ox0 && xn < p.ox1 && yn >= p.oy0 && yn < p.oy1)
                        acc += 2.0f * (float)cx(q) * (wf(q) + g[q][j]);
                }
            }
        }
#pragma unroll
        for (int off = 16; off > 0; off >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, off);
        if (lane == 0) {
            const int slot = (y - p.ry0) * (p.rs1 - p.rs0 + 1) + (seg - p.rs0);
            p.partials[((int64_t)c * p.batch_cap + p.step_in_batch) * p.n_slots + slot] = acc;
        }
    }

    if (active) {
#pragma unroll
        for (int q = 0; q < 9; ++q) {
            Vec<T, V> o;
#pragma unroll
            for (int j = 0; j < V; ++j) o.e[j] = C::enc(g[q][j], wf(q), p.scale);
            st_stream<T, V>(dst + q * p.plane + row_off + x0, o);
        }
    }
}

template <int S, int V, int WARPS>
cudaError_t launch_step(const StepParams& p, int grid, cudaStream_t s)
{
    step_kernel<S, V, WARPS><<<grid, WARPS * 32, 0, s>>>(p);
    return cudaGetLastError();
}

}  // namespace lbm
