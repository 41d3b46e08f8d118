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
// array.  Thread = V consecutive sites of one row; warp = 32 V sites; block =
// WARPS rows of the same 32 V-site segment; grid = (segments, row blocks,
// listed clones), so no index arithmetic needs a division.  Every plane is
// read with one aligned V-wide vector load per thread (16 bytes for V *
// sizeof(T) = 16), all nine issued before any is used; the one-site shift of
// directions with c_x = +-1 is done in registers with a warp shuffle, and only
// the two warp-edge elements are fetched separately (sectors the neighbouring
// warp reads, so they come from L2).  Each population value is read once and
// written once: there is no reuse for shared memory or TMA staging to
// exploit, and the kernel is bound by HBM bandwidth at 2 * 9 * sizeof(T)
// bytes per site.
//
// Interior warps (no wall row, away from the obstacle) take a path without
// any boundary test; the few warps on the walls and around the obstacle take
// the general path, which also produces the drag partial of the warp.
#pragma once
#include <type_traits>
#include "internal.h"
#include "lbm_device.cuh"

namespace lbm {

// The collision carries the shifted value g = f - w_q for every storage
// format.  For FP32 storage the shift is applied on load and undone on store:
// the float weights do not sum to one exactly (4/9 + 4/9 + 1/9 rounds to
// 1 + 7.5e-9), and carrying f itself would turn that into a systematic mass
// drift of om * 7.5e-9 per node and step; with g the same float w_q cancels
// between load and store.
// SCALED = false compiles the 2^s storage scale out (s = 0).
template <int S, bool SCALED> struct Carry {
    using T = typename Codec<S>::T;
    __device__ static float in(T v, float w, float inv_scale) { return Codec<S>::dec(v, w, SCALED ? inv_scale : 1.0f); }
    __device__ static T out(float g, float w, float scale) { return Codec<S>::enc(g, w, SCALED ? scale : 1.0f); }
    __device__ static float2 in2(const T* v, float w, float inv_scale)
    {
        return Codec<S>::dec2(v, w, SCALED ? inv_scale : 1.0f);
    }
    __device__ static void out2(T* o, float a, float b, float w, float scale)
    {
        Codec<S>::enc2(o, a, b, w, SCALED ? scale : 1.0f);
    }
};

// one opposite pair (q, opp q) of the collision, from the shared E and O terms
__device__ __forceinline__ void bgk_pair(float& gq, float& go, float cu, float A, float B, float wq, float P, float Qc,
                                         float a0, float omm)
{
    const float E = fmaf(cu, fmaf(Qc, cu, A), a0);
    const float O = fmaf(P, cu, B);
    gq = fmaf(wq, E + O, omm * gq);
    go = fmaf(wq, E - O, omm * go);
}

// BGK collision with Guo forcing of site j, in place on the carried values
// g = f - w, in the pairwise form of BgkConsts.  FORCE = false compiles the
// force terms out (a channel without body force: the open channel)
template <int V, bool FORCE = true>
__device__ __forceinline__ void bgk_collide(float (&g)[9][V], int j, const BgkConsts& k)
{
    const float s1 = g[1][j] + g[3][j], d1 = g[1][j] - g[3][j];
    const float s2 = g[2][j] + g[4][j], d2 = g[2][j] - g[4][j];
    const float s5 = g[5][j] + g[7][j], d5 = g[5][j] - g[7][j];
    const float s6 = g[6][j] + g[8][j], d6 = g[6][j] - g[8][j];
    const float drho = (g[0][j] + s1) + (s2 + (s5 + s6));
    const float jx = d1 + (d5 - d6), jy = d2 + (d5 + d6);
    const float inv = __fdividef(1.0f, 1.0f + drho);
    if constexpr (FORCE) {
        const float ux = (jx + k.hgx) * inv, uy = (jy + k.hgy) * inv;
        const float P = fmaf(k.om3, drho, k.om3);  // 3 om rho
        const float Qc = 1.5f * P;                  // 4.5 om rho
        const float u2 = fmaf(ux, ux, uy * uy);
        float a0 = fmaf(k.om, drho, -(0.5f * P) * u2);
        a0 = fmaf(-k.kgx, ux, fmaf(-k.kgy, uy, a0));
        g[0][j] = fmaf(wf(0), a0, k.omm * g[0][j]);
        bgk_pair(g[1][j], g[3][j], ux, k.A[0], k.B[0], wf(1), P, Qc, a0, k.omm);
        bgk_pair(g[2][j], g[4][j], uy, k.A[1], k.B[1], wf(2), P, Qc, a0, k.omm);
        bgk_pair(g[5][j], g[7][j], ux + uy, k.A[2], k.B[2], wf(5), P, Qc, a0, k.omm);
        bgk_pair(g[6][j], g[8][j], uy - ux, k.A[3], k.B[3], wf(6), P, Qc, a0, k.omm);
    } else {
        // F = 0: A = B = 0 and no force in a0 or u
        const float ux = jx * inv, uy = jy * inv;
        const float P = fmaf(k.om3, drho, k.om3);
        const float Qc = 1.5f * P;
        const float u2 = fmaf(ux, ux, uy * uy);
        const float a0 = fmaf(k.om, drho, -(0.5f * P) * u2);
        g[0][j] = fmaf(wf(0), a0, k.omm * g[0][j]);
        bgk_pair(g[1][j], g[3][j], ux, 0.0f, 0.0f, wf(1), P, Qc, a0, k.omm);
        bgk_pair(g[2][j], g[4][j], uy, 0.0f, 0.0f, wf(2), P, Qc, a0, k.omm);
        bgk_pair(g[5][j], g[7][j], ux + uy, 0.0f, 0.0f, wf(5), P, Qc, a0, k.omm);
        bgk_pair(g[6][j], g[8][j], uy - ux, 0.0f, 0.0f, wf(6), P, Qc, a0, k.omm);
    }
}

// central-moment collision of site j, in place on the carried values g = f - w
// (CmConsts): raw moments of g from the pair sums, the moments of
// f - f^eq + S/2 from the closed-form moments of the discrete equilibrium and
// of the Guo term, binomial shift to central moments, relaxation, shift back,
// and the D2Q9 inverse of the raw-moment transform.  FORCE = false: the same
// without body force (the open channel), the force terms compiled out
template <int V, bool FORCE = true>
__device__ __forceinline__ void cm_collide(float (&g)[9][V], int j, const BgkConsts& k, const CmConsts& m)
{
    const float s1 = g[1][j] + g[3][j], d1 = g[1][j] - g[3][j];
    const float s2 = g[2][j] + g[4][j], d2 = g[2][j] - g[4][j];
    const float s5 = g[5][j] + g[7][j], d5 = g[5][j] - g[7][j];
    const float s6 = g[6][j] + g[8][j], d6 = g[6][j] - g[8][j];
    const float drho = (g[0][j] + s1) + (s2 + (s5 + s6));
    const float jx = d1 + (d5 - d6), jy = d2 + (d5 + d6);
    const float rho = 1.0f + drho;
    const float inv = __fdividef(1.0f, rho);
    // raw moments of g
    const float m22 = s5 + s6, m20 = s1 + m22, m02 = s2 + m22, m11 = s5 - s6, m21 = d5 + d6, m12 = d5 - d6;
    if constexpr (FORCE) {
        const float ux = (jx + k.hgx) * inv, uy = (jy + k.hgy) * inv;
        const float fx = m.fx, fy = m.fy;
        // moments of f - f^eq + S/2 (those of order 0 and 1 vanish)
        const float rux = rho * ux, ruy = rho * uy, uF = ux * fx + uy * fy;
        const float M20 = m20 - drho * (1.0f / 3.0f) - rux * ux + ux * fx;
        const float M02 = m02 - drho * (1.0f / 3.0f) - ruy * uy + uy * fy;
        const float M11 = m11 - rux * uy + 0.5f * (ux * fy + uy * fx);
        const float M21 = m21 - ruy * (1.0f / 3.0f) + fy * (1.0f / 6.0f);
        const float M12 = m12 - rux * (1.0f / 3.0f) + fx * (1.0f / 6.0f);
        const float M22 = m22 - drho * (1.0f / 9.0f) - (rux * ux + ruy * uy) * (1.0f / 3.0f) + uF * (1.0f / 3.0f);
        // central moments, relaxed
        const float k21 = M21 - 2.0f * ux * M11 - uy * M20;
        const float k12 = M12 - 2.0f * uy * M11 - ux * M02;
        const float k22 = M22 - 2.0f * ux * M12 - 2.0f * uy * M21 + ux * ux * M02 + uy * uy * M20 + 4.0f * ux * uy * M11;
        const float r20 = m.a * M20 + m.b * M02, r02 = m.b * M20 + m.a * M02, r11 = m.ws * M11;
        const float r21 = m.w3 * k21, r12 = m.w3 * k12, r22 = m.w4 * k22;
        // back to raw moments
        const float R21 = r21 + 2.0f * ux * r11 + uy * r20;
        const float R12 = r12 + 2.0f * uy * r11 + ux * r02;
        const float R22 = r22 + 2.0f * ux * r12 + 2.0f * uy * r21 + ux * ux * r02 + uy * uy * r20 + 4.0f * ux * uy * r11;
        // Guo term S_q = w_q (3 c.F - 3 u.F + 9 (c.u)(c.F)) and the update g + S - x
        const float t0 = -3.0f * uF;
        g[0][j] = g[0][j] + wf(0) * t0 - (R22 - r20 - r02);
        const float cu1 = ux, cF1 = fx, cu2 = uy, cF2 = fy;
        const float cu5 = ux + uy, cF5 = fx + fy, cu6 = uy - ux, cF6 = fy - fx;
        const float e1 = t0 + 9.0f * cu1 * cF1, e2 = t0 + 9.0f * cu2 * cF2;
        const float e5 = t0 + 9.0f * cu5 * cF5, e6 = t0 + 9.0f * cu6 * cF6;
        g[1][j] = g[1][j] + wf(1) * (e1 + 3.0f * cF1) - 0.5f * (r20 - R12 - R22);
        g[3][j] = g[3][j] + wf(3) * (e1 - 3.0f * cF1) - 0.5f * (r20 + R12 - R22);
        g[2][j] = g[2][j] + wf(2) * (e2 + 3.0f * cF2) - 0.5f * (r02 - R21 - R22);
        g[4][j] = g[4][j] + wf(4) * (e2 - 3.0f * cF2) - 0.5f * (r02 + R21 - R22);
        g[5][j] = g[5][j] + wf(5) * (e5 + 3.0f * cF5) - 0.25f * (r11 + R21 + R12 + R22);
        g[7][j] = g[7][j] + wf(7) * (e5 - 3.0f * cF5) - 0.25f * (r11 - R21 - R12 + R22);
        g[6][j] = g[6][j] + wf(6) * (e6 + 3.0f * cF6) - 0.25f * (-r11 + R21 - R12 + R22);
        g[8][j] = g[8][j] + wf(8) * (e6 - 3.0f * cF6) - 0.25f * (-r11 - R21 + R12 + R22);
    } else {
        // the same collision with F = 0: no Guo term, u = sum c g / rho
        const float ux = jx * inv, uy = jy * inv;
        const float rux = rho * ux, ruy = rho * uy;
        const float M20 = m20 - drho * (1.0f / 3.0f) - rux * ux;
        const float M02 = m02 - drho * (1.0f / 3.0f) - ruy * uy;
        const float M11 = m11 - rux * uy;
        const float M21 = m21 - ruy * (1.0f / 3.0f);
        const float M12 = m12 - rux * (1.0f / 3.0f);
        const float M22 = m22 - drho * (1.0f / 9.0f) - (rux * ux + ruy * uy) * (1.0f / 3.0f);
        const float k21 = M21 - 2.0f * ux * M11 - uy * M20;
        const float k12 = M12 - 2.0f * uy * M11 - ux * M02;
        const float k22 = M22 - 2.0f * ux * M12 - 2.0f * uy * M21 + ux * ux * M02 + uy * uy * M20 + 4.0f * ux * uy * M11;
        const float r20 = m.a * M20 + m.b * M02, r02 = m.b * M20 + m.a * M02, r11 = m.ws * M11;
        const float r21 = m.w3 * k21, r12 = m.w3 * k12, r22 = m.w4 * k22;
        const float R21 = r21 + 2.0f * ux * r11 + uy * r20;
        const float R12 = r12 + 2.0f * uy * r11 + ux * r02;
        const float R22 = r22 + 2.0f * ux * r12 + 2.0f * uy * r21 + ux * ux * r02 + uy * uy * r20 + 4.0f * ux * uy * r11;
        g[0][j] = g[0][j] - (R22 - r20 - r02);
        g[1][j] = g[1][j] - 0.5f * (r20 - R12 - R22);
        g[3][j] = g[3][j] - 0.5f * (r20 + R12 - R22);
        g[2][j] = g[2][j] - 0.5f * (r02 - R21 - R22);
        g[4][j] = g[4][j] - 0.5f * (r02 + R21 - R22);
        g[5][j] = g[5][j] - 0.25f * (r11 + R21 + R12 + R22);
        g[7][j] = g[7][j] - 0.25f * (r11 - R21 - R12 + R22);
        g[6][j] = g[6][j] - 0.25f * (-r11 + R21 - R12 + R22);
        g[8][j] = g[8][j] - 0.25f * (-r11 - R21 + R12 + R22);
    }
}

// the collision selected at compile time: 0 BGK, 1 central moments
template <int COLL, int V>
__device__ __forceinline__ void collide(float (&g)[9][V], int j, const StepParams& p)
{
    if constexpr (COLL == 0)
        bgk_collide<V>(g, j, p.bgk);
    else
        cm_collide<V>(g, j, p.bgk, p.cm);
}

// the same collision at the relaxation rate om of a sponge column, without
// body force (open channel, Sec. 2: the force terms are compiled out and only
// the rate-dependent constants change; the central-moment collision relaxes
// the shear moments at om)
template <int COLL, int V>
__device__ __forceinline__ void collide_at(float (&g)[9][V], int j, const StepParams& p, float om)
{
    BgkConsts k = p.bgk;
    k.om = om;
    k.omm = 1.0f - om;
    k.om3 = 3.0f * om;
    if constexpr (COLL == 0) {
        bgk_collide<V, false>(g, j, k);
    } else {
        CmConsts m = p.cm;
        m.ws = om;
        m.a = 0.5f * (m.wb + om);
        m.b = 0.5f * (m.wb - om);
        cm_collide<V, false>(g, j, k, m);
    }
}

// velocity sum c f / sum f of a node from its carried values g = f - w (no
// body force: the velocity of a post-collision state of an open channel)
__device__ __forceinline__ void open_velocity9(const float (&g)[9], float& ux, float& uy)
{
    const float drho = (g[0] + (g[1] + g[3])) + ((g[2] + g[4]) + ((g[5] + g[7]) + (g[6] + g[8])));
    const float jx = (g[1] - g[3]) + ((g[5] - g[7]) - (g[6] - g[8]));
    const float jy = (g[2] - g[4]) + ((g[5] - g[7]) + (g[6] - g[8]));
    const float inv = 1.0f / (1.0f + drho);
    ux = jx * inv;
    uy = jy * inv;
}

// carried value g_q = f_q - w_q of the open channel's outlet column (x = nx - 1)
// at one row, regularized (Latt et al. 2008) from the velocities of columns
// nx-2 and nx-3:
//   rho = 1,  u = 2 u(nx-2) - u(nx-3),
//   f_q = f_q^eq(1, u) + w_q / (2 cs2^2) Q_q : Pi,  Q_q = c_q c_q - cs2 I,
//   Pi = bc_pre S,  bc_pre = -2 cs2 (tau(nx-1) - 1),
// S the strain rate by finite differences: x one-sided from the two upstream
// columns, y central on the extrapolated column (one-sided on the wall rows).
// Every operation is rounded explicitly (no contraction), so that the kernel
// that stores the column and a step that pulls from it without the stored
// column (outlet_from_u) compute the same value bit for bit.
// the twelve velocity components one outlet row needs: columns nx-2 (2) and
// nx-3 (3) at the row itself and at its neighbours ym, yp (the row itself on a
// wall row), and whether the y difference spans two rows
struct OutletU {
    float u2, v2, u3, v3;          // row y
    float u2m, u3m, v2m, v3m;      // row ym
    float u2p, u3p, v2p, v3p;      // row yp
    bool two;                      // yp - ym == 2
};

__device__ __forceinline__ float outlet_g(const OutletU& a, float cxq, float cyq, float wq, float bc_pre)
{
    const float exm = __fsub_rn(__fmul_rn(2.0f, a.u2m), a.u3m);
    const float exp_ = __fsub_rn(__fmul_rn(2.0f, a.u2p), a.u3p);
    const float eym = __fsub_rn(__fmul_rn(2.0f, a.v2m), a.v3m);
    const float eyp = __fsub_rn(__fmul_rn(2.0f, a.v2p), a.v3p);
    const float inv_dy = a.two ? 0.5f : 1.0f;
    const float dxux = __fsub_rn(a.u2, a.u3), dxuy = __fsub_rn(a.v2, a.v3);
    const float dyux = __fmul_rn(__fsub_rn(exp_, exm), inv_dy), dyuy = __fmul_rn(__fsub_rn(eyp, eym), inv_dy);
    const float pxx = __fmul_rn(bc_pre, dxux), pyy = __fmul_rn(bc_pre, dyuy);
    const float pxy = __fmul_rn(__fmul_rn(bc_pre, 0.5f), __fadd_rn(dyux, dxuy));
    const float ux = __fsub_rn(__fmul_rn(2.0f, a.u2), a.u3), uy = __fsub_rn(__fmul_rn(2.0f, a.v2), a.v3);
    const float usq = __fadd_rn(__fmul_rn(ux, ux), __fmul_rn(uy, uy));
    const float cu = __fadd_rn(__fmul_rn(cxq, ux), __fmul_rn(cyq, uy));
    const float qp = __fadd_rn(__fadd_rn(__fmul_rn(__fsub_rn(__fmul_rn(cxq, cxq), 1.0f / 3.0f), pxx),
                                         __fmul_rn(__fmul_rn(2.0f * cxq, cyq), pxy)),
                               __fmul_rn(__fsub_rn(__fmul_rn(cyq, cyq), 1.0f / 3.0f), pyy));
    const float t = __fadd_rn(__fsub_rn(__fadd_rn(__fmul_rn(3.0f, cu), __fmul_rn(__fmul_rn(4.5f, cu), cu)),
                                        __fmul_rn(1.5f, usq)),
                              __fmul_rn(4.5f, qp));
    return __fmul_rn(wq, t);
}

// the velocities of outlet row y from the buffer the step kernel writes
__device__ __forceinline__ OutletU outlet_u_at(const float* __restrict__ u, int ny, int y)
{
    const int ym = y > 0 ? y - 1 : y, yp = y < ny - 1 ? y + 1 : y;
    OutletU a;
    // written by the step kernel just before (L2 loads)
    a.u2 = __ldcg(u + y);
    a.v2 = __ldcg(u + ny + y);
    a.u3 = __ldcg(u + 2 * ny + y);
    a.v3 = __ldcg(u + 3 * ny + y);
    a.u2m = __ldcg(u + ym);
    a.u3m = __ldcg(u + 2 * ny + ym);
    a.v2m = __ldcg(u + ny + ym);
    a.v3m = __ldcg(u + 3 * ny + ym);
    a.u2p = __ldcg(u + yp);
    a.u3p = __ldcg(u + 2 * ny + yp);
    a.v2p = __ldcg(u + ny + yp);
    a.v3p = __ldcg(u + 3 * ny + yp);
    a.two = yp - ym == 2;
    return a;
}

// The pulls of a step whose previous step (in the same chunk) left the outlet
// column unwritten: directions 3, 6 and 7 at column nx - 2 come from the outlet
// at rows y, y - 1 and y + 1.  The warp holding column nx - 2 loads the twenty
// velocity values of rows y - 2 .. y + 2 (clamped to the channel) in phase 1,
// one per lane; lanes 0, 1 and 2 gather by shuffles what their outlet row
// needs and compute one direction each, in the storage format and back (as a
// pull from the stored column would load it); the owner of column nx - 2 takes
// the three values by shuffles.
struct OutletPrefetch {
    float v;    // lane l < 20: component l / 5 at row clamp(y - 2 + l % 5)
};

__device__ __forceinline__ OutletPrefetch outlet_prefetch(const StepParams& p, int y, int lane)
{
    OutletPrefetch f{0.f};
    if (lane < 20) {
        int r = y - 2 + lane % 5;
        r = r < 0 ? 0 : (r >= p.ny ? p.ny - 1 : r);
        f.v = __ldcg(p.open_u_prev + ((int64_t)blockIdx.z * 4 + lane / 5) * p.ny + r);
    }
    return f;
}

template <int S, bool SCALED>
__device__ __forceinline__ void outlet_pulls(const StepParams& p, const OutletPrefetch& f, int y, int lane,
                                             float& g3, float& g6, float& g7)
{
    using K = Carry<S, SCALED>;
    // lane 0: direction 3 from row y; lane 1: 6 from row y - 1; lane 2: 7 from row y + 1
    const int k = lane < 3 ? lane : 0;
    const int yo_raw = y + (k == 1 ? -1 : (k == 2 ? 1 : 0));
    const int yo = yo_raw < 0 ? 0 : (yo_raw >= p.ny ? p.ny - 1 : yo_raw);
    const int ym = yo > 0 ? yo - 1 : yo, yp = yo < p.ny - 1 ? yo + 1 : yo;
    // rows yo, ym, yp lie within y - 2 .. y + 2: index component * 5 + (row - y + 2)
    auto at = [&](int comp, int row) { return __shfl_sync(0xffffffffu, f.v, comp * 5 + (row - y + 2)); };
    OutletU a;
    a.u2 = at(0, yo);
    a.v2 = at(1, yo);
    a.u3 = at(2, yo);
    a.v3 = at(3, yo);
    a.u2m = at(0, ym);
    a.v2m = at(1, ym);
    a.u3m = at(2, ym);
    a.v3m = at(3, ym);
    a.u2p = at(0, yp);
    a.v2p = at(1, yp);
    a.u3p = at(2, yp);
    a.v3p = at(3, yp);
    a.two = yp - ym == 2;
    const int q = k == 0 ? 3 : (k == 1 ? 6 : 7);
    const float wq = k == 0 ? wf(3) : wf(6);
    const float r = K::in(K::out(outlet_g(a, -1.0f, k == 0 ? 0.0f : (k == 1 ? 1.0f : -1.0f), wq, p.bc_pre), wq,
                                 p.scale),
                          wq, p.inv_scale);
    (void)q;
    g3 = __shfl_sync(0xffffffffu, r, 0);
    g6 = __shfl_sync(0xffffffffu, r, 1);
    g7 = __shfl_sync(0xffffffffu, r, 2);
}

template <int S, int V, bool GENERAL, bool SCALED, int COLL, bool OPEN>
__device__ __forceinline__ void step_warp(const StepParams& p, const typename Codec<S>::T* __restrict__ src,
                                          typename Codec<S>::T* __restrict__ dst, int c, int y, int seg, int lane,
                                          bool grid_warp = false)
{
    using T = typename Codec<S>::T;
    using K = Carry<S, SCALED>;
    const int x0 = seg * 32 * V + lane * V;
    const bool active = x0 < p.nx;
    const int row = y * p.pitch;
    const int plane = (int)p.plane;  // a clone holds < 2^31 values (checked at creation)
    const int ox0 = p.ox0, ox1 = p.ox1, oy0 = p.oy0, oy1 = p.oy1;

    // ---- phase 1: issue every load
    Vec<T, V> v[9];
    T edge[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int ex = cx(q), ey = cy(q);
        int srow = y - ey;
        int plane_q = q;
        if (GENERAL && (srow < 0 || srow >= p.ny)) {
            // the wall sends back the population that left this node
            srow = y;
            plane_q = opp(q);
        }
        const T* rp = src + plane_q * plane + srow * p.pitch;
        if constexpr (OPEN) {
            // lanes past the last column (nx need not be a multiple of 32 V)
            // feed only the outlet column, which the boundary kernel rewrites
            if (active)
                v[q] = ld_stream<T, V>(rp + x0);
            else
                v[q] = Vec<T, V>{};
        } else {
            v[q] = ld_stream<T, V>(rp + x0);
        }
        if (ex == 1) {
            const int xs = x0 == 0 ? p.nx - 1 : x0 - 1;
            if (lane == 0 || x0 == 0) edge[q] = ld_one(rp + xs);
        } else if (ex == -1) {
            const int xs = x0 + V >= p.nx ? 0 : x0 + V;
            if (lane == 31 || x0 + V >= p.nx) edge[q] = ld_one(rp + xs);
        }
    }

    // the warp holding column nx - 2 of an open channel, inside a chunk: the
    // velocities for the outlet it pulls from, loaded with the populations
    const bool outlet_warp = OPEN && p.outlet_from_u && seg * 32 * V <= p.nx - 2 && p.nx - 2 < (seg + 1) * 32 * V;
    OutletPrefetch opf{0.f};
    if constexpr (OPEN) {
        if (outlet_warp) opf = outlet_prefetch(p, y, lane);
    }

    // ---- phase 2: assemble the pulled values of the V sites
    float g[9][V];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        const int ex = cx(q), ey = cy(q);
        const bool wall = GENERAL && ((y - ey) < 0 || (y - ey) >= p.ny);
        float d[V];
        if constexpr (V % 2 == 0) {
#pragma unroll
            for (int j = 0; j < V; j += 2) {
                const float2 f = K::in2(&v[q].e[j], wf(q), p.inv_scale);
                d[j] = f.x;
                d[j + 1] = f.y;
            }
        } else {
#pragma unroll
            for (int j = 0; j < V; ++j) d[j] = K::in(v[q].e[j], wf(q), p.inv_scale);
        }
        if (ex == 0 || wall) {
#pragma unroll
            for (int j = 0; j < V; ++j) g[q][j] = d[j];
        } else if (ex == 1) {
            float e = __shfl_up_sync(0xffffffffu, d[V - 1], 1);
            if (lane == 0 || x0 == 0) e = K::in(edge[q], wf(q), p.inv_scale);
            g[q][0] = e;
#pragma unroll
            for (int j = 1; j < V; ++j) g[q][j] = d[j - 1];
        } else {
            float e = __shfl_down_sync(0xffffffffu, d[0], 1);
            if (lane == 31 || x0 + V >= p.nx) e = K::in(edge[q], wf(q), p.inv_scale);
#pragma unroll
            for (int j = 0; j < V - 1; ++j) g[q][j] = d[j + 1];
            g[q][V - 1] = e;
        }
    }
    if constexpr (OPEN) {
        if (GENERAL || grid_warp) {
            // links whose upstream node is solid (the square, or a bar of the
            // open channel's grid) bounce back at this node; the bar rows among
            // y - 1, y, y + 1 from one remainder.  Warps around the grid that
            // are not wall or ring warps come here from the test-free path.
            const int r0 = y % p.gperiod;
            const bool bar_m = y > 0 && (r0 == 0 ? p.gperiod - 1 : r0 - 1) >= p.ggap;
            const bool bar_0 = r0 >= p.ggap;
            const bool bar_p = y + 1 < p.ny && (r0 + 1 == p.gperiod ? 0 : r0 + 1) >= p.ggap;
#pragma unroll
            for (int q = 1; q < 9; ++q) {
                const int ex = cx(q), ys = y - cy(q);
                const bool sq_row = ys >= oy0 && ys < oy1;
                const bool grid_row = cy(q) == 1 ? bar_m : (cy(q) == 0 ? bar_0 : bar_p);
                if (!sq_row && !grid_row) continue;
                bool hit[V];
                bool any = false;
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const int xs = x0 + j - ex;
                    hit[j] = (sq_row && xs >= ox0 && xs < ox1) || (grid_row && xs >= p.gx0 && xs < p.gx1);
                    any |= hit[j];
                }
                if (any) {
                    const Vec<T, V> o = ld_stream<T, V>(src + opp(q) * plane + row + x0);
#pragma unroll
                    for (int j = 0; j < V; ++j)
                        if (hit[j]) g[q][j] = K::in(o.e[j], wf(q), p.inv_scale);
                }
            }
        }
    } else if (GENERAL && ox1 > ox0) {
        // links whose upstream node is solid bounce back at this node
#pragma unroll
        for (int q = 1; q < 9; ++q) {
            const int ex = cx(q), ys = y - cy(q);
            if (ys < oy0 || ys >= oy1) continue;
            bool any = false;
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int xs = x0 + j - ex;
                any |= (xs >= ox0 && xs < ox1);
            }
            if (any) {
                const Vec<T, V> o = ld_stream<T, V>(src + opp(q) * plane + row + x0);
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const int xs = x0 + j - ex;
                    if (xs >= ox0 && xs < ox1) g[q][j] = K::in(o.e[j], wf(q), p.inv_scale);
                }
            }
        }
    }

    if constexpr (OPEN) {
        // the previous step of this chunk left the outlet column unwritten: the
        // pulls from it (directions 3, 6 and 7 at column nx - 2, from rows y,
        // y - 1 and y + 1) take the outlet that step's velocities give, as the
        // stored column would hold it; a wall row keeps its bounce-back
        if (outlet_warp) {
            float o3, o6, o7;
            outlet_pulls<S, SCALED>(p, opf, y, lane, o3, o6, o7);
#pragma unroll
            for (int j = 0; j < V; ++j)
                if (x0 + j == p.nx - 2) {
                    g[3][j] = o3;
                    if (y > 0) g[6][j] = o6;
                    if (y + 1 < p.ny) g[7][j] = o7;
                }
        }
    }

    // ---- phase 3: BGK collision with Guo forcing
    if constexpr (OPEN) {
        // one collision body per site: the rate of a sponge column, else 1/tau
        const bool sponge = x0 + V > p.sx0;
#pragma unroll
        for (int j = 0; j < V; ++j) {
            const int x = x0 + j;
            const float om = sponge && x >= p.sx0 && x < p.nx ? __ldg(p.om_col + x) : p.bgk.om;
            collide_at<COLL, V>(g, j, p, om);
        }
    } else {
#pragma unroll
        for (int j = 0; j < V; ++j) collide<COLL, V>(g, j, p);
    }
    if constexpr (OPEN) {
        if ((GENERAL || grid_warp) && y % p.gperiod >= p.ggap) {  // this row is a bar row
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int x = x0 + j;
                if (x >= p.gx0 && x < p.gx1) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) g[q][j] = 0.f;  // a bar of the grid: rest state
                }
            }
        }
        // the inlet column holds the equilibrium of the inlet profile
        if (x0 == 0) {
#pragma unroll
            for (int q = 0; q < 9; ++q) g[q][0] = __ldg(p.inlet_g + q * p.ny + y);
        }
        // an open channel's nx need not be a multiple of V: sites past the
        // last column (row padding) are kept at rest
        if (x0 + V > p.nx) {
#pragma unroll
            for (int j = 0; j < V; ++j)
                if (x0 + j >= p.nx) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) g[q][j] = 0.f;
                }
        }
        // the velocities of columns nx-2 and nx-3 as they are stored (encoded
        // and decoded), from which the boundary kernel extrapolates the outlet
        if (x0 + V > p.nx - 3 && x0 <= p.nx - 2) {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int x = x0 + j;
                if (x == p.nx - 2 || x == p.nx - 3) {
                    float h[9];
#pragma unroll
                    for (int q = 0; q < 9; ++q) h[q] = K::in(K::out(g[q][j], wf(q), p.scale), wf(q), p.inv_scale);
                    float ux, uy;
                    open_velocity9(h, ux, uy);
                    float* u = p.open_u + ((int64_t)blockIdx.z * 4 + (x == p.nx - 2 ? 0 : 2)) * p.ny + y;
                    u[0] = ux;
                    u[p.ny] = uy;
                }
            }
        }
    }

    if (GENERAL && ox1 > ox0) {
        if (y >= oy0 && y < oy1) {
#pragma unroll
            for (int j = 0; j < V; ++j) {
                const int x = x0 + j;
                if (x >= ox0 && x < ox1) {
#pragma unroll
                    for (int q = 0; q < 9; ++q) g[q][j] = 0.f;  // solid node: rest state f = w
                }
            }
        }
        // momentum exchange with the obstacle, one partial per warp of the ring
        if (y >= p.ry0 && y <= p.ry1 && seg >= p.rs0 && seg <= p.rs1) {
            float acc = 0.f;
            if (active) {
#pragma unroll
                for (int j = 0; j < V; ++j) {
                    const int x = x0 + j;
                    if (y >= oy0 && y < oy1 && x >= ox0 && x < ox1) continue;
#pragma unroll
                    for (int q = 1; q < 9; ++q) {
                        if (cx(q) == 0) continue;
                        const int xn = x + cx(q), yn = y + cy(q);
                        if (xn >= ox0 && xn < ox1 && yn >= oy0 && yn < oy1) {
                            acc += 2.0f * (float)cx(q) * (wf(q) + g[q][j]);
                        }
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
    }

    // ---- phase 4: store
    if (active) {
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
            st_stream<T, V>(dst + q * plane + row + x0, o);
        }
    }
}

// ---------------------------------------------------------------- open channel
// Boundary columns of the open channel (Sec. 2), in the state a step launch
// produces (post-collision populations):
//   inlet  x = 0:      f = f^eq(rho = 1, (u_in(y), 0)): the step kernel's
//                      thread for x = 0 stores p.inlet_g (FP64 on the host,
//                      then FP32) instead of its collision result;
//   outlet x = nx-1:   rho = 1 and u = 2 u(nx-2) - u(nx-3), the populations
//                      regularized (Latt et al. 2008):
//                      f = f^eq(1, u) + w_q / (2 cs2^2) Q_q : Pi,  Q_q = c_q c_q - cs2 I,
//                      Pi = bc_pre * S,  bc_pre = -2 cs2 (tau(nx-1) - 1),
//                      S the strain rate by finite differences: x one-sided from
//                      the two upstream columns, y central on the extrapolated
//                      column (one-sided on the wall rows).
// The threads that own columns nx-2 and nx-3 leave their velocities (as
// stored) in p.open_u ([list index][ux(nx-2), uy(nx-2), ux(nx-3), uy(nx-3)][ny],
// one buffer per step parity).  Within a chunk of steps the outlet column is
// not written: the next step's thread of column nx-2 computes the three outlet
// populations it pulls from those velocities (outlet_from_u).  After the
// chunk's last step open_bc_kernel writes the column from them, so that every
// state seen outside a chunk (checkpoints, copies, reads) is whole.  A row
// segment that would hold column nx-1 alone is not launched.  (Writing the outlet from the
// block that finishes last for each clone instead, with an arrival counter,
// measured slower: every block waits at a barrier before it can retire, and
// the last clone's outlet lands on the kernel's tail.)

// outlet populations of row y of listed clone li, into the state st
template <int S, bool SCALED>
__device__ __forceinline__ void open_outlet_row(const StepParams& p, typename Codec<S>::T* st, int li, int y)
{
    using K = Carry<S, SCALED>;
    const float* u = p.open_u + (int64_t)li * 4 * p.ny;
    typename Codec<S>::T* o = st + (int64_t)y * p.pitch + (p.nx - 1);
    const OutletU a = outlet_u_at(u, p.ny, y);
#pragma unroll
    for (int q = 0; q < 9; ++q)
        o[q * p.plane] = K::out(outlet_g(a, (float)cx(q), (float)cy(q), wf(q), p.bc_pre), wf(q), p.scale);
}

// one warp's row segment of a fused-step launch (grid: segments, row blocks,
// listed clones)
template <int S, int V, int WARPS, bool SCALED, int COLL, bool OPEN>
__device__ __forceinline__ void step_block(const StepParams& p)
{
    using T = typename Codec<S>::T;
    const int lane = threadIdx.x;
    const int y = blockIdx.y * WARPS + threadIdx.y;
    if (y >= p.ny) return;  // warp-uniform
    const int seg = blockIdx.x;
    const int c = p.clone_list[blockIdx.z];
    const int cur = p.parity[c] ^ (p.step_in_batch & 1);
    const T* src = static_cast<const T*>(cur ? p.buf1 : p.buf0) + (int64_t)c * p.clone_stride;
    T* dst = static_cast<T*>(cur ? p.buf0 : p.buf1) + (int64_t)c * p.clone_stride;
    const bool wall_row = y == 0 || y == p.ny - 1;
    const bool ring = p.ox1 > p.ox0 && y >= p.ry0 && y <= p.ry1 && seg >= p.rs0 && seg <= p.rs1;
    if constexpr (OPEN) {
        // segments around the entrance grid, in rows that are bars or next to
        // one (a row whose neighbours are fluid has no link into a bar)
        bool grid = false;
        if (seg >= p.gs0 && seg <= p.gs1) {
            const bool bar = y % p.gperiod >= p.ggap;
            const bool bar_below = y > 0 && (y - 1) % p.gperiod >= p.ggap;
            const bool bar_above = y + 1 < p.ny && (y + 1) % p.gperiod >= p.ggap;
            grid = bar || bar_below || bar_above;
        }
        if (wall_row || ring)
            step_warp<S, V, true, SCALED, COLL, true>(p, src, dst, c, y, seg, lane, grid);
        else
            step_warp<S, V, false, SCALED, COLL, true>(p, src, dst, c, y, seg, lane, grid);
    } else {
        if (wall_row || ring)
            step_warp<S, V, true, SCALED, COLL, false>(p, src, dst, c, y, seg, lane);
        else
            step_warp<S, V, false, SCALED, COLL, false>(p, src, dst, c, y, seg, lane);
    }
}

// the periodic channel's fused step
template <int S, int V, int WARPS, bool SCALED, int COLL>
__global__ void __launch_bounds__(WARPS * 32) step_kernel(const StepParams p)
{
    step_block<S, V, WARPS, SCALED, COLL, false>(p);
}

// the open channel's fused step
template <int S, int V, int WARPS, bool SCALED, int COLL>
__global__ void __launch_bounds__(WARPS * 32) step_kernel_open(const StepParams p)
{
    step_block<S, V, WARPS, SCALED, COLL, true>(p);
}

// the same held to 64 registers, for 16-bit storage at up to 4 sites per
// thread: 32 resident warps per SM instead of 24; issue-bound, it gains more
// from the warps in flight than it loses to a few spilled bytes (FP32 storage
// measured slower so)
template <int S, int V, int WARPS, bool SCALED, int COLL>
__global__ void __launch_bounds__(WARPS * 32, 1024 / (WARPS * 32)) step_kernel_open64(const StepParams p)
{
    step_block<S, V, WARPS, SCALED, COLL, true>(p);
}

// the outlet column of an open channel, one thread per (row, listed clone),
// launched after the step on the same stream
constexpr int kBcThreads = 128;

template <int S, bool SCALED>
__global__ void __launch_bounds__(kBcThreads) open_bc_kernel(const StepParams p)
{
    using T = typename Codec<S>::T;
    const int y = blockIdx.x * kBcThreads + threadIdx.x;
    const int li = blockIdx.y;
    const int c = p.clone_list[li];
    const int cur = p.parity[c] ^ (p.step_in_batch & 1);
    T* st = static_cast<T*>(cur ? p.buf0 : p.buf1) + (int64_t)c * p.clone_stride;
    if (y < p.ny) open_outlet_row<S, SCALED>(p, st, li, y);
}

template <int S, int V, int WARPS>
cudaError_t launch_step(const StepParams& p, cudaStream_t s)
{
    const dim3 block(32, WARPS);
    const dim3 grid(p.nseg, (p.ny + WARPS - 1) / WARPS, p.n_list);
    auto go = [&](auto coll) {
        constexpr int C = decltype(coll)::value;
        if constexpr (S == kFP32) {
            step_kernel<S, V, WARPS, false, C><<<grid, block, 0, s>>>(p);
        } else {
            if (p.scale == 1.0f)
                step_kernel<S, V, WARPS, false, C><<<grid, block, 0, s>>>(p);
            else
                step_kernel<S, V, WARPS, true, C><<<grid, block, 0, s>>>(p);
        }
    };
    if (p.coll == 1)
        go(std::integral_constant<int, 1>{});
    else
        go(std::integral_constant<int, 0>{});
    return cudaGetLastError();
}

// one step of an open channel: the fused step's open-channel instantiation
// (which also writes the inlet column), then, after a chunk's last step, the
// outlet column.  (Launching
// the outlet kernel as a programmatic dependent of the step measured slower:
// its waiting blocks hold SM slots during the step's tail.)
template <int S, int V, int WARPS>
cudaError_t launch_step_open(const StepParams& p, cudaStream_t s)
{
    const dim3 block(32, WARPS);
    const dim3 grid(p.nseg, (p.ny + WARPS - 1) / WARPS, p.n_list);
    const dim3 bc_grid((p.ny + kBcThreads - 1) / kBcThreads, p.n_list);
    auto go = [&](auto coll, auto scaled) {
        constexpr int C = decltype(coll)::value;
        constexpr bool SC = decltype(scaled)::value;
        if constexpr (S != kFP32 && V <= 4)
            step_kernel_open64<S, V, WARPS, SC, C><<<grid, block, 0, s>>>(p);
        else
            step_kernel_open<S, V, WARPS, SC, C><<<grid, block, 0, s>>>(p);
        if (p.write_outlet) open_bc_kernel<S, SC><<<bc_grid, kBcThreads, 0, s>>>(p);
    };
    auto by_scale = [&](auto coll) {
        if constexpr (S == kFP32) {
            go(coll, std::false_type{});
        } else {
            if (p.scale != 1.0f)
                go(coll, std::true_type{});
            else
                go(coll, std::false_type{});
        }
    };
    if (p.coll == 1)
        by_scale(std::integral_constant<int, 1>{});
    else
        by_scale(std::integral_constant<int, 0>{});
    return cudaGetLastError();
}

}  // namespace lbm
