// Launch parameters of the fused step kernels: the only host data a step
// kernel reads.  Kept apart from the runtime's other internals so that a
// change here, and only here or in the kernels, changes what was profiled.
#pragma once
#include <cstdint>

namespace lbm {

// Constants of the BGK collision with Guo forcing, in the pairwise form the
// step kernels use (the BGK collision and D2Q9 equilibrium of App. A with
// Guo's body-force term, expanded).  With the carried value g = f - w,
// drho = sum g, u = (sum c g + F/2) / rho and kap3 = 3 (1 - om/2), the
// post-collision value of direction q is
//   g*_q = (1 - om) g_q + w_q t_q,
//   t_q  = a0 + kap3 cF + cu (3 om rho + 3 kap3 cF + 4.5 om rho cu),
//   a0   = om drho - 1.5 om rho u.u - kap3 u.F,   cu = c_q.u,  cF = c_q.F.
// For the opposite direction cu and cF change sign, so a pair shares
//   E = a0 + cu (A + 4.5 om rho cu),  O = B + 3 om rho cu,
//   t_q = E + O,  t_opp = E - O,      A = 3 kap3 cF,  B = kap3 cF,
// for the pairs (1,3), (2,4), (5,7), (6,8) with cF = F_x, F_y, F_x + F_y,
// F_y - F_x.  Computed once on the host so that every kernel reads them as
// launch constants.
struct BgkConsts {
    float om, omm, om3;  // omega, 1 - omega, 3 omega
    float hgx, hgy;      // F/2
    float kgx, kgy;      // kap3 F
    float A[4], B[4];    // per direction pair
};

inline BgkConsts bgk_consts(float om, float gx, float gy)
{
    BgkConsts k;
    const float kap3 = 3.0f * (1.0f - 0.5f * om);
    k.om = om;
    k.omm = 1.0f - om;
    k.om3 = 3.0f * om;
    k.hgx = 0.5f * gx;
    k.hgy = 0.5f * gy;
    k.kgx = kap3 * gx;
    k.kgy = kap3 * gy;
    const float cf[4] = {gx, gy, gx + gy, gy - gx};
    for (int i = 0; i < 4; ++i) {
        k.B[i] = kap3 * cf[i];
        k.A[i] = 3.0f * k.B[i];
    }
    return k;
}

// Constants of the central-moment collision (the multiple-relaxation-time
// collision on central moments of App. A's production runs), the
// generalisation of the BGK collision above:
//   g* = g + S - T^{-1} Omega T (f - f^eq + S/2),
// T(u) the D2Q9 central-moment transform (moments 00 10 01 20 02 11 21 12 22),
// f^eq the same discrete equilibrium, S the Guo term.  Omega relaxes k20 - k02
// and k11 at ws = 1/tau, k20 + k02 at wb, k21 and k12 at w3, k22 at w4; equal
// rates give the BGK collision exactly.
struct CmConsts {
    float ws, wb, w3, w4;
    float a, b;    // (wb + ws)/2 and (wb - ws)/2: the k20, k02 block of Omega
    float fx, fy;  // F
};

inline CmConsts cm_consts(float ws, float wb, float w3, float w4, float gx, float gy)
{
    CmConsts m;
    m.ws = ws;
    m.wb = wb;
    m.w3 = w3;
    m.w4 = w4;
    m.a = 0.5f * (wb + ws);
    m.b = 0.5f * (wb - ws);
    m.fx = gx;
    m.fy = gy;
    return m;
}

// Everything one fused stream-collide launch needs.  Populations of clone c
// live at buf[p] + c * clone_stride, direction q at + q * plane, row y at
// + y * pitch; p alternates per clone with its own parity.
struct StepParams {
    void* buf0;
    void* buf1;
    const int32_t* parity;      // [N] current buffer of each clone
    const int32_t* clone_list;  // clones advanced by this launch
    int32_t n_list;
    int32_t nx, ny, pitch;
    int64_t plane, clone_stride;
    int32_t nseg;               // row segments of 32*V sites
    // obstacle: solid cells [ox0, ox1) x [oy0, oy1); ox1 == ox0 for none
    int32_t ox0, ox1, oy0, oy1;
    // drag ring: rows [ry0, ry1], segments [rs0, rs1]; one partial per warp
    int32_t ry0, ry1, rs0, rs1, n_slots, batch_cap;
    float* partials;            // [N][batch_cap][n_slots]
    float omega;                // 1/tau
    float gx, gy;               // body-force density
    float scale, inv_scale;     // 16-bit shift scale 2^s and its inverse
    int32_t step_in_batch;
    int32_t* err_flag;          // set to 1 when a bounded device-side wait runs out (may be null)
    BgkConsts bgk;              // bgk_consts(omega, gx, gy)
    int32_t coll;               // 0: BGK; 1: central-moment collision with cm
    CmConsts cm;
    // open channel (Sec. 2; launched through the open-channel instantiations
    // only): the grid of bars, the sponge and the two boundary columns
    int32_t open;               // 1: open channel
    int32_t gx0, gx1, ggap, gperiod;  // grid cells x in [gx0, gx1), y mod gperiod >= ggap
    int32_t gs0, gs1;           // segments whose warps take the general path for the grid
    int32_t sx0;                // first sponge column (nx: no sponge)
    const float* om_col;        // [nx] relaxation rate 1/tau(x) of each column
    const float* inlet_g;       // [9][ny] inlet populations minus w_q (FP32 of the FP64 values)
    float bc_pre;               // outlet stress factor -2 cs2 (tau(nx-1) - 1)
    float* open_u;              // [list index][4][ny] velocities of columns nx-2, nx-3 (this step writes)
    const float* open_u_prev;   // the same, written by the previous step of the chunk
    int32_t outlet_from_u;      // 1: the pulls from the outlet column use the outlet computed from
                                // open_u_prev (the previous step left that column unwritten)
    int32_t write_outlet;       // 1: the launch also writes the outlet column (the chunk's last step)
    int32_t tb_steps;           // steps of one launch of the temporally blocked kernel (odd)
};

// consumer warps of the row-staged step kernel; each writes its own drag
// partial for every obstacle-ring row it computes
constexpr int kRowWarps = 8;

// the temporally blocked step kernel: tiles of kTbTx x kTbTy sites with a halo
// of kTbHalo sites (a 32 x 16 region, one site per thread), at most kTbHalo
// steps per launch; one drag partial per tile of the obstacle ring and step
constexpr int kTbHalo = 3, kTbRw = 32, kTbRh = 16;
constexpr int kTbTx = kTbRw - 2 * kTbHalo, kTbTy = kTbRh - 2 * kTbHalo;  // 26 x 10
constexpr int kTbThreads = kTbRw * kTbRh;                              // 512

}  // namespace lbm
