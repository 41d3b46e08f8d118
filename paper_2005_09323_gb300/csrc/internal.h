// Host-side internals shared by the translation units of liblbmrare.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "lbmrare.h"

namespace lbm {

void set_error(const std::string& msg);
// every kernel the library launches is counted (lbm_launch_count)
void count_launches(int64_t n);
int fail(int code, const std::string& msg);
int cuda_fail(cudaError_t err, const char* what);

#define LBM_CUDA(call)                                        \
    do {                                                      \
        cudaError_t err_ = (call);                            \
        if (err_ != cudaSuccess) return cuda_fail(err_, #call); \
    } while (0)

// Everything one fused stream-collide launch needs.  Populations of clone c
// live at buf[p] + c * clone_stride, direction q at + q * plane, row y at
// + y * pitch; p alternates per clone with its own parity.
// Constants of the BGK collision with Guo forcing, in the pairwise form the
// step kernels use (the BGK collision and D2Q9 equilibrium of App. A with
// Guo's body-force term, expanded).  With the
// carried value g = f - w, drho = sum g, u = (sum c g + F/2) / rho and
// kap3 = 3 (1 - om/2), the post-collision value of direction q is
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
};

// consumer warps of the row-staged step kernel; each writes its own drag
// partial for every obstacle-ring row it computes
constexpr int kRowWarps = 8;

struct StepVariant {
    int storage;
    int vec;    // sites per thread
    int warps;  // warps per block
    cudaError_t (*launch)(const StepParams&, cudaStream_t);
    int kind;   // 0: register-staged row segments per warp; 1: whole rows staged by bulk copies
    bool (*supports)(const StepParams&);  // null: every shape
};

// all compiled variants of the fused step (lbm_step.cu)
const std::vector<StepVariant>& step_variants();

// network input of clones listed on the device (cnn.cu); no synchronisation
int fields_launch(lbm_ensemble* e, const int32_t* list_dev, int32_t n, int32_t factor, float rho_scale, float u_scale,
                  void* dst_dev);
// learned score of the listed clones (host list) into out[c * stride + k] (surrogate.cu)
int score_clones(lbm_ensemble* e, const int32_t* clones, int32_t n, double* out, int32_t stride, int32_t k);

}  // namespace lbm

struct cnn_model;

struct lbm_ensemble {
    lbm_config cfg;
    int32_t n;
    uint64_t seed;
    cudaStream_t stream;
    int device;
    int elem_bytes;
    int32_t pitch;
    int64_t plane, clone_stride;  // in elements
    float scale, inv_scale;
    void* buf[2];
    int32_t* parity_dev;
    int32_t* t_dev;
    std::vector<int32_t> parity_host, t_host;
    int32_t* list_dev;        // clone list of the current step call
    int32_t* all_dev;         // 0..N-1
    float* partials;          // [N][batch_cap][n_slots]
    int32_t batch_cap, n_slots;
    int32_t ry0, ry1, rs0, rs1;
    double* drag;             // [N][max_steps]
    int32_t* flag_dev;        // [0]: nonzero once a drag value was not finite; [1]: scratch int
    // App. D snapshot bank
    void* snaps;
    double* snap_mass;        // [n_snapshots]
    int32_t n_snaps_set;
    // AMS checkpoints every ckpt_stride steps: [N][n_ckpt] states
    void* ckpt;
    int32_t n_ckpt;
    // scratch for deterministic reductions
    double* red_partials;     // [N][red_blocks] (or larger)
    int32_t red_blocks;
    double* mass_dev;         // [N]
    double* scores;           // [N][max_steps] trailing means
    int32_t score_window, score_t_begin, score_t_end;  // arguments of the last lbm_ensemble_scores
    int32_t* fields_list_dev; // clone list of field extractions
    // learned score attached to the ensemble (lbm_ensemble_attach_score)
    cnn_model* cnn;
    int32_t cnn_factor;
    float cnn_rho_scale, cnn_u_scale;
    void* cnn_x;              // [max_batch][H][W][8] BF16 network input
    float* cnn_pred;          // [max_batch]
    double* cnn_score;        // [N][n_ckpt] score at every checkpoint (NaN until evaluated)
    double* pot[3];           // GKTL potential: now, previous, start (per slot)
    double* pot_tmp[2];
    // selected step variant (index into step_variants())
    int variant;
    // optional timing of the fused step launches
    bool timing;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    double timed_ms;
    int64_t timed_launches;
};
