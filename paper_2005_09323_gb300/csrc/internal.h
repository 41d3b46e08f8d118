// Host-side internals shared by the translation units of liblbmrare.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "lbmrare.h"
#include "step_params.h"

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

struct StepVariant {
    using Launch = cudaError_t (*)(const StepParams&, cudaStream_t);
    int storage;
    int vec;    // sites per thread
    int warps;  // warps per block
    cudaError_t (*launch)(const StepParams&, cudaStream_t);
    int kind;   // 0: register-staged row segments per warp; 1: whole rows staged by bulk copies;
                // 2: tiles in shared memory, several steps per launch (temporal blocking)
    bool (*supports)(const StepParams&);  // null: every shape
    // the open channel's step (fused step + boundary columns); null: this
    // variant has no open-channel instantiation
    Launch launch_open = nullptr;
    int multi = 1;  // most steps one launch runs (kind 2; an odd number per launch)
};

// LBM_ERR_ARG unless the collision fields of c are valid (lbm_ensemble.cu)
int check_collision(const lbm_config& c);
// LBM_ERR_ARG unless the open-channel fields of c are valid (lbm_ensemble.cu)
int check_open(const lbm_config& c);

// all compiled variants of the fused step (lbm_step.cu)
const std::vector<StepVariant>& step_variants();

// tensor-core (tcgen05) 3x3 convolution 32 -> 32 channels over NHWC BF16
// activations (conv_tc.cu): bwd = false: ReLU(conv(x, w) + bias); bwd = true:
// conv(x, w) masked by mask > 0.  err (device int) is set on a device-side
// timeout.  Supported shapes: W a multiple of 128 or a divisor of 128 (>= 8),
// H a multiple of 2 * 128 / min(W, 128).
bool conv3x3_tc_supported(int B, int H, int W);
// weight gradient of a 32 -> 32 layer on the tensor cores (conv_tc.cu): per-CTA
// partial sums [nblk][32][304] (bias at column 288) for the fixed-order
// reduction; supported for widths that are a multiple of 128
bool conv3x3_wgrad_tc_supported(int B, int H, int W);
int conv3x3_wgrad_tc(const void* x, const void* dy, float* partial, int B, int H, int W, int32_t* err,
                     cudaStream_t s, int* nblk);
int conv3x3_tc(const void* x, const void* w, const void* mask, void* out, int B, int H, int W, bool bwd,
               int32_t* err, cudaStream_t s);

// network input of clones listed on the device (cnn.cu); no synchronisation
int fields_launch(lbm_ensemble* e, const int32_t* list_dev, int32_t n, int32_t factor, float rho_scale, float u_scale,
                  void* dst_dev);
// learned score of the listed clones (host list) into out[c * stride + k] (surrogate.cu)
int score_clones(lbm_ensemble* e, const int32_t* clones, int32_t n, double* out, int32_t stride, int32_t k);

// one launch of the observables kernel for step `step` of a chunk over the
// listed clones (observables.cu)
int observables_launch(lbm_ensemble* e, const int32_t* list_dev, int32_t n_list, int32_t step, cudaStream_t s);

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
    int32_t perturb_mode;     // coefficients alpha_n: 0 uniform in [0, 1) (App. D); 1 centred, minus 1/2
    double* snap_mass;        // [n_snapshots]
    int32_t n_snaps_set;
    // AMS checkpoints every ckpt_stride steps: [N][n_ckpt] states
    void* ckpt;
    int32_t n_ckpt;
    // scratch for deterministic reductions
    double* red_partials;     // [N][red_blocks] (or larger)
    int32_t red_blocks;
    double* mass_dev;         // [N]
    float* om_col;            // open channel: [nx] relaxation rate of each column
    float* inlet_g;           // open channel: [9][ny] inlet populations minus w_q
    float* open_u;            // open channel: [2][N][4][ny] velocities of columns nx-2, nx-3, per step parity
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
    // selected step variants (indices into step_variants()): one for step
    // calls over many sites, one for calls below kSmallSites (an AMS branch)
    int variant;
    int variant_small;
    // step chunks captured once as CUDA graphs and replayed: one cached
    // executable per (variant, clone list, list length, chunk length)
    struct StepGraph {
        int variant;
        const int32_t* list;
        int32_t n_list, chunk;
        cudaGraphExec_t exec;
        uint64_t used;
    };
    std::vector<StepGraph> graphs;
    uint64_t graph_clock;
    bool use_graphs;          // on by default (lbm_ensemble_set_graphs)
    cudaStream_t cap_stream;  // private stream the chunks are captured on
    // optional timing of the fused step launches
    bool timing;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> events;
    double timed_ms;
    int64_t timed_launches;
    // observables of the square after every step (lbm_ensemble_set_observables)
    bool observe;
    double* obs;              // [N][max_steps][4]: p_fb, p_base, gamma_top, gamma_bottom
};

