/*
 * lbmrare: ensemble lattice-Boltzmann channel flows past a square obstacle,
 * advanced on one NVIDIA GB300 (sm_103a) and resampled by the GKTL and AMS
 * rare-event algorithms, after Lestang, Bouchet & Leveque, "Numerical study of
 * extreme mechanical force exerted by a turbulent flow on a bluff body by
 * direct and rare-event sampling techniques" (arXiv 2005.09323).
 *
 * Conventions for every entry point:
 *   - returns LBM_OK (0) or a negative lbm_status; lbm_last_error() gives a
 *     message for the calling thread.  No exception crosses this boundary.
 *   - arguments named *_dev are device pointers in the ensemble's (or the
 *     given) stream order; the call enqueues work and returns without waiting.
 *     Other pointers are host memory, owned by the caller, and the call has
 *     finished with them when it returns (it synchronises the stream).
 *   - arguments are validated on the host before anything is enqueued; on
 *     LBM_ERR_ARG nothing was enqueued and the ensemble is unchanged.
 *   - population arrays on the host are FP64, [9][ny][nx], direction q with
 *     velocity c_q: q=0 (0,0); 1 (1,0); 2 (0,1); 3 (-1,0); 4 (0,-1);
 *     5 (1,1); 6 (-1,1); 7 (-1,-1); 8 (1,-1).
 *   - time t counts lattice steps; D(t) is the drag of the state after step t.
 */
#ifndef LBMRARE_H
#define LBMRARE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    LBM_OK = 0,
    LBM_ERR_ARG = -1,        /* invalid argument; nothing enqueued */
    LBM_ERR_CUDA = -2,       /* a CUDA call failed; message names it */
    LBM_ERR_NONFINITE = -3,  /* a drag value, weight or score is not finite */
    LBM_ERR_TIMEOUT = -4,    /* a bounded device-side wait ran out */
    LBM_ERR_OOM = -5,        /* device allocation failed */
    LBM_ERR_STATE = -6       /* call not valid in the ensemble's current state */
} lbm_status;

typedef enum {
    LBM_FP32 = 0,            /* populations f stored as FP32 (72 B per site update) */
    LBM_FP16_SHIFTED = 1,    /* (f - w_q) * 2^shift_exp stored as FP16 (36 B) */
    LBM_BF16_SHIFTED = 2     /* (f - w_q) * 2^shift_exp stored as BF16 (36 B) */
} lbm_storage;

/* One channel flow (Sec. 2 and App. A): D2Q9 lattice-BGK on nx x ny nodes,
 * periodic in x, no-slip walls halfway below row 0 and above row ny-1, a square
 * obstacle of solid cells [obs_x0, obs_x0+obs_w) x [obs_y0, obs_y0+obs_h) with
 * halfway bounce-back on its surface, and a constant body-force density
 * (gx, gy) on fluid nodes (Guo forcing). */
typedef struct {
    int32_t nx, ny;            /* nx a multiple of 8 (any nx >= 8 for an open channel), nx >= 8, ny >= 2 */
    int32_t obs_x0, obs_y0, obs_w, obs_h;  /* obs_w = 0: no obstacle; else 1 <= obs_x0, obs_x0+obs_w <= nx-1
                                              (<= nx-3 in an open channel) */
    double tau;                /* BGK relaxation time (> 1/2); nu = (tau - 1/2)/3 */
    double gx, gy;             /* force density per fluid node */
    int32_t storage;           /* lbm_storage */
    int32_t shift_exp;         /* 16-bit storage scale 2^shift_exp (0 for FP32) */
    int32_t max_steps;         /* capacity of the drag history per clone */
    int32_t ckpt_stride;       /* AMS: keep the state every ckpt_stride steps; 0 = none */
    int32_t n_snapshots;       /* capacity of the App. D snapshot bank (N_s) */
    double init_amp;           /* initial velocity perturbation amplitude */
    /* collision (App. A): 0 = BGK with Guo forcing; 1 = central moments with
     * multiple relaxation times, the production collision the paper names:
     *   f* = f + S - T^{-1} Omega T (f - f^eq + S/2),
     * T(u) the D2Q9 central-moment transform, f^eq the same discrete
     * equilibrium, S the Guo term; Omega relaxes k20 - k02 and k11 at 1/tau
     * (the viscosity), k20 + k02 at omega_bulk, k21 and k12 at omega_3, k22 at
     * omega_4 (each in (0, 2)); all rates 1/tau is BGK.  Zero-initialised
     * configurations are BGK. */
    int32_t collision;
    double omega_bulk, omega_3, omega_4;
    /* open channel (Sec. 2); open_x = 0 (zero-initialised) is the periodic,
     * body-forced channel.  open_x = 1:
     *   inlet   column x = 0 holds the equilibrium of rho = 1 and u = (u_in(y), 0),
     *           u_in(y) = 4 u_in (y + 1/2)(ny - y - 1/2) / ny^2, the parabola that
     *           vanishes on the halfway walls with centreline value u_in;
     *   outlet  column x = nx-1 takes rho = 1 and the velocity extrapolated to
     *           second order from columns nx-2 and nx-3, its populations
     *           regularized with the finite-difference strain rate (Latt et al.
     *           2008); the paper extrapolates the density too, which leaves the
     *           mean pressure drop free (a drifting neutral mode);
     *   grid    bars of grid_bar rows separated by grid_gap fluid rows (a gap at
     *           the bottom wall) over columns [grid_x0, grid_x0 + grid_w);
     *           grid_w = 0: none.  The drag counts the square's links only;
     *   sponge  tau(x) = tau + (sponge_tau - tau) s^2 over the last sponge_len
     *           columns, s = (x - nx + sponge_len + 1) / sponge_len;
     * each step the boundary columns are overwritten after the collision.
     * Requires gx = gy = 0, 8 <= nx (any nx, not only multiples of 8), ny >= 3,
     * the square and the grid inside columns [1, nx-3), tau at the outlet
     * (sponge_tau, or tau without a sponge) at most 1 (larger values made the
     * outlet unstable), |u_in| < 0.3.  Open channels run on register-staged
     * step variants only and not through lbm_step_noalloc. */
    int32_t open_x;
    double u_in;
    int32_t grid_x0, grid_w, grid_bar, grid_gap;
    int32_t sponge_len;
    double sponge_tau;
} lbm_config;

typedef struct lbm_ensemble lbm_ensemble;

/* message of the last failure on the calling thread ("" if none) */
const char* lbm_last_error(void);

/* number of CUDA kernels this library has launched in the process so far */
int64_t lbm_launch_count(void);

/* ---------------------------------------------------------------- ensemble */

/* Create N independent trajectories of the flow (ensemble of Sec. 4 and
 * App. C.1) on the current CUDA device and initialise each at equilibrium
 * (Sec. 2: "initial distributions ... at equilibrium") with rho = 1 and a
 * seeded velocity u = init_amp * (2 U - 1) per component, U from Philox4x64-10
 * with counter (5, clone, y*nx + x, 0) and key (seed, 0); solid nodes hold the
 * rest weights.  The ensemble owns all its device memory; stream may be NULL
 * (the legacy default stream).  Errors: LBM_ERR_ARG, LBM_ERR_OOM, LBM_ERR_CUDA. */
int lbm_ensemble_create(const lbm_config* cfg, int32_t n_clones, uint64_t seed, void* stream,
                        lbm_ensemble** out);

/* Free everything the ensemble owns (waits for its stream). */
int lbm_ensemble_destroy(lbm_ensemble* e);

/* Advance every clone by n_steps lattice steps (App. A: exact streaming with
 * halfway bounce-back, then BGK collision with Guo forcing; one fused kernel per
 * step) and record the momentum-exchange drag of eq. (drag_definition) after each
 * step.  All clones must be at the same time; t + n_steps <= max_steps.  States
 * are saved every ckpt_stride steps when checkpoints are enabled.  Asynchronous:
 * a non-finite drag is reported by the next synchronising call as
 * LBM_ERR_NONFINITE. */
int lbm_ensemble_step(lbm_ensemble* e, int32_t n_steps);

/* As lbm_ensemble_step, for the n listed clones only (host array of distinct
 * indices, all at the same time) - the re-simulation of a branched AMS
 * trajectory (App. B.1). */
int lbm_ensemble_step_clones(lbm_ensemble* e, int32_t n_steps, const int32_t* clones, int32_t n);

/* Copy each clone's current time (host int32[N]). */
int lbm_ensemble_time(lbm_ensemble* e, int32_t* t);

/* Drag history D(t), t0 < t <= t1, of every clone into dst[N][t1-t0] (FP64);
 * t1 may not exceed the latest clone time, and entries past a clone's own
 * time are not part of its trajectory.
 * dst_on_device != 0: dst is a device pointer and the copy is enqueued;
 * otherwise dst is host memory and the call waits.  Errors: LBM_ERR_ARG,
 * LBM_ERR_NONFINITE (a recorded drag value was not finite). */
int lbm_ensemble_drag(lbm_ensemble* e, int32_t t0, int32_t t1, double* dst, int32_t dst_on_device);

/* Overwrite the drag history D(t), t0 < t <= t1, of every clone with
 * src[N][t1-t0] (host, FP64, finite; t1 at most the latest clone time), for
 * the statistics, window sums, scores and estimators that read it: a run
 * restored from saved state, or a given series to evaluate them on.  The
 * populations are untouched.  Waits.  Errors: LBM_ERR_ARG. */
int lbm_ensemble_set_drag(lbm_ensemble* e, int32_t t0, int32_t t1, const double* src);

/* GKTL exponent of eq. (Weight): out_dev[n] = k * sum_{t0 < t <= t1} D_n(t)
 * (dt = one lattice step), FP64, fixed summation order. */
int lbm_ensemble_window_sum(lbm_ensemble* e, int32_t t0, int32_t t1, double k, double* out_dev);

/* Time-averaged drag of eq. (def_time_averaged_drag) with a window of T steps,
 * F(t) = (1/T) sum_{s=t-T+1}^{t} D(s) for t_begin + T <= t <= t_end (the
 * trajectory starts at t_begin), FP64, stored in the ensemble; out_dev[n] (may
 * be NULL) receives max_t F_n(t) (-inf if t_end < t_begin + T): the AMS score
 * maximum Q_n (App. B.1) and the GKTL event amplitude (App. C.2). */
int lbm_ensemble_scores(lbm_ensemble* e, int32_t window, int32_t t_begin, int32_t t_end, double* out_dev);

/* First t with F_clone(t) > level in the last lbm_ensemble_scores result (the
 * AMS branching time of App. B.1); *t = -1 if none.  Host output; waits. */
int lbm_ensemble_first_crossing(lbm_ensemble* e, int32_t clone, double level, int32_t* t);

/* Fill the App. D snapshot bank with the current states of the n_s listed
 * clones (host array) and record their masses. */
int lbm_ensemble_set_snapshots(lbm_ensemble* e, int32_t n_s, const int32_t* clones);

/* As lbm_ensemble_set_snapshots, from the states the listed clones held at
 * checkpoint k (time k * ckpt_stride). */
int lbm_ensemble_set_snapshots_from_checkpoint(lbm_ensemble* e, int32_t n_s, const int32_t* clones, int32_t k);

/* GKTL cloning (App. C.1) with the App. D perturbation: every slot s with
 * parent_dev[s] != s (a killed trajectory) becomes a copy of its parent's state,
 * time and drag history, perturbed by eq. (perturb_pop),
 *   f <- (f + eps sum_n alpha_n f^(n)) * M / (M + eps sum_n alpha_n M^(n)),
 * M the fluid mass, alpha_n uniform from Philox4x64-10 counter (4, iter, s, n),
 * key (seed, 0), minus 1/2 in the centred mode (lbm_ensemble_set_perturbation).
 * A parent must keep its own slot (parent_dev[p] == p), as
 * gktl_select guarantees.  eps = 0 copies exactly.  Needs the snapshot bank
 * when eps != 0.  A parent index outside [0, N) (a rejected selection writes
 * -1) leaves that slot unchanged and is reported as LBM_ERR_NONFINITE by the
 * next synchronising call. */
int lbm_ensemble_clone(lbm_ensemble* e, const int32_t* parent_dev, double eps, uint64_t seed,
                       uint64_t iter);

/* AMS branching (App. B.1): trajectory dst becomes a copy of src up to time t_b
 * (state restored from src's last checkpoint at or before t_b and replayed
 * bit-for-bit, drag history and checkpoints copied), perturbed as in
 * lbm_ensemble_clone with counter (4, iter, dst, n); dst is then at time t_b.
 * Needs ckpt_stride > 0 and src at time >= t_b. */
int lbm_ensemble_branch(lbm_ensemble* e, int32_t dst, int32_t src, int32_t t_b, double eps,
                        uint64_t seed, uint64_t iter);

/* The App. D perturbation of eq. (perturb_pop) applied in place to the n listed
 * clones (host array of distinct indices): f <- (f + eps sum_n alpha_n f^(n)) *
 * M / (M + eps sum_n alpha_n M^(n)) on fluid nodes, alpha_n from counter
 * (4, iter, clone, n) as in lbm_ensemble_clone.  This is the periodic
 * perturbation of the paper's check that the perturbation leaves the drag
 * statistics unchanged (App. D).  eps = 0 does nothing; otherwise needs the
 * snapshot bank.  Waits.  Errors: LBM_ERR_ARG, LBM_ERR_STATE. */
int lbm_ensemble_perturb(lbm_ensemble* e, int32_t n, const int32_t* clones, double eps, uint64_t seed,
                         uint64_t iter);

/* The coefficients alpha_n of every App. D perturbation of the ensemble
 * (cloning, branching, lbm_ensemble_perturb).  mode 0 (the default): uniform in
 * [0, 1), as eq. (perturb_pop) prints them.  Since they are positive, each
 * application then moves the state about eps sum_n alpha_n / 2 ~ 1% of the way
 * towards the mean of the bank's snapshots, which carries weaker fluctuations;
 * GKTL copies the trajectories that carry the tail again and again, and on the
 * open channel of Sec. 2 its estimate of a tail probability was measured to
 * fall as eps grows.  mode 1 (centred): alpha_n - 1/2, uniform in [-1/2, 1/2):
 * the same random directions with no mean pull.
 * Kept by lbm_ensemble_save.  Errors: LBM_ERR_ARG. */
int lbm_ensemble_set_perturbation(lbm_ensemble* e, int32_t mode);

/* Observables of the square after every step (Sec. 2.1 eq. drag_approx, Sec.
 * 3.2 eq. avg_shear_def), recorded from the next step on while enabled, from
 * the post-collision state of each step:
 *   [0] p_fb   = cs2 sum over rows [obs_y0, obs_y0+obs_h) of rho(obs_x0 - 1, y):
 *               the pressure integrated over the upstream face (forebody);
 *   [1] p_base = the same at x = obs_x0 + obs_w (the base); f_d ~ p_fb - p_base;
 *   [2] gamma_top, [3] gamma_bottom: the mean over the face's obs_w columns of
 *       d u_x / d y at the halfway wall, (9 u_1 - u_2)/3 from the fluid rows at
 *       distances 1/2 and 3/2 (negated on the bottom face, whose rows lie
 *       below), with rho u = sum c f - F/2.
 * FP64, fixed summation order.  Enabling needs a square with two fluid rows
 * above and below it (obs_y0 >= 2, obs_y0 + obs_h <= ny - 2) and allocates
 * [N][max_steps][4] doubles; each step then adds one small kernel.  Cloning
 * and branching copy the history with the drag's.  Errors: LBM_ERR_ARG.
 * lbm_ensemble_observables copies entries t0 <= t < t1 (t as in
 * lbm_ensemble_drag) of every clone into dst[N][t1-t0][4] (host, waits; or
 * device with dst_on_device != 0).  Errors: LBM_ERR_STATE if never enabled. */
int lbm_ensemble_set_observables(lbm_ensemble* e, int32_t enable);
int lbm_ensemble_observables(lbm_ensemble* e, int32_t t0, int32_t t1, double* dst, int32_t dst_on_device);

/* Fluid mass and momentum sum_x sum_q f_q (1, c_q) per clone (host double[N]
 * each; any may be NULL), FP64 deterministic reduction.  Waits. */
int lbm_ensemble_moments(lbm_ensemble* e, double* mass, double* px, double* py);

/* Read / overwrite one clone's populations as FP64 [9][ny][nx] host arrays
 * (decoded from, or encoded to, the storage format).  Wait. */
int lbm_ensemble_get_populations(lbm_ensemble* e, int32_t clone, double* host);
int lbm_ensemble_set_populations(lbm_ensemble* e, int32_t clone, const double* host);

/* Run resume.  No passage of the paper defines it: it lets a long direct-
 * sampling run (Sec. 3) or a GKTL loop driven step by step (App. C.1) stop and
 * continue in a later process.
 * lbm_ensemble_save writes the ensemble's run state into the caller-owned host
 * buffer dst of capacity bytes: a versioned header with the configuration,
 * then each clone's time and current populations in the storage format, the
 * drag history up to the latest clone time (and the observables' history when
 * enabled), the App. D snapshot bank with its masses, and the AMS checkpoints
 * up to the latest clone time.  *bytes receives the size the state needs;
 * dst = NULL only reports it.  Waits.  Errors: LBM_ERR_ARG (null e or bytes,
 * capacity too small; nothing written).
 * lbm_ensemble_load overwrites ensemble e with a state written by
 * lbm_ensemble_save.  e must have been created with the same configuration
 * (every lbm_config field equal) and clone count, and with observables enabled
 * exactly when the saved ensemble had them; its seed and perturbation mode
 * become the saved ones.
 * An attached learned score is not part of the state: attach it after loading
 * (LBM_ERR_STATE otherwise).  The loaded ensemble continues bit for bit as the
 * saved one would have.  Waits.  Errors: LBM_ERR_ARG (not a saved state,
 * another version, size, configuration or layout; nothing changed),
 * LBM_ERR_STATE, LBM_ERR_CUDA. */
int lbm_ensemble_save(lbm_ensemble* e, void* dst, uint64_t capacity, uint64_t* bytes);
int lbm_ensemble_load(lbm_ensemble* e, const void* src, uint64_t bytes);

/* Pick the fastest compiled variant of the fused step (sites per thread, warps
 * per block) for this ensemble by timing each on its own state; the state and
 * the drag history are left unchanged.  *variant (may be NULL) gets the index. */
int lbm_ensemble_autotune(lbm_ensemble* e, int32_t* variant);
/* Force a variant by index for every step call (-1 restores the defaults);
 * describe any index.  Without a forced variant, step calls over at most 2^18
 * sites (clones x nx x ny, e.g. one AMS branch) use a separate small-list
 * variant (default: the narrowest register-staged variant with 8 warps, which
 * puts the most threads on a small grid); lbm_ensemble_autotune picks both. */
int lbm_ensemble_set_variant(lbm_ensemble* e, int32_t variant);
int lbm_step_variant_info(int32_t variant, int32_t* storage, int32_t* vec, int32_t* warps);
int32_t lbm_step_variant_count(void);
/* Data movement of a variant: 0 = register-staged row segments, one warp per
 * segment (lbm_step.cuh); 1 = whole rows staged in shared memory by bulk
 * copies (lbm_step_rows.cuh).  LBM_ERR_ARG for an index out of range. */
int32_t lbm_step_variant_kind(int32_t variant);

/* Failure-detection self test of the bounded device-side waits used by the
 * row-staged step kernels: one thread polls an mbarrier that nothing arrives
 * at, `spins` times, then gives up; *status (host) receives LBM_ERR_TIMEOUT.
 * The context stays usable.  Waits. */
int lbm_selftest_bounded_wait(int64_t spins, void* stream, int32_t* status);

/* CUDA graphs (on by default): each chunk of fused-step launches between two
 * drag finalisations is captured once per (variant, clone list, chunk length)
 * into a CUDA graph, cached (24 per ensemble, least recently used dropped) and
 * replayed on the ensemble's stream.  The replay does the same work as the
 * launches; it removes the per-launch host cost, which bounds the step rate
 * of small ensembles such as one AMS branch.  enable = 0 launches each step
 * directly.  Errors: LBM_ERR_ARG for a null ensemble. */
int lbm_ensemble_set_graphs(lbm_ensemble* e, int32_t enable);

/* Kernel timing: when enabled, every batch of fused-step launches is bracketed
 * by CUDA events on the ensemble's stream; lbm_ensemble_kernel_time waits and
 * returns the summed milliseconds and launch count since the last reset. */
int lbm_ensemble_set_timing(lbm_ensemble* e, int32_t enable);
int lbm_ensemble_kernel_time(lbm_ensemble* e, double* ms, int64_t* launches, int32_t reset);

/* ---------------------------------------------------------------- direct sampling (Sec. 3) */

/* Drag statistics of direct sampling.  The clones are independent
 * trajectories; their drag series over the steps [t0, t1) are pooled (every
 * clone must have reached t1).  FP64, every sum in a fixed order.
 *
 * lbm_drag_autocorrelation: c_dev[tau] (device, max_lag + 1 doubles) =
 *   mean_{clones, t} f~(t + tau) f~(t) / mean f~^2,   f~ = f_d - mean f_d,
 * the autocorrelation of the caption of Fig. pdf_drag; each lag averages the
 * n (t1 - t0 - tau) products inside the series.  *tau_c (host, may be NULL)
 * receives the correlation time, the first lag with C <= 0 (C(tau_c) = 0 in
 * the paper), or -1 if C stays positive up to max_lag (then waits).
 * 0 <= max_lag < t1 - t0.
 *
 * lbm_drag_return_times: the waiting-time return time of Sec. 3 for each of
 * n_levels levels (levels_dev, device doubles).  An event of level a starts
 * where a series crosses from below a to >= a, unless it was >= a within the
 * last gap steps (then it is the same fluctuation; gap = tau_c declusters).
 * events[j] (host) = events over all clones; r[j] (host) = n (t1 - t0) /
 * events[j], the mean waiting time in steps, +inf without events.  Waits. */
int lbm_drag_autocorrelation(lbm_ensemble* e, int32_t t0, int32_t t1, int32_t max_lag, double* c_dev, int32_t* tau_c);
int lbm_drag_return_times(lbm_ensemble* e, int32_t t0, int32_t t1, int32_t n_levels, const double* levels_dev,
                          int32_t gap, int64_t* events, double* r);

/* ---------------------------------------------------------------- drivers */

/* GKTL run (App. C.1), from the ensemble's current time t0 (all clones equal):
 * n_periods times, advance period steps, form s_n = k sum_{period} D_n(t)
 * (gktl exponent of eq. (Weight)), the weights and log R_i, resample
 * (gktl_select with iter = i) and clone with the App. D perturbation eps
 * (lbm_ensemble_clone, iter = i).  Device outputs: logR_dev[n_periods] (their
 * sum is ln Z), parent_dev[n_periods][N] (the genealogy), and, when non-NULL,
 * integral_dev[N] = sum_{t0 < t <= t_end} D_n(t) of each final trajectory
 * (histories follow the clones) and maxima_dev[N] = max_t F_T(t) with T =
 * window steps (lbm_ensemble_scores from t0).  Waits at the end; a rejected
 * resampling or a non-finite drag returns LBM_ERR_NONFINITE / LBM_ERR_ARG. */
typedef struct {
    int32_t period;       /* cloning period tau, in steps */
    int32_t n_periods;    /* T_a / tau */
    double k;             /* bias per step of drag (exponent k * sum D) */
    double eps;           /* App. D perturbation amplitude; 0 copies exactly */
    uint64_t seed;        /* selection and perturbation streams */
    int32_t window;       /* T of the time-averaged drag for maxima_dev (0: none) */
    double kappa;         /* learned pre-screen: exponent += kappa (V(t_i) - V(t_{i-1})), V the
                             attached learned score; 0 = off */
    int32_t refresh_snapshots;  /* 1: before each cloning step refill the App. D bank from the
                             current states of evenly spaced clones (needed when the flow is not
                             stationary: stale snapshots pull clones toward an earlier mean flow) */
} lbm_gktl_params;
/* correction_dev[N] (may be NULL) receives kappa (V(t_end) - V(t0)) of each final
 * trajectory: the log-weight the estimator removes (gktl_probability). */
int lbm_gktl_run(lbm_ensemble* e, const lbm_gktl_params* p, double* logR_dev, int32_t* parent_dev,
                 double* integral_dev, double* maxima_dev, double* correction_dev);

/* GKTL return-time estimator (App. C.2, sign read as the inversion of eq.
 * (Biased_Path_Approximation) requires): for each level a_j,
 *   p_dev[j] = (1/N) sum_n exp(ln Z - k I_n - c_n) 1{A_n >= a_j},  ln Z = sum_i logR_dev[i],
 *   r_dev[j] = -(t_a - t_window) / ln(1 - p_dev[j])   (r_dev may be NULL),
 * I_n = integral_dev[n], A_n = maxima_dev[n], c_n = correction_dev[n] (NULL: 0).
 * FP64, fixed summation order. */
int gktl_probability(int32_t n, double k, const double* logR_dev, int32_t n_periods, const double* integral_dev,
                     const double* maxima_dev, const double* correction_dev, int32_t n_levels,
                     const double* levels_dev, double t_a, double t_window, double* p_dev, double* r_dev,
                     void* stream);

/* AMS run (App. B.1) on trajectories of t_a steps from the ensemble's current
 * time t0 (all clones equal, t0 a multiple of ckpt_stride): advance every
 * clone t_a steps, score = time-averaged drag over window steps; then for
 * j = 1..max_iter: ams_select (iter = j), stop if the level z_j >= level or
 * every score ties, else branch each killed trajectory from its survivor at
 * the first time the survivor's score exceeds z_j (perturbation eps, iter = j)
 * and re-simulate it to t0 + t_a.  Outputs: *iterations (kills done),
 * *log_weight = sum_j ln(1 - |K_j|/N), Q_dev[N] the final score maxima, and
 * on the host levels[j-1] = z_j and n_killed[j-1] = |K_j| (either may be NULL;
 * max_iter entries; ties at the minimum are killed together), and
 * killed_max[(j-1) * N + i] (may be NULL; max_iter * N entries) the event
 * maximum - the time-averaged drag over window, maximised over the run - of the
 * i-th trajectory killed at iteration j, taken before it is replaced.  The
 * generalised AMS estimator counts these killed trajectories (ams_probability);
 * with the drag as score each one's maximum is z_j.  Waits. */
typedef struct {
    int32_t t_a;          /* trajectory duration, steps */
    int32_t window;       /* score window T, steps */
    int32_t max_iter;     /* J */
    double level;         /* stop once the killed level reaches it (+inf: run J) */
    double eps;           /* App. D perturbation amplitude at branching */
    uint64_t seed;
    int32_t score_kind;   /* 0: time-averaged drag over window (every step);
                             1: the attached learned score at every checkpoint
                             (branching then restores a checkpoint exactly) */
    int32_t refresh_snapshots;  /* 1: before each branch refill the App. D bank with the states of
                             evenly spaced trajectories at the branching checkpoint */
} lbm_ams_params;
int lbm_ams_run(lbm_ensemble* e, const lbm_ams_params* p, int32_t* iterations, double* log_weight, double* Q_dev,
                double* levels, int32_t* n_killed, double* killed_max);

/* AMS estimator (generalised AMS, Brehier-Lelievre-Rousset 2016; the paper
 * states none): every trajectory the run has seen counts with its weight,
 * p_dev[l] = (exp(log_weight) #{n : Q_n >= a_l}
 *            + sum_r exp(rec_logw_dev[r]) 1{rec_max_dev[r] >= a_l}) / N,
 * with Q_dev[N] the final ensemble's event maxima and one record r per killed
 * trajectory: the log weight before its iteration, sum_{i<j} ln(1 - |K_i|/N),
 * and its event maximum (lbm_ams_run's killed_max).  n_records = 0 counts the
 * final ensemble only, which is exact when the score is the event's own
 * observable and a_l lies above the last killed level.  FP64, fixed-order sums. */
int ams_probability(int32_t n, double log_weight, const double* Q_dev, int32_t n_records, const double* rec_logw_dev,
                    const double* rec_max_dev, int32_t n_levels, const double* levels_dev, double* p_dev,
                    void* stream);

/* ---------------------------------------------------------------- learned score */

/* A CNN surrogate of the future time-averaged drag: the paper's conclusion
 * proposes learning the score function of the rare-event algorithms; this is
 * that function, trained on trajectories the method itself produces.
 * Network: conv3x3(8 -> 32) + ReLU, 3 x [conv3x3(32 -> 32) + ReLU], global mean
 * pool, linear 32 -> 1.  Input x_dev: BF16 [batch][height][width][8] (NHWC;
 * channels 0..2 the fields of lbm_ensemble_fields, 3..7 zero).  BF16 weights
 * and activations, FP32 tensor-core accumulation, FP32 master parameters and
 * Adam.  Parameter vector (FP32, cnn_param_count entries): for conv layer l,
 * W_l[co][k] with k = (3 ky + kx) * C_in + ci (C_in = 8, then 32), the bias at
 * k = 9 C_in, zero padding to 80 (layer 0) or 304 columns; then the head
 * weights v[32] and its bias.  height % 8 == 0, width % 16 == 0. */
typedef struct cnn_model cnn_model;
int cnn_create(int32_t height, int32_t width, int32_t max_batch, uint64_t seed, cnn_model** out);
int cnn_destroy(cnn_model* m);
int64_t cnn_param_count(const cnn_model* m);
int cnn_get_params(cnn_model* m, float* host);        /* waits */
int cnn_set_params(cnn_model* m, const float* host);  /* waits; rejects non-finite values */
/* pred_dev[b] (FP32) for a batch of inputs */
int cnn_forward(cnn_model* m, const void* x_dev, int32_t batch, float* pred_dev, void* stream);
/* gradient of the mean squared error (1/B) sum_b (pred_b - y_b)^2 with respect
 * to every parameter, into the model's gradient buffer; *loss_dev (may be NULL)
 * receives the loss.  cnn_get_gradient copies it to the host (waits). */
int cnn_gradient(cnn_model* m, const void* x_dev, const float* y_dev, int32_t batch, float* loss_dev, void* stream);
int cnn_get_gradient(cnn_model* m, float* host);
/* Adam (Kingma & Ba 2015) with bias correction on the master parameters */
int cnn_adam_step(cnn_model* m, float lr, float beta1, float beta2, float eps, void* stream);
/* cnn_gradient then cnn_adam_step(lr, 0.9, 0.999, 1e-8) */
int cnn_train_step(cnn_model* m, const void* x_dev, const float* y_dev, int32_t batch, float lr, float* loss_dev,
                   void* stream);

int cnn_shape(const cnn_model* m, int32_t* height, int32_t* width, int32_t* max_batch);
/* Kernels of the three hidden 32 -> 32 layers (forward and data gradient).
 * path 0 (default): fifth-generation tensor cores (tcgen05.mma with the
 * accumulator in tensor memory, operands staged by TMA) wherever the shape
 * allows: width a multiple of 128 or a divisor of 128 (>= 8) and height a
 * multiple of 256 / min(width, 128); other shapes use path 1.  path 1: the
 * warp-level mma.sync kernels.  Both compute the same layer (FP32 accumulation
 * of BF16 products; the summation order differs).  The input layer and the
 * weight gradients use mma.sync.  LBM_ERR_ARG for another path. */
int cnn_set_conv_path(cnn_model* m, int32_t path);
/* Waits for the stream, then LBM_ERR_TIMEOUT if a bounded device-side wait of
 * a tensor-core convolution ran out since the model was created (the kernel
 * records it and returns; the context stays usable), else LBM_OK.  cnn_fit
 * checks the same flag after every minibatch. */
int cnn_status(cnn_model* m, void* stream);
/* Which hidden-layer kernels a step of this batch size runs: *conv_tc = 1 if
 * the 32 -> 32 forward and data-gradient convolutions run on the tcgen05
 * kernels (else mma.sync), *wgrad_tc = 1 likewise for their weight gradient.
 * The tensor-core path needs a width that is a multiple of 128, or a divisor
 * of 128 for the forward kernels; a width of exactly 128 with more than 148
 * output rows (batch x height) stays on mma.sync, because a GPU fault of
 * unknown cause was once recorded at 32 x 128 with batch 64.  No GPU work. */
int cnn_tensor_core_paths(const cnn_model* m, int32_t batch, int32_t* conv_tc, int32_t* wgrad_tc);
/* predictions for n inputs (any n; evaluated in batches of max_batch) */
int cnn_predict(cnn_model* m, const void* x_dev, int64_t n, float* pred_dev, void* stream);
/* epochs of minibatch Adam over a data set x_dev [n][H][W][8], y_dev[n] (FP32):
 * each epoch visits the samples in a Fisher-Yates order from Philox4x64-10
 * stream 8 (key (seed, 0), counter (8, epoch, i, 0)); epoch_loss[ep] (host, may
 * be NULL) gets the mean minibatch loss.  Waits. */
int cnn_fit(cnn_model* m, const void* x_dev, const float* y_dev, int64_t n, int32_t batch, int32_t epochs, float lr,
            uint64_t seed, float* epoch_loss, void* stream);

/* Attach a learned score to an ensemble (m = NULL detaches; the model stays the
 * caller's): from now on every checkpointed state of every stepped clone is
 * scored, the series following branches (lbm_ams_run with score_kind 1), and
 * lbm_gktl_run may use it as a pre-screen potential (kappa).  The model input is
 * the ensemble's fields downsampled by factor; its height and width must be
 * ny/factor and nx/factor (floor division, as lbm_ensemble_fields). */
int lbm_ensemble_attach_score(lbm_ensemble* e, cnn_model* m, int32_t factor, float rho_scale, float u_scale);
/* score of every clone now, into out_dev[N] (device) */
int lbm_ensemble_evaluate_score(lbm_ensemble* e, double* out_dev);
/* the checkpoint score series, host double[N][max_steps/ckpt_stride + 1] (NaN where
 * not evaluated).  Waits. */
int lbm_ensemble_score_history(lbm_ensemble* e, double* host);

/* Training data for the learned score from an ensemble run: n_snaps snapshots
 * of every clone, every `every` steps from the current time t0, as network
 * inputs x_dev [n_snaps * N][ny/factor][nx/factor][8] (snapshot-major), with
 * labels y_dev[i * N + c] = the time-averaged drag of clone c over the next
 * `horizon` steps (eq. (def_time_averaged_drag)), normalised to zero mean and unit
 * variance; *label_mean, *label_std (may be NULL) receive the scaling.  The
 * ensemble advances (n_snaps - 1) * every + horizon steps.  Waits. */
int lbm_surrogate_dataset(lbm_ensemble* e, int32_t n_snaps, int32_t every, int32_t horizon, int32_t factor,
                          float rho_scale, float u_scale, void* x_dev, float* y_dev, double* label_mean,
                          double* label_std);

/* Network input of the listed clones (host array): the block mean over
 * factor x factor nodes of (rho - 1) * rho_scale, u_x * u_scale, u_y * u_scale,
 * with u = (sum f c - F/2)/rho the velocity of the stored post-collision state,
 * into dst_dev BF16 [n][ny/factor][nx/factor][8] (channels 3..7 zero).  The
 * blocks tile the lattice from node (0, 0) with floor division: rows and
 * columns past the last whole block (the outlet column and top row of a
 * 513 x 129 open channel at factor 4) are not in the input.  LBM_ERR_ARG
 * unless 1 <= factor <= min(nx, ny).  Waits. */
int lbm_ensemble_fields(lbm_ensemble* e, const int32_t* clones, int32_t n, int32_t factor, float rho_scale,
                        float u_scale, void* dst_dev);

/* ---------------------------------------------------------------- no allocation */

/* One fused step (as lbm_ensemble_step, for one time step) over population
 * buffers the caller owns, for callers that cannot allocate device memory: a
 * program whose device memory belongs to another allocator (a framework's
 * pool, an arena fixed at start-up) or a loop that cannot afford the implicit
 * synchronisation of cudaMalloc.  The paper has no counterpart; it is an
 * interface of this library only.
 *   f_in_dev / f_out_dev: device arrays [n_clones][9][ny][pitch] in cfg->storage
 *     (FP32 f, or 16-bit (f - w_q) * 2^shift_exp), pitch = nx rounded up to a
 *     multiple of 256 elements, 16-byte aligned, distinct; padding columns are
 *     read but never written.  f_out_dev receives the state one step later.
 *   drag_dev: device double[n_clones], 8-byte aligned: the momentum-exchange
 *     drag of the new state, as lbm_ensemble_drag reports it.
 *   cfg: the flow (max_steps, ckpt_stride and n_snapshots are ignored).
 * Misaligned buffers, a non-finite force and shift_exp outside [-20, 20] are
 * rejected with LBM_ERR_ARG before anything is enqueued.
 * The call allocates nothing: its scratch (the per-warp drag partials and two
 * index tables) is a fixed 1 MiB device array inside the library, which every
 * device that loads the library holds until the process exits.  Sizes whose
 * scratch exceeds 1 MiB (n_clones x drag slots x 4 bytes plus the tables) are
 * rejected with LBM_ERR_ARG.  The first call on a device looks up that
 * array's device address (cudaGetSymbolAddress) with the device current; make
 * that first call before any stream capture.  Every call uses the same array:
 * calls that may overlap on the GPU (different streams without ordering)
 * race on it.  Enqueued on stream; returns without waiting. */
int lbm_step_noalloc(const lbm_config* cfg, int32_t n_clones, const void* f_in_dev, void* f_out_dev,
                     double* drag_dev, void* stream);

/* ---------------------------------------------------------------- selection */

/* GKTL weights, eq. (Weight): with m = max s, W_dev[n] = N e^{s_n - m} / S and
 * logR_dev[0] = m + ln(S / N), S = sum_n e^{s_n - m} (fixed-order FP64 sum), so
 * that sum W = N and ln Z = sum over cloning steps of logR (App. C.1).  One
 * block, N <= 4096.  Writes flag_dev-free: a non-finite s makes every W NaN and
 * gktl_select then fails with LBM_ERR_NONFINITE. */
int gktl_weights(int32_t n, const double* s_dev, double* W_dev, double* logR_dev, void* stream);

/* GKTL resampling to N copies with mean copy number W_n (App. C.1; scheme:
 * residual resampling with a systematic draw of the residuals, uniform from
 * Philox4x64-10 counter (1, iter, 0, 0), key (seed, 0)); a trajectory with at
 * least one copy keeps its slot, extra copies fill the emptied slots in
 * ascending order.  parent_dev[N] receives the parent of each slot.  W must be
 * finite, non-negative and sum to N (relative 1e-9): otherwise parent_dev is
 * filled with -1 and status_dev (may be NULL) receives LBM_ERR_NONFINITE or
 * LBM_ERR_ARG.  One block, N <= 4096. */
int gktl_select(int32_t n, const double* W_dev, uint64_t seed, uint64_t iter, int32_t* parent_dev,
                int32_t* status_dev, void* stream);

/* AMS selection (App. B.1): level z = min_n Q_n; every n with Q_n == z is
 * killed (killed_dev, ascending; *n_killed_dev = their number); for the k-th
 * killed index, survivor_dev[k] is the r-th non-killed index in ascending order,
 * r = floor(x * (N - |K|) / 2^64), x word 0 of Philox4x64-10 counter
 * (3, iter, killed, 0), key (seed, 0).  *n_killed_dev = N means every score
 * equals z (nothing survives).  A NaN score gives *n_killed_dev = -1. */
int ams_select(int32_t n, const double* Q_dev, uint64_t seed, uint64_t iter, int32_t* killed_dev,
               int32_t* n_killed_dev, int32_t* survivor_dev, double* level_dev, void* stream);

#ifdef __cplusplus
}
#endif
#endif
