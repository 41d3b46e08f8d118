/*
 * Oracle: plain, slow, single-threaded FP64 CPU implementation of the
 * ensemble lattice-Boltzmann rare-event method of Lestang, Bouchet & Leveque,
 * "Numerical study of extreme mechanical force exerted by a turbulent flow on
 * a bluff body by direct and rare-event sampling techniques" (arXiv 2005.09323).
 *
 * THIS IS TEST INFRASTRUCTURE.  Only the test suite, the smoke check and the
 * CPU-baseline leg of the benchmark may load it.  It shares no code, header,
 * table or constant generator with the CUDA library; each side writes the
 * lattice, the random-number generator and the selection rules on its own.
 *
 * Layout of every population array: f[(q*ny + y)*nx + x], q = 0..8, FP64.
 *
 * Functions and what pins them (tests/test_oracle_*.py):
 *   orc_philox4x64          numpy.random.Philox (library routine)
 *   orc_feq / orc_guo       closed-form moments (App. A)
 *   orc_lbm_step            rest-state invariance, mass conservation,
 *                           momentum balance (pins the drag), Poiseuille
 *   orc_cm_collide          equal rates = BGK; every central moment relaxes
 *                           at its own rate (numpy sums); mass and momentum
 *                           balance; shear-wave decay at nu = (tau - 1/2)/3
 *   orc_perturb             exact mass preservation; eps = 0 gives a copy
 *   orc_gktl_weights/select sum of weights = N, k = 0 identity, brute-force
 *                           mean copy counts; OU closed-form SCGF (App. C)
 *   orc_ams_select          OU brute-force exceedance probability (App. B)
 *   open channel (Sec. 2)   rest state kept; per-step mass balance through
 *                           the boundary columns; developed flow: one mass
 *                           flux through every cut, parabolic profile,
 *                           cs2 drho/dx = nu(x) rho u'' in bulk and sponge;
 *                           inlet equilibrium; outlet moments (numpy);
 *                           grid geometry; drag over the square's links only
 */
#ifndef LBMRARE_ORACLE_H
#define LBMRARE_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ---------------- counter-based random numbers ----------------------- */
/* Philox4x64-10 (Salmon, Moraes, Dror & Shaw, SC'11).  Counter and key are
 * little-endian words.  Streams used by the method (word 0 of the counter):
 *   1 GKTL systematic-resampling uniform, 3 AMS survivor draw,
 *   4 perturbation coefficients alpha_n, 5 initial velocity field,
 *   6 OU noise (test process).                                                */
void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4]);
double orc_u01(uint64_t x);                    /* (x >> 11) * 2^-53, in [0,1) */
uint64_t orc_below(uint64_t x, uint64_t m);    /* floor(x * m / 2^64), in [0,m) */

/* ---------------- D2Q9 lattice-BGK channel (App. A, Sec. 2) ---------- */
typedef struct {
    int32_t nx, ny;                 /* periodic in x; walls halfway below y=0 and above y=ny-1 */
    int32_t ox0, oy0, ow, oh;       /* solid cells [ox0,ox0+ow) x [oy0,oy0+oh); ow=0: no obstacle */
    double tau;                     /* BGK relaxation time, nu = (tau - 1/2)/3 */
    double gx, gy;                  /* constant body-force density on fluid nodes */
    int32_t collision;              /* 0: BGK; 1: central-moment multiple relaxation times */
    double omega_bulk, omega_3, omega_4;  /* collision 1: rates of the bulk (k20 + k02), third-
                                       order (k21, k12) and fourth-order (k22) central moments;
                                       shear (k20 - k02, k11) relaxes at 1/tau */
    /* open channel (Sec. 2): x not periodic; inlet column x = 0 held at the
     * equilibrium of rho = 1 and the parabolic profile of centreline u_in;
     * outlet column x = nx-1: rho = 1, u extrapolated (second order), the
     * populations regularized with the finite-difference strain rate.        */
    int32_t open_x;
    double u_in;
    int32_t grid_x0, grid_w, grid_bar, grid_gap;  /* entrance grid: cells x in [grid_x0, grid_x0+grid_w)
                                       with y mod (bar + gap) >= gap are solid; grid_w = 0: none */
    int32_t sponge_len;             /* tau rises to sponge_tau over the last sponge_len columns */
    double sponge_tau;
} orc_cfg;

int orc_is_solid(const orc_cfg* c, int x, int y);   /* obstacle or entrance grid */
/* relaxation time of column x (tau, or the sponge profile of an open channel) */
double orc_tau_at(const orc_cfg* c, int x);
/* inlet velocity of row y of an open channel */
double orc_inlet_u(const orc_cfg* c, int y);
/* equilibrium populations for density rho and velocity (ux, uy) */
void orc_feq(double rho, double ux, double uy, double feq[9]);
/* Guo forcing term S_q for velocity u and force density (gx, gy) */
void orc_guo(double ux, double uy, double gx, double gy, double S[9]);
/* central-moment collision of one node (App. A's production collision):
 *   out = f + S - T^{-1} Omega T (f - feq + S/2),
 * T_{pq,i} = (c_ix - ux)^p (c_iy - uy)^q, pq = 00 10 01 20 02 11 21 12 22;
 * Omega relaxes k20 - k02 and k11 at rates[0], k20 + k02 at rates[1], k21 and
 * k12 at rates[2], k22 at rates[3] (the conserved moments are unaffected).
 * rates all equal to omega give the BGK collision with Guo forcing.            */
void orc_cm_collide(const double f[9], double ux, double uy, const double feq[9], const double S[9],
                    const double rates[4], double out[9]);
/* equilibrium start with rho = 1 and a seeded uniform velocity perturbation of
 * amplitude amp on fluid nodes; solid nodes hold the rest weights w_q. */
void orc_init(const orc_cfg* c, uint64_t seed, int32_t clone, double amp, double* f);
/* one time step t -> t+1 of post-collision populations: stream (halfway
 * bounce-back on walls and obstacle) then BGK collision with Guo forcing.
 * force_obs[2] receives the momentum-exchange force on the obstacle and
 * force_wall[2] that on the two walls, both from the new populations.
 * Either may be NULL. */
void orc_step(const orc_cfg* c, const double* fin, double* fout,
              double* force_obs, double* force_wall);
/* run n steps from f (in place, using scratch of the same size); drag[t] =
 * x-force on the obstacle after step t+1 (may be NULL) */
void orc_run(const orc_cfg* c, double* f, double* scratch, int32_t n, double* drag);
/* total mass and momentum over fluid nodes */
void orc_moments(const orc_cfg* c, const double* f, double* mass, double* px, double* py);
/* density and velocity fields of post-collision populations:
 * rho = sum f, rho u = sum f c - F/2 (the step's force counted half) */
void orc_macro(const orc_cfg* c, const double* f, double* rho, double* ux, double* uy);

/* observables of the square (Sec. 2.1 and Sec. 3.2), from post-collision
 * populations (velocity as orc_macro):
 *   out[0] p_fb    = cs2 * sum of rho over the fluid column just upstream of
 *                    the square (x = ox0 - 1), its rows [oy0, oy0 + oh): the
 *                    forebody pressure integrated over the upstream face;
 *   out[1] p_base  = the same over the column just downstream (x = ox0 + ow);
 *                    eq. (drag_approx): f_d ~ p_fb - p_base;
 *   out[2] gamma_top, out[3] gamma_bottom: eq. (avg_shear_def), the mean over
 *                    the face's ow columns of d u_x / d y at the halfway wall,
 *                    from the two fluid rows beside it (distances 1/2 and 3/2):
 *                    du/dy = (9 u_1 - u_2) / 3 on the top face, the negative of
 *                    that with the rows below on the bottom face (exact for
 *                    u_x quadratic in the distance with u_x = 0 at the wall).
 * Returns -1 (out untouched) without a square, or when the square leaves fewer
 * than two fluid rows above or below it or no fluid column beside it. */
int orc_observables(const orc_cfg* c, const double* f, double out[4]);

/* ---------------- branching perturbation (App. D) -------------------- */
void orc_perturb_alphas(uint64_t seed, uint64_t iter, int32_t slot, int32_t n_s, double* alpha);
/* f_out = (f + eps * sum_n alpha_n snap_n) rescaled to the mass of f, fluid nodes only */
void orc_perturb(const orc_cfg* c, const double* f, int32_t n_s, const double* snaps,
                 const double* alpha, double eps, double* f_out);

/* ---------------- GKTL (App. C) -------------------------------------- */
/* W_n = N e^{s_n} / sum e^{s_m};  logR = log((1/N) sum e^{s_n}) */
int orc_gktl_weights(int32_t n, const double* s, double* W, double* logR);
/* residual-systematic resampling to N copies, slot assignment -> parent[N];
 * the weights must sum to N (relative 1e-9) */
int orc_gktl_select(int32_t n, const double* W, uint64_t seed, uint64_t iter, int32_t* parent);

/* ---------------- AMS (App. B.1) ------------------------------------- */
/* kill the trajectories holding the minimum maximum score; one survivor per
 * killed trajectory.  n_killed = n signals that all scores are equal (stop). */
int orc_ams_select(int32_t n, const double* Q, uint64_t seed, uint64_t iter,
                   int32_t* killed, int32_t* n_killed, int32_t* survivor, double* level);

/* ---------------- Ornstein-Uhlenbeck test process (App. B.2) ---------- */
/* exact AR(1) discretisation of dx = -x dt + dW with <dW dW> = dt */
double orc_ou_noise(uint64_t seed, uint64_t a, uint64_t b, uint64_t c);
/* GKTL on the OU process with observable A = x and potential kappa V, V = x
 * (kappa = 0: the plain algorithm).  Returns log Z = sum_i log R_i; every
 * output may be NULL:
 *   final_int[N]    time integral over [0, T_a] of each final trajectory;
 *   final_max_mean  with window T: max over t of (1/T) int_{t-T}^t x;
 *   final_hist      [N][M + 1] each final trajectory x_0..x_M (its genealogy);
 *   final_corr[N]   kappa (V(x_{T_a}) - V(x_0)) of each final trajectory;
 *   logR_out        [n_periods] log R_i of each cloning step. */
double orc_ou_gktl(int32_t n, int32_t n_periods, int32_t steps_per_period, double dt, double k, double kappa,
                   uint64_t seed, double* final_int, int32_t window_steps, double* final_max_mean,
                   double* final_hist, double* final_corr, double* logR_out);
/* direct sampling: fraction of n trajectories (stationary start) whose max over
 * steps 0..n_steps of x reaches each level a[j] */
void orc_ou_direct_max(int64_t n, int32_t n_steps, double dt, uint64_t seed,
                       int32_t n_a, const double* a, double* frac);
/* AMS on the OU process, score = x, fixed duration n_steps, stopping when the
 * killed level reaches a or after j_max iterations.  Returns the estimate of
 * P(max x >= a); *iters receives the number of iterations. */
double orc_ou_ams(int32_t n, int32_t n_steps, double dt, double a, int32_t j_max,
                  uint64_t seed, int32_t* iters);
/* AMS on the OU process with the trailing mean of x over score_window steps,
 * taken at every stride-th step, as score; stops when the killed level reaches
 * score_level or after j_max iterations.  Returns the estimate of
 * P(max_t x >= a), the killed trajectories included; *out_logw =
 * sum_j ln(1 - |K_j|/N) and out_event_max[N] = max_t x of each final
 * trajectory; one record per killed trajectory, in kill order, of the log
 * weight before its iteration (rec_logw) and its max_t x (rec_max), the first
 * rec_cap of them stored, their number in *n_rec (outputs may be NULL). */
double orc_ou_ams_score(int32_t n, int32_t n_steps, double dt, int32_t stride, int32_t score_window,
                        double score_level, double a, int32_t j_max, uint64_t seed, int32_t* iters,
                        double* out_logw, double* out_event_max, int32_t rec_cap, int32_t* n_rec,
                        double* rec_logw, double* rec_max);

#ifdef __cplusplus
}
#endif
#endif
