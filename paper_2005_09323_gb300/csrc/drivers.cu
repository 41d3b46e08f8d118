// Native drivers of the two rare-event algorithms on an ensemble, and the
// estimators that turn their output into probabilities and return times.
//   GKTL (App. C.1): periods of tau steps; after each, weights from the drag
//   integral, resampling, cloning with the App. D perturbation; log Z = sum_i
//   log R_i.  Estimator (App. C.2): P(F_T >= a) = (1/N) sum_j Z e^{-k I_j}
//   1{max F_T^(j) >= a}, r(a) = -(T_a - T) / ln(1 - P).
//   AMS (App. B.1): trajectories of fixed duration T_a, score = time-averaged
//   drag over a window (or a learned score); kill the minimum maximum, branch a
//   survivor at the killed level, re-simulate.  Estimator (generalised AMS):
//   every trajectory the run has seen counts with its weight over N - a killed
//   one with prod_{i<j} (1 - |K_i|/N), a final one with prod_j (1 - |K_j|/N) -
//   times 1{its time-averaged drag maximum >= a}.  With the drag as score the
//   killed ones all lie below the levels above the last killed one.
#include <algorithm>
#include <cmath>
#include <vector>

#include "internal.h"
#include "lbm_device.cuh"

namespace lbm {

constexpr int kEstThreads = 256;

// one block per level; fixed-order FP64 sums
__global__ void gktl_probability_kernel(int32_t n, double k, const double* logR, int32_t n_periods,
                                        const double* integral, const double* maxima, const double* correction,
                                        const double* levels, double t_a, double t_window, double* p_out,
                                        double* r_out)
{
    __shared__ double sh[kEstThreads];
    __shared__ double logz;
    if (threadIdx.x == 0) {
        double z = 0.0;
        for (int i = 0; i < n_periods; ++i) z += logR[i];
        logz = z;
    }
    __syncthreads();
    const double a = levels[blockIdx.x];
    double acc = 0.0;
    for (int j = threadIdx.x; j < n; j += kEstThreads)
        if (maxima[j] >= a) acc += exp(logz - k * integral[j] - (correction ? correction[j] : 0.0));
    sh[threadIdx.x] = acc;
    __syncthreads();
    for (int off = kEstThreads / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) sh[threadIdx.x] += sh[threadIdx.x + off];
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        const double p = sh[0] / (double)n;
        p_out[blockIdx.x] = p;
        if (r_out) r_out[blockIdx.x] = -(t_a - t_window) / log1p(-p);
    }
}

// one block per level: the final ensemble's count and the killed records'
// weighted sum, fixed-order reductions
__global__ void ams_probability_kernel(int32_t n, double log_weight, const double* Q, int32_t n_rec,
                                       const double* rec_logw, const double* rec_max, const double* levels,
                                       double* p_out)
{
    __shared__ int sh[kEstThreads];
    __shared__ double shr[kEstThreads];
    const double a = levels[blockIdx.x];
    int cnt = 0;
    for (int j = threadIdx.x; j < n; j += kEstThreads) cnt += Q[j] >= a ? 1 : 0;
    double acc = 0.0;
    for (int r = threadIdx.x; r < n_rec; r += kEstThreads)
        if (rec_max[r] >= a) acc += exp(rec_logw[r]);
    sh[threadIdx.x] = cnt;
    shr[threadIdx.x] = acc;
    __syncthreads();
    for (int off = kEstThreads / 2; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off) {
            sh[threadIdx.x] += sh[threadIdx.x + off];
            shr[threadIdx.x] += shr[threadIdx.x + off];
        }
        __syncthreads();
    }
    if (threadIdx.x == 0) p_out[blockIdx.x] = (exp(log_weight) * (double)sh[0] + shr[0]) / (double)n;
}

// s_n += kappa (V_now - V_prev): the telescoping potential of the exponent
__global__ void add_potential_kernel(double* s, const double* vnow, const double* vprev, double kappa, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) s[i] += kappa * (vnow[i] - vprev[i]);
}

// per-slot potentials follow the clones: out_a[s] = a[parent[s]], out_b[s] = b[parent[s]]
__global__ void gather2_kernel(const int32_t* parent, const double* a, const double* b, double* out_a, double* out_b,
                               int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    const int p = parent[i];
    const int q = (p >= 0 && p < n) ? p : i;
    out_a[i] = a[q];
    out_b[i] = b[q];
}

__global__ void correction_kernel(const double* vend, const double* v0, double kappa, double* out, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = kappa * (vend[i] - v0[i]);
}

// Q_n = max over checkpoints k0..k1 of the learned score
__global__ void score_max_kernel(const double* score, int32_t n_ckpt, int32_t k0, int32_t k1, double* Q, int n)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    double m = -INFINITY;
    for (int k = k0; k <= k1; ++k) m = fmax(m, score[(int64_t)i * n_ckpt + k]);
    Q[i] = m;
}

}  // namespace lbm

using namespace lbm;

extern "C" {

int gktl_probability(int32_t n, double k, const double* logR_dev, int32_t n_periods, const double* integral_dev,
                     const double* maxima_dev, const double* correction_dev, int32_t n_levels,
                     const double* levels_dev, double t_a, double t_window, double* p_dev, double* r_dev, void* stream)
{
    if (n < 1 || n_periods < 0 || n_levels < 1 || n_levels > 65535) return fail(LBM_ERR_ARG, "gktl_probability: sizes");
    if ((n_periods > 0 && !logR_dev) || !integral_dev || !maxima_dev || !levels_dev || !p_dev)
        return fail(LBM_ERR_ARG, "gktl_probability: null pointer");
    if (!std::isfinite(k)) return fail(LBM_ERR_ARG, "gktl_probability: k must be finite");
    gktl_probability_kernel<<<n_levels, kEstThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        n, k, logR_dev, n_periods, integral_dev, maxima_dev, correction_dev, levels_dev, t_a, t_window, p_dev, r_dev);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    return LBM_OK;
}

int ams_probability(int32_t n, double log_weight, const double* Q_dev, int32_t n_records, const double* rec_logw_dev,
                    const double* rec_max_dev, int32_t n_levels, const double* levels_dev, double* p_dev, void* stream)
{
    if (n < 1 || n_levels < 1 || n_levels > 65535 || n_records < 0) return fail(LBM_ERR_ARG, "ams_probability: sizes");
    if (!Q_dev || !levels_dev || !p_dev) return fail(LBM_ERR_ARG, "ams_probability: null pointer");
    if (n_records > 0 && (!rec_logw_dev || !rec_max_dev))
        return fail(LBM_ERR_ARG, "ams_probability: null killed records");
    ams_probability_kernel<<<n_levels, kEstThreads, 0, static_cast<cudaStream_t>(stream)>>>(
        n, log_weight, Q_dev, n_records, rec_logw_dev, rec_max_dev, levels_dev, p_dev);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    return LBM_OK;
}

int lbm_gktl_run(lbm_ensemble* e, const lbm_gktl_params* prm, double* logR_dev, int32_t* parent_dev,
                 double* integral_dev, double* maxima_dev, double* correction_dev)
{
    if (!e || !prm) return fail(LBM_ERR_ARG, "lbm_gktl_run: null argument");
    const lbm_gktl_params p = *prm;
    if (p.period < 1 || p.n_periods < 1) return fail(LBM_ERR_ARG, "lbm_gktl_run: period and n_periods must be >= 1");
    if (!std::isfinite(p.k) || !std::isfinite(p.eps) || p.eps < 0) return fail(LBM_ERR_ARG, "lbm_gktl_run: k, eps");
    if (!logR_dev || !parent_dev) return fail(LBM_ERR_ARG, "lbm_gktl_run: logR_dev and parent_dev are required");
    const int32_t t0 = e->t_host[0];
    for (int i = 1; i < e->n; ++i)
        if (e->t_host[i] != t0) return fail(LBM_ERR_STATE, "lbm_gktl_run: clones at different times");
    const int64_t t_end = (int64_t)t0 + (int64_t)p.period * p.n_periods;
    if (t_end > e->cfg.max_steps) return fail(LBM_ERR_ARG, "lbm_gktl_run: the run exceeds max_steps");
    if (p.window < 0 || p.window > t_end - t0) return fail(LBM_ERR_ARG, "lbm_gktl_run: window longer than the run");
    if (p.eps != 0.0 && e->n_snaps_set < 1) return fail(LBM_ERR_STATE, "lbm_gktl_run: perturbation needs snapshots");
    if (e->n > 4096) return fail(LBM_ERR_ARG, "lbm_gktl_run: at most 4096 clones");
    if (!std::isfinite(p.kappa)) return fail(LBM_ERR_ARG, "lbm_gktl_run: kappa must be finite");
    const bool pot = p.kappa != 0.0;
    if (pot && !e->cnn) return fail(LBM_ERR_STATE, "lbm_gktl_run: kappa != 0 needs a learned score attached");
    // weights and exponents live in the ensemble's reduction scratch
    double* s = e->red_partials;
    double* W = e->red_partials + e->n;
    int32_t* status = e->flag_dev + 1;
    int rc;
    std::vector<int32_t> all(e->n);
    for (int i = 0; i < e->n; ++i) all[i] = i;
    // clones whose current states refill the App. D bank (evenly spaced)
    std::vector<int32_t> bank;
    const int n_bank = std::min(e->cfg.n_snapshots, e->n);
    for (int i = 0; i < n_bank; ++i) bank.push_back((int32_t)((int64_t)i * e->n / n_bank));
    const int nb = (e->n + 127) / 128;
    if (pot) {  // V at the start of every trajectory: pot[2] (start) and pot[1] (previous)
        if ((rc = score_clones(e, all.data(), e->n, e->pot[2], 1, 0))) return rc;
        LBM_CUDA(cudaMemcpyAsync(e->pot[1], e->pot[2], sizeof(double) * e->n, cudaMemcpyDeviceToDevice, e->stream));
    }
    for (int32_t i = 0; i < p.n_periods; ++i) {
        const int32_t ta = t0 + i * p.period;
        int32_t* par = parent_dev + (int64_t)i * e->n;
        if ((rc = lbm_ensemble_step(e, p.period))) return rc;
        if ((rc = lbm_ensemble_window_sum(e, ta, ta + p.period, p.k, s))) return rc;
        if (pot) {
            if ((rc = score_clones(e, all.data(), e->n, e->pot[0], 1, 0))) return rc;
            add_potential_kernel<<<nb, 128, 0, e->stream>>>(s, e->pot[0], e->pot[1], p.kappa, e->n);
            LBM_CUDA(cudaGetLastError());
            count_launches(1);
        }
        if ((rc = gktl_weights(e->n, s, W, logR_dev + i, e->stream))) return rc;
        if ((rc = gktl_select(e->n, W, p.seed, (uint64_t)i, par, status, e->stream))) return rc;
        if (p.refresh_snapshots && p.eps != 0.0) {  // contemporaneous perturbation directions
            if ((rc = lbm_ensemble_set_snapshots(e, (int32_t)bank.size(), bank.data()))) return rc;
        }
        if ((rc = lbm_ensemble_clone(e, par, p.eps, p.seed, (uint64_t)i))) return rc;
        if (pot) {
            gather2_kernel<<<nb, 128, 0, e->stream>>>(par, e->pot[0], e->pot[2], e->pot_tmp[0], e->pot_tmp[1], e->n);
            LBM_CUDA(cudaGetLastError());
            count_launches(1);
            std::swap(e->pot[1], e->pot_tmp[0]);  // previous = now, of the parent
            std::swap(e->pot[2], e->pot_tmp[1]);  // start, of the parent
        }
    }
    if (correction_dev) {
        if (pot) {
            correction_kernel<<<nb, 128, 0, e->stream>>>(e->pot[1], e->pot[2], p.kappa, correction_dev, e->n);
            LBM_CUDA(cudaGetLastError());
            count_launches(1);
        } else {
            LBM_CUDA(cudaMemsetAsync(correction_dev, 0, sizeof(double) * e->n, e->stream));
        }
    }
    if (integral_dev && (rc = lbm_ensemble_window_sum(e, t0, (int32_t)t_end, 1.0, integral_dev))) return rc;
    if (maxima_dev && p.window > 0 && (rc = lbm_ensemble_scores(e, p.window, t0, (int32_t)t_end, maxima_dev)))
        return rc;
    int32_t st = 0;
    LBM_CUDA(cudaMemcpyAsync(&st, status, sizeof(int32_t), cudaMemcpyDeviceToHost, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    if (st != 0) return fail(st, "lbm_gktl_run: a resampling step rejected its weights (non-finite drag?)");
    int32_t flag = 0;
    LBM_CUDA(cudaMemcpy(&flag, e->flag_dev, sizeof(int32_t), cudaMemcpyDeviceToHost));
    if (flag) return fail(LBM_ERR_NONFINITE, "lbm_gktl_run: a drag value became non-finite");
    return LBM_OK;
}

int lbm_ams_run(lbm_ensemble* e, const lbm_ams_params* prm, int32_t* iterations, double* log_weight, double* Q_dev,
                double* levels, int32_t* n_killed, double* killed_max)
{
    if (!e || !prm || !iterations || !log_weight || !Q_dev) return fail(LBM_ERR_ARG, "lbm_ams_run: null argument");
    const lbm_ams_params p = *prm;
    if (p.t_a < 1 || p.window < 1 || p.window > p.t_a || p.max_iter < 0)
        return fail(LBM_ERR_ARG, "lbm_ams_run: need 1 <= window <= t_a and max_iter >= 0");
    if (!std::isfinite(p.eps) || p.eps < 0 || std::isnan(p.level)) return fail(LBM_ERR_ARG, "lbm_ams_run: eps, level");
    if (e->cfg.ckpt_stride <= 0) return fail(LBM_ERR_STATE, "lbm_ams_run: branching needs checkpoints");
    if (p.eps != 0.0 && e->n_snaps_set < 1) return fail(LBM_ERR_STATE, "lbm_ams_run: perturbation needs snapshots");
    if (e->n < 2 || e->n > 4096) return fail(LBM_ERR_ARG, "lbm_ams_run: 2 to 4096 trajectories");
    const int32_t t0 = e->t_host[0];
    for (int i = 1; i < e->n; ++i)
        if (e->t_host[i] != t0) return fail(LBM_ERR_STATE, "lbm_ams_run: clones at different times");
    if (t0 % e->cfg.ckpt_stride != 0) return fail(LBM_ERR_STATE, "lbm_ams_run: start time not on a checkpoint");
    const int32_t t_end = t0 + p.t_a;
    if ((int64_t)t_end > e->cfg.max_steps) return fail(LBM_ERR_ARG, "lbm_ams_run: t_a exceeds max_steps");
    const bool learned = p.score_kind == 1;
    if (p.score_kind != 0 && !learned) return fail(LBM_ERR_ARG, "lbm_ams_run: score_kind is 0 (drag) or 1 (learned)");
    if (learned && !e->cnn) return fail(LBM_ERR_STATE, "lbm_ams_run: the learned score needs a model attached");
    if (learned && p.t_a % e->cfg.ckpt_stride) return fail(LBM_ERR_ARG, "lbm_ams_run: t_a not a multiple of ckpt_stride");
    const int32_t C = e->cfg.ckpt_stride, k0 = t0 / C, k1 = t_end / C;
    std::vector<int32_t> all(e->n);
    for (int i = 0; i < e->n; ++i) all[i] = i;
    std::vector<int32_t> bank;
    const int n_bank = std::min(e->cfg.n_snapshots, e->n);
    for (int i = 0; i < n_bank; ++i) bank.push_back((int32_t)((int64_t)i * e->n / n_bank));
    // score maxima of the current ensemble
    auto maxima = [&]() -> int {
        if (!learned) return lbm_ensemble_scores(e, p.window, t0, t_end, Q_dev);
        score_max_kernel<<<(e->n + 127) / 128, 128, 0, e->stream>>>(e->cnn_score, e->n_ckpt, k0, k1, Q_dev, e->n);
        LBM_CUDA(cudaGetLastError());
        count_launches(1);
        return LBM_OK;
    };
    // first time the survivor's score exceeds the level (a checkpoint time for the learned score)
    std::vector<double> row(learned ? e->n_ckpt : 0);
    auto crossing = [&](int32_t surv, double z, int32_t* tb) -> int {
        if (!learned) return lbm_ensemble_first_crossing(e, surv, z, tb);
        LBM_CUDA(cudaMemcpyAsync(row.data(), e->cnn_score + (size_t)surv * e->n_ckpt, sizeof(double) * e->n_ckpt,
                                 cudaMemcpyDeviceToHost, e->stream));
        LBM_CUDA(cudaStreamSynchronize(e->stream));
        *tb = -1;
        for (int32_t k = k0; k <= k1; ++k)
            if (row[k] > z) {
                *tb = k * C;
                break;
            }
        return LBM_OK;
    };
    int rc;
    if (learned && (rc = score_clones(e, all.data(), e->n, e->cnn_score, e->n_ckpt, k0))) return rc;
    if ((rc = lbm_ensemble_step(e, p.t_a))) return rc;
    if ((rc = maxima())) return rc;
    int32_t* killed = reinterpret_cast<int32_t*>(e->red_partials);
    int32_t* surv = killed + e->n;
    int32_t* nk_dev = surv + e->n;
    double* z_dev = e->red_partials + 2 * (size_t)e->n;  // after the two int tables (2n ints = n doubles)
    double* ev_dev = e->red_partials + 3 * (size_t)e->n;  // event maxima before a kill (learned score)
    std::vector<int32_t> hk(e->n), hs(e->n);
    std::vector<double> ev(learned ? e->n : 0);
    double lw = 0.0;
    int32_t done = 0;
    for (int32_t j = 1; j <= p.max_iter; ++j) {
        if ((rc = ams_select(e->n, Q_dev, p.seed, (uint64_t)j, killed, nk_dev, surv, z_dev, e->stream))) return rc;
        int32_t nk = 0;
        double z = 0.0;
        LBM_CUDA(cudaMemcpyAsync(&nk, nk_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, e->stream));
        LBM_CUDA(cudaMemcpyAsync(&z, z_dev, sizeof(double), cudaMemcpyDeviceToHost, e->stream));
        LBM_CUDA(cudaStreamSynchronize(e->stream));
        if (nk < 0) return fail(LBM_ERR_NONFINITE, "lbm_ams_run: a score is NaN");
        if (z >= p.level || nk >= e->n) break;
        LBM_CUDA(cudaMemcpyAsync(hk.data(), killed, sizeof(int32_t) * nk, cudaMemcpyDeviceToHost, e->stream));
        LBM_CUDA(cudaMemcpyAsync(hs.data(), surv, sizeof(int32_t) * nk, cudaMemcpyDeviceToHost, e->stream));
        if (learned && killed_max) {  // the killed trajectories' own event maxima, before they are replaced
            if ((rc = lbm_ensemble_scores(e, p.window, t0, t_end, ev_dev))) return rc;
            LBM_CUDA(cudaMemcpyAsync(ev.data(), ev_dev, sizeof(double) * e->n, cudaMemcpyDeviceToHost, e->stream));
        }
        LBM_CUDA(cudaStreamSynchronize(e->stream));
        if (killed_max)  // with the drag as score a killed trajectory's maximum is the level itself
            for (int32_t i = 0; i < nk; ++i) killed_max[(int64_t)(j - 1) * e->n + i] = learned ? ev[hk[i]] : z;
        // branching times from the scores of the survivors (not modified here)
        std::vector<int32_t> tb(nk);
        for (int32_t i = 0; i < nk; ++i) {
            if ((rc = crossing(hs[i], z, &tb[i]))) return rc;
            if (tb[i] < 0) return fail(LBM_ERR_STATE, "lbm_ams_run: survivor never exceeds the level");
        }
        for (int32_t i = 0; i < nk; ++i) {
            if (p.refresh_snapshots && p.eps != 0.0) {  // states of the flow at the branching checkpoint
                const int32_t kc = tb[i] / C;
                if ((rc = lbm_ensemble_set_snapshots_from_checkpoint(e, (int32_t)bank.size(), bank.data(), kc)))
                    return rc;
            }
            if ((rc = lbm_ensemble_branch(e, hk[i], hs[i], tb[i], p.eps, p.seed, (uint64_t)j))) return rc;
            if (t_end > tb[i] && (rc = lbm_ensemble_step_clones(e, t_end - tb[i], &hk[i], 1))) return rc;
        }
        if ((rc = maxima())) return rc;
        lw += std::log1p(-(double)nk / (double)e->n);
        if (levels) levels[j - 1] = z;
        if (n_killed) n_killed[j - 1] = nk;
        done = j;
    }
    *iterations = done;
    *log_weight = lw;
    int32_t flag = 0;
    LBM_CUDA(cudaMemcpyAsync(&flag, e->flag_dev, sizeof(int32_t), cudaMemcpyDeviceToHost, e->stream));
    LBM_CUDA(cudaStreamSynchronize(e->stream));
    if (flag) return fail(LBM_ERR_NONFINITE, "lbm_ams_run: a drag value became non-finite");
    return LBM_OK;
}

}  // extern "C"
