/*
 * Oracle (test infrastructure): the Ornstein-Uhlenbeck test process of
 * App. B.2, dx/dt = -x + eta with <eta(t) eta(t')> = delta(t - t'), driven by
 * the GKTL (App. C.1) and AMS (App. B.1) algorithms of the oracle.
 *
 * Discretisation: the exact AR(1) update over a step dt,
 *   x_{m+1} = a x_m + sqrt((1 - a^2)/2) xi_m,  a = e^{-dt},  xi_m ~ N(0,1),
 * whose stationary law N(0, 1/2) is that of the continuous process.  Time
 * integrals are right-point sums dt * sum_m x_m.
 *
 * Noise counters (stream 6): GKTL  (step, slot, 0);
 *                            AMS   (step, slot, 0) initially, (step, slot, j) on
 *                                  the branch made at iteration j >= 1.
 *
 * GKTL with a potential (the learned score's role in selection): the exponent
 * of period i gains kappa (V(x_{t_i}) - V(x_{t_{i-1}})), V(x) = x here.  The
 * sum telescopes along a genealogy to kappa (V(x_{T_a}) - V(x_0)), so App. C.2's
 * estimator stays exact once each final trajectory is weighted by
 * e^{-kappa (V(x_{T_a}) - V(x_0))}, x_0 being the start of its ancestor; the
 * potential changes which trajectories are cloned, not what is estimated.
 *
 * AMS with a score other than the event's observable (generalised AMS,
 * Brehier, Lelievre & Rousset 2016): the score is the trailing mean of x over
 * score_window steps, seen only every `stride` steps (checkpoint times); the
 * event is max_t x >= a.  Killing, branching and the weights follow the score.
 * The estimate of E[phi(X)] sums every trajectory the run has seen with its
 * weight: a trajectory killed at iteration j counts with
 * prod_{i<j} (1 - |K_i|/N) / N, a final one with prod_{all j} (1 - |K_j|/N) / N.
 * When the event is the score reaching a (the plain AMS) every killed
 * trajectory lies below a and only the final ensemble counts; with another
 * score a killed trajectory may hold the event, and leaving it out biases the
 * estimate low.  When every score ties (all would be killed) the run stops and
 * the ensemble counts with the current weight, which equals killing them all.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

double orc_ou_gktl(int32_t n, int32_t n_periods, int32_t steps_per_period, double dt, double k, double kappa,
                   uint64_t seed, double* final_int, int32_t window_steps, double* final_max_mean,
                   double* final_hist, double* final_corr, double* logR_out)
{
    const double a = exp(-dt), sig = sqrt((1.0 - a * a) / 2.0);
    const int32_t M = n_periods * steps_per_period;
    double* x = (double*)malloc(sizeof(double) * n);
    double* xn = (double*)malloc(sizeof(double) * n);
    double* integ = (double*)calloc((size_t)n, sizeof(double));
    double* integn = (double*)malloc(sizeof(double) * n);
    double* v0 = (double*)malloc(sizeof(double) * n);     /* V at the start of the ancestor */
    double* v0n = (double*)malloc(sizeof(double) * n);
    double* vprev = (double*)malloc(sizeof(double) * n);  /* V at the last cloning time */
    double* s = (double*)malloc(sizeof(double) * n);
    double* W = (double*)malloc(sizeof(double) * n);
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * n);
    double* hist = (double*)malloc(sizeof(double) * (size_t)n * (M + 1));
    double* histn = (double*)malloc(sizeof(double) * (size_t)n * (M + 1));
    for (int32_t i = 0; i < n; ++i) {
        x[i] = sqrt(0.5) * orc_ou_noise(seed, 0u, (uint64_t)i, 0u);
        hist[(size_t)i * (M + 1)] = x[i];
        v0[i] = x[i];
        vprev[i] = x[i];
    }
    double logZ = 0.0;
    for (int32_t p = 0; p < n_periods; ++p) {
        for (int32_t i = 0; i < n; ++i) {
            double acc = 0.0;
            for (int32_t m = 0; m < steps_per_period; ++m) {
                int32_t step = p * steps_per_period + m + 1;
                x[i] = a * x[i] + sig * orc_ou_noise(seed, (uint64_t)step, (uint64_t)i, 0u);
                hist[(size_t)i * (M + 1) + step] = x[i];
                acc += dt * x[i];
            }
            integ[i] += acc;
            s[i] = k * acc + kappa * (x[i] - vprev[i]);
        }
        double logR;
        orc_gktl_weights(n, s, W, &logR);
        logZ += logR;
        if (logR_out) logR_out[p] = logR;
        orc_gktl_select(n, W, seed, (uint64_t)p, parent);
        for (int32_t i = 0; i < n; ++i) {
            xn[i] = x[parent[i]];
            integn[i] = integ[parent[i]];
            v0n[i] = v0[parent[i]];
            memcpy(histn + (size_t)i * (M + 1), hist + (size_t)parent[i] * (M + 1), sizeof(double) * (M + 1));
        }
        memcpy(x, xn, sizeof(double) * n);
        memcpy(integ, integn, sizeof(double) * n);
        memcpy(v0, v0n, sizeof(double) * n);
        memcpy(vprev, xn, sizeof(double) * n);
        double* t = hist; hist = histn; histn = t;
    }
    for (int32_t i = 0; i < n; ++i) {
        if (final_int) final_int[i] = integ[i];
        if (final_corr) final_corr[i] = kappa * (x[i] - v0[i]);
        if (final_hist) memcpy(final_hist + (size_t)i * (M + 1), hist + (size_t)i * (M + 1), sizeof(double) * (M + 1));
        if (final_max_mean) {
            double best = -INFINITY;
            for (int32_t t = window_steps; t <= M; ++t) {
                double acc = 0.0;
                for (int32_t m = t - window_steps + 1; m <= t; ++m) acc += hist[(size_t)i * (M + 1) + m];
                double mean = acc / window_steps;
                if (mean > best) best = mean;
            }
            final_max_mean[i] = best;
        }
    }
    free(x); free(xn); free(integ); free(integn); free(v0); free(v0n); free(vprev); free(s); free(W); free(parent);
    free(hist); free(histn);
    return logZ;
}

void orc_ou_direct_max(int64_t n, int32_t n_steps, double dt, uint64_t seed,
                       int32_t n_a, const double* alev, double* frac)
{
    const double a = exp(-dt), sig = sqrt((1.0 - a * a) / 2.0);
    int64_t* hits = (int64_t*)calloc((size_t)n_a, sizeof(int64_t));
    for (int64_t i = 0; i < n; ++i) {
        double x = sqrt(0.5) * orc_ou_noise(seed, 0u, (uint64_t)i, 0u), mx = x;
        for (int32_t m = 1; m <= n_steps; ++m) {
            x = a * x + sig * orc_ou_noise(seed, (uint64_t)m, (uint64_t)i, 0u);
            if (x > mx) mx = x;
        }
        for (int32_t j = 0; j < n_a; ++j)
            if (mx >= alev[j]) hits[j]++;
    }
    for (int32_t j = 0; j < n_a; ++j) frac[j] = (double)hits[j] / (double)n;
    free(hits);
}

/* score of a stored path at step t: mean of x over the score_window steps
 * ending at t (fewer at the start of the path) */
static double ams_score_at(const double* xs, int32_t t, int32_t score_window)
{
    int32_t m0 = t - score_window + 1;
    if (m0 < 0) m0 = 0;
    double acc = 0.0;
    for (int32_t m = m0; m <= t; ++m) acc += xs[m];
    return acc / (double)(t - m0 + 1);
}

/* maximum of the score over the checkpoint times 0, stride, 2 stride, ... */
static double ams_score_max(const double* xs, int32_t n_steps, int32_t stride, int32_t score_window)
{
    double q = -INFINITY;
    for (int32_t t = 0; t <= n_steps; t += stride) {
        double v = ams_score_at(xs, t, score_window);
        if (v > q) q = v;
    }
    return q;
}

static double path_max(const double* xs, int32_t n_steps)
{
    double mx = -INFINITY;
    for (int32_t m = 0; m <= n_steps; ++m) if (xs[m] > mx) mx = xs[m];
    return mx;
}

double orc_ou_ams_score(int32_t n, int32_t n_steps, double dt, int32_t stride, int32_t score_window,
                        double score_level, double alev, int32_t j_max, uint64_t seed, int32_t* iters,
                        double* out_logw, double* out_event_max, int32_t rec_cap, int32_t* n_rec,
                        double* rec_logw, double* rec_max)
{
    const double a = exp(-dt), sig = sqrt((1.0 - a * a) / 2.0);
    const int32_t L = n_steps + 1;
    double* x = (double*)malloc(sizeof(double) * (size_t)n * L);
    double* Q = (double*)malloc(sizeof(double) * n);
    int32_t* killed = (int32_t*)malloc(sizeof(int32_t) * n);
    int32_t* surv = (int32_t*)malloc(sizeof(int32_t) * n);
    for (int32_t i = 0; i < n; ++i) {
        double* xi = x + (size_t)i * L;
        xi[0] = sqrt(0.5) * orc_ou_noise(seed, 0u, (uint64_t)i, 0u);
        for (int32_t m = 1; m <= n_steps; ++m)
            xi[m] = a * xi[m - 1] + sig * orc_ou_noise(seed, (uint64_t)m, (uint64_t)i, 0u);
        Q[i] = ams_score_max(xi, n_steps, stride, score_window);
    }
    double logw = 0.0, p_killed = 0.0;
    int32_t done = 0, nr = 0;
    for (int32_t j = 1; j <= j_max; ++j) {
        int32_t nk;
        double z;
        orc_ams_select(n, Q, seed, (uint64_t)j, killed, &nk, surv, &z);
        if (z >= score_level) break;
        if (nk == n) break;  /* every score ties: the ensemble counts as it stands */
        for (int32_t kk = 0; kk < nk; ++kk) {  /* the killed trajectories, with the weight before j */
            const double mk = path_max(x + (size_t)killed[kk] * L, n_steps);
            if (mk >= alev) p_killed += exp(logw) / (double)n;
            if (nr < rec_cap) { rec_logw[nr] = logw; rec_max[nr] = mk; }
            nr++;
        }
        logw += log1p(-(double)nk / (double)n);
        done = j;
        for (int32_t kk = 0; kk < nk; ++kk) {
            double* xd = x + (size_t)killed[kk] * L;
            const double* xs = x + (size_t)surv[kk] * L;
            /* first checkpoint time where the survivor's score exceeds z; its
             * maximum exceeds z, so one exists */
            int32_t tb = 0;
            while (tb <= n_steps && !(ams_score_at(xs, tb, score_window) > z)) tb += stride;
            memcpy(xd, xs, sizeof(double) * (size_t)(tb + 1));
            for (int32_t m = tb + 1; m <= n_steps; ++m)
                xd[m] = a * xd[m - 1] + sig * orc_ou_noise(seed, (uint64_t)m, (uint64_t)killed[kk], (uint64_t)j);
            Q[killed[kk]] = ams_score_max(xd, n_steps, stride, score_window);
        }
    }
    if (iters) *iters = done;
    if (n_rec) *n_rec = nr;
    int32_t hit = 0;
    for (int32_t i = 0; i < n; ++i) {
        const double mx = path_max(x + (size_t)i * L, n_steps);
        if (out_event_max) out_event_max[i] = mx;
        if (mx >= alev) hit++;
    }
    if (out_logw) *out_logw = logw;
    double p = p_killed + exp(logw) * (double)hit / (double)n;
    free(x); free(Q); free(killed); free(surv);
    return p;
}

double orc_ou_ams(int32_t n, int32_t n_steps, double dt, double alev, int32_t j_max,
                  uint64_t seed, int32_t* iters)
{
    /* score = x at every step; the event is the score reaching a */
    return orc_ou_ams_score(n, n_steps, dt, 1, 1, alev, alev, j_max, seed, iters, NULL, NULL, 0, NULL, NULL, NULL);
}
