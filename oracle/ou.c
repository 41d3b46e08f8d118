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
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>
#include <string.h>

double orc_ou_gktl(int32_t n, int32_t n_periods, int32_t steps_per_period, double dt, double k,
                   uint64_t seed, double* final_int, int32_t window_steps, double* final_max_mean)
{
    const double a = exp(-dt), sig = sqrt((1.0 - a * a) / 2.0);
    const int32_t M = n_periods * steps_per_period;
    double* x = (double*)malloc(sizeof(double) * n);
    double* xn = (double*)malloc(sizeof(double) * n);
    double* integ = (double*)calloc((size_t)n, sizeof(double));
    double* integn = (double*)malloc(sizeof(double) * n);
    double* s = (double*)malloc(sizeof(double) * n);
    double* W = (double*)malloc(sizeof(double) * n);
    int32_t* parent = (int32_t*)malloc(sizeof(int32_t) * n);
    double* hist = (double*)malloc(sizeof(double) * (size_t)n * (M + 1));
    double* histn = (double*)malloc(sizeof(double) * (size_t)n * (M + 1));
    for (int32_t i = 0; i < n; ++i) {
        x[i] = sqrt(0.5) * orc_ou_noise(seed, 0u, (uint64_t)i, 0u);
        hist[(size_t)i * (M + 1)] = x[i];
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
            s[i] = k * acc;
        }
        double logR;
        orc_gktl_weights(n, s, W, &logR);
        logZ += logR;
        orc_gktl_select(n, W, seed, (uint64_t)p, parent);
        for (int32_t i = 0; i < n; ++i) {
            xn[i] = x[parent[i]];
            integn[i] = integ[parent[i]];
            memcpy(histn + (size_t)i * (M + 1), hist + (size_t)parent[i] * (M + 1), sizeof(double) * (M + 1));
        }
        memcpy(x, xn, sizeof(double) * n);
        memcpy(integ, integn, sizeof(double) * n);
        double* t = hist; hist = histn; histn = t;
    }
    for (int32_t i = 0; i < n; ++i) {
        if (final_int) final_int[i] = integ[i];
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
    free(x); free(xn); free(integ); free(integn); free(s); free(W); free(parent); free(hist); free(histn);
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

double orc_ou_ams(int32_t n, int32_t n_steps, double dt, double alev, int32_t j_max,
                  uint64_t seed, int32_t* iters)
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
        Q[i] = xi[0];
        for (int32_t m = 1; m <= n_steps; ++m) {
            xi[m] = a * xi[m - 1] + sig * orc_ou_noise(seed, (uint64_t)m, (uint64_t)i, 0u);
            if (xi[m] > Q[i]) Q[i] = xi[m];
        }
    }
    double logw = 0.0;
    int32_t done = 0;
    for (int32_t j = 1; j <= j_max; ++j) {
        int32_t nk;
        double z;
        orc_ams_select(n, Q, seed, (uint64_t)j, killed, &nk, surv, &z);
        if (z >= alev) break;
        if (nk == n) { logw = -INFINITY; break; }
        logw += log1p(-(double)nk / (double)n);
        done = j;
        for (int32_t kk = 0; kk < nk; ++kk) {
            double* xd = x + (size_t)killed[kk] * L;
            const double* xs = x + (size_t)surv[kk] * L;
            int32_t tb = 0;
            while (tb <= n_steps && !(xs[tb] > z)) tb++;
            /* the survivor's maximum exceeds z, so tb <= n_steps */
            memcpy(xd, xs, sizeof(double) * (size_t)(tb + 1));
            double q = -INFINITY;
            for (int32_t m = 0; m <= tb; ++m) if (xd[m] > q) q = xd[m];
            for (int32_t m = tb + 1; m <= n_steps; ++m) {
                xd[m] = a * xd[m - 1] + sig * orc_ou_noise(seed, (uint64_t)m, (uint64_t)killed[kk], (uint64_t)j);
                if (xd[m] > q) q = xd[m];
            }
            Q[killed[kk]] = q;
        }
    }
    if (iters) *iters = done;
    int32_t hit = 0;
    for (int32_t i = 0; i < n; ++i) if (Q[i] >= alev) hit++;
    double p = exp(logw) * (double)hit / (double)n;
    free(x); free(Q); free(killed); free(surv);
    return p;
}
