/*
 * Oracle (test infrastructure): selection rules of the two rare-event
 * algorithms, FP64 and integer, one thread.
 *
 * GKTL (App. C.1, eq. (Weight)): W_n = e^{s_n} / R with
 * R = (1/N) sum_n e^{s_n}, so that sum_n W_n = N.  The weights set how many
 * copies of each trajectory the next period starts from; the paper leaves the
 * resampling scheme to its references.  Reading used here: the copy number
 * must have mean W_n with the ensemble size held at N, which residual
 * resampling (Liu & Chen 1998) with a systematic draw of the residuals
 * (Kitagawa 1996; Carpenter, Clifford & Fearnhead 1999) achieves exactly:
 *   1. c_n = floor(W_n), residual r_n = W_n - floor(W_n), R = N - sum_n c_n;
 *   2. one uniform U; the R points (U + k) * C/R, k = 0..R-1, where C is the
 *      running sum of the residuals taken in ascending n, each add one copy to
 *      the trajectory whose residual interval [C_{n-1}, C_n) holds it;
 *   3. a trajectory with c_n >= 1 keeps its own slot n; its extra copies, taken
 *      in ascending n, fill the emptied slots in ascending order.
 *
 * AMS (App. B.1): the trajectories whose maximum score equals the minimum z
 * over the ensemble are discarded; each is replaced by a branch of a survivor
 * drawn uniformly among the others, taken in ascending order of the killed
 * index.
 */
#include "oracle.h"
#include <math.h>
#include <stdlib.h>

static uint64_t stream_word(uint64_t purpose, uint64_t seed, uint64_t a, uint64_t b)
{
    uint64_t ctr[4] = {purpose, a, b, 0u}, key[2] = {seed, 0u}, o[4];
    orc_philox4x64(ctr, key, o);
    return o[0];
}

int orc_gktl_weights(int32_t n, const double* s, double* W, double* logR)
{
    if (n <= 0) return -1;
    double m = -INFINITY;
    for (int32_t i = 0; i < n; ++i) {
        if (!isfinite(s[i])) return -3;
        if (s[i] > m) m = s[i];
    }
    double sum = 0.0;
    for (int32_t i = 0; i < n; ++i) sum += exp(s[i] - m);
    for (int32_t i = 0; i < n; ++i) W[i] = (double)n * exp(s[i] - m) / sum;
    if (logR) *logR = m + log(sum / (double)n);
    return 0;
}

int orc_gktl_select(int32_t n, const double* W, uint64_t seed, uint64_t iter, int32_t* parent)
{
    if (n <= 0) return -1;
    double total_w = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        if (!isfinite(W[i]) || W[i] < 0.0) return -3;
        total_w += W[i];
    }
    if (fabs(total_w - (double)n) > 1e-9 * (double)n) return -1; /* weights must sum to N */
    int32_t* cnt = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    double* res = (double*)malloc(sizeof(double) * (size_t)n);
    int64_t whole = 0;
    double csum = 0.0;
    for (int32_t i = 0; i < n; ++i) {
        double fl = floor(W[i]);
        cnt[i] = (int32_t)fl;
        res[i] = W[i] - fl;
        whole += cnt[i];
        csum += res[i];
    }
    int64_t R = (int64_t)n - whole;
    if (R < 0 || (R > 0 && !(csum > 0.0))) { free(cnt); free(res); return -1; }
    if (R > 0) {
        double U = orc_u01(stream_word(1u, seed, iter, 0u));
        double spacing = csum / (double)R;
        int32_t i = 0;
        double edge = res[0];
        for (int64_t k = 0; k < R; ++k) {
            double point = (U + (double)k) * spacing;
            while (point >= edge && i < n - 1) {
                i++;
                edge += res[i];
            }
            cnt[i] += 1;
        }
    }
    /* slot assignment */
    int32_t next_empty = 0;
    for (int32_t i = 0; i < n; ++i) parent[i] = (cnt[i] >= 1) ? i : -1;
    for (int32_t i = 0; i < n; ++i)
        for (int32_t e = 1; e < cnt[i]; ++e) {
            while (parent[next_empty] != -1) next_empty++;
            parent[next_empty] = i;
        }
    free(cnt);
    free(res);
    return 0;
}

int orc_ams_select(int32_t n, const double* Q, uint64_t seed, uint64_t iter,
                   int32_t* killed, int32_t* n_killed, int32_t* survivor, double* level)
{
    if (n <= 0) return -1;
    double z = INFINITY;
    for (int32_t i = 0; i < n; ++i) {
        if (isnan(Q[i])) return -3;
        if (Q[i] < z) z = Q[i];
    }
    int32_t nk = 0;
    for (int32_t i = 0; i < n; ++i)
        if (Q[i] == z) killed[nk++] = i;
    *n_killed = nk;
    *level = z;
    if (nk == n) return 0; /* every trajectory sits at the level: nothing survives */
    for (int32_t k = 0; k < nk; ++k) {
        uint64_t r = orc_below(stream_word(3u, seed, iter, (uint64_t)killed[k]), (uint64_t)(n - nk));
        int64_t seen = 0;
        for (int32_t i = 0; i < n; ++i) {
            if (Q[i] == z) continue;
            if (seen == (int64_t)r) { survivor[k] = i; break; }
            seen++;
        }
    }
    return 0;
}
