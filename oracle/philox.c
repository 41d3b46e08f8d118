/*
 * Oracle (test infrastructure): counter-based random numbers.
 *
 * Philox4x64-10 as defined by Salmon, Moraes, Dror & Shaw, "Parallel random
 * numbers: as easy as 1, 2, 3" (SC'11): ten rounds of two 64x64->128-bit
 * multiplications whose halves are xor-ed with the other two counter words
 * and the key, the key being bumped by two Weyl constants between rounds.
 * Pinned against numpy.random.Philox (the same generator) in the tests.
 */
#include "oracle.h"
#include <math.h>

static void mulhilo64(uint64_t a, uint64_t b, uint64_t* hi, uint64_t* lo)
{
    unsigned __int128 p = (unsigned __int128)a * (unsigned __int128)b;
    *hi = (uint64_t)(p >> 64);
    *lo = (uint64_t)p;
}

void orc_philox4x64(const uint64_t ctr[4], const uint64_t key[2], uint64_t out[4])
{
    /* round multipliers and key increments from the SC'11 paper */
    const uint64_t M0 = 0xD2E7470EE14C6C93ULL, M1 = 0xCA5A826395121157ULL;
    const uint64_t W0 = 0x9E3779B97F4A7C15ULL, W1 = 0xBB67AE8584CAA73BULL;
    uint64_t x0 = ctr[0], x1 = ctr[1], x2 = ctr[2], x3 = ctr[3];
    uint64_t k0 = key[0], k1 = key[1];
    for (int r = 0; r < 10; ++r) {
        if (r > 0) { k0 += W0; k1 += W1; }
        uint64_t hi0, lo0, hi1, lo1;
        mulhilo64(M0, x0, &hi0, &lo0);
        mulhilo64(M1, x2, &hi1, &lo1);
        uint64_t y0 = hi1 ^ x1 ^ k0;
        uint64_t y1 = lo1;
        uint64_t y2 = hi0 ^ x3 ^ k1;
        uint64_t y3 = lo0;
        x0 = y0; x1 = y1; x2 = y2; x3 = y3;
    }
    out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

double orc_u01(uint64_t x)
{
    return (double)(x >> 11) * (1.0 / 9007199254740992.0); /* 2^-53 */
}

uint64_t orc_below(uint64_t x, uint64_t m)
{
    unsigned __int128 p = (unsigned __int128)x * (unsigned __int128)m;
    return (uint64_t)(p >> 64);
}

/* standard normal by the Box-Muller transform of two uniforms of one block */
double orc_ou_noise(uint64_t seed, uint64_t a, uint64_t b, uint64_t c)
{
    uint64_t ctr[4] = {6u, a, b, c}, key[2] = {seed, 0u}, o[4];
    orc_philox4x64(ctr, key, o);
    double u1 = 1.0 - orc_u01(o[0]); /* (0, 1] */
    double u2 = orc_u01(o[1]);
    return sqrt(-2.0 * log(u1)) * cos(6.283185307179586476925 * u2);
}
