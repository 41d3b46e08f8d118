// Device-side building blocks of the ensemble lattice-Boltzmann library:
// the D2Q9 lattice, the counter-based random-number generator and the
// population storage codecs.  sm_103a only.
#pragma once
#include <cstdint>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

namespace lbm {

// ---------------------------------------------------------------- lattice
// D2Q9 velocities (App. A): rest, the four axis links, the four diagonal
// links; weights 4/9, 1/9, 1/36; c_s^2 = 1/3.
__host__ __device__ constexpr int cx(int q) { return q == 1 || q == 5 || q == 8 ? 1 : (q == 3 || q == 6 || q == 7 ? -1 : 0); }
__host__ __device__ constexpr int cy(int q) { return q == 2 || q == 5 || q == 6 ? 1 : (q == 4 || q == 7 || q == 8 ? -1 : 0); }
__host__ __device__ constexpr int opp(int q) { return q == 0 ? 0 : (q <= 4 ? ((q + 1) & 3) + 1 : ((q - 3) & 3) + 5); }
__host__ __device__ constexpr float wf(int q) { return q == 0 ? 4.0f / 9.0f : (q <= 4 ? 1.0f / 9.0f : 1.0f / 36.0f); }
__host__ __device__ constexpr double wd(int q) { return q == 0 ? 4.0 / 9.0 : (q <= 4 ? 1.0 / 9.0 : 1.0 / 36.0); }

static_assert(opp(1) == 3 && opp(2) == 4 && opp(3) == 1 && opp(4) == 2, "axis opposites");
static_assert(opp(5) == 7 && opp(6) == 8 && opp(7) == 5 && opp(8) == 6, "diagonal opposites");
static_assert(cx(opp(5)) == -cx(5) && cy(opp(6)) == -cy(6), "opposite velocity");

// Solid cells (Sec. 2): the square [ox0, ox1) x [oy0, oy1) whose drag is
// measured (ox1 == ox0 for none) and, in an open channel, the entrance grid of
// bars: cells x in [gx0, gx1) with y mod period >= gap (gx1 == gx0 for none;
// bars of period - gap rows separated by gap fluid rows, a gap at the bottom).
struct Solids {
    int32_t ox0, ox1, oy0, oy1;
    int32_t gx0, gx1, gap, period;
    __host__ __device__ bool square(int x, int y) const { return x >= ox0 && x < ox1 && y >= oy0 && y < oy1; }
    __host__ __device__ bool grid(int x, int y) const { return x >= gx0 && x < gx1 && y % period >= gap; }
    __host__ __device__ bool at(int x, int y) const { return square(x, y) || grid(x, y); }
};

// ---------------------------------------------------------------- random numbers
// Philox4x64-10 of Salmon, Moraes, Dror & Shaw (SC'11): ten rounds of two
// 64x64 -> 128-bit products whose halves are mixed with the other counter
// words and the key; the key advances by two Weyl increments between rounds.
struct u64x4 { uint64_t v[4]; };

__host__ __device__ inline void mul_hi_lo(uint64_t a, uint64_t b, uint64_t& hi, uint64_t& lo)
{
#ifdef __CUDA_ARCH__
    hi = __umul64hi(a, b);
    lo = a * b;
#else
    unsigned __int128 p = (unsigned __int128)a * b;
    hi = (uint64_t)(p >> 64);
    lo = (uint64_t)p;
#endif
}

__host__ __device__ inline u64x4 philox(uint64_t c0, uint64_t c1, uint64_t c2, uint64_t c3, uint64_t k0, uint64_t k1)
{
    constexpr uint64_t kMulA = 0xD2E7470EE14C6C93ULL, kMulB = 0xCA5A826395121157ULL;
    constexpr uint64_t kWeylA = 0x9E3779B97F4A7C15ULL, kWeylB = 0xBB67AE8584CAA73BULL;
    for (int r = 0; r < 10; ++r) {
        uint64_t hA, lA, hB, lB;
        mul_hi_lo(kMulA, c0, hA, lA);
        mul_hi_lo(kMulB, c2, hB, lB);
        const uint64_t n0 = hB ^ c1 ^ k0, n2 = hA ^ c3 ^ k1;
        c0 = n0; c1 = lB; c2 = n2; c3 = lA;
        k0 += kWeylA;
        k1 += kWeylB;
    }
    return u64x4{{c0, c1, c2, c3}};
}

// Stream identifiers (counter word 0) shared with the published definition
// of each random draw of the method.
enum : uint64_t { kStreamGktl = 1, kStreamAms = 3, kStreamPerturb = 4, kStreamInit = 5 };

__host__ __device__ inline double unit_double(uint64_t x) { return (double)(x >> 11) * 0x1.0p-53; }

__host__ __device__ inline uint64_t index_below(uint64_t x, uint64_t m)
{
    uint64_t hi, lo;
    mul_hi_lo(x, m, hi, lo);
    return hi;
}

// ---------------------------------------------------------------- storage
// Populations are stored per direction plane either as FP32 values f, or as
// 16-bit shifted values h = (f - w_q) * 2^s (FP16 or BF16, round to nearest
// even); arithmetic is always FP32 on the shifted value g = f - w_q.
enum Storage : int { kFP32 = 0, kFP16 = 1, kBF16 = 2 };

template <int S> struct Codec;

// dec2/enc2 move two neighbouring elements with one packed conversion.
template <> struct Codec<kFP32> {
    using T = float;
    __device__ static float dec(T v, float w, float) { return v - w; }
    __device__ static T enc(float g, float w, float) { return g + w; }
    __device__ static float2 dec2(const T* v, float w, float) { return make_float2(v[0] - w, v[1] - w); }
    __device__ static void enc2(T* out, float a, float b, float w, float)
    {
        out[0] = a + w;
        out[1] = b + w;
    }
};
template <> struct Codec<kFP16> {
    using T = __half;
    __device__ static float dec(T v, float, float inv_scale) { return __half2float(v) * inv_scale; }
    __device__ static T enc(float g, float, float scale) { return __float2half_rn(g * scale); }
    __device__ static float2 dec2(const T* v, float, float inv_scale)
    {
        const float2 f = __half22float2(*reinterpret_cast<const __half2*>(v));
        return make_float2(f.x * inv_scale, f.y * inv_scale);
    }
    __device__ static void enc2(T* out, float a, float b, float, float scale)
    {
        *reinterpret_cast<__half2*>(out) = __floats2half2_rn(a * scale, b * scale);
    }
};
template <> struct Codec<kBF16> {
    using T = __nv_bfloat16;
    __device__ static float dec(T v, float, float inv_scale) { return __bfloat162float(v) * inv_scale; }
    __device__ static T enc(float g, float, float scale) { return __float2bfloat16_rn(g * scale); }
    __device__ static float2 dec2(const T* v, float, float inv_scale)
    {
        const float2 f = __bfloat1622float2(*reinterpret_cast<const __nv_bfloat162*>(v));
        return make_float2(f.x * inv_scale, f.y * inv_scale);
    }
    __device__ static void enc2(T* out, float a, float b, float, float scale)
    {
        *reinterpret_cast<__nv_bfloat162*>(out) = __floats2bfloat162_rn(a * scale, b * scale);
    }
};

// V consecutive stored elements moved as one aligned vector access.
template <typename T, int V> struct alignas(sizeof(T) * V) Vec { T e[V]; };

// Streaming-store / evict-first hints for the population planes: each element
// is read once and written once per step, so neither side benefits from L2.
template <typename T, int V>
__device__ inline Vec<T, V> ld_stream(const T* p)
{
    Vec<T, V> r;
    if constexpr (sizeof(T) * V == 16) {
        uint4 u = __ldcs(reinterpret_cast<const uint4*>(p));
        r = *reinterpret_cast<Vec<T, V>*>(&u);
    } else if constexpr (sizeof(T) * V == 8) {
        uint2 u = __ldcs(reinterpret_cast<const uint2*>(p));
        r = *reinterpret_cast<Vec<T, V>*>(&u);
    } else if constexpr (sizeof(T) * V == 4) {
        unsigned u = __ldcs(reinterpret_cast<const unsigned*>(p));
        r = *reinterpret_cast<Vec<T, V>*>(&u);
    } else {
        static_assert(sizeof(T) * V == 2, "vector width");
        unsigned short u = __ldcs(reinterpret_cast<const unsigned short*>(p));
        r = *reinterpret_cast<Vec<T, V>*>(&u);
    }
    return r;
}

template <typename T, int V>
__device__ inline void st_stream(T* p, const Vec<T, V>& v)
{
    if constexpr (sizeof(T) * V == 16) {
        __stcs(reinterpret_cast<uint4*>(p), *reinterpret_cast<const uint4*>(&v));
    } else if constexpr (sizeof(T) * V == 8) {
        __stcs(reinterpret_cast<uint2*>(p), *reinterpret_cast<const uint2*>(&v));
    } else if constexpr (sizeof(T) * V == 4) {
        __stcs(reinterpret_cast<unsigned*>(p), *reinterpret_cast<const unsigned*>(&v));
    } else {
        __stcs(reinterpret_cast<unsigned short*>(p), *reinterpret_cast<const unsigned short*>(&v));
    }
}

template <typename T>
__device__ inline T ld_one(const T* p) { return *p; }

}  // namespace lbm
