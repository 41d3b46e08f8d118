// Learned score function (the paper's conclusion suggests learning the score;
// here a small CNN surrogate): downsampled (rho, u_x, u_y) fields of a flow
// state -> predicted future time-averaged drag.
//
// Network: conv3x3(8 -> 32) + ReLU, three conv3x3(32 -> 32) + ReLU, global
// mean pool, linear 32 -> 1.  Inputs and activations are BF16 in NHWC layout
// ([B][H][W][C], C = 8 for the input: 3 fields + 5 zero channels, 32 after),
// weights BF16 with FP32 master copies, every product accumulated in FP32 on
// the tensor cores (mma.sync m16n8k16 BF16).
//
// Every 3x3 'same' convolution is an implicit GEMM: M = pixels, N = 32 output
// channels, K = 9 * C_in input taps plus one constant-1 column that carries
// the bias (so the weight gradient produces the bias gradient too), padded to
// a multiple of 16.  Block = 8 x 16 output pixels of one sample, 4 warps of
// 2 x 16 pixels x 32 channels; the input tile with its 1-pixel halo and the
// weights are staged in shared memory (16-byte chunks XOR-swizzled by pixel
// to keep ldmatrix free of bank conflicts).
//   forward          conv(x, W) + ReLU
//   data gradient    conv(dY, W') masked by ReLU'(previous activation), with
//                    W'[ci][ky][kx][co] = W[co][2-ky][2-kx][ci]
//   weight gradient  dW[co][k] = sum over pixels dY[p][co] patch[p][k]: GEMM
//                    with the pixels as the reduction dimension, per-block
//                    partials summed in a fixed order.
#include <cmath>
#include <algorithm>
#include <cstring>
#include <vector>

#include "internal.h"
#include "lbm_device.cuh"

namespace lbm {

using bf16 = __nv_bfloat16;

constexpr int kTH = 8, kTW = 16;           // output tile
constexpr int kHH = kTH + 2, kHW = kTW + 2;  // halo tile
constexpr int kHPix = kHH * kHW;           // 180
constexpr int kC = 32;                     // channels of every hidden layer
constexpr int kCin0 = 8;                   // input channels (3 fields + 5 zeros)
constexpr int kLayers = 4;
constexpr int kWgradBlocks = 608;          // 4 per SM on 152 SMs
constexpr int kInputConvBlocks = 1216;     // 8 per SM on 152 SMs

__host__ __device__ constexpr int kpad_fwd(int cin) { return cin == 32 ? 304 : 80; }

// ---------------------------------------------------------------- PTX helpers
__device__ inline uint32_t smem_u32(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ inline void ldsm_x4(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ inline void ldsm_x4_t(uint32_t addr, uint32_t& r0, uint32_t& r1, uint32_t& r2, uint32_t& r3)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
                 : "=r"(r0), "=r"(r1), "=r"(r2), "=r"(r3)
                 : "r"(addr));
}
__device__ inline void ldsm_x2_t(uint32_t addr, uint32_t& r0, uint32_t& r1)
{
    asm volatile("ldmatrix.sync.aligned.m8n8.x2.trans.shared.b16 {%0,%1}, [%2];\n" : "=r"(r0), "=r"(r1) : "r"(addr));
}
__device__ inline void mma_bf16(float (&d)[4], const uint32_t (&a)[4], uint32_t b0, uint32_t b1)
{
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

constexpr uint32_t kBf16One = 0x3F80u;  // 1.0 in BF16

// shared-memory element offset of channel chunk `ch` (8 channels) of halo pixel
// `pix`; chunks are XOR-swizzled by the pixel index when a pixel holds 4 chunks
template <int CIN>
__device__ inline int halo_off(int pix, int ch)
{
    if constexpr (CIN == 32) return pix * 32 + ((ch ^ (pix & 3)) << 3);
    else return pix * CIN + (ch << 3);
}

// stage the (kTH+2) x (kTW+2) x CIN input tile of sample b with zero padding
template <int CIN>
__device__ inline void load_halo(bf16* s_in, const bf16* __restrict__ x, int b, int ty0, int tx0, int H, int W)
{
    constexpr int CH = CIN / 8;
    for (int i = threadIdx.x; i < kHPix * CH; i += blockDim.x) {
        const int pix = i / CH, ch = i - pix * CH;
        const int hr = pix / kHW, hc = pix - hr * kHW;
        const int gy = ty0 + hr - 1, gx = tx0 + hc - 1;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (gy >= 0 && gy < H && gx >= 0 && gx < W)
            v = *reinterpret_cast<const uint4*>(x + (((int64_t)b * H + gy) * W + gx) * CIN + ch * 8);
        *reinterpret_cast<uint4*>(s_in + halo_off<CIN>(pix, ch)) = v;
    }
}

// ---------------------------------------------------------------- convolution
// BWD = false: out = ReLU(conv(x, w)) with the bias column; BWD = true: out =
// conv(x, w) * (mask > 0), no bias column (x = dY of the next layer, w = W').
template <int CIN, bool BWD>
__global__ void __launch_bounds__(128) conv3x3_kernel(const bf16* __restrict__ x, const bf16* __restrict__ w,
                                                      const bf16* __restrict__ mask, bf16* __restrict__ out, int H,
                                                      int W)
{
    constexpr int KP = BWD ? 288 : kpad_fwd(CIN);
    constexpr int KS = KP + 8;  // padded row stride of the weight tile
    constexpr int NSTEP = KP / 16;
    __shared__ __align__(16) bf16 s_in[kHPix * CIN];
    __shared__ __align__(16) bf16 s_w[kC * KS];
    const int b = blockIdx.z, ty0 = blockIdx.y * kTH, tx0 = blockIdx.x * kTW;
    for (int i = threadIdx.x; i < kC * KP / 8; i += blockDim.x) {
        const int co = i / (KP / 8), kc = i - co * (KP / 8);
        *reinterpret_cast<uint4*>(s_w + co * KS + kc * 8) = *reinterpret_cast<const uint4*>(w + co * KP + kc * 8);
    }
    load_halo<CIN>(s_in, x, b, ty0, tx0, H, W);
    __syncthreads();

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int arow = (lane & 7) + ((lane >> 3) & 1) * 8;  // pixel of the m16 tile this lane addresses
    const int akh = lane >> 4;                            // k half (8 columns) it addresses
    const int bn = (lane >> 4) * 8 + (lane & 7);          // output channel row of the weight tile
    const int bkh = (lane >> 3) & 1;
    float acc[2][4][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < 4; ++n)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[m][n][r] = 0.f;

#pragma unroll 2
    for (int s = 0; s < NSTEP; ++s) {
        uint32_t a[2][4];
        const bool bias_step = !BWD && CIN == 32 && s == NSTEP - 1;
        if (bias_step) {
            const uint32_t one = t == 0 ? kBf16One : 0u;  // column 0 of this step is the bias input
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                a[m][0] = one;
                a[m][1] = one;
                a[m][2] = 0u;
                a[m][3] = 0u;
            }
        } else {
            int pos, ch;
            if (CIN == 32) {
                pos = s >> 1;
                ch = ((s & 1) << 1) + akh;
            } else {
                pos = 2 * s + akh;
                ch = 0;
                if (pos > 8) pos = 8;  // the bias half of the last step is set below
            }
            const int ky = pos / 3, kx = pos - ky * 3;
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int py = warp * 2 + m;
                const int hpix = (py + ky) * kHW + arow + kx;
                ldsm_x4(smem_u32(s_in + halo_off<CIN>(hpix, ch)), a[m][0], a[m][1], a[m][2], a[m][3]);
            }
            if (CIN == 8 && s == NSTEP - 1) {  // k 8..15 of the last step: bias column, zeros
                const uint32_t one = t == 0 ? kBf16One : 0u;
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    a[m][2] = one;
                    a[m][3] = one;
                }
            }
        }
        uint32_t bfr[4][2];
#pragma unroll
        for (int np = 0; np < 2; ++np) {
            const int co = np * 16 + bn, k = s * 16 + bkh * 8;
            ldsm_x4(smem_u32(s_w + co * KS + k), bfr[2 * np][0], bfr[2 * np][1], bfr[2 * np + 1][0],
                    bfr[2 * np + 1][1]);
        }
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int n = 0; n < 4; ++n) mma_bf16(acc[m][n], a[m], bfr[n][0], bfr[n][1]);
    }

#pragma unroll
    for (int m = 0; m < 2; ++m) {
        const int gy = ty0 + warp * 2 + m;
#pragma unroll
        for (int n = 0; n < 4; ++n) {
            const int co = n * 8 + 2 * t;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int gx = tx0 + g + 8 * h;
                const int64_t o = (((int64_t)b * H + gy) * W + gx) * kC + co;
                float v0 = acc[m][n][2 * h], v1 = acc[m][n][2 * h + 1];
                if (!BWD) {
                    v0 = fmaxf(v0, 0.f);
                    v1 = fmaxf(v1, 0.f);
                } else {
                    const __nv_bfloat162 mk = *reinterpret_cast<const __nv_bfloat162*>(mask + o);
                    if (!(__bfloat162float(mk.x) > 0.f)) v0 = 0.f;
                    if (!(__bfloat162float(mk.y) > 0.f)) v1 = 0.f;
                }
                *reinterpret_cast<__nv_bfloat162*>(out + o) = __floats2bfloat162_rn(v0, v1);
            }
        }
    }
}

// 16 bytes global -> shared through L2 (cp.async); src_bytes = 0 fills zeros
__device__ inline void cp_async16(void* dst, const void* src, uint32_t src_bytes)
{
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(smem_u32(dst)), "l"(src), "r"(src_bytes)
                 : "memory");
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// The input layer's forward pass: out = ReLU(conv3x3(x, w) + bias) from the
// 8-channel input (three fields and five zero channels).  It moves 16 B in and
// 64 B out per pixel for 2 x 80 x 32 FLOP, so HBM bounds it.  Persistent
// blocks stage the weights once, fetch the next tile's halo with cp.async while
// the current tile is computed, and stage each output tile in shared memory
// (80-byte pixel stride: the fragment writes are free of bank conflicts) so
// that it leaves as whole 512-byte runs of 16-byte stores.
constexpr int kOutStride = kC + 8;  // elements per pixel of the staged output tile

__global__ void __launch_bounds__(128, 8) input_conv_kernel(const bf16* __restrict__ x, const bf16* __restrict__ w,
                                                         bf16* __restrict__ out, int B, int H, int W)
{
    constexpr int CIN = kCin0, KP = kpad_fwd(kCin0), KS = KP + 8, NSTEP = KP / 16;
    __shared__ __align__(16) bf16 s_in[2][kHPix * CIN];
    __shared__ __align__(16) bf16 s_w[kC * KS];
    __shared__ __align__(16) bf16 s_out[kTH * kTW * kOutStride];
    const int tiles_x = W / kTW, tiles_y = H / kTH;
    const int total = B * tiles_x * tiles_y;
    for (int i = threadIdx.x; i < kC * KP / 8; i += blockDim.x) {
        const int co = i / (KP / 8), kc = i - co * (KP / 8);
        *reinterpret_cast<uint4*>(s_w + co * KS + kc * 8) = *reinterpret_cast<const uint4*>(w + co * KP + kc * 8);
    }
    auto origin = [&](int tile, int& b, int& ty0, int& tx0) {
        b = tile / (tiles_x * tiles_y);
        const int rem = tile - b * tiles_x * tiles_y;
        ty0 = (rem / tiles_x) * kTH;
        tx0 = (rem - (rem / tiles_x) * tiles_x) * kTW;
    };
    // the halo of a tile into buffer buf: one 16-byte pixel per copy, zeros outside the image
    auto fetch = [&](int tile, int buf) {
        int b, ty0, tx0;
        origin(tile, b, ty0, tx0);
        for (int pix = threadIdx.x; pix < kHPix; pix += blockDim.x) {
            const int hr = pix / kHW, hc = pix - hr * kHW;
            const int gy = ty0 + hr - 1, gx = tx0 + hc - 1;
            const bool in = gy >= 0 && gy < H && gx >= 0 && gx < W;
            const bf16* src = in ? x + (((int64_t)b * H + gy) * W + gx) * CIN : x;
            cp_async16(s_in[buf] + pix * CIN, src, in ? 16u : 0u);
        }
        cp_async_commit();
    };

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    const int arow = (lane & 7) + ((lane >> 3) & 1) * 8;
    const int akh = lane >> 4;
    const int bn = (lane >> 4) * 8 + (lane & 7);
    const int bkh = (lane >> 3) & 1;

    if ((int)blockIdx.x < total) fetch(blockIdx.x, 0);
    for (int tile = blockIdx.x, k = 0; tile < total; tile += gridDim.x, ++k) {
        const int buf = k & 1;
        if (tile + (int)gridDim.x < total) {
            fetch(tile + gridDim.x, buf ^ 1);
            cp_async_wait<1>();
        } else {
            cp_async_wait<0>();
        }
        __syncthreads();  // this tile's halo (and, the first time, the weights) is in place
        const bf16* si = s_in[buf];
        float acc[2][4][4];
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int n = 0; n < 4; ++n)
#pragma unroll
                for (int r = 0; r < 4; ++r) acc[m][n][r] = 0.f;
#pragma unroll
        for (int st = 0; st < NSTEP; ++st) {
            uint32_t a[2][4];
            int pos = 2 * st + akh;
            if (pos > 8) pos = 8;  // the bias half of the last step is set below
            const int ky = pos / 3, kx = pos - ky * 3;
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int hpix = (warp * 2 + m + ky) * kHW + arow + kx;
                ldsm_x4(smem_u32(si + hpix * CIN), a[m][0], a[m][1], a[m][2], a[m][3]);
            }
            if (st == NSTEP - 1) {  // k 8..15 of the last step: the bias column, then zeros
                const uint32_t one = t == 0 ? kBf16One : 0u;
#pragma unroll
                for (int m = 0; m < 2; ++m) {
                    a[m][2] = one;
                    a[m][3] = one;
                }
            }
            uint32_t bfr[4][2];
#pragma unroll
            for (int np = 0; np < 2; ++np) {
                const int co = np * 16 + bn, kk = st * 16 + bkh * 8;
                ldsm_x4(smem_u32(s_w + co * KS + kk), bfr[2 * np][0], bfr[2 * np][1], bfr[2 * np + 1][0],
                        bfr[2 * np + 1][1]);
            }
#pragma unroll
            for (int m = 0; m < 2; ++m)
#pragma unroll
                for (int n = 0; n < 4; ++n) mma_bf16(acc[m][n], a[m], bfr[n][0], bfr[n][1]);
        }
        // ReLU, BF16, into the staged tile: pixel (row warp*2 + m, column g + 8h)
#pragma unroll
        for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int n = 0; n < 4; ++n)
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    const int pix = (warp * 2 + m) * kTW + g + 8 * h;
                    *reinterpret_cast<__nv_bfloat162*>(s_out + pix * kOutStride + n * 8 + 2 * t) =
                        __floats2bfloat162_rn(fmaxf(acc[m][n][2 * h], 0.f), fmaxf(acc[m][n][2 * h + 1], 0.f));
                }
        __syncthreads();
        int b, ty0, tx0;
        origin(tile, b, ty0, tx0);
#pragma unroll
        for (int j = 0; j < kTH * kTW * 4 / 128; ++j) {
            const int i = threadIdx.x + j * 128, pix = i >> 2, c = i & 3;
            const int gy = ty0 + pix / kTW, gx = tx0 + (pix & (kTW - 1));
            *reinterpret_cast<uint4*>(out + (((int64_t)b * H + gy) * W + gx) * kC + c * 8) =
                *reinterpret_cast<const uint4*>(s_out + pix * kOutStride + c * 8);
        }
        __syncthreads();  // the staged tile and this halo buffer are free again
    }
}

// dW partials: block-persistent over output tiles; D[co][k] += dY^T patch
template <int CIN>
__global__ void __launch_bounds__(128) conv_wgrad_kernel(const bf16* __restrict__ x, const bf16* __restrict__ dy,
                                                         int B, int H, int W, float* __restrict__ partial)
{
    constexpr int KP = kpad_fwd(CIN);
    constexpr int NT = KP / 8;           // feature tiles of 8
    constexpr int NTW = (NT + 3) / 4;    // per warp
    constexpr int REAL_NT = 9 * CIN / 8; // tiles of real taps; the next one holds the bias column
    __shared__ __align__(16) bf16 s_in[kHPix * CIN];
    __shared__ __align__(16) bf16 s_dy[kTH * kTW * kC];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int g = lane >> 2, t = lane & 3;
    float acc[2][NTW][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int n = 0; n < NTW; ++n)
#pragma unroll
            for (int r = 0; r < 4; ++r) acc[m][n][r] = 0.f;
    const int tiles_x = W / kTW, tiles_y = H / kTH;
    const int total = B * tiles_x * tiles_y;
    for (int tile = blockIdx.x; tile < total; tile += gridDim.x) {
        const int b = tile / (tiles_x * tiles_y);
        const int rem = tile - b * tiles_x * tiles_y;
        const int ty0 = (rem / tiles_x) * kTH, tx0 = (rem % tiles_x) * kTW;
        __syncthreads();
        load_halo<CIN>(s_in, x, b, ty0, tx0, H, W);
        for (int i = threadIdx.x; i < kTH * kTW * 4; i += blockDim.x) {
            const int pix = i >> 2, ch = i & 3;
            const int gy = ty0 + pix / kTW, gx = tx0 + (pix % kTW);
            *reinterpret_cast<uint4*>(s_dy + halo_off<32>(pix, ch)) =
                *reinterpret_cast<const uint4*>(dy + (((int64_t)b * H + gy) * W + gx) * kC + ch * 8);
        }
        __syncthreads();
#pragma unroll 1
        for (int r = 0; r < kTH; ++r) {
            // A = dY^T (co x 16 pixels of tile row r) via transposed ldmatrix
            uint32_t a[2][4];
#pragma unroll
            for (int m = 0; m < 2; ++m) {
                const int j = lane >> 3;
                const int pix = r * kTW + (j >> 1) * 8 + (lane & 7);
                const int ch = m * 2 + (j & 1);
                ldsm_x4_t(smem_u32(s_dy + halo_off<32>(pix, ch)), a[m][0], a[m][1], a[m][2], a[m][3]);
            }
#pragma unroll
            for (int i = 0; i < NTW; ++i) {
                const int nt = warp * NTW + i;
                if (nt >= NT) break;
                uint32_t b0, b1;
                if (nt < REAL_NT) {
                    int pos, ch;
                    if (CIN == 32) {
                        pos = nt >> 2;
                        ch = nt & 3;
                    } else {
                        pos = nt;
                        ch = 0;
                    }
                    const int ky = pos / 3, kx = pos - ky * 3;
                    const int px = ((lane >> 3) & 1) * 8 + (lane & 7);  // lanes 0..15 address the two matrices
                    const int hpix = (r + ky) * kHW + px + kx;
                    ldsm_x2_t(smem_u32(s_in + halo_off<CIN>(hpix, ch)), b0, b1);
                } else {
                    // bias column (first feature of tile REAL_NT) is the constant 1
                    const uint32_t one = (nt == REAL_NT && g == 0) ? (kBf16One | (kBf16One << 16)) : 0u;
                    b0 = one;
                    b1 = one;
                }
#pragma unroll
                for (int m = 0; m < 2; ++m) mma_bf16(acc[m][i], a[m], b0, b1);
            }
        }
    }
    float* out = partial + (int64_t)blockIdx.x * kC * KP;
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int i = 0; i < NTW; ++i) {
            const int nt = warp * NTW + i;
            if (nt >= NT) break;
            const int k = nt * 8 + 2 * t;
            out[(m * 16 + g) * KP + k] = acc[m][i][0];
            out[(m * 16 + g) * KP + k + 1] = acc[m][i][1];
            out[(m * 16 + g + 8) * KP + k] = acc[m][i][2];
            out[(m * 16 + g + 8) * KP + k + 1] = acc[m][i][3];
        }
}

__global__ void reduce_partials_kernel(const float* partial, int nblk, int n, float* out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    float s = 0.f;
    for (int b = 0; b < nblk; ++b) s += partial[(int64_t)b * n + i];
    out[i] = s;
}

// global mean pool over the pixels of the last activation, then the linear head
__global__ void head_forward_kernel(const bf16* __restrict__ act, int P, const float* __restrict__ head,
                                   float* __restrict__ pooled, float* __restrict__ pred)
{
    __shared__ float sh[256][kC + 1];
    const int b = blockIdx.x;
    float s[kC];
#pragma unroll
    for (int c = 0; c < kC; ++c) s[c] = 0.f;
    for (int p = threadIdx.x; p < P; p += 256) {
        const uint4* src = reinterpret_cast<const uint4*>(act + ((int64_t)b * P + p) * kC);
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const uint4 u = src[q];
            const __nv_bfloat162* h2 = reinterpret_cast<const __nv_bfloat162*>(&u);
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const float2 f = __bfloat1622float2(h2[e]);
                s[q * 8 + 2 * e] += f.x;
                s[q * 8 + 2 * e + 1] += f.y;
            }
        }
    }
#pragma unroll
    for (int c = 0; c < kC; ++c) sh[threadIdx.x][c] = s[c];
    __syncthreads();
    for (int off = 128; off > 0; off >>= 1) {
        if ((int)threadIdx.x < off)
            for (int c = 0; c < kC; ++c) sh[threadIdx.x][c] += sh[threadIdx.x + off][c];
        __syncthreads();
    }
    if (threadIdx.x < kC) pooled[b * kC + threadIdx.x] = sh[0][threadIdx.x] / (float)P;
    __syncthreads();
    if (threadIdx.x == 0) {
        float v = head[kC];
        for (int c = 0; c < kC; ++c) v += head[c] * (sh[0][c] / (float)P);
        pred[b] = v;
    }
}

// MSE loss, head gradients and the per-(sample, channel) seed of dY4
__global__ void head_backward_kernel(int B, int P, const float* pooled, const float* pred, const float* y,
                                     const float* head, float* grad_head, float* seed, float* loss)
{
    __shared__ float dp[1024];
    const int tid = threadIdx.x;
    for (int b = tid; b < B; b += blockDim.x) dp[b] = 2.f * (pred[b] - y[b]) / (float)B;
    __syncthreads();
    if (tid < kC) {
        float gv = 0.f;
        for (int b = 0; b < B; ++b) gv += dp[b] * pooled[b * kC + tid];
        grad_head[tid] = gv;
    }
    if (tid == kC) {
        float gb = 0.f, l = 0.f;
        for (int b = 0; b < B; ++b) {
            gb += dp[b];
            const float e = pred[b] - y[b];
            l += e * e;
        }
        grad_head[kC] = gb;
        if (loss) *loss = l / (float)B;
    }
    for (int i = tid; i < B * kC; i += blockDim.x) seed[i] = dp[i / kC] * head[i % kC] / (float)P;
}

// dY4[b][p][c] = seed[b][c] * (act4 > 0): grid.y = image, one thread per
// 16-byte vector (8 channels of a pixel), no index division
__global__ void head_spread_kernel(const bf16* __restrict__ act, const float* __restrict__ seed, int P,
                                   bf16* __restrict__ dy)
{
    __shared__ float sd[kC];
    const int b = blockIdx.y;
    if (threadIdx.x < kC) sd[threadIdx.x] = seed[b * kC + threadIdx.x];
    __syncthreads();
    const uint4* a = reinterpret_cast<const uint4*>(act + (int64_t)b * P * kC);
    uint4* d = reinterpret_cast<uint4*>(dy + (int64_t)b * P * kC);
    const int64_t nv = (int64_t)P * (kC / 8);
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < nv; i += (int64_t)gridDim.x * blockDim.x) {
        const int c0 = (int)(i & (kC / 8 - 1)) * 8;  // channel of the vector's first element
        const uint4 v = a[i];
        const __nv_bfloat162* e = reinterpret_cast<const __nv_bfloat162*>(&v);
        uint4 o;
        __nv_bfloat162* oe = reinterpret_cast<__nv_bfloat162*>(&o);
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const float v0 = __bfloat162float(e[k].x) > 0.f ? sd[c0 + 2 * k] : 0.f;
            const float v1 = __bfloat162float(e[k].y) > 0.f ? sd[c0 + 2 * k + 1] : 0.f;
            oe[k] = __floats2bfloat162_rn(v0, v1);
        }
        d[i] = o;
    }
}

// Adam on the FP32 master parameters; conv weights re-exported to BF16
__global__ void adam_kernel(float* master, const float* grad, float* m, float* v, int64_t n, float lr, float b1,
                            float b2, float eps, float c1, float c2)
{
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        const float gi = grad[i];
        const float mi = b1 * m[i] + (1.f - b1) * gi;
        const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
        m[i] = mi;
        v[i] = vi;
        master[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
    }
}

// BF16 copies of the conv weights and the flipped, transposed W' of layers 1..3
__global__ void export_weights_kernel(const float* master, const int64_t* off, bf16* const* w, bf16* const* wt)
{
    const int l = blockIdx.y;
    const int cin = l == 0 ? kCin0 : kC;
    const int kp = kpad_fwd(cin);
    const float* src = master + off[l];
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kC * kp; i += gridDim.x * blockDim.x)
        w[l][i] = __float2bfloat16_rn(src[i]);
    if (l == 0) return;
    // W'[ci][pos' * 32 + co] = W[co][(8 - pos') * 32 + ci]
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < kC * 288; i += gridDim.x * blockDim.x) {
        const int ci = i / 288, k = i - ci * 288;
        const int posp = k / kC, co = k - posp * kC;
        wt[l][i] = __float2bfloat16_rn(src[co * kp + (8 - posp) * kC + ci]);
    }
}

// minibatch gather: rows idx[j] of the data set into the staging buffers
__global__ void gather_kernel(const bf16* __restrict__ x, const float* __restrict__ y, const int32_t* idx, int batch,
                              int64_t row_chunks, bf16* __restrict__ xb, float* __restrict__ yb)
{
    const int j = blockIdx.y;
    const int64_t src = (int64_t)idx[j] * row_chunks, dst = (int64_t)j * row_chunks;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < row_chunks; i += (int64_t)gridDim.x * blockDim.x)
        reinterpret_cast<uint4*>(xb)[dst + i] = reinterpret_cast<const uint4*>(x)[src + i];
    if (blockIdx.x == 0 && threadIdx.x == 0 && y) yb[j] = y[idx[j]];
}

// K8: block-mean of (rho, u_x, u_y) over factor x factor nodes of each listed
// clone -> [n][ny/factor][nx/factor][8] BF16 network input (floor division:
// rows and columns past the last whole block, e.g. the outlet column and top
// row of a 513 x 129 open channel at factor 4, are left out)
template <int S>
__global__ void fields_kernel(const void* buf0, const void* buf1, const int32_t* parity, const int32_t* list, int n,
                              int64_t clone_stride, int64_t plane, int32_t pitch, int32_t nx, int32_t ny, int factor,
                              float gx, float gy, float rho_scale, float u_scale, float inv_scale, bf16* out)
{
    using T = typename Codec<S>::T;
    const int Hc = ny / factor, Wc = nx / factor;
    const int64_t total = (int64_t)n * Hc * Wc;
    for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < total; i += (int64_t)gridDim.x * blockDim.x) {
        const int li = (int)(i / ((int64_t)Hc * Wc));
        const int rem = (int)(i - (int64_t)li * Hc * Wc);
        const int Y = rem / Wc, X = rem - Y * Wc;
        const int c = list[li];
        const T* base = static_cast<const T*>(parity[c] ? buf1 : buf0) + (int64_t)c * clone_stride;
        float sr = 0.f, sx = 0.f, sy = 0.f;
        for (int dy = 0; dy < factor; ++dy)
            for (int dx = 0; dx < factor; ++dx) {
                const int y = Y * factor + dy, x = X * factor + dx;
                float drho = 0.f, jx = 0.f, jy = 0.f;
#pragma unroll
                for (int q = 0; q < 9; ++q) {
                    const float gq = Codec<S>::dec(base[q * plane + (int64_t)y * pitch + x], wf(q), inv_scale);
                    drho += gq;
                    jx += cx(q) * gq;
                    jy += cy(q) * gq;
                }
                const float rho = 1.f + drho;
                sr += drho;
                sx += (jx - 0.5f * gx) / rho;  // velocity of a post-collision state
                sy += (jy - 0.5f * gy) / rho;
            }
        const float inv = 1.f / (float)(factor * factor);
        __align__(16) bf16 v[8];
        v[0] = __float2bfloat16_rn(sr * inv * rho_scale);
        v[1] = __float2bfloat16_rn(sx * inv * u_scale);
        v[2] = __float2bfloat16_rn(sy * inv * u_scale);
        for (int e = 3; e < 8; ++e) v[e] = __float2bfloat16_rn(0.f);
        *reinterpret_cast<uint4*>(out + i * 8) = *reinterpret_cast<const uint4*>(v);
    }
}

// network input of the clones listed on the device (no synchronisation)
int fields_launch(lbm_ensemble* e, const int32_t* list_dev, int32_t n, int32_t factor, float rho_scale, float u_scale,
                  void* dst_dev)
{
    if (factor < 1 || factor > e->cfg.nx || factor > e->cfg.ny)
        return fail(LBM_ERR_ARG, "fields: factor must be in [1, min(nx, ny)]");
    const int64_t total = (int64_t)n * (e->cfg.ny / factor) * (e->cfg.nx / factor);
    const int grid = (int)std::min<int64_t>((total + 255) / 256, 152 * 16);
    auto launch = [&](auto tag) {
        constexpr int S = decltype(tag)::value;
        fields_kernel<S><<<grid, 256, 0, e->stream>>>(e->buf[0], e->buf[1], e->parity_dev, list_dev, n,
                                                     e->clone_stride, e->plane, e->pitch, e->cfg.nx, e->cfg.ny, factor,
                                                     (float)e->cfg.gx, (float)e->cfg.gy, rho_scale, u_scale,
                                                     e->inv_scale, static_cast<bf16*>(dst_dev));
    };
    if (e->cfg.storage == kFP32) launch(std::integral_constant<int, kFP32>{});
    else if (e->cfg.storage == kFP16) launch(std::integral_constant<int, kFP16>{});
    else launch(std::integral_constant<int, kBF16>{});
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    return LBM_OK;
}

}  // namespace lbm

using namespace lbm;

struct cnn_model {
    int H, W, max_batch;
    int64_t off[kLayers + 1];  // parameter offsets; off[4] = head (v[32], bias)
    int64_t n_params;
    float* master;
    float* grad;
    float* adam_m;
    float* adam_v;
    int64_t* off_dev;
    bf16* w[kLayers];
    bf16* wt[kLayers];
    bf16** w_dev;   // device arrays of the pointers above
    bf16** wt_dev;
    bf16* act[kLayers];
    bf16* dy[2];
    float* pooled;
    float* pred;
    float* seed;
    float* wpart;
    bf16* xb;       // minibatch staging [max_batch][H][W][8]
    float* yb;      // [max_batch]
    float* lossb;   // [1]
    int32_t* idx;   // [max_batch] sample indices of the minibatch
    int64_t adam_t;
    int32_t conv_path;  // 0: tensor-core (tcgen05) hidden layers where the shape allows; 1: mma.sync everywhere
    int32_t* err;       // device flag: a bounded device-side wait ran out
};

namespace {

int cnn_check(const cnn_model* m, int batch)
{
    if (!m) return fail(LBM_ERR_ARG, "null model");
    if (batch < 1 || batch > m->max_batch) return fail(LBM_ERR_ARG, "batch outside [1, max_batch]");
    return LBM_OK;
}

int export_weights(cnn_model* m, cudaStream_t s)
{
    export_weights_kernel<<<dim3(16, kLayers), 256, 0, s>>>(m->master, m->off_dev, m->w_dev, m->wt_dev);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    return LBM_OK;
}

bool use_tc(const cnn_model* m, int batch)
{
    return m->conv_path == 0 && conv3x3_tc_supported(batch, m->H, m->W);
}

// one hidden 32 -> 32 layer: forward (ReLU(conv + bias)) or data gradient
// (conv with W' masked by the layer below)
int conv32(cnn_model* m, const bf16* x, const bf16* w, const bf16* mask, bf16* out, int batch, bool bwd,
           cudaStream_t s)
{
    if (use_tc(m, batch)) return conv3x3_tc(x, w, mask, out, batch, m->H, m->W, bwd, m->err, s);
    const dim3 grid(m->W / kTW, m->H / kTH, batch);
    if (bwd)
        conv3x3_kernel<kC, true><<<grid, 128, 0, s>>>(x, w, mask, out, m->H, m->W);
    else
        conv3x3_kernel<kC, false><<<grid, 128, 0, s>>>(x, w, nullptr, out, m->H, m->W);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    return LBM_OK;
}

int forward(cnn_model* m, const bf16* x, int batch, cudaStream_t s)
{
    const int tiles = batch * (m->H / kTH) * (m->W / kTW);
    const int blocks = tiles < kInputConvBlocks ? tiles : kInputConvBlocks;
    input_conv_kernel<<<blocks, 128, 0, s>>>(x, m->w[0], m->act[0], batch, m->H, m->W);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    for (int l = 1; l < kLayers; ++l)
        if (int rc = conv32(m, m->act[l - 1], m->w[l], nullptr, m->act[l], batch, false, s)) return rc;
    head_forward_kernel<<<batch, 256, 0, s>>>(m->act[kLayers - 1], m->H * m->W, m->master + m->off[kLayers],
                                             m->pooled, m->pred);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    return LBM_OK;
}

int wgrad(cnn_model* m, int l, const bf16* x, const bf16* dy, int batch, cudaStream_t s)
{
    const int cin = l == 0 ? kCin0 : kC;
    const int kp = kpad_fwd(cin);
    int nblk = 0;
    if (cin == kC && m->conv_path == 0 && conv3x3_wgrad_tc_supported(batch, m->H, m->W)) {
        // hidden layers on the tensor cores (tcgen05): partial sums per CTA
        if (int rc = conv3x3_wgrad_tc(x, dy, m->wpart, batch, m->H, m->W, m->err, s, &nblk)) return rc;
    } else {
        const int tiles = batch * (m->H / kTH) * (m->W / kTW);
        // the input layer's partials (32 x 80) are a quarter of a hidden layer's
        // (32 x 304), so twice the blocks fit the same buffer: 8 resident per SM,
        // twice the loads in flight for a kernel bound by their latency
        const int cap = cin == kC ? kWgradBlocks : 2 * kWgradBlocks;
        nblk = tiles < cap ? tiles : cap;
        if (cin == kC)
            conv_wgrad_kernel<kC><<<nblk, 128, 0, s>>>(x, dy, batch, m->H, m->W, m->wpart);
        else
            conv_wgrad_kernel<kCin0><<<nblk, 128, 0, s>>>(x, dy, batch, m->H, m->W, m->wpart);
        count_launches(1);
    }
    const int n = kC * kp;
    reduce_partials_kernel<<<(n + 255) / 256, 256, 0, s>>>(m->wpart, nblk, n, m->grad + m->off[l]);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    return LBM_OK;
}

int gradient(cnn_model* m, const bf16* x, const float* y, int batch, float* loss, cudaStream_t s)
{
    int rc;
    if ((rc = forward(m, x, batch, s))) return rc;
    const int P = m->H * m->W;
    head_backward_kernel<<<1, 256, 0, s>>>(batch, P, m->pooled, m->pred, y, m->master + m->off[kLayers],
                                          m->grad + m->off[kLayers], m->seed, loss);
    {
        const int64_t nv = (int64_t)P * (kC / 8);
        const int gx = (int)std::min<int64_t>((nv + 255) / 256, 64);
        head_spread_kernel<<<dim3(gx, batch), 256, 0, s>>>(m->act[kLayers - 1], m->seed, P, m->dy[0]);
    }
    LBM_CUDA(cudaGetLastError());
    count_launches(2);
    int cur = 0;
    for (int l = kLayers - 1; l >= 0; --l) {
        const bf16* in = l == 0 ? x : m->act[l - 1];
        if ((rc = wgrad(m, l, in, m->dy[cur], batch, s))) return rc;
        if (l > 0) {
            if ((rc = conv32(m, m->dy[cur], m->wt[l], m->act[l - 1], m->dy[cur ^ 1], batch, true, s))) return rc;
            cur ^= 1;
        }
    }
    return LBM_OK;
}

}  // namespace

extern "C" {

int cnn_create(int32_t height, int32_t width, int32_t max_batch, uint64_t seed, cnn_model** out)
{
    if (!out) return fail(LBM_ERR_ARG, "cnn_create: null output");
    *out = nullptr;
    if (height < kTH || height % kTH || width < kTW || width % kTW)
        return fail(LBM_ERR_ARG, "cnn_create: height must be a multiple of 8 and width of 16");
    if (max_batch < 1 || max_batch > 1024) return fail(LBM_ERR_ARG, "cnn_create: max_batch in [1, 1024]");
    auto* m = new cnn_model();
    std::memset(m, 0, sizeof(*m));
    m->H = height;
    m->W = width;
    m->max_batch = max_batch;
    int64_t o = 0;
    for (int l = 0; l < kLayers; ++l) {
        m->off[l] = o;
        o += (int64_t)kC * kpad_fwd(l == 0 ? kCin0 : kC);
    }
    m->off[kLayers] = o;
    o += kC + 1;
    m->n_params = o;
    // deterministic initialisation (He-uniform conv weights, zero biases,
    // uniform head) from Philox4x64-10 stream 7
    std::vector<float> host(o, 0.f);
    for (int l = 0; l < kLayers; ++l) {
        const int cin = l == 0 ? 3 : kC, cin_s = l == 0 ? kCin0 : kC, kp = kpad_fwd(cin_s);
        const double a = std::sqrt(6.0 / (9.0 * cin));
        for (int co = 0; co < kC; ++co)
            for (int pos = 0; pos < 9; ++pos)
                for (int ci = 0; ci < cin; ++ci) {
                    const u64x4 r = philox(7u, (uint64_t)l, (uint64_t)(co * 9 + pos), (uint64_t)ci, seed, 0u);
                    host[m->off[l] + co * kp + pos * cin_s + ci] = (float)(a * (2.0 * unit_double(r.v[0]) - 1.0));
                }
    }
    for (int c = 0; c < kC; ++c) {
        const u64x4 r = philox(7u, 9u, (uint64_t)c, 0u, seed, 0u);
        host[m->off[kLayers] + c] = (float)((2.0 * unit_double(r.v[0]) - 1.0) / std::sqrt((double)kC));
    }
    const int64_t P = (int64_t)height * width;
    auto cleanup = [&](int code) {
        cnn_destroy(m);
        return code;
    };
    cudaError_t err;
#define ALLOC(ptr, bytes)                                                          \
    err = cudaMalloc((void**)&(ptr), (bytes));                                     \
    if (err != cudaSuccess) return cleanup(cuda_fail(err, "cudaMalloc " #ptr));
    ALLOC(m->master, sizeof(float) * o);
    ALLOC(m->grad, sizeof(float) * o);
    ALLOC(m->adam_m, sizeof(float) * o);
    ALLOC(m->adam_v, sizeof(float) * o);
    ALLOC(m->off_dev, sizeof(int64_t) * (kLayers + 1));
    ALLOC(m->w_dev, sizeof(bf16*) * kLayers);
    ALLOC(m->wt_dev, sizeof(bf16*) * kLayers);
    for (int l = 0; l < kLayers; ++l) {
        ALLOC(m->w[l], sizeof(bf16) * kC * kpad_fwd(l == 0 ? kCin0 : kC));
        ALLOC(m->wt[l], sizeof(bf16) * kC * 288);
        ALLOC(m->act[l], sizeof(bf16) * max_batch * P * kC);
    }
    ALLOC(m->dy[0], sizeof(bf16) * max_batch * P * kC);
    ALLOC(m->dy[1], sizeof(bf16) * max_batch * P * kC);
    ALLOC(m->pooled, sizeof(float) * max_batch * kC);
    ALLOC(m->pred, sizeof(float) * max_batch);
    ALLOC(m->seed, sizeof(float) * max_batch * kC);
    ALLOC(m->wpart, sizeof(float) * kWgradBlocks * kC * 304);
    ALLOC(m->xb, sizeof(bf16) * max_batch * P * kCin0);
    ALLOC(m->yb, sizeof(float) * max_batch);
    ALLOC(m->lossb, sizeof(float));
    ALLOC(m->idx, sizeof(int32_t) * max_batch);
    ALLOC(m->err, sizeof(int32_t));
#undef ALLOC
    if ((err = cudaMemcpy(m->master, host.data(), sizeof(float) * o, cudaMemcpyHostToDevice)) != cudaSuccess)
        return cleanup(cuda_fail(err, "cnn_create upload"));
    cudaMemset(m->err, 0, sizeof(int32_t));
    cudaMemset(m->grad, 0, sizeof(float) * o);
    cudaMemset(m->adam_m, 0, sizeof(float) * o);
    cudaMemset(m->adam_v, 0, sizeof(float) * o);
    cudaMemcpy(m->off_dev, m->off, sizeof(int64_t) * (kLayers + 1), cudaMemcpyHostToDevice);
    cudaMemcpy(m->w_dev, m->w, sizeof(bf16*) * kLayers, cudaMemcpyHostToDevice);
    cudaMemcpy(m->wt_dev, m->wt, sizeof(bf16*) * kLayers, cudaMemcpyHostToDevice);
    int rc = export_weights(m, nullptr);
    if (rc) return cleanup(rc);
    if ((err = cudaDeviceSynchronize()) != cudaSuccess) return cleanup(cuda_fail(err, "cnn_create"));
    *out = m;
    return LBM_OK;
}

int cnn_destroy(cnn_model* m)
{
    if (!m) return LBM_OK;
    cudaDeviceSynchronize();
    void* ptrs[] = {m->master, m->grad, m->adam_m, m->adam_v, m->off_dev, m->w_dev, m->wt_dev, m->dy[0], m->dy[1],
                    m->pooled, m->pred, m->seed, m->wpart, m->xb, m->yb, m->lossb, m->idx, m->err};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int l = 0; l < kLayers; ++l) {
        if (m->w[l]) cudaFree(m->w[l]);
        if (m->wt[l]) cudaFree(m->wt[l]);
        if (m->act[l]) cudaFree(m->act[l]);
    }
    delete m;
    return LBM_OK;
}

int64_t cnn_param_count(const cnn_model* m) { return m ? m->n_params : -1; }

int cnn_get_params(cnn_model* m, float* host)
{
    if (!m || !host) return fail(LBM_ERR_ARG, "cnn_get_params: null argument");
    LBM_CUDA(cudaDeviceSynchronize());
    LBM_CUDA(cudaMemcpy(host, m->master, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

int cnn_set_params(cnn_model* m, const float* host)
{
    if (!m || !host) return fail(LBM_ERR_ARG, "cnn_set_params: null argument");
    for (int64_t i = 0; i < m->n_params; ++i)
        if (!std::isfinite(host[i])) return fail(LBM_ERR_NONFINITE, "cnn_set_params: parameter not finite");
    LBM_CUDA(cudaDeviceSynchronize());
    LBM_CUDA(cudaMemcpy(m->master, host, sizeof(float) * m->n_params, cudaMemcpyHostToDevice));
    int rc = export_weights(m, nullptr);
    if (rc) return rc;
    LBM_CUDA(cudaDeviceSynchronize());
    return LBM_OK;
}

int cnn_get_gradient(cnn_model* m, float* host)
{
    if (!m || !host) return fail(LBM_ERR_ARG, "cnn_get_gradient: null argument");
    LBM_CUDA(cudaDeviceSynchronize());
    LBM_CUDA(cudaMemcpy(host, m->grad, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
    return LBM_OK;
}

int cnn_forward(cnn_model* m, const void* x_dev, int32_t batch, float* pred_dev, void* stream)
{
    int rc = cnn_check(m, batch);
    if (rc) return rc;
    if (!x_dev || !pred_dev) return fail(LBM_ERR_ARG, "cnn_forward: null pointer");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if ((rc = forward(m, static_cast<const bf16*>(x_dev), batch, s))) return rc;
    LBM_CUDA(cudaMemcpyAsync(pred_dev, m->pred, sizeof(float) * batch, cudaMemcpyDeviceToDevice, s));
    return LBM_OK;
}

int cnn_gradient(cnn_model* m, const void* x_dev, const float* y_dev, int32_t batch, float* loss_dev, void* stream)
{
    int rc = cnn_check(m, batch);
    if (rc) return rc;
    if (!x_dev || !y_dev) return fail(LBM_ERR_ARG, "cnn_gradient: null pointer");
    return gradient(m, static_cast<const bf16*>(x_dev), y_dev, batch, loss_dev, static_cast<cudaStream_t>(stream));
}

int cnn_adam_step(cnn_model* m, float lr, float beta1, float beta2, float eps, void* stream)
{
    if (!m) return fail(LBM_ERR_ARG, "cnn_adam_step: null model");
    if (!(lr > 0.f) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) || !(eps > 0.f))
        return fail(LBM_ERR_ARG, "cnn_adam_step: hyper-parameters");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    m->adam_t += 1;
    const float c1 = 1.f - std::pow(beta1, (float)m->adam_t), c2 = 1.f - std::pow(beta2, (float)m->adam_t);
    adam_kernel<<<64, 256, 0, s>>>(m->master, m->grad, m->adam_m, m->adam_v, m->n_params, lr, beta1, beta2, eps, c1, c2);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    return export_weights(m, s);
}

int cnn_train_step(cnn_model* m, const void* x_dev, const float* y_dev, int32_t batch, float lr, float* loss_dev,
                   void* stream)
{
    int rc = cnn_gradient(m, x_dev, y_dev, batch, loss_dev, stream);
    if (rc) return rc;
    return cnn_adam_step(m, lr, 0.9f, 0.999f, 1e-8f, stream);
}

int cnn_set_conv_path(cnn_model* m, int32_t path)
{
    if (!m) return fail(LBM_ERR_ARG, "cnn_set_conv_path: null model");
    if (path != 0 && path != 1) return fail(LBM_ERR_ARG, "cnn_set_conv_path: path must be 0 or 1");
    m->conv_path = path;
    return LBM_OK;
}

int cnn_tensor_core_paths(const cnn_model* m, int32_t batch, int32_t* conv_tc, int32_t* wgrad_tc)
{
    if (int rc = cnn_check(m, batch)) return rc;
    if (!conv_tc || !wgrad_tc) return fail(LBM_ERR_ARG, "cnn_tensor_core_paths: null output");
    *conv_tc = use_tc(m, batch) ? 1 : 0;
    *wgrad_tc = (m->conv_path == 0 && conv3x3_wgrad_tc_supported(batch, m->H, m->W)) ? 1 : 0;
    return LBM_OK;
}

int cnn_status(cnn_model* m, void* stream)
{
    if (!m) return fail(LBM_ERR_ARG, "cnn_status: null model");
    int32_t err = 0;
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    LBM_CUDA(cudaMemcpyAsync(&err, m->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
    LBM_CUDA(cudaStreamSynchronize(s));
    if (err) return fail(LBM_ERR_TIMEOUT, "cnn: a bounded device-side wait of the convolution ran out");
    return LBM_OK;
}

int cnn_shape(const cnn_model* m, int32_t* height, int32_t* width, int32_t* max_batch)
{
    if (!m) return fail(LBM_ERR_ARG, "cnn_shape: null model");
    if (height) *height = m->H;
    if (width) *width = m->W;
    if (max_batch) *max_batch = m->max_batch;
    return LBM_OK;
}

int cnn_predict(cnn_model* m, const void* x_dev, int64_t n, float* pred_dev, void* stream)
{
    if (!m || !x_dev || !pred_dev || n < 1) return fail(LBM_ERR_ARG, "cnn_predict: arguments");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t per = (int64_t)m->H * m->W * kCin0;
    for (int64_t b0 = 0; b0 < n; b0 += m->max_batch) {
        const int batch = (int)std::min<int64_t>(m->max_batch, n - b0);
        int rc = forward(m, static_cast<const bf16*>(x_dev) + b0 * per, batch, s);
        if (rc) return rc;
        LBM_CUDA(cudaMemcpyAsync(pred_dev + b0, m->pred, sizeof(float) * batch, cudaMemcpyDeviceToDevice, s));
    }
    return LBM_OK;
}

int cnn_fit(cnn_model* m, const void* x_dev, const float* y_dev, int64_t n, int32_t batch, int32_t epochs, float lr,
            uint64_t seed, float* epoch_loss, void* stream)
{
    if (!m || !x_dev || !y_dev) return fail(LBM_ERR_ARG, "cnn_fit: null argument");
    if (n < 1 || n > INT32_MAX || batch < 1 || batch > m->max_batch || epochs < 0)
        return fail(LBM_ERR_ARG, "cnn_fit: sizes");
    if (!(lr > 0.f)) return fail(LBM_ERR_ARG, "cnn_fit: lr");
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const int64_t row_chunks = (int64_t)m->H * m->W * kCin0 / 8;
    std::vector<int32_t> perm(n);
    for (int32_t ep = 0; ep < epochs; ++ep) {
        // Fisher-Yates shuffle driven by Philox4x64-10 stream 8
        for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
        for (int64_t i = n - 1; i > 0; --i) {
            const u64x4 r = philox(8u, (uint64_t)ep, (uint64_t)i, 0u, seed, 0u);
            const int64_t j = (int64_t)index_below(r.v[0], (uint64_t)(i + 1));
            std::swap(perm[i], perm[j]);
        }
        double total = 0.0;
        int64_t nb = 0;
        for (int64_t b0 = 0; b0 + batch <= n; b0 += batch) {
            LBM_CUDA(cudaMemcpyAsync(m->idx, perm.data() + b0, sizeof(int32_t) * batch, cudaMemcpyHostToDevice, s));
            gather_kernel<<<dim3(64, batch), 256, 0, s>>>(static_cast<const bf16*>(x_dev), y_dev, m->idx, batch,
                                                          row_chunks, m->xb, m->yb);
            LBM_CUDA(cudaGetLastError());
            count_launches(1);
            int rc = gradient(m, m->xb, m->yb, batch, m->lossb, s);
            if (rc) return rc;
            rc = cnn_adam_step(m, lr, 0.9f, 0.999f, 1e-8f, s);
            if (rc) return rc;
            float l = 0.f;
            int32_t err = 0;
            LBM_CUDA(cudaMemcpyAsync(&l, m->lossb, sizeof(float), cudaMemcpyDeviceToHost, s));
            LBM_CUDA(cudaMemcpyAsync(&err, m->err, sizeof(int32_t), cudaMemcpyDeviceToHost, s));
            LBM_CUDA(cudaStreamSynchronize(s));  // also keeps perm alive for the index copy
            if (err) return fail(LBM_ERR_TIMEOUT, "cnn_fit: a bounded device-side wait of the convolution ran out");
            if (!std::isfinite(l)) return fail(LBM_ERR_NONFINITE, "cnn_fit: loss not finite");
            total += l;
            ++nb;
        }
        if (epoch_loss) epoch_loss[ep] = nb ? (float)(total / nb) : 0.f;
    }
    return LBM_OK;
}

int lbm_ensemble_fields(lbm_ensemble* e, const int32_t* clones, int32_t n, int32_t factor, float rho_scale,
                        float u_scale, void* dst_dev)
{
    if (!e || !clones || !dst_dev) return fail(LBM_ERR_ARG, "lbm_ensemble_fields: null argument");
    if (n < 1 || n > e->n) return fail(LBM_ERR_ARG, "lbm_ensemble_fields: clone count");
    for (int i = 0; i < n; ++i)
        if (clones[i] < 0 || clones[i] >= e->n) return fail(LBM_ERR_ARG, "lbm_ensemble_fields: clone index");
    LBM_CUDA(cudaMemcpyAsync(e->fields_list_dev, clones, sizeof(int32_t) * n, cudaMemcpyHostToDevice, e->stream));
    int rc = lbm::fields_launch(e, e->fields_list_dev, n, factor, rho_scale, u_scale, dst_dev);
    if (rc) return rc;
    LBM_CUDA(cudaStreamSynchronize(e->stream));  // the host index list must outlive its copy
    return LBM_OK;
}

}  // extern "C"
