// 3x3 'same' convolution with 32 input and 32 output channels on the fifth-
// generation tensor cores (tcgen05), for the hidden layers of the learned-score
// CNN: the forward pass (bias + ReLU) and the data gradient (masked by the
// ReLU derivative of the layer below).  Implicit GEMM: M = output pixels,
// K = 9 taps x 32 input channels, FP32 accumulators in tensor memory, operands
// staged in shared memory by TMA, one thread issuing the MMAs, a persistent
// CTA per SM with warp roles (TMA producer, MMA issuer, epilogue warps that
// read the accumulators with tcgen05.ld and store BF16 NHWC rows).
//
// Two kernels:
//   conv_row_kernel  widths that are a multiple of 128 (the 64 x 256 input of
//                    the 1024 x 256 channel): the three ky taps stacked along
//                    N = 96, six MMAs per 128-pixel input row;
//   conv_tc_kernel   narrower inputs (width a divisor of 128): 128-pixel
//                    blocks of 128 / W rows, N = 32, one MMA per tap and K-step.
// Measured on this GPU, a chain of MMAs into one accumulator costs about 80
// cycles per MMA for M = 128 and any N up to 128 (about 150 at N = 256), and
// MMAs into an accumulator the previous MMAs are still writing serialise; the
// row kernel's layout follows from both.  Every mbarrier wait is bounded by
// clock cycles; on timeout the CTA records the error, waits (bounded) for its
// own copies and MMAs in flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <mutex>

#include "async_copy.cuh"
#include "internal.h"

namespace lbm {
namespace {

using bf16 = __nv_bfloat16;

constexpr int kTcThreads = 192;
constexpr int kTcT = 2;                     // 128-pixel blocks per CTA tile
constexpr int kTcStages = 2;                // input ring depth
constexpr int kTcAcc = 2;                   // accumulator buffers (CTA tiles) in tensor memory
constexpr uint32_t kTcCols = kTcAcc * kTcT * 32;  // tensor-memory columns (power of 2, >= 32)
constexpr uint32_t kTapBytes = 32 * 64;     // one tap of the weights: 32 rows x 64 B
constexpr uint32_t kWBytes = 9 * kTapBytes;
constexpr long long kTcWaitCycles = 4000000000ll;  // about 2 s at 2 GHz

// instruction descriptor of tcgen05.mma .kind::f16: FP32 accumulator (bits
// 4-5 = 1), A and B BF16 (bits 7-9, 10-12 = 1), both K-major (bits 15, 16 =
// 0), N >> 3 in bits 17-22, M >> 4 in bits 24-28
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((32u >> 3) << 17) | ((128u >> 4) << 24);

struct TcShape {
    int B, H, W;
    int Wt, R, rows;   // pixels per row of a block, rows per block, output rows per CTA tile
    int xt, yt, n_ct;  // CTA tiles along x, along y, in total
    uint32_t box_bytes, copy_stride;
};

// shared-memory matrix descriptor: K-major, 64-byte swizzle (rows of 64 B,
// 8-row groups 512 B apart), descriptor version 1 (bits 46-47)
__device__ inline uint64_t sw64_desc(uint32_t saddr)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;            // leading-dimension offset: unused for swizzled K-major
    d |= (uint64_t)(512 >> 4) << 32;   // stride-dimension offset: next 8 rows
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;            // SWIZZLE_64B
    return d;
}

__device__ inline void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1, int c2, int c3, uint32_t bar)
{
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, "
        "%5}], [%6];\n" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
        : "memory");
}

__device__ inline void umma_f16(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc), "r"(accumulate)
        : "memory");
}

__device__ inline void umma_commit(uint32_t bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(bar)
                 : "memory");
}

__device__ inline void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory"); }
__device__ inline void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory"); }

// 32 consecutive FP32 columns of this thread's tensor-memory lane
__device__ inline void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];\n"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
}

__device__ inline void tile_origin(const TcShape& sh, int ct, int& b, int& y0, int& x0)
{
    const int xt = ct % sh.xt, rest = ct / sh.xt;
    x0 = xt * sh.Wt;
    y0 = (rest % sh.yt) * sh.rows;
    b = rest / sh.yt;
}

// one output pixel from its 32 FP32 accumulators: bias + ReLU (forward) or
// the ReLU' mask of the layer below (data gradient), BF16, one 64-byte store
template <bool BWD>
__device__ inline void epilogue_pixel(const uint32_t (&r)[32], const float* bias_s, const bf16* __restrict__ mask,
                                      bf16* __restrict__ out, int64_t o)
{
    uint4 mk[4];
    if (BWD) {
#pragma unroll
        for (int c = 0; c < 4; ++c) mk[c] = *reinterpret_cast<const uint4*>(mask + o + 8 * c);
    }
    uint32_t packed[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
        float v0 = __uint_as_float(r[2 * i]), v1 = __uint_as_float(r[2 * i + 1]);
        if (!BWD) {
            v0 = fmaxf(v0 + bias_s[2 * i], 0.f);
            v1 = fmaxf(v1 + bias_s[2 * i + 1], 0.f);
        } else {
            const uint32_t mw = reinterpret_cast<const uint32_t*>(mk)[i];
            const __nv_bfloat162 m2 = *reinterpret_cast<const __nv_bfloat162*>(&mw);
            if (!(__bfloat162float(m2.x) > 0.f)) v0 = 0.f;
            if (!(__bfloat162float(m2.y) > 0.f)) v1 = 0.f;
        }
        const __nv_bfloat162 p2 = __floats2bfloat162_rn(v0, v1);
        packed[i] = *reinterpret_cast<const uint32_t*>(&p2);
    }
#pragma unroll
    for (int c = 0; c < 4; ++c)
        *reinterpret_cast<uint4*>(out + o + 8 * c) =
            make_uint4(packed[4 * c], packed[4 * c + 1], packed[4 * c + 2], packed[4 * c + 3]);
}

// weights of the 9 taps into shared memory, 64-byte swizzled: 16-byte chunk c
// of row n of tap t lands at chunk c ^ ((n >> 1) & 3); KS = row stride of w
template <int KS>
__device__ inline void stage_weights(unsigned char* smem, const bf16* __restrict__ w, int nthreads)
{
    for (int i = threadIdx.x; i < 9 * 32 * 4; i += nthreads) {
        const int t = i >> 7, n = (i >> 2) & 31, c = i & 3;
        const uint4 v = *reinterpret_cast<const uint4*>(w + n * KS + t * 32 + c * 8);
        *reinterpret_cast<uint4*>(smem + t * kTapBytes + n * 64 + ((c ^ ((n >> 1) & 3)) << 4)) = v;
    }
}

// Block kernel for narrow inputs.  A block of 128 pixels is R = 128 / Wt rows
// of Wt = W pixels; a CTA tile stacks T = 2 blocks (T R rows).  The A operand
// of tap (ky, kx) for block j is the input shifted by (ky - 1, kx - 1): TMA
// loads the T R + 2 input rows of the tile three times, at x offsets kx - 1 =
// -1, 0, 1, into 64-byte-swizzled shared memory (each pixel's 32 channels one
// 64-byte row), where rows j R + ky .. of copy kx are exactly the K-major
// operand; 18 MMAs (9 taps x 2 K-steps) of N = 32 per block, two CTA-tile
// accumulators so the epilogue overlaps the next tile's MMAs.
//
// BWD = false: out = ReLU(conv(x, W) + bias), W = w[n][t*32 + k] (row stride
// 304, bias at column 288); BWD = true: out = conv(x, W') * (mask > 0), W' =
// w[n][t*32 + k] with row stride 288, no bias.
template <bool BWD>
__global__ void __launch_bounds__(kTcThreads, 1)
    conv_tc_kernel(const __grid_constant__ CUtensorMap tmap, const bf16* __restrict__ w,
                   const bf16* __restrict__ mask, bf16* __restrict__ out, const TcShape sh, int32_t* err)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kTcStages];
    __shared__ __align__(8) uint64_t empty[kTcStages];
    __shared__ __align__(8) uint64_t accf[kTcAcc];
    __shared__ __align__(8) uint64_t acce[kTcAcc];
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t tmem_slot;
    __shared__ float bias_s[32];
    __shared__ volatile int abort_flag;

    const uint32_t raw = smem_addr(smem_raw);
    unsigned char* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);  // 1024-byte aligned (swizzle atoms)
    const uint32_t w_s = smem_addr(smem);
    const uint32_t in_s = w_s + kWBytes;
    const uint32_t stage_stride = 3 * sh.copy_stride;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int KS = BWD ? 288 : 304;

    stage_weights<KS>(smem, w, kTcThreads);
    if (!BWD && threadIdx.x < 32) bias_s[threadIdx.x] = __bfloat162float(w[threadIdx.x * KS + 288]);
    if (threadIdx.x == 0) {
        for (int s = 0; s < kTcStages; ++s) {
            mbar_init(smem_addr(&full[s]), 1);
            mbar_init(smem_addr(&empty[s]), 1);
        }
        for (int a = 0; a < kTcAcc; ++a) {
            mbar_init(smem_addr(&accf[a]), 1);
            mbar_init(smem_addr(&acce[a]), 4);
        }
        mbar_init(smem_addr(&done), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_slot)),
                     "r"(kTcCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // weights -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer
        if (lane == 0) {
            int k = 0, issued = -1;
            for (int ct = blockIdx.x; ct < sh.n_ct; ct += gridDim.x, ++k) {
                const int s = k % kTcStages;
                if (k >= kTcStages && !mbar_wait_cycles(smem_addr(&empty[s]), ((k / kTcStages) - 1) & 1, kTcWaitCycles)) {
                    abort_flag = 1;
                    break;
                }
                if (abort_flag) break;
                int b, y0, x0;
                tile_origin(sh, ct, b, y0, x0);
                const uint32_t bar = smem_addr(&full[s]);
                mbar_expect_tx(bar, 3 * sh.box_bytes);
#pragma unroll
                for (int kx = 0; kx < 3; ++kx)
                    tma_load_4d(in_s + s * stage_stride + kx * sh.copy_stride, &tmap, 0, x0 + kx - 1, y0 - 1, b, bar);
                issued = k;
            }
            // the shared memory must outlive every copy issued into it
            for (int kk = issued - kTcStages + 1 > 0 ? issued - kTcStages + 1 : 0; kk <= issued; ++kk)
                mbar_wait_cycles(smem_addr(&full[kk % kTcStages]), (kk / kTcStages) & 1, kTcWaitCycles);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer
        if (lane == 0) {
            int k = 0;
            bool any = false;
            for (int ct = blockIdx.x; ct < sh.n_ct; ct += gridDim.x, ++k) {
                const int s = k % kTcStages, ab = k & 1;
                if (!mbar_wait_cycles(smem_addr(&full[s]), (k / kTcStages) & 1, kTcWaitCycles)) {
                    abort_flag = 1;
                    break;
                }
                if (k >= kTcAcc && !mbar_wait_cycles(smem_addr(&acce[ab]), ((k >> 1) - 1) & 1, kTcWaitCycles)) {
                    abort_flag = 1;
                    break;
                }
                if (abort_flag) break;
                tc_fence_after();
                const uint32_t sb = in_s + s * stage_stride;
#pragma unroll 1
                for (int j = 0; j < kTcT; ++j) {
                    const uint32_t d = tmem + (uint32_t)((ab * kTcT + j) * 32);
#pragma unroll
                    for (int tap = 0; tap < 9; ++tap) {
                        const int ky = tap / 3, kx = tap - 3 * (tap / 3);
                        const uint32_t a0 = sb + kx * sh.copy_stride + (uint32_t)((j * sh.R + ky) * sh.Wt * 64);
                        const uint32_t b0 = w_s + tap * kTapBytes;
#pragma unroll
                        for (int ks = 0; ks < 2; ++ks)
                            umma_f16(d, sw64_desc(a0 + ks * 32), sw64_desc(b0 + ks * 32), (tap | ks) != 0);
                    }
                }
                umma_commit(smem_addr(&accf[ab]));  // accumulators ready for the epilogue
                umma_commit(smem_addr(&empty[s]));  // input stage free for the producer
                any = true;
            }
            if (any) {  // every MMA issued has completed before the tensor memory is freed
                umma_commit(smem_addr(&done));
                mbar_wait_cycles(smem_addr(&done), 0, kTcWaitCycles);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warp w reads tensor-memory lanes 32 (w % 4) ..
        const int q = warp & 3;
        const int m = 32 * q + lane;  // pixel of the 128-pixel block
        int k = 0;
        for (int ct = blockIdx.x; ct < sh.n_ct; ct += gridDim.x, ++k) {
            const int ab = k & 1;
            if (!mbar_wait_cycles(smem_addr(&accf[ab]), (k >> 1) & 1, kTcWaitCycles)) abort_flag = 1;
            if (abort_flag) break;
            tc_fence_after();
            int b, y0, x0;
            tile_origin(sh, ct, b, y0, x0);
#pragma unroll 1
            for (int j = 0; j < kTcT; ++j) {
                uint32_t r[32];
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)((ab * kTcT + j) * 32), r);
                const int y = y0 + j * sh.R + m / sh.Wt, x = x0 + m % sh.Wt;
                const int64_t o = (((int64_t)b * sh.H + y) * sh.W + x) * 32;
                epilogue_pixel<BWD>(r, bias_s, mask, out, o);
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(smem_addr(&acce[ab]));  // accumulator buffer free again
        }
    }

    tc_fence_before();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0 && err) atomicExch(err, 1);
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kTcCols) : "memory");
    }
}

// ---------------------------------------------------------------------------
// Row kernel for widths that are a multiple of 128.  The three ky taps share
// their input row, so their weights are stacked along N: for input row r and
// its 128-pixel column segment,
//   D_r[p][32 ky + co] = sum_kx sum_ci X[r][x0 + p + kx - 1][ci] W[co][3 ky + kx][ci],
// six MMAs (3 kx x 2 K-steps of 16) of M = 128 pixels, N = 96, into one
// tensor-memory accumulator, and output row y is
//   out[y] = D_{y-1}[ky = 0] + D_y[ky = 1] + D_{y+1}[ky = 2]
// summed by the epilogue thread that owns the pixel (all three blocks sit in
// its own tensor-memory lane).  An MMA's cost hardly depends on N up to 128,
// so this does the layer in a third of the MMAs of one N = 32 MMA per tap.
// Each input row has an accumulator of its own: MMAs into an accumulator that
// the previous row's MMAs are still writing would serialise on it.
//
// Input rows are staged once (four 8-channel TMA boxes of the 130-pixel
// segment with its halo, in the interleaved K-major layout: channel chunk c of
// pixel p at chunk base + 16 p); the operand of shift kx starts 16 kx bytes
// into the chunk (8-pixel groups 128 B apart, the two 8-channel halves of a
// K-step one chunk apart).  TMA fills the zero padding at the borders.
//
// A persistent CTA walks a contiguous range of output rows down its (sample,
// 128-pixel column); for a run of output rows y_a .. y_b it computes D for
// input rows y_a - 1 .. y_b + 1.  An input slot is free once its row's MMAs
// complete; an accumulator once the (up to three) output rows that read it
// have loaded it: each reader's four warps arrive on the accumulator's
// barrier, the last reader also for the readers a run edge leaves out (12
// arrivals a use).
constexpr int kRowSlots = 12;                         // input-row ring
constexpr int kRowPairSlots = kRowSlots / 2;          // its pairs (one full / empty barrier each)
constexpr int kRowBufs = 4;                           // accumulators in tensor memory, 128 columns apart
constexpr int kRowPairBufs = kRowBufs / 2;            // accumulator pairs (one dfull / dfree barrier each)
constexpr int kRowEpi = 4;                            // epilogue warpgroups: output rows k = e mod kRowEpi
constexpr int kRowThreads = 64 + 128 * kRowEpi;
constexpr uint32_t kRowCols = 512;
constexpr uint32_t kChunkBytes = 2176;                // 130 pixels x 16 B, rounded up to 128 B
constexpr uint32_t kSlotBytes = 4 * kChunkBytes;
constexpr uint32_t kRowBoxBytes = 4 * 130 * 16;       // what one input row's four boxes deliver
constexpr uint32_t kStackBytes = 96 * 64;             // weights of one kx: 96 rows (ky, co) x 64 B
constexpr uint32_t kIdesc96 = (1u << 4) | (1u << 7) | (1u << 10) | ((96u >> 3) << 17) | ((128u >> 4) << 24);

struct RowShape {
    int B, H, W, xt;
    int64_t G;  // output rows (sample, column, y) in total
};

// interleaved K-major descriptor: 8-row core matrices of 16-byte rows
__device__ inline uint64_t interleave_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;  // version; layout bits 61-63 = 0: no swizzle
    return d;
}

__device__ inline void umma_f16_n96(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdesc96), "r"(accumulate)
        : "memory");
}

__device__ inline void mbar_arrive_n(uint32_t bar, uint32_t n)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(n) : "memory");
}

// walks the CTA's output rows [g0, g1): row(b, y, x0, ya, yb) with [ya, yb] the
// run down one column that y belongs to; stops when row returns false.
// Incremental: one division for the starting row, none per row.
template <typename F>
__device__ inline void walk_rows(const RowShape& sh, int64_t g0, int64_t g1, F&& row)
{
    if (g0 >= g1) return;
    int col = (int)(g0 / sh.H), y = (int)(g0 - (int64_t)col * sh.H);
    int b = col / sh.xt, xc = col - b * sh.xt;
    const int count = (int)(g1 - g0);
    int ya = y;
    for (int i = 0; i < count; ++i) {
        if (y == 0) ya = 0;
        const int left = count - 1 - i;
        const int yb = y + (sh.H - 1 - y < left ? sh.H - 1 - y : left);
        if (!row(b, y, xc * 128, ya, yb)) return;
        if (++y == sh.H) {
            y = 0;
            if (++xc == sh.xt) {
                xc = 0;
                ++b;
            }
        }
    }
}

// input rows a CTA computes D for: its output rows [g0, g1) plus two per run
// down a column (a run ends where a column does)
__device__ inline int row_count(const RowShape& sh, int64_t g0, int64_t g1)
{
    return g1 > g0 ? (int)(g1 - g0) + 2 * (int)((g1 - 1) / sh.H - g0 / sh.H + 1) : 0;
}

// stacked weights: for each kx, rows n = 32 ky + co of W[co][3 ky + kx][.],
// 64-byte swizzled (16-byte chunk c of row n at chunk c ^ ((n >> 1) & 3))
template <int KS>
__device__ inline void stage_stacked_weights(unsigned char* smem, const bf16* __restrict__ w, int nthreads)
{
    for (int i = threadIdx.x; i < 3 * 96 * 4; i += nthreads) {
        const int kx = i / 384, n = (i >> 2) % 96, c = i & 3;
        const int ky = n >> 5, co = n & 31;
        const uint4 v = *reinterpret_cast<const uint4*>(w + co * KS + (3 * ky + kx) * 32 + c * 8);
        *reinterpret_cast<uint4*>(smem + kx * kStackBytes + n * 64 + ((c ^ ((n >> 1) & 3)) << 4)) = v;
    }
}

template <bool BWD>
__global__ void __launch_bounds__(kRowThreads, 1)
    conv_row_kernel(const __grid_constant__ CUtensorMap tmap, const bf16* __restrict__ w,
                    const bf16* __restrict__ mask, bf16* __restrict__ out, const RowShape sh, int32_t* err)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full[kRowPairSlots];   // per pair of input rows
    __shared__ __align__(8) uint64_t empty[kRowPairSlots];
    __shared__ __align__(8) uint64_t dfull[kRowPairBufs];   // per pair of accumulators
    __shared__ __align__(8) uint64_t dfree[kRowPairBufs];
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t tmem_slot;
    __shared__ float bias_s[32];
    __shared__ volatile int abort_flag;

    const uint32_t raw = smem_addr(smem_raw);
    unsigned char* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);
    const uint32_t w_s = smem_addr(smem);
    const uint32_t ring_s = w_s + 3 * kStackBytes;  // 18432: 1024-aligned
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr int KS = BWD ? 288 : 304;
    const int64_t g0 = sh.G * blockIdx.x / gridDim.x, g1 = sh.G * (blockIdx.x + 1) / gridDim.x;

    stage_stacked_weights<KS>(smem, w, kRowThreads);
    if (!BWD && threadIdx.x < 32) bias_s[threadIdx.x] = __bfloat162float(w[threadIdx.x * KS + 288]);
    if (threadIdx.x == 0) {
        for (int i = 0; i < kRowPairSlots; ++i) {
            mbar_init(smem_addr(&full[i]), 1);
            mbar_init(smem_addr(&empty[i]), 2);  // one arrival per input row of the pair
        }
        for (int i = 0; i < kRowPairBufs; ++i) {
            mbar_init(smem_addr(&dfull[i]), 1);
            mbar_init(smem_addr(&dfree[i]), 24);  // 3 readers x 4 warps per accumulator
        }
        mbar_init(smem_addr(&done), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_slot)),
                     "r"(kRowCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer: input rows in the order the MMAs use them,
        // in pairs that share a full/empty barrier (the last pair of an odd count
        // holds one row).  The single thread's loop is the pipeline's pace, so its
        // bookkeeping is ring counters (pair slot, phase) rather than divisions.
        if (lane == 0) {
            const int n_in = row_count(sh, g0, g1);
            int n = 0, ps = 0;
            uint32_t par = 0;  // phase parity of the current pass over the pair slots
            auto load_row = [&](int b, int yr, int x0) -> bool {
                const uint32_t bar = smem_addr(&full[ps]);
                if ((n & 1) == 0) {  // the first row of a pair claims the pair slot
                    if (n >= 2 * kRowPairSlots && !mbar_wait_cycles(smem_addr(&empty[ps]), par ^ 1u, kTcWaitCycles)) {
                        abort_flag = 1;
                        return false;
                    }
                    if (abort_flag) return false;
                    mbar_expect_tx(bar, n + 1 < n_in ? 2 * kRowBoxBytes : kRowBoxBytes);
                }
                const uint32_t dst = ring_s + (uint32_t)(2 * ps + (n & 1)) * kSlotBytes;
#pragma unroll
                for (int c = 0; c < 4; ++c) tma_load_4d(dst + c * kChunkBytes, &tmap, 8 * c, x0 - 1, yr, b, bar);
                if ((++n & 1) == 0 && ++ps == kRowPairSlots) {
                    ps = 0;
                    par ^= 1u;
                }
                return true;
            };
            walk_rows(sh, g0, g1, [&](int b, int y, int x0, int ya, int) {
                if (y == ya && !(load_row(b, y - 1, x0) && load_row(b, y, x0))) return false;
                return load_row(b, y + 1, x0);
            });
            const int np = (n + 1) >> 1;  // pairs issued
            for (int k = np - kRowPairSlots > 0 ? np - kRowPairSlots : 0; k < np; ++k)
                mbar_wait_cycles(smem_addr(&full[k % kRowPairSlots]), (uint32_t)((k / kRowPairSlots) & 1),
                                 kTcWaitCycles);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer: D_s for every input row s, in order, two
        // rows an iteration.  The issuing thread's loop is the layer's pace: a
        // barrier wait, a commit and the loop cost it about as much as the six
        // MMAs of a row, so each iteration waits once for a pair of input rows
        // and a pair of accumulators and commits once.  The input rows are the
        // output rows plus two per run down a column; their MMAs do not depend on
        // which output row they serve, so the loop is a plain count, and the
        // descriptors of slot i are those of slot 0 advanced by i slots (the
        // start-address field holds address / 16 in 14 bits, which no
        // shared-memory address overflows).
        if (lane == 0) {
            const int n_in = row_count(sh, g0, g1);
            uint64_t ad[6], bd[6];
#pragma unroll
            for (int kx = 0; kx < 3; ++kx)
#pragma unroll
                for (int ks = 0; ks < 2; ++ks) {
                    ad[2 * kx + ks] = interleave_desc(ring_s + 2 * ks * kChunkBytes + 16 * kx, kChunkBytes, 128);
                    bd[2 * kx + ks] = sw64_desc(w_s + kx * kStackBytes + ks * 32);
                }
            int ps = 0, pb = 0;
            uint32_t fpar = 0, dround = 0;  // full's phase parity; passes over the accumulator pairs
            for (int sq = 0; sq < n_in; sq += 2) {
                // a failed wait elsewhere ends this loop through a failed wait here
                if (!mbar_wait_cycles(smem_addr(&full[ps]), fpar, kTcWaitCycles) ||
                    (sq >= 2 * kRowPairBufs &&
                     !mbar_wait_cycles(smem_addr(&dfree[pb]), (dround - 1u) & 1u, kTcWaitCycles))) {
                    abort_flag = 1;
                    break;
                }
                tc_fence_after();
                const int rows = sq + 1 < n_in ? 2 : 1;
                for (int r = 0; r < rows; ++r) {
                    const uint64_t so = (uint64_t)(((uint32_t)(2 * ps + r) * kSlotBytes) >> 4);
                    const uint32_t d = tmem + (uint32_t)((2 * pb + r) * 128);
#pragma unroll
                    for (int j = 0; j < 6; ++j) umma_f16_n96(d, ad[j] + so, bd[j], j != 0);
                }
                // both D ready for the epilogue, which also frees the input slots
                umma_commit(smem_addr(&dfull[pb]));
                if (++ps == kRowPairSlots) {
                    ps = 0;
                    fpar ^= 1u;
                }
                if (++pb == kRowPairBufs) {
                    pb = 0;
                    ++dround;
                }
            }
            if (n_in > 0) {
                umma_commit(smem_addr(&done));
                mbar_wait_cycles(smem_addr(&done), 0, kTcWaitCycles);
            }
        }
        __syncwarp();
    } else {
        // ---------------- epilogue: warpgroup e takes output rows k = e mod kRowEpi,
        // one pixel (tensor-memory lane 32 (warp % 4) + lane) per thread
        const int q = warp & 3;
        const int e = (warp - 2) >> 2;
        const int m = 32 * q + lane;
        const uint32_t lane_addr = tmem + ((uint32_t)(32 * q) << 16);
        int64_t n = 0;
        int k = 0;
        walk_rows(sh, g0, g1, [&](int b, int y, int x0, int ya, int yb) {
            if (y == ya) n += 2;
            const int64_t sq[3] = {n - 2, n - 1, n};  // input rows y - 1, y, y + 1
            ++n;
            if (k++ % kRowEpi != e) return true;
            // the pairs of input rows sq[0..2] (D of pair p in accumulator pair p mod 2)
            for (int j = 0; j < 3; ++j) {
                const int64_t pr = sq[j] >> 1;
                if (!mbar_wait_cycles(smem_addr(&dfull[pr % kRowPairBufs]), (uint32_t)((pr / kRowPairBufs) & 1),
                                      kTcWaitCycles)) {
                    abort_flag = 1;
                    return false;
                }
            }
            if (abort_flag) return false;
            tc_fence_after();
            // the MMAs of input rows sq[0..2] are complete: free the input slot of
            // the last (each input row is some output row's sq[2], but for the
            // two rows before a run's first, which its first output row frees)
            if (q == 0 && lane == 0) {
                mbar_arrive(smem_addr(&empty[(int)((sq[2] >> 1) % kRowPairSlots)]));
                if (y == ya) {
                    mbar_arrive(smem_addr(&empty[(int)((sq[0] >> 1) % kRowPairSlots)]));
                    mbar_arrive(smem_addr(&empty[(int)((sq[1] >> 1) % kRowPairSlots)]));
                }
            }
            uint32_t r[32], t[32];
            tmem_ld32(lane_addr + (uint32_t)((sq[0] % kRowBufs) * 128), r);
#pragma unroll
            for (int j = 1; j < 3; ++j) {
                tmem_ld32(lane_addr + (uint32_t)((sq[j] % kRowBufs) * 128 + 32 * j), t);
#pragma unroll
                for (int i = 0; i < 32; ++i) r[i] = __float_as_uint(__uint_as_float(r[i]) + __uint_as_float(t[i]));
            }
            // the sums are in registers: release the accumulators before the arithmetic
            tc_fence_before();
            __syncwarp();
            if (lane == 0) {
                // readers of input row y - 1: output rows y - 2 .. y within the run;
                // this row is its last, so it also arrives for the readers outside
                const uint32_t users_m1 = (uint32_t)(y - (y - 2 > ya ? y - 2 : ya) + 1);
                mbar_arrive_n(smem_addr(&dfree[(sq[0] >> 1) % kRowPairBufs]), 4 - users_m1);
                if (y == yb) {  // input rows y and y + 1 are read by no later row of the run
                    mbar_arrive_n(smem_addr(&dfree[(sq[1] >> 1) % kRowPairBufs]), y > ya ? 2u : 3u);
                    mbar_arrive_n(smem_addr(&dfree[(sq[2] >> 1) % kRowPairBufs]), 3);
                } else {
                    mbar_arrive_n(smem_addr(&dfree[(sq[1] >> 1) % kRowPairBufs]), 1);
                    mbar_arrive_n(smem_addr(&dfree[(sq[2] >> 1) % kRowPairBufs]), 1);
                }
            }
            epilogue_pixel<BWD>(r, bias_s, mask, out, (((int64_t)b * sh.H + y) * sh.W + x0 + m) * 32);
            return true;
        });
    }

    tc_fence_before();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0 && err) atomicExch(err, 1);
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kRowCols) : "memory");
    }
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder()
{
    static std::once_flag once;
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    std::call_once(once, [] {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

bool tc_shape(int B, int H, int W, TcShape& sh)
{
    if (B < 1 || H < 1 || W < 1) return false;
    sh.B = B;
    sh.H = H;
    sh.W = W;
    sh.Wt = W < 128 ? W : 128;
    if (128 % sh.Wt || W % sh.Wt || sh.Wt < 8) return false;
    sh.R = 128 / sh.Wt;
    sh.rows = kTcT * sh.R;
    if (H % sh.rows || sh.rows + 2 > 256) return false;
    sh.xt = W / sh.Wt;
    sh.yt = H / sh.rows;
    sh.n_ct = B * sh.xt * sh.yt;
    sh.box_bytes = (uint32_t)(64 * sh.Wt * (sh.rows + 2));
    sh.copy_stride = (sh.box_bytes + 1023u) & ~1023u;
    return true;
}

size_t tc_smem_bytes(const TcShape& sh) { return 1024 + kWBytes + (size_t)kTcStages * 3 * sh.copy_stride; }

// ---------------------------------------------------------------------------
// Weight gradient of a 32 -> 32 hidden layer (the layer's input x, its output
// gradient dy, both NHWC BF16) on the tensor cores:
//   dW[co][(ky*3 + kx)*32 + ci] = sum over pixels p of dy[p][co] x[p + (ky - 1, kx - 1)][ci],
//   db[co] = sum over pixels of dy[p][co],
// with x zero outside the image (the forward pass's padding).  The reduction
// runs over pixels.  A CTA takes bands of kWgBand output rows y0 .. y1 - 1 of
// one 128-pixel half x0 of an image.  For each input row r = y0 - 1 .. y1 one
// chain of 8 MMAs (K = 16 pixels each) accumulates
//   D[m][n] += sum_p A_r[m][p] B_r[n][p],
//   A_r[kx*32 + ci][p] = x[r][x0 + p + kx - 1][ci]   (kx = 0, 1, 2),
//   A_r[96 + c][p]     = (c == 0),
//   B_r[ky*32 + co][p] = dy[r - ky + 1][x0 + p][co]  if that row is in the band, else 0,
// so that D[kx*32 + ci][ky*32 + co] is dW of tap (ky, kx) and D[96][32 + co]
// is db.  M = 128, N = 96: each input row is read once and serves all nine taps.
// Both operands are MN-major with 64-byte swizzle, as TMA lays out the NHWC
// rows (a pixel's 32 channels one 64-byte row: 32 elements along MN, the pixel
// along K), 8-pixel groups 512 B apart (the descriptors' stride offset):
//   A: the three copies of the input row TMA loads at x offsets -1, 0, +1 and
//      a constant plane, kWgCopy bytes apart (the leading offset);
//   B: three consecutive slots of a ring of output-gradient rows, kWgCopy
//      bytes apart.  The ring runs to lower addresses (stream row t in slot
//      kWgDySlots - 1 - t mod kWgDySlots), so rows r + 1, r, r - 1 are slots
//      s, s + 1, s + 2; the rows in slots 0 and 1 are written a second time
//      into slots kWgDySlots and kWgDySlots + 1, so the three are contiguous
//      at the wrap too.  The rows just outside a band enter the stream as zero
//      rows (TMA loads far outside the image, zero-filled).
// The accumulator (96 columns) stays in tensor memory for the CTA's whole
// share; the epilogue writes the CTA's partial sums in the layout of the
// fixed-order cross-CTA reduction ([co][304], bias at column 288).
constexpr int kWgThreads = 192;             // TMA producer, MMA issuer, 4 epilogue warps
// output rows per work unit: a unit loads its band's input rows plus one halo
// row on each side, and the CTAs take whole units, so the slowest CTA's input
// rows are ceil(units / CTAs) x (kWgBand + 2); at 64 rows x 2 halves x 256
// images on 152 CTAs that is 7 x 34 = 238 for 32 against 14 x 18 = 252 for 16
constexpr int kWgBand = 32;
constexpr int kWgInSlots = 3;               // input-row ring (5 slots measured the same)
constexpr int kWgDySlots = 6;               // output-gradient ring (plus two mirror slots)
constexpr uint32_t kWgCopy = 128 * 64;      // one 128-pixel row of 32 channels
constexpr uint32_t kWgSlot = 4 * kWgCopy;   // three x-shifted copies and the constant plane
constexpr uint32_t kWgCols = 128;           // tensor-memory columns (power of 2; 96 used)
constexpr int kWgDoneRing = 4;              // row-completion barriers (more than kWgInSlots)
constexpr int kWgZeroRow = -64;             // a row far outside any image: TMA fills zeros
// kind::f16, FP32 accumulate, BF16 A and B, both MN-major (bits 15, 16), N = 96, M = 128
constexpr uint32_t kIdescMN =
    (1u << 4) | (1u << 7) | (1u << 10) | (1u << 15) | (1u << 16) | ((96u >> 3) << 17) | ((128u >> 4) << 24);

// shared-memory descriptor of an MN-major operand with 64-byte swizzle: the
// 64-byte rows are successive K (pixels), 8-row groups 512 B apart (stride
// offset); successive 32-element groups along MN lbo bytes apart (leading
// offset), descriptor version 1
__device__ inline uint64_t sw64_mn_desc(uint32_t saddr, uint32_t lbo)
{
    uint64_t d = (uint64_t)((saddr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)(512 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;  // SWIZZLE_64B
    return d;
}

__device__ inline void umma_f16_mn(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
        "l"(adesc), "l"(bdesc), "r"(kIdescMN), "r"(accumulate)
        : "memory");
}

struct WgShape {
    int B, H, W;
    int halves, bands, n_units;  // units: (image, band of output rows, 128-pixel half)
};

__device__ inline void wg_unit(const WgShape& sh, int u, int& b, int& y0, int& y1, int& x0)
{
    const int half = u % sh.halves, rest = u / sh.halves;
    const int band = rest % sh.bands;
    b = rest / sh.bands;
    x0 = half * 128;
    y0 = band * kWgBand;
    y1 = y0 + kWgBand < sh.H ? y0 + kWgBand : sh.H;
}

// ring slot of output-gradient stream row t (the ring runs to lower addresses)
__device__ inline int wg_dy_slot(int t) { return kWgDySlots - 1 - t % kWgDySlots; }

__global__ void __launch_bounds__(kWgThreads, 1)
    conv_wgrad_tc_kernel(const __grid_constant__ CUtensorMap xmap, const __grid_constant__ CUtensorMap dymap,
                         const WgShape sh, float* __restrict__ partial, int32_t* err)
{
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t in_full[kWgInSlots];
    __shared__ __align__(8) uint64_t in_empty[kWgInSlots];
    __shared__ __align__(8) uint64_t dy_empty[kWgDySlots];
    __shared__ __align__(8) uint64_t row_done[kWgDoneRing];
    __shared__ __align__(8) uint64_t done;
    __shared__ uint32_t tmem_slot;
    __shared__ volatile int abort_flag;

    const uint32_t raw = smem_addr(smem_raw);
    unsigned char* smem = smem_raw + (((raw + 1023u) & ~1023u) - raw);  // 1024-byte aligned (swizzle atoms)
    const uint32_t in_s = smem_addr(smem);
    const uint32_t dy_s = in_s + kWgInSlots * kWgSlot;  // kWgDySlots + 2 slots of kWgCopy
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;

    // the constant plane of every input slot: channel 0 = 1 and the rest 0 in
    // each pixel row (lane 96 of A), swizzled as TMA would: logical 16-byte
    // chunk 0 of row p sits at chunk (p >> 1) & 3
    for (int i = threadIdx.x; i < kWgInSlots * 128 * 4; i += kWgThreads) {
        const int sl = i / 512, p = (i >> 2) & 127, c = i & 3;
        const uint4 v = c == ((p >> 1) & 3) ? make_uint4(0x3F80u, 0u, 0u, 0u) : make_uint4(0u, 0u, 0u, 0u);
        *reinterpret_cast<uint4*>(smem + sl * kWgSlot + 3 * kWgCopy + p * 64 + c * 16) = v;
    }
    if (threadIdx.x == 0) {
        for (int k = 0; k < kWgInSlots; ++k) {
            mbar_init(smem_addr(&in_full[k]), 1);
            mbar_init(smem_addr(&in_empty[k]), 1);
        }
        for (int k = 0; k < kWgDySlots; ++k) mbar_init(smem_addr(&dy_empty[k]), 1);
        for (int k = 0; k < kWgDoneRing; ++k) mbar_init(smem_addr(&row_done[k]), 1);
        mbar_init(smem_addr(&done), 1);
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_addr(&tmem_slot)),
                     "r"(kWgCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n" ::: "memory");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");  // constant planes -> tensor-core reads
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        // ---------------- TMA producer.  Per unit the stream of output-
        // gradient rows is: zero, zero, dy rows y0 .. y1 - 1, zero, zero; input
        // row i (r = y0 - 1 + i) needs stream rows i .. i + 2.  The stream rows an
        // input row needs first (three for the unit's first, then one) complete
        // on that input row's barrier with its own copies, so that the MMA
        // issuer waits once a row: its shared-memory accesses queue behind the
        // tensor core's operand reads and cost it about as much as three MMAs.
        if (lane == 0) {
            int nin = 0, ndy = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < sh.n_units && ok; u += gridDim.x) {
                int b, y0, y1, x0;
                wg_unit(sh, u, b, y0, y1, x0);
                const int n_out = y1 - y0;
                for (int i = 0; i < n_out + 2 && ok; ++i) {
                    // claim the slots: the input row's, then its new stream rows'
                    const int sl = nin % kWgInSlots;
                    if (nin >= kWgInSlots &&
                        !mbar_wait_cycles(smem_addr(&in_empty[sl]), ((nin / kWgInSlots) - 1) & 1, kTcWaitCycles)) {
                        ok = false;
                        break;
                    }
                    const int n_new = i == 0 ? 3 : 1;
                    uint32_t bytes = 3 * kWgCopy;
                    for (int k = 0; k < n_new && ok; ++k) {
                        const int t = ndy + k, dsl = wg_dy_slot(t);
                        if (t >= kWgDySlots &&
                            !mbar_wait_cycles(smem_addr(&dy_empty[dsl]), ((t / kWgDySlots) - 1) & 1, kTcWaitCycles))
                            ok = false;
                        bytes += dsl < 2 ? 2 * kWgCopy : kWgCopy;  // slots 0 and 1 are mirrored past the end
                    }
                    if (!ok) break;
                    const uint32_t bar = smem_addr(&in_full[sl]);
                    mbar_expect_tx(bar, bytes);
                    for (int k = 0; k < n_new; ++k) {
                        // stream row i + 2 - (n_new - 1 - k): zero rows before and after the band
                        const int srow = i + 2 - (n_new - 1 - k);
                        const int y = srow >= 2 && srow - 2 < n_out ? y0 + srow - 2 : kWgZeroRow;
                        const int dsl = wg_dy_slot(ndy);
                        tma_load_4d(dy_s + dsl * kWgCopy, &dymap, 0, x0, y, b, bar);
                        if (dsl < 2) tma_load_4d(dy_s + (kWgDySlots + dsl) * kWgCopy, &dymap, 0, x0, y, b, bar);
                        ++ndy;
                    }
#pragma unroll
                    for (int kx = 0; kx < 3; ++kx)
                        tma_load_4d(in_s + sl * kWgSlot + kx * kWgCopy, &xmap, 0, x0 + kx - 1, y0 - 1 + i, b, bar);
                    ++nin;
                }
            }
            if (!ok) abort_flag = 1;
            // the shared memory must outlive every copy issued into it
            for (int kk = nin - kWgInSlots > 0 ? nin - kWgInSlots : 0; kk < nin; ++kk)
                mbar_wait_cycles(smem_addr(&in_full[kk % kWgInSlots]), (kk / kWgInSlots) & 1, kTcWaitCycles);
        }
        __syncwarp();
    } else if (warp == 1) {
        // ---------------- MMA issuer.  Its loop sets the pipeline's pace, so the
        // rings are followed with counters (slot, phase parity) and the operand
        // descriptors are those of slot 0 advanced by the slot's offset (the
        // start-address field holds address / 16 in 14 bits, which no shared-
        // memory address overflows).
        if (lane == 0) {
            uint64_t ad[8], bd[8];
#pragma unroll
            for (int ks = 0; ks < 8; ++ks) {
                ad[ks] = sw64_mn_desc(in_s + ks * 1024, kWgCopy);
                bd[ks] = sw64_mn_desc(dy_s + ks * 1024, kWgCopy);
            }
            int isl = 0, tm = 0, last = 0;  // input slot; stream row mod kWgDySlots; slot of the newest stream row
            int dr = 0;                     // row_done slot of this input row
            uint32_t ipar = 0;
            bool first = true, ok = true;
            for (int u = blockIdx.x; u < sh.n_units && ok && !abort_flag; u += gridDim.x) {
                int b, y0, y1, x0;
                wg_unit(sh, u, b, y0, y1, x0);
                const int n_out = y1 - y0;
                for (int i = 0; i < n_out + 2 && ok; ++i) {
                    // stream rows up to t0 + i + 2 (three new for the unit's first input
                    // row, then one) arrive on the input row's own barrier
                    for (int k = i == 0 ? 3 : 1; k > 0; --k) {
                        last = kWgDySlots - 1 - tm;
                        if (++tm == kWgDySlots) tm = 0;
                    }
                    ok = mbar_wait_cycles(smem_addr(&in_full[isl]), ipar, kTcWaitCycles);
                    if (!ok || abort_flag) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    // B: rows r + 1, r, r - 1 in slots last, last + 1, last + 2 (mirrored past the end)
                    const uint64_t ao = (uint64_t)(((uint32_t)isl * kWgSlot) >> 4);
                    const uint64_t bo = (uint64_t)(((uint32_t)last * kWgCopy) >> 4);
#pragma unroll
                    for (int ks = 0; ks < 8; ++ks)
                        umma_f16_mn(tmem, ad[ks] + ao, bd[ks] + bo, (first && ks == 0) ? 0u : 1u);
                    first = false;
                    // one commit a row (it costs the issuing thread about as much as
                    // two MMAs); the relay thread frees the slots this row read
                    umma_commit(smem_addr(&row_done[dr]));
                    if (++dr == kWgDoneRing) dr = 0;
                    if (++isl == kWgInSlots) {
                        isl = 0;
                        ipar ^= 1u;
                    }
                }
            }
            if (!ok) abort_flag = 1;
            // every MMA issued completes before the epilogue reads or the memory is freed
            umma_commit(smem_addr(&done));
        }
        __syncwarp();
    } else {
        // ---------------- relay: one thread follows the input rows in the MMA
        // issuer's order and, as each row's MMAs complete, frees its input slot
        // and the output-gradient row that leaves the window (at a unit's last
        // row also the window's last two).  The issuer runs at most kWgInSlots
        // rows ahead of it, so a row_done barrier is never a phase ahead of it.
        if (warp == 2 && lane == 0) {
            int isl = 0, tm = 0, dr = 0;  // as in the issuer
            uint32_t dpar = 0;
            bool ok = true;
            for (int u = blockIdx.x; u < sh.n_units && ok; u += gridDim.x) {
                int b, y0, y1, x0;
                wg_unit(sh, u, b, y0, y1, x0);
                const int n_out = y1 - y0;
                for (int i = 0; i < n_out + 2 && ok; ++i) {
                    ok = mbar_wait_cycles(smem_addr(&row_done[dr]), dpar, kTcWaitCycles);
                    if (!ok) break;
                    if (++dr == kWgDoneRing) {
                        dr = 0;
                        dpar ^= 1u;
                    }
                    mbar_arrive(smem_addr(&in_empty[isl]));
                    if (++isl == kWgInSlots) isl = 0;
                    // stream row t0 + i (slot kWgDySlots - 1 - (t0 + i) mod kWgDySlots)
                    mbar_arrive(smem_addr(&dy_empty[kWgDySlots - 1 - tm]));
                    if (++tm == kWgDySlots) tm = 0;
                }
                if (!ok) break;
                for (int k = 0; k < 2; ++k) {  // stream rows t0 + n_out + 2, t0 + n_out + 3
                    mbar_arrive(smem_addr(&dy_empty[kWgDySlots - 1 - tm]));
                    if (++tm == kWgDySlots) tm = 0;
                }
            }
            if (!ok) abort_flag = 1;
        }
        __syncwarp();
        // ---------------- epilogue: warp w reads tensor-memory lanes 32 (w % 4) ..
        const int q = warp & 3, m = 32 * q + lane;
        float* out = partial + (int64_t)blockIdx.x * 32 * 304;
        const bool work = (int)blockIdx.x < sh.n_units;
        bool ok = mbar_wait_cycles(smem_addr(&done), 0, kTcWaitCycles);
        ok = __all_sync(0xffffffffu, ok) && !abort_flag;
        if (!ok) abort_flag = 1;
        tc_fence_after();
#pragma unroll 1
        for (int ky = 0; ky < 3; ++ky) {
            uint32_t r[32];
            if (ok && work) {
                tmem_ld32(tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)(ky * 32), r);
            } else {
#pragma unroll
                for (int c = 0; c < 32; ++c) r[c] = 0u;
            }
            if (m < 96) {
                const int col = (ky * 3 + m / 32) * 32 + (m & 31);
#pragma unroll
                for (int co = 0; co < 32; ++co) out[co * 304 + col] = __uint_as_float(r[co]);
            } else if (m == 96 && ky == 1) {
#pragma unroll
                for (int co = 0; co < 32; ++co) out[co * 304 + 288] = __uint_as_float(r[co]);
            }
        }
        if (m < 32)  // padding columns of co = m
            for (int c = 289; c < 304; ++c) out[m * 304 + c] = 0.f;
    }

    tc_fence_before();
    __syncthreads();
    if (abort_flag && threadIdx.x == 0 && err) atomicExch(err, 1);
    if (warp == 1) {
        __syncwarp();
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem), "r"(kWgCols) : "memory");
    }
}

}  // namespace

// One 128-pixel column (W = 128) with more output rows than a wave of CTAs
// (several rows per CTA, runs crossing image boundaries) is the shape of the
// one GPU fault recorded for this library (CNN training at 32 x 128, batch 64;
// Xid 13 and 43).  Reading the row-ring and weight-gradient kernels found no
// out-of-range index for it, so the shape is kept off the tensor-core path:
// the mma.sync kernels take it.  148 rows: at most one per CTA on a 148-SM or
// larger part, the W = 128 shapes that run and are tested on this path.
constexpr int64_t kW128MaxRows = 148;

bool w128_cleared(int B, int H, int W) { return W != 128 || (int64_t)B * H <= kW128MaxRows; }

bool conv3x3_tc_supported(int B, int H, int W)
{
    if (tensor_map_encoder() == nullptr || B < 1 || H < 1) return false;
    if (W >= 128 && W % 128 == 0) return w128_cleared(B, H, W);  // row-ring kernel
    TcShape sh;
    return tc_shape(B, H, W, sh) && tc_smem_bytes(sh) <= 227 * 1024;
}

namespace {

int launch_ring(const void* x, const void* w, const void* mask, void* out, int B, int H, int W, bool bwd,
                int32_t* err, cudaStream_t s, PFN_cuTensorMapEncodeTiled_v12000 encode, int sms)
{
    CUtensorMap map;
    const cuuint64_t dims[4] = {32, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[3] = {64, (cuuint64_t)W * 64, (cuuint64_t)H * W * 64};
    const cuuint32_t box[4] = {8, 130, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LBM_ERR_CUDA, "conv3x3_tc: cuTensorMapEncodeTiled failed");
    RowShape sh{B, H, W, W / 128, (int64_t)B * (W / 128) * H};
    const size_t smem = 1024 + 3 * kStackBytes + (size_t)kRowSlots * kSlotBytes;
    const int grid = sh.G < sms ? (int)sh.G : sms;
    auto launch = [&](auto kernel) -> int {
        LBM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kernel<<<grid, kRowThreads, smem, s>>>(map, static_cast<const bf16*>(w), static_cast<const bf16*>(mask),
                                               static_cast<bf16*>(out), sh, err);
        LBM_CUDA(cudaGetLastError());
        count_launches(1);
        return LBM_OK;
    };
    return bwd ? launch(conv_row_kernel<true>) : launch(conv_row_kernel<false>);
}

}  // namespace

int conv3x3_tc(const void* x, const void* w, const void* mask, void* out, int B, int H, int W, bool bwd,
               int32_t* err, cudaStream_t s)
{
    auto encode = tensor_map_encoder();
    if (!encode) return fail(LBM_ERR_CUDA, "conv3x3_tc: cuTensorMapEncodeTiled unavailable");
    int dev = 0, sms = 152;
    LBM_CUDA(cudaGetDevice(&dev));
    LBM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (B >= 1 && H >= 1 && W >= 128 && W % 128 == 0)
        return launch_ring(x, w, mask, out, B, H, W, bwd, err, s, encode, sms);
    TcShape sh;
    if (!tc_shape(B, H, W, sh) || tc_smem_bytes(sh) > 227 * 1024)
        return fail(LBM_ERR_ARG, "conv3x3_tc: shape not supported by the tensor-core convolution");
    CUtensorMap map;
    const cuuint64_t dims[4] = {32, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[3] = {64, (cuuint64_t)W * 64, (cuuint64_t)H * W * 64};
    const cuuint32_t box[4] = {32, (cuuint32_t)sh.Wt, (cuuint32_t)(sh.rows + 2), 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    const CUresult r = encode(&map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(x), dims, strides, box, estr,
                              CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                              CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS) return fail(LBM_ERR_CUDA, "conv3x3_tc: cuTensorMapEncodeTiled failed");
    const size_t smem = tc_smem_bytes(sh);
    const int grid = sh.n_ct < sms ? sh.n_ct : sms;
    auto launch = [&](auto kernel) -> int {
        LBM_CUDA(cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        kernel<<<grid, kTcThreads, smem, s>>>(map, static_cast<const bf16*>(w), static_cast<const bf16*>(mask),
                                              static_cast<bf16*>(out), sh, err);
        LBM_CUDA(cudaGetLastError());
        count_launches(1);
        return LBM_OK;
    };
    return bwd ? launch(conv_tc_kernel<true>) : launch(conv_tc_kernel<false>);
}

bool conv3x3_wgrad_tc_supported(int B, int H, int W)
{
    return tensor_map_encoder() != nullptr && B >= 1 && H >= 1 && W >= 128 && W % 128 == 0 && w128_cleared(B, H, W);
}

int conv3x3_wgrad_tc(const void* x, const void* dy, float* partial, int B, int H, int W, int32_t* err,
                     cudaStream_t s, int* nblk)
{
    auto encode = tensor_map_encoder();
    if (!encode) return fail(LBM_ERR_CUDA, "conv3x3_wgrad_tc: cuTensorMapEncodeTiled unavailable");
    if (!conv3x3_wgrad_tc_supported(B, H, W)) return fail(LBM_ERR_ARG, "conv3x3_wgrad_tc: width must be a multiple of 128");
    int dev = 0, sms = 152;
    LBM_CUDA(cudaGetDevice(&dev));
    LBM_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    CUtensorMap maps[2];
    const void* src[2] = {x, dy};
    const cuuint64_t dims[4] = {32, (cuuint64_t)W, (cuuint64_t)H, (cuuint64_t)B};
    const cuuint64_t strides[3] = {64, (cuuint64_t)W * 64, (cuuint64_t)H * W * 64};
    const cuuint32_t box[4] = {32, 128, 1, 1};
    const cuuint32_t estr[4] = {1, 1, 1, 1};
    for (int k = 0; k < 2; ++k) {
        const CUresult r = encode(&maps[k], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void*>(src[k]), dims, strides,
                                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B,
                                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
        if (r != CUDA_SUCCESS) return fail(LBM_ERR_CUDA, "conv3x3_wgrad_tc: cuTensorMapEncodeTiled failed");
    }
    WgShape sh{B, H, W, W / 128, (H + kWgBand - 1) / kWgBand, 0};
    sh.n_units = B * sh.bands * sh.halves;
    const int grid = sh.n_units < sms ? sh.n_units : sms;
    const size_t smem = 1024 + (size_t)kWgInSlots * kWgSlot + (size_t)(kWgDySlots + 2) * kWgCopy;
    LBM_CUDA(cudaFuncSetAttribute(conv_wgrad_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    conv_wgrad_tc_kernel<<<grid, kWgThreads, smem, s>>>(maps[0], maps[1], sh, partial, err);
    LBM_CUDA(cudaGetLastError());
    count_launches(1);
    *nblk = grid;
    return LBM_OK;
}

}  // namespace lbm
