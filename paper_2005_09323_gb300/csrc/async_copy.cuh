// Asynchronous-copy and mbarrier helpers shared by the kernels that stage
// data in shared memory with the bulk-copy engine (inline PTX, sm_100+).
// Every wait is bounded: a caller that gets `false` back records an error and
// winds down instead of spinning forever.
#pragma once
#include <cstdint>

namespace lbm {

constexpr long long kWaitCycles = 4000000000ll;  // SM clock cycles before a cycle-bounded wait gives up (about 2 s)

__device__ inline uint32_t smem_addr(const void* p) { return static_cast<uint32_t>(__cvta_generic_to_shared(p)); }

__device__ inline void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count));
}

__device__ inline void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(bar), "r"(bytes) : "memory");
}

__device__ inline void mbar_arrive(uint32_t bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(bar) : "memory");
}

__device__ inline bool mbar_try_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ inline void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(dst),
                 "l"(src), "r"(bytes), "r"(bar)
                 : "memory");
}

// one try that suspends the thread in hardware until the phase completes or
// about `ns` nanoseconds pass (the suspend-time hint of mbarrier.try_wait), so
// that a waiting warp issues no instructions meanwhile
__device__ inline bool mbar_try_wait_suspend(uint32_t bar, uint32_t parity, uint32_t ns)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// bounded by elapsed SM clock cycles instead of a poll count.  After a first
// plain try the thread waits in suspended tries: a warp that polled instead
// would keep issuing barrier reads through the shared-memory pipe, which the
// warps that issue the copies and the MMAs need as well.
__device__ inline bool mbar_wait_cycles(uint32_t bar, uint32_t parity, long long limit_cycles)
{
    if (mbar_try_wait(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try_wait_suspend(bar, parity, 20000u))
        if (clock64() - t0 > limit_cycles) return false;
    return true;
}

}  // namespace lbm
