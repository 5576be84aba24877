// cw_tma.cuh -- 1D bulk asynchronous copies (TMA, cp.async.bulk) into shared memory, completed
// on an mbarrier, with bounded waits.
//
// A CTA's tile of consecutive cells is one contiguous span of each cell-wise array, so a single
// bulk copy per array moves it (no tensor map). A bulk copy needs 16-byte aligned source and
// destination and a size that is a multiple of 16; callers check this per tile and load the
// tile with ordinary loads otherwise (e.g. a ragged last tile).
#pragma once
#include <cstdint>

namespace cw {

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

// global -> shared bulk copy completing `bytes` transactions on `bar`
__device__ __forceinline__ void bulk_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

// bulk prefetch of a global range into L2 (no shared memory, no completion to wait for)
__device__ __forceinline__ void bulk_prefetch_l2(const void *src, uint32_t bytes)
{
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(src), "r"(bytes) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Bounded wait for phase `parity` of `bar`: returns false if the phase did not complete within
// `limit` polls (each poll may suspend the thread for a hardware-defined time).
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t *bar, uint32_t parity, uint32_t limit = 1u << 22)
{
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity)) return true;
    return false;
}

__device__ __forceinline__ bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

// Poll limits of the staged tiles' waits: the normal bound (far above any real copy time), and the
// short bound used when a test arms a barrier that cannot complete (see the fault-injection hook).
constexpr uint32_t kWaitLimit = 1u << 22;
constexpr uint32_t kWaitLimitInjected = 1u << 10;
// bit set in an operator's device status word when a bounded wait expired
constexpr unsigned kDevStatusTimeout = 1u;

}  // namespace cw
