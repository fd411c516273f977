// mbarrier and bulk-copy (TMA engine, cp.async.bulk) wrappers shared by the
// matching kernels.  Every wait is bounded: mbar_wait gives up after
// kWaitLimitNs of the global timer (or kBulkWaitLimit polls, whichever comes
// first) and returns false, and the caller records a timeout, drains its
// copies in flight and returns.  A poll may suspend the thread for up to
// kSuspendNs (it wakes as soon as the phase completes), so a waiting warp
// takes few issue slots from the warps that work.
#pragma once

#include <stdint.h>

namespace kmx {

constexpr uint32_t kBulkWaitLimit = 1u << 22;
constexpr uint64_t kWaitLimitNs = 1000000000ull;  // 1 s
constexpr uint32_t kSuspendNs = 20000;

__device__ __forceinline__ uint32_t smem_u32(const void* p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_fence_init() { asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory"); }

__device__ __forceinline__ void mbar_expect_tx(uint64_t* bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ uint64_t global_ns()
{
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// One poll of the phase with the given parity (potentially blocking for up
// to kSuspendNs).
__device__ __forceinline__ bool mbar_try(uint32_t a, uint32_t parity)
{
    uint32_t done;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(a), "r"(parity), "r"(kSuspendNs)
        : "memory");
    return done != 0;
}

// Bounded wait for the phase with the given parity; false on timeout.
__device__ __forceinline__ bool mbar_wait(uint64_t* bar, uint32_t parity)
{
    const uint32_t a = smem_u32(bar);
    if (mbar_try(a, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < kBulkWaitLimit; ++it) {
        if (mbar_try(a, parity)) return true;
        if (global_ns() - t0 > kWaitLimitNs) return false;
    }
    return false;
}

// Global -> shared copy of `bytes` (a multiple of 16, both addresses 16-byte
// aligned), completing as transaction bytes on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_u32(dst)),
                 "l"(src), "r"(bytes), "r"(smem_u32(bar))
                 : "memory");
}

}  // namespace kmx
