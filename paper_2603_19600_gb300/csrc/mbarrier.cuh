// Shared-memory mbarriers with bounded waits (producer/consumer hand-off inside one CTA).
// A wait that has not completed within its budget of SM cycles records an error word in global
// memory and returns false; the caller then leaves its loop, so a kernel always terminates.
//
// The handle's device control block (kCtlWords 32-bit words, furax_pointing::d_err):
//   [0]    error word (kErrWaitTimeout once a wait gave up; cleared by furax_device_status)
//   [1]    hold flag: the loader of the cached FP32 operator issues no copies while it is set
//          (furax_debug_hold_loader), so that the other roles' waits run out
//   [2..3] wait budget in SM cycles (int64; 0 selects kWaitCycles)
#pragma once
#include <cstdint>

namespace fx {

constexpr long long kWaitCycles = 1LL << 32;   // ~2 s at 2 GHz: far above any legitimate wait
constexpr unsigned kErrWaitTimeout = 1u;

// The budget a kernel's waits use, read once at kernel start.
__device__ __forceinline__ long long wait_budget(const unsigned *ctl)
{
    const long long b = *reinterpret_cast<const volatile long long *>(ctl + 2);
    return b > 0 ? b : kWaitCycles;
}

__device__ __forceinline__ bool loader_held(const unsigned *ctl)
{
    return *reinterpret_cast<const volatile unsigned *>(ctl + 1) != 0u;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

// Arrive (release: this thread's prior shared-memory writes become visible to the waiters).
__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ bool mbar_test(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// L2 policy for data read once (the pointing stream): evict first, so that it does not displace
// the randomly accessed map and accumulators.
__device__ __forceinline__ uint64_t evict_first_policy()
{
    uint64_t pol;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(pol));
    return pol;
}

// Global -> shared bulk copy completing on `bar` (bytes counted); dst, src and bytes multiples of
// 16. With hint, the source is read under the L2 policy pol.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar, bool hint,
                                              uint64_t pol)
{
    if (hint)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint [%0], [%1], %2, [%3], %4;" ::"r"(
                smem_u32(dst)),
            "l"(src), "r"(bytes), "r"(smem_u32(bar)), "l"(pol)
            : "memory");
    else
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                         smem_u32(dst)),
                     "l"(src), "r"(bytes), "r"(smem_u32(bar))
                     : "memory");
}

// Wait until the phase with the given parity has completed (acquire). Bounded by `budget` cycles.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned *err, long long budget)
{
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (clock64() - t0 > budget) {
            atomicOr(err, kErrWaitTimeout);
            return false;
        }
    }
    return true;
}

}  // namespace fx
