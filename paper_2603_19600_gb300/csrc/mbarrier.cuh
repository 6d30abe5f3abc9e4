// Shared-memory mbarriers with bounded waits (producer/consumer hand-off inside one CTA).
// A wait that has not completed after kWaitCycles SM cycles records an error word in global
// memory and returns false; the caller then leaves its loop, so a kernel always terminates.
#pragma once
#include <cstdint>

namespace fx {

constexpr long long kWaitCycles = 1LL << 32;   // ~2 s at 2 GHz: far above any legitimate wait
constexpr unsigned kErrWaitTimeout = 1u;

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

// Wait until the phase with the given parity has completed (acquire). Bounded.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned *err)
{
    if (mbar_test(bar, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_test(bar, parity)) {
        if (clock64() - t0 > kWaitCycles) {
            atomicOr(err, kErrWaitTimeout);
            return false;
        }
    }
    return true;
}

}  // namespace fx
