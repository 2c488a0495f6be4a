// Bounded waits on shared-memory mbarriers, used by every kernel of the library that waits on asynchronous
// work (the FFT's bulk-copy ring, the tensor-core kernels' pipelines) and by the wait self-test
// (pusch_selftest_wait). A wait polls the barrier phase and gives up once %globaltimer has passed a
// deadline, so that a copy or an MMA that never completes turns into an error bit the host can read instead
// of a kernel that never ends.
#pragma once

#include <stdint.h>

namespace pusch {
namespace bw {

constexpr uint64_t kWaitNs = 2000000000ull;  // the library kernels' limit: 2 s

__device__ __forceinline__ uint64_t globaltimer() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}

// Waits until the phase with the given parity of the barrier at shared address `bar` has completed, for at
// most limit_ns nanoseconds of %globaltimer. Returns false when the limit passed first.
__device__ __forceinline__ bool mbar_wait_for(uint32_t bar, uint32_t parity, uint64_t limit_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t deadline = globaltimer() + limit_ns;
    while (!mbar_try_wait(bar, parity))
        if (globaltimer() > deadline) return false;
    return true;
}

}  // namespace bw
}  // namespace pusch
