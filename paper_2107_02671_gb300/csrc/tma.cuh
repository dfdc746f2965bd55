// tma.cuh -- bulk copies global -> shared memory through the Tensor Memory Accelerator
// (cp.async.bulk with an mbarrier transaction count), with bounded waits.
//
// One thread of a block arms the barrier with the byte count and issues the copy; every
// thread that needs the data waits on the barrier's phase.  A wait gives up after
// `limit` SM clock cycles: the caller then records a timeout in the plan's status word
// (NNFFT_ETIMEOUT at the next nnfft_sync) and, before the block exits, waits once more
// (bounded again) so that no copy is still writing its shared memory.
//
// Copies must start at 16-byte aligned addresses (source and destination) and move a
// multiple of 16 bytes; the barrier's transaction count holds at most 2^20 - 1 bytes.
// Only this GPU's own memory is read (no cluster multicast).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

namespace nnfft {
namespace tma {

// about one second at the GB300's 2.07 GHz SM clock
constexpr long long WAIT_LIMIT_CYCLES = 2000000000LL;

__device__ __forceinline__ unsigned smem_addr(const void *p) {
    return (unsigned)__cvta_generic_to_shared(p);
}

// one thread: barrier with an arrival count of 1, made visible to the async proxy
__device__ __forceinline__ void bar_init(uint64_t *bar) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(bar)) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// one thread: arrive on the barrier announcing `bytes` of transactions for this phase
__device__ __forceinline__ void bar_expect(uint64_t *bar, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                 ::"r"(smem_addr(bar)), "r"(bytes) : "memory");
}

// one thread: global -> shared bulk copy completing `bytes` transactions on the barrier
__device__ __forceinline__ void copy_g2s(void *dst, const void *src, unsigned bytes,
                                         uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
        ::"r"(smem_addr(dst)), "l"(src), "r"(bytes), "r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ bool bar_test(uint64_t *bar, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// wait for the barrier's phase `parity` to complete; false after `limit` cycles
__device__ __forceinline__ bool bar_wait(uint64_t *bar, unsigned parity, long long limit) {
    const long long t0 = clock64();
    while (!bar_test(bar, parity)) {
        if (clock64() - t0 > limit) return false;
    }
    return true;
}

}  // namespace tma
}  // namespace nnfft
