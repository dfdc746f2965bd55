// gridsync.cuh -- a grid-wide barrier with bounded waits for kernels launched cooperatively
// (every block resident at once), used by the fused grid-stage kernel.
//
// The barrier is one 64-bit arrival counter in global memory that only grows: block b's
// thread 0 adds 1 when it arrives and waits until the counter reaches the next multiple
// of the launch's block count.  A launch whose every barrier completes leaves the counter
// at a multiple of the block count, so the next launch over the same counter needs no
// reset.  A wait gives up after `limit` SM clock cycles: the block ORs STATUS_TIMEOUT into
// the plan's status word and raises the abort word, which every other waiting block sees
// and leaves on at once; each block then skips its remaining stages and returns.  The host
// zeroes both words after reporting the timeout (the counter is then no longer a multiple
// of the block count).
#pragma once

#include <cuda_runtime.h>
#include <cstdint>

#include "internal.h"

namespace nnfft {
namespace gsync {


__device__ __forceinline__ unsigned long long ld_acquire(const unsigned long long *p) {
    unsigned long long v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// words[0]: arrival counter, words[1]: abort word (nonzero: some block gave up).
// `expected` is the number of blocks that arrive at every barrier (gridDim.x for the
// kernels of this library).  Returns false (in every thread of the block) when this
// block gave up or another block did: the caller returns without touching shared data.
__device__ __forceinline__ bool grid_barrier(unsigned long long *words, unsigned expected,
                                             long long limit, int *status) {
    __shared__ int ok_s;
    __syncthreads();                              // the block's work before the barrier
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned *abort_word = reinterpret_cast<unsigned *>(words + 1);
        __threadfence();                          // publish the block's writes (cumulative)
        const unsigned long long old = atomicAdd(words, 1ULL);
        const unsigned long long target = (old / expected + 1ULL) * expected;
        const long long t0 = clock64();
        while (ld_acquire(words) < target) {
            if (ld_acquire(abort_word) != 0u) {
                ok = 0;
                break;
            }
            if (clock64() - t0 > limit) {
                atomicOr(status, STATUS_TIMEOUT);
                atomicExch(abort_word, 1u);
                ok = 0;
                break;
            }
            __nanosleep(64);
        }
        __threadfence();                          // see the other blocks' writes
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

}  // namespace gsync
}  // namespace nnfft
