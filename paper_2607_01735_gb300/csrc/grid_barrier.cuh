// Bounded grid barrier for kernels whose blocks are all resident at once (cooperative
// launch).  One counter per launch, zeroed before it.  At every barrier each block's
// thread 0, after the block barrier, fences the block's writes and adds one; it then polls
// (acquire) until the counter reaches `target` = the number of blocks times the barriers
// passed so far.  The wait is bounded: after `max_polls` polls, or as soon as the status
// word is nonzero (another block gave up), the block sets bit 1 of the status and the
// function returns false; the caller then leaves the kernel.
#pragma once

#include <cstdint>

namespace rbgs {

__device__ __forceinline__ unsigned ld_acquire_gpu(const unsigned *p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ bool grid_barrier(unsigned *counter, unsigned target, int *status, uint32_t max_polls) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();  // the block's stores of this phase, before its arrival
        atomicAdd(counter, 1u);
        int ok = 1;
        for (uint32_t q = 0; ld_acquire_gpu(counter) < target; ++q) {
            if (q >= max_polls || *reinterpret_cast<volatile int *>(status) != 0) {
                ok = 0;
                break;
            }
        }
        if (!ok) atomicOr(status, 2);
        s_ok = ok;
    }
    __syncthreads();
    return s_ok != 0;
}

}  // namespace rbgs
