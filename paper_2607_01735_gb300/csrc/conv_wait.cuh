// Bounded mbarrier waits with a block-wide abort flag, for the warp-specialised
// convolution kernels.  Their roles (loader, MMA issuer, epilogue) wait on one another's
// barriers; if one role gives up, the others must leave too, or they would wait for
// hand-offs that never come.  Every wait therefore polls a bounded number of times and,
// between polls, the abort flag: the first role to run out of polls sets the flag and
// the failure word, and every other role returns as soon as it sees the flag.
#pragma once

#include "tma.cuh"

namespace rbgs {

// One poll that suspends the thread until the phase with `parity` completes or about
// `ns` nanoseconds have passed (a hint; the hardware may return earlier).
__device__ __forceinline__ bool mbar_try_wait_suspend(uint64_t *bar, uint32_t parity, uint32_t ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity), "r"(ns)
        : "memory");
    return ok != 0;
}

// Suspending wait: at most `polls` polls of up to `ns` each.  Returns true when the phase
// completed; false when another role aborted, or when this wait ran out (it then sets
// the abort flag and the failure word).
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                              uint32_t polls, uint32_t ns, int *fail_word) {
    for (uint32_t q = 0; q < polls; ++q) {
        if (mbar_try_wait_suspend(bar, parity, ns)) return true;
        if (*abort_flag) return false;
    }
    *abort_flag = 1;
    atomicOr(fail_word, 1);
    return false;
}

// Polling wait without a suspend hint, for single issuing threads whose hand-offs sit on
// the critical path of every stage; the abort flag is read every 256 polls.
__device__ __forceinline__ bool wait_or_abort_spin(uint64_t *bar, uint32_t parity, volatile int *abort_flag,
                                                   uint32_t polls, int *fail_word) {
    for (uint32_t q = 0; q < polls; ++q) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((q & 255u) == 255u && *abort_flag) return false;
    }
    *abort_flag = 1;
    atomicOr(fail_word, 1);
    return false;
}

}  // namespace rbgs
