// Test harness for the library's bounded mbarrier waits.
//  * csrc/tma.cuh: one kernel waits on a barrier that nothing completes and must give up
//    after `polls` polls and report it; a control kernel arrives on the barrier first
//    and must see it complete.
//  * csrc/grid_barrier.cuh (the cooperative FP64 sweep launch): two blocks of a cooperative
//    launch meet at the barrier; with one block absent (it leaves at once), the other's wait
//    must run out after `polls` polls and set the status instead of waiting forever.
//  * csrc/conv_wait.cuh (the convolution kernels' abort protocol): one role spins on a
//    barrier that nothing completes, another role waits (suspending) on a second barrier
//    that nothing completes either.  The side with the short limit must give up and raise
//    the abort flag; the other must leave through the flag, long before its own limit.
// Test infrastructure only.
#include "../../paper_2607_01735_gb300/csrc/conv_wait.cuh"
#include "../../paper_2607_01735_gb300/csrc/grid_barrier.cuh"
#include "../../paper_2607_01735_gb300/csrc/tma.cuh"

namespace {

__global__ void wait_kernel(unsigned polls, int arrive, int *status) {
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) {
        rbgs::mbar_init(&bar, 1);
        rbgs::fence_barrier_init();
    }
    __syncthreads();
    if (arrive && threadIdx.x == 0) {
        asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(rbgs::smem_addr(&bar)) : "memory");
    }
    const bool ok = rbgs::mbar_wait_bounded(&bar, 0, polls);
    if (!ok) atomicOr(status, 1);   // the wait gave up
    if (ok) atomicOr(status, 2);    // the barrier completed
}

// Thread 0 plays the single issuing thread (spinning wait, `polls` polls); warp 1 plays
// the epilogue (suspending waits of at most 1 ms, `waiter_polls` of them).
__global__ void abort_kernel(unsigned polls, unsigned waiter_polls, int *status, int *fail_issuer,
                             int *fail_waiter) {
    __shared__ uint64_t a, b;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        rbgs::mbar_init(&a, 1);
        rbgs::mbar_init(&b, 1);
        abort_flag = 0;
        rbgs::fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        const bool ok = rbgs::wait_or_abort_spin(&a, 0, &abort_flag, polls, fail_issuer);
        atomicOr(status, ok ? 4 : 1);  // 1: the issuer gave up
    } else if (threadIdx.x >= 32) {
        const bool ok = rbgs::wait_or_abort(&b, 0, &abort_flag, waiter_polls, 1000000u, fail_waiter);
        atomicOr(status, ok ? 4 : 2);  // 2: a waiter left without completion
    }
}

__global__ void grid_barrier_kernel(unsigned *counter, int *status, int absent, unsigned polls, int *passed) {
    if (absent && blockIdx.x == 1) return;  // this block never arrives
    const bool ok = rbgs::grid_barrier(counter, gridDim.x, status, polls);
    if (ok && threadIdx.x == 0) atomicAdd(passed, 1);
}

}  // namespace

// out_host[0]: the status word, out_host[1]: blocks that passed the barrier.
extern "C" int run_grid_barrier_check(int absent, unsigned polls, int *out_host) {
    unsigned *counter = nullptr;
    int *d = nullptr;
    if (cudaMalloc(&counter, sizeof(unsigned)) != cudaSuccess) return 1;
    if (cudaMalloc(&d, 2 * sizeof(int)) != cudaSuccess) {
        cudaFree(counter);
        return 1;
    }
    cudaMemset(counter, 0, sizeof(unsigned));
    cudaMemset(d, 0, 2 * sizeof(int));
    int *status = d, *passed = d + 1;
    void *args[] = {&counter, &status, &absent, &polls, &passed};
    cudaError_t e = cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(grid_barrier_kernel), dim3(2),
                                                dim3(64), args, 0, 0);
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(out_host, d, 2 * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(counter);
    cudaFree(d);
    return e == cudaSuccess ? 0 : 2;
}

extern "C" int run_abort_check(unsigned polls, unsigned waiter_polls, int *out_host) {
    int *d = nullptr;
    if (cudaMalloc(&d, 3 * sizeof(int)) != cudaSuccess) return 1;
    cudaMemset(d, 0, 3 * sizeof(int));
    abort_kernel<<<1, 64>>>(polls, waiter_polls, d, d + 1, d + 2);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(out_host, d, 3 * sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : 2;
}

extern "C" int run_wait_check(unsigned polls, int arrive, int *status_host) {
    int *d = nullptr;
    if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) return 1;
    cudaMemset(d, 0, sizeof(int));
    wait_kernel<<<1, 64>>>(polls, arrive, d);
    cudaError_t e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(status_host, d, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(d);
    return e == cudaSuccess ? 0 : 2;
}
