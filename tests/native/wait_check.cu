// Test harness for the library's bounded mbarrier wait (csrc/tma.cuh): one kernel waits
// on a barrier that nothing completes and must give up after `polls` polls and report
// it; a control kernel arrives on the barrier first and must see it complete.
// Test infrastructure only.
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

}  // namespace

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
