// Mixed-precision defect correction: the FP64 update of the refinement loop.
//
// One outer step of the refinement (the loop lives in api.cu):
//   1. rt = h^2 (b - A u) in FP64 and max |rt| (residual.cu, exact max);
//   2. e = the binary exponent of max |rt|; r32 = (float)(rt * 2^-e)   (exact scaling,
//      one rounding to binary32);
//   3. d = m FP32 red-black sweeps of (4 I - Adj) d = r32 from d = 0 with a zero ring
//      (the update of Eq. (1) with h^2 f replaced by r32);
//   4. u = u + (double)d * 2^e at interior points   (this file).
// Steps 1-2 and 4 touch the FP64 iterate; only step 3 runs in FP32.
#include "common.cuh"

namespace rbgs {
namespace {

constexpr int kThreads = 256;

__global__ void __launch_bounds__(kThreads)
correct_kernel(double *__restrict__ red, double *__restrict__ black, const float *__restrict__ d_red,
               const float *__restrict__ d_black, int n, int W, int W32, double scale) {
    const int k = blockIdx.x * kThreads + threadIdx.x;
    if (k > (n + 1) / 2) return;
    for (int i = 1 + blockIdx.y; i <= n; i += gridDim.y) {
        // colour c of row i holds natural column j = 2k + ((i + c) & 1)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
            const int j = 2 * k + ((i + c) & 1);
            if (j < 1 || j > n) continue;
            double *u = c ? black : red;
            const float *d = c ? d_black : d_red;
            const size_t q = (size_t)i * W + k;
            u[q] = __dadd_rn(u[q], __dmul_rn((double)d[(size_t)i * W32 + k], scale));
        }
    }
}

}  // namespace

rbgs_status launch_correct(const rbgs_ctx *c, double scale, cudaStream_t s) {
    const int n = c->g.n;
    const int kmax = (n + 1) / 2 + 1;
    int gy = n < 65535 ? n : 65535;
    dim3 grid((kmax + kThreads - 1) / kThreads, gy);
    correct_kernel<<<grid, kThreads, 0, s>>>(c->f64.u[0], c->f64.u[1], c->f32.u[0], c->f32.u[1], n, c->g.W,
                                             c->f32.W, scale);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

}  // namespace rbgs
