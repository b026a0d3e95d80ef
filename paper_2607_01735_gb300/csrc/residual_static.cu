// rbgs_residual_static: the relative residual of a natural-layout iterate, computed
// without allocating any memory.
//
// rbgs_residual needs a solver context, and creating one allocates device buffers.  Some
// callers cannot do that: code that runs under a fixed device-memory budget decided up
// front (embedded or real-time services, plugins hosted by a framework that owns all
// allocations), code called from inside an allocator or a memory-pool callback, and
// code that must not trigger the implicit device synchronisation that cudaMalloc and
// cudaFree can cause.  This entry point takes the caller's buffers and writes the
// result into the caller's memory; its only scratch is a fixed array in the library's
// own device image (a file-scope __device__ array, present on every GPU that loads the
// library until the process exits).
//
// Scratch: kStaticBlocks partial sums of rt^2 and of (h^2 b)^2, one pair per block of
// kStaticRows grid rows, so n may be at most kStaticBlocks * kStaticRows = 32768.
// Every call overwrites every slot it reads before reading it, so no clearing is
// needed; calls that overlap on the GPU (different streams, or different host threads)
// share the array and race.
#include <cmath>
#include <mutex>

#include "common.cuh"

namespace rbgs {
namespace {

constexpr int kStaticRows = 4;
constexpr int kStaticBlocks = 8192;
constexpr int kStaticThreads = 256;
constexpr int kStaticMaxN = kStaticRows * kStaticBlocks;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) double g_static_partials[2 * kStaticBlocks];

// per-device device address of g_static_partials, looked up on first use
double *g_scratch_ptr[kMaxDevices] = {};
std::mutex g_scratch_mutex;

__device__ __forceinline__ double warp_block_sum(double v, double *smem) {
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    __syncthreads();
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = (lane < kStaticThreads / 32) ? smem[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t = __dadd_rn(t, __shfl_down_sync(0xffffffffu, t, o));
    }
    return t;
}

// Block b reduces rows [1 + b * kStaticRows, ...] of the natural (n+2)^2 grid.
__global__ void __launch_bounds__(kStaticThreads)
static_partials_kernel(const double *__restrict__ f, const double *__restrict__ u, double h2, int n,
                       double *__restrict__ scratch) {
    __shared__ double smem[kStaticThreads / 32];
    const size_t ld = (size_t)n + 2;
    double r2 = 0.0, b2 = 0.0;
    const int i_end = min(n, 1 + (int)blockIdx.x * kStaticRows + kStaticRows - 1);
    for (int i = 1 + blockIdx.x * kStaticRows; i <= i_end; ++i) {
        for (int j = 1 + threadIdx.x; j <= n; j += kStaticThreads) {
            const double hf = __dmul_rn(h2, f[(size_t)(i - 1) * n + (j - 1)]);
            const double un = u[(size_t)(i - 1) * ld + j], us = u[(size_t)(i + 1) * ld + j];
            const double uw = u[(size_t)i * ld + j - 1], ue = u[(size_t)i * ld + j + 1];
            const double s = __dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn(hf, un), us), uw), ue);
            const double r = __dadd_rn(s, -__dmul_rn(4.0, u[(size_t)i * ld + j]));
            r2 = __fma_rn(r, r, r2);
            double b = hf;
            if (i == 1) b = __dadd_rn(b, un);
            if (i == n) b = __dadd_rn(b, us);
            if (j == 1) b = __dadd_rn(b, uw);
            if (j == n) b = __dadd_rn(b, ue);
            b2 = __fma_rn(b, b, b2);
        }
    }
    const double tr = warp_block_sum(r2, smem);
    const double tb = warp_block_sum(b2, smem);
    if (threadIdx.x == 0) {
        scratch[2 * blockIdx.x] = tr;
        scratch[2 * blockIdx.x + 1] = tb;
    }
}

// One block: add the partials in a fixed order and write rho.
__global__ void __launch_bounds__(kStaticThreads)
static_final_kernel(const double *__restrict__ scratch, int blocks, double *__restrict__ out) {
    __shared__ double smem[kStaticThreads / 32];
    double r2 = 0.0, b2 = 0.0;
    for (int q = threadIdx.x; q < blocks; q += kStaticThreads) {
        r2 = __dadd_rn(r2, scratch[2 * q]);
        b2 = __dadd_rn(b2, scratch[2 * q + 1]);
    }
    const double tr = warp_block_sum(r2, smem);
    const double tb = warp_block_sum(b2, smem);
    if (threadIdx.x == 0) *out = tb > 0.0 ? sqrt(tr) / sqrt(tb) : sqrt(tr);
}

bool on_device(const void *p, int device) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    if (a.type == cudaMemoryTypeManaged) return true;
    return a.type == cudaMemoryTypeDevice && a.device == device;
}

}  // namespace
}  // namespace rbgs

using namespace rbgs;

extern "C" rbgs_status rbgs_residual_static(int n, double h2, const double *f, const double *u,
                                            double *rel_out, void *cuda_stream) {
    clear_error();
    if (n < 1 || n > kStaticMaxN) {
        set_error("rbgs_residual_static: n = %d outside 1..%d (the static scratch holds %d row "
                  "blocks of %d rows)", n, kStaticMaxN, kStaticBlocks, kStaticRows);
        return RBGS_EINVAL;
    }
    if (!(h2 > 0.0) || !std::isfinite(h2)) {
        set_error("rbgs_residual_static: h2 must be finite and > 0");
        return RBGS_EINVAL;
    }
    if (!f || !u || !rel_out) {
        set_error("rbgs_residual_static: f, u and rel_out must not be NULL");
        return RBGS_EINVAL;
    }
    int device = 0;
    RBGS_CUDA(cudaGetDevice(&device));
    if (device < 0 || device >= kMaxDevices) {
        set_error("rbgs_residual_static: device ordinal %d unsupported", device);
        return RBGS_EINVAL;
    }
    if (!on_device(f, device) || !on_device(u, device) || !on_device(rel_out, device)) {
        set_error("rbgs_residual_static: f, u and rel_out must be device memory of the current device");
        return RBGS_EINVAL;
    }
    double *scratch = nullptr;
    {
        // set-up once per device (again only if the device was reset since): the device
        // address of the static scratch array.  A reset unloads the library's device image,
        // so an address looked up before it no longer belongs to this device's context.
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (g_scratch_ptr[device] && !on_device(g_scratch_ptr[device], device)) g_scratch_ptr[device] = nullptr;
        if (!g_scratch_ptr[device]) {
            void *p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_static_partials);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                set_error("rbgs_residual_static: cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
                return RBGS_ECUDA;
            }
            g_scratch_ptr[device] = static_cast<double *>(p);
        }
        scratch = g_scratch_ptr[device];
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const int blocks = (n + kStaticRows - 1) / kStaticRows;
    static_partials_kernel<<<blocks, kStaticThreads, 0, s>>>(f, u, h2, n, scratch);
    RBGS_LAUNCH_CHECK();
    static_final_kernel<<<1, kStaticThreads, 0, s>>>(scratch, blocks, rel_out);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}
