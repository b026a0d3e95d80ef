// The 3D variant of the red-black scheme (the paper's outlook, Section 5): the 7-point
// update u = (h2 f + N + S + W + E + D + U) / 6 over one colour at a time, i + j + k even
// (red) then odd (black).  C ABI in include/rbgs3d.h.
//
// Layout: the 2D colour split applied along k.  For every grid line (i, j), 0 <= i, j <=
// N+1, colour c holds a row of W values; element m is the point k = 2m + ((i + j + c) & 1).
// A point and its four neighbours in i and j share m (those lines have the other parity);
// its k-neighbours sit in the other colour's row of the same line, at m-1/m or m/m+1.
// W = ceil((N+2)/2) rounded up to 32 values (256-byte rows).
//
// Half-sweep: the colour's (line, pair of values) items are flattened over a grid-stride
// loop; each item reads the other colour's rows of lines (i-1, j), (i+1, j), (i, j-1),
// (i, j+1) and (i, j) and h2 f, and writes its own two values.  Neighbouring lines in j are
// adjacent in the item order and lines i+-1 one plane apart, so the re-reads of the other
// colour hit the caches (a plane of a 511^3 grid is 1.2 MB).  Arithmetic: six adds in the
// order above, each one correctly rounded fused multiply-add by a run-time 1.0, and one
// correctly rounded division by 6 (div6 in div6.cuh: three FP64 operations instead of the
// division sequence): the same bits as the plain sequential loop.
#include <algorithm>
#include <cmath>
#include <new>

#include "../../include/rbgs3d.h"
#include "common.cuh"
#include "div6.cuh"
#include "fp64.cuh"
#include "sweep_impl.cuh"

struct rbgs3d_ctx {
    int n, W;
    double h2;
    cudaStream_t stream;
    double *u[2], *hf[2];
    double *staging;   // natural-layout (N+2)^3 buffer for host inputs and outputs
    double *partials;  // [2 * kBlocks3]: per block sum rt^2, sum hb^2
    double *dsum;      // [2]
    double *hsum;      // pinned mirror of dsum
    double den2;
};

namespace rbgs {
namespace {

constexpr int kThreads3 = 256;
constexpr int kBlocks3 = 4096;  // grid-stride blocks of the reductions (<= partial slots)
constexpr int kMaxN3 = 2048;

__host__ __device__ inline int width3(int n) {
    const int w = (n + 3) / 2;
    return (w + 31) / 32 * 32;
}

// natural (N+2)^3 u -> colour rows; f (N^3) -> h2 f colour rows, zero off the interior.
__global__ void pack3_kernel(const double *__restrict__ u_nat, const double *__restrict__ f_nat, double h2,
                             double *__restrict__ u0, double *__restrict__ u1, double *__restrict__ hf0,
                             double *__restrict__ hf1, int n, int W) {
    const int L = n + 2;
    const size_t total = (size_t)L * L * W;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(q % W);
        const size_t line = q / W;
        const int i = (int)(line / L), j = (int)(line % L);
        const int k = 2 * m;
        // colour of (i, j, k) is (i + j) & 1; (i, j, k + 1) the other one
        const double a = k <= n + 1 ? u_nat[line * L + k] : 0.0;
        const double b = k + 1 <= n + 1 ? u_nat[line * L + k + 1] : 0.0;
        const bool in_line = i >= 1 && i <= n && j >= 1 && j <= n;
        const size_t fl = ((size_t)(i - 1) * n + (j - 1)) * n;
        const double fa = (in_line && k >= 1 && k <= n) ? __dmul_rn(h2, f_nat[fl + k - 1]) : 0.0;
        const double fb = (in_line && k + 1 <= n) ? __dmul_rn(h2, f_nat[fl + k]) : 0.0;
        const bool even = ((i + j) & 1) == 0;
        (even ? u0 : u1)[q] = a;
        (even ? u1 : u0)[q] = b;
        (even ? hf0 : hf1)[q] = fa;
        (even ? hf1 : hf0)[q] = fb;
    }
}

__global__ void unpack3_kernel(const double *__restrict__ u0, const double *__restrict__ u1,
                               double *__restrict__ u_nat, int n, int W) {
    const int L = n + 2;
    const size_t total = (size_t)L * L * W;
    for (size_t q = (size_t)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (size_t)gridDim.x * blockDim.x) {
        const int m = (int)(q % W);
        const size_t line = q / W;
        const int i = (int)(line / L), j = (int)(line % L);
        const int k = 2 * m;
        const bool even = ((i + j) & 1) == 0;
        if (k <= n + 1) u_nat[line * L + k] = (even ? u0 : u1)[q];
        if (k + 1 <= n + 1) u_nat[line * L + k + 1] = (even ? u1 : u0)[q];
    }
}

// One half-sweep of colour C: items (interior line, pair of values) over the grid.
template <int C>
__global__ void __launch_bounds__(kThreads3)
half_sweep3_kernel(double *__restrict__ self, const double *__restrict__ other, const double *__restrict__ hf,
                   int n, int W, int kact, double one) {
    const int L = n + 2;
    const int npairs = kact / 2;
    const size_t items = (size_t)n * n * npairs;
    for (size_t q = (size_t)blockIdx.x * kThreads3 + threadIdx.x; q < items; q += (size_t)gridDim.x * kThreads3) {
        const int pr = (int)(q % npairs);
        const size_t ln = q / npairs;
        const int i = 1 + (int)(ln / n), j = 1 + (int)(ln % n);
        const int m0 = 2 * pr;
        const int p = (i + j + C) & 1;  // k offset of this colour on line (i, j)
        const size_t row = ((size_t)i * L + j) * W;
        const size_t plane = (size_t)L * W;
        const double2 vn = __ldg(reinterpret_cast<const double2 *>(other + row - plane + m0));
        const double2 vs = __ldg(reinterpret_cast<const double2 *>(other + row + plane + m0));
        const double2 vw = __ldg(reinterpret_cast<const double2 *>(other + row - W + m0));
        const double2 ve = __ldg(reinterpret_cast<const double2 *>(other + row + W + m0));
        const double2 vm = __ldg(reinterpret_cast<const double2 *>(other + row + m0));
        const double2 f2 = __ldg(reinterpret_cast<const double2 *>(hf + row + m0));
        double d0, u0, d1, u1;  // k-1 and k+1 neighbours of the two values
        if (p == 0) {  // value v at k = 2(m0+v): k-1 at m0+v-1, k+1 at m0+v
            d0 = m0 > 0 ? __ldg(other + row + m0 - 1) : 0.0;
            u0 = vm.x;
            d1 = vm.x;
            u1 = vm.y;
        } else {  // at 2(m0+v)+1: k-1 at m0+v, k+1 at m0+v+1
            d0 = vm.x;
            u0 = vm.y;
            d1 = vm.y;
            u1 = m0 + 2 < W ? __ldg(other + row + m0 + 2) : 0.0;
        }
        double s0 = add_fma(f2.x, vn.x, one);
        s0 = add_fma(s0, vs.x, one);
        s0 = add_fma(s0, vw.x, one);
        s0 = add_fma(s0, ve.x, one);
        s0 = add_fma(s0, d0, one);
        s0 = add_fma(s0, u0, one);
        double s1 = add_fma(f2.y, vn.y, one);
        s1 = add_fma(s1, vs.y, one);
        s1 = add_fma(s1, vw.y, one);
        s1 = add_fma(s1, ve.y, one);
        s1 = add_fma(s1, d1, one);
        s1 = add_fma(s1, u1, one);
        const int k0 = 2 * m0 + p;  // natural k of value 0; value 1 at k0 + 2
        if (k0 >= 1 && k0 <= n) self[row + m0] = div6(s0);
        if (k0 + 2 <= n) self[row + m0 + 1] = div6(s1);
    }
}

// Per-block sums of rt^2 and (h^2 b)^2 over every interior point (both colours).
__global__ void __launch_bounds__(kThreads3)
residual3_kernel(const double *__restrict__ u0, const double *__restrict__ u1, const double *__restrict__ hf0,
                 const double *__restrict__ hf1, int n, int W, double *__restrict__ partials) {
    __shared__ double smem[kThreads3 / 32];
    const int L = n + 2;
    const size_t total = (size_t)n * n * n;
    double r2 = 0.0, b2 = 0.0;
    auto at = [&](int i, int j, int k) {
        const bool even = ((i + j + k) & 1) == 0;
        return (even ? u0 : u1)[((size_t)i * L + j) * W + (k >> 1)];
    };
    for (size_t q = (size_t)blockIdx.x * kThreads3 + threadIdx.x; q < total; q += (size_t)gridDim.x * kThreads3) {
        const int k = 1 + (int)(q % n);
        const size_t t = q / n;
        const int j = 1 + (int)(t % n), i = 1 + (int)(t / n);
        const bool even = ((i + j + k) & 1) == 0;
        const double hf = (even ? hf0 : hf1)[((size_t)i * L + j) * W + (k >> 1)];
        const double vn = at(i - 1, j, k), vs = at(i + 1, j, k), vw = at(i, j - 1, k), ve = at(i, j + 1, k);
        const double vd = at(i, j, k - 1), vu = at(i, j, k + 1);
        double s = __dadd_rn(hf, vn);
        s = __dadd_rn(s, vs);
        s = __dadd_rn(s, vw);
        s = __dadd_rn(s, ve);
        s = __dadd_rn(s, vd);
        s = __dadd_rn(s, vu);
        const double r = __dadd_rn(s, -__dmul_rn(6.0, at(i, j, k)));
        r2 = __fma_rn(r, r, r2);
        double b = hf;
        if (i == 1) b = __dadd_rn(b, vn);
        if (i == n) b = __dadd_rn(b, vs);
        if (j == 1) b = __dadd_rn(b, vw);
        if (j == n) b = __dadd_rn(b, ve);
        if (k == 1) b = __dadd_rn(b, vd);
        if (k == n) b = __dadd_rn(b, vu);
        b2 = __fma_rn(b, b, b2);
    }
    const double tr = block_sum<kThreads3>(r2, smem);
    __syncthreads();
    const double tb = block_sum<kThreads3>(b2, smem);
    if (threadIdx.x == 0) {
        partials[2 * blockIdx.x] = tr;
        partials[2 * blockIdx.x + 1] = tb;
    }
}

// The blocks' partial sums added in a fixed order (one block).
__global__ void __launch_bounds__(kThreads3)
final3_kernel(const double *__restrict__ partials, int blocks, double *__restrict__ out) {
    __shared__ double smem[kThreads3 / 32];
    double r2 = 0.0, b2 = 0.0;
    for (int q = threadIdx.x; q < blocks; q += kThreads3) {
        r2 = __dadd_rn(r2, partials[2 * q]);
        b2 = __dadd_rn(b2, partials[2 * q + 1]);
    }
    const double tr = block_sum<kThreads3>(r2, smem);
    __syncthreads();
    const double tb = block_sum<kThreads3>(b2, smem);
    if (threadIdx.x == 0) {
        out[0] = tr;
        out[1] = tb;
    }
}

int grid_for(size_t items) {
    static const int cap = [] {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            sms = 152;
        }
        return 8 * sms;
    }();
    const size_t want = (items + kThreads3 - 1) / kThreads3;
    return (int)(want < (size_t)cap ? (want < 1 ? 1 : want) : cap);
}

bool dev_ptr(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

void free3(rbgs3d_ctx *c) {
    if (!c) return;
    for (int q = 0; q < 2; ++q) {
        cudaFree(c->u[q]);
        cudaFree(c->hf[q]);
    }
    cudaFree(c->staging);
    cudaFree(c->partials);
    cudaFree(c->dsum);
    if (c->hsum) cudaFreeHost(c->hsum);
    delete c;
}

// rho's two sums into dsum (stream-ordered)
rbgs_status enqueue_residual3(rbgs3d_ctx *c) {
    const size_t total = (size_t)c->n * c->n * c->n;
    const int blocks = std::min(grid_for(total), kBlocks3);
    residual3_kernel<<<blocks, kThreads3, 0, c->stream>>>(c->u[0], c->u[1], c->hf[0], c->hf[1], c->n, c->W,
                                                          c->partials);
    RBGS_LAUNCH_CHECK();
    final3_kernel<<<1, kThreads3, 0, c->stream>>>(c->partials, blocks, c->dsum);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

}  // namespace
}  // namespace rbgs

using namespace rbgs;

extern "C" {

rbgs_status rbgs3d_create(int n, double h2, const double *f, const double *u_init, void *cuda_stream,
                          rbgs3d_t *out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return RBGS_EINVAL; }
    *out = nullptr;
    if (n < 1 || n > kMaxN3) { set_error("n = %d outside 1..%d", n, kMaxN3); return RBGS_EINVAL; }
    if (!(h2 > 0.0) || !std::isfinite(h2)) { set_error("h2 must be finite and > 0"); return RBGS_EINVAL; }
    if (!f || !u_init) { set_error("f and u_init must not be NULL"); return RBGS_EINVAL; }
    rbgs3d_ctx *c = new (std::nothrow) rbgs3d_ctx();
    if (!c) { set_error("out of host memory"); return RBGS_ENOMEM; }
    c->n = n;
    c->W = width3(n);
    c->h2 = h2;
    c->stream = (cudaStream_t)cuda_stream;
    const size_t L = (size_t)n + 2;
    const size_t colour = L * L * c->W * sizeof(double);
    bool ok = true;
    for (int q = 0; q < 2 && ok; ++q)
        ok = cudaMalloc(&c->u[q], colour) == cudaSuccess && cudaMalloc(&c->hf[q], colour) == cudaSuccess;
    ok = ok && cudaMalloc(&c->partials, 2 * kBlocks3 * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMalloc(&c->dsum, 2 * sizeof(double)) == cudaSuccess;
    ok = ok && cudaMallocHost(&c->hsum, 2 * sizeof(double)) == cudaSuccess;
    const bool host_in = !dev_ptr(f) || !dev_ptr(u_init);
    ok = ok && (!host_in || cudaMalloc(&c->staging, L * L * L * sizeof(double)) == cudaSuccess);
    if (!ok) {
        cudaGetLastError();
        free3(c);
        set_error("allocation of the 3D solver's %zu-byte buffers failed", 4 * colour);
        return RBGS_ENOMEM;
    }
    // inputs in host memory go through device copies (u_init through the staging buffer,
    // f through a temporary one); device inputs are read in place
    const double *fv = f, *uv = u_init;
    const size_t nf = (size_t)n * n * n, nu = L * L * L;
    double *fstage = nullptr;
    if (host_in) {
        if (!dev_ptr(f)) {
            if (cudaMalloc(&fstage, nf * sizeof(double)) != cudaSuccess) {
                cudaGetLastError();
                free3(c);
                set_error("allocation of the 3D solver's f staging failed");
                return RBGS_ENOMEM;
            }
            if (cudaMemcpyAsync(fstage, f, nf * sizeof(double), cudaMemcpyDefault, c->stream) != cudaSuccess) {
                cudaGetLastError();
                cudaFree(fstage);
                free3(c);
                set_error("copy of f failed");
                return RBGS_ECUDA;
            }
            fv = fstage;
        }
        if (!dev_ptr(u_init)) {
            if (cudaMemcpyAsync(c->staging, u_init, nu * sizeof(double), cudaMemcpyDefault, c->stream) != cudaSuccess) {
                cudaGetLastError();
                cudaFree(fstage);
                free3(c);
                set_error("copy of u_init failed");
                return RBGS_ECUDA;
            }
            uv = c->staging;
        }
    }
    pack3_kernel<<<grid_for(L * L * c->W), kThreads3, 0, c->stream>>>(uv, fv, h2, c->u[0], c->u[1], c->hf[0],
                                                                      c->hf[1], n, c->W);
    rbgs_status st = cudaGetLastError() == cudaSuccess ? RBGS_OK : RBGS_ECUDA;
    if (st == RBGS_OK) st = enqueue_residual3(c);
    if (st == RBGS_OK && (cudaMemcpyAsync(c->hsum, c->dsum, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream) !=
                              cudaSuccess ||
                          cudaStreamSynchronize(c->stream) != cudaSuccess)) {
        cudaGetLastError();
        st = RBGS_ECUDA;
    }
    cudaFree(fstage);
    if (st != RBGS_OK) {
        set_error("3D set-up failed");
        free3(c);
        return st;
    }
    c->den2 = c->hsum[1];
    *out = c;
    return RBGS_OK;
}

rbgs_status rbgs3d_sweep(rbgs3d_t c, long nsweeps) {
    clear_error();
    if (!c) { set_error("ctx is NULL"); return RBGS_EINVAL; }
    if (nsweeps < 0) { set_error("nsweeps < 0"); return RBGS_EINVAL; }
    const int kact = active_width(c->n);
    const size_t items = (size_t)c->n * c->n * (kact / 2);
    const int grid = grid_for(items);
    for (long it = 0; it < nsweeps; ++it) {
        half_sweep3_kernel<0><<<grid, kThreads3, 0, c->stream>>>(c->u[0], c->u[1], c->hf[0], c->n, c->W, kact, 1.0);
        RBGS_LAUNCH_CHECK();
        half_sweep3_kernel<1><<<grid, kThreads3, 0, c->stream>>>(c->u[1], c->u[0], c->hf[1], c->n, c->W, kact, 1.0);
        RBGS_LAUNCH_CHECK();
    }
    return RBGS_OK;
}

rbgs_status rbgs3d_residual(rbgs3d_t c, double *rel) {
    clear_error();
    if (!c || !rel) { set_error("ctx and rel must not be NULL"); return RBGS_EINVAL; }
    rbgs_status st = enqueue_residual3(c);
    if (st != RBGS_OK) return st;
    RBGS_CUDA(cudaMemcpyAsync(c->hsum, c->dsum, 2 * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    RBGS_CUDA(cudaStreamSynchronize(c->stream));
    const double r2 = c->hsum[0];
    *rel = c->den2 > 0.0 ? std::sqrt(r2) / std::sqrt(c->den2) : std::sqrt(r2);
    if (!std::isfinite(*rel)) {
        set_error("residual is not finite");
        return RBGS_ENONFINITE;
    }
    return RBGS_OK;
}

rbgs_status rbgs3d_get_solution(rbgs3d_t c, double *u_out) {
    clear_error();
    if (!c || !u_out) { set_error("ctx and u_out must not be NULL"); return RBGS_EINVAL; }
    const size_t L = (size_t)c->n + 2, nu = L * L * L;
    const int grid = grid_for(L * L * c->W);
    if (dev_ptr(u_out)) {
        unpack3_kernel<<<grid, kThreads3, 0, c->stream>>>(c->u[0], c->u[1], u_out, c->n, c->W);
        RBGS_LAUNCH_CHECK();
        return RBGS_OK;
    }
    if (!c->staging && cudaMalloc(&c->staging, nu * sizeof(double)) != cudaSuccess) {
        cudaGetLastError();
        set_error("staging allocation failed");
        return RBGS_ENOMEM;
    }
    unpack3_kernel<<<grid, kThreads3, 0, c->stream>>>(c->u[0], c->u[1], c->staging, c->n, c->W);
    RBGS_LAUNCH_CHECK();
    RBGS_CUDA(cudaMemcpyAsync(u_out, c->staging, nu * sizeof(double), cudaMemcpyDefault, c->stream));
    RBGS_CUDA(cudaStreamSynchronize(c->stream));
    return RBGS_OK;
}

void rbgs3d_destroy(rbgs3d_t c) {
    if (!c) return;
    cudaStreamSynchronize(c->stream);
    free3(c);
}

}  // extern "C"
