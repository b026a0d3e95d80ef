// Grid operations of the learned initial guess (C ABI in include/rbgs_unet.h): the
// transfinite interpolation of the Dirichlet ring that the network's correction is added
// to, the network's four input channels, the training target, the guess itself, and the
// transfer between a fine grid and the training grid (block averages of f down, bilinear
// interpolation up).  One thread per output point; everything stays on the device.
//
// Transfinite (Coons) interpolation of the ring of an (n+2)^2 grid, g = n+2, at point
// (i, j) with x = i/(g-1), y = j/(g-1): the blended sum of the four edge interpolants minus
// the bilinear corner term,
//   (1-x) N_j + x S_j + (1-y) W_i + y E_i
//     - ((1-x)(1-y) c00 + (1-x) y c01 + x (1-y) c10 + x y c11),
// N = row 0, S = row g-1, W = column 0, E = column g-1, c the corners.  It reproduces ring
// data that is linear in x and in y exactly, and the ring itself.
#include <cuda_runtime.h>

#include "../../include/rbgs_unet.h"
#include "common.cuh"

namespace rbgs {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ double coons(const double *__restrict__ u, int g, int i, int j) {
    const double x = (double)i / (double)(g - 1), y = (double)j / (double)(g - 1);
    const double c00 = u[0], c01 = u[g - 1], c10 = u[(size_t)(g - 1) * g], c11 = u[(size_t)(g - 1) * g + g - 1];
    const double edges = (1.0 - x) * u[j] + x * u[(size_t)(g - 1) * g + j] + (1.0 - y) * u[(size_t)i * g] +
                         y * u[(size_t)i * g + g - 1];
    const double corners = (1.0 - x) * (1.0 - y) * c00 + (1.0 - x) * y * c01 + x * (1.0 - y) * c10 + x * y * c11;
    return edges - corners;
}

__global__ void blend_kernel(const double *__restrict__ u, int g, double *__restrict__ out) {
    const long total = (long)g * g;
    for (long q = (long)blockIdx.x * kT + threadIdx.x; q < total; q += (long)gridDim.x * kT)
        out[q] = coons(u, g, (int)(q / g), (int)(q % g));
}

// x[(i*size + j)*4 + c]: f (interior), ring mask, ring values, the blend; zero off the grid
__global__ void input_kernel(const double *__restrict__ f, const double *__restrict__ u, int n, int size,
                             float *__restrict__ x) {
    const int g = n + 2;
    const long total = (long)size * size;
    for (long q = (long)blockIdx.x * kT + threadIdx.x; q < total; q += (long)gridDim.x * kT) {
        const int i = (int)(q / size), j = (int)(q % size);
        float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
        if (i < g && j < g) {
            const bool ring = i == 0 || j == 0 || i == g - 1 || j == g - 1;
            v.x = ring ? 0.f : (float)f[(size_t)(i - 1) * n + (j - 1)];
            v.y = ring ? 1.f : 0.f;
            v.z = ring ? (float)u[(size_t)i * g + j] : 0.f;
            v.w = (float)coons(u, g, i, j);
        }
        reinterpret_cast<float4 *>(x)[q] = v;
    }
}

// t = sol - blend on the (n+2)^2 grid, 0 elsewhere on the size^2 grid
__global__ void target_kernel(const double *__restrict__ sol, const double *__restrict__ u, int n, int size,
                              float *__restrict__ t) {
    const int g = n + 2;
    const long total = (long)size * size;
    for (long q = (long)blockIdx.x * kT + threadIdx.x; q < total; q += (long)gridDim.x * kT) {
        const int i = (int)(q / size), j = (int)(q % size);
        t[q] = (i < g && j < g) ? (float)(sol[(size_t)i * g + j] - coons(u, g, i, j)) : 0.f;
    }
}

// u0: the ring of u; interior = blend + pred (pred on the size^2 grid)
__global__ void assemble_kernel(const double *__restrict__ u, const float *__restrict__ pred, int n, int size,
                                double *__restrict__ u0) {
    const int g = n + 2;
    const long total = (long)g * g;
    for (long q = (long)blockIdx.x * kT + threadIdx.x; q < total; q += (long)gridDim.x * kT) {
        const int i = (int)(q / g), j = (int)(q % g);
        const bool ring = i == 0 || j == 0 || i == g - 1 || j == g - 1;
        u0[q] = ring ? u[q] : coons(u, g, i, j) + (double)pred[(size_t)i * size + j];
    }
}

// coarse node c = (ci, cj), 1 <= ci, cj <= nc, sits on fine node (ci r, cj r): fc = the mean
// of f over the (2r-1)^2 fine nodes around it (all interior); uc = u sampled at stride r
__global__ void coarsen_kernel(const double *__restrict__ f, const double *__restrict__ u, int n, int nc, int r,
                               double *__restrict__ fc, double *__restrict__ uc) {
    const int gc = nc + 2, g = n + 2;
    const long total = (long)gc * gc;
    const double inv = 1.0 / (double)((2 * r - 1) * (2 * r - 1));
    for (long q = (long)blockIdx.x * kT + threadIdx.x; q < total; q += (long)gridDim.x * kT) {
        const int ci = (int)(q / gc), cj = (int)(q % gc);
        uc[q] = u[(size_t)(ci * r) * g + cj * r];
        if (ci >= 1 && ci <= nc && cj >= 1 && cj <= nc) {
            double s = 0.0;
            for (int di = -(r - 1); di <= r - 1; ++di)
                for (int dj = -(r - 1); dj <= r - 1; ++dj)
                    s += f[(size_t)(ci * r + di - 1) * n + (cj * r + dj - 1)];
            fc[(size_t)(ci - 1) * nc + (cj - 1)] = s * inv;
        }
    }
}

// fine interior point (i, j) at coarse coordinates (i/r, j/r): bilinear interpolation of
// uc between the surrounding coarse nodes; the fine ring is kept
__global__ void refine_kernel(const double *__restrict__ uc, int nc, const double *__restrict__ u, int n, int r,
                              double *__restrict__ u0) {
    const int gc = nc + 2, g = n + 2;
    const long total = (long)g * g;
    for (long q = (long)blockIdx.x * kT + threadIdx.x; q < total; q += (long)gridDim.x * kT) {
        const int i = (int)(q / g), j = (int)(q % g);
        if (i == 0 || j == 0 || i == g - 1 || j == g - 1) {
            u0[q] = u[q];
            continue;
        }
        const int i0 = i / r, j0 = j / r;
        const int i1 = i0 + 1 < gc ? i0 + 1 : i0, j1 = j0 + 1 < gc ? j0 + 1 : j0;
        const double a = (double)(i - i0 * r) / r, b = (double)(j - j0 * r) / r;
        const double v00 = uc[(size_t)i0 * gc + j0], v01 = uc[(size_t)i0 * gc + j1];
        const double v10 = uc[(size_t)i1 * gc + j0], v11 = uc[(size_t)i1 * gc + j1];
        u0[q] = (1.0 - a) * ((1.0 - b) * v00 + b * v01) + a * ((1.0 - b) * v10 + b * v11);
    }
}

int blocks_for(long total) {
    const long b = (total + kT - 1) / kT;
    return (int)(b < 4096 ? (b < 1 ? 1 : b) : 4096);
}

bool on_dev(const void *p) {
    cudaPointerAttributes a;
    if (!p || cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

}  // namespace
}  // namespace rbgs

using namespace rbgs;

extern "C" {

rbgs_status rbgs_guess_blend(const double *u_ring, int n, double *out, void *cuda_stream) {
    clear_error();
    if (n < 1 || !on_dev(u_ring) || !on_dev(out)) {
        set_error("rbgs_guess_blend: n >= 1 and device buffers required");
        return RBGS_EINVAL;
    }
    const int g = n + 2;
    blend_kernel<<<blocks_for((long)g * g), kT, 0, (cudaStream_t)cuda_stream>>>(u_ring, g, out);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

rbgs_status rbgs_guess_input(const double *f, const double *u_ring, int n, int size, float *x, void *cuda_stream) {
    clear_error();
    if (n < 1 || size < n + 2 || size % 8 || !on_dev(f) || !on_dev(u_ring) || !on_dev(x)) {
        set_error("rbgs_guess_input: n >= 1, size >= n + 2 and a multiple of 8, device buffers required");
        return RBGS_EINVAL;
    }
    input_kernel<<<blocks_for((long)size * size), kT, 0, (cudaStream_t)cuda_stream>>>(f, u_ring, n, size, x);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

rbgs_status rbgs_guess_target(const double *sol, const double *u_ring, int n, int size, float *t,
                              void *cuda_stream) {
    clear_error();
    if (n < 1 || size < n + 2 || !on_dev(sol) || !on_dev(u_ring) || !on_dev(t)) {
        set_error("rbgs_guess_target: n >= 1, size >= n + 2, device buffers required");
        return RBGS_EINVAL;
    }
    target_kernel<<<blocks_for((long)size * size), kT, 0, (cudaStream_t)cuda_stream>>>(sol, u_ring, n, size, t);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

rbgs_status rbgs_guess_assemble(const double *u_ring, const float *pred, int n, int size, double *u0,
                                void *cuda_stream) {
    clear_error();
    if (n < 1 || size < n + 2 || !on_dev(u_ring) || !on_dev(pred) || !on_dev(u0)) {
        set_error("rbgs_guess_assemble: n >= 1, size >= n + 2, device buffers required");
        return RBGS_EINVAL;
    }
    const int g = n + 2;
    assemble_kernel<<<blocks_for((long)g * g), kT, 0, (cudaStream_t)cuda_stream>>>(u_ring, pred, n, size, u0);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

rbgs_status rbgs_guess_coarsen(const double *f, const double *u_ring, int n, int nc, double *fc, double *uc_ring,
                               void *cuda_stream) {
    clear_error();
    if (n < 1 || nc < 1 || (n + 1) % (nc + 1) || !on_dev(f) || !on_dev(u_ring) || !on_dev(fc) || !on_dev(uc_ring)) {
        set_error("rbgs_guess_coarsen: (n + 1) must be a multiple of (nc + 1), device buffers required");
        return RBGS_EINVAL;
    }
    const int r = (n + 1) / (nc + 1);
    coarsen_kernel<<<blocks_for((long)(nc + 2) * (nc + 2)), kT, 0, (cudaStream_t)cuda_stream>>>(f, u_ring, n, nc, r,
                                                                                               fc, uc_ring);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

rbgs_status rbgs_guess_refine(const double *uc, int nc, const double *u_ring, int n, double *u0, void *cuda_stream) {
    clear_error();
    if (n < 1 || nc < 1 || (n + 1) % (nc + 1) || !on_dev(uc) || !on_dev(u_ring) || !on_dev(u0)) {
        set_error("rbgs_guess_refine: (n + 1) must be a multiple of (nc + 1), device buffers required");
        return RBGS_EINVAL;
    }
    const int r = (n + 1) / (nc + 1);
    const int g = n + 2;
    refine_kernel<<<blocks_for((long)g * g), kT, 0, (cudaStream_t)cuda_stream>>>(uc, nc, u_ring, n, r, u0);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

}  // extern "C"
