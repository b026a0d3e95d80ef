// Device helpers shared by the sweep and residual kernels.
#pragma once

#include "common.cuh"
#include "fp64.cuh"

namespace rbgs {

constexpr int kSweepThreads = 128;

// Number of colour values per row that can hold a grid point: ceil((n+2)/2), rounded up
// to even so that threads always own whole 16-byte pairs.  Always <= W.
__host__ __device__ inline int active_width(int n) { return (((n + 3) / 2) + 1) & ~1; }

__device__ __forceinline__ double2 ldg2(const double *p) {
    return __ldg(reinterpret_cast<const double2 *>(p));
}

__device__ __forceinline__ void stg2(double *p, double2 v) {
    *reinterpret_cast<double2 *>(p) = v;
}

template <int PTS>
__device__ __forceinline__ void load_row(double *v, const double *p, bool act) {
#pragma unroll
    for (int q = 0; q < PTS; q += 2) {
        const double2 t = act ? ldg2(p + q) : make_double2(0.0, 0.0);
        v[q] = t.x;
        v[q + 1] = t.y;
    }
}

template <int PTS>
__device__ __forceinline__ void store_row(double *p, const double *v) {
#pragma unroll
    for (int q = 0; q < PTS; q += 2) stg2(p + q, make_double2(v[q], v[q + 1]));
}

// (((hf + vn) + vs) + vw) + ve, times 0.25.  Bit q of m routes add q to the integer pipe;
// m is a compile-time constant at every call site (unrolled loops), so the branches fold.
template <bool PLAIN>
__device__ __forceinline__ double update_f64(int m, double hf, double vn, double vs, double vw,
                                             double ve, double one) {
    if (PLAIN) {
        double s = __dadd_rn(hf, vn);
        s = __dadd_rn(s, vs);
        s = __dadd_rn(s, vw);
        s = __dadd_rn(s, ve);
        return __dmul_rn(s, 0.25);
    }
    double s = (m & 1) ? add_int(hf, vn) : add_fma(hf, vn, one);
    s = (m & 2) ? add_int(s, vs) : add_fma(s, vs, one);
    s = (m & 4) ? add_int(s, vw) : add_fma(s, vw, one);
    s = (m & 8) ? add_int(s, ve) : add_fma(s, ve, one);
    return quarter(s);
}

// Block-wide sum of one double per thread, fixed reduction tree (deterministic).
template <int THREADS>
__device__ __forceinline__ double block_sum(double v, double *smem) {
    for (int o = 16; o > 0; o >>= 1) v = __dadd_rn(v, __shfl_down_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = (lane < THREADS / 32) ? smem[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t = __dadd_rn(t, __shfl_down_sync(0xffffffffu, t, o));
    }
    return t;  // valid in thread 0
}

// Block-wide max of one non-negative double per thread.
template <int THREADS>
__device__ __forceinline__ double block_max(double v, double *smem) {
    for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) smem[warp] = v;
    __syncthreads();
    double t = 0.0;
    if (warp == 0) {
        t = (lane < THREADS / 32) ? smem[lane] : 0.0;
        for (int o = 16; o > 0; o >>= 1) t = fmax(t, __shfl_down_sync(0xffffffffu, t, o));
    }
    return t;  // valid in thread 0
}

bool emulation_split_supported(int m);

}  // namespace rbgs
