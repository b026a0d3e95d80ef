// FP32 half-sweeps (the inner solver of the mixed-precision refinement): the update of
// Eq. (1) in binary32, (((hf + N) + S) + W) + E, times 0.25, each step correctly
// rounded with no contraction, so the result equals a sequential binary32 C loop in
// that order.  Same strip walk as the FP64 kernel; a thread owns 4 values (one 16-byte
// vector) per row.  12 bytes of DRAM traffic per update.
#include "common.cuh"
#include "sweep_impl.cuh"

namespace rbgs {
namespace {

constexpr int kPts32 = 4;

__device__ __forceinline__ float update_f32(float hf, float vn, float vs, float vw, float ve) {
    float s = __fadd_rn(hf, vn);
    s = __fadd_rn(s, vs);
    s = __fadd_rn(s, vw);
    s = __fadd_rn(s, ve);
    return __fmul_rn(s, 0.25f);
}

__device__ __forceinline__ void load4(float *v, const float *p, bool act) {
    const float4 t = act ? __ldg(reinterpret_cast<const float4 *>(p)) : make_float4(0.f, 0.f, 0.f, 0.f);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}

template <int COLOUR>
__global__ void __launch_bounds__(kSweepThreads)
half_sweep_f32(float *__restrict__ self, const float *__restrict__ other, const float *__restrict__ hf,
               int n, int W, int kact, int rows_per_block) {
    const int lane = threadIdx.x & 31;
    const int k0 = kPts32 * (blockIdx.x * kSweepThreads + threadIdx.x);
    const bool act = k0 < kact;  // k0 + 3 < W: W is a multiple of 64
    const int i0 = 1 + blockIdx.y * rows_per_block;
    if (i0 > n) return;
    const int i1 = min(n, i0 + rows_per_block - 1);
    float up[4], mid[4], dn[4], f[4], r[4];
    load4(up, other + (size_t)(i0 - 1) * W + k0, act);
    load4(mid, other + (size_t)i0 * W + k0, act);
    for (int i = i0; i <= i1; ++i) {
        const size_t row = (size_t)i * W;
        load4(dn, other + row + W + k0, act);
        load4(f, hf + row + k0, act);
        const int p = (i + COLOUR) & 1;
        if (p == 0) {
            float prev = __shfl_up_sync(0xffffffffu, mid[3], 1);
            if (lane == 0) prev = (act && k0 > 0) ? __ldg(other + row + k0 - 1) : 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) r[q] = update_f32(f[q], up[q], dn[q], q ? mid[q - 1] : prev, mid[q]);
        } else {
            float next = __shfl_down_sync(0xffffffffu, mid[0], 1);
            if (lane == 31) next = (k0 + 4 < kact) ? __ldg(other + row + k0 + 4) : 0.f;
#pragma unroll
            for (int q = 0; q < 4; ++q) r[q] = update_f32(f[q], up[q], dn[q], mid[q], q < 3 ? mid[q + 1] : next);
        }
        const int j0 = 2 * k0 + p;
        float *sp = self + row + k0;
        if (act && j0 >= 1 && j0 + 6 <= n) {
            *reinterpret_cast<float4 *>(sp) = make_float4(r[0], r[1], r[2], r[3]);
        } else if (act) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (j0 + 2 * q >= 1 && j0 + 2 * q <= n) sp[q] = r[q];
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            up[q] = mid[q];
            mid[q] = dn[q];
        }
    }
}

}  // namespace

rbgs_status launch_sweeps_f32(const ColourField<float> &fld, long nsweeps, cudaStream_t s) {
    const int n = fld.n;
    // active values per row, rounded up to whole 4-value vectors
    const int kact = (((n + 3) / 2) + 3) & ~3;
    // strips of up to 32 rows, fewer when that leaves fewer than ~600 blocks
    const int gx = (kact + kPts32 * kSweepThreads - 1) / (kPts32 * kSweepThreads);
    long r = (long)n * gx / 600;
    const int rows = (int)(r < 1 ? 1 : (r > 32 ? 32 : r));
    dim3 grid(gx, (n + rows - 1) / rows);
    for (long it = 0; it < nsweeps; ++it) {
        half_sweep_f32<0><<<grid, kSweepThreads, 0, s>>>(fld.u[0], fld.u[1], fld.hf[0], n, fld.W, kact, rows);
        RBGS_LAUNCH_CHECK();
        half_sweep_f32<1><<<grid, kSweepThreads, 0, s>>>(fld.u[1], fld.u[0], fld.hf[1], n, fld.W, kact, rows);
        RBGS_LAUNCH_CHECK();
    }
    return RBGS_OK;
}

}  // namespace rbgs
