// Many FP64 sweeps in one cooperative launch.
//
// Every block of a grid that is resident as a whole (cooperative launch) walks all the
// sweeps: it updates its share of one colour (Section 2, Eq. (1)), then waits at a grid
// barrier until every block has finished that colour, then does the same for the other
// colour: the two phases of Algorithm 1, with the barrier between them.  On small grids
// this removes the gaps between one-per-colour launches.  On large ones it measured faster
// than the row-strip kernel too (GB300, 16383^2: 1.15x): no launch ramps or tails, and the
// flattened items spread every half-sweep evenly over all resident warps, so the FP64 pipe
// stays busier.
//
// Work: the colour's (row, group of 4 values) items from 768^2 on, (row, pair) items below,
// flattened and strided over all threads of the grid, so each thread carries 4 (or 2)
// independent update chains per item (pairs measured 4.5% slower at 16383^2, groups of 8
// 5.6% slower: fewer resident warps); a warp runs an iteration while any of its lanes has an
// item (the FP64 x0.25 votes across the warp).  Loads of the other colour go through L2 (`ld.global.cg`): it
// was written by other blocks during this launch.  The update is the library's, step by
// step correctly rounded, so the iterate is bit-identical to one launch per colour.
//
// Grid barrier (grid_barrier.cuh): one counter per launch, zeroed before it.  Every wait is
// bounded: after kBarrierPolls polls, or as soon as another block has given up, the block
// records a status and leaves; the host reports it as RBGS_ETIMEOUT at its next
// synchronising call.
#include "common.cuh"
#include "fp64.cuh"
#include "grid_barrier.cuh"
#include "sweep_impl.cuh"

namespace rbgs {
namespace {

constexpr int kPThreads = 256;
constexpr uint32_t kBarrierPolls = 1u << 22;
constexpr long long kMaxSweepsPerLaunch = 1LL << 20;

template <typename T>
struct PArgs {
    T *u0, *u1;
    const T *hf0, *hf1;
    int n, W, kact;
    long long nsweeps;
    unsigned *counter;
    int *status;
    double one;  // 1.0 at run time: the FP64 adds stay fused multiply-adds with it
};

__device__ __forceinline__ double upd(double hf, double vn, double vs, double vw, double ve, double one) {
    return update_f64<false>(0, hf, vn, vs, vw, ve, one);
}

template <typename V>
__device__ __forceinline__ V make_vec() {
    V v;
    v.x = 0, v.y = 0;
    return v;
}

template <typename T>
struct Pair;
template <>
struct Pair<double> {
    using V = double2;
};

// One half-sweep of colour C by the whole grid: items of 2 * NP values (NP pairs) each.
template <typename T, int C, int NP>
__device__ __forceinline__ void half_sweep(const PArgs<T> &a) {
    using V = typename Pair<T>::V;
    constexpr int NV = 2 * NP;
    T *self = C ? a.u1 : a.u0;
    const T *other = C ? a.u0 : a.u1;
    const T *hf = C ? a.hf1 : a.hf0;
    const int n = a.n, W = a.W, kact = a.kact, ngroups = (kact + NV - 1) / NV;
    const int items = n * ngroups;
    const int gt = blockIdx.x * kPThreads + threadIdx.x;
    const int stride = gridDim.x * kPThreads;
    for (int base = 0; base < items; base += stride) {
        if (base + (gt & ~31) >= items) break;  // warp-uniform: no item left for this warp
        const int q = base + gt;
        const bool act = q < items;
        const int qq = act ? q : 0;
        const int i = 1 + qq / ngroups, k0 = NV * (qq % ngroups);
        const int p = (i + C) & 1;
        const size_t row = (size_t)i * W;
        T m[NV], uv[NV], dv[NV], fv[NV];
#pragma unroll
        for (int h = 0; h < NP; ++h) {
            // pairs past the active width (the row's last group only) are not read
            V u_ = make_vec<V>(), m_ = make_vec<V>(), d_ = make_vec<V>(), f_ = make_vec<V>();
            if (h == 0 || k0 + 2 * h < kact) {
                u_ = __ldcg(reinterpret_cast<const V *>(other + row - W + k0 + 2 * h));
                m_ = __ldcg(reinterpret_cast<const V *>(other + row + k0 + 2 * h));
                d_ = __ldcg(reinterpret_cast<const V *>(other + row + W + k0 + 2 * h));
                f_ = __ldg(reinterpret_cast<const V *>(hf + row + k0 + 2 * h));
            }
            m[2 * h] = m_.x, m[2 * h + 1] = m_.y;
            uv[2 * h] = u_.x, uv[2 * h + 1] = u_.y;
            dv[2 * h] = d_.x, dv[2 * h + 1] = d_.y;
            fv[2 * h] = f_.x, fv[2 * h + 1] = f_.y;
        }
        T wv[NV], ev[NV];
        if (p == 0) {  // value v at natural column 2(k0+v): west/east at k0+v-1, k0+v
            wv[0] = k0 > 0 ? __ldcg(other + row + k0 - 1) : T(0);
#pragma unroll
            for (int v = 1; v < NV; ++v) wv[v] = m[v - 1];
#pragma unroll
            for (int v = 0; v < NV; ++v) ev[v] = m[v];
        } else {  // at 2(k0+v)+1: west/east at k0+v, k0+v+1
#pragma unroll
            for (int v = 0; v < NV; ++v) wv[v] = m[v];
#pragma unroll
            for (int v = 0; v + 1 < NV; ++v) ev[v] = k0 + v + 1 < kact ? m[v + 1] : T(0);
            ev[NV - 1] = k0 + NV < kact ? __ldcg(other + row + k0 + NV) : T(0);
        }
        const int j0 = 2 * k0 + p;
#pragma unroll
        for (int v = 0; v < NV; ++v) {
            const T r = upd(fv[v], uv[v], dv[v], wv[v], ev[v], a.one);
            if (act && j0 + 2 * v >= 1 && j0 + 2 * v <= n) self[row + k0 + v] = r;
        }
    }
}

template <typename T, int NP>
__global__ void __launch_bounds__(kPThreads) persistent_sweeps(const PArgs<T> a) {
    unsigned target = 0;
    for (long long s = 0; s < a.nsweeps; ++s) {
        half_sweep<T, 0, NP>(a);
        target += gridDim.x;
        if (!grid_barrier(a.counter, target, a.status, kBarrierPolls)) return;
        half_sweep<T, 1, NP>(a);
        target += gridDim.x;
        if (!grid_barrier(a.counter, target, a.status, kBarrierPolls)) return;
    }
}

// Blocks the grid needs (at most what can be resident at once).
template <typename T, int NP>
int persistent_grid(int n) {
    // resident blocks of the whole GPU, per template instance (initialised once, thread-safely;
    // 0 when the query fails)
    static const long cap = [] {
        int dev = 0, sms = 0, per_sm = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_sweeps<T, NP>, kPThreads, 0) !=
                cudaSuccess) {
            cudaGetLastError();
            return 0L;
        }
        return (long)per_sm * sms;
    }();
    const long items = (long)n * ((active_width(n) + 2 * NP - 1) / (2 * NP));
    const long want = (items + kPThreads - 1) / kPThreads;
    return (int)(want < cap ? want : cap);
}

template <typename T, int NP>
rbgs_status launch_np(ColourField<T> &fld, long nsweeps, unsigned *counter, int *status, cudaStream_t s) {
    const int grid = persistent_grid<T, NP>(fld.n);
    if (grid < 1) {
        set_error("persistent sweeps: no resident block fits");
        return RBGS_ECUDA;
    }
    PArgs<T> a;
    a.u0 = fld.u[0], a.u1 = fld.u[1], a.hf0 = fld.hf[0], a.hf1 = fld.hf[1];
    a.n = fld.n, a.W = fld.W, a.kact = active_width(fld.n);
    a.counter = counter, a.status = status, a.one = 1.0;
    // the barrier counter reaches 2 * grid per sweep and must stay below 2^32
    long long per_launch = (0xffffffffLL / (2LL * grid)) - 1;
    if (per_launch > kMaxSweepsPerLaunch) per_launch = kMaxSweepsPerLaunch;
    while (nsweeps > 0) {
        a.nsweeps = nsweeps < per_launch ? nsweeps : per_launch;
        RBGS_CUDA(cudaMemsetAsync(counter, 0, sizeof(unsigned), s));
        void *args[] = {&a};
        RBGS_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(persistent_sweeps<T, NP>), dim3(grid),
                                              dim3(kPThreads), args, 0, s));
        nsweeps -= a.nsweeps;
    }
    return RBGS_OK;
}

}  // namespace

// Items of 4 values where the grid gives every resident thread several of them; pairs on
// smaller grids, where more threads are worth more than longer items (GB300: quads 1.046x
// at 16383^2 and 1.03x at 1023^2 over pairs, but slower at 511^2).
template <typename T>
rbgs_status launch_persistent_sweeps(ColourField<T> &fld, long nsweeps, unsigned *counter, int *status,
                                     cudaStream_t s) {
    if (nsweeps <= 0) return RBGS_OK;
    return fld.n >= 768 ? launch_np<T, 2>(fld, nsweeps, counter, status, s)
                        : launch_np<T, 1>(fld, nsweeps, counter, status, s);
}

template rbgs_status launch_persistent_sweeps<double>(ColourField<double> &, long, unsigned *, int *,
                                                      cudaStream_t);

}  // namespace rbgs
