// Many FP64 sweeps in one cooperative launch.
//
// Every block of a grid that is resident as a whole (cooperative launch) walks all the
// sweeps: it updates its share of one colour (Section 2, Eq. (1)), then waits at a grid
// barrier until every block has finished that colour, then does the same for the other
// colour: the two phases of Algorithm 1, with the barrier between them.  On small grids
// this removes the gaps between one-per-colour launches.  On large ones it measured faster
// than the row-strip kernel too (GB300, 16383^2: 1.10x): no launch ramps or tails, and the
// flattened items spread every half-sweep evenly over all resident warps, so the FP64 pipe
// stays busier.
//
// Work: the colour's (row, pair of values) items, flattened and strided over all threads of
// the grid; a warp runs an iteration while any of its lanes has an item (the FP64 x0.25
// votes across the warp).  Loads of the other colour go through L2 (`ld.global.cg`): it
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

template <typename T>
struct Pair;
template <>
struct Pair<double> {
    using V = double2;
};

// One half-sweep of colour C by the whole grid.
template <typename T, int C>
__device__ __forceinline__ void half_sweep(const PArgs<T> &a) {
    using V = typename Pair<T>::V;
    T *self = C ? a.u1 : a.u0;
    const T *other = C ? a.u0 : a.u1;
    const T *hf = C ? a.hf1 : a.hf0;
    const int n = a.n, W = a.W, kact = a.kact, npairs = kact / 2;
    const int items = n * npairs;
    const int gt = blockIdx.x * kPThreads + threadIdx.x;
    const int stride = gridDim.x * kPThreads;
    for (int base = 0; base < items; base += stride) {
        if (base + (gt & ~31) >= items) break;  // warp-uniform: no item left for this warp
        const int q = base + gt;
        const bool act = q < items;
        const int qq = act ? q : 0;
        const int i = 1 + qq / npairs, k0 = 2 * (qq % npairs);
        const int p = (i + C) & 1;
        const size_t row = (size_t)i * W;
        const V up = __ldcg(reinterpret_cast<const V *>(other + row - W + k0));
        const V mid = __ldcg(reinterpret_cast<const V *>(other + row + k0));
        const V dn = __ldcg(reinterpret_cast<const V *>(other + row + W + k0));
        const V f = __ldg(reinterpret_cast<const V *>(hf + row + k0));
        T w0, e0, w1, e1;
        if (p == 0) {  // values at natural columns 2k0, 2k0+2: west/east at k-1, k
            w0 = k0 > 0 ? __ldcg(other + row + k0 - 1) : T(0);
            e0 = mid.x, w1 = mid.x, e1 = mid.y;
        } else {  // at 2k0+1, 2k0+3: west/east at k, k+1
            w0 = mid.x, e0 = mid.y, w1 = mid.y;
            e1 = k0 + 2 < kact ? __ldcg(other + row + k0 + 2) : T(0);
        }
        const T r0 = upd(f.x, up.x, dn.x, w0, e0, a.one);
        const T r1 = upd(f.y, up.y, dn.y, w1, e1, a.one);
        const int j0 = 2 * k0 + p;
        if (act && j0 >= 1 && j0 <= n) self[row + k0] = r0;
        if (act && j0 + 2 <= n) self[row + k0 + 1] = r1;
    }
}

template <typename T>
__global__ void __launch_bounds__(kPThreads) persistent_sweeps(const PArgs<T> a) {
    unsigned target = 0;
    for (long long s = 0; s < a.nsweeps; ++s) {
        half_sweep<T, 0>(a);
        target += gridDim.x;
        if (!grid_barrier(a.counter, target, a.status, kBarrierPolls)) return;
        half_sweep<T, 1>(a);
        target += gridDim.x;
        if (!grid_barrier(a.counter, target, a.status, kBarrierPolls)) return;
    }
}

// Blocks the grid needs (at most what can be resident at once).
template <typename T>
int persistent_grid(int n) {
    static int per_sm = 0, sms = 0;
    if (!per_sm) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, persistent_sweeps<T>, kPThreads, 0) !=
                cudaSuccess) {
            cudaGetLastError();
            per_sm = 0;
            return 0;
        }
    }
    const long items = (long)n * (active_width(n) / 2);
    const long want = (items + kPThreads - 1) / kPThreads;
    const long cap = (long)per_sm * sms;
    return (int)(want < cap ? want : cap);
}

}  // namespace

template <typename T>
rbgs_status launch_persistent_sweeps(ColourField<T> &fld, long nsweeps, unsigned *counter, int *status,
                                     cudaStream_t s) {
    if (nsweeps <= 0) return RBGS_OK;
    const int grid = persistent_grid<T>(fld.n);
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
        RBGS_CUDA(cudaLaunchCooperativeKernel(reinterpret_cast<const void *>(persistent_sweeps<T>), dim3(grid),
                                              dim3(kPThreads), args, 0, s));
        nsweeps -= a.nsweeps;
    }
    return RBGS_OK;
}

template rbgs_status launch_persistent_sweeps<double>(ColourField<double> &, long, unsigned *, int *,
                                                      cudaStream_t);

}  // namespace rbgs
