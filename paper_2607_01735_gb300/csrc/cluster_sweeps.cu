// The FP32 inner sweeps of the mixed-precision refinement on small grids, in one launch of
// one thread-block cluster.
//
// On a small grid a half-sweep is less work than a kernel launch, and one launch per colour
// (even from a CUDA graph) spends its time between kernels.  Here the CS blocks of one
// cluster (one block per SM) hold the correction d in their shared memory, a band of rows
// each, both colours.  Every half-sweep (Section 2, Eq. (1), on the defect equation) updates
// the band's values of one colour from the other colour's rows: the band's own rows from
// local shared memory, the row just above and just below the band from the neighbouring
// blocks' shared memory (distributed shared memory).  The cluster's hardware barrier
// separates the colours, as the phases of Algorithm 1.  The right-hand side (the scaled
// defect) stays in global memory and is read through L1.  d is read from global memory once
// at the start and written back once at the end.
//
// The update is the one of the FP32 half-sweep kernels, (((r + N) + S) + W) + E times 0.25,
// each step correctly rounded in binary32, so the result is bit-identical to them.  All
// blocks of the cluster run the same number of barriers (the sweep count is a kernel
// argument); nothing waits on anything outside the cluster.
#include <atomic>

#include "common.cuh"

namespace rbgs {
namespace {

constexpr int kCThreads = 1024;

struct CArgs {
    float *d0, *d1;          // correction, colour-split (row pitch W), ring rows and columns 0
    const float *r0, *r1;    // scaled defect
    int n, W, hb;            // interior size, row pitch, rows per block
    int nsweeps;
};

__device__ __forceinline__ int cta_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}

__device__ __forceinline__ void cluster_sync() {
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// float at shared-memory address `local` in block `rank` of the cluster
__device__ __forceinline__ float ld_remote(const float *local, int rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    float v;
    asm volatile("ld.shared::cluster.f32 %0, [%1];" : "=f"(v) : "r"(ra) : "memory");
    return v;
}

__device__ __forceinline__ float upd(float hf, float vn, float vs, float vw, float ve) {
    float s = __fadd_rn(hf, vn);
    s = __fadd_rn(s, vs);
    s = __fadd_rn(s, vw);
    s = __fadd_rn(s, ve);
    return __fmul_rn(s, 0.25f);
}

// Shared memory of a block: sm[c * hb * W + rl * W + k] holds d of colour c, band row rl.
template <int CS>
__global__ void __launch_bounds__(kCThreads) cluster_sweeps_f32(const CArgs a) {
    extern __shared__ __align__(16) float sm[];
    const int rank = cta_rank();
    const int n = a.n, W = a.W, hb = a.hb;
    const int r0 = 1 + rank * hb;                       // first grid row of the band
    const int nr = max(0, min(n + 1, r0 + hb) - r0);    // rows in the band
    const int kact = (n + 3) / 2;                       // values of a colour row that can be interior
    const size_t plane = (size_t)hb * W;  // one colour's band

    for (int q = threadIdx.x; q < 2 * nr * W; q += kCThreads) {
        const int c = q / (nr * W), rem = q % (nr * W);
        sm[c * plane + rem] = (c ? a.d1 : a.d0)[(size_t)(r0 + rem / W) * W + rem % W];
    }
    cluster_sync();

    const int items = nr * kact;
    for (int s = 0; s < a.nsweeps; ++s) {
        for (int c = 0; c < 2; ++c) {
            const float *oth = sm + (c ^ 1) * plane;
            float *self = sm + c * plane;
            const float *rr = c ? a.r1 : a.r0;
            for (int q = threadIdx.x; q < items; q += kCThreads) {
                const int rl = q / kact, k = q % kact;
                const int i = r0 + rl;
                const int p = (i + c) & 1;
                const int j = 2 * k + p;  // natural column
                if (j < 1 || j > n) continue;
                const float *mid = oth + (size_t)rl * W;
                // north / south: this band, a neighbouring block's band, or the ring (0)
                float vn, vs;
                if (rl > 0) vn = mid[k - W];
                else if (i == 1) vn = 0.f;
                else vn = ld_remote(oth + (size_t)(hb - 1) * W + k, rank - 1);
                if (rl + 1 < nr) vs = mid[k + W];
                else if (i == n) vs = 0.f;
                else vs = ld_remote(oth + k, rank + 1);
                const float vw = p ? mid[k] : (k > 0 ? mid[k - 1] : 0.f);
                const float ve = p ? mid[k + 1] : mid[k];
                self[(size_t)rl * W + k] = upd(__ldg(rr + (size_t)i * W + k), vn, vs, vw, ve);
            }
            cluster_sync();
        }
    }

    for (int q = threadIdx.x; q < 2 * nr * W; q += kCThreads) {
        const int c = q / (nr * W), rem = q % (nr * W);
        (c ? a.d1 : a.d0)[(size_t)(r0 + rem / W) * W + rem % W] = sm[c * plane + rem];
    }
}

// Shared memory per block for an n^2 grid (row pitch W) spread over a cluster of CS blocks.
template <int CS>
size_t cluster_smem(int n, int W) {
    const int hb = (n + CS - 1) / CS;
    return (size_t)2 * hb * W * sizeof(float);
}

template <int CS>
bool cluster_fits(int n, int W) {
    // largest shared memory per block known to fit, per CS (the occupancy query runs once
    // per new maximum)
    static std::atomic<int> checked_bytes{-1};
    const size_t smem = cluster_smem<CS>(n, W);
    if (smem > 200 * 1024) return false;
    const int known = checked_bytes.load();
    if (known >= 0 && smem <= (size_t)known) return true;
    if (cudaFuncSetAttribute(cluster_sweeps_f32<CS>, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) !=
            cudaSuccess ||
        (CS > 8 && cudaFuncSetAttribute(cluster_sweeps_f32<CS>, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) !=
                       cudaSuccess)) {
        cudaGetLastError();
        return false;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS);
    cfg.blockDim = dim3(kCThreads);
    cfg.dynamicSmemBytes = smem;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, cluster_sweeps_f32<CS>, &cfg) != cudaSuccess || nc < 1) {
        cudaGetLastError();
        return false;
    }
    int prev = checked_bytes.load();
    while ((int)smem > prev && !checked_bytes.compare_exchange_weak(prev, (int)smem)) {
    }
    return true;
}

template <int CS>
rbgs_status launch_cs(ColourField<float> &fld, long nsweeps, cudaStream_t s) {
    CArgs a;
    a.d0 = fld.u[0], a.d1 = fld.u[1], a.r0 = fld.hf[0], a.r1 = fld.hf[1];
    a.n = fld.n, a.W = fld.W, a.hb = (fld.n + CS - 1) / CS;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS);
    cfg.blockDim = dim3(kCThreads);
    cfg.dynamicSmemBytes = cluster_smem<CS>(fld.n, fld.W);
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    while (nsweeps > 0) {
        a.nsweeps = (int)(nsweeps < (1L << 30) ? nsweeps : (1L << 30));
        RBGS_CUDA(cudaLaunchKernelEx(&cfg, cluster_sweeps_f32<CS>, a));
        nsweeps -= a.nsweeps;
    }
    return RBGS_OK;
}

}  // namespace

bool cluster_sweeps_f32_fit(int n, int W) { return cluster_fits<16>(n, W) || cluster_fits<8>(n, W); }

rbgs_status launch_cluster_sweeps_f32(ColourField<float> &fld, long nsweeps, cudaStream_t s) {
    if (nsweeps <= 0) return RBGS_OK;
    if (cluster_fits<16>(fld.n, fld.W)) return launch_cs<16>(fld, nsweeps, s);
    if (cluster_fits<8>(fld.n, fld.W)) return launch_cs<8>(fld, nsweeps, s);
    set_error("FP32 cluster sweeps: %d^2 does not fit one cluster", fld.n);
    return RBGS_EINVAL;
}

}  // namespace rbgs
