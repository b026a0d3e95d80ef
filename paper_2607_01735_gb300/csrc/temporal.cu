// Temporally blocked sweeps: K red+black sweeps per pass over HBM, without a grid-wide
// barrier between colours.
//
// Each thread block owns an output tile of TR rows x TK colour values (both colours).
// It loads the tile plus a halo of H = 2K rows above and below and HK >= K+1 colour
// values left and right (the region a point's value after K sweeps depends on: one grid
// step per half-sweep) for u_red, u_black, hf_red, hf_black with four 2D TMA copies
// (cp.async.bulk.tensor, completion on one mbarrier; zero fill outside the grid).  It
// then runs the 2K half-sweeps of Eq. (1) (red first, Algorithms 1-2's order) in shared
// memory.  After half-sweep s only points at distance > s from the loaded region's edge
// are final, so step s updates exactly those (the halo is recomputed by every tile that
// needs it).  The inner TR x TK values of both colours are then written to the partner
// buffer (ping-pong: no tile reads what another tile writes in the same launch).
//
// The arithmetic per update is the same sequence of correctly rounded operations as the
// one-launch-per-colour kernels, so K sweeps here equal K sweeps there bit for bit.
//
// DRAM traffic per pass: (4 loaded arrays x halo factor + 2 stored) per tile, i.e.
// roughly (4 (TR+2H)(TK+2HK)/(TR TK) + 2) * sizeof(T) / (2K) bytes per update.
#include <cstring>

#include <cudaTypedefs.h>

#include "common.cuh"
#include "sweep_impl.cuh"
#include "tma.cuh"

namespace rbgs {

cudaError_t encode_tensor_map_2d(CUtensorMap *map, const void *base, int elem_bytes, uint64_t width,
                                 uint64_t rows, uint64_t pitch_elems, uint32_t box_w, uint32_t box_h) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        cudaError_t e = cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000,
                                                         cudaEnableDefault, &q);
        if (e != cudaSuccess) return e;
        if (q != cudaDriverEntryPointSuccess || !fn) return cudaErrorNotSupported;
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    cuuint64_t dims[2] = {width, rows};
    cuuint64_t strides[1] = {pitch_elems * (cuuint64_t)elem_bytes};
    cuuint32_t box[2] = {box_w, box_h};
    cuuint32_t estr[2] = {1, 1};
    CUtensorMapDataType dt = elem_bytes == 8 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT64 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32;
    CUresult r = encode(map, dt, 2, const_cast<void *>(base), dims, strides, box, estr,
                        CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                        CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

namespace {

constexpr int kTThreads = 512;
constexpr uint32_t kWaitPolls = 1u << 22;  // bounded mbarrier wait

template <typename T, int K, int TR, int TK>
struct TCfg {
    static constexpr int H = 2 * K;                       // halo rows
    static constexpr int ALIGN = 16 / (int)sizeof(T);     // TMA x alignment in elements
    static constexpr int HK = ((K + 1) + ALIGN - 1) / ALIGN * ALIGN;
    static constexpr int ER = TR + 2 * H;
    static constexpr int EK = TK + 2 * HK;
    static constexpr int ARR = ER * EK;
    static constexpr size_t ARR_BYTES = ((size_t)ARR * sizeof(T) + 127) / 128 * 128;
    static constexpr size_t SMEM = 4 * ARR_BYTES + 128 + 128;  // arrays, barrier, alignment slack
    static_assert(EK <= 256 && ER <= 256, "TMA box dimensions are limited to 256");
    static_assert((EK * sizeof(T)) % 16 == 0, "TMA box rows must be whole 16-byte units");
    static_assert(TK % ALIGN == 0, "tile x origin must be 16-byte aligned");
    static_assert(EK % 32 == 0 && kTThreads % EK == 0, "row bands must hold whole warps");
};

template <typename T>
struct Update;

template <>
struct Update<double> {
    __device__ static __forceinline__ double go(double hf, double vn, double vs, double vw, double ve,
                                                double one) {
        return update_f64<false>(0, hf, vn, vs, vw, ve, one);
    }
};

template <>
struct Update<float> {
    __device__ static __forceinline__ float go(float hf, float vn, float vs, float vw, float ve, double) {
        float s = __fadd_rn(hf, vn);
        s = __fadd_rn(s, vs);
        s = __fadd_rn(s, vw);
        s = __fadd_rn(s, ve);
        return __fmul_rn(s, 0.25f);
    }
};

// One row of a half-step: the row's colour offset P (0 or 1) is a compile-time constant,
// so the neighbour that comes from the adjacent lane, and its direction, are fixed.
template <typename T, int EK, int P>
__device__ __forceinline__ void tile_row(T *__restrict__ self, const T *__restrict__ oth, const T *__restrict__ fh,
                                         int ii, int kk, int lane, T &up, T &mid, bool store, double one) {
    const T dn = oth[(ii + 1) * EK + kk];
    const T fv = fh[ii * EK + kk];
    T vw, ve;
    if (P == 0) {  // west neighbour is column kk-1 (the previous lane)
        T prev = __shfl_up_sync(0xffffffffu, mid, 1);
        if (lane == 0) prev = kk > 0 ? oth[ii * EK + kk - 1] : T(0);
        vw = prev;
        ve = mid;
    } else {       // east neighbour is column kk+1 (the next lane)
        T next = __shfl_down_sync(0xffffffffu, mid, 1);
        if (lane == 31) next = kk + 1 < EK ? oth[ii * EK + kk + 1] : T(0);
        vw = mid;
        ve = next;
    }
    const T r = Update<T>::go(fv, up, dn, vw, ve, one);
    if (store) self[ii * EK + kk] = r;
    up = mid;
    mid = dn;
}

// Rows [r0, r1) of one half-step, in pairs (the colour offset alternates row by row).
template <typename T, int EK, int P0>
__device__ __forceinline__ void tile_rows(T *__restrict__ self, const T *__restrict__ oth, const T *__restrict__ fh,
                                          int r0, int r1, int row_lo, int row_hi, int kk, int lane, bool col0,
                                          bool col1, double one) {
    T up = oth[(r0 - 1) * EK + kk];
    T mid = oth[r0 * EK + kk];
    for (int ii = r0; ii < r1; ii += 2) {
        tile_row<T, EK, P0>(self, oth, fh, ii, kk, lane, up, mid,
                            (P0 == 0 ? col0 : col1) && ii >= row_lo && ii < row_hi, one);
        if (ii + 1 < r1)
            tile_row<T, EK, 1 - P0>(self, oth, fh, ii + 1, kk, lane, up, mid,
                                    (P0 == 0 ? col1 : col0) && ii + 1 >= row_lo && ii + 1 < row_hi, one);
    }
}

template <typename T, int K, int TR, int TK>
__global__ void __launch_bounds__(kTThreads, 2)
temporal_tile(const __grid_constant__ CUtensorMap mu0, const __grid_constant__ CUtensorMap mu1,
              const __grid_constant__ CUtensorMap mf0, const __grid_constant__ CUtensorMap mf1,
              T *__restrict__ out0, T *__restrict__ out1, int n, int W, double one, int *status) {
    using C = TCfg<T, K, TR, TK>;
    extern __shared__ unsigned char smem_raw[];
    unsigned char *base = reinterpret_cast<unsigned char *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~static_cast<uintptr_t>(127));
    T *const su0 = reinterpret_cast<T *>(base);
    T *const su1 = reinterpret_cast<T *>(base + C::ARR_BYTES);
    T *const sf0 = reinterpret_cast<T *>(base + 2 * C::ARR_BYTES);
    T *const sf1 = reinterpret_cast<T *>(base + 3 * C::ARR_BYTES);
    uint64_t *bar = reinterpret_cast<uint64_t *>(base + 4 * C::ARR_BYTES);

    const int r0 = blockIdx.y * TR, k0 = blockIdx.x * TK;
    const int R0 = r0 - C::H, E0 = k0 - C::HK;
    if (threadIdx.x == 0) {
        prefetch_tensormap(&mu0);
        prefetch_tensormap(&mu1);
        prefetch_tensormap(&mf0);
        prefetch_tensormap(&mf1);
        mbar_init(bar, 1);
        fence_barrier_init();
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        mbar_arrive_expect_tx(bar, (uint32_t)(4 * C::ARR * sizeof(T)));
        tma_load_2d(su0, &mu0, E0, R0, bar);
        tma_load_2d(su1, &mu1, E0, R0, bar);
        tma_load_2d(sf0, &mf0, E0, R0, bar);
        tma_load_2d(sf1, &mf1, E0, R0, bar);
    }
    if (!mbar_wait_bounded(bar, 0, kWaitPolls)) {
        if (threadIdx.x == 0) atomicOr(status, 1);
        mbar_wait_bounded(bar, 0, kWaitPolls);  // let copies in flight land before exiting
        return;
    }

    // Half-step s of colour c updates the points at distance > s from the region's edge.
    // Thread t owns column kk = t % EK and marches down band t / EK of the step's rows,
    // keeping the other colour's rows i-1, i, i+1 in registers; the horizontal neighbour
    // that is not in its own column comes from the adjacent lane (or, at a warp edge,
    // from shared memory).  Bands hold whole warps, so every loop below is warp-uniform.
    constexpr int BANDS = kTThreads / C::EK;
    const int kk = threadIdx.x % C::EK, band = threadIdx.x / C::EK;
    const int lane = threadIdx.x & 31;
    // interior rows of the grid, as smem row indices: R0 + ii in [1, n]
    const int row_lo = 1 - R0, row_hi = n + 1 - R0;
    for (int s = 0; s < 2 * K; ++s) {
        const int c = s & 1;
        T *const self = c ? su1 : su0;
        const T *const oth = c ? su0 : su1;
        const T *const fh = c ? sf1 : sf0;
        const int rlo = s + 1, rhi = C::ER - 1 - s;  // rows [rlo, rhi)
        const int per = (rhi - rlo + BANDS - 1) / BANDS;
        const int r0 = rlo + band * per;
        const int r1 = r0 + per < rhi ? r0 + per : rhi;
        // column kk holds natural column jj = 2 kk + p of the region (p = the row's offset);
        // it is updated at this step if it lies at distance > s from the region's edge and
        // inside the grid
        bool colok[2];
#pragma unroll
        for (int p = 0; p < 2; ++p) {
            const int jj = 2 * kk + p, j = 2 * E0 + jj;
            colok[p] = jj >= s + 1 && (2 * C::EK - 1 - jj) >= s + 1 && j >= 1 && j <= n;
        }
        if (r0 < r1) {
            if (((R0 + r0 + c) & 1) == 0)
                tile_rows<T, C::EK, 0>(self, oth, fh, r0, r1, row_lo, row_hi, kk, lane, colok[0], colok[1], one);
            else
                tile_rows<T, C::EK, 1>(self, oth, fh, r0, r1, row_lo, row_hi, kk, lane, colok[0], colok[1], one);
        }
        __syncthreads();
    }

    // inner tile of both colours -> partner buffers (rows 0..n+1, values 0..W-1)
    if (kk >= C::HK && kk < C::HK + TK) {
        const int k = k0 + kk - C::HK;
        for (int rr = band; rr < TR; rr += BANDS) {
            const int i = r0 + rr;
            if (i <= n + 1 && k < W) {
                const int sidx = (rr + C::H) * C::EK + kk;
                out0[(size_t)i * W + k] = su0[sidx];
                out1[(size_t)i * W + k] = su1[sidx];
            }
        }
    }
}

template <typename T, int K, int TR, int TK>
rbgs_status run_pass(ColourField<T> &fld, int *status, cudaStream_t s) {
    using C = TCfg<T, K, TR, TK>;
    const int n = fld.n;
    if (!fld.maps_ready || fld.maps_box_w != C::EK || fld.maps_box_h != C::ER) {
        const T *ptrs[6] = {fld.u[0], fld.u[1], fld.alt[0], fld.alt[1], fld.hf[0], fld.hf[1]};
        for (int q = 0; q < 6; ++q) {
            cudaError_t e = encode_tensor_map_2d(&fld.maps[q], ptrs[q], (int)sizeof(T), (uint64_t)fld.W,
                                                 (uint64_t)(n + 2), (uint64_t)fld.W, C::EK, C::ER);
            if (e != cudaSuccess) {
                set_error("tensor map encoding failed: %s", cudaGetErrorString(e));
                return RBGS_ECUDA;
            }
        }
        fld.maps_ready = true;
        fld.maps_box_w = C::EK;
        fld.maps_box_h = C::ER;
    }
    // set once per template instance, thread-safely; a failure is reported on every call
    static const cudaError_t attr = cudaFuncSetAttribute(temporal_tile<T, K, TR, TK>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)C::SMEM);
    RBGS_CUDA(attr);
    const int kact = ((n + 3) / 2 + C::ALIGN - 1) / C::ALIGN * C::ALIGN;
    dim3 grid((kact + TK - 1) / TK, (n + 2 + TR - 1) / TR);
    temporal_tile<T, K, TR, TK><<<grid, kTThreads, C::SMEM, s>>>(fld.maps[0], fld.maps[1], fld.maps[4],
                                                                  fld.maps[5], fld.alt[0], fld.alt[1], n,
                                                                  fld.W, 1.0, status);
    RBGS_LAUNCH_CHECK();
    // the partner buffers now hold the iterate
    for (int q = 0; q < 2; ++q) {
        T *t = fld.u[q];
        fld.u[q] = fld.alt[q];
        fld.alt[q] = t;
        CUtensorMap m;
        std::memcpy(&m, &fld.maps[q], sizeof(m));
        std::memcpy(&fld.maps[q], &fld.maps[2 + q], sizeof(m));
        std::memcpy(&fld.maps[2 + q], &m, sizeof(m));
    }
    return RBGS_OK;
}

}  // namespace

template <>
rbgs_status launch_temporal_pass<double>(ColourField<double> &fld, int k, int *status, cudaStream_t s) {
    switch (k) {  // tiles of 32 rows x (64 - 2 HK) values: EK = 64 = one quarter of the block
    case 1: return run_pass<double, 1, 32, 60>(fld, status, s);
    case 2: return run_pass<double, 2, 32, 56>(fld, status, s);
    case 4: return run_pass<double, 4, 32, 52>(fld, status, s);
    default: set_error("FP64 temporal depth must be 1, 2 or 4 (got %d)", k); return RBGS_EINVAL;
    }
}

template <>
rbgs_status launch_temporal_pass<float>(ColourField<float> &fld, int k, int *status, cudaStream_t s) {
    switch (k) {  // tiles of 32 rows x (128 - 2 HK) values: EK = 128 = half of the block
    case 2: return run_pass<float, 2, 32, 120>(fld, status, s);
    case 4: return run_pass<float, 4, 32, 112>(fld, status, s);
    case 8: return run_pass<float, 8, 32, 104>(fld, status, s);
    default: set_error("FP32 temporal depth must be 2, 4 or 8 (got %d)", k); return RBGS_EINVAL;
    }
}

// K sweeps per pass over the FP64 iterate; the remainder runs as one-launch-per-colour
// half-sweeps on the current buffers (identical arithmetic).
rbgs_status launch_temporal_sweeps(rbgs_ctx *c, long nsweeps, cudaStream_t s) {
    const int k = c->tblock_k;
    long passes = nsweeps / k;
    for (long q = 0; q < passes; ++q) {
        rbgs_status st = launch_temporal_pass<double>(c->f64, k, c->dstatus, s);
        if (st != RBGS_OK) return st;
    }
    return launch_sweeps_f64(c, nsweeps - passes * k, s);
}

}  // namespace rbgs
