// Fused FP64 half-sweeps (rbgs_opts.fma = 1): the update of Eq. (1) with one rounding.
//
// The bit-exact update rounds four times ((((h2f + N) + S) + W) + E, each add rounded) and
// on GB300 its four FP64 adds per point bound the sweep well below HBM.  The fused update
// sums the five terms exactly in 64-bit fixed point and rounds the quotient by 4 once
// (fixed64.cuh), with integer instructions only: no FP64 pipe, so the sweep can stream at
// the memory's rate.
//
// A block of at most kFusedChunk sweeps runs at one scale 2^e:
//   1. absmax_kernel: B = max |u| over both colours (ring and padding included, padding is
//      zero) into words[0] (an atomic max over the bit patterns of |u|: for non-negative
//      binary64 values the order of the bits is the order of the values, and Inf and NaN
//      patterns sort above every finite value); Q = max |h2 f| is kept in words[1] from
//      the problem's load;
//   2. prepare_kernel: e = scale_exponent(B, Q, sweeps of the block) into words[2] (or
//      kNoScale); h2 f of both colours converted once to the fixed-point grid (hq, int64),
//      so the sweeps read it as is;
//   3. the block's sweeps: per colour one launch of fused_half_sweep.
// A non-finite B or Q (a NaN or Inf in the iterate or in f) leaves no valid scale: the
// block's half-sweeps then write NaN to every point they update, so the next residual
// reports RBGS_ENONFINITE.
//
// Work decomposition of a half-sweep: that of the bit-exact strip kernel (sweep.cu).  A
// thread owns PTS neighbouring values of its colour row and walks down a strip of rows
// with the other colour's rows i-1, i, i+1 in registers, here already converted to the
// fixed-point grid, so each value of the other colour is converted once per strip; the
// west/east neighbour owned by the adjacent lane arrives by warp shuffle.  24 bytes of DRAM
// traffic per update, as the bit-exact kernel.
#include <cmath>

#include "common.cuh"
#include "fixed64.cuh"
#include "sweep_impl.cuh"

namespace rbgs {
namespace {

constexpr int kMaxThreads = 256;
constexpr unsigned long long kNoScale = 0x8000000000000000ull;  // words[2]: B or Q not finite

__device__ __forceinline__ unsigned long long warp_max_u64(unsigned long long v) {
    for (int o = 16; o > 0; o >>= 1) {
        const unsigned long long w = __shfl_down_sync(0xffffffffu, v, o);
        v = w > v ? w : v;
    }
    return v;
}

// max |a0[q]|, |a1[q]| over q < count (count even, both arrays 16-byte aligned), as the
// bit pattern of the non-negative value, atomically maxed into *word.
__global__ void __launch_bounds__(kMaxThreads)
absmax_kernel(const double *__restrict__ a0, const double *__restrict__ a1, size_t count,
              unsigned long long *__restrict__ word) {
    __shared__ unsigned long long smem[kMaxThreads / 32];
    const unsigned long long mask = 0x7FFFFFFFFFFFFFFFull;
    unsigned long long m = 0;
    const size_t pairs = count / 2;
    const double2 *p0 = reinterpret_cast<const double2 *>(a0), *p1 = reinterpret_cast<const double2 *>(a1);
    for (size_t q = (size_t)blockIdx.x * kMaxThreads + threadIdx.x; q < pairs; q += (size_t)gridDim.x * kMaxThreads) {
        const double2 x = __ldg(p0 + q), y = __ldg(p1 + q);
        const unsigned long long b0 = dbits(x.x) & mask, b1 = dbits(x.y) & mask;
        const unsigned long long b2 = dbits(y.x) & mask, b3 = dbits(y.y) & mask;
        const unsigned long long m01 = b0 > b1 ? b0 : b1, m23 = b2 > b3 ? b2 : b3;
        const unsigned long long mm = m01 > m23 ? m01 : m23;
        m = mm > m ? mm : m;
    }
    m = warp_max_u64(m);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) smem[warp] = m;
    __syncthreads();
    if (warp == 0) {
        m = lane < kMaxThreads / 32 ? smem[lane] : 0ull;
        m = warp_max_u64(m);
        if (lane == 0) atomicMax(word, m);
    }
}

// h2 f of both colours on the block's fixed-point grid (nothing to do without a scale).
__global__ void __launch_bounds__(kMaxThreads)
prepare_kernel(const double *__restrict__ hf0, const double *__restrict__ hf1, int64_t *__restrict__ hq0,
               int64_t *__restrict__ hq1, size_t count, unsigned long long *__restrict__ words,
               long long nsweeps) {
    int e = 0;
    const bool ok = scale_exponent(bitsd(words[0]), bitsd(words[1]), nsweeps, &e);
    if (blockIdx.x == 0 && threadIdx.x == 0) words[2] = ok ? (unsigned long long)(long long)e : kNoScale;
    if (!ok) return;
    for (size_t q = (size_t)blockIdx.x * kMaxThreads + threadIdx.x; q < count; q += (size_t)gridDim.x * kMaxThreads) {
        hq0[q] = to_fixed(__ldg(hf0 + q), e);
        hq1[q] = to_fixed(__ldg(hf1 + q), e);
    }
}

template <int PTS>
__device__ __forceinline__ void load_fixed(int64_t *v, const double *p, bool act, int e) {
#pragma unroll
    for (int q = 0; q < PTS; q += 2) {
        const double2 t = act ? ldg2(p + q) : make_double2(0.0, 0.0);
        v[q] = to_fixed(t.x, e);
        v[q + 1] = to_fixed(t.y, e);
    }
}

template <int PTS>
__device__ __forceinline__ void load_i64(int64_t *v, const int64_t *p, bool act) {
#pragma unroll
    for (int q = 0; q < PTS; q += 2) {
        const longlong2 t = act ? __ldg(reinterpret_cast<const longlong2 *>(p + q)) : make_longlong2(0, 0);
        v[q] = t.x;
        v[q + 1] = t.y;
    }
}

// One half-sweep of colour COLOUR over rows [i0, i1] of a strip; PTS values per thread.
template <int COLOUR, int PTS>
__global__ void __launch_bounds__(kSweepThreads)
fused_half_sweep(double *__restrict__ self, const double *__restrict__ other, const int64_t *__restrict__ hq,
                 int n, int W, int kact, int rows_per_block, const unsigned long long *__restrict__ words) {
    const int i0 = 1 + blockIdx.y * rows_per_block;
    if (i0 > n) return;  // uniform over the block
    const int i1 = min(n, i0 + rows_per_block - 1);
    const unsigned long long ew = words[2];
    const bool ok = ew != kNoScale;
    const int e = ok ? (int)(long long)ew : 0;
    const double poison = __longlong_as_double(0x7FF8000000000000ll);
    const int lane = threadIdx.x & 31;
    const int k0 = PTS * (blockIdx.x * kSweepThreads + threadIdx.x);
    const bool act = k0 < kact;  // k0 + PTS - 1 < W as W is a multiple of 32
    int64_t up[PTS], mid[PTS], dn[PTS], f[PTS];
    load_fixed<PTS>(up, other + (size_t)(i0 - 1) * W + k0, act, e);
    load_fixed<PTS>(mid, other + (size_t)i0 * W + k0, act, e);
    for (int i = i0; i <= i1; ++i) {
        const size_t row = (size_t)i * W;
        load_fixed<PTS>(dn, other + row + W + k0, act, e);
        load_i64<PTS>(f, hq + row + k0, act);
        const int p = (i + COLOUR) & 1;  // column offset of this colour in row i
        double r[PTS];
        if (p == 0) {
            // value q sits at natural column 2(k0+q): west = other[k0+q-1], east = other[k0+q]
            int64_t prev = __shfl_up_sync(0xffffffffu, mid[PTS - 1], 1);
            if (lane == 0) prev = (act && k0 > 0) ? to_fixed(__ldg(other + row + k0 - 1), e) : 0;
#pragma unroll
            for (int q = 0; q < PTS; ++q) r[q] = fused_update(f[q], up[q], dn[q], q ? mid[q - 1] : prev, mid[q], e);
        } else {
            // value q sits at 2(k0+q)+1: west = other[k0+q], east = other[k0+q+1]
            int64_t next = __shfl_down_sync(0xffffffffu, mid[0], 1);
            if (lane == 31) next = (k0 + PTS < kact) ? to_fixed(__ldg(other + row + k0 + PTS), e) : 0;
#pragma unroll
            for (int q = 0; q < PTS; ++q)
                r[q] = fused_update(f[q], up[q], dn[q], mid[q], q + 1 < PTS ? mid[q + 1] : next, e);
        }
        if (!ok) {
#pragma unroll
            for (int q = 0; q < PTS; ++q) r[q] = poison;
        }
        const int j0 = 2 * k0 + p;  // natural column of value 0; value q is at j0 + 2q
        double *sp = self + row + k0;
        if (act && j0 >= 1 && j0 + 2 * (PTS - 1) <= n) {
            store_row<PTS>(sp, r);
        } else if (act) {
#pragma unroll
            for (int q = 0; q < PTS; ++q)
                if (j0 + 2 * q >= 1 && j0 + 2 * q <= n) sp[q] = r[q];
        }
#pragma unroll
        for (int q = 0; q < PTS; ++q) {
            up[q] = mid[q];
            mid[q] = dn[q];
        }
    }
}

int reduce_grid(size_t count) {
    static const int cap = [] {
        int dev = 0, sms = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            sms = 152;
        }
        return 8 * sms;
    }();
    const size_t want = (count / 2 + kMaxThreads - 1) / kMaxThreads;
    return (int)(want < (size_t)cap ? (want < 1 ? 1 : want) : cap);
}

template <int PTS>
rbgs_status launch_fused_colour(const rbgs_ctx *c, int colour, cudaStream_t s) {
    const Geometry &g = c->g;
    const int kact = active_width(g.n);
    const int rows = c->tile_rows;
    const int per_block = PTS * kSweepThreads;
    dim3 grid((kact + per_block - 1) / per_block, (g.n + rows - 1) / rows);
    if (colour == 0)
        fused_half_sweep<0, PTS><<<grid, kSweepThreads, 0, s>>>(c->f64.u[0], c->f64.u[1], c->hq[0], g.n, g.W, kact,
                                                                rows, c->fwords);
    else
        fused_half_sweep<1, PTS><<<grid, kSweepThreads, 0, s>>>(c->f64.u[1], c->f64.u[0], c->hq[1], g.n, g.W, kact,
                                                                rows, c->fwords);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

}  // namespace

// Q = max |h2 f| of the loaded problem into words[1] (stream-ordered).
rbgs_status launch_fused_rhs_max(const rbgs_ctx *c, cudaStream_t s) {
    const size_t count = c->g.colour_elems();
    RBGS_CUDA(cudaMemsetAsync(c->fwords + 1, 0, sizeof(unsigned long long), s));
    absmax_kernel<<<reduce_grid(count), kMaxThreads, 0, s>>>(c->f64.hf[0], c->f64.hf[1], count, c->fwords + 1);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

// The scale of a block of `nsweeps` sweeps from the current iterate, and h2 f on its grid.
rbgs_status launch_fused_prepare(const rbgs_ctx *c, long long nsweeps, cudaStream_t s) {
    const size_t count = c->g.colour_elems();
    RBGS_CUDA(cudaMemsetAsync(c->fwords, 0, sizeof(unsigned long long), s));
    const int grid = reduce_grid(count);
    absmax_kernel<<<grid, kMaxThreads, 0, s>>>(c->f64.u[0], c->f64.u[1], count, c->fwords);
    RBGS_LAUNCH_CHECK();
    prepare_kernel<<<grid, kMaxThreads, 0, s>>>(c->f64.hf[0], c->f64.hf[1], c->hq[0], c->hq[1], count, c->fwords,
                                                nsweeps);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

// One fused half-sweep of `colour` at the scale the last launch_fused_prepare chose.
rbgs_status launch_fused_half_sweep(const rbgs_ctx *c, int colour, cudaStream_t s) {
    return c->pts == 4 ? launch_fused_colour<4>(c, colour, s) : launch_fused_colour<2>(c, colour, s);
}

}  // namespace rbgs
