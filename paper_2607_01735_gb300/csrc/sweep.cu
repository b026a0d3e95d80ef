// Half-sweep kernels: one launch updates every point of one colour (Section 2, Eq. (1);
// the red-then-black phases of Algorithm 1), reading only the other colour.
//
// Work decomposition.  A thread owns PTS (2 or 4) neighbouring values k0.. of its colour
// in a row, loaded and stored as 16-byte vectors, and walks down `rows` consecutive
// rows of a strip, one or two rows per loop step.  The other colour's rows i-1, i, i+1 live in registers as the strip
// advances, so every value of the other colour is loaded from memory once per strip
// (plus the two rows shared with neighbouring strips), h2*f once, and the own colour is
// only written: 24 bytes of DRAM traffic per point update in FP64.  The west/east
// neighbour that belongs to the adjacent thread arrives by warp shuffle; at warp edges
// it is loaded directly.
//
// Arithmetic.  Each update is (((h2f + N) + S) + W) + E, times 0.25, every step
// correctly rounded (see fp64.cuh).  Template parameter M picks, per add, the FP64 pipe
// (fma(a, one, b), one = 1.0 passed at run time) or the exact integer-pipe add; bits 0-3
// are the four adds of the thread's even values, bits 4-7 of its odd values.  PLAIN
// selects the textbook add and multiply instructions.  Every choice yields the same bits.
#include "common.cuh"
#include "fp64.cuh"
#include "sweep_impl.cuh"

namespace rbgs {
namespace {

// PTS values per thread (2 or 4) and ROWS rows per loop step (1 or 2): both give the FP64
// pipe more independent update chains per thread (all updates of one colour are
// independent of each other).
template <int COLOUR, int M, bool PLAIN, int PTS>
__device__ __forceinline__ void update_row(double *__restrict__ self, const double *__restrict__ other,
                                           const double *up, const double *mid, const double *dn,
                                           const double *f, int i, int k0, int n, int W, int kact, bool act,
                                           int lane, double one) {
    const size_t row = (size_t)i * W;
    const int p = (i + COLOUR) & 1;  // column offset of this colour in row i
    double r[PTS];
    if (p == 0) {
        // value q sits at natural column 2(k0+q): west = other[k0+q-1], east = other[k0+q]
        double prev = __shfl_up_sync(0xffffffffu, mid[PTS - 1], 1);
        if (lane == 0) prev = (act && k0 > 0) ? __ldg(other + row + k0 - 1) : 0.0;
#pragma unroll
        for (int q = 0; q < PTS; ++q)
            r[q] = update_f64<PLAIN>((M >> (4 * (q & 1))) & 15, f[q], up[q], dn[q], q ? mid[q - 1] : prev, mid[q],
                                     one);
    } else {
        // value q sits at 2(k0+q)+1: west = other[k0+q], east = other[k0+q+1]
        double next = __shfl_down_sync(0xffffffffu, mid[0], 1);
        if (lane == 31) next = (k0 + PTS < kact) ? __ldg(other + row + k0 + PTS) : 0.0;
#pragma unroll
        for (int q = 0; q < PTS; ++q)
            r[q] = update_f64<PLAIN>((M >> (4 * (q & 1))) & 15, f[q], up[q], dn[q], mid[q],
                                     q + 1 < PTS ? mid[q + 1] : next, one);
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
}

// Rows i0..i1 of one strip (the body of a half-sweep block).
template <int COLOUR, int M, bool PLAIN, int PTS, int ROWS>
__device__ __forceinline__ void march_strip(double *__restrict__ self, const double *__restrict__ other,
                                            const double *__restrict__ hf, int n, int W, int kact, int i0, int i1,
                                            double one) {
    static_assert(PTS == 2 || PTS == 4, "2 or 4 values per thread");
    static_assert(ROWS == 1 || ROWS == 2, "1 or 2 rows per step");
    const int lane = threadIdx.x & 31;
    const int k0 = PTS * (blockIdx.x * kSweepThreads + threadIdx.x);
    const bool act = k0 < kact;  // k0 + PTS - 1 < W as W is a multiple of 32
    double up[PTS], mid[PTS], dn[PTS], f[PTS];
    load_row<PTS>(up, other + (size_t)(i0 - 1) * W + k0, act);
    load_row<PTS>(mid, other + (size_t)i0 * W + k0, act);
    int i = i0;
    if (ROWS == 2) {
        double dn2[PTS], f2[PTS];
        for (; i + 1 <= i1; i += 2) {
            const size_t row = (size_t)i * W;
            load_row<PTS>(dn, other + row + W + k0, act);
            load_row<PTS>(dn2, other + row + 2 * (size_t)W + k0, act);
            load_row<PTS>(f, hf + row + k0, act);
            load_row<PTS>(f2, hf + row + W + k0, act);
            update_row<COLOUR, M, PLAIN, PTS>(self, other, up, mid, dn, f, i, k0, n, W, kact, act, lane, one);
            update_row<COLOUR, M, PLAIN, PTS>(self, other, mid, dn, dn2, f2, i + 1, k0, n, W, kact, act, lane, one);
#pragma unroll
            for (int q = 0; q < PTS; ++q) {
                up[q] = dn[q];
                mid[q] = dn2[q];
            }
        }
    }
    for (; i <= i1; ++i) {
        const size_t row = (size_t)i * W;
        load_row<PTS>(dn, other + row + W + k0, act);
        load_row<PTS>(f, hf + row + k0, act);
        update_row<COLOUR, M, PLAIN, PTS>(self, other, up, mid, dn, f, i, k0, n, W, kact, act, lane, one);
#pragma unroll
        for (int q = 0; q < PTS; ++q) {
            up[q] = mid[q];
            mid[q] = dn[q];
        }
    }
}

template <int COLOUR, int M, bool PLAIN, int PTS, int ROWS>
__global__ void __launch_bounds__(kSweepThreads)
half_sweep_f64(double *__restrict__ self, const double *__restrict__ other,
               const double *__restrict__ hf, int n, int W, int kact, int rows_per_block,
               double one) {
    const int i0 = 1 + blockIdx.y * rows_per_block;
    if (i0 > n) return;  // uniform over the block
    const int i1 = min(n, i0 + rows_per_block - 1);
    march_strip<COLOUR, M, PLAIN, PTS, ROWS>(self, other, hf, n, W, kact, i0, i1, one);
}

// Hybrid half-sweep: the rows are cut into repeating pairs of strips, rows_fp rows whose
// adds run on the FP64 pipe and rows_int rows whose adds run on the integer pipe (exact
// IEEE addition, fp64.cuh).  Block y handles strip y; both kinds of blocks are resident on
// every SM at once, so the two pipes work in parallel while each warp stays on one pipe.
// The result is bit-identical to every other variant.
template <int COLOUR, int PTS>
__global__ void __launch_bounds__(kSweepThreads)
half_sweep_f64_hybrid(double *__restrict__ self, const double *__restrict__ other,
                      const double *__restrict__ hf, int n, int W, int kact, int rows_fp, int rows_int,
                      double one) {
    const int period = rows_fp + rows_int;
    const int pair = blockIdx.y >> 1, kind = blockIdx.y & 1;
    const int i0 = 1 + pair * period + (kind ? rows_fp : 0);
    if (i0 > n) return;  // uniform over the block
    const int i1 = min(n, i0 + (kind ? rows_int : rows_fp) - 1);
    if (kind == 0)
        march_strip<COLOUR, 0x00, false, PTS, 1>(self, other, hf, n, W, kact, i0, i1, one);
    else
        march_strip<COLOUR, 0xFF, false, PTS, 1>(self, other, hf, n, W, kact, i0, i1, one);
}

template <int M, bool PLAIN, int PTS, int ROWS>
rbgs_status launch_colour(const rbgs_ctx *c, int colour, cudaStream_t s) {
    const Geometry &g = c->g;
    const int kact = active_width(g.n);
    const int rows = c->tile_rows;
    const int per_block = PTS * kSweepThreads;
    dim3 grid((kact + per_block - 1) / per_block, (g.n + rows - 1) / rows);
    if (colour == 0)
        half_sweep_f64<0, M, PLAIN, PTS, ROWS><<<grid, kSweepThreads, 0, s>>>(c->f64.u[0], c->f64.u[1], c->f64.hf[0],
                                                                         g.n, g.W, kact, rows, 1.0);
    else
        half_sweep_f64<1, M, PLAIN, PTS, ROWS><<<grid, kSweepThreads, 0, s>>>(c->f64.u[1], c->f64.u[0], c->f64.hf[1],
                                                                         g.n, g.W, kact, rows, 1.0);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

template <int PTS>
rbgs_status launch_hybrid(const rbgs_ctx *c, int colour, cudaStream_t s) {
    const Geometry &g = c->g;
    const int kact = active_width(g.n);
    const int rf = c->tile_rows, ri = c->int_rows;
    const int per_block = PTS * kSweepThreads;
    const int pairs = (g.n + rf + ri - 1) / (rf + ri);
    dim3 grid((kact + per_block - 1) / per_block, 2 * pairs);
    if (colour == 0)
        half_sweep_f64_hybrid<0, PTS><<<grid, kSweepThreads, 0, s>>>(c->f64.u[0], c->f64.u[1], c->f64.hf[0], g.n, g.W,
                                                                     kact, rf, ri, 1.0);
    else
        half_sweep_f64_hybrid<1, PTS><<<grid, kSweepThreads, 0, s>>>(c->f64.u[1], c->f64.u[0], c->f64.hf[1], g.n, g.W,
                                                                     kact, rf, ri, 1.0);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

template <int PTS>
rbgs_status launch_pts(const rbgs_ctx *c, int colour, cudaStream_t s) {
    if (c->int_rows > 0) return launch_hybrid<PTS>(c, colour, s);
    if (c->sweep_rows == 2 && c->emulate == 0x00) return launch_colour<0x00, false, PTS, 2>(c, colour, s);
    switch (c->emulate) {
    case -2: return launch_colour<0x00, true, PTS, 1>(c, colour, s);
    case 0x00: return launch_colour<0x00, false, PTS, 1>(c, colour, s);
    case 0x08: return launch_colour<0x08, false, PTS, 1>(c, colour, s);
    case 0x88: return launch_colour<0x88, false, PTS, 1>(c, colour, s);
    case 0x8C: return launch_colour<0x8C, false, PTS, 1>(c, colour, s);
    case 0xCC: return launch_colour<0xCC, false, PTS, 1>(c, colour, s);
    case 0xFF: return launch_colour<0xFF, false, PTS, 1>(c, colour, s);
    default:
        set_error("unsupported FP64 emulation split 0x%x", c->emulate);
        return RBGS_EINVAL;
    }
}

}  // namespace

// emulate: -2 = textbook add/multiply instructions; otherwise the mask of integer-pipe
// adds (bits 0-3: the four adds of even values, bits 4-7: of odd values).
rbgs_status launch_half_sweep(const rbgs_ctx *c, int colour, cudaStream_t s) {
    return c->pts == 4 ? launch_pts<4>(c, colour, s) : launch_pts<2>(c, colour, s);
}

rbgs_status launch_sweeps_f64(const rbgs_ctx *c, long nsweeps, cudaStream_t s) {
    for (long it = 0; it < nsweeps; ++it) {
        rbgs_status st = launch_half_sweep(c, 0, s);
        if (st != RBGS_OK) return st;
        st = launch_half_sweep(c, 1, s);
        if (st != RBGS_OK) return st;
    }
    return RBGS_OK;
}

bool emulation_split_supported(int m) {
    switch (m) {
    case -2: case 0x00: case 0x08: case 0x88: case 0x8C: case 0xCC: case 0xFF:
        return true;
    default:
        return false;
    }
}

}  // namespace rbgs
