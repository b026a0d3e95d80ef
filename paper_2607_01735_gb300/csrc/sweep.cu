// Half-sweep kernels: one launch updates every point of one colour (Section 2, Eq. (1);
// the red-then-black phases of Algorithm 1), reading only the other colour.
//
// Work decomposition.  A thread owns two neighbouring values (k0, k0+1) of its colour
// in a row, loaded and stored as one 16-byte vector, and walks down `rows` consecutive
// rows of a strip.  The other colour's rows i-1, i, i+1 live in registers as the strip
// advances, so every value of the other colour is loaded from memory once per strip
// (plus the two rows shared with neighbouring strips), h2*f once, and the own colour is
// only written: 24 bytes of DRAM traffic per point update in FP64.  The west/east
// neighbour that belongs to the adjacent thread arrives by warp shuffle; at warp edges
// it is loaded directly.
//
// Arithmetic.  Each update is (((h2f + N) + S) + W) + E, times 0.25, every step
// correctly rounded (see fp64.cuh).  Template parameter M picks, per add, the FP64 pipe
// (fma(a, one, b), one = 1.0 passed at run time) or the exact integer-pipe add; bits 0-3 are the four adds of the
// thread's first point, bits 4-7 of its second.  PLAIN selects the textbook add and
// multiply instructions.  Every choice yields the same bits.
#include "common.cuh"
#include "fp64.cuh"
#include "sweep_impl.cuh"

namespace rbgs {
namespace {

template <int COLOUR, int M, bool PLAIN>
__global__ void __launch_bounds__(kSweepThreads)
half_sweep_f64(double *__restrict__ self, const double *__restrict__ other,
               const double *__restrict__ hf, int n, int W, int kact, int rows_per_block,
               double one) {
    const int lane = threadIdx.x & 31;
    const int k0 = 2 * (blockIdx.x * kSweepThreads + threadIdx.x);
    const bool act = k0 < kact;
    const int i0 = 1 + blockIdx.y * rows_per_block;
    if (i0 > n) return;  // uniform over the block
    const int i1 = min(n, i0 + rows_per_block - 1);
    const double2 zero = make_double2(0.0, 0.0);
    double2 up = act ? ldg2(other + (size_t)(i0 - 1) * W + k0) : zero;
    double2 mid = act ? ldg2(other + (size_t)i0 * W + k0) : zero;
    for (int i = i0; i <= i1; ++i) {
        const size_t row = (size_t)i * W;
        const double2 dn = act ? ldg2(other + row + W + k0) : zero;
        const double2 f2 = act ? ldg2(hf + row + k0) : zero;
        const int p = (i + COLOUR) & 1;  // column offset of this colour in row i
        double w0, e0, w1, e1;
        if (p == 0) {
            double prev = __shfl_up_sync(0xffffffffu, mid.y, 1);
            if (lane == 0) prev = (act && k0 > 0) ? __ldg(other + row + k0 - 1) : 0.0;
            w0 = prev; e0 = mid.x; w1 = mid.x; e1 = mid.y;
        } else {
            double next = __shfl_down_sync(0xffffffffu, mid.x, 1);
            if (lane == 31) next = (k0 + 2 < kact) ? __ldg(other + row + k0 + 2) : 0.0;
            w0 = mid.x; e0 = mid.y; w1 = mid.y; e1 = next;
        }
        const double r0 = update_f64<(M & 15), PLAIN>(f2.x, up.x, dn.x, w0, e0, one);
        const double r1 = update_f64<(M >> 4), PLAIN>(f2.y, up.y, dn.y, w1, e1, one);
        const int j0 = 2 * k0 + p;  // natural column of the first value; second is j0 + 2
        const bool in0 = act && j0 >= 1 && j0 <= n;
        const bool in1 = act && j0 + 2 <= n;
        double *sp = self + row + k0;
        if (in0 && in1) {
            stg2(sp, make_double2(r0, r1));
        } else {
            if (in0) sp[0] = r0;
            if (in1) sp[1] = r1;
        }
        up = mid;
        mid = dn;
    }
}

template <int M, bool PLAIN>
rbgs_status launch_colour(const rbgs_ctx *c, int colour, cudaStream_t s) {
    const Geometry &g = c->g;
    const int kact = active_width(g.n);
    const int rows = c->tile_rows;
    dim3 grid((kact + 2 * kSweepThreads - 1) / (2 * kSweepThreads), (g.n + rows - 1) / rows);
    if (colour == 0)
        half_sweep_f64<0, M, PLAIN><<<grid, kSweepThreads, 0, s>>>(c->u[0], c->u[1], c->hf[0],
                                                                    g.n, g.W, kact, rows, 1.0);
    else
        half_sweep_f64<1, M, PLAIN><<<grid, kSweepThreads, 0, s>>>(c->u[1], c->u[0], c->hf[1],
                                                                    g.n, g.W, kact, rows, 1.0);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

}  // namespace

// emulate: -2 = textbook add/multiply instructions; otherwise the mask of integer-pipe
// adds (a few tuned splits are instantiated; others round to the nearest below).
rbgs_status launch_half_sweep(const rbgs_ctx *c, int colour, cudaStream_t s) {
    switch (c->emulate) {
    case -2: return launch_colour<0x00, true>(c, colour, s);
    case 0x00: return launch_colour<0x00, false>(c, colour, s);
    case 0x08: return launch_colour<0x08, false>(c, colour, s);
    case 0x88: return launch_colour<0x88, false>(c, colour, s);
    case 0x8C: return launch_colour<0x8C, false>(c, colour, s);
    case 0xCC: return launch_colour<0xCC, false>(c, colour, s);
    case 0xCE: return launch_colour<0xCE, false>(c, colour, s);
    case 0xEE: return launch_colour<0xEE, false>(c, colour, s);
    case 0xFF: return launch_colour<0xFF, false>(c, colour, s);
    default:
        set_error("unsupported FP64 emulation split 0x%x", c->emulate);
        return RBGS_EINVAL;
    }
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
    case -2: case 0x00: case 0x08: case 0x88: case 0x8C: case 0xCC: case 0xCE: case 0xEE: case 0xFF:
        return true;
    default:
        return false;
    }
}

}  // namespace rbgs
