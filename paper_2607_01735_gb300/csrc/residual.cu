// Residual-norm reduction (the convergence test of the solver).
//
// For every interior point, rt = ((((h2f + N) + S) + W) + E) - 4 u equals h^2 (b - A u)
// for the linear system of Eq. (1) with the ring folded into b.  The kernels walk the
// colour-split grid the same way the half-sweeps do (strip of rows per block, other
// colour's rows i-1, i, i+1 in registers), square each rt and reduce: warp shuffle,
// then the block, then one partial per block; a single-block kernel adds the partials
// in a fixed order.  The result is the same on every run.
//
// The adds run as fused multiply-adds by a run-time 1.0 (one rounding of the exact sum,
// the same value as the add, on GB300's faster-issuing DFMA path), and rt as
// fma(-4, u, s), the same value as s + (-4u) because 4u is exact.  GB300's FP64 pipe, not
// HBM, bounds this walk.
//
// ||h^2 b|| depends only on f and the ring; it is reduced once per problem by
// rhs_norm_kernel (h2f plus the ring neighbours of each boundary-adjacent point), walking
// the colour rows without any index division.
//
// Right after a full sweep the black points' rt is exactly zero: each black value was set
// to s * 0.25 from the very sum s the residual forms (the red values have not moved since),
// and 4 (s * 0.25) = s exactly (where s * 0.25 is subnormal and rounded, |rt| < 2^-1072 and
// its square adds nothing to the sum).  The red-black ordering gives this for any right-hand
// side (Section 2, Eq. (1)).  So after a sweep only the red points are walked: half the
// work, and the same sum bit for bit (the black partials were exact zeros).
//
// The same walk also serves the mixed-precision refinement: max |rt| (exact, order-
// independent) and the FP32 scaled defect (float)(rt * 2^-e) for the inner solver.
#include "common.cuh"
#include "fp64.cuh"
#include "sweep_impl.cuh"

namespace rbgs {
namespace {

constexpr int kFinalThreads = 1024;

// MAX: also reduce max |rt| (into partials[kMaxPartials + block]).  WRITE: also store
// (float)(rt * scale) into the FP32 colour array r32 (pitch W32) at interior points: the
// scaled defect that the mixed-precision refinement hands to its FP32 inner solver.
template <int COLOUR, bool MAX, bool WRITE>
__global__ void __launch_bounds__(kSweepThreads)
residual_colour_kernel(const double *__restrict__ self, const double *__restrict__ other,
                       const double *__restrict__ hf, int n, int W, int kact,
                       int rows_per_block, double *__restrict__ partials, float *__restrict__ r32,
                       int W32, double scale, double one) {
    __shared__ double red_smem[kSweepThreads / 32];
    const int lane = threadIdx.x & 31;
    const int k0 = 2 * (blockIdx.x * kSweepThreads + threadIdx.x);
    const bool act = k0 < kact;
    const int i0 = 1 + blockIdx.y * rows_per_block;
    const int i1 = min(n, i0 + rows_per_block - 1);
    const double2 zero = make_double2(0.0, 0.0);
    double acc = 0.0, mx = 0.0;
    if (i0 <= n) {
        double2 up = act ? ldg2(other + (size_t)(i0 - 1) * W + k0) : zero;
        double2 mid = act ? ldg2(other + (size_t)i0 * W + k0) : zero;
        for (int i = i0; i <= i1; ++i) {
            const size_t row = (size_t)i * W;
            const double2 dn = act ? ldg2(other + row + W + k0) : zero;
            const double2 f2 = act ? ldg2(hf + row + k0) : zero;
            const double2 me = act ? ldg2(self + row + k0) : zero;
            const int p = (i + COLOUR) & 1;
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
            const int j0 = 2 * k0 + p;
            if (act && j0 >= 1 && j0 <= n) {
                const double s = add_fma(add_fma(add_fma(add_fma(f2.x, up.x, one), dn.x, one), w0, one), e0, one);
                const double r = __fma_rn(-4.0, me.x, s);
                acc = __fma_rn(r, r, acc);
                if (MAX) mx = fmax(mx, fabs(r));
                if (WRITE) r32[(size_t)i * W32 + k0] = __double2float_rn(__dmul_rn(r, scale));
            }
            if (act && j0 + 2 <= n) {
                const double s = add_fma(add_fma(add_fma(add_fma(f2.y, up.y, one), dn.y, one), w1, one), e1, one);
                const double r = __fma_rn(-4.0, me.y, s);
                acc = __fma_rn(r, r, acc);
                if (MAX) mx = fmax(mx, fabs(r));
                if (WRITE) r32[(size_t)i * W32 + k0 + 1] = __double2float_rn(__dmul_rn(r, scale));
            }
            up = mid;
            mid = dn;
        }
    }
    const size_t slot = (size_t)COLOUR * gridDim.x * gridDim.y + (size_t)blockIdx.y * gridDim.x + blockIdx.x;
    const double t = block_sum<kSweepThreads>(acc, red_smem);
    if (threadIdx.x == 0) partials[slot] = t;
    if (MAX) {
        __syncthreads();
        const double m = block_max<kSweepThreads>(mx, red_smem);
        if (threadIdx.x == 0) partials[kMaxPartials + slot] = m;
    }
}

// Max of `count` partials -> *out (order-independent, exact).
__global__ void __launch_bounds__(kFinalThreads)
final_max_kernel(const double *__restrict__ partials, int count, double *__restrict__ out) {
    __shared__ double smem[kFinalThreads / 32];
    double v = 0.0;
    for (int q = threadIdx.x; q < count; q += kFinalThreads) v = fmax(v, partials[q]);
    const double t = block_max<kFinalThreads>(v, smem);
    if (threadIdx.x == 0) *out = t;
}

// Sum of `count` partials in a fixed order -> *out.
__global__ void __launch_bounds__(kFinalThreads)
final_sum_kernel(const double *__restrict__ partials, int count, double *__restrict__ out) {
    __shared__ double smem[kFinalThreads / 32];
    double v = 0.0;
    for (int q = threadIdx.x; q < count; q += kFinalThreads) v = __dadd_rn(v, partials[q]);
    const double t = block_sum<kFinalThreads>(v, smem);
    if (threadIdx.x == 0) *out = t;
}

__device__ __forceinline__ double at(const double *const *u, int W, int i, int j) {
    return u[(i + j) & 1][(size_t)i * W + (j >> 1)];
}

struct ColourPtrs { const double *p[2]; };

// Partial sums of (h^2 b)^2: h2f plus, in N, S, W, E order, the neighbours on the ring.
// Thread t of block (x, y) takes elements k0 = 2t and k0 + 1 of both colour rows (one 16-byte
// load per colour row) down the block's rows, loading four rows ahead of their use so that
// eight loads are in flight.  Away from the first and last interior row and column, b is h2f
// itself (no ring neighbour), so those rows take four fused multiply-adds and no index
// arithmetic: the walk is bound by HBM, not by instruction issue.
constexpr int kNormThreads = 256;
constexpr int kNormRowsAhead = 4;

__global__ void __launch_bounds__(kNormThreads)
rhs_norm_kernel(ColourPtrs u, ColourPtrs hf, int n, int W, int kact, int rows_per_block,
                double *__restrict__ partials) {
    __shared__ double smem[kNormThreads / 32];
    const int k0 = 2 * (blockIdx.x * kNormThreads + threadIdx.x);
    const int i0 = 1 + blockIdx.y * rows_per_block, i1 = min(n, i0 + rows_per_block - 1);
    // this thread's columns 2 k0 + {0..3} all lie in 2..n-1
    const bool inner_cols = k0 > 0 && 2 * k0 + 3 < n;
    double acc = 0.0;
    if (k0 < kact) {  // k0 + 1 < W always (W is even and at least kact)
        for (int i = i0; i <= i1; i += kNormRowsAhead) {
            double2 v[kNormRowsAhead][2];
#pragma unroll
            for (int r = 0; r < kNormRowsAhead; ++r) {
                const size_t row = (size_t)min(i + r, i1) * W;  // rows past i1: reloaded, unused
                v[r][0] = ldg2(hf.p[0] + row + k0);
                v[r][1] = ldg2(hf.p[1] + row + k0);
            }
#pragma unroll
            for (int r = 0; r < kNormRowsAhead; ++r) {
                const int ii = i + r;
                if (ii > i1) break;
                if (inner_cols && ii > 1 && ii < n) {
                    acc = __fma_rn(v[r][0].x, v[r][0].x, acc);
                    acc = __fma_rn(v[r][0].y, v[r][0].y, acc);
                    acc = __fma_rn(v[r][1].x, v[r][1].x, acc);
                    acc = __fma_rn(v[r][1].y, v[r][1].y, acc);
                    continue;
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int c = q >> 1, k = k0 + (q & 1);
                    const int j = 2 * k + ((ii + c) & 1);  // natural column of element k, colour c
                    if (j < 1 || j > n) continue;
                    double b = (q & 1) ? v[r][c].y : v[r][c].x;
                    if (ii == 1) b = __dadd_rn(b, at(u.p, W, 0, j));
                    if (ii == n) b = __dadd_rn(b, at(u.p, W, n + 1, j));
                    if (j == 1) b = __dadd_rn(b, at(u.p, W, ii, 0));
                    if (j == n) b = __dadd_rn(b, at(u.p, W, ii, n + 1));
                    acc = __fma_rn(b, b, acc);
                }
            }
        }
    }
    const double t = block_sum<kNormThreads>(acc, smem);
    if (threadIdx.x == 0) partials[(size_t)blockIdx.y * gridDim.x + blockIdx.x] = t;
}

int residual_rows(int n, int kact) {
    // enough blocks to fill the GPU, at most kMaxPartials / 2 per colour
    const int bx = (kact + 2 * kSweepThreads - 1) / (2 * kSweepThreads);
    int rows = 16;
    while ((size_t)bx * ((n + rows - 1) / rows) > (size_t)kMaxPartials / 2) rows *= 2;
    return rows;
}

}  // namespace

namespace {

// red_only: the black points' rt is known to be zero (the iterate is the result of a full
// sweep); only the red partials are formed and summed.
template <bool MAX, bool WRITE>
rbgs_status residual_passes(const rbgs_ctx *c, double scale, cudaStream_t s, bool red_only) {
    const Geometry &g = c->g;
    const int kact = active_width(g.n);
    const int rows = residual_rows(g.n, kact);
    dim3 grid((kact + 2 * kSweepThreads - 1) / (2 * kSweepThreads), (g.n + rows - 1) / rows);
    float *r0 = WRITE ? c->f32.hf[0] : nullptr, *r1 = WRITE ? c->f32.hf[1] : nullptr;
    residual_colour_kernel<0, MAX, WRITE><<<grid, kSweepThreads, 0, s>>>(
        c->f64.u[0], c->f64.u[1], c->f64.hf[0], g.n, g.W, kact, rows, c->partials, r0, c->f32.W, scale, 1.0);
    RBGS_LAUNCH_CHECK();
    if (!red_only) {
        residual_colour_kernel<1, MAX, WRITE><<<grid, kSweepThreads, 0, s>>>(
            c->f64.u[1], c->f64.u[0], c->f64.hf[1], g.n, g.W, kact, rows, c->partials, r1, c->f32.W, scale, 1.0);
        RBGS_LAUNCH_CHECK();
    }
    const int count = (red_only ? 1 : 2) * (int)(grid.x * grid.y);
    final_sum_kernel<<<1, kFinalThreads, 0, s>>>(c->partials, count, c->dsum);
    RBGS_LAUNCH_CHECK();
    if (MAX) {
        final_max_kernel<<<1, kFinalThreads, 0, s>>>(c->partials + kMaxPartials, count, c->dsum + 2);
        RBGS_LAUNCH_CHECK();
    }
    return RBGS_OK;
}

}  // namespace

rbgs_status launch_residual_sum(const rbgs_ctx *c, cudaStream_t s) {
    return residual_passes<false, false>(c, 1.0, s, c->black_fresh);
}

// write_r32 = false: sum rt^2 -> dsum[0], max |rt| -> dsum[2].
// write_r32 = true:  r32 = (float)(rt * scale) at interior points (and the sum again).
rbgs_status launch_defect(const rbgs_ctx *c, bool write_r32, double scale, cudaStream_t s) {
    return write_r32 ? residual_passes<false, true>(c, scale, s, false) : residual_passes<true, false>(c, scale, s, false);
}

rbgs_status launch_rhs_norm(const rbgs_ctx *c, cudaStream_t s) {
    const Geometry &g = c->g;
    ColourPtrs u{{c->f64.u[0], c->f64.u[1]}}, hf{{c->f64.hf[0], c->f64.hf[1]}};
    const int kact = active_width(g.n);
    const int bx = (kact + 2 * kNormThreads - 1) / (2 * kNormThreads);
    int rows = 16;
    while ((size_t)bx * ((g.n + rows - 1) / rows) > (size_t)kMaxPartials) rows *= 2;
    const dim3 grid(bx, (g.n + rows - 1) / rows);
    rhs_norm_kernel<<<grid, kNormThreads, 0, s>>>(u, hf, g.n, g.W, kact, rows, c->partials);
    RBGS_LAUNCH_CHECK();
    final_sum_kernel<<<1, kFinalThreads, 0, s>>>(c->partials, (int)(grid.x * grid.y), c->dsum + 1);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

}  // namespace rbgs
