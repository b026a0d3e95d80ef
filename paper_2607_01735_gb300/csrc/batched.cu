// Batched solve of many independent Poisson problems of uneven sizes in persistent launches
// (rbgs_solve_batched).
//
// Design.  The problems are independent, so the batch shards by problem with no data
// exchange.  A persistent grid of thread blocks pulls problem indices, largest first, from
// an atomic work counter; a team that claims a problem solves it to tolerance on its own:
// red half-sweep, team barrier, black half-sweep, team barrier (the colour phases of
// Algorithm 1), a deterministic reduction of the residual every `check_every` sweeps
// (FP64), or the mixed-precision refinement loop (FP64 defect/correction, FP32 sweeps).
// A team is one block, or the blocks of one thread-block cluster for the largest problems
// left over after full waves (the phased plan: a launch of full waves, one block per
// problem, then a launch in which clusters take the leftover largest problems and single
// blocks the rest).  No block waits on a block outside its cluster; a cluster's blocks
// reach the same barriers on every path.  Each problem records %globaltimer stamps when
// its team starts and finishes it.
//
// The arithmetic per update is the one of the single-problem kernels (same operations,
// same order), so every problem's iterate equals the oracle's after the same sweeps.
// The host side packs all problems into one device pool (colour-split layout), captures
// pack -> persistent launches -> unpack into a CUDA graph and launches it.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <mutex>
#include <numeric>
#include <vector>

#include "common.cuh"
#include "sweep_impl.cuh"

namespace rbgs {
namespace {

struct DevProblem {
    int n, W, W32, pad;
    double h2;
    double *u[2];
    double *hf[2];
    float *d[2];   // FP32 correction (refinement)
    float *r[2];   // FP32 scaled defect (refinement)
    const double *f_nat;   // natural-layout inputs (device-readable)
    const double *u_nat;
    double *out_nat;       // natural-layout output (device)
};

struct DevResult {
    int status;
    int pad;
    long long sweeps;
    double rel;
    unsigned long long t_start, t_end;
};

// Limits of a batch: a problem stops (RBGS_ENOTCONV) when rho has not reached a new
// minimum for stall_limit consecutive checks (<= 0: never), and every problem stops
// (RBGS_ETIMEOUT) once budget_ns of %globaltimer time have passed since the batch's first
// problem started (*t_first, the minimum over the teams' start stamps; 0: no budget).
struct BatchLimits {
    int stall_limit;
    unsigned long long budget_ns;
    unsigned long long *t_first;
};

__device__ __forceinline__ unsigned long long globaltimer() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %globaltimer;" : "=l"(t));
    return t;
}

// ---- teams.  A problem is solved by a team: one thread block, or the CS blocks of one
// thread-block cluster (one block per SM).  The team's VT = CS * THREADS threads act as one
// block: thread vt = rank * THREADS + threadIdx.x takes every VT-th work item, a team
// barrier separates the colour phases, and reductions combine the blocks' partials in
// rank order, so every block of the team sees the same residual and takes the same
// decisions (the same number of barriers on every path).

__device__ __forceinline__ int cluster_rank() {
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return (int)r;
}

// Barrier over the team: the block for CS = 1, else the cluster barrier with release /
// acquire at cluster scope, which makes every global write of the team made before it
// visible to every thread of the team after it.  Reached by all threads of the team on
// the same paths (decisions come from team-wide values only).
template <int CS>
__device__ __forceinline__ void team_sync() {
    if (CS == 1) {
        __syncthreads();
    } else {
        asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
    }
}

// Shared-memory value of block `rank` of this cluster (distributed shared memory).
__device__ __forceinline__ uint32_t dsmem_addr(const void *local, int rank) {
    const uint32_t a = (uint32_t)__cvta_generic_to_shared(local);
    uint32_t ra;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(ra) : "r"(a), "r"(rank));
    return ra;
}
__device__ __forceinline__ double ld_dsmem(const double *local, int rank) {
    double v;
    asm volatile("ld.shared::cluster.f64 %0, [%1];" : "=d"(v) : "r"(dsmem_addr(local, rank)) : "memory");
    return v;
}
__device__ __forceinline__ int ld_dsmem(const int *local, int rank) {
    int v;
    asm volatile("ld.shared::cluster.s32 %0, [%1];" : "=r"(v) : "r"(dsmem_addr(local, rank)) : "memory");
    return v;
}

// Load of an array that other blocks of the team write: through L2 only for teams of
// several blocks (an L1 line of this SM may predate the last team barrier).
template <int CS, typename V>
__device__ __forceinline__ V ldt(const V *p) {
    if (CS == 1) return *p;
    return __ldcg(p);
}

// Team-wide deterministic sum / max, the same value in every thread of the team: block
// reduction (fixed tree), then the blocks' results added in rank order.
template <int THREADS, int CS>
__device__ __forceinline__ double team_sum(double v, double *smem, double *slot) {
    const double t = block_sum<THREADS>(v, smem);
    if (threadIdx.x == 0) *slot = t;
    team_sync<CS>();
    double r;
    if (CS == 1) {
        r = *slot;
    } else {
        r = ld_dsmem(slot, 0);
        for (int q = 1; q < CS; ++q) r = __dadd_rn(r, ld_dsmem(slot, q));
    }
    team_sync<CS>();
    return r;
}

template <int THREADS, int CS>
__device__ __forceinline__ double team_max(double v, double *smem, double *slot) {
    const double t = block_max<THREADS>(v, smem);
    if (threadIdx.x == 0) *slot = t;
    team_sync<CS>();
    double r;
    if (CS == 1) {
        r = *slot;
    } else {
        r = ld_dsmem(slot, 0);
        for (int q = 1; q < CS; ++q) r = fmax(r, ld_dsmem(slot, q));
    }
    team_sync<CS>();
    return r;
}

__device__ __forceinline__ int kact_of(int n) { return (((n + 3) / 2) + 1) & ~1; }

// FP32 half-sweep of colour C over the whole problem by this team, as a row-band walk:
// work item (column group g, band b) is a strip of V values (16 bytes) of the colour rows
// walked down the band's rows with the other colour's rows i-1, i, i+1 in registers, so
// each row of the other colour is loaded once per item (plus the band edges) and h2f once.
// The west/east value that lies outside the item is read directly.  Loads are ordinary
// (coherent) loads, through L2 for multi-block teams: the other colour was written by the
// team one half-sweep earlier.  Every thread of the team runs the same number of row
// steps, on rows of the same parity; steps past an item's band, and threads without an
// item, compute on a valid row and store nothing (warps without any item skip the pass).
template <typename T>
struct BandVec;
template <>
struct BandVec<float> {
    static constexpr int V = 4;
    template <int CS>
    __device__ static void load(float *v, const float *p) {
        const float4 t = ldt<CS>(reinterpret_cast<const float4 *>(p));
        v[0] = t.x, v[1] = t.y, v[2] = t.z, v[3] = t.w;
    }
    __device__ static void store(float *p, const float *v) {
        *reinterpret_cast<float4 *>(p) = make_float4(v[0], v[1], v[2], v[3]);
    }
    __device__ static float update(float hf, float vn, float vs, float vw, float ve) {
        float s = __fadd_rn(hf, vn);
        s = __fadd_rn(s, vs);
        s = __fadd_rn(s, vw);
        s = __fadd_rn(s, ve);
        return __fmul_rn(s, 0.25f);
    }
};
template <typename T, int C, int VT, int CS>
__device__ void block_half_sweep_band(T *__restrict__ self, const T *other, const T *hf, int n, int W, int vt) {
    using BV = BandVec<T>;
    constexpr int V = BV::V;
    const int kact = kact_of(n);
    const int ncol = (kact + V - 1) / V;
    const int bands = ncol < VT ? VT / ncol : 1;
    // rows per band, even: every band starts on an odd row, so at each step all bands sit
    // on rows of one parity and the colour-offset branch stays uniform across a warp that
    // spans two bands
    const int rb = ((n + bands - 1) / bands + 1) & ~1;
    const int passes = (ncol * bands + VT - 1) / VT;  // > 1 only when ncol > VT
    for (int pass = 0; pass < passes; ++pass) {
        const int item = pass * VT + vt;
        const bool has = item < ncol * bands;
        if (__all_sync(0xffffffffu, !has)) continue;  // warp-uniform: no item in this warp
        const int g = has ? item % ncol : 0, b = has ? item / ncol : 0;
        const int k0 = V * g;
        const int i0 = 1 + b * rb, i1 = min(n, i0 + rb - 1);
        // rows i-1, i, i+1 of the other colour and h2f of row i, plus the next step's row
        // i+2 / h2f i+1 / edge values loaded one step ahead (their latency overlaps a step)
        T up[V], mid[V], dn[V], f[V], dn2[V], f2[V];
        BV::template load<CS>(up, other + (size_t)min(i0 - 1, n) * W + k0);
        BV::template load<CS>(mid, other + (size_t)min(i0, n) * W + k0);
        BV::template load<CS>(dn, other + (size_t)(min(i0, n) + 1) * W + k0);
        BV::template load<CS>(f, hf + (size_t)min(i0, n) * W + k0);
        auto edge = [&](int ic) {  // the west (k0-1) or east (k0+V) value of row ic
            const size_t row = (size_t)ic * W;
            if (((ic + C) & 1) == 0) return k0 > 0 ? ldt<CS>(other + row + k0 - 1) : T(0);
            return k0 + V < kact ? ldt<CS>(other + row + k0 + V) : T(0);
        };
        T ew = edge(min(i0, n));
        for (int r = 0; r < rb; ++r) {
            const int i = i0 + r;
            const bool live = has && i <= i1;
            // past row n (last band only): a valid row of the same parity (n or n - 1, the
            // ring row 0 when n = 1) for the steps that store nothing
            const int ic = i <= n ? i : n - ((i - n) & 1);
            const int in = i + 1 <= n ? i + 1 : n - ((i + 1 - n) & 1);
            BV::template load<CS>(dn2, other + (size_t)(in + 1) * W + k0);
            BV::template load<CS>(f2, hf + (size_t)in * W + k0);
            const T ew2 = edge(in);
            const int p = (ic + C) & 1;
            const size_t row = (size_t)ic * W;
            T res[V];
            if (p == 0) {  // west/east at k-1, k
#pragma unroll
                for (int q = 0; q < V; ++q) res[q] = BV::update(f[q], up[q], dn[q], q ? mid[q - 1] : ew, mid[q]);
            } else {  // at k, k+1
#pragma unroll
                for (int q = 0; q < V; ++q)
                    res[q] = BV::update(f[q], up[q], dn[q], mid[q], q + 1 < V ? mid[q + 1] : ew);
            }
            if (live) {
                const int j0 = 2 * k0 + p;  // natural column of value q: j0 + 2q
                if (j0 >= 1 && j0 + 2 * (V - 1) <= n) {
                    BV::store(self + row + k0, res);
                } else {
#pragma unroll
                    for (int q = 0; q < V; ++q)
                        if (j0 + 2 * q >= 1 && j0 + 2 * q <= n) self[row + k0 + q] = res[q];
                }
            }
#pragma unroll
            for (int q = 0; q < V; ++q) {
                up[q] = mid[q];
                mid[q] = dn[q];
                dn[q] = dn2[q];
                f[q] = f2[q];
            }
            ew = ew2;
        }
    }
}

// One FP64 half-sweep of colour C over the whole problem by this team, one pair of values
// per thread per iteration (flattened over rows and pairs: every thread busy, which suits
// the FP64 pipe).  quarter() votes across the warp, so a warp runs an iteration whenever
// any of its lanes has an item and leaves the loop as a whole.  Loads of the other colour
// are ordinary (coherent) loads, through L2 for multi-block teams: the team wrote it one
// half-sweep earlier.
template <int C, int VT, int CS>
__device__ void block_half_sweep_f64(const DevProblem &P, int vt) {
    double *self = P.u[C];
    const double *other = P.u[C ^ 1];
    const double *hf = P.hf[C];
    const int n = P.n, W = P.W, kact = kact_of(n), npairs = kact / 2;
    const int items = n * npairs;
    for (int base = 0; base < items; base += VT) {
        if (base + (vt & ~31) >= items) break;  // warp-uniform: no item left for this warp
        const int q = base + vt;
        const bool act = q < items;
        const int qq = act ? q : 0;
        const int i = 1 + qq / npairs, k0 = 2 * (qq % npairs);
        const int p = (i + C) & 1;
        const size_t row = (size_t)i * W;
        const double2 up = ldt<CS>(reinterpret_cast<const double2 *>(other + row - W + k0));
        const double2 mid = ldt<CS>(reinterpret_cast<const double2 *>(other + row + k0));
        const double2 dn = ldt<CS>(reinterpret_cast<const double2 *>(other + row + W + k0));
        const double2 f2 = *reinterpret_cast<const double2 *>(hf + row + k0);
        double w0, e0, w1, e1;
        if (p == 0) {
            w0 = k0 > 0 ? ldt<CS>(other + row + k0 - 1) : 0.0;
            e0 = mid.x; w1 = mid.x; e1 = mid.y;
        } else {
            w0 = mid.x; e0 = mid.y; w1 = mid.y;
            e1 = (k0 + 2 < kact) ? ldt<CS>(other + row + k0 + 2) : 0.0;
        }
        const double r0 = update_f64<false>(0, f2.x, up.x, dn.x, w0, e0, 1.0);
        const double r1 = update_f64<false>(0, f2.y, up.y, dn.y, w1, e1, 1.0);
        const int j0 = 2 * k0 + p;
        if (act && j0 >= 1 && j0 <= n) self[row + k0] = r0;
        if (act && j0 + 2 <= n) self[row + k0 + 1] = r1;
    }
}

// FP32 half-sweep of the defect equation (h^2 f replaced by the scaled defect r).
template <int C, int VT, int CS>
__device__ void block_half_sweep_f32(const DevProblem &P, int vt) {
    block_half_sweep_band<float, C, VT, CS>(P.d[C], P.d[C ^ 1], P.r[C], P.n, P.W32, vt);
}

// Per-thread partial of sum rt^2 (and max |rt|; optionally write (float)(rt * scale)) over
// the first `colours` colours.  Right after a full FP64 sweep the black points' rt is exactly
// zero (their values are s * 0.25 of the very sums s formed here, and 4 (s * 0.25) = s), so
// the red points alone give the same sum bit for bit: colours = 1 there.
template <int VT, int CS, bool WRITE>
__device__ void block_residual(const DevProblem &P, double scale, double &r2, double &mx, int vt,
                               int colours = 2) {
    const int n = P.n, W = P.W, kact = kact_of(n);
    r2 = 0.0;
    mx = 0.0;
    for (int c = 0; c < colours; ++c) {
        const double *self = P.u[c], *other = P.u[c ^ 1], *hf = P.hf[c];
        const int items = n * kact;
        for (int q = vt; q < items; q += VT) {
            const int i = 1 + q / kact, k = q % kact;
            const int p = (i + c) & 1;
            const int j = 2 * k + p;
            if (j < 1 || j > n) continue;
            const size_t row = (size_t)i * W;
            double s = __dadd_rn(hf[row + k], ldt<CS>(other + row - W + k));
            s = __dadd_rn(s, ldt<CS>(other + row + W + k));
            s = __dadd_rn(s, ldt<CS>(other + row + k - 1 + p));
            s = __dadd_rn(s, ldt<CS>(other + row + k + p));
            const double r = __dadd_rn(s, -__dmul_rn(4.0, ldt<CS>(self + row + k)));
            r2 = __fma_rn(r, r, r2);
            mx = fmax(mx, fabs(r));
            if (WRITE) P.r[c][(size_t)i * P.W32 + k] = __double2float_rn(__dmul_rn(r, scale));
        }
    }
}

// Per-thread partial of sum (h^2 b)^2: h2f plus the ring neighbours, as in rhs_norm_kernel
// (the ring is never written, h2f only by the packing kernel).
template <int VT>
__device__ double rhs_norm2_partial(const DevProblem &P, int vt) {
    const int n = P.n, W = P.W;
    double acc = 0.0;
    const int total = n * n;
    for (int q = vt; q < total; q += VT) {
        const int i = 1 + q / n, j = 1 + q % n;
        auto at = [&](const double *const *a, int ii, int jj) { return a[(ii + jj) & 1][(size_t)ii * W + (jj >> 1)]; };
        double b = at(P.hf, i, j);
        if (i == 1) b = __dadd_rn(b, at(P.u, 0, j));
        if (i == n) b = __dadd_rn(b, at(P.u, n + 1, j));
        if (j == 1) b = __dadd_rn(b, at(P.u, i, 0));
        if (j == n) b = __dadd_rn(b, at(P.u, i, n + 1));
        acc = __fma_rn(b, b, acc);
    }
    return acc;
}

__device__ __forceinline__ double rho_of(double r2, double den2) {
    return den2 > 0.0 ? sqrt(r2) / sqrt(den2) : sqrt(r2);
}

// Solve one problem with a team of CS blocks (rank: this block's place in it).  The sweep
// limit is max_sweeps, scaled by (n / cap_n)^2 when cap_n > 0 (the autotuner's probes: the
// work per problem then grows like n^4, as in a solve to tolerance).
// Whether the batch's time budget is spent, the same answer in every thread of the team
// (the team's leader reads the clock; the value reaches the others through a team sum).
template <int THREADS, int CS>
__device__ __forceinline__ bool budget_spent(const BatchLimits &L, int rank, double *smem, double *slot) {
    if (L.budget_ns == 0) return false;
    double v = 0.0;
    if (rank == 0 && threadIdx.x == 0) {
        const unsigned long long first = *reinterpret_cast<volatile unsigned long long *>(L.t_first);
        const unsigned long long now = globaltimer();
        v = (now > first && now - first > L.budget_ns) ? 1.0 : 0.0;
    }
    return team_sum<THREADS, CS>(v, smem, slot) > 0.5;
}

template <int THREADS, int CS>
__device__ void solve_problem(const DevProblem &P, DevResult &R, double tol, int check_every,
                              long long max_sweeps, int inner, bool refine, int cap_n, const BatchLimits &L,
                              int rank, double *smem, double *slot) {
    constexpr int VT = THREADS * CS;
    const int vt = rank * THREADS + (int)threadIdx.x;
    const unsigned long long t0 = globaltimer();
    if (rank == 0 && threadIdx.x == 0 && L.t_first) atomicMin(L.t_first, t0);
    if (cap_n > 0) {
        const double frac = ((double)P.n * P.n) / ((double)cap_n * cap_n);
        max_sweeps = max(1LL, (long long)(frac * (double)max_sweeps));
    }
    const double den2 = team_sum<THREADS, CS>(rhs_norm2_partial<VT>(P, vt), smem, slot);
    double r2, mx;
    block_residual<VT, CS, false>(P, 1.0, r2, mx, vt);
    r2 = team_sum<THREADS, CS>(r2, smem, slot);
    mx = team_max<THREADS, CS>(mx, smem, slot);
    double rho = rho_of(r2, den2);
    long long done = 0;
    double best = rho;
    int since_best = 0;
    bool stalled = false;
    bool spent = budget_spent<THREADS, CS>(L, rank, smem, slot);
    while (!(rho <= tol) && done < max_sweeps && isfinite(rho) && !stalled && !spent) {
        if (!refine) {
            long long k = check_every;
            if (k > max_sweeps - done) k = max_sweeps - done;
            for (long long it = 0; it < k; ++it) {
                block_half_sweep_f64<0, VT, CS>(P, vt);
                team_sync<CS>();
                block_half_sweep_f64<1, VT, CS>(P, vt);
                team_sync<CS>();
            }
            done += k;
        } else {
            int e = 0;
            frexp(mx, &e);
            const double down = ldexp(1.0, -e), up = ldexp(1.0, e);
            double t2, tm;
            block_residual<VT, CS, true>(P, down, t2, tm, vt);  // writes the scaled defect
            const size_t elems = (size_t)(P.n + 2) * P.W32;
            for (size_t q = vt; q < elems; q += VT) {
                P.d[0][q] = 0.0f;
                P.d[1][q] = 0.0f;
            }
            team_sync<CS>();
            long long k = inner;
            if (k > max_sweeps - done) k = max_sweeps - done;
            for (long long it = 0; it < k; ++it) {
                block_half_sweep_f32<0, VT, CS>(P, vt);
                team_sync<CS>();
                block_half_sweep_f32<1, VT, CS>(P, vt);
                team_sync<CS>();
            }
            // u += (double)d * 2^e at interior points
            const int n = P.n, kact = kact_of(n);
            for (int c = 0; c < 2; ++c) {
                for (int q = vt; q < n * kact; q += VT) {
                    const int i = 1 + q / kact, kk = q % kact;
                    const int j = 2 * kk + ((i + c) & 1);
                    if (j < 1 || j > n) continue;
                    double *uu = P.u[c] + (size_t)i * P.W + kk;
                    *uu = __dadd_rn(ldt<CS>(uu), __dmul_rn((double)ldt<CS>(P.d[c] + (size_t)i * P.W32 + kk), up));
                }
            }
            team_sync<CS>();
            done += k;
        }
        // after FP64 sweeps the black rt is zero; the refinement's correction moves every point
        block_residual<VT, CS, false>(P, 1.0, r2, mx, vt, refine ? 2 : 1);
        r2 = team_sum<THREADS, CS>(r2, smem, slot);
        mx = team_max<THREADS, CS>(mx, smem, slot);
        rho = rho_of(r2, den2);
        // rho, best and since_best are the same in every thread of the team
        if (rho < best) {
            best = rho;
            since_best = 0;
        } else if (L.stall_limit > 0 && ++since_best >= L.stall_limit) {
            stalled = true;
        }
        spent = budget_spent<THREADS, CS>(L, rank, smem, slot);
    }
    if (rank == 0 && threadIdx.x == 0) {
        R.status = !isfinite(rho) ? RBGS_ENONFINITE
                   : rho <= tol   ? RBGS_OK
                   : spent        ? RBGS_ETIMEOUT
                                  : RBGS_ENOTCONV;
        R.sweeps = done;
        R.rel = rho;
        R.t_start = t0;
        R.t_end = globaltimer();
    }
}

// Persistent solver over problems order[0 .. nprob).  The first nteam of them (the
// largest) are solved by teams of CS blocks: block rank 0 of a cluster claims the next one
// from queues[0] and the cluster solves it together.  After that every block claims the
// rest one at a time from queues[1] and solves each on its own; no block waits on a block
// outside its cluster, and a cluster's blocks part only after their last team barrier.
template <int THREADS, int CS>
__global__ void __launch_bounds__(THREADS)
batched_persistent_kernel(const DevProblem *__restrict__ probs, DevResult *__restrict__ res,
                          const int *__restrict__ order, int nprob, int nteam, int *queues, double tol,
                          int check_every, long long max_sweeps, int inner, int refine, int cap_n,
                          const BatchLimits L) {
    __shared__ double smem[THREADS / 32 + 1];
    __shared__ double slot;
    __shared__ int s_q;
    if (CS > 1) {
        const int rank = cluster_rank();
        for (;;) {
            if (rank == 0 && threadIdx.x == 0) s_q = atomicAdd(&queues[0], 1);
            team_sync<CS>();
            const int q = ld_dsmem(&s_q, 0);
            team_sync<CS>();  // every block has read the claim before it is replaced
            if (q >= nteam) break;
            const int p = order[q];
            const DevProblem P = probs[p];
            solve_problem<THREADS, CS>(P, res[p], tol, check_every, max_sweeps, inner, refine != 0, cap_n, L,
                                       rank, smem, &slot);
        }
    }
    for (;;) {
        if (threadIdx.x == 0) s_q = atomicAdd(&queues[1], 1);
        __syncthreads();
        const int q = (CS > 1 ? nteam : 0) + s_q;
        __syncthreads();
        if (q >= nprob) break;
        const int p = order[q];
        const DevProblem P = probs[p];
        solve_problem<THREADS, 1>(P, res[p], tol, check_every, max_sweeps, inner, refine != 0, cap_n, L, 0,
                                  smem, &slot);
        __syncthreads();
    }
}

// Pack every problem's natural-layout inputs into its colour-split arrays (blockIdx.z =
// problem) and unpack the solutions afterwards.
__global__ void batch_pack_kernel(const DevProblem *__restrict__ probs) {
    const DevProblem P = probs[blockIdx.z];
    const int n = P.n, W = P.W, ld = n + 2;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= W) return;
    for (int i = blockIdx.y; i < n + 2; i += gridDim.y) {
        const int j = 2 * k;
        const double a = (j <= n + 1) ? P.u_nat[(size_t)i * ld + j] : 0.0;
        const double b = (j + 1 <= n + 1) ? P.u_nat[(size_t)i * ld + j + 1] : 0.0;
        double *ev = (i & 1) ? P.u[1] : P.u[0];
        double *od = (i & 1) ? P.u[0] : P.u[1];
        ev[(size_t)i * W + k] = a;
        od[(size_t)i * W + k] = b;
        const bool row_in = i >= 1 && i <= n;
        const double fa = (row_in && j >= 1 && j <= n) ? __dmul_rn(P.h2, P.f_nat[(size_t)(i - 1) * n + (j - 1)]) : 0.0;
        const double fb = (row_in && j + 1 <= n) ? __dmul_rn(P.h2, P.f_nat[(size_t)(i - 1) * n + j]) : 0.0;
        double *fev = (i & 1) ? P.hf[1] : P.hf[0];
        double *fod = (i & 1) ? P.hf[0] : P.hf[1];
        fev[(size_t)i * W + k] = fa;
        fod[(size_t)i * W + k] = fb;
    }
}

__global__ void batch_unpack_kernel(const DevProblem *__restrict__ probs) {
    const DevProblem P = probs[blockIdx.z];
    const int n = P.n, W = P.W, ld = n + 2;
    const int k = blockIdx.x * blockDim.x + threadIdx.x;
    const int j = 2 * k;
    if (j > n + 1) return;
    for (int i = blockIdx.y; i < n + 2; i += gridDim.y) {
        const double *ev = (i & 1) ? P.u[1] : P.u[0];
        const double *od = (i & 1) ? P.u[0] : P.u[1];
        P.out_nat[(size_t)i * ld + j] = ev[(size_t)i * W + k];
        if (j + 1 <= n + 1) P.out_nat[(size_t)i * ld + j + 1] = od[(size_t)i * W + k];
    }
}

size_t align256(size_t x) { return (x + 255) / 256 * 256; }

bool device_readable(const void *p) {
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Launch shape of the persistent solver.  team > 1: the phased plan, all with one block of
// 1024 threads per SM: first as many full waves of the largest problems as the SMs hold,
// one block per problem; then the remaining largest problems by clusters of `team` blocks,
// and everything else one block per problem (team_waves, grid1, grid2 are filled in by
// plan_phases).
struct LaunchConfig {
    int threads;       // 256, 512 or 1024
    int blocks_per_sm;
    int team;          // 1: one phase, one block per problem
    int first = 0;     // problems (largest first) solved one per block in the first phase
    int nteam = 0;     // problems after those solved by teams in the second phase
    int grid1 = 0, grid2 = 0;
};

template <int THREADS, int CS>
rbgs_status launch_one(int grid, const DevProblem *d_probs, DevResult *d_res, const int *d_order, int nprob,
                       int nteam, int *d_queues, double tol, int check_every, long long max_sweeps, int inner,
                       int refine, int cap_n, const BatchLimits &L, cudaStream_t s) {
    RBGS_CUDA(cudaMemsetAsync(d_queues, 0, 2 * sizeof(int), s));
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(THREADS);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = CS > 1 ? 1 : 0;
    RBGS_CUDA(cudaLaunchKernelEx(&cfg, batched_persistent_kernel<THREADS, CS>, d_probs, d_res, d_order, nprob, nteam,
                                 d_queues, tol, check_every, max_sweeps, inner, refine, cap_n, L));
    return RBGS_OK;
}

// Clusters of CS blocks of 1024 threads that fit on the device at once (0 if none).
template <int CS>
int max_clusters() {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(CS * 64);
    cfg.blockDim = dim3(1024);
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = CS;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    int nc = 0;
    if (cudaOccupancyMaxActiveClusters(&nc, batched_persistent_kernel<1024, CS>, &cfg) != cudaSuccess) {
        cudaGetLastError();
        return 0;
    }
    return nc;
}

int max_clusters_of(int cs) { return cs == 2 ? max_clusters<2>() : (cs == 4 ? max_clusters<4>() : 0); }

// The phased plan for the problems in order (largest first): m = the problems at the
// largest size.  Phase one takes floor(m / sms) * sms of them, one block per SM each;
// phase two gives the remaining ones to clusters of `team` blocks and the rest to single
// blocks.
void plan_phases(LaunchConfig &lc, const std::vector<int> &sizes_desc, int sms) {
    const int nmax = sizes_desc.empty() ? 0 : sizes_desc[0];
    int m = 0;
    while (m < (int)sizes_desc.size() && sizes_desc[m] == nmax) ++m;
    lc.first = (m / sms) * sms;
    lc.nteam = m - lc.first;
    lc.grid1 = sms;
    const int nc = max_clusters_of(lc.team);
    lc.grid2 = lc.team * std::max(1, nc);
}

rbgs_status launch_persistent(const LaunchConfig &lc, int sms, const DevProblem *d_probs, DevResult *d_res,
                              const int *d_order, int nprob, int *d_queues, double tol, int check_every,
                              long long max_sweeps, int inner, int refine, int cap_n, const BatchLimits &L,
                              cudaStream_t s) {
    if (lc.team > 1) {
        rbgs_status st = RBGS_OK;
        if (lc.first > 0)
            st = launch_one<1024, 1>(lc.grid1, d_probs, d_res, d_order, lc.first, 0, d_queues, tol, check_every,
                                     max_sweeps, inner, refine, cap_n, L, s);
        if (st != RBGS_OK || lc.first >= nprob) return st;
        const int *rest = d_order + lc.first;
        const int nrest = nprob - lc.first;
        if (lc.team == 2)
            return launch_one<1024, 2>(lc.grid2, d_probs, d_res, rest, nrest, lc.nteam, d_queues, tol, check_every,
                                       max_sweeps, inner, refine, cap_n, L, s);
        return launch_one<1024, 4>(lc.grid2, d_probs, d_res, rest, nrest, lc.nteam, d_queues, tol, check_every,
                                   max_sweeps, inner, refine, cap_n, L, s);
    }
    const int grid = std::max(1, std::min(nprob, sms * lc.blocks_per_sm));
    switch (lc.threads) {
    case 256:
        return launch_one<256, 1>(grid, d_probs, d_res, d_order, nprob, 0, d_queues, tol, check_every, max_sweeps,
                                  inner, refine, cap_n, L, s);
    case 512:
        return launch_one<512, 1>(grid, d_probs, d_res, d_order, nprob, 0, d_queues, tol, check_every, max_sweeps,
                                  inner, refine, cap_n, L, s);
    default:
        return launch_one<1024, 1>(grid, d_probs, d_res, d_order, nprob, 0, d_queues, tol, check_every, max_sweeps,
                                   inner, refine, cap_n, L, s);
    }
}

// Autotuner: block size and blocks per SM for the persistent kernel, and the phased plan
// with clusters of 2 or 4 blocks per large problem.  The iterate of every problem is the
// same under all of them; each candidate runs a probe of the real batch (after which the
// problems are re-packed), the fastest wins.  Cached per process by (device, precision,
// team option, sizes).
struct TuneKey {
    int device, refine, team;
    std::vector<int> sizes;
    bool operator==(const TuneKey &o) const {
        return device == o.device && refine == o.refine && team == o.team && sizes == o.sizes;
    }
};
std::mutex g_tune_mutex;
thread_local LaunchConfig g_last_shape{0, 0, 0};
std::vector<std::pair<TuneKey, LaunchConfig>> g_tune_cache;

}  // namespace
}  // namespace rbgs

using namespace rbgs;

extern "C" rbgs_status rbgs_solve_batched(int nprob, const rbgs_problem *probs, double tol,
                                          const rbgs_opts *opts, void *cuda_stream, double **u_out,
                                          rbgs_result *res) {
    clear_error();
    if (nprob < 0 || (nprob > 0 && (!probs || !u_out || !res))) {
        set_error("bad batched arguments");
        return RBGS_EINVAL;
    }
    if (!(tol >= 0.0)) { set_error("tol must be >= 0"); return RBGS_EINVAL; }
    if (nprob == 0) return RBGS_OK;
    rbgs_opts o;
    rbgs_default_opts(&o);
    if (opts) o = *opts;
    if (o.check_every <= 0) o.check_every = 100;
    if (o.max_sweeps <= 0) o.max_sweeps = 1000000000L;
    const int inner = o.inner_sweeps > 0 ? o.inner_sweeps : 100;
    const int refine = o.precision == RBGS_FP32_REFINE ? 1 : 0;
    if (o.precision != RBGS_FP64 && o.precision != RBGS_FP32_REFINE) {
        set_error("unknown precision %d", o.precision);
        return RBGS_EINVAL;
    }
    if (o.stall_checks < -1) {
        set_error("stall_checks must be >= -1");
        return RBGS_EINVAL;
    }
    if (!(o.max_seconds >= 0.0) || !std::isfinite(o.max_seconds) || o.max_seconds > 1e9) {
        set_error("max_seconds must be finite, >= 0 and at most 1e9");
        return RBGS_EINVAL;
    }
    for (int p = 0; p < nprob; ++p) {
        if (probs[p].n < 1 || probs[p].n > 32768 || !(probs[p].h2 > 0.0) || !probs[p].f || !probs[p].u_init || !u_out[p]) {
            set_error("problem %d: n must be in 1..32768, h2 > 0, pointers non-NULL", p);
            return RBGS_EINVAL;
        }
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int device = 0, sms = 0;
    RBGS_CUDA(cudaGetDevice(&device));
    RBGS_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));

    // ---- device pool: colour-split state per problem + natural staging where needed
    std::vector<DevProblem> hp(nprob);
    std::vector<size_t> off_u(nprob), off_nat_f(nprob), off_nat_u(nprob), off_out(nprob);
    size_t total = 0;
    for (int p = 0; p < nprob; ++p) {
        const int n = probs[p].n;
        const int W = colour_width(n), W32 = colour_width_bytes(n, 4);
        const size_t c64 = align256((size_t)(n + 2) * W * sizeof(double));
        const size_t c32 = align256((size_t)(n + 2) * W32 * sizeof(float));
        off_u[p] = total;
        total += 4 * c64 + (refine ? 4 * c32 : 0);
        const size_t natf = align256((size_t)n * n * sizeof(double));
        const size_t natu = align256((size_t)(n + 2) * (n + 2) * sizeof(double));
        off_nat_f[p] = device_readable(probs[p].f) ? (size_t)-1 : (total += natf, total - natf);
        off_nat_u[p] = device_readable(probs[p].u_init) ? (size_t)-1 : (total += natu, total - natu);
        off_out[p] = device_readable(u_out[p]) ? (size_t)-1 : (total += natu, total - natu);
        hp[p].n = n;
        hp[p].W = W;
        hp[p].W32 = W32;
        hp[p].h2 = probs[p].h2;
    }
    char *pool = nullptr;
    if (cudaMalloc(&pool, total) != cudaSuccess) {
        cudaGetLastError();
        set_error("batched pool allocation of %zu bytes failed", total);
        return RBGS_ENOMEM;
    }
    DevProblem *d_probs = nullptr;
    DevResult *d_res = nullptr;
    int *d_order = nullptr, *d_queue = nullptr;
    unsigned long long *d_tfirst = nullptr;
    rbgs_status st = RBGS_OK;
    auto fail_cuda = [&](cudaError_t e, const char *what) {
        if (e != cudaSuccess && st == RBGS_OK) {
            set_error("%s: %s", what, cudaGetErrorString(e));
            st = RBGS_ECUDA;
        }
    };
    fail_cuda(cudaMalloc(&d_probs, nprob * sizeof(DevProblem)), "cudaMalloc");
    fail_cuda(cudaMalloc(&d_res, nprob * sizeof(DevResult)), "cudaMalloc");
    fail_cuda(cudaMalloc(&d_order, nprob * sizeof(int)), "cudaMalloc");
    fail_cuda(cudaMalloc(&d_queue, 2 * sizeof(int)), "cudaMalloc");
    fail_cuda(cudaMalloc(&d_tfirst, sizeof(unsigned long long)), "cudaMalloc");
    // the solve's limits (the autotuner's probes run without them: a fixed sweep count)
    const BatchLimits limits{o.stall_checks == 0 ? 64 : o.stall_checks,
                             (unsigned long long)(o.max_seconds * 1e9), d_tfirst};
    const BatchLimits probe_limits{-1, 0ull, nullptr};
    if (st == RBGS_OK) fail_cuda(cudaMemsetAsync(pool, 0, total, s), "cudaMemsetAsync");
    for (int p = 0; p < nprob && st == RBGS_OK; ++p) {
        const int n = probs[p].n;
        const size_t c64 = align256((size_t)(n + 2) * hp[p].W * sizeof(double));
        const size_t c32 = align256((size_t)(n + 2) * hp[p].W32 * sizeof(float));
        char *b = pool + off_u[p];
        hp[p].u[0] = (double *)b;
        hp[p].u[1] = (double *)(b + c64);
        hp[p].hf[0] = (double *)(b + 2 * c64);
        hp[p].hf[1] = (double *)(b + 3 * c64);
        hp[p].d[0] = refine ? (float *)(b + 4 * c64) : nullptr;
        hp[p].d[1] = refine ? (float *)(b + 4 * c64 + c32) : nullptr;
        hp[p].r[0] = refine ? (float *)(b + 4 * c64 + 2 * c32) : nullptr;
        hp[p].r[1] = refine ? (float *)(b + 4 * c64 + 3 * c32) : nullptr;
        if (off_nat_f[p] == (size_t)-1) {
            hp[p].f_nat = probs[p].f;
        } else {
            hp[p].f_nat = (const double *)(pool + off_nat_f[p]);
            fail_cuda(cudaMemcpyAsync(pool + off_nat_f[p], probs[p].f, (size_t)n * n * sizeof(double),
                                      cudaMemcpyDefault, s), "cudaMemcpyAsync");
        }
        if (off_nat_u[p] == (size_t)-1) {
            hp[p].u_nat = probs[p].u_init;
        } else {
            hp[p].u_nat = (const double *)(pool + off_nat_u[p]);
            fail_cuda(cudaMemcpyAsync(pool + off_nat_u[p], probs[p].u_init, (size_t)(n + 2) * (n + 2) * sizeof(double),
                                      cudaMemcpyDefault, s), "cudaMemcpyAsync");
        }
        hp[p].out_nat = off_out[p] == (size_t)-1 ? u_out[p] : (double *)(pool + off_out[p]);
    }
    // largest problems first (longest-processing-time order balances the blocks)
    std::vector<int> order(nprob);
    std::iota(order.begin(), order.end(), 0);
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return probs[a].n > probs[b].n; });
    int maxW = 0, maxRows = 0;
    for (int p = 0; p < nprob; ++p) {
        maxW = std::max(maxW, hp[p].W);
        maxRows = std::max(maxRows, hp[p].n + 2);
    }
    if (st == RBGS_OK) fail_cuda(cudaMemcpyAsync(d_probs, hp.data(), nprob * sizeof(DevProblem), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
    if (st == RBGS_OK) fail_cuda(cudaMemcpyAsync(d_order, order.data(), nprob * sizeof(int), cudaMemcpyHostToDevice, s), "cudaMemcpyAsync");
    const dim3 pgrid((maxW + 255) / 256, std::min(maxRows, 64), nprob);

    // ---- autotune the launch shape (per process, per device/precision/size mix/team option)
    std::vector<int> sizes_desc(nprob);
    for (int q = 0; q < nprob; ++q) sizes_desc[q] = probs[order[q]].n;
    LaunchConfig lc{1024, 1, 1};
    if (st == RBGS_OK && nprob > 65535) { set_error("at most 65535 problems per batch"); st = RBGS_EINVAL; }
    if (st == RBGS_OK && o.team_size != 0 && o.team_size != 1 && o.team_size != 2 && o.team_size != 4) {
        set_error("team_size must be 0, 1, 2 or 4");
        st = RBGS_EINVAL;
    }
    if (st == RBGS_OK && o.team_size > 1) {
        // explicit request: the phased plan with clusters of team_size blocks
        lc = LaunchConfig{1024, 1, o.team_size};
        if (max_clusters_of(o.team_size) < 1) {
            set_error("clusters of %d blocks of 1024 threads do not fit on this device", o.team_size);
            st = RBGS_EINVAL;
        } else {
            plan_phases(lc, sizes_desc, sms);
        }
    } else if (st == RBGS_OK) {
        TuneKey key{device, refine, o.team_size, {}};
        for (int p = 0; p < nprob; ++p) key.sizes.push_back(probs[p].n);
        std::sort(key.sizes.begin(), key.sizes.end());
        bool found = false;
        {
            std::lock_guard<std::mutex> lock(g_tune_mutex);
            for (auto &e : g_tune_cache)
                if (e.first == key) { lc = e.second; found = true; }
        }
        const bool tune = o.tile_rows == 0 && !found;
        if (o.tile_rows > 0) {
            // explicit request: tile_rows selects the block size, tblock_k the blocks per SM
            lc.threads = o.tile_rows >= 1024 ? 1024 : (o.tile_rows >= 512 ? 512 : 256);
            lc.blocks_per_sm = o.tblock_k > 0 ? o.tblock_k : 1;
        }
        if (tune) {
            std::vector<LaunchConfig> cands = {{1024, 1, 1}, {512, 2, 1}, {512, 1, 1}, {256, 4, 1}, {256, 2, 1}};
            if (o.team_size == 0) {
                for (int cs : {2, 4}) {
                    if (max_clusters_of(cs) < 1) continue;
                    LaunchConfig c{1024, 1, cs};
                    plan_phases(c, sizes_desc, sms);
                    cands.push_back(c);
                }
            }
            cudaEvent_t e0, e1;
            fail_cuda(cudaEventCreate(&e0), "cudaEventCreate");
            fail_cuda(cudaEventCreate(&e1), "cudaEventCreate");
            float best = 1e30f;
            // each probe runs the largest problems `probe` sweeps and a problem of size n
            // probe * (n / n_max)^2 (at least one), so that its work grows like n^4, as in
            // a solve to tolerance, and the probe sees the real load balance.  The refined
            // form probes one whole outer step (FP64 residual, `inner` FP32 sweeps,
            // correction), the unit its solves repeat.
            const long long probe = refine ? std::min<long long>(inner, 256) : 32;
            for (const LaunchConfig &cand : cands) {
                if (st != RBGS_OK) break;
                batch_pack_kernel<<<pgrid, 256, 0, s>>>(d_probs);
                fail_cuda(cudaGetLastError(), "pack launch");
                fail_cuda(cudaEventRecord(e0, s), "cudaEventRecord");
                // tol < 0 is never reached: every problem runs its probe sweeps
                if (st == RBGS_OK)
                    st = launch_persistent(cand, sms, d_probs, d_res, d_order, nprob, d_queue, -1.0,
                                           (int)probe, probe, (int)probe, refine, sizes_desc[0], probe_limits, s);
                fail_cuda(cudaEventRecord(e1, s), "cudaEventRecord");
                fail_cuda(cudaEventSynchronize(e1), "cudaEventSynchronize");
                float ms = 0.f;
                fail_cuda(cudaEventElapsedTime(&ms, e0, e1), "cudaEventElapsedTime");
                if (st == RBGS_OK && ms < best) {
                    best = ms;
                    lc = cand;
                }
            }
            cudaEventDestroy(e0);
            cudaEventDestroy(e1);
            if (st == RBGS_OK) {
                std::lock_guard<std::mutex> lock(g_tune_mutex);
                g_tune_cache.push_back({key, lc});
            }
        }
    }
    g_last_shape = lc;

    // ---- the batch: pack -> persistent solve -> unpack, captured as one CUDA graph
    if (st == RBGS_OK) {
        cudaStream_t cap = nullptr;
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        fail_cuda(cudaStreamCreateWithFlags(&cap, cudaStreamNonBlocking), "cudaStreamCreate");
        if (st == RBGS_OK) fail_cuda(cudaStreamBeginCapture(cap, cudaStreamCaptureModeThreadLocal), "capture");
        if (st == RBGS_OK) {
            batch_pack_kernel<<<pgrid, 256, 0, cap>>>(d_probs);
            fail_cuda(cudaGetLastError(), "pack launch");
            fail_cuda(cudaMemsetAsync(d_tfirst, 0xFF, sizeof(unsigned long long), cap), "cudaMemsetAsync");
            rbgs_status ls = launch_persistent(lc, sms, d_probs, d_res, d_order, nprob, d_queue, tol,
                                               o.check_every, o.max_sweeps, inner, refine, 0, limits, cap);
            if (ls != RBGS_OK && st == RBGS_OK) st = ls;
            batch_unpack_kernel<<<pgrid, 256, 0, cap>>>(d_probs);
            fail_cuda(cudaGetLastError(), "unpack launch");
            cudaError_t e = cudaStreamEndCapture(cap, &graph);
            fail_cuda(e, "end capture");
        }
        if (st == RBGS_OK) fail_cuda(cudaGraphInstantiate(&exec, graph, 0), "graph instantiate");
        if (st == RBGS_OK) fail_cuda(cudaGraphLaunch(exec, s), "graph launch");
        if (exec) cudaGraphExecDestroy(exec);
        if (graph) cudaGraphDestroy(graph);
        if (cap) cudaStreamDestroy(cap);
    }
    // ---- results and host outputs
    std::vector<DevResult> hr(nprob);
    if (st == RBGS_OK) fail_cuda(cudaMemcpyAsync(hr.data(), d_res, nprob * sizeof(DevResult), cudaMemcpyDeviceToHost, s), "cudaMemcpyAsync");
    for (int p = 0; p < nprob && st == RBGS_OK; ++p) {
        if (off_out[p] != (size_t)-1)
            fail_cuda(cudaMemcpyAsync(u_out[p], pool + off_out[p], (size_t)(probs[p].n + 2) * (probs[p].n + 2) * sizeof(double),
                                      cudaMemcpyDefault, s), "cudaMemcpyAsync");
    }
    fail_cuda(cudaStreamSynchronize(s), "cudaStreamSynchronize");
    rbgs_status first = st;
    if (st == RBGS_OK) {
        unsigned long long t_begin = ~0ull;
        for (int p = 0; p < nprob; ++p) t_begin = std::min(t_begin, hr[p].t_start);
        for (int p = 0; p < nprob; ++p) {
            res[p].status = hr[p].status;
            res[p].sweeps = (long)hr[p].sweeps;
            res[p].rel = hr[p].rel;
            res[p].latency_ms = (double)(hr[p].t_end - t_begin) * 1e-6;
            if (hr[p].status != RBGS_OK && first == RBGS_OK) {
                first = (rbgs_status)hr[p].status;
                set_error("problem %d: status %d after %lld sweeps (rho = %.3e)", p, hr[p].status,
                          hr[p].sweeps, hr[p].rel);
            }
        }
    }
    cudaFree(pool);
    cudaFree(d_probs);
    cudaFree(d_res);
    cudaFree(d_order);
    cudaFree(d_queue);
    cudaFree(d_tfirst);
    return first;
}

extern "C" void rbgs_batched_last_shape(int *threads, int *blocks_per_sm, int *team, int *first, int *nteam) {
    if (threads) *threads = g_last_shape.threads;
    if (blocks_per_sm) *blocks_per_sm = g_last_shape.blocks_per_sm;
    if (team) *team = g_last_shape.team;
    if (first) *first = g_last_shape.first;
    if (nteam) *nteam = g_last_shape.nteam;
}
