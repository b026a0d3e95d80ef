// Temporally blocked sweeps as a register wavefront: K sweeps (2K half-sweeps of Eq. (1),
// red then black as in Algorithm 1) per pass over memory, with the iterate of a strip
// held in registers while a warp marches down the grid.
//
// Wavefront.  Half-sweep h (h = 1..2K; odd h red, even h black) of row i needs half-sweep
// h-1 of rows i-1, i, i+1.  So at step t a warp applies half-sweep h to row t-h+1 for
// h = 1, 2, ..., 2K in that order: half-sweep h-1 has just reached row t-h+2, and
// half-sweep h+1 has not yet touched row t-h.  Row t-2K+1 is then final and is stored.
// The live rows of the iterate (t-2K .. t+3, loaded three steps ahead) sit in a ring of
// 2K+4 register slots; the step loop is unrolled over the ring so every slot index is a
// compile-time constant.  The live rows of h2f (t-2K+1 .. t+2) sit in a ring of the same
// slots in shared memory, filled by cp.async three steps ahead (which frees the registers
// for more resident warps).  Rows of the iterate further ahead are prefetched into L1.
//
// Decomposition.  A warp owns a strip of 64 values of each colour row (2 per lane) and a
// segment of rows.  The west/east neighbour across lanes comes by shuffle; at the strip's
// edges it is wrong, and the damage moves inward by at most K values of a colour row over
// the 2K half-sweeps (checked by simulation), so each strip stores only its middle
// 64 - 2H values (H = K rounded up to even) and neighbouring strips overlap by 2H.  In
// the same way a segment that outputs rows [a, b) starts marching 2K rows above a and
// runs 2K-1 rows past b.  The ring rows and columns are copied through, so the output
// buffer receives a complete iterate and the pass ends by swapping it with the input.
//
// Arithmetic is the library's update, (((h2f + N) + S) + W) + E times 0.25, each step
// correctly rounded, so a pass equals K one-launch-per-colour sweeps bit for bit.
// Traffic per pass: the iterate read and written once and h2f read once (plus the
// overlaps): 12 bytes per point per K sweeps in FP32, 24 in FP64.
#include <type_traits>

#include "common.cuh"
#include "fp64.cuh"
#include "sweep_impl.cuh"

namespace rbgs {
namespace {

constexpr int kWfWarps = 4;  // warps per block; each warp is an independent work item
constexpr int kWfThreads = 32 * kWfWarps;
constexpr int kWfPrefetch = 4;  // rows ahead of the loads that are prefetched into L1
constexpr int kWfP = 2;         // values of each colour per lane

template <typename T>
struct WfArgs {
    const T *u0, *u1;    // input iterate (red, black)
    const T *hf0, *hf1;  // right-hand-side term
    T *o0, *o1;          // output iterate
    int n, W, kmax;        // kmax: values of a colour row holding columns 0..n+1
    int strips, ow, halo;  // strip: values computed 32 P, stored ow, overlap halo per side
    int seg_h, items;      // rows per segment (even), work items = strips x segments
    double one;            // 1.0, for the FP64 update's fma form
};

__device__ __forceinline__ float wf_update(float hf, float vn, float vs, float vw, float ve, double) {
    float s = __fadd_rn(hf, vn);
    s = __fadd_rn(s, vs);
    s = __fadd_rn(s, vw);
    s = __fadd_rn(s, ve);
    return __fmul_rn(s, 0.25f);
}

__device__ __forceinline__ double wf_update(double hf, double vn, double vs, double vw, double ve, double one) {
    return update_f64<false>(0, hf, vn, vs, vw, ve, one);
}

// the lane's 2 values of one colour row
__device__ __forceinline__ void wf_load(float *v, const float *p) {
    const float2 t = __ldg(reinterpret_cast<const float2 *>(p));
    v[0] = t.x, v[1] = t.y;
}

__device__ __forceinline__ void wf_load(double *v, const double *p) {
    const double2 t = __ldg(reinterpret_cast<const double2 *>(p));
    v[0] = t.x, v[1] = t.y;
}

__device__ __forceinline__ void wf_load_shared(float *v, const float *p) {
    const float2 t = *reinterpret_cast<const float2 *>(p);
    v[0] = t.x, v[1] = t.y;
}

__device__ __forceinline__ void wf_load_shared(double *v, const double *p) {
    const double2 t = *reinterpret_cast<const double2 *>(p);
    v[0] = t.x, v[1] = t.y;
}

__device__ __forceinline__ void wf_store(float *p, const float *v) {
    *reinterpret_cast<float2 *>(p) = make_float2(v[0], v[1]);
}

__device__ __forceinline__ void wf_store(double *p, const double *v) {
    *reinterpret_cast<double2 *>(p) = make_double2(v[0], v[1]);
}

// cp.async of the lane's 2 values (8 or 16 bytes) into shared memory; src_valid = false
// fills zeros without reading
template <typename T>
__device__ __forceinline__ void wf_cp_async(T *dst, const T *src, bool src_valid) {
    const uint32_t d = static_cast<uint32_t>(__cvta_generic_to_shared(dst));
    if (sizeof(T) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8, %2;" ::"r"(d), "l"(src), "r"(src_valid ? 8 : 0)
                     : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(d), "l"(src), "r"(src_valid ? 16 : 0)
                     : "memory");
}

__device__ __forceinline__ void wf_cp_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

__device__ __forceinline__ void wf_cp_wait3() { asm volatile("cp.async.wait_group 3;" ::: "memory"); }

__device__ __forceinline__ void wf_prefetch(const void *p) {
    asm volatile("prefetch.global.L1 [%0];" ::"l"(p));
}

// Ring of WS = 2K + 4 row slots, for the iterate (registers) and h2f (shared memory) alike.  With t_s the first
// step and rho(i) = i - t_s + 2K, row i lives in slot rho(i) mod WS.  At step t (t - t_s =
// u mod WS): the iterate's row t+3 is loaded into slot u-1, h2f's row t+3 into slot u-1,
// half-sweep h works on row t-h+1 in slot u-3-h (its neighbours in the slots on either
// side), and row t-2K+1 (slot u+1) is stored.  A slot is refilled only after its row's
// last use: the iterate's row i is last read at step i+2K, h2f's at step i+2K-1.
template <typename T, int K>
__global__ void __launch_bounds__(kWfThreads) wavefront_kernel(const WfArgs<T> a) {
    constexpr int P = kWfP;
    constexpr int WS = 2 * K + 4;
    const int wid = blockIdx.x * kWfWarps + (threadIdx.x >> 5);
    if (wid >= a.items) return;  // whole warps only
    const int lane = threadIdx.x & 31;
    const int n = a.n, W = a.W;
    const int strip = wid % a.strips, seg = wid / a.strips;
    const int ks = strip * a.ow - a.halo;
    const int k0 = ks + lane * P;  // a multiple of P
    // lanes outside the grid's columns hold 1.0 (any finite non-zero value: their results
    // are discarded, and 1.0 keeps the FP64 quarter on its exponent path)
    const bool kin = k0 >= 0 && k0 < a.kmax;
    unsigned msk0 = 0, msk1 = 0;  // interior columns for row parity offset 0 / 1
#pragma unroll
    for (int q = 0; q < P; ++q) {
        const int j = 2 * (k0 + q);
        if (kin && j >= 1 && j <= n) msk0 |= 1u << q;
        if (kin && j + 1 >= 1 && j + 1 <= n) msk1 |= 1u << q;
    }
    const int olo = max(ks + a.halo, 0), ohi = min(ks + a.halo + a.ow, a.kmax);
    const int row_a = seg * a.seg_h, row_b = min(row_a + a.seg_h, n + 2);
    const int t_s = row_a - 2 * K;  // even: row parities below are compile-time constants
    const int t_e = min(row_b + 2 * K - 2, n + 2 * K);

    // the iterate's ring in registers; h2f's ring in shared memory, filled by cp.async and
    // read back by the lane that copied it (no barrier: each lane reads its own bytes)
    T uw[WS][2][P];
    __shared__ __align__(16) T fsm[kWfWarps][WS][2][32 * P];
    T(*fw)[2][32 * P] = fsm[threadIdx.x >> 5];
    auto load_f = [&](int slot, int r) {
        const bool ok = kin && r >= 0 && r <= n + 1;
        const size_t off = ok ? (size_t)r * W + k0 : 0;
        wf_cp_async(&fw[slot][0][lane * P], a.hf0 + off, ok);
        wf_cp_async(&fw[slot][1][lane * P], a.hf1 + off, ok);
    };
    auto load2 = [&](T (&dst)[2][P], const T *p0, const T *p1, int r) {
        if (kin && r >= 0 && r <= n + 1) {
            wf_load(dst[0], p0 + (size_t)r * W + k0);
            wf_load(dst[1], p1 + (size_t)r * W + k0);
        } else {
#pragma unroll
            for (int q = 0; q < P; ++q) dst[0][q] = dst[1][q] = T(1);
        }
    };
    auto prefetch2 = [&](const T *p0, const T *p1, int r) {
        if (kin && r >= 0 && r <= n + 1) {
            wf_prefetch(p0 + (size_t)r * W + k0);
            wf_prefetch(p1 + (size_t)r * W + k0);
        }
    };
    // rows t_s - 2K .. t_s + 2 of the iterate, t_s - 2K + 1 .. t_s + 2 of h2f
#pragma unroll
    for (int r = 0; r <= 2 * K + 2; ++r) load2(uw[r], a.u0, a.u1, t_s - 2 * K + r);
#pragma unroll
    for (int r = 1; r <= 2 * K + 2; ++r) load_f(r, t_s - 2 * K + r);
    wf_cp_commit();
    wf_cp_commit();  // three empty groups: the first step's wait then covers the rows above
    wf_cp_commit();
    wf_cp_commit();
#pragma unroll
    for (int d = 0; d < kWfPrefetch; ++d) {
        prefetch2(a.u0, a.u1, t_s + 3 + d);
    }

    // Blocks of WS steps whose rows, loads and stores all lie inside the grid and the
    // segment, on a strip with no boundary column, run without any of those checks: every
    // lane is inside the grid's columns, and a lane either stores both of its values or
    // (in the overlap) none.
    const bool full_cols = __all_sync(0xffffffffu, msk0 == (1u << P) - 1 && msk1 == (1u << P) - 1);
    const bool store_vec = k0 >= olo && k0 + P <= ohi;
    auto run_block = [&](int base, auto fast_tag) {
        constexpr bool FAST = decltype(fast_tag)::value;
#pragma unroll
        for (int u = 0; u < WS; ++u) {
            const int t = base + u;  // t - t_s = u (mod WS), and t has the parity of u
            if (FAST || t <= t_e) {
                if (FAST) {
                    const size_t ur = (size_t)(t + 3) * W + k0;
                    wf_load(uw[(u + WS - 1) % WS][0], a.u0 + ur);
                    wf_load(uw[(u + WS - 1) % WS][1], a.u1 + ur);
                    const int fs = (u + WS - 1) % WS;
                    const size_t fr = (size_t)(t + 3) * W + k0;
                    wf_cp_async(&fw[fs][0][lane * P], a.hf0 + fr, true);
                    wf_cp_async(&fw[fs][1][lane * P], a.hf1 + fr, true);
                } else {
                    prefetch2(a.u0, a.u1, t + 3 + kWfPrefetch);
                    load2(uw[(u + WS - 1) % WS], a.u0, a.u1, t + 3);
                    load_f((u + WS - 1) % WS, t + 3);
                }
                wf_cp_commit();
                wf_cp_wait3();  // h2f rows up to t (issued three steps ago) have landed
#pragma unroll
                for (int h = 1; h <= 2 * K; ++h) {
                    const int i = t - h + 1;
                    if (FAST || (i >= 1 && i <= n)) {
                        const int c = (h - 1) & 1;          // colour updated by half-sweep h
                        const int p = (u - h + 1 + c) & 1;  // (i + c) & 1
                        const int sm = (u - 3 - h + 2 * WS) % WS;  // slot of row i
                        const int su = (sm + WS - 1) % WS, sd = (sm + 1) % WS;
                        T f[P];
                        wf_load_shared(f, &fw[sm][c][lane * P]);
                        const T *mid = uw[sm][1 - c];
                        const T *up = uw[su][1 - c];
                        const T *dn = uw[sd][1 - c];
                        T *self = uw[sm][c];
                        const unsigned msk = p ? msk1 : msk0;
                        if (p == 0) {  // west/east neighbours at k-1, k
                            const T prev = __shfl_up_sync(0xffffffffu, mid[P - 1], 1);
#pragma unroll
                            for (int q = 0; q < P; ++q) {
                                const T r = wf_update(f[q], up[q], dn[q], q ? mid[q - 1] : prev, mid[q], a.one);
                                if (FAST || ((msk >> q) & 1u)) self[q] = r;
                            }
                        } else {  // at k, k+1
                            const T next = __shfl_down_sync(0xffffffffu, mid[0], 1);
#pragma unroll
                            for (int q = 0; q < P; ++q) {
                                const T r = wf_update(f[q], up[q], dn[q], mid[q], q + 1 < P ? mid[q + 1] : next, a.one);
                                if (FAST || ((msk >> q) & 1u)) self[q] = r;
                            }
                        }
                    }
                }
                const int r = t - 2 * K + 1;  // final: every half-sweep has passed it
                if (FAST) {
                    if (store_vec) {
                        const T(&v)[2][P] = uw[(u + 1) % WS];
                        wf_store(a.o0 + (size_t)r * W + k0, v[0]);
                        wf_store(a.o1 + (size_t)r * W + k0, v[1]);
                    }
                } else if (r >= row_a && r < row_b && kin) {
                    const T(&v)[2][P] = uw[(u + 1) % WS];
                    T *d0 = a.o0 + (size_t)r * W + k0, *d1 = a.o1 + (size_t)r * W + k0;
                    if (k0 >= olo && k0 + P <= ohi) {
                        wf_store(d0, v[0]);
                        wf_store(d1, v[1]);
                    } else {
#pragma unroll
                        for (int q = 0; q < P; ++q) {
                            if (k0 + q >= olo && k0 + q < ohi) {
                                d0[q] = v[0][q];
                                d1[q] = v[1][q];
                            }
                        }
                    }
                }
            }
        }
    };
    for (int base = t_s; base <= t_e; base += WS) {
        const bool fast = full_cols && base >= 2 * K && base + WS + 2 <= n + 1 && base + WS - 1 <= t_e &&
                          base - 2 * K + 1 >= row_a && base + WS - 2 * K < row_b;
        if (fast)
            run_block(base, std::true_type{});
        else
            run_block(base, std::false_type{});
    }
}

int sm_count_wf() {
    static const int sms = [] {  // initialised once, thread-safely
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) {
            cudaGetLastError();
            v = 152;
        }
        return v;
    }();
    return sms;
}

template <typename T, int K>
rbgs_status run_wavefront(ColourField<T> &fld, cudaStream_t s) {
    constexpr int P = kWfP;
    const int n = fld.n;
    WfArgs<T> a;
    a.u0 = fld.u[0], a.u1 = fld.u[1], a.hf0 = fld.hf[0], a.hf1 = fld.hf[1];
    a.o0 = fld.alt[0], a.o1 = fld.alt[1];
    a.n = n, a.W = fld.W, a.one = 1.0;
    a.kmax = (n + 3) / 2;
    a.halo = (K + P - 1) / P * P;
    a.ow = 32 * P - 2 * a.halo;
    a.strips = (a.kmax + a.ow - 1) / a.ow;
    // segments: as many as fill the warps that can be resident at once (one wave: a
    // second, partial wave would leave most SMs idle), each at least 8K rows tall so that
    // the 4K extra rows a segment marches stay a small share
    static const int per_sm = [] {  // resident blocks per SM, per template instance
        int v = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&v, wavefront_kernel<T, K>, kWfThreads, 0) !=
                cudaSuccess ||
            v < 1) {
            cudaGetLastError();
            v = 1;
        }
        return v;
    }();
    const long capacity = (long)per_sm * kWfWarps * sm_count_wf();
    long want = capacity / a.strips;
    if (want < 1) want = 1;
    long seg = (n + 2 + want - 1) / want;
    if (seg < 8 * K) seg = 8 * K;
    if (seg > n + 2) seg = n + 2;
    seg = (seg + 1) & ~1L;
    a.seg_h = (int)seg;
    const long segs = (n + 2 + seg - 1) / seg;
    const long items = segs * a.strips;
    if (items > 0x7fffffffL / 2) {
        set_error("wavefront pass: grid too large");
        return RBGS_EINVAL;
    }
    a.items = (int)items;
    const unsigned blocks = (unsigned)((items + kWfWarps - 1) / kWfWarps);
    wavefront_kernel<T, K><<<blocks, kWfThreads, 0, s>>>(a);
    RBGS_LAUNCH_CHECK();
    for (int q = 0; q < 2; ++q) {
        T *t = fld.u[q];
        fld.u[q] = fld.alt[q];
        fld.alt[q] = t;
    }
    fld.maps_ready = false;  // tensor maps of the TMA kernel name the old buffers
    return RBGS_OK;
}

}  // namespace

template <>
rbgs_status launch_wavefront_pass<double>(ColourField<double> &fld, int k, cudaStream_t s) {
    switch (k) {
    case 2: return run_wavefront<double, 2>(fld, s);
    case 4: return run_wavefront<double, 4>(fld, s);
    default: set_error("FP64 wavefront depth must be 2 or 4 (got %d)", k); return RBGS_EINVAL;
    }
}

template <>
rbgs_status launch_wavefront_pass<float>(ColourField<float> &fld, int k, cudaStream_t s) {
    switch (k) {
    case 2: return run_wavefront<float, 2>(fld, s);
    case 4: return run_wavefront<float, 4>(fld, s);
    case 6: return run_wavefront<float, 6>(fld, s);
    default: set_error("FP32 wavefront depth must be 2, 4 or 6 (got %d)", k); return RBGS_EINVAL;
    }
}

}  // namespace rbgs
