// Convolution kernels of the learned initial guess on the 5th-generation tensor cores:
// implicit GEMM with tcgen05.mma, FP32 accumulators in tensor memory (TMEM).
//
// The three products of a convolution layer are the GEMMs listed in conv.cu, tiled here
// as (M x N output tile, K in stages of 64 bf16):
//   forward      M = pixels,     N = Cout, K = taps*Cin    A, B K-major
//   data grad    M = pixels,     N = Cin,  K = taps*Cout   A, B K-major
//   weight grad  M = taps*Cin,   N = Cout, K = pixels      A, B MN-major, K split in chunks
// (the weight gradient is formed transposed, dW^T[(t,c), o], so that the long dimension
// taps*Cin fills the 128 TMEM lanes; its partial tiles are added with FP32 atomics).
//
// Persistent, warp-specialised CTA (one per SM, 13 warps), over tiles blockIdx.x,
// blockIdx.x + gridDim.x, ...:
//   warps 0-7   producers: gather the operand tiles of each K stage with 16-byte cp.async
//               copies (zero-filled outside the image, the channels and the pixel range)
//               into a ring of shared-memory stages, then signal the stage's `full`
//               mbarrier once their copies have landed (two further stages are issued
//               before a thread waits for a stage's copies);
//   warp 8      one thread issues four 128 x bn x 16 MMAs per stage and commits them to
//               the stage's `empty` mbarrier (which frees it for the producers), and after
//               a tile's last stage to the `tfull` mbarrier of its accumulator buffer;
//   warps 9-12  epilogue: read the finished accumulator rows with tcgen05.ld (warp w owns
//               TMEM lanes 32 (w mod 4) .. +31, one output row per thread), apply bias /
//               ReLU / rounding or the atomic add, and release the buffer (`tempty`).
// Two accumulator buffers of bn TMEM columns let the MMAs of tile i+1 run while the
// epilogue drains tile i.  Every wait is bounded; a wait that gives up sets a CTA-wide
// abort flag (all roles leave their loops) and a global flag read by rbgs_conv_check.
//
// Shared-memory operand layouts (bf16, one stage = A 128 x 64 then B bn x 64):
//   K-major, 128-byte swizzle: row r of the tile is 128 bytes (64 k); its 16-byte chunk
//     c sits at chunk position c ^ (r mod 8) inside the 8-row, 1024-byte atom of rows
//     8 (r / 8) ..; descriptor SBO = 1024 B, LBO unused, K step of 16 = +32 bytes.
//   MN-major, 128-byte swizzle (weight-grad A): atoms of 8 k-rows x 64 mn; within an atom
//     k-row q holds 128 bytes of mn values with chunk c at position c ^ q; the two mn
//     atoms of a k group are 1024 B apart (LBO), k groups 2048 B apart (SBO).
//   MN-major, no swizzle (weight-grad B): core matrix (mn group i, k group j) = 8 k-rows of
//     16 bytes at (j bn/8 + i) 128; LBO (next k group) = 16 bn B, SBO (next mn group) = 128 B.
// The producer mapping puts the 8 threads of each quarter-warp on 8 different rows of
// one chunk column, so their 16-byte writes fall in 8 distinct bank groups.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <cuda_bf16.h>

#include <cstring>

#include "common.cuh"
#include "conv_wait.cuh"
#include "tma.cuh"
#include "../../include/rbgs_unet.h"

namespace rbgs {

// Set when a bounded wait of a tcgen05 convolution gave up; read and cleared by
// rbgs_conv_check.
__device__ int g_conv_wait_failed;

namespace {

constexpr int UM = 128;              // tile rows = TMEM lanes
constexpr int UK = 64;               // K per stage: 128 bytes of bf16 per row
constexpr int kProducers = 256;      // warps 0-7
constexpr int kMmaWarp = 8;
constexpr int kEpiWarp0 = 9;         // warps 9-12
constexpr int kThreads = 416;
constexpr int kMaxStages = 10;
constexpr int kLag = 2;                   // stages in flight per producer before it signals
constexpr uint32_t kPolls = 4000;          // x kSuspendNs: a wait gives up after about 4 s
constexpr uint32_t kSuspendNs = 1000000;  // each poll sleeps until the phase completes or 1 ms
constexpr uint32_t kSpinPolls = 1u << 22; // spinning polls of the issuing threads
constexpr int kMaxBn = 256;
constexpr uint32_t kRingBudget = 200 * 1024;
constexpr size_t kMaxSmem = kRingBudget + 1024;

enum UMode { U_FWD = 0, U_BWD_DATA = 1, U_BWD_WEIGHT = 2 };

// Division of 0 <= n < 2^31 by an invariant d >= 1 with a multiply-high and a shift
// (Granlund and Montgomery, "Division by invariant integers using multiplication", 1994):
// with l = ceil(log2 d) and p = 31 + l, mul = ceil(2^p / d) < 2^32 and n / d =
// (n mul) >> p, since n (mul d - 2^p) < 2^31 d <= 2^p.
struct FastDiv {
    uint32_t d, mul, shr;
};

FastDiv make_fastdiv(uint32_t d) {
    FastDiv f{d, 0u, 0u};
    if (d > 1) {
        uint32_t l = 0;
        while ((1ull << l) < d) ++l;
        const uint32_t p = 31 + l;
        f.mul = (uint32_t)(((1ull << p) + d - 1) / d);
        f.shr = p - 32;
    }
    return f;
}

__device__ __forceinline__ uint32_t fdiv(uint32_t n, const FastDiv &f) {
    return f.d == 1 ? n : (__umulhi(n, f.mul) >> f.shr);
}

struct UArgs {
    const uint16_t *X;   // NHWC bf16 activations
    const uint16_t *Wt;  // forward: [Cout][taps][Cin]; data grad: transposed [taps][Cin][Cout]
    const uint16_t *G;   // NHWC bf16 gradient of the pre-activation output
    const float *bias;
    void *out;
    int H, W, Cin, Cout, ks;
    int relu, y_fp32, accumulate;
    int M, N, K;         // GEMM sizes
    int bn, stages;
    int m_tiles, n_tiles, k_chunk, num_tiles;
    int log2_groups;     // weight grad: log2(bn / 8)
    uint32_t tmem_cols;  // power of two >= max(32, 2 bn)
    FastDiv div_w, div_hw;
};

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_addr(bar)) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor: start address, leading / stride byte offsets,
// descriptor version 1, swizzle mode (0 none, 2 = 128-byte).
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t swizzle) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46) | ((uint64_t)swizzle << 61);
}

// Instruction descriptor of kind::f16: FP32 accumulator, bf16 A and B, major-ness of each
// operand (0 K-major, 1 MN-major), N >> 3 and M >> 4.
__host__ __device__ constexpr uint32_t instr_desc(int m, int n, int a_mn, int b_mn) {
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)a_mn << 15) | ((uint32_t)b_mn << 16) |
           ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void umma_bf16(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t idesc,
                                          uint32_t accumulate) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(idesc), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void umma_commit(uint64_t *bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t *r) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, "
        "[%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
    const __nv_bfloat16 a = __float2bfloat16_rn(lo), b = __float2bfloat16_rn(hi);
    return (uint32_t)__bfloat16_as_ushort(a) | ((uint32_t)__bfloat16_as_ushort(b) << 16);
}

// The kernels' waits: suspending polls for the many-thread roles, spinning polls for the
// single issuing threads (conv_wait.cuh).  A suspending wait gives up after about 4 s, a
// spinning one after 2^22 polls, each of which blocks for a hardware-defined time slice.
__device__ __forceinline__ bool wait_or_abort(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    return rbgs::wait_or_abort(bar, parity, abort_flag, kPolls, kSuspendNs, &g_conv_wait_failed);
}

__device__ __forceinline__ bool wait_or_abort_spin(uint64_t *bar, uint32_t parity, volatile int *abort_flag) {
    return rbgs::wait_or_abort_spin(bar, parity, abort_flag, kSpinPolls, &g_conv_wait_failed);
}

struct Tile {
    int m0, n0, kbeg, kend, KT;
};

template <int MODE>
__device__ __forceinline__ Tile decode_tile(const UArgs &a, int tile) {
    Tile t;
    int rest = tile;
    t.kbeg = 0;
    t.kend = a.K;
    if (MODE == U_BWD_WEIGHT) {
        const int per = a.m_tiles * a.n_tiles;
        const int chunk = tile / per;
        rest = tile - chunk * per;
        t.kbeg = chunk * a.k_chunk;
        t.kend = min(a.K, t.kbeg + a.k_chunk);
    }
    const int mt = rest / a.n_tiles;
    t.m0 = mt * UM;
    t.n0 = (rest - mt * a.n_tiles) * a.bn;
    t.KT = (t.kend - t.kbeg + UK - 1) / UK;
    return t;
}

// ------------------------------------------------------------------ producers
template <int MODE>
__device__ void produce(const UArgs &a, uint32_t sbase, uint32_t stage_bytes, uint64_t *full_bar,
                        uint64_t *empty_bar, volatile int *abort_flag) {
    const int ptid = threadIdx.x;  // 0..255
    const int bn = a.bn, S = a.stages;
    const uint32_t a_bytes = UM * UK * 2;
    const int b_vecs = bn * 8;
    const int pad = a.ks / 2;
    const uint32_t HW = (uint32_t)a.H * (uint32_t)a.W;
    uint32_t s = 0, ph = 0, s_arr = 0;
    int issued = 0, arrived = 0;
    bool live = true;

    if (MODE != U_BWD_WEIGHT) {
        // K-major A and B: this thread fills rows 8 (rh0 + 4 it) + row_lo, chunk kc.
        const int row_lo = ptid & 7, kc = (ptid >> 3) & 7, rh0 = ptid >> 6;
        const uint32_t sw = (uint32_t)(row_lo * 128 + ((kc ^ row_lo) << 4));
        const int CK = MODE == U_FWD ? a.Cin : a.Cout;
        const uint16_t *src = MODE == U_FWD ? a.X : a.G;
        const int t_init = (kc * 8) / CK, ch_init = kc * 8 - t_init * CK;
        const int tx_init = t_init % a.ks, ty_init = t_init / a.ks;
        for (int tile = blockIdx.x; tile < a.num_tiles && live; tile += gridDim.x) {
            const Tile T = decode_tile<MODE>(a, tile);
            int pyx[4];
            long mbase[4];
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const int m = T.m0 + (rh0 + 4 * it) * 8 + row_lo;
                if (m < a.M) {
                    const uint32_t r = (uint32_t)m - fdiv((uint32_t)m, a.div_hw) * HW;
                    const uint32_t y = fdiv(r, a.div_w);
                    pyx[it] = (int)((y << 16) | (r - y * (uint32_t)a.W));
                    mbase[it] = (long)m * CK;
                } else {
                    pyx[it] = -1;
                    mbase[it] = 0;
                }
            }
            int ch = ch_init, tx = tx_init, ty = ty_init;
            for (int kt = 0; kt < T.KT; ++kt) {
                if (!wait_or_abort(&empty_bar[s], ph ^ 1u, abort_flag)) {
                    live = false;
                    break;
                }
                const uint32_t sa = sbase + s * stage_bytes, sb = sa + a_bytes;
                const bool kval = ty < a.ks;  // tap index < taps
                int dy = ty - pad, dx = tx - pad;
                if (MODE == U_BWD_DATA) dy = -dy, dx = -dx;
                const long delta = ((long)dy * a.W + dx) * CK + ch;
#pragma unroll
                for (int it = 0; it < 4; ++it) {
                    const int yx = pyx[it];
                    const int y = (yx >> 16) + dy, x = (yx & 0xFFFF) + dx;
                    const bool ok = kval && yx >= 0 && y >= 0 && y < a.H && x >= 0 && x < a.W;
                    cp_async16(sa + (uint32_t)(rh0 + 4 * it) * 1024u + sw, ok ? src + mbase[it] + delta : src, ok);
                }
#pragma unroll
                for (int it = 0; it < kMaxBn * 8 / kProducers; ++it) {
                    const int v = ptid + kProducers * it;
                    if (v >= b_vecs) break;
                    const int n = T.n0 + (rh0 + 4 * it) * 8 + row_lo;
                    const bool ok = kval && n < a.N;
                    const uint16_t *p = a.Wt;
                    if (ok) {
                        if (MODE == U_FWD)
                            p = a.Wt + (long)n * a.K + kt * UK + kc * 8;  // Wt[o][t][c], k = t Cin + c
                        else
                            p = a.Wt + ((long)(ty * a.ks + tx) * a.Cin + n) * a.Cout + ch;  // Wt_t[t][c][o]
                    }
                    cp_async16(sb + (uint32_t)(rh0 + 4 * it) * 1024u + sw, p, ok);
                }
                cp_async_commit();
                ++issued;
                if (issued > kLag) {
                    cp_async_wait<kLag>();
                    fence_proxy_async_smem();
                    mbar_arrive(&full_bar[s_arr]);
                    ++arrived;
                    if (++s_arr == (uint32_t)S) s_arr = 0;
                }
                ch += UK;
                while (ch >= CK) {
                    ch -= CK;
                    if (++tx == a.ks) tx = 0, ++ty;
                }
                if (++s == (uint32_t)S) s = 0, ph ^= 1u;
            }
        }
    } else {
        // MN-major A (128B swizzle): mn group ig of the tile, k rows 8 (j0 + 2 it) + kr.
        const int kr = ptid & 7, ig = (ptid >> 3) & 15, j0 = ptid >> 7;
        const uint32_t a_sw = (uint32_t)((ig >> 3) * 1024 + kr * 128 + (((ig & 7) ^ kr) << 4));
        const int gmask = (1 << a.log2_groups) - 1;
        for (int tile = blockIdx.x; tile < a.num_tiles && live; tile += gridDim.x) {
            const Tile T = decode_tile<MODE>(a, tile);
            const int m = T.m0 + ig * 8;  // (t, c) of this thread's 8 rows
            const bool mval = m < a.M;
            int dy = 0, dx = 0, c = 0;
            if (mval) {
                const int t = m / a.Cin;
                c = m - t * a.Cin;
                dy = t / a.ks - pad;
                dx = t % a.ks - pad;
            }
            const long shift = ((long)dy * a.W + dx) * a.Cin + c;
            // image coordinates of the thread's 4 pixels, advanced by UK pixels per stage
            int py[4], px[4];
#pragma unroll
            for (int it = 0; it < 4; ++it) {
                const uint32_t p = (uint32_t)(T.kbeg + (j0 + 2 * it) * 8 + kr);
                const uint32_t r = p - fdiv(p, a.div_hw) * HW;
                py[it] = (int)fdiv(r, a.div_w);
                px[it] = (int)r - py[it] * a.W;
            }
            for (int kt = 0; kt < T.KT; ++kt) {
                if (!wait_or_abort(&empty_bar[s], ph ^ 1u, abort_flag)) {
                    live = false;
                    break;
                }
                const uint32_t sa = sbase + s * stage_bytes, sb = sa + a_bytes;
                const int k0 = T.kbeg + kt * UK;
#pragma unroll
                for (int it = 0; it < 4; ++it) {
                    const int p = k0 + (j0 + 2 * it) * 8 + kr;
                    const int y = py[it] + dy, x = px[it] + dx;
                    const bool ok = mval && p < T.kend && y >= 0 && y < a.H && x >= 0 && x < a.W;
                    cp_async16(sa + (uint32_t)(j0 + 2 * it) * 2048u + a_sw,
                               ok ? a.X + (long)p * a.Cin + shift : a.X, ok);
                    px[it] += UK;  // the same pixel lane of the next stage
                    while (px[it] >= a.W) {
                        px[it] -= a.W;
                        if (++py[it] == a.H) py[it] = 0;
                    }
                }
#pragma unroll
                for (int it = 0; it < kMaxBn * 8 / kProducers; ++it) {
                    const int v = ptid + kProducers * it;
                    if (v >= b_vecs) break;
                    const int g = v >> 3;
                    const int p = k0 + (g >> a.log2_groups) * 8 + (v & 7);
                    const int n = T.n0 + (g & gmask) * 8;
                    const bool ok = p < T.kend && n < a.N;
                    cp_async16(sb + (uint32_t)v * 16u, ok ? a.G + (long)p * a.Cout + n : a.G, ok);
                }
                cp_async_commit();
                ++issued;
                if (issued > kLag) {
                    cp_async_wait<kLag>();
                    fence_proxy_async_smem();
                    mbar_arrive(&full_bar[s_arr]);
                    ++arrived;
                    if (++s_arr == (uint32_t)S) s_arr = 0;
                }
                if (++s == (uint32_t)S) s = 0, ph ^= 1u;
            }
        }
    }
    cp_async_wait<0>();
    fence_proxy_async_smem();
    while (arrived < issued) {
        mbar_arrive(&full_bar[s_arr]);
        ++arrived;
        if (++s_arr == (uint32_t)S) s_arr = 0;
    }
}

// ------------------------------------------------------------------ MMA issuer
template <int MODE>
__device__ void issue_mmas(const UArgs &a, uint32_t sbase, uint32_t stage_bytes, uint32_t tmem,
                           uint64_t *full_bar, uint64_t *empty_bar, uint64_t *tfull_bar, uint64_t *tempty_bar,
                           volatile int *abort_flag) {
    constexpr bool MN = MODE == U_BWD_WEIGHT;
    const int bn = a.bn, S = a.stages;
    const uint32_t a_bytes = UM * UK * 2;
    const uint32_t idesc = instr_desc(UM, bn, MN ? 1 : 0, MN ? 1 : 0);
    uint32_t s = 0, ph = 0;
    int local = 0;
    for (int tile = blockIdx.x; tile < a.num_tiles; tile += gridDim.x, ++local) {
        const Tile T = decode_tile<MODE>(a, tile);
        const int buf = local & 1;
        if (!wait_or_abort(&tempty_bar[buf], (((uint32_t)local >> 1) & 1u) ^ 1u, abort_flag)) return;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(buf * bn);
        for (int kt = 0; kt < T.KT; ++kt) {
            if (!wait_or_abort(&full_bar[s], ph, abort_flag)) return;
            tc_fence_after();
            const uint32_t sa = sbase + s * stage_bytes, sb = sa + a_bytes;
#pragma unroll
            for (int kk = 0; kk < UK / 16; ++kk) {
                uint64_t ad, bd;
                if (!MN) {
                    ad = smem_desc(sa + kk * 32, 16, 1024, 2);
                    bd = smem_desc(sb + kk * 32, 16, 1024, 2);
                } else {
                    ad = smem_desc(sa + kk * 4096, 1024, 2048, 2);
                    bd = smem_desc(sb + kk * (uint32_t)bn * 32u, (uint32_t)bn * 16u, 128, 0);
                }
                umma_bf16(acc, ad, bd, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
            }
            umma_commit(&empty_bar[s]);
            if (++s == (uint32_t)S) s = 0, ph ^= 1u;
        }
        umma_commit(&tfull_bar[buf]);
    }
}

// ------------------------------------------------------------------ epilogue
template <int MODE>
__device__ void drain(const UArgs &a, uint32_t tmem, uint64_t *tfull_bar, uint64_t *tempty_bar,
                      volatile int *abort_flag) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int bn = a.bn;
    int local = 0;
    for (int tile = blockIdx.x; tile < a.num_tiles; tile += gridDim.x, ++local) {
        const Tile T = decode_tile<MODE>(a, tile);
        const int buf = local & 1;
        // warp-uniform: the tcgen05.ld below needs every lane of the warp
        const bool ok = wait_or_abort(&tfull_bar[buf], ((uint32_t)local >> 1) & 1u, abort_flag);
        if (!__all_sync(0xffffffffu, ok)) return;
        tc_fence_after();
        const int m = T.m0 + q * 32 + lane;
#pragma unroll 1
        for (int c0 = 0; c0 < bn; c0 += 16) {
            uint32_t r[16];
            tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * bn + c0), r);
            if (m >= a.M) continue;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const int n = T.n0 + c0 + h * 8;
                if (n >= a.N) continue;  // N is a multiple of 8: all 8 columns or none
                float v[8];
#pragma unroll
                for (int e = 0; e < 8; ++e) v[e] = __uint_as_float(r[h * 8 + e]);
                if (MODE == U_FWD) {
                    if (a.bias) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) v[e] += a.bias[n + e];
                    }
                    if (a.relu) {
#pragma unroll
                        for (int e = 0; e < 8; ++e) v[e] = fmaxf(v[e], 0.f);
                    }
                    const long o = (long)m * a.N + n;
                    if (a.y_fp32) {
                        float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.out) + o);
                        dst[0] = make_float4(v[0], v[1], v[2], v[3]);
                        dst[1] = make_float4(v[4], v[5], v[6], v[7]);
                    } else {
                        *reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(a.out) + o) =
                            make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                       pack_bf16(v[6], v[7]));
                    }
                } else if (MODE == U_BWD_DATA) {
                    float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.out) + (long)m * a.N + n);
                    float4 p0 = make_float4(v[0], v[1], v[2], v[3]), p1 = make_float4(v[4], v[5], v[6], v[7]);
                    if (a.accumulate) {
                        const float4 q0 = dst[0], q1 = dst[1];
                        p0.x += q0.x, p0.y += q0.y, p0.z += q0.z, p0.w += q0.w;
                        p1.x += q1.x, p1.y += q1.y, p1.z += q1.z, p1.w += q1.w;
                    }
                    dst[0] = p0;
                    dst[1] = p1;
                } else {
                    float *dw = reinterpret_cast<float *>(a.out);  // dW[o][t][c] = dW[n M + m]
#pragma unroll
                    for (int e = 0; e < 8; ++e) atomicAdd(dw + (long)(n + e) * a.M + m, v[e]);
                }
            }
        }
        tc_fence_before();
        mbar_arrive(&tempty_bar[buf]);
    }
}

// ------------------------------------------------------------------ kernel
template <int MODE>
__global__ void __launch_bounds__(kThreads, 1) conv_umma_kernel(const UArgs a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], tfull_bar[2], tempty_bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_word;
    volatile int *abort_flag = &abort_word;
    const int warp = threadIdx.x >> 5;
    const uint32_t stage_bytes = (uint32_t)(UM + a.bn) * UK * 2;
    const uint32_t sbase = (smem_addr(smem_raw) + 1023u) & ~1023u;  // swizzle atoms are 1024-aligned

    if (warp == kMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&full_bar[s], kProducers);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull_bar[b], 1);
            mbar_init(&tempty_bar[b], 128);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp < kMmaWarp) {
        produce<MODE>(a, sbase, stage_bytes, full_bar, empty_bar, abort_flag);
    } else if (warp == kMmaWarp) {
        if ((threadIdx.x & 31) == 0)
            issue_mmas<MODE>(a, sbase, stage_bytes, tmem, full_bar, empty_bar, tfull_bar, tempty_bar, abort_flag);
    } else if (warp >= kEpiWarp0) {
        drain<MODE>(a, tmem, tfull_bar, tempty_bar, abort_flag);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                     : "memory");
}

// ------------------------------------------------------------------ host side
int sm_count() {
    static const int sms = [] {  // initialised once, thread-safely
        int dev = 0, v = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
            cudaGetLastError();
            v = 1;
        }
        return v > 0 ? v : 1;
    }();
    return sms;
}

// N tile for K-major B: the fewest tiles of at most 256 columns, each a multiple of 16.
int pick_bn(int N) {
    const int tiles = (N + kMaxBn - 1) / kMaxBn;
    const int per = (N + tiles - 1) / tiles;
    return (per + 15) / 16 * 16;
}

// N tile for the weight gradient's MN-major B: a power of two in [16, 256].
int pick_bn_pow2(int N) {
    int bn = 16;
    while (bn < N && bn < kMaxBn) bn <<= 1;
    return bn;
}

void finish_args(UArgs &a, int B) {
    a.stages = (int)(kRingBudget / ((uint32_t)(UM + a.bn) * UK * 2));
    if (a.stages > kMaxStages) a.stages = kMaxStages;
    uint32_t cols = 32;
    while ((int)cols < 2 * a.bn) cols <<= 1;
    a.tmem_cols = cols;
    a.m_tiles = (a.M + UM - 1) / UM;
    a.n_tiles = (a.N + a.bn - 1) / a.bn;
    a.div_w = make_fastdiv((uint32_t)a.W);
    a.div_hw = make_fastdiv((uint32_t)a.H * (uint32_t)a.W);
    (void)B;
}

template <int MODE>
rbgs_status launch(const UArgs &a, cudaStream_t s) {
    // set once per kernel instance, thread-safely; a failure is reported on every call
    static const cudaError_t attr = cudaFuncSetAttribute(conv_umma_kernel<MODE>,
                                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kMaxSmem);
    RBGS_CUDA(attr);
    const size_t smem = (size_t)a.stages * (UM + a.bn) * UK * 2 + 1024;
    const int grid = a.num_tiles < sm_count() ? a.num_tiles : sm_count();
    conv_umma_kernel<MODE><<<grid, kThreads, smem, s>>>(a);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

bool sizes_fit(int B, int H, int W) { return (long)B * H * W < (1L << 31) - UK; }

#include "conv_tma.cuh"
#include "conv_wgrad.cuh"
#include "conv_wgrad_ring.cuh"

}  // namespace

rbgs_status umma_conv_forward(const uint16_t *X, const uint16_t *Wt, const float *bias, void *Y, int B, int H,
                              int W, int Cin, int Cout, int ks, int relu, int y_fp32, cudaStream_t s) {
    if (!sizes_fit(B, H, W)) {
        set_error("tcgen05 convolution: at most 2^31 - 64 pixels");
        return RBGS_EINVAL;
    }
    // (the TMA-fed kernel also takes the forward product, but measured slower there than
    // the cp.async gathers: its weight box reads bn rows 9 Cin apart per tap)
    UArgs a{};
    a.X = X, a.Wt = Wt, a.bias = bias, a.out = Y;
    a.H = H, a.W = W, a.Cin = Cin, a.Cout = Cout, a.ks = ks, a.relu = relu, a.y_fp32 = y_fp32;
    a.M = B * H * W, a.N = Cout, a.K = ks * ks * Cin;
    a.bn = pick_bn(a.N);
    finish_args(a, B);
    a.num_tiles = a.m_tiles * a.n_tiles;
    return launch<U_FWD>(a, s);
}

rbgs_status umma_conv_backward_data(const uint16_t *Wtt, const uint16_t *G, float *dX, int B, int H, int W,
                                    int Cin, int Cout, int ks, int accumulate, bool tma, cudaStream_t s) {
    if (!sizes_fit(B, H, W)) {
        set_error("tcgen05 convolution: at most 2^31 - 64 pixels");
        return RBGS_EINVAL;
    }
    rbgs_status st = RBGS_OK;
    if (tma && tma_conv_launch<U_BWD_DATA>(G, Wtt, nullptr, dX, B, H, W, Cin, Cout, ks, 0, 0, accumulate, s, &st))
        return st;
    UArgs a{};
    a.Wt = Wtt, a.G = G, a.out = dX;
    a.H = H, a.W = W, a.Cin = Cin, a.Cout = Cout, a.ks = ks, a.accumulate = accumulate;
    a.M = B * H * W, a.N = Cin, a.K = ks * ks * Cout;
    a.bn = pick_bn(a.N);
    finish_args(a, B);
    a.num_tiles = a.m_tiles * a.n_tiles;
    return launch<U_BWD_DATA>(a, s);
}

rbgs_status umma_conv_backward_weight(const uint16_t *X, const uint16_t *G, float *dW, int B, int H, int W,
                                      int Cin, int Cout, int ks, int kind, cudaStream_t s) {
    if (!sizes_fit(B, H, W)) {
        set_error("tcgen05 convolution: at most 2^31 - 64 pixels");
        return RBGS_EINVAL;
    }
    // 3x3 layers: the ring kernel (conv_wgrad_ring.cuh) or the tap-row kernel (conv_wgrad.cuh),
    // whose epilogue adds 16-byte vectors, else the gather kernel below.  The automatic choice
    // follows the per-layer measurements on GB300 (U-Net layers at 16 x 256^2, TFLOP/s, ring /
    // tap row / gather): Cin <= 32, 256^2 and 128^2 rows: 88-166 / 45-144 / 75-157; the other
    // layers with >= 40 tap-row stages per SM and rows >= 64 pixels: 326-514 (tap row) vs
    // 163-273 (gather); the rest (stages per SM ~20, or 32-pixel rows): 234-317 (gather) vs
    // 163-275 (tap row).
    if (ks == 3 && kind != RBGS_WGRAD_GATHER && (reinterpret_cast<uintptr_t>(dW) & 15u) == 0) {
        bool launched = false;
        rbgs_status st = RBGS_OK;
        if (kind == RBGS_WGRAD_RING || (kind == RBGS_WGRAD_AUTO && Cin <= 32)) {
            st = wr_launch(X, G, dW, B, H, W, Cin, Cout, s, &launched);
            if (st != RBGS_OK || launched) return st;
        }
        WgPlan pl;
        const bool fits = wg_plan(B, H, W, Cin, Cout, sm_count(), pl);
        if (fits && (kind != RBGS_WGRAD_AUTO || (W >= 64 && pl.a.f_per_cta >= 40))) {
            st = wg_launch(pl, X, G, dW, s);
            if (st != RBGS_OK) return st;
            return RBGS_OK;
        }
    }
    UArgs a{};
    a.X = X, a.G = G, a.out = dW;
    a.H = H, a.W = W, a.Cin = Cin, a.Cout = Cout, a.ks = ks;
    a.M = ks * ks * Cin, a.N = Cout, a.K = B * H * W;
    a.bn = pick_bn_pow2(a.N);
    int lg = 0;
    while ((8 << lg) < a.bn) ++lg;
    a.log2_groups = lg;
    finish_args(a, B);
    // split the pixels so that about two tiles fall to each SM
    const int mn_tiles = a.m_tiles * a.n_tiles;
    int chunks = (2 * sm_count() + mn_tiles - 1) / mn_tiles;
    const int max_chunks = (a.K + 4 * UK - 1) / (4 * UK);  // at least four stages per chunk
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    int chunk = (a.K + chunks - 1) / chunks;
    chunk = (chunk + UK - 1) / UK * UK;
    a.k_chunk = chunk;
    chunks = (a.K + chunk - 1) / chunk;  // every chunk non-empty
    a.num_tiles = mn_tiles * chunks;
    return launch<U_BWD_WEIGHT>(a, s);
}

rbgs_status umma_conv_check(cudaStream_t s) {
    RBGS_CUDA(cudaStreamSynchronize(s));
    int failed = 0;
    RBGS_CUDA(cudaMemcpyFromSymbol(&failed, g_conv_wait_failed, sizeof(int)));
    if (failed) {
        const int zero = 0;
        RBGS_CUDA(cudaMemcpyToSymbol(g_conv_wait_failed, &zero, sizeof(int)));
        set_error("a tcgen05 convolution gave up waiting for its tensor-core work");
        return RBGS_ETIMEOUT;
    }
    return RBGS_OK;
}

}  // namespace rbgs
