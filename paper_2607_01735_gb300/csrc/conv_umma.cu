// Convolution kernels of the learned initial guess on the 5th-generation tensor cores:
// implicit GEMM with tcgen05.mma, FP32 accumulators in tensor memory (TMEM).
//
// The three products of a convolution layer are the GEMMs listed in conv.cu; here they
// are tiled for tcgen05 as follows (M x N output tile, K in stages of 64):
//   forward      M = pixels,       N = Cout, K = taps*Cin   A, B K-major
//   data grad    M = pixels,       N = Cin,  K = taps*Cout  A, B K-major
//   weight grad  M = taps*Cin,     N = Cout, K = pixels     A, B MN-major (split over K)
// (the weight gradient is computed transposed, dW^T[(t,c), o], so that the long
// dimension taps*Cin fills the 128 TMEM lanes and Cout <= 256 is one N tile).
//
// One CTA of 128 threads owns a 128 x bn tile (bn a multiple of 16, at most 256).
// All threads gather operand tiles with 16-byte cp.async copies (zero-filled outside the
// image, the channel range and the pixel range) straight into the canonical
// no-swizzle core-matrix layout: vector v of a tile lands at byte 16 v, which makes the
// shared-memory writes conflict-free and the global reads of 8 threads one 128-byte row.
//   K-major tile (R rows x 64 k): core matrix (rows 8i..8i+7, k 8j..8j+7) at (8 i + j) 128;
//     descriptor LBO (next core matrix along K) = 128 B, SBO (next 8 rows) = 1024 B.
//   MN-major tile: core matrix (mn 8i.., k 8j..) at (j R/8 + i) 128 with one k per
//     16-byte row; LBO (along K) = 16 R B, SBO (along MN) = 128 B.
// A four-stage ring overlaps the gathers of stages kt+1..kt+3 with the MMAs of stage kt;
// thread 0 issues four 128 x bn x 16 MMAs per stage and commits them to the stage's
// mbarrier, which every thread waits on (bounded) before refilling that stage.  The
// epilogue reads the accumulator rows with tcgen05.ld (warp w owns lanes 32w..32w+31,
// one output row per thread) and applies bias / ReLU / bf16 rounding, or adds the
// partial weight gradient with FP32 atomics.
#include <cuda_bf16.h>

#include "common.cuh"
#include "tma.cuh"
#include "../../include/rbgs_unet.h"

namespace rbgs {

// Set when a bounded wait of a tcgen05 convolution gave up; read and cleared by
// rbgs_conv_check.
__device__ int g_conv_wait_failed;

namespace {

constexpr int UM = 128;        // tile rows = TMEM lanes
constexpr int UK = 64;         // K per stage: 128 bytes of bf16 per row
constexpr int USTAGES = 4;
constexpr int UTHREADS = 128;
constexpr uint32_t kUmmaPolls = 1u << 22;
constexpr int kMaxBn = 256;
constexpr size_t kMaxSmem = (size_t)USTAGES * (UM + kMaxBn) * UK * 2;

enum UMode { U_FWD = 0, U_BWD_DATA = 1, U_BWD_WEIGHT = 2 };

struct UArgs {
    const uint16_t *X;   // NHWC bf16 activations
    const uint16_t *Wt;  // forward: [Cout][taps][Cin]; data grad: transposed [taps][Cin][Cout]
    const uint16_t *G;   // NHWC bf16 gradient of the pre-activation output
    const float *bias;
    void *out;
    int H, W, Cin, Cout, ks;
    int relu, y_fp32, accumulate;
    long M, N, K;        // GEMM sizes
    int bn;              // N tile
    long k_chunk;        // weight grad: pixels per CTA (multiple of UK)
    uint32_t tmem_cols;  // power of two >= max(32, bn)
};

// ------------------------------------------------------------------ PTX wrappers
__device__ __forceinline__ void cp_async16(uint32_t dst, const void *src, bool valid) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], 16, %2;" ::"r"(dst), "l"(src), "r"(valid ? 16 : 0)
                 : "memory");
}

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }

template <int N>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor, no swizzle: start address, leading (K-direction) and
// stride (MN-direction) byte offsets between core matrices, descriptor version 1.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | ((uint64_t)1 << 46);
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

// ------------------------------------------------------------------ kernel
template <int MODE>
__global__ void __launch_bounds__(UTHREADS) conv_umma_kernel(UArgs a) {
    extern __shared__ __align__(128) unsigned char smem[];
    __shared__ __align__(8) uint64_t mma_bar[USTAGES];
    __shared__ uint32_t tmem_slot;
    constexpr bool MN = MODE == U_BWD_WEIGHT;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int bn = a.bn;
    const uint32_t a_bytes = UM * UK * 2, b_bytes = (uint32_t)bn * UK * 2;
    const uint32_t stage_bytes = a_bytes + b_bytes;
    const uint32_t sbase = smem_addr(smem);
    const long m0 = (long)blockIdx.x * UM, n0 = (long)blockIdx.y * bn;
    long kbeg = 0, kend = a.K;
    if (MODE == U_BWD_WEIGHT) {
        kbeg = (long)blockIdx.z * a.k_chunk;
        kend = kbeg + a.k_chunk < a.K ? kbeg + a.k_chunk : a.K;
    }
    const int KT = kend > kbeg ? (int)((kend - kbeg + UK - 1) / UK) : 0;
    const int pad = a.ks / 2;
    const long HW = (long)a.H * a.W;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        for (int s = 0; s < USTAGES; ++s) mbar_init(&mma_bar[s], 1);
        fence_barrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    // Per-thread constants of the A gather.  K-major A: this thread fills vectors
    // tid + 128 it (it = 0..7), i.e. rows 8 ((tid >> 6) + 2 it) + (tid & 7) at k chunk
    // (tid >> 3) & 7.  MN-major A: mn group (tid >> 3) & 15 at k rows 8 it + (tid & 7).
    int pyx[8];  // K-major: (y << 16 | x) of the row's pixel, -1 past the last pixel
    int a_dy = 0, a_dx = 0, a_c = 0;
    bool a_mval = false;
    if (!MN) {
#pragma unroll
        for (int it = 0; it < 8; ++it) {
            const long m = m0 + ((tid >> 6) + 2 * it) * 8 + (tid & 7);
            if (m < a.M) {
                const int r = (int)(m % HW);
                pyx[it] = ((r / a.W) << 16) | (r % a.W);
            } else {
                pyx[it] = -1;
            }
        }
    } else {
        const long m = m0 + ((tid >> 3) & 15) * 8;  // (t, c) index of the thread's 8 rows
        a_mval = m < a.M;
        if (a_mval) {
            const int t = (int)(m / a.Cin);
            a_c = (int)(m - (long)t * a.Cin);
            a_dy = t / a.ks - pad;
            a_dx = t % a.ks - pad;
        }
    }

    auto load_tile = [&](int kt, int s) {
        const uint32_t sa = sbase + (uint32_t)s * stage_bytes, sb = sa + a_bytes;
        const long k0 = kbeg + (long)kt * UK;
        if (!MN) {
            const long k = k0 + ((tid >> 3) & 7) * 8;
            const int CK = MODE == U_FWD ? a.Cin : a.Cout;
            const uint16_t *src = MODE == U_FWD ? a.X : a.G;
            const bool kval = k < a.K;
            int dy = 0, dx = 0, ch = 0;
            if (kval) {
                const int t = (int)(k / CK);
                ch = (int)(k - (long)t * CK);
                dy = t / a.ks - pad;
                dx = t % a.ks - pad;
                if (MODE == U_BWD_DATA) dy = -dy, dx = -dx;
            }
#pragma unroll
            for (int it = 0; it < 8; ++it) {
                const int yx = pyx[it];
                const int y = (yx >> 16) + dy, x = (yx & 0xFFFF) + dx;
                const bool ok = kval && yx >= 0 && y >= 0 && y < a.H && x >= 0 && x < a.W;
                const long m = m0 + ((tid >> 6) + 2 * it) * 8 + (tid & 7);
                const uint16_t *p = ok ? src + ((m + (long)dy * a.W + dx) * CK + ch) : src;
                cp_async16(sa + (uint32_t)(tid + it * UTHREADS) * 16, p, ok);
            }
            for (int v = tid; v < bn * 8; v += UTHREADS) {
                const long n = n0 + (v >> 6) * 8 + (v & 7);
                const long kb = k0 + ((v >> 3) & 7) * 8;
                const bool ok = n < a.N && kb < a.K;
                const uint16_t *p = a.Wt;
                if (ok) {
                    if (MODE == U_FWD) {
                        p = a.Wt + n * a.K + kb;  // Wt[o][t][c], k = t Cin + c
                    } else {
                        const int t = (int)(kb / a.Cout);
                        const int o = (int)(kb - (long)t * a.Cout);
                        p = a.Wt + ((long)t * a.Cin + n) * a.Cout + o;  // Wt_t[t][c][o]
                    }
                }
                cp_async16(sb + (uint32_t)v * 16, p, ok);
            }
        } else {
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const long p = k0 + j * 8 + (tid & 7);
                bool ok = a_mval && p < kend;
                const uint16_t *q = a.X;
                if (ok) {
                    const int r = (int)(p % HW);
                    const int y = r / a.W + a_dy, x = r % a.W + a_dx;
                    ok = y >= 0 && y < a.H && x >= 0 && x < a.W;
                    if (ok) q = a.X + (p + (long)a_dy * a.W + a_dx) * a.Cin + a_c;
                }
                cp_async16(sa + (uint32_t)(tid + j * UTHREADS) * 16, q, ok);
            }
            const int groups = bn >> 3;
            for (int v = tid; v < bn * 8; v += UTHREADS) {
                const int g = v >> 3;
                const long p = k0 + (g / groups) * 8 + (v & 7);
                const long n = n0 + (g % groups) * 8;
                const bool ok = p < kend && n < a.N;
                cp_async16(sb + (uint32_t)v * 16, ok ? a.G + p * a.Cout + n : a.G, ok);
            }
        }
    };

    const uint32_t idesc = instr_desc(UM, bn, MN ? 1 : 0, MN ? 1 : 0);
    const uint32_t a_lbo = MN ? UM * 16 : 128, a_sbo = MN ? 128 : 1024;
    const uint32_t b_lbo = MN ? (uint32_t)bn * 16 : 128, b_sbo = MN ? 128 : 1024;
    const uint32_t a_kstep = MN ? UM * 32 : 256, b_kstep = MN ? (uint32_t)bn * 32 : 256;
    bool waits_ok = true;

#pragma unroll 1
    for (int kt = 0; kt < USTAGES - 1; ++kt) {
        if (kt < KT) load_tile(kt, kt);
        cp_async_commit();
    }
#pragma unroll 1
    for (int kt = 0; kt < KT; ++kt) {
        const int s = kt % USTAGES;
        cp_async_wait<USTAGES - 2>();
        fence_proxy_async_smem();
        __syncthreads();
        if (tid == 0) {
            tc_fence_after();
            const uint32_t sa = sbase + (uint32_t)s * stage_bytes, sb = sa + a_bytes;
#pragma unroll
            for (int kk = 0; kk < UK / 16; ++kk) {
                const uint64_t ad = smem_desc(sa + kk * a_kstep, a_lbo, a_sbo);
                const uint64_t bd = smem_desc(sb + kk * b_kstep, b_lbo, b_sbo);
                umma_bf16(tmem, ad, bd, idesc, (kt > 0 || kk > 0) ? 1u : 0u);
            }
            umma_commit(&mma_bar[s]);
        }
        const int nt = kt + USTAGES - 1;
        if (nt < KT) {
            if (kt >= 1) {
                const int j = kt - 1;  // the stage being refilled last held tile kt - 1
                if (!mbar_wait_bounded(&mma_bar[j % USTAGES], (uint32_t)(j / USTAGES) & 1u, kUmmaPolls))
                    waits_ok = false;
            }
            load_tile(nt, nt % USTAGES);
        }
        cp_async_commit();
    }
    cp_async_wait<0>();
    if (KT > 0) {
        const int j = KT - 1;  // its commit arrives once every MMA of the CTA has completed
        if (!mbar_wait_bounded(&mma_bar[j % USTAGES], (uint32_t)(j / USTAGES) & 1u, kUmmaPolls))
            waits_ok = false;
    }
    if (!waits_ok) atomicOr(&g_conv_wait_failed, 1);
    tc_fence_after();

    // ---- epilogue: thread (warp w, lane l) owns output row 32 w + l
    const long m = m0 + warp * 32 + lane;
#pragma unroll 1
    for (int c0 = 0; c0 < bn; c0 += 16) {
        uint32_t r[16];
        tmem_ld16(tmem + ((uint32_t)(warp * 32) << 16) + (uint32_t)c0, r);
        if (m >= a.M || KT == 0 || !waits_ok) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const long n = n0 + c0 + h * 8;
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
                if (a.y_fp32) {
                    float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.out) + m * a.N + n);
                    o[0] = make_float4(v[0], v[1], v[2], v[3]);
                    o[1] = make_float4(v[4], v[5], v[6], v[7]);
                } else {
                    *reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(a.out) + m * a.N + n) =
                        make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                   pack_bf16(v[6], v[7]));
                }
            } else if (MODE == U_BWD_DATA) {
                float4 *o = reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.out) + m * a.N + n);
                float4 p0 = make_float4(v[0], v[1], v[2], v[3]), p1 = make_float4(v[4], v[5], v[6], v[7]);
                if (a.accumulate) {
                    const float4 q0 = o[0], q1 = o[1];
                    p0.x += q0.x, p0.y += q0.y, p0.z += q0.z, p0.w += q0.w;
                    p1.x += q1.x, p1.y += q1.y, p1.z += q1.z, p1.w += q1.w;
                }
                o[0] = p0;
                o[1] = p1;
            } else {
                float *dw = reinterpret_cast<float *>(a.out);  // dW[o][t][c] = dW[n M + m]
#pragma unroll
                for (int e = 0; e < 8; ++e) atomicAdd(dw + (n + e) * a.M + m, v[e]);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                     : "memory");
}

// N tile: the fewest tiles of at most 256 columns, each a multiple of 16.
int pick_bn(long N) {
    const long tiles = (N + kMaxBn - 1) / kMaxBn;
    const long per = (N + tiles - 1) / tiles;
    return (int)((per + 15) / 16 * 16);
}

uint32_t tmem_columns(int bn) {
    uint32_t c = 32;
    while ((int)c < bn) c <<= 1;
    return c;
}

template <int MODE>
rbgs_status launch(UArgs a, dim3 grid, cudaStream_t s) {
    static bool attr_set = false;
    if (!attr_set) {
        RBGS_CUDA(cudaFuncSetAttribute(conv_umma_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       (int)kMaxSmem));
        attr_set = true;
    }
    const size_t smem = (size_t)USTAGES * (UM + a.bn) * UK * 2;
    conv_umma_kernel<MODE><<<grid, UTHREADS, smem, s>>>(a);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

int sm_count() {
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0) sms = 1;
    }
    return sms;
}

}  // namespace

rbgs_status umma_conv_forward(const uint16_t *X, const uint16_t *Wt, const float *bias, void *Y, int B, int H,
                              int W, int Cin, int Cout, int ks, int relu, int y_fp32, cudaStream_t s) {
    UArgs a{};
    a.X = X, a.Wt = Wt, a.bias = bias, a.out = Y;
    a.H = H, a.W = W, a.Cin = Cin, a.Cout = Cout, a.ks = ks, a.relu = relu, a.y_fp32 = y_fp32;
    a.M = (long)B * H * W, a.N = Cout, a.K = (long)ks * ks * Cin;
    a.bn = pick_bn(a.N), a.tmem_cols = tmem_columns(a.bn);
    dim3 grid((unsigned)((a.M + UM - 1) / UM), (unsigned)((a.N + a.bn - 1) / a.bn), 1);
    return launch<U_FWD>(a, grid, s);
}

rbgs_status umma_conv_backward_data(const uint16_t *Wtt, const uint16_t *G, float *dX, int B, int H, int W,
                                    int Cin, int Cout, int ks, int accumulate, cudaStream_t s) {
    UArgs a{};
    a.Wt = Wtt, a.G = G, a.out = dX;
    a.H = H, a.W = W, a.Cin = Cin, a.Cout = Cout, a.ks = ks, a.accumulate = accumulate;
    a.M = (long)B * H * W, a.N = Cin, a.K = (long)ks * ks * Cout;
    a.bn = pick_bn(a.N), a.tmem_cols = tmem_columns(a.bn);
    dim3 grid((unsigned)((a.M + UM - 1) / UM), (unsigned)((a.N + a.bn - 1) / a.bn), 1);
    return launch<U_BWD_DATA>(a, grid, s);
}

rbgs_status umma_conv_backward_weight(const uint16_t *X, const uint16_t *G, float *dW, int B, int H, int W,
                                      int Cin, int Cout, int ks, cudaStream_t s) {
    UArgs a{};
    a.X = X, a.G = G, a.out = dW;
    a.H = H, a.W = W, a.Cin = Cin, a.Cout = Cout, a.ks = ks;
    a.M = (long)ks * ks * Cin, a.N = Cout, a.K = (long)B * H * W;
    a.bn = pick_bn(a.N), a.tmem_cols = tmem_columns(a.bn);
    const long tiles = ((a.M + UM - 1) / UM) * ((a.N + a.bn - 1) / a.bn);
    // split the pixels so that the grid covers about two waves of the SMs
    long chunks = (2L * sm_count() + tiles - 1) / tiles;
    const long max_chunks = (a.K + UK - 1) / UK;
    if (chunks > max_chunks) chunks = max_chunks;
    if (chunks < 1) chunks = 1;
    long chunk = (a.K + chunks - 1) / chunks;
    chunk = (chunk + UK - 1) / UK * UK;
    a.k_chunk = chunk;
    chunks = (a.K + chunk - 1) / chunk;
    dim3 grid((unsigned)((a.M + UM - 1) / UM), (unsigned)((a.N + a.bn - 1) / a.bn), (unsigned)chunks);
    return launch<U_BWD_WEIGHT>(a, grid, s);
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
