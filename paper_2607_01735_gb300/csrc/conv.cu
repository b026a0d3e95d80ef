// Convolution kernels of the learned initial guess: implicit GEMM on the tensor cores.
//
// Two engines compute the same products: the tcgen05 kernels of conv_umma.cu (TMEM
// accumulators, the default) and the mma.sync kernels below (register accumulators),
// kept as the reference engine that rbgs_conv_set_engine selects.
//
// All three products of a 3x3 (or 1x1) convolution layer are one GEMM with a gathered
// operand (M x N += M x K times K x N, bf16 operands, FP32 accumulation) computed with
// mma.sync m16n8k16 bf16 tiles:
//   forward      M = pixels, N = Cout, K = taps*Cin :  A(p, (t,c)) = X[p + off(t), c]
//                                                       B((t,c), o) = Wt[o, t, c]
//   data grad    M = pixels, N = Cin,  K = taps*Cout:  A(p, (t,o)) = G[p - off(t), o]
//                                                       B((t,o), c) = Wt[o, t, c]
//   weight grad  M = Cout,   N = taps*Cin, K = pixels: A(o, p) = G[p, o]
//                                                       B(p, (t,c)) = X[p + off(t), c]
// (off(t) = (dy - 1, dx - 1) for a 3x3 kernel; rows outside the image read zero.)  A
// thread block computes a 64 x 64 tile of C in 32-wide K steps: the gathered A and B
// tiles are staged in shared memory (16-byte vector loads along the contiguous
// channel dimension), four warps each own a 32 x 32 sub-tile (2 x 4 mma tiles).  The
// weight gradient splits K (pixels) over gridDim.z and adds its partial tile to dW
// with FP32 atomics.
#include <cuda_bf16.h>

#include "common.cuh"
#include "../../include/rbgs_unet.h"

namespace rbgs {
namespace {

constexpr int BM = 64, BN = 64, BK = 32, KPAD = 8, THREADS = 128;
constexpr int LDS = BK + KPAD;  // shared row stride (bf16): 80 B, conflict-free fragments

enum Mode { FWD = 0, BWD_DATA = 1, BWD_WEIGHT = 2 };

struct ConvArgs {
    const uint16_t *X;   // activations (forward input), NHWC bf16
    const uint16_t *Wt;  // weights [Cout][ks][ks][Cin] bf16 (or transposed [ks*ks][Cin][Cout])
    const uint16_t *G;   // gradient w.r.t. the pre-activation output, NHWC bf16
    const float *bias;
    void *out;           // FWD: Y (bf16 or fp32); BWD_DATA: dX fp32; BWD_WEIGHT: dW fp32
    int B, H, W, Cin, Cout, ks;
    int relu, y_fp32, accumulate;
    int k_chunk;         // BWD_WEIGHT: pixels per block (multiple of BK)
};

__device__ __forceinline__ uint4 zero4() { return make_uint4(0u, 0u, 0u, 0u); }

__device__ __forceinline__ uint4 ld16(const uint16_t *p) { return *reinterpret_cast<const uint4 *>(p); }

__device__ __forceinline__ void mma_bf16(float *d, const uint32_t *a, const uint32_t *b) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
        "{%0,%1,%2,%3};"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b[0]), "r"(b[1]));
}

// Pixel index p -> (b, y, x) and a spatially shifted neighbour's linear index (or -1).
__device__ __forceinline__ long shifted(long p, int H, int W, int sy, int sx) {
    const long hw = (long)H * W;
    const long b = p / hw;
    const int r = (int)(p - b * hw);
    const int y = r / W + sy, x = r % W + sx;
    if (y < 0 || y >= H || x < 0 || x >= W) return -1;
    return b * hw + (long)y * W + x;
}

template <int MODE>
__global__ void __launch_bounds__(THREADS) conv_igemm_kernel(ConvArgs a) {
    __shared__ __align__(16) uint16_t As[BM][LDS];
    __shared__ __align__(16) uint16_t Bs[BN][LDS];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int wm = (warp >> 1) * 32, wn = (warp & 1) * 32;
    const int g = lane >> 2, tg = lane & 3;
    const long P = (long)a.B * a.H * a.W;
    const int taps = a.ks * a.ks, pad = a.ks / 2;
    long M, N, K;
    if (MODE == FWD) { M = P; N = a.Cout; K = (long)taps * a.Cin; }
    else if (MODE == BWD_DATA) { M = P; N = a.Cin; K = (long)taps * a.Cout; }
    else { M = a.Cout; N = (long)taps * a.Cin; K = P; }
    const long m0 = (long)blockIdx.x * BM, n0 = (long)blockIdx.y * BN;
    long kbeg = 0, kend = K;
    if (MODE == BWD_WEIGHT) {
        kbeg = (long)blockIdx.z * a.k_chunk;
        kend = kbeg + a.k_chunk < K ? kbeg + a.k_chunk : K;
    }
    float acc[2][4][4];
#pragma unroll
    for (int i = 0; i < 2; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[i][j][q] = 0.f;

    for (long k0 = kbeg; k0 < kend; k0 += BK) {
        // ---- stage A (BM x BK) and B (BN x BK) as [row][k]
#pragma unroll
        for (int it = 0; it < 2; ++it) {
            const int v = tid + it * THREADS;  // 256 vectors of 8 bf16 per tile
            if (MODE == FWD || MODE == BWD_DATA) {
                const int ml = v >> 2, k8 = (v & 3) * 8;
                const long m = m0 + ml, k = k0 + k8;
                uint4 val = zero4();
                const int CK = MODE == FWD ? a.Cin : a.Cout;  // channels per tap
                if (m < M && k < K) {
                    const int t = (int)(k / CK), ch = (int)(k % CK);
                    const int dy = t / a.ks - pad, dx = t % a.ks - pad;
                    const long q = MODE == FWD ? shifted(m, a.H, a.W, dy, dx) : shifted(m, a.H, a.W, -dy, -dx);
                    if (q >= 0) val = ld16((MODE == FWD ? a.X : a.G) + q * CK + ch);
                }
                *reinterpret_cast<uint4 *>(&As[ml][k8]) = val;
                // B tile
                const int nl = v >> 2;
                const long n = n0 + nl;
                uint4 bv = zero4();
                if (n < N && k < K) {
                    if (MODE == FWD) {
                        bv = ld16(a.Wt + n * K + k);  // Wt[o][t][c], k = t*Cin + c
                    } else {
                        const int t = (int)(k / a.Cout), o = (int)(k % a.Cout);
                        bv = ld16(a.Wt + ((long)t * a.Cin + n) * a.Cout + o);  // transposed [t][c][o]
                    }
                }
                *reinterpret_cast<uint4 *>(&Bs[nl][k8]) = bv;
            } else {
                // weight gradient: rows of the tiles are o (A) and (t,c) (B); k is a pixel
                const int kl = v >> 3, r8 = (v & 7) * 8;
                const long p = k0 + kl;
                uint4 av = zero4(), bv = zero4();
                const long mo = m0 + r8, n = n0 + r8;
                if (p < kend) {
                    if (mo < M) av = ld16(a.G + p * a.Cout + mo);
                    if (n < N) {
                        const int t = (int)(n / a.Cin), c = (int)(n % a.Cin);
                        const long q = shifted(p, a.H, a.W, t / a.ks - pad, t % a.ks - pad);
                        if (q >= 0) bv = ld16(a.X + q * a.Cin + c);
                    }
                }
                const uint16_t *ae = reinterpret_cast<const uint16_t *>(&av);
                const uint16_t *be = reinterpret_cast<const uint16_t *>(&bv);
#pragma unroll
                for (int j = 0; j < 8; ++j) {
                    As[r8 + j][kl] = ae[j];
                    Bs[r8 + j][kl] = be[j];
                }
            }
        }
        __syncthreads();
        // ---- two m16n8k16 steps per BK
#pragma unroll
        for (int kk = 0; kk < BK; kk += 16) {
            uint32_t af[2][4], bf[4][2];
#pragma unroll
            for (int i = 0; i < 2; ++i) {
                const int r = wm + i * 16 + g;
                af[i][0] = *reinterpret_cast<const uint32_t *>(&As[r][kk + tg * 2]);
                af[i][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + tg * 2]);
                af[i][2] = *reinterpret_cast<const uint32_t *>(&As[r][kk + tg * 2 + 8]);
                af[i][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][kk + tg * 2 + 8]);
            }
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = wn + j * 8 + g;
                bf[j][0] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + tg * 2]);
                bf[j][1] = *reinterpret_cast<const uint32_t *>(&Bs[c][kk + tg * 2 + 8]);
            }
#pragma unroll
            for (int i = 0; i < 2; ++i)
#pragma unroll
                for (int j = 0; j < 4; ++j) mma_bf16(acc[i][j], af[i], bf[j]);
        }
        __syncthreads();
    }

    // ---- epilogue
#pragma unroll
    for (int i = 0; i < 2; ++i) {
#pragma unroll
        for (int j = 0; j < 4; ++j) {
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const long m = m0 + wm + i * 16 + g + h * 8;
                const long n = n0 + wn + j * 8 + tg * 2;
                if (m >= M) continue;
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    if (n + e >= N) continue;
                    float v = acc[i][j][h * 2 + e];
                    if (MODE == FWD) {
                        if (a.bias) v += a.bias[n + e];
                        if (a.relu) v = fmaxf(v, 0.f);
                        if (a.y_fp32) {
                            reinterpret_cast<float *>(a.out)[m * N + n + e] = v;
                        } else {
                            __nv_bfloat16 bv = __float2bfloat16_rn(v);
                            reinterpret_cast<__nv_bfloat16 *>(a.out)[m * N + n + e] = bv;
                        }
                    } else if (MODE == BWD_DATA) {
                        float *o = reinterpret_cast<float *>(a.out) + m * N + n + e;
                        *o = a.accumulate ? *o + v : v;
                    } else {
                        atomicAdd(reinterpret_cast<float *>(a.out) + m * N + n + e, v);
                    }
                }
            }
        }
    }
}

// Wt[o][t][c] -> Wt_t[t][c][o]
__global__ void transpose_weights_kernel(const uint16_t *__restrict__ Wt, uint16_t *__restrict__ Wtt,
                                         int Cout, int taps, int Cin) {
    const long total = (long)Cout * taps * Cin;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const int c = (int)(q % Cin);
        const int t = (int)((q / Cin) % taps);
        const int o = (int)(q / ((long)Cin * taps));
        Wtt[((long)t * Cin + c) * Cout + o] = Wt[q];
    }
}

// db[o] += sum over pixels of G[p][o].  A thread owns 8 channels (one 16-byte vector) of
// a pixel lane and strides over pixels; the lanes of a block are then summed in a fixed
// order in shared memory and added to db once per block.
constexpr int kBiasThreads = 256;

__global__ void __launch_bounds__(kBiasThreads) bias_grad_kernel(const uint16_t *__restrict__ G,
                                                                 float *__restrict__ db, long P, int Cout) {
    __shared__ float part[kBiasThreads][8];
    const int groups = Cout >> 3;  // 1..32
    const int lanes = kBiasThreads / groups;
    const int g = threadIdx.x % groups, r = threadIdx.x / groups;
    float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
    if (r < lanes) {
        // four pixels per step, their loads issued together
        const long stride = (long)gridDim.x * lanes;
        for (long p = (long)blockIdx.x * lanes + r; p < P; p += 4 * stride) {
            uint4 v[4];
#pragma unroll
            for (int u = 0; u < 4; ++u)
                v[u] = p + u * stride < P ? ld16(G + (p + u * stride) * Cout + g * 8) : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                const uint32_t w[4] = {v[u].x, v[u].y, v[u].z, v[u].w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                    acc[2 * e] += __uint_as_float(w[e] << 16);
                    acc[2 * e + 1] += __uint_as_float(w[e] & 0xFFFF0000u);
                }
            }
        }
    }
#pragma unroll
    for (int e = 0; e < 8; ++e) part[threadIdx.x][e] = acc[e];
    __syncthreads();
    if (r == 0) {
        float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
        for (int q = 0; q < lanes; ++q)
#pragma unroll
            for (int e = 0; e < 8; ++e) s[e] += part[q * groups + g][e];
#pragma unroll
        for (int e = 0; e < 8; ++e) atomicAdd(db + g * 8 + e, s[e]);
    }
}

bool aligned16(const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

int g_engine = RBGS_CONV_TCGEN05;
int g_wgrad_kind = RBGS_WGRAD_AUTO;

}  // namespace

rbgs_status umma_conv_forward(const uint16_t *X, const uint16_t *Wt, const float *bias, void *Y, int B, int H,
                              int W, int Cin, int Cout, int ks, int relu, int y_fp32, cudaStream_t s);
rbgs_status umma_conv_backward_data(const uint16_t *Wtt, const uint16_t *G, float *dX, int B, int H, int W,
                                    int Cin, int Cout, int ks, int accumulate, bool tma, cudaStream_t s);
rbgs_status umma_conv_backward_weight(const uint16_t *X, const uint16_t *G, float *dW, int B, int H, int W,
                                      int Cin, int Cout, int ks, int kind, cudaStream_t s);
rbgs_status umma_conv_check(cudaStream_t s);

rbgs_status conv_forward(const uint16_t *X, const uint16_t *Wt, const float *bias, void *Y, int B, int H,
                         int W, int Cin, int Cout, int ks, int relu, int y_fp32, cudaStream_t s) {
    if (g_engine != RBGS_CONV_MMA_SYNC)
        return umma_conv_forward(X, Wt, bias, Y, B, H, W, Cin, Cout, ks, relu, y_fp32, s);
    ConvArgs a{X, Wt, nullptr, bias, Y, B, H, W, Cin, Cout, ks, relu, y_fp32, 0, 0};
    const long P = (long)B * H * W;
    dim3 grid((unsigned)((P + BM - 1) / BM), (unsigned)((Cout + BN - 1) / BN), 1);
    conv_igemm_kernel<FWD><<<grid, THREADS, 0, s>>>(a);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

rbgs_status conv_backward(const uint16_t *X, const uint16_t *Wt, const uint16_t *G, float *dX, float *dW,
                          float *db, uint16_t *Wtt, int B, int H, int W, int Cin, int Cout, int ks,
                          int accumulate, cudaStream_t s) {
    const long P = (long)B * H * W;
    const int taps = ks * ks;
    if (dX) {
        transpose_weights_kernel<<<256, 256, 0, s>>>(Wt, Wtt, Cout, taps, Cin);
        RBGS_LAUNCH_CHECK();
        if (g_engine != RBGS_CONV_MMA_SYNC) {
            const rbgs_status st = umma_conv_backward_data(Wtt, G, dX, B, H, W, Cin, Cout, ks, accumulate,
                                                           g_engine == RBGS_CONV_TCGEN05, s);
            if (st != RBGS_OK) return st;
        } else {
            ConvArgs a{X, Wtt, G, nullptr, dX, B, H, W, Cin, Cout, ks, 0, 0, accumulate, 0};
            dim3 grid((unsigned)((P + BM - 1) / BM), (unsigned)((Cin + BN - 1) / BN), 1);
            conv_igemm_kernel<BWD_DATA><<<grid, THREADS, 0, s>>>(a);
            RBGS_LAUNCH_CHECK();
        }
    }
    if (dW && g_engine != RBGS_CONV_MMA_SYNC) {
        const rbgs_status st = umma_conv_backward_weight(
            X, G, dW, B, H, W, Cin, Cout, ks, g_engine == RBGS_CONV_TCGEN05 ? g_wgrad_kind : RBGS_WGRAD_GATHER, s);
        if (st != RBGS_OK) return st;
    } else if (dW) {
        const int chunk = 4096;
        ConvArgs a{X, Wt, G, nullptr, dW, B, H, W, Cin, Cout, ks, 0, 0, 1, chunk};
        dim3 grid((unsigned)((Cout + BM - 1) / BM), (unsigned)((taps * Cin + BN - 1) / BN),
                  (unsigned)((P + chunk - 1) / chunk));
        conv_igemm_kernel<BWD_WEIGHT><<<grid, THREADS, 0, s>>>(a);
        RBGS_LAUNCH_CHECK();
    }
    if (db) {
        bias_grad_kernel<<<2 * 152, kBiasThreads, 0, s>>>(G, db, P, Cout);
        RBGS_LAUNCH_CHECK();
    }
    return RBGS_OK;
}

bool conv_shapes_ok(int B, int H, int W, int Cin, int Cout, int ks) {
    return B >= 1 && H >= 1 && W >= 1 && Cin >= 8 && Cout >= 8 && Cin % 8 == 0 && Cout % 8 == 0 &&
           Cout <= 256 * 8 && (ks == 1 || ks == 3) && H <= 32767 && W <= 32767 && (long)B * H * W < (1L << 40);
}

}  // namespace rbgs

using namespace rbgs;

extern "C" rbgs_status rbgs_conv_forward(const uint16_t *X, const uint16_t *Wt, const float *bias, void *Y,
                                         int B, int H, int W, int Cin, int Cout, int ksize, int relu,
                                         int y_fp32, void *cuda_stream) {
    clear_error();
    if (!X || !Wt || !Y || !conv_shapes_ok(B, H, W, Cin, Cout, ksize) || !aligned16(X) || !aligned16(Wt)) {
        set_error("rbgs_conv_forward: bad arguments (channels multiples of 8, ksize 1 or 3, 16-byte aligned)");
        return RBGS_EINVAL;
    }
    return conv_forward(X, Wt, bias, Y, B, H, W, Cin, Cout, ksize, relu, y_fp32, (cudaStream_t)cuda_stream);
}

extern "C" rbgs_status rbgs_conv_backward(const uint16_t *X, const uint16_t *Wt, const uint16_t *G, float *dX,
                                          float *dW, float *db, uint16_t *Wt_t, int B, int H, int W, int Cin,
                                          int Cout, int ksize, int accumulate, void *cuda_stream) {
    clear_error();
    if (!X || !Wt || !G || (dX && !Wt_t) || !conv_shapes_ok(B, H, W, Cin, Cout, ksize) || !aligned16(X) ||
        !aligned16(G) || !aligned16(Wt) || (Wt_t && !aligned16(Wt_t))) {
        set_error("rbgs_conv_backward: bad arguments");
        return RBGS_EINVAL;
    }
    return conv_backward(X, Wt, G, dX, dW, db, Wt_t, B, H, W, Cin, Cout, ksize, accumulate,
                         (cudaStream_t)cuda_stream);
}

extern "C" rbgs_status rbgs_conv_set_engine(int engine) {
    clear_error();
    if (engine != RBGS_CONV_TCGEN05 && engine != RBGS_CONV_MMA_SYNC && engine != RBGS_CONV_TCGEN05_GATHER) {
        set_error("rbgs_conv_set_engine: unknown engine %d", engine);
        return RBGS_EINVAL;
    }
    g_engine = engine;
    return RBGS_OK;
}

extern "C" int rbgs_conv_get_engine(void) { return g_engine; }

extern "C" rbgs_status rbgs_conv_set_wgrad_kernel(int kind) {
    clear_error();
    if (kind != RBGS_WGRAD_AUTO && kind != RBGS_WGRAD_RING && kind != RBGS_WGRAD_TAPROW &&
        kind != RBGS_WGRAD_GATHER) {
        set_error("rbgs_conv_set_wgrad_kernel: unknown kernel %d", kind);
        return RBGS_EINVAL;
    }
    g_wgrad_kind = kind;
    return RBGS_OK;
}

extern "C" int rbgs_conv_get_wgrad_kernel(void) { return g_wgrad_kind; }

extern "C" rbgs_status rbgs_conv_check(void *cuda_stream) {
    clear_error();
    return umma_conv_check((cudaStream_t)cuda_stream);
}
