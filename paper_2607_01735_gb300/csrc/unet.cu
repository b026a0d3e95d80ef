// The learned initial guess: a 4-level U-Net trained and run by the library's own
// kernels (conv.cu for the convolutions; pooling, upsampling, concatenation, loss and
// Adam here).  Layer order, shapes and the parameter layout are fixed:
//
//   level 0 (H x W):      e0a 16->32, e0b 32->32                       -> skip0
//   level 1 (H/2 x W/2):  e1a 32->64, e1b 64->64                       -> skip1
//   level 2 (H/4 x W/4):  e2a 64->128, e2b 128->128                    -> skip2
//   level 3 (H/8 x W/8):  b3a 128->256, b3b 256->256
//   level 2: concat(up(b3b), skip2) 384 -> d2a 384->128, d2b 128->128
//   level 1: concat(up(d2b), skip1) 192 -> d1a 192->64, d1b 64->64
//   level 0: concat(up(d1b), skip0)  96 -> d0a 96->32, d0b 32->32
//   out: 1x1 conv 32->8 (channel 0 is the prediction), no activation
// 3x3 convolutions with ReLU; 2x2 average pooling; nearest-neighbour upsampling.
// Parameters (FP32, in this order per layer): weights [Cout][k][k][Cin], then bias[Cout].
#include <cuda_bf16.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "common.cuh"
#include "../../include/rbgs_unet.h"

namespace rbgs {

rbgs_status conv_forward(const uint16_t *X, const uint16_t *Wt, const float *bias, void *Y, int B, int H,
                         int W, int Cin, int Cout, int ks, int relu, int y_fp32, cudaStream_t s);
rbgs_status umma_conv_check(cudaStream_t s);
rbgs_status conv_backward(const uint16_t *X, const uint16_t *Wt, const uint16_t *G, float *dX, float *dW,
                          float *db, uint16_t *Wtt, int B, int H, int W, int Cin, int Cout, int ks,
                          int accumulate, cudaStream_t s);

namespace {

struct Layer {
    int cin, cout, ks, relu, level;
    long w_off, b_off;  // offsets into the parameter vector
};

constexpr int kInCh = 16;  // f, mask, g, boundary interpolation, zero padding
constexpr int kXCh = 4;    // channels of the caller's input
const int kSpec[15][5] = {
    // cin, cout, ks, relu, level
    {16, 32, 3, 1, 0},   {32, 32, 3, 1, 0},   {32, 64, 3, 1, 1},   {64, 64, 3, 1, 1},
    {64, 128, 3, 1, 2},  {128, 128, 3, 1, 2}, {128, 256, 3, 1, 3}, {256, 256, 3, 1, 3},
    {384, 128, 3, 1, 2}, {128, 128, 3, 1, 2}, {192, 64, 3, 1, 1},  {64, 64, 3, 1, 1},
    {96, 32, 3, 1, 0},   {32, 32, 3, 1, 0},   {32, 8, 1, 0, 0}};

// ------------------------------------------------------------------ elementwise kernels
__global__ void pack_input_kernel(const float *__restrict__ x, __nv_bfloat16 *__restrict__ out, long P) {
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long)gridDim.x * blockDim.x) {
#pragma unroll
        for (int c = 0; c < kInCh; ++c) out[p * kInCh + c] = __float2bfloat16_rn(c < kXCh ? x[p * kXCh + c] : 0.f);
    }
}

// G = bf16(dY * (Y > 0)) (relu != 0) or bf16(dY)
__global__ void act_grad_kernel(const float *__restrict__ dY, const __nv_bfloat16 *__restrict__ Y,
                                __nv_bfloat16 *__restrict__ G, long n, int relu) {
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
        float v = dY[q];
        if (relu && !(__bfloat162float(Y[q]) > 0.f)) v = 0.f;
        G[q] = __float2bfloat16_rn(v);
    }
}

// 2x2 average pooling: in [B][H][W][C] -> out [B][H/2][W/2][C]
__global__ void avgpool_kernel(const __nv_bfloat16 *__restrict__ in, __nv_bfloat16 *__restrict__ out, int B,
                               int H, int W, int C) {
    const int h = H / 2, w = W / 2;
    const long total = (long)B * h * w * C;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const int c = (int)(q % C);
        const long pix = q / C;
        const int x = (int)(pix % w), y = (int)((pix / w) % h);
        const long b = pix / ((long)w * h);
        const long base = ((b * H + 2 * y) * W + 2 * x) * C + c;
        const float s = __bfloat162float(in[base]) + __bfloat162float(in[base + C]) +
                        __bfloat162float(in[base + (long)W * C]) + __bfloat162float(in[base + (long)W * C + C]);
        out[q] = __float2bfloat16_rn(0.25f * s);
    }
}

// backward of avg pooling: dIn[.., 2y+a, 2x+b, c] += dOut[.., y, x, c] / 4
__global__ void avgpool_bwd_kernel(const float *__restrict__ dOut, float *__restrict__ dIn, int B, int H, int W,
                                   int C) {
    const long total = (long)B * H * W * C;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const int c = (int)(q % C);
        const long pix = q / C;
        const int x = (int)(pix % W), y = (int)((pix / W) % H);
        const long b = pix / ((long)W * H);
        dIn[q] += 0.25f * dOut[((b * (H / 2) + y / 2) * (W / 2) + x / 2) * C + c];
    }
}

// concat(up(lo), skip): out [B][H][W][Clo + Cs]
__global__ void up_concat_kernel(const __nv_bfloat16 *__restrict__ lo, const __nv_bfloat16 *__restrict__ skip,
                                 __nv_bfloat16 *__restrict__ out, int B, int H, int W, int Clo, int Cs) {
    const int Ct = Clo + Cs;
    const long total = (long)B * H * W * Ct;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const int c = (int)(q % Ct);
        const long pix = q / Ct;
        const int x = (int)(pix % W), y = (int)((pix / W) % H);
        const long b = pix / ((long)W * H);
        out[q] = c < Clo ? lo[((b * (H / 2) + y / 2) * (W / 2) + x / 2) * Clo + c] : skip[pix * Cs + (c - Clo)];
    }
}

// split the concat gradient: dLo = sum over each 2x2 block of dCat[.., :Clo] (assigned);
// dSkip (+)= dCat[.., Clo:]
__global__ void up_concat_bwd_lo_kernel(const float *__restrict__ dCat, float *__restrict__ dLo, int B, int H,
                                        int W, int Clo, int Cs) {
    const int Ct = Clo + Cs, h = H / 2, w = W / 2;
    const long total = (long)B * h * w * Clo;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const int c = (int)(q % Clo);
        const long pix = q / Clo;
        const int x = (int)(pix % w), y = (int)((pix / w) % h);
        const long b = pix / ((long)w * h);
        const long base = ((b * H + 2 * y) * W + 2 * x) * Ct + c;
        dLo[q] = dCat[base] + dCat[base + Ct] + dCat[base + (long)W * Ct] + dCat[base + (long)W * Ct + Ct];
    }
}

__global__ void concat_bwd_skip_kernel(const float *__restrict__ dCat, float *__restrict__ dSkip, long P, int Clo,
                                       int Cs, int accumulate) {
    const int Ct = Clo + Cs;
    const long total = P * Cs;
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < total; q += (long)gridDim.x * blockDim.x) {
        const long pix = q / Cs;
        const int c = (int)(q % Cs);
        const float v = dCat[pix * Ct + Clo + c];
        dSkip[q] = accumulate ? dSkip[q] + v : v;
    }
}

__global__ void mask_sum_kernel(const float *__restrict__ mask, float *__restrict__ count, long P) {
    __shared__ float sm[32];
    float acc = 0.f;
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long)gridDim.x * blockDim.x)
        acc += mask[p];
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = threadIdx.x < blockDim.x / 32 ? sm[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) atomicAdd(count, t);
    }
}

// prediction (channel 0 of the 8-channel output) and masked MSE: loss partials, dOut
__global__ void loss_kernel(const float *__restrict__ out8, const float *__restrict__ target,
                            const float *__restrict__ mask, const float *__restrict__ count,
                            float *__restrict__ dOut8, float *__restrict__ loss, long P) {
    __shared__ float sm[32];
    const float inv_count = *count > 0.f ? 1.f / *count : 0.f;
    float acc = 0.f;
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long)gridDim.x * blockDim.x) {
        const float d = out8[p * 8] - target[p];
        const float m = mask[p];
        acc += m * d * d;
#pragma unroll
        for (int c = 0; c < 8; ++c) dOut8[p * 8 + c] = c == 0 ? 2.f * m * d * inv_count : 0.f;
    }
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x < 32) {
        float t = threadIdx.x < blockDim.x / 32 ? sm[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) t += __shfl_down_sync(0xffffffffu, t, o);
        if (threadIdx.x == 0) atomicAdd(loss, t * inv_count);
    }
}

__global__ void extract_pred_kernel(const float *__restrict__ out8, float *__restrict__ y, long P) {
    for (long p = (long)blockIdx.x * blockDim.x + threadIdx.x; p < P; p += (long)gridDim.x * blockDim.x)
        y[p] = out8[p * 8];
}

__global__ void adam_kernel(float *__restrict__ w, const float *__restrict__ g, float *__restrict__ m,
                            float *__restrict__ v, __nv_bfloat16 *__restrict__ wb, long n, float lr, float b1,
                            float b2, float c1, float c2, float eps) {
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x) {
        const float gq = g[q];
        const float mq = b1 * m[q] + (1.f - b1) * gq;
        const float vq = b2 * v[q] + (1.f - b2) * gq * gq;
        m[q] = mq;
        v[q] = vq;
        const float wq = w[q] - lr * (mq * c1) / (sqrtf(vq * c2) + eps);
        w[q] = wq;
        wb[q] = __float2bfloat16_rn(wq);
    }
}

__global__ void to_bf16_kernel(const float *__restrict__ w, __nv_bfloat16 *__restrict__ wb, long n) {
    for (long q = (long)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (long)gridDim.x * blockDim.x)
        wb[q] = __float2bfloat16_rn(w[q]);
}

int nblocks(long n) {
    long b = (n + 255) / 256;
    return (int)(b < 4096 ? (b > 0 ? b : 1) : 4096);
}

uint64_t splitmix(uint64_t &s) {
    uint64_t z = (s += 0x9E3779B97F4A7C15ull);
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

}  // namespace
}  // namespace rbgs

using namespace rbgs;

struct rbgs_unet {
    cudaStream_t stream;
    std::vector<Layer> layers;
    long nparams;
    float *w, *grad, *m, *v;   // FP32 master weights, gradient, Adam moments
    uint16_t *wb;               // bf16 copy used by the forward and backward
    uint16_t *wtt;              // transposed-weight scratch (largest layer)
    long step;
    // activation / gradient buffers for one (B, H, W)
    int B, H, W;
    std::vector<void *> bufs;
    uint16_t *act[22];          // bf16 activations (see forward for the order)
    float *gr[22];              // fp32 gradients of the same tensors
    uint16_t *gbf;              // bf16 pre-activation gradient scratch
    float *out8, *dout8, *dloss, *hloss;
};

namespace {

// activation tensors: index, channels, level
enum {
    A_IN = 0, A_E0A, A_S0, A_P0, A_E1A, A_S1, A_P1, A_E2A, A_S2, A_P2, A_B3A, A_B3B,
    A_C2, A_D2A, A_D2B, A_C1, A_D1A, A_D1B, A_C0, A_D0A, A_D0B, A_COUNT
};
const int kActCh[A_COUNT] = {16, 32, 32, 32, 64, 64, 64, 128, 128, 128, 256, 256, 384, 128, 128, 192, 64, 64, 96, 32, 32};
const int kActLv[A_COUNT] = {0, 0, 0, 1, 1, 1, 2, 2, 2, 3, 3, 3, 2, 2, 2, 1, 1, 1, 0, 0, 0};

rbgs_status ensure_buffers(rbgs_unet *net, int B, int H, int W) {
    if (net->B == B && net->H == H && net->W == W) return RBGS_OK;
    for (void *p : net->bufs) cudaFree(p);
    net->bufs.clear();
    net->B = net->H = net->W = 0;
    auto alloc = [&](size_t bytes, void **p) {
        if (cudaMalloc(p, bytes) != cudaSuccess) {
            cudaGetLastError();
            *p = nullptr;
            return false;
        }
        net->bufs.push_back(*p);
        return true;
    };
    size_t gmax = 0;
    for (int a = 0; a < A_COUNT; ++a) {
        const long pix = (long)B * (H >> kActLv[a]) * (W >> kActLv[a]);
        const size_t n = (size_t)pix * kActCh[a];
        if (!alloc(n * 2, (void **)&net->act[a]) || !alloc(n * 4, (void **)&net->gr[a])) {
            set_error("U-Net activation buffers: out of device memory");
            return RBGS_ENOMEM;
        }
        gmax = n > gmax ? n : gmax;
    }
    const size_t P = (size_t)B * H * W;
    if (!alloc(gmax * 2, (void **)&net->gbf) || !alloc(P * 8 * 4, (void **)&net->out8) ||
        !alloc(P * 8 * 4, (void **)&net->dout8) || !alloc(8, (void **)&net->dloss)) {
        set_error("U-Net buffers: out of device memory");
        return RBGS_ENOMEM;
    }
    net->B = B;
    net->H = H;
    net->W = W;
    return RBGS_OK;
}

#define UNET_TRY(x)                              \
    do {                                         \
        rbgs_status st_ = (x);                   \
        if (st_ != RBGS_OK) return st_;          \
    } while (0)

rbgs_status forward(rbgs_unet *net, const float *x) {
    const int B = net->B, H = net->H, W = net->W;
    cudaStream_t s = net->stream;
    const long P = (long)B * H * W;
    pack_input_kernel<<<nblocks(P), 256, 0, s>>>(x, (__nv_bfloat16 *)net->act[A_IN], P);
    RBGS_LAUNCH_CHECK();
    auto conv = [&](int li, int in, int out) {
        const Layer &L = net->layers[li];
        return conv_forward(net->act[in], net->wb + L.w_off, net->w + L.b_off, net->act[out], B, H >> L.level,
                            W >> L.level, L.cin, L.cout, L.ks, L.relu, 0, s);
    };
    auto pool = [&](int in, int out) {
        const int lv = kActLv[in];
        avgpool_kernel<<<nblocks((long)B * (H >> lv) * (W >> lv) * kActCh[in] / 4), 256, 0, s>>>(
            (const __nv_bfloat16 *)net->act[in], (__nv_bfloat16 *)net->act[out], B, H >> lv, W >> lv, kActCh[in]);
        return cudaGetLastError() == cudaSuccess ? RBGS_OK : RBGS_ECUDA;
    };
    auto upcat = [&](int lo, int skip, int out) {
        const int lv = kActLv[out];
        up_concat_kernel<<<nblocks((long)B * (H >> lv) * (W >> lv) * kActCh[out]), 256, 0, s>>>(
            (const __nv_bfloat16 *)net->act[lo], (const __nv_bfloat16 *)net->act[skip], (__nv_bfloat16 *)net->act[out],
            B, H >> lv, W >> lv, kActCh[lo], kActCh[skip]);
        return cudaGetLastError() == cudaSuccess ? RBGS_OK : RBGS_ECUDA;
    };
    UNET_TRY(conv(0, A_IN, A_E0A));
    UNET_TRY(conv(1, A_E0A, A_S0));
    UNET_TRY(pool(A_S0, A_P0));
    UNET_TRY(conv(2, A_P0, A_E1A));
    UNET_TRY(conv(3, A_E1A, A_S1));
    UNET_TRY(pool(A_S1, A_P1));
    UNET_TRY(conv(4, A_P1, A_E2A));
    UNET_TRY(conv(5, A_E2A, A_S2));
    UNET_TRY(pool(A_S2, A_P2));
    UNET_TRY(conv(6, A_P2, A_B3A));
    UNET_TRY(conv(7, A_B3A, A_B3B));
    UNET_TRY(upcat(A_B3B, A_S2, A_C2));
    UNET_TRY(conv(8, A_C2, A_D2A));
    UNET_TRY(conv(9, A_D2A, A_D2B));
    UNET_TRY(upcat(A_D2B, A_S1, A_C1));
    UNET_TRY(conv(10, A_C1, A_D1A));
    UNET_TRY(conv(11, A_D1A, A_D1B));
    UNET_TRY(upcat(A_D1B, A_S0, A_C0));
    UNET_TRY(conv(12, A_C0, A_D0A));
    UNET_TRY(conv(13, A_D0A, A_D0B));
    const Layer &L = net->layers[14];
    return conv_forward(net->act[A_D0B], net->wb + L.w_off, net->w + L.b_off, net->out8, B, H, W, L.cin, L.cout,
                        L.ks, 0, 1, s);
}

// Backward from dout8 (gradient of the 8-channel output); fills net->grad.
rbgs_status backward(rbgs_unet *net) {
    const int B = net->B, H = net->H, W = net->W;
    cudaStream_t s = net->stream;
    RBGS_CUDA(cudaMemsetAsync(net->grad, 0, net->nparams * sizeof(float), s));
    // layer li: input activation `in` (bf16), output activation `out` whose fp32 gradient
    // gr[out] is complete; writes gr[in] (assigned, or accumulated when acc != 0)
    auto conv_bwd = [&](int li, int in, const float *dOut, const uint16_t *Yout, int acc, bool need_dx) {
        const Layer &L = net->layers[li];
        const int h = H >> L.level, w = W >> L.level;
        const long n = (long)B * h * w * L.cout;
        act_grad_kernel<<<nblocks(n), 256, 0, s>>>(dOut, (const __nv_bfloat16 *)Yout, (__nv_bfloat16 *)net->gbf, n,
                                                  L.relu);
        if (cudaGetLastError() != cudaSuccess) {
            set_error("act_grad launch failed");
            return RBGS_ECUDA;
        }
        return conv_backward(net->act[in], net->wb + L.w_off, net->gbf, need_dx ? net->gr[in] : nullptr,
                             net->grad + L.w_off, net->grad + L.b_off, net->wtt, B, h, w, L.cin, L.cout, L.ks, acc,
                             s);
    };
    auto upcat_bwd = [&](int cat, int lo, int skip, int acc_skip) {
        const int lv = kActLv[cat];
        const int h = H >> lv, w = W >> lv;
        up_concat_bwd_lo_kernel<<<nblocks((long)B * h * w * kActCh[lo] / 4), 256, 0, s>>>(
            net->gr[cat], net->gr[lo], B, h, w, kActCh[lo], kActCh[skip]);
        concat_bwd_skip_kernel<<<nblocks((long)B * h * w * kActCh[skip]), 256, 0, s>>>(
            net->gr[cat], net->gr[skip], (long)B * h * w, kActCh[lo], kActCh[skip], acc_skip);
        return cudaGetLastError() == cudaSuccess ? RBGS_OK : RBGS_ECUDA;
    };
    auto pool_bwd = [&](int pooled, int src) {
        const int lv = kActLv[src];
        avgpool_bwd_kernel<<<nblocks((long)B * (H >> lv) * (W >> lv) * kActCh[src]), 256, 0, s>>>(
            net->gr[pooled], net->gr[src], B, H >> lv, W >> lv, kActCh[src]);
        return cudaGetLastError() == cudaSuccess ? RBGS_OK : RBGS_ECUDA;
    };
    // output layer (1x1, linear): its "output activation" is the fp32 out8
    {
        const Layer &L = net->layers[14];
        const long n = (long)B * H * W * 8;
        act_grad_kernel<<<nblocks(n), 256, 0, s>>>(net->dout8, nullptr, (__nv_bfloat16 *)net->gbf, n, 0);
        RBGS_LAUNCH_CHECK();
        UNET_TRY(conv_backward(net->act[A_D0B], net->wb + L.w_off, net->gbf, net->gr[A_D0B], net->grad + L.w_off,
                               net->grad + L.b_off, net->wtt, B, H, W, L.cin, L.cout, L.ks, 0, s));
    }
    UNET_TRY(conv_bwd(13, A_D0A, net->gr[A_D0B], net->act[A_D0B], 0, true));
    UNET_TRY(conv_bwd(12, A_C0, net->gr[A_D0A], net->act[A_D0A], 0, true));
    UNET_TRY(upcat_bwd(A_C0, A_D1B, A_S0, 0));
    UNET_TRY(conv_bwd(11, A_D1A, net->gr[A_D1B], net->act[A_D1B], 0, true));
    UNET_TRY(conv_bwd(10, A_C1, net->gr[A_D1A], net->act[A_D1A], 0, true));
    UNET_TRY(upcat_bwd(A_C1, A_D2B, A_S1, 0));
    UNET_TRY(conv_bwd(9, A_D2A, net->gr[A_D2B], net->act[A_D2B], 0, true));
    UNET_TRY(conv_bwd(8, A_C2, net->gr[A_D2A], net->act[A_D2A], 0, true));
    UNET_TRY(upcat_bwd(A_C2, A_B3B, A_S2, 0));
    UNET_TRY(conv_bwd(7, A_B3A, net->gr[A_B3B], net->act[A_B3B], 0, true));
    UNET_TRY(conv_bwd(6, A_P2, net->gr[A_B3A], net->act[A_B3A], 0, true));
    UNET_TRY(pool_bwd(A_P2, A_S2));
    UNET_TRY(conv_bwd(5, A_E2A, net->gr[A_S2], net->act[A_S2], 0, true));
    UNET_TRY(conv_bwd(4, A_P1, net->gr[A_E2A], net->act[A_E2A], 0, true));
    UNET_TRY(pool_bwd(A_P1, A_S1));
    UNET_TRY(conv_bwd(3, A_E1A, net->gr[A_S1], net->act[A_S1], 0, true));
    UNET_TRY(conv_bwd(2, A_P0, net->gr[A_E1A], net->act[A_E1A], 0, true));
    UNET_TRY(pool_bwd(A_P0, A_S0));
    UNET_TRY(conv_bwd(1, A_E0A, net->gr[A_S0], net->act[A_S0], 0, true));
    UNET_TRY(conv_bwd(0, A_IN, net->gr[A_E0A], net->act[A_E0A], 0, false));
    return RBGS_OK;
}

}  // namespace

extern "C" {

rbgs_status rbgs_unet_create(uint64_t seed, void *cuda_stream, rbgs_unet_t *out) {
    clear_error();
    if (!out) { set_error("out is NULL"); return RBGS_EINVAL; }
    *out = nullptr;
    rbgs_unet *net = new (std::nothrow) rbgs_unet();
    if (!net) { set_error("out of host memory"); return RBGS_ENOMEM; }
    net->stream = (cudaStream_t)cuda_stream;
    long off = 0, wmax = 0;
    for (int li = 0; li < 15; ++li) {
        Layer L{kSpec[li][0], kSpec[li][1], kSpec[li][2], kSpec[li][3], kSpec[li][4], 0, 0};
        const long nw = (long)L.cout * L.ks * L.ks * L.cin;
        L.w_off = off;
        off += nw;
        L.b_off = off;
        off += L.cout;
        wmax = nw > wmax ? nw : wmax;
        net->layers.push_back(L);
    }
    net->nparams = off;
    // He-uniform weights (fan-in = k*k*real input channels), zero biases
    std::vector<float> h(off, 0.f);
    uint64_t st = seed;
    for (const Layer &L : net->layers) {
        const int real_in = L.cin == kInCh ? kXCh : L.cin;
        const float a = std::sqrt(6.0f / (float)(L.ks * L.ks * real_in));
        const long nw = (long)L.cout * L.ks * L.ks * L.cin;
        for (long q = 0; q < nw; ++q) {
            const double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
            h[L.w_off + q] = (float)((2.0 * u - 1.0) * a);
        }
    }
    bool ok = cudaMalloc(&net->w, off * 4) == cudaSuccess && cudaMalloc(&net->grad, off * 4) == cudaSuccess &&
              cudaMalloc(&net->m, off * 4) == cudaSuccess && cudaMalloc(&net->v, off * 4) == cudaSuccess &&
              cudaMalloc(&net->wb, off * 2) == cudaSuccess && cudaMalloc(&net->wtt, wmax * 2) == cudaSuccess &&
              cudaMallocHost(&net->hloss, 4) == cudaSuccess;
    if (ok) {
        ok = cudaMemcpyAsync(net->w, h.data(), off * 4, cudaMemcpyHostToDevice, net->stream) == cudaSuccess &&
             cudaMemsetAsync(net->m, 0, off * 4, net->stream) == cudaSuccess &&
             cudaMemsetAsync(net->v, 0, off * 4, net->stream) == cudaSuccess;
        to_bf16_kernel<<<nblocks(off), 256, 0, net->stream>>>(net->w, (__nv_bfloat16 *)net->wb, off);
        ok = ok && cudaGetLastError() == cudaSuccess && cudaStreamSynchronize(net->stream) == cudaSuccess;
    }
    if (!ok) {
        cudaGetLastError();
        rbgs_unet_destroy(net);
        set_error("U-Net allocation failed");
        return RBGS_ENOMEM;
    }
    *out = net;
    return RBGS_OK;
}

long rbgs_unet_num_params(rbgs_unet_t net) { return net ? net->nparams : 0; }

rbgs_status rbgs_unet_get_params(rbgs_unet_t net, float *params) {
    clear_error();
    if (!net || !params) { set_error("NULL argument"); return RBGS_EINVAL; }
    RBGS_CUDA(cudaMemcpyAsync(params, net->w, net->nparams * 4, cudaMemcpyDefault, net->stream));
    RBGS_CUDA(cudaStreamSynchronize(net->stream));
    return RBGS_OK;
}

rbgs_status rbgs_unet_set_params(rbgs_unet_t net, const float *params) {
    clear_error();
    if (!net || !params) { set_error("NULL argument"); return RBGS_EINVAL; }
    RBGS_CUDA(cudaMemcpyAsync(net->w, params, net->nparams * 4, cudaMemcpyDefault, net->stream));
    to_bf16_kernel<<<nblocks(net->nparams), 256, 0, net->stream>>>(net->w, (__nv_bfloat16 *)net->wb, net->nparams);
    RBGS_LAUNCH_CHECK();
    RBGS_CUDA(cudaMemsetAsync(net->m, 0, net->nparams * 4, net->stream));
    RBGS_CUDA(cudaMemsetAsync(net->v, 0, net->nparams * 4, net->stream));
    net->step = 0;
    RBGS_CUDA(cudaStreamSynchronize(net->stream));
    return RBGS_OK;
}

rbgs_status rbgs_unet_forward(rbgs_unet_t net, const float *x, float *y, int B, int H, int W) {
    clear_error();
    if (!net || !x || !y || B < 1 || H < 8 || W < 8 || H % 8 || W % 8) {
        set_error("rbgs_unet_forward: bad arguments (H, W multiples of 8)");
        return RBGS_EINVAL;
    }
    UNET_TRY(ensure_buffers(net, B, H, W));
    UNET_TRY(forward(net, x));
    const long P = (long)B * H * W;
    extract_pred_kernel<<<nblocks(P), 256, 0, net->stream>>>(net->out8, y, P);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}

rbgs_status rbgs_unet_train_step(rbgs_unet_t net, const float *x, const float *target, const float *mask_loss,
                                 int B, int H, int W, float lr, float *loss, float *grads) {
    clear_error();
    if (!net || !x || !target || !mask_loss || B < 1 || H < 8 || W < 8 || H % 8 || W % 8) {
        set_error("rbgs_unet_train_step: bad arguments");
        return RBGS_EINVAL;
    }
    UNET_TRY(ensure_buffers(net, B, H, W));
    UNET_TRY(forward(net, x));
    const long P = (long)B * H * W;
    RBGS_CUDA(cudaMemsetAsync(net->dloss, 0, 8, net->stream));  // [0] loss, [1] sum(mask)
    mask_sum_kernel<<<nblocks(P), 256, 0, net->stream>>>(mask_loss, net->dloss + 1, P);
    RBGS_LAUNCH_CHECK();
    loss_kernel<<<nblocks(P), 256, 0, net->stream>>>(net->out8, target, mask_loss, net->dloss + 1, net->dout8,
                                                    net->dloss, P);
    RBGS_LAUNCH_CHECK();
    UNET_TRY(backward(net));
    if (grads) {
        RBGS_CUDA(cudaMemcpyAsync(grads, net->grad, net->nparams * 4, cudaMemcpyDefault, net->stream));
    } else {
        net->step += 1;
        const float b1 = 0.9f, b2 = 0.999f;
        const float c1 = 1.f / (1.f - std::pow(b1, (float)net->step));
        const float c2 = 1.f / (1.f - std::pow(b2, (float)net->step));
        adam_kernel<<<nblocks(net->nparams), 256, 0, net->stream>>>(net->w, net->grad, net->m, net->v,
                                                                    (__nv_bfloat16 *)net->wb, net->nparams, lr, b1,
                                                                    b2, c1, c2, 1e-8f);
        RBGS_LAUNCH_CHECK();
    }
    RBGS_CUDA(cudaMemcpyAsync(net->hloss, net->dloss, 4, cudaMemcpyDeviceToHost, net->stream));
    RBGS_CUDA(cudaStreamSynchronize(net->stream));
    if (loss) *loss = *net->hloss;
    return umma_conv_check(net->stream);
}

void rbgs_unet_destroy(rbgs_unet_t net) {
    if (!net) return;
    cudaStreamSynchronize(net->stream);
    for (void *p : net->bufs) cudaFree(p);
    cudaFree(net->w);
    cudaFree(net->grad);
    cudaFree(net->m);
    cudaFree(net->v);
    cudaFree(net->wb);
    cudaFree(net->wtt);
    if (net->hloss) cudaFreeHost(net->hloss);
    delete net;
}

}  // extern "C"
