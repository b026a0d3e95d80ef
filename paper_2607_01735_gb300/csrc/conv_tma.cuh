// TMA-fed tcgen05 convolution for the data-gradient product (written for the forward
// product too, which measured faster with the cp.async gathers).  Included by conv_umma.cu
// inside its anonymous namespace: it shares that file's PTX helpers, bounded waits and
// wait-failure flag.
//
// M tile = a tw x th rectangle of 128 pixels of one image (tw = 128 when W >= 128, else
// the power of two >= W); N tile = bn output channels.  The K loop runs over (tap t,
// channel chunk) pairs; a chunk is 64, 32 or 16 channels, loaded with the 128-, 64- or
// 32-byte swizzle whose K-major UMMA layout has rows of exactly that width (SBO = 8 rows).
// When the channels are a single chunk of 16 or 32, a stage carries 4 or 2 taps (each in
// its own sub-buffer, with its own descriptors), so every stage holds 64 of K.
// Per stage one thread issues two TMA loads on the stage's mbarrier (transaction bytes):
//   A: the 4D box (chunk, tw, th, 1) of the activations (forward) or of the output
//      gradient (data gradient) at the tap's offset (x0 + dx, y0 + dy); coordinates
//      outside the image read zeros, which is the convolution's zero padding;
//   B: the 3D box of the weights for that tap and chunk, [Cout][taps][Cin] (forward) or
//      the transposed [taps][Cin][Cout] (data gradient).
// Roles: warp 0 lane 0 issues the TMA loads, warp 1 lane 0 the MMAs (w/16 per stage) and
// the commits, warps 2-9 drain the double-buffered TMEM accumulators: warp w reads lanes
// 32 (w mod 4) .. of every other 16-column slice (two warps per lane quarter, since with
// few output channels the drain, not the MMAs, sets the pace).  Waits are bounded exactly
// as in the cp.async kernel.

constexpr int kTmaThreads = 320;  // warp 0 TMA, warp 1 MMA, warps 2-9 epilogue
constexpr int kTmaEpiThreads = 256;
constexpr int kTmaMaxChunks = 8;
constexpr uint32_t kTmaRing = 200 * 1024;

struct TMaps {
    CUtensorMap a[3], b[3];  // by chunk width: 16, 32, 64 channels
};

struct TArgs {
    const float *bias;
    void *out;
    int H, W, B, ks, pad, taps;
    int relu, y_fp32, accumulate;
    int M, N;  // pixels, output channels of this product
    int bn, stages;
    int tw, th, tiles_x, tiles_y, n_tiles, num_tiles;
    int nchunks, chunk_off[kTmaMaxChunks], chunk_w[kTmaMaxChunks];
    int group;   // taps per stage: 64 / w when the channels are one chunk of w < 64, else 1
    int kstages; // stages per tile
    uint32_t tmem_cols;
};

__device__ __forceinline__ int chunk_index(int w) { return w == 64 ? 2 : (w == 32 ? 1 : 0); }

// tcgen05 descriptor swizzle field for a K-major row of w bf16: 128B = 2, 64B = 4, 32B = 6
__device__ __forceinline__ uint32_t chunk_swizzle(int w) { return w == 64 ? 2u : (w == 32 ? 4u : 6u); }

__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2, int c3,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.4d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4, %5}], "
        "[%6];" ::"r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap *map, int c0, int c1, int c2,
                                            uint64_t *bar) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3, %4}], [%5];" ::
            "r"(dst),
        "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(smem_addr(bar))
        : "memory");
}

struct TTile {
    int b, y0, x0, n0;
};

__device__ __forceinline__ TTile decode_ttile(const TArgs &a, int tile) {
    const int nt = tile % a.n_tiles;
    int rest = tile / a.n_tiles;
    const int tx = rest % a.tiles_x;
    rest /= a.tiles_x;
    const int ty = rest % a.tiles_y;
    return TTile{rest / a.tiles_y, ty * a.th, tx * a.tw, nt * a.bn};
}

template <int MODE>
__global__ void __launch_bounds__(kTmaThreads, 1) conv_tma_kernel(const __grid_constant__ TMaps maps, const TArgs a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kMaxStages], empty_bar[kMaxStages], tfull_bar[2], tempty_bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_word;
    volatile int *abort_flag = &abort_word;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int bn = a.bn, S = a.stages;
    const uint32_t a_room = UM * UK * 2;                       // A box of the widest chunk
    const uint32_t stage_bytes = (uint32_t)(UM + bn) * UK * 2;  // multiple of 2048
    const uint32_t sbase = (smem_addr(smem_raw) + 1023u) & ~1023u;
    const int KT = a.kstages;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full_bar[s], 1);
            mbar_init(&empty_bar[s], 1);
        }
        for (int b = 0; b < 2; ++b) {
            mbar_init(&tfull_bar[b], 1);
            mbar_init(&tempty_bar[b], kTmaEpiThreads);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            for (int q = 0; q < 3; ++q) {
                prefetch_tensormap(&maps.a[q]);
                prefetch_tensormap(&maps.b[q]);
            }
            uint32_t s = 0, ph = 0;
            bool live = true;
            for (int tile = blockIdx.x; tile < a.num_tiles && live; tile += gridDim.x) {
                const TTile T = decode_ttile(a, tile);
                for (int kt = 0; kt < KT; ++kt) {
                    if (!wait_or_abort_spin(&empty_bar[s], ph ^ 1u, abort_flag)) {
                        live = false;
                        break;
                    }
                    // stage kt: taps t0 .. t0 + cnt - 1 of chunk j, each into its own
                    // sub-buffer (A: 128 w bf16, B: bn w bf16) of the stage
                    const int G = a.group;
                    const int j = G > 1 ? 0 : kt % a.nchunks;
                    const int t0 = G > 1 ? kt * G : kt / a.nchunks;
                    const int cnt = min(G, a.taps - t0);
                    const int w = a.chunk_w[j], c0 = a.chunk_off[j], wi = chunk_index(w);
                    const uint32_t sa = sbase + s * stage_bytes, sb = sa + a_room;
                    mbar_arrive_expect_tx(&full_bar[s], (uint32_t)cnt * (uint32_t)(UM + bn) * (uint32_t)w * 2u);
                    for (int g = 0; g < cnt; ++g) {
                        const int t = t0 + g;
                        int dy = t / a.ks - a.pad, dx = t % a.ks - a.pad;
                        if (MODE == U_BWD_DATA) dy = -dy, dx = -dx;
                        const uint32_t da = sa + (uint32_t)g * UM * (uint32_t)w * 2u;
                        const uint32_t db = sb + (uint32_t)g * (uint32_t)bn * (uint32_t)w * 2u;
                        tma_load_4d(da, &maps.a[wi], c0, T.x0 + dx, T.y0 + dy, T.b, &full_bar[s]);
                        if (MODE == U_FWD)
                            tma_load_3d(db, &maps.b[wi], c0, t, T.n0, &full_bar[s]);
                        else
                            tma_load_3d(db, &maps.b[wi], c0, T.n0, t, &full_bar[s]);
                    }
                    if (++s == (uint32_t)S) s = 0, ph ^= 1u;
                }
            }
        }
    } else if (warp == 1) {
        if (lane == 0) {
            const uint32_t idesc = instr_desc(UM, bn, 0, 0);
            uint32_t s = 0, ph = 0;
            int local = 0;
            bool live = true;
            for (int tile = blockIdx.x; tile < a.num_tiles && live; tile += gridDim.x, ++local) {
                const int buf = local & 1;
                if (!wait_or_abort_spin(&tempty_bar[buf], (((uint32_t)local >> 1) & 1u) ^ 1u, abort_flag)) break;
                tc_fence_after();
                const uint32_t acc = tmem + (uint32_t)(buf * bn);
                for (int kt = 0; kt < KT; ++kt) {
                    if (!wait_or_abort_spin(&full_bar[s], ph, abort_flag)) {
                        live = false;
                        break;
                    }
                    tc_fence_after();
                    const int G = a.group;
                    const int w = a.chunk_w[G > 1 ? 0 : kt % a.nchunks];
                    const int cnt = G > 1 ? min(G, a.taps - kt * G) : 1;
                    const uint32_t sw = chunk_swizzle(w), sbo = 16u * (uint32_t)w;
                    const uint32_t sa = sbase + s * stage_bytes, sb = sa + a_room;
                    for (int g = 0; g < cnt; ++g) {
                        const uint32_t da = sa + (uint32_t)g * UM * (uint32_t)w * 2u;
                        const uint32_t db = sb + (uint32_t)g * (uint32_t)bn * (uint32_t)w * 2u;
                        for (int kk = 0; kk < w / 16; ++kk) {
                            const uint64_t ad = smem_desc(da + kk * 32, 16, sbo, sw);
                            const uint64_t bd = smem_desc(db + kk * 32, 16, sbo, sw);
                            umma_bf16(acc, ad, bd, idesc, (kt > 0 || g > 0 || kk > 0) ? 1u : 0u);
                        }
                    }
                    umma_commit(&empty_bar[s]);
                    if (++s == (uint32_t)S) s = 0, ph ^= 1u;
                }
                if (!live) break;
                umma_commit(&tfull_bar[buf]);
            }
        }
    } else {
        const int q = warp & 3;             // TMEM lane quarter
        const int half = (warp - 2) >> 2;   // which 16-column slices: half, half + 2, ...
        const int row = q * 32 + lane;
        const int yy = row / a.tw, xx = row - yy * a.tw;
        int local = 0;
        for (int tile = blockIdx.x; tile < a.num_tiles; tile += gridDim.x, ++local) {
            const TTile T = decode_ttile(a, tile);
            const int buf = local & 1;
            const bool ok = wait_or_abort(&tfull_bar[buf], ((uint32_t)local >> 1) & 1u, abort_flag);
            if (!__all_sync(0xffffffffu, ok)) break;
            tc_fence_after();
            const int y = T.y0 + yy, x = T.x0 + xx;
            const bool pix = y < a.H && x < a.W;
            const long m = ((long)T.b * a.H + y) * a.W + x;
#pragma unroll 1
            for (int c0 = half * 16; c0 < bn; c0 += 32) {
                uint32_t r[16];
                tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * bn + c0), r);
                if (!pix) continue;
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
                        const long o = m * a.N + n;
                        if (a.y_fp32) {
                            float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.out) + o);
                            dst[0] = make_float4(v[0], v[1], v[2], v[3]);
                            dst[1] = make_float4(v[4], v[5], v[6], v[7]);
                        } else {
                            *reinterpret_cast<uint4 *>(reinterpret_cast<uint16_t *>(a.out) + o) =
                                make_uint4(pack_bf16(v[0], v[1]), pack_bf16(v[2], v[3]), pack_bf16(v[4], v[5]),
                                           pack_bf16(v[6], v[7]));
                        }
                    } else {
                        float4 *dst = reinterpret_cast<float4 *>(reinterpret_cast<float *>(a.out) + m * a.N + n);
                        float4 p0 = make_float4(v[0], v[1], v[2], v[3]), p1 = make_float4(v[4], v[5], v[6], v[7]);
                        if (a.accumulate) {
                            const float4 q0 = dst[0], q1 = dst[1];
                            p0.x += q0.x, p0.y += q0.y, p0.z += q0.z, p0.w += q0.w;
                            p1.x += q1.x, p1.y += q1.y, p1.z += q1.z, p1.w += q1.w;
                        }
                        dst[0] = p0;
                        dst[1] = p1;
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&tempty_bar[buf]);
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                     : "memory");
}

// ---- host side
CUresult encode_bf16_map(CUtensorMap *map, const void *base, int rank, const uint64_t *dims,
                         const uint64_t *strides_bytes, const uint32_t *box, int w) {
    static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
    if (!encode) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult qr;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &qr) !=
                cudaSuccess ||
            qr != cudaDriverEntryPointSuccess || !fn) {
            cudaGetLastError();
            return CUDA_ERROR_NOT_SUPPORTED;
        }
        encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
    }
    cuuint64_t d[5], st[4];
    cuuint32_t bx[5], es[5];
    for (int i = 0; i < rank; ++i) {
        d[i] = dims[i];
        bx[i] = box[i];
        es[i] = 1;
        if (i + 1 < rank) st[i] = strides_bytes[i];
    }
    const CUtensorMapSwizzle sw =
        w == 64 ? CU_TENSOR_MAP_SWIZZLE_128B : (w == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_32B);
    return encode(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, (cuuint32_t)rank, const_cast<void *>(base), d, st, bx, es,
                  CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                  CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

// The TMA path takes channel counts that split into chunks of 64, 32 and 16.
bool tma_chunks(int CK, TArgs &a) {
    if (CK % 16 != 0) return false;
    int n = 0, off = 0;
    while (CK - off >= 64 && n < kTmaMaxChunks) a.chunk_off[n] = off, a.chunk_w[n++] = 64, off += 64;
    if (CK - off >= 32 && n < kTmaMaxChunks) a.chunk_off[n] = off, a.chunk_w[n++] = 32, off += 32;
    if (CK - off >= 16 && n < kTmaMaxChunks) a.chunk_off[n] = off, a.chunk_w[n++] = 16, off += 16;
    a.nchunks = n;
    // one chunk narrower than 64: several taps per stage, so that a stage carries 64 of K
    a.group = (n == 1 && a.chunk_w[0] < 64) ? 64 / a.chunk_w[0] : 1;
    return off == CK;
}

// src: NHWC bf16 activations (forward) or output gradient (data gradient), CK channels;
// wts: Wt [Cout][taps][Cin] (forward) or Wt_t [taps][Cin][Cout] (data gradient).
// Returns false (nothing launched) when the shape is not one the TMA path takes.
template <int MODE>
bool tma_conv_launch(const uint16_t *src, const uint16_t *wts, const float *bias, void *out, int B, int H, int W,
                     int Cin, int Cout, int ks, int relu, int y_fp32, int accumulate, cudaStream_t s,
                     rbgs_status *st) {
    TArgs a{};
    const int CK = MODE == U_FWD ? Cin : Cout;
    const int N = MODE == U_FWD ? Cout : Cin;
    if (!tma_chunks(CK, a)) return false;
    a.bias = bias, a.out = out;
    a.H = H, a.W = W, a.B = B, a.ks = ks, a.pad = ks / 2, a.taps = ks * ks;
    a.kstages = a.group > 1 ? (a.taps + a.group - 1) / a.group : a.taps * a.nchunks;
    a.relu = relu, a.y_fp32 = y_fp32, a.accumulate = accumulate;
    a.M = B * H * W, a.N = N;
    a.bn = pick_bn(N);
    a.tw = 128;
    if (W < 128) {
        a.tw = 1;
        while (a.tw < W) a.tw <<= 1;
    }
    a.th = UM / a.tw;
    a.tiles_x = (W + a.tw - 1) / a.tw;
    a.tiles_y = (H + a.th - 1) / a.th;
    a.n_tiles = (N + a.bn - 1) / a.bn;
    const long tiles = (long)B * a.tiles_x * a.tiles_y * a.n_tiles;
    if (tiles > 0x7fffffffL) return false;
    a.num_tiles = (int)tiles;
    const uint32_t stage_bytes = (uint32_t)(UM + a.bn) * UK * 2;
    a.stages = (int)(kTmaRing / stage_bytes);
    if (a.stages > kMaxStages) a.stages = kMaxStages;
    uint32_t cols = 32;
    while ((int)cols < 2 * a.bn) cols <<= 1;
    a.tmem_cols = cols;

    TMaps maps;
    std::memset(&maps, 0, sizeof(maps));
    for (int wi = 0; wi < 3; ++wi) {
        const int w = 16 << wi;
        const uint64_t ad[4] = {(uint64_t)CK, (uint64_t)W, (uint64_t)H, (uint64_t)B};
        const uint64_t as[3] = {(uint64_t)CK * 2, (uint64_t)W * CK * 2, (uint64_t)H * W * CK * 2};
        const uint32_t abox[4] = {(uint32_t)w, (uint32_t)a.tw, (uint32_t)a.th, 1u};
        CUresult r = encode_bf16_map(&maps.a[wi], src, 4, ad, as, abox, w);
        if (r == CUDA_SUCCESS) {
            if (MODE == U_FWD) {
                const uint64_t bd[3] = {(uint64_t)Cin, (uint64_t)a.taps, (uint64_t)Cout};
                const uint64_t bs[2] = {(uint64_t)Cin * 2, (uint64_t)a.taps * Cin * 2};
                const uint32_t bbox[3] = {(uint32_t)w, 1u, (uint32_t)a.bn};
                r = encode_bf16_map(&maps.b[wi], wts, 3, bd, bs, bbox, w);
            } else {
                const uint64_t bd[3] = {(uint64_t)Cout, (uint64_t)Cin, (uint64_t)a.taps};
                const uint64_t bs[2] = {(uint64_t)Cout * 2, (uint64_t)Cin * Cout * 2};
                const uint32_t bbox[3] = {(uint32_t)w, (uint32_t)a.bn, 1u};
                r = encode_bf16_map(&maps.b[wi], wts, 3, bd, bs, bbox, w);
            }
        }
        if (r != CUDA_SUCCESS) {
            set_error("tensor map encoding for the TMA convolution failed (%d)", (int)r);
            *st = RBGS_ECUDA;
            return true;
        }
    }
    static const cudaError_t attr = [] {  // set once per instance, thread-safely
        const cudaError_t e = cudaFuncSetAttribute(conv_tma_kernel<MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)(kTmaRing + 1024));
        if (e != cudaSuccess) cudaGetLastError();
        return e;
    }();
    if (attr != cudaSuccess) {
        set_error("cudaFuncSetAttribute failed for the TMA convolution");
        *st = RBGS_ECUDA;
        return true;
    }
    const size_t smem = (size_t)a.stages * stage_bytes + 1024;
    const int grid = a.num_tiles < sm_count() ? a.num_tiles : sm_count();
    conv_tma_kernel<MODE><<<grid, kTmaThreads, smem, s>>>(maps, a);
    const cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
        set_error("TMA convolution launch failed: %s", cudaGetErrorString(e));
        *st = RBGS_ECUDA;
        return true;
    }
    *st = RBGS_OK;
    return true;
}
