// Weight gradient of a 3x3 convolution on tcgen05 with the tap's column shift taken in the
// shared-memory descriptor.  Included by conv_umma.cu inside its anonymous namespace, after
// the PTX wrappers, the bounded waits and the cp.async helpers it uses.
//
//   dW[o][ty][tx][c] = sum over pixels (b, y, x) of g[b, y, x, o] x[b, y + ty - 1, x + tx - 1, c]
//
// (zero outside the image).  The pixels are the GEMM's K.  A stage is one segment of `seg`
// pixels of one image row.  For a fixed tap row ty the segment's activation row y + ty - 1
// is staged once, with one pixel of halo on each side, and the three taps tx = 0, 1, 2 read
// it at pixel offsets 0, 1 and 2.  The staging layout is MN-major without swizzle: the
// pixels of one 8-channel group are consecutive 16-byte rows (channel group i, pixel p at
// (i len + p) 16 bytes), so the descriptor's K-group stride (LBO) is 128 bytes, its
// channel-group stride (SBO) is 16 len bytes, and a shift by one pixel is a shift of the
// start address by 16 bytes.  Nothing is gathered per tap: a stage loads seg + 2
// activation pixels and seg gradient pixels with 16-byte cp.async copies (each producer
// thread's arrival on the stage's barrier is tied to its copies' completion with
// cp.async.mbarrier.arrive, so every stage of the ring can be in flight) and issues
// 3 seg / 16 MMAs (the gather kernel re-reads the activations once per tap and the
// gradient once per M tile).
//
// Operands, chosen per layer so that the 128 rows of A are least padded:
//   xa = 0: A = gradient tile (M = Cout channels of an M tile), B = activations (N = Cin tile)
//   xa = 1: A = activation tile (M = Cin channels), B = gradient (N = Cout tile)
// Rows of A beyond the tile's channels read whatever follows the A slot in shared memory;
// their accumulator rows are never stored, and the host checks that every address a
// descriptor can form lies inside the allocation.
//
// Accumulators: the three taps of one tap row, 3 N TMEM columns (N <= 160), two buffers
// where 6 N <= 512.  A work item is (tap row, M tile, N tile, run of stages).  The stage
// sequence is cut into blocks of `lb` stages; within a block the items of every
// (tap row, tile) follow one another, so that the three tap rows of the same pixels run
// close together in time and their re-reads of the activation rows can hit L2 (on a layer
// whose inputs exceed L2, such as 96 channels at 16 x 256^2, they measured as DRAM reads,
// three per input).  The flattened
// (block, combination, stage) sequence is split evenly over the CTAs, and each CTA adds its
// items' partial sums to dW with FP32 atomics (dW must hold zeros, or the sum to add to).
//
// Roles (13 warps, one CTA per SM): warps 0-7 stage the operands, warp 8 issues the MMAs
// (one thread), warps 9-12 drain the accumulators.  Every wait is bounded, as in the
// gather kernel.

constexpr int kWgProducers = 256;  // warps 0-7
constexpr int kWgMmaWarp = 8;
constexpr int kWgEpiWarp0 = 9;     // warps 9-12
constexpr int kWgThreads = 416;
constexpr int kWgMaxStages = 16;
constexpr int kWgMinStages = 4;
constexpr int kWgGoodStages = 6;
constexpr uint32_t kWgBudget = 210 * 1024;
constexpr int kWgMaxN = 160;
// Pixel rows per channel group in a slot: seg, and seg + 2 halo pixels for activations
// (rounded up to 8).  (Rows padded to 1 mod 8, against bank conflicts between channel
// groups, measured the same.)
constexpr int kWgPadG = 0, kWgPadX = 8;

struct WgArgs {
    const uint16_t *X, *G;  // NHWC bf16 activations and output gradient
    float *dW;              // [Cout][3][3][Cin]
    int H, W, Cin, Cout;
    int xa;                 // 1: A = activations, B = gradient; 0: A = gradient, B = activations
    int ngA, ngB;           // 8-channel groups staged per A / B pixel
    int lenA, lenB;         // pixel rows per channel group of the A / B slot
    int N;                  // MMA N, a multiple of 16
    int m_tiles, n_tiles, ncombo;  // ncombo = 3 m_tiles n_tiles
    int seg, nseg, nk;      // pixels per stage, segments per image row, seg / 16
    int total_stages;       // B H nseg
    int lb;                 // stages per block
    long long f_per_cta;
    int stages;
    uint32_t a_slot, b_slot, b_ring;  // bytes; the B ring starts at b_ring
    uint32_t tmem_cols;
    int nbuf;
};

struct WgItem {
    int combo, s0, len;
};

// The next non-empty item of the flattened sequence [f, f_end); false at its end.
__device__ __forceinline__ bool wg_next(const WgArgs &a, long long &f, long long f_end, WgItem &it) {
    const long long per_blk = (long long)a.ncombo * a.lb;
    while (f < f_end) {
        const long long blk = f / per_blk;
        const long long rem = f - blk * per_blk;
        const int combo = (int)(rem / a.lb);
        const int j0 = (int)(rem - (long long)combo * a.lb);
        const long long s0 = blk * a.lb + j0;
        long long len = (long long)(a.lb - j0);
        if (len > f_end - f) len = f_end - f;
        f += len;
        const long long avail = (long long)a.total_stages - s0;
        if (avail <= 0) continue;  // the tail of the last block
        it.combo = combo;
        it.s0 = (int)s0;
        it.len = (int)(len < avail ? len : avail);
        return true;
    }
    return false;
}

__device__ __forceinline__ void wg_combo(const WgArgs &a, int combo, int &ty, int &mt, int &nt) {
    const int tiles = a.m_tiles * a.n_tiles;
    ty = combo / tiles;
    const int rest = combo - ty * tiles;
    mt = rest / a.n_tiles;
    nt = rest - mt * a.n_tiles;
}

// Staging tables: the 16-byte copies of one staged row that a producer thread issues, fixed
// per launch (units u = ptid, ptid + 256, ... of the row; pixel-major with channel groups
// fastest, so that a warp's copies read consecutive bytes of consecutive pixels).  Built
// once per kernel, so a stage costs each copy an add, a bounds check and its address.
constexpr int kWgMaxUnits = 8;

struct WgUnits {
    uint32_t dst[kWgMaxUnits];  // byte offset in the slot
    int pc[kWgMaxUnits];        // pixel offset from the segment's first pixel (high 16 bits,
                                // signed) and channel offset from the tile's first channel
    int n;
};

__device__ __forceinline__ int wg_pack_pc(int pix, int ch) { return (int)((uint32_t)pix << 16) | ch; }

// Plain layout: unit (pixel p, group g) of ng groups x npix pixels at (g len + p) 16 bytes,
// image pixel x0 + p + pix0.
__device__ __forceinline__ WgUnits wg_units_plain(int ng, int npix, int len, int pix0, int ptid) {
    WgUnits t;
    t.n = 0;
#pragma unroll
    for (int k = 0; k < kWgMaxUnits; ++k) {
        const int u = ptid + k * kWgProducers;
        const int p = u / ng, g = u - p * ng;
        t.dst[k] = (uint32_t)(g * len + p) * 16u;
        t.pc[k] = wg_pack_pc(p + pix0, g * 8);
        if (u < ng * npix) t.n = k + 1;
    }
    return t;
}

// Issues a thread's copies of one staged row: image pixels x0 + pix, channels c0 + ch;
// pixels outside the image row, channels beyond C and rows outside the image (row_ok
// false) are zero-filled.
__device__ __forceinline__ void wg_stage_units(const WgUnits &t, const uint16_t *row, bool row_ok, int C, int c0,
                                               int x0, int W, uint32_t slot) {
#pragma unroll
    for (int k = 0; k < kWgMaxUnits; ++k) {
        if (k < t.n) {
            const int x = x0 + (t.pc[k] >> 16), c = c0 + (t.pc[k] & 0xFFFF);
            const bool ok = row_ok && (unsigned)x < (unsigned)W && c < C;
            cp_async16(slot + t.dst[k], ok ? row + (long)x * C + c : row, ok);
        }
    }
}

__device__ void wg_produce(const WgArgs &a, uint32_t sbase, uint64_t *full_bar, uint64_t *empty_bar,
                           volatile int *abort_flag, long long f, long long f_end) {
    const int ptid = threadIdx.x;  // 0..255
    const int S = a.stages;
    const int ngx = a.xa ? a.ngA : a.ngB, ngg = a.xa ? a.ngB : a.ngA;
    const int lenx = a.xa ? a.lenA : a.lenB, leng = a.xa ? a.lenB : a.lenA;
    const WgUnits ux = wg_units_plain(ngx, a.seg + 2, lenx, -1, ptid);
    const WgUnits ug = wg_units_plain(ngg, a.seg, leng, 0, ptid);
    uint32_t s = 0, ph = 0;
    bool live = true;
    WgItem it;
    while (live && wg_next(a, f, f_end, it)) {
        int ty, mt, nt;
        wg_combo(a, it.combo, ty, mt, nt);
        const int xc0 = a.xa ? mt * 128 : nt * a.N;
        const int gc0 = a.xa ? nt * a.N : mt * 128;
        // the item's first stage, then one segment (and row, image) further per stage
        int r = it.s0 / a.nseg;
        int sg = it.s0 - r * a.nseg;
        int b = r / a.H, y = r - b * a.H;
        for (int j = 0; j < it.len; ++j) {
            if (!wait_or_abort(&empty_bar[s], ph ^ 1u, abort_flag)) {
                live = false;
                break;
            }
            const int x0 = sg * a.seg;
            const uint32_t sa = sbase + s * a.a_slot, sb = sbase + a.b_ring + s * a.b_slot;
            const int yy = y + ty - 1;  // the activation row of this tap row
            const bool rx = yy >= 0 && yy < a.H;
            const uint16_t *xrow = a.X + (long)(b * a.H + (rx ? yy : y)) * a.W * a.Cin;
            wg_stage_units(ux, xrow, rx, a.Cin, xc0, x0, a.W, a.xa ? sa : sb);
            const uint16_t *grow = a.G + (long)(b * a.H + y) * a.W * a.Cout;
            wg_stage_units(ug, grow, true, a.Cout, gc0, x0, a.W, a.xa ? sb : sa);
            // the stage's full barrier counts this thread's arrival once all its copies above
            // have landed; the thread itself moves on, so the whole ring can be in flight
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(&full_bar[s]))
                         : "memory");
            if (++s == (uint32_t)S) s = 0, ph ^= 1u;
            if (++sg == a.nseg) {
                sg = 0;
                if (++y == a.H) y = 0, ++b;
            }
        }
    }
    cp_async_wait<0>();
}

__device__ void wg_issue(const WgArgs &a, uint32_t sbase, uint32_t tmem, uint64_t *full_bar, uint64_t *empty_bar,
                         uint64_t *tfull_bar, uint64_t *tempty_bar, volatile int *abort_flag, long long f,
                         long long f_end) {
    const uint32_t idesc = instr_desc(UM, a.N, 1, 1);
    const uint32_t sbo_a = (uint32_t)a.lenA * 16u, sbo_b = (uint32_t)a.lenB * 16u;
    const uint32_t sh_a = a.xa ? 1u : 0u, sh_b = a.xa ? 0u : 1u;  // which operand the tap shifts
    const int S = a.stages;
    uint32_t s = 0, ph = 0;
    int local = 0;
    WgItem it;
    while (wg_next(a, f, f_end, it)) {
        const int buf = a.nbuf == 2 ? (local & 1) : 0;
        const uint32_t use = a.nbuf == 2 ? ((uint32_t)local >> 1) : (uint32_t)local;
        if (!wait_or_abort_spin(&tempty_bar[buf], (use & 1u) ^ 1u, abort_flag)) return;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(buf * 3 * a.N);
        for (int j = 0; j < it.len; ++j) {
            if (!wait_or_abort_spin(&full_bar[s], ph, abort_flag)) return;
            // the copies were written through the generic proxy; the MMAs read through the
            // async proxy
            fence_proxy_async_smem();
            tc_fence_after();
            // descriptors of the stage's slots; the start-address field is the address in
            // 16-byte units, so adding a row count moves the start by that many pixels
            const uint64_t da = smem_desc(sbase + s * a.a_slot, 128, sbo_a, 0);
            const uint64_t db = smem_desc(sbase + a.b_ring + s * a.b_slot, 128, sbo_b, 0);
            for (int kk = 0; kk < a.nk; ++kk) {
#pragma unroll
                for (int tx = 0; tx < 3; ++tx) {
                    const uint64_t ad = da + (uint64_t)(16 * kk) + sh_a * (uint64_t)tx;
                    const uint64_t bd = db + (uint64_t)(16 * kk) + sh_b * (uint64_t)tx;
                    umma_bf16(acc + (uint32_t)(tx * a.N), ad, bd, idesc, (j > 0 || kk > 0) ? 1u : 0u);
                }
            }
            umma_commit(&empty_bar[s]);
            if (++s == (uint32_t)S) s = 0, ph ^= 1u;
        }
        umma_commit(&tfull_bar[buf]);
        ++local;
    }
}

__device__ void wg_drain(const WgArgs &a, uint32_t tmem, uint64_t *tfull_bar, uint64_t *tempty_bar,
                         volatile int *abort_flag, long long f, long long f_end) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int mdim = a.xa ? a.Cin : a.Cout, ndim = a.xa ? a.Cout : a.Cin;
    int local = 0;
    WgItem it;
    while (wg_next(a, f, f_end, it)) {
        const int buf = a.nbuf == 2 ? (local & 1) : 0;
        const uint32_t use = a.nbuf == 2 ? ((uint32_t)local >> 1) : (uint32_t)local;
        const bool ok = wait_or_abort(&tfull_bar[buf], use & 1u, abort_flag);
        if (!__all_sync(0xffffffffu, ok)) return;
        tc_fence_after();
        int ty, mt, nt;
        wg_combo(a, it.combo, ty, mt, nt);
        const int m = mt * UM + q * 32 + lane;  // channel on the A side
        if (mt * UM + q * 32 < mdim) {          // warp-uniform: the quarter holds real rows
            for (int tx = 0; tx < 3; ++tx) {
#pragma unroll 1
                for (int c0 = 0; c0 < a.N; c0 += 16) {
                    uint32_t r[16];
                    tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 3 * a.N + tx * a.N + c0), r);
                    const int n0 = nt * a.N + c0;
                    if (m >= mdim || n0 >= ndim) continue;
                    if (!a.xa) {  // m = o, columns c = n0 .. n0 + 15
                        float *dst = a.dW + ((long)(m * 3 + ty) * 3 + tx) * a.Cin + n0;
#pragma unroll
                        for (int h = 0; h < 4; ++h) {
                            if (n0 + 4 * h < ndim)
                                atomicAdd(reinterpret_cast<float4 *>(dst + 4 * h),
                                          make_float4(__uint_as_float(r[4 * h]), __uint_as_float(r[4 * h + 1]),
                                                      __uint_as_float(r[4 * h + 2]), __uint_as_float(r[4 * h + 3])));
                        }
                    } else {  // m = c, columns o = n0 .. n0 + 15
#pragma unroll
                        for (int e = 0; e < 16; ++e) {
                            if (n0 + e < ndim)
                                atomicAdd(a.dW + ((long)((n0 + e) * 3 + ty) * 3 + tx) * a.Cin + m, __uint_as_float(r[e]));
                        }
                    }
                }
            }
        }
        tc_fence_before();
        mbar_arrive(&tempty_bar[buf]);
        ++local;
    }
}

__global__ void __launch_bounds__(kWgThreads, 1) wgrad_shift_kernel(const WgArgs a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kWgMaxStages], empty_bar[kWgMaxStages], tfull_bar[2], tempty_bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_word;
    volatile int *abort_flag = &abort_word;
    const int warp = threadIdx.x >> 5;
    const uint32_t sbase = (smem_addr(smem_raw) + 1023u) & ~1023u;
    const long long f0 = (long long)blockIdx.x * a.f_per_cta;
    const long long per_blk = (long long)a.ncombo * a.lb;
    const long long f_total = ((long long)a.total_stages + a.lb - 1) / a.lb * per_blk;
    const long long f1 = f0 + a.f_per_cta < f_total ? f0 + a.f_per_cta : f_total;

    if (warp == kWgMmaWarp) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                         smem_addr(&tmem_slot)),
                     "r"(a.tmem_cols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < a.stages; ++s) {
            mbar_init(&full_bar[s], kWgProducers);
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

    if (warp < kWgMmaWarp) {
        wg_produce(a, sbase, full_bar, empty_bar, abort_flag, f0, f1);
    } else if (warp == kWgMmaWarp) {
        if ((threadIdx.x & 31) == 0)
            wg_issue(a, sbase, tmem, full_bar, empty_bar, tfull_bar, tempty_bar, abort_flag, f0, f1);
    } else if (warp >= kWgEpiWarp0) {
        wg_drain(a, tmem, tfull_bar, tempty_bar, abort_flag, f0, f1);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kWgMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                     : "memory");
}

// ------------------------------------------------------------------ host side
struct WgPlan {
    WgArgs a;
    size_t smem;
    int grid;
};

// Tiles of at most kWgMaxN columns covering ndim channels, each a multiple of 16.
void wg_tiles(int ndim, int &n_tiles, int &N) {
    const int pad = (ndim + 15) / 16 * 16;
    n_tiles = (pad + kWgMaxN - 1) / kWgMaxN;
    N = ((ndim + n_tiles - 1) / n_tiles + 15) / 16 * 16;
}

// Plans the launch; false if no layout fits (the caller then uses the gather kernel).
// Checks, for every slot, that the addresses the descriptors can form stay inside the
// allocation: B reads stay inside their slot; A reads (128 rows, possibly beyond the
// tile's channels) end before the end of the allocation.
bool wg_plan(int B, int H, int W, int Cin, int Cout, int sms, WgPlan &pl) {
    WgArgs &a = pl.a;
    a = WgArgs{};
    a.H = H, a.W = W, a.Cin = Cin, a.Cout = Cout;
    int ntg, ng_, ntx, nx_;
    wg_tiles(Cin, ntg, ng_);   // A = gradient: N over Cin
    wg_tiles(Cout, ntx, nx_);  // A = activations: N over Cout
    const int mtg = (Cout + UM - 1) / UM, mtx = (Cin + UM - 1) / UM;
    a.xa = (long)mtx * ntx * nx_ < (long)mtg * ntg * ng_ ? 1 : 0;
    const int mdim = a.xa ? Cin : Cout;
    a.m_tiles = a.xa ? mtx : mtg;
    a.n_tiles = a.xa ? ntx : ntg;
    a.N = a.xa ? nx_ : ng_;
    a.ngA = (mdim + 7) / 8 < 16 ? (mdim + 7) / 8 : 16;
    a.ngB = a.N / 8;
    a.ncombo = 3 * a.m_tiles * a.n_tiles;
    // the longest segment that leaves a ring of kWgGoodStages stages, else kWgMinStages
    const int seg0 = W < 128 ? (W + 15) / 16 * 16 : 128;
    const int cands[4] = {seg0, 64, 32, 16};
    for (int ci = 0; ci < 8 && !a.seg; ++ci) {
        const int seg = cands[ci & 3];
        const int min_stages = ci < 4 ? kWgGoodStages : kWgMinStages;
        if ((ci & 3) > 0 && seg >= seg0) continue;
        const int xp = seg + kWgPadX, gp = seg + kWgPadG, nk = seg / 16;
        const int lenA = a.xa ? xp : gp, lenB = a.xa ? gp : xp;
        const uint32_t as = (uint32_t)(a.ngA * lenA * 16), bs = (uint32_t)(a.ngB * lenB * 16);
        const uint32_t b_reach = (uint32_t)((16 * (nk - 1) + (a.xa ? 0 : 2)) * 16 + (a.ngB - 1) * lenB * 16 + 256);
        if (b_reach > bs) continue;
        // every staged row fits the producers' unit tables
        const int ngx = a.xa ? a.ngA : a.ngB, ngg = a.xa ? a.ngB : a.ngA;
        if (ngx * (seg + 2) > kWgMaxUnits * kWgProducers || ngg * seg > kWgMaxUnits * kWgProducers) continue;
        for (int S = kWgMaxStages; S >= min_stages; --S) {
            const uint32_t rings = (uint32_t)S * (as + bs);
            const uint32_t a_reach =
                (uint32_t)(S - 1) * as + (uint32_t)((16 * (nk - 1) + (a.xa ? 2 : 0)) * 16 + 15 * lenA * 16 + 256);
            const uint32_t total = rings > a_reach ? rings : a_reach;
            if (total <= kWgBudget) {
                a.seg = seg, a.nk = nk, a.lenA = lenA, a.lenB = lenB, a.a_slot = as, a.b_slot = bs;
                a.b_ring = (uint32_t)S * as;
                a.stages = S;
                pl.smem = total + 1024;
                break;
            }
        }
    }
    if (!a.seg) return false;
    a.nseg = (W + a.seg - 1) / a.seg;
    const long long stages = (long long)B * H * a.nseg;
    if (stages >= (1LL << 31)) return false;
    a.total_stages = (int)stages;
    const int cols = 3 * a.N;
    a.nbuf = 2 * cols <= 512 ? 2 : 1;
    uint32_t tc = 32;
    while ((int)tc < a.nbuf * cols) tc <<= 1;
    a.tmem_cols = tc;
    // even split of the flattened sequence; blocks of about a third of a CTA's share, so
    // that a CTA drains a handful of items
    const long long work = stages * a.ncombo;
    const long long per = (work + sms - 1) / sms;
    long long lb = per / 3;
    if (lb < 8) lb = 8;
    if (lb > 256) lb = 256;
    a.lb = (int)lb;
    const long long f_total = (stages + lb - 1) / lb * a.ncombo * lb;
    a.f_per_cta = (f_total + sms - 1) / sms;
    pl.grid = (int)((f_total + a.f_per_cta - 1) / a.f_per_cta);
    return true;
}

// Launches the tap-row weight gradient for a plan of wg_plan.
rbgs_status wg_launch(WgPlan pl, const uint16_t *X, const uint16_t *G, float *dW, cudaStream_t s) {
    static const cudaError_t attr = cudaFuncSetAttribute(wgrad_shift_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)(kWgBudget + 1024));
    RBGS_CUDA(attr);
    pl.a.X = X, pl.a.G = G, pl.a.dW = dW;
    wgrad_shift_kernel<<<pl.grid, kWgThreads, pl.smem, s>>>(pl.a);
    RBGS_LAUNCH_CHECK();
    return RBGS_OK;
}
