// Weight gradient of a 3x3 convolution on tcgen05, all nine taps per stage: the activation
// rows stay in a ring while the output rows walk down an image.  Included by conv_umma.cu
// after conv_wgrad.cuh (whose helpers it uses), inside the anonymous namespace.
//
//   dW[o][ty][tx][c] = sum over pixels (b, y, x) of g[b, y, x, o] x[b, y + ty - 1, x + tx - 1, c]
//
// GEMM per tap row ty: M = (tx, c), 3 Cin rows; N = o; K = the pixels of the stage's row
// segment.  A is the activation row y + ty - 1 staged as three copies shifted by tx = 0, 1, 2
// pixels, so that the three taps share one MMA whose 128 rows hold (tx, c) with c fastest.
// A's layout is MN-major with the 128-byte swizzle: atoms of 8 pixels x 64 rows of M
// (1024 bytes, the 16-byte chunk ch of pixel row r at position ch ^ r), the MN atoms of a
// pixel group 1024 bytes apart (LBO) and pixel groups n_atoms 1024 bytes apart (SBO); the
// pre-shifted copies keep every descriptor start on an atom.  B is the gradient row y,
// MN-major without swizzle (channel group i, pixel p at (i seg + p) 16 bytes).  (The
// layouts without swizzle fed the tensor cores at about 45 bytes per clock and SM in this
// kernel's first form, a third of what the swizzled forward operands reach.)
//
// A stage is the row segment of one output row: it loads the gradient row and one new
// activation row (the first stage of an item three: y - 1, y, y + 1), and issues
// 3 m_tiles seg / 16 MMAs of 128 x N x 16.  Each activation row is loaded once per
// item and used by the stages of rows y - 1, y and y + 1; it lives in a ring of xr slots,
// each with an `xempty` barrier that the MMA thread's commit arrives on once the row's last
// stage has finished (the row above the current one after every stage; all three rows after
// an item's last stage).  Accumulators: (ty, M tile) x N columns, 3 m_tiles N per buffer.
//
// Compared with the per-tap-row kernel (conv_wgrad.cuh) a row segment costs a third of the
// MMAs (three taps in one MMA, and 3 Cin of the 128 rows used instead of Cout) and a third
// of the gradient loads; the activation row is copied three times, from L2.
//
// Work: the stages of every (image, column segment) strip, rows innermost; the flattened
// (block, N tile, stage) sequence is split evenly over the CTAs, and an item is a run of
// rows of one strip and one N tile.  Rows of A beyond 3 Cin (last M tile) read what follows
// the activation slot in shared memory and are never stored; the host checks that every
// address a descriptor can form lies inside the allocation.

constexpr int kWrMaxXr = kWgMaxStages + 2;

struct WrArgs {
    const uint16_t *X, *G;  // NHWC bf16 activations and output gradient
    float *dW;              // [Cout][3][3][Cin]
    int H, W, Cin, Cout;
    int ncc;                // Cin / 8
    int m_tiles;            // ceil(3 Cin / 128)
    int n_atoms;            // ceil(3 Cin / 64): 64-row MN atoms of an activation slot
    int N, n_tiles;         // MMA N (multiple of 16) and N tiles over Cout
    int seg, nseg, nk;      // pixels per stage, segments per image row, seg / 16
    int total;              // stages per N tile: B nseg H
    int lb;                 // stages per block
    long long f_per_cta;
    int stages, xr;         // gradient ring depth, activation ring depth (stages + 2)
    uint32_t x_slot, g_slot, g_ring;  // bytes; the activation ring first, the gradient ring at g_ring
    uint32_t tmem_cols;
    int nbuf, acc_cols;     // accumulator buffers, 3 m_tiles N columns each
};

struct WrItem {
    int nt, s0, len;
};

// The next item of [f, f_end): a run of rows of one strip and one N tile.
__device__ __forceinline__ bool wr_next(const WrArgs &a, long long &f, long long f_end, WrItem &it) {
    const long long per_blk = (long long)a.n_tiles * a.lb;
    while (f < f_end) {
        const long long blk = f / per_blk;
        const long long rem = f - blk * per_blk;
        const int nt = (int)(rem / a.lb);
        const int j0 = (int)(rem - (long long)nt * a.lb);
        const long long s0 = blk * a.lb + j0;
        long long len = (long long)(a.lb - j0);
        if (len > f_end - f) len = f_end - f;
        const long long avail = (long long)a.total - s0;
        if (avail <= 0) {  // the tail of the last block
            f += len;
            continue;
        }
        if (len > avail) len = avail;
        const long long to_strip_end = a.H - s0 % a.H;
        if (len > to_strip_end) len = to_strip_end;
        f += len;
        it.nt = nt;
        it.s0 = (int)s0;
        it.len = (int)len;
        return true;
    }
    return false;
}

// Staging table of the activation row's three shifted copies in the swizzled layout: unit
// (tx, pixel p, group g), groups fastest, holds channels 8g.. of image pixel x0 - 1 + p + tx
// at M row group mg = tx ncc + g: atom (p / 8, mg / 8), pixel row r = p mod 8, chunk
// (mg mod 8) ^ r.
__device__ __forceinline__ WgUnits wr_units_x(int ncc, int n_atoms, int seg, int ptid) {
    WgUnits t;
    t.n = 0;
#pragma unroll
    for (int k = 0; k < kWgMaxUnits; ++k) {
        const int u = ptid + k * kWgProducers;
        const int q = u / ncc, g = u - q * ncc;  // q = tx seg + p
        const int tx = q >= 2 * seg ? 2 : (q >= seg ? 1 : 0);
        const int p = q - tx * seg;
        const int mg = tx * ncc + g, r8 = p & 7;
        t.dst[k] = ((uint32_t)((p >> 3) * n_atoms + (mg >> 3)) << 10) + ((uint32_t)r8 << 7) +
                   ((uint32_t)((mg & 7) ^ r8) << 4);
        t.pc[k] = wg_pack_pc(p + tx - 1, g * 8);
        if (u < 3 * ncc * seg) t.n = k + 1;
    }
    return t;
}

__device__ void wr_produce(const WrArgs &a, uint32_t sbase, uint64_t *full_bar, uint64_t *empty_bar,
                           uint64_t *xempty_bar, volatile int *abort_flag, long long f, long long f_end) {
    const int ptid = threadIdx.x;  // 0..255
    const int S = a.stages;
    const WgUnits ux = wr_units_x(a.ncc, a.n_atoms, a.seg, ptid);
    const WgUnits ug = wg_units_plain(a.N / 8, a.seg, a.seg, 0, ptid);
    uint32_t s = 0, ph = 0;
    int xs = 0;         // slot of the next activation row
    uint32_t xph = 0;   // parity of that slot's uses so far
    bool live = true;
    WrItem it;
    while (live && wr_next(a, f, f_end, it)) {
        const int gc0 = it.nt * a.N;
        const int strip = it.s0 / a.H, b = strip / a.nseg;
        const int x0 = (strip - b * a.nseg) * a.seg;
        int y = it.s0 - strip * a.H;
        for (int j = 0; j < it.len && live; ++j, ++y) {
            if (!wait_or_abort(&empty_bar[s], ph ^ 1u, abort_flag)) {
                live = false;
                break;
            }
            // activation rows: y - 1, y, y + 1 at an item's first stage, else y + 1
            for (int r = j == 0 ? -1 : 1; r <= 1; ++r) {
                if (!wait_or_abort(&xempty_bar[xs], xph ^ 1u, abort_flag)) {
                    live = false;
                    break;
                }
                const int yy = y + r;
                const bool rok = yy >= 0 && yy < a.H;
                const uint16_t *xrow = a.X + (long)(b * a.H + (rok ? yy : y)) * a.W * a.Cin;
                wg_stage_units(ux, xrow, rok, a.Cin, 0, x0, a.W, sbase + (uint32_t)xs * a.x_slot);
                if (++xs == a.xr) xs = 0, xph ^= 1u;
            }
            if (!live) break;
            const uint16_t *grow = a.G + (long)(b * a.H + y) * a.W * a.Cout;
            wg_stage_units(ug, grow, true, a.Cout, gc0, x0, a.W, sbase + a.g_ring + s * a.g_slot);
            asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];" ::"r"(smem_addr(&full_bar[s]))
                         : "memory");
            if (++s == (uint32_t)S) s = 0, ph ^= 1u;
        }
    }
    cp_async_wait<0>();
}

__device__ void wr_issue(const WrArgs &a, uint32_t sbase, uint32_t tmem, uint64_t *full_bar, uint64_t *empty_bar,
                         uint64_t *xempty_bar, uint64_t *tfull_bar, uint64_t *tempty_bar, volatile int *abort_flag,
                         long long f, long long f_end) {
    const uint32_t idesc = instr_desc(UM, a.N, 1, 1);
    const uint32_t sbo = (uint32_t)a.seg * 16u;                 // B: channel-group stride
    const uint32_t a_sbo = (uint32_t)a.n_atoms << 10;           // A: pixel-group stride
    const uint64_t a_kstep = (uint64_t)(2u * a_sbo) >> 4;       // 16 pixels, in 16-byte units
    const int S = a.stages;
    uint32_t s = 0, ph = 0;
    int xs = 0;  // slot of the item's first activation row (row y0 - 1)
    int local = 0;
    WrItem it;
    while (wr_next(a, f, f_end, it)) {
        const int buf = a.nbuf == 2 ? (local & 1) : 0;
        const uint32_t use = a.nbuf == 2 ? ((uint32_t)local >> 1) : (uint32_t)local;
        if (!wait_or_abort_spin(&tempty_bar[buf], (use & 1u) ^ 1u, abort_flag)) return;
        tc_fence_after();
        const uint32_t acc = tmem + (uint32_t)(buf * a.acc_cols);
        int sj = xs;  // slot of activation row y - 1 (y = y0 + j)
        for (int j = 0; j < it.len; ++j) {
            if (!wait_or_abort_spin(&full_bar[s], ph, abort_flag)) return;
            fence_proxy_async_smem();  // cp.async wrote through the generic proxy
            tc_fence_after();
            const uint64_t bd = smem_desc(sbase + a.g_ring + s * a.g_slot, 128, sbo, 0);
            for (int ty = 0; ty < 3; ++ty) {
                int slot = sj + ty;  // activation row y + ty - 1
                if (slot >= a.xr) slot -= a.xr;
                const uint32_t xbase = sbase + (uint32_t)slot * a.x_slot;
                for (int mt = 0; mt < a.m_tiles; ++mt) {
                    // M tile mt: MN atoms 2 mt and 2 mt + 1
                    const uint64_t ad = smem_desc(xbase + ((uint32_t)mt << 11), 1024, a_sbo, 2);
                    const uint32_t d = acc + (uint32_t)((ty * a.m_tiles + mt) * a.N);
                    for (int kk = 0; kk < a.nk; ++kk)
                        umma_bf16(d, ad + (uint64_t)kk * a_kstep, bd + (uint64_t)(16 * kk), idesc,
                                  (j > 0 || kk > 0) ? 1u : 0u);
                }
            }
            umma_commit(&empty_bar[s]);
            // the row above this one is used by no later stage; after the item's last stage,
            // neither are the other two
            umma_commit(&xempty_bar[sj]);
            if (j == it.len - 1) {
                umma_commit(&xempty_bar[sj + 1 < a.xr ? sj + 1 : sj + 1 - a.xr]);
                umma_commit(&xempty_bar[sj + 2 < a.xr ? sj + 2 : sj + 2 - a.xr]);
            }
            if (++s == (uint32_t)S) s = 0, ph ^= 1u;
            if (++sj == a.xr) sj = 0;
        }
        xs = (xs + it.len + 2) % a.xr;
        umma_commit(&tfull_bar[buf]);
        ++local;
    }
}

__device__ void wr_drain(const WrArgs &a, uint32_t tmem, uint64_t *tfull_bar, uint64_t *tempty_bar,
                         volatile int *abort_flag, long long f, long long f_end) {
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int q = warp & 3;  // TMEM lane quarter this warp may access
    const int mrows = 3 * a.Cin;
    int local = 0;
    WrItem it;
    while (wr_next(a, f, f_end, it)) {
        const int buf = a.nbuf == 2 ? (local & 1) : 0;
        const uint32_t use = a.nbuf == 2 ? ((uint32_t)local >> 1) : (uint32_t)local;
        const bool ok = wait_or_abort(&tfull_bar[buf], use & 1u, abort_flag);
        if (!__all_sync(0xffffffffu, ok)) return;
        tc_fence_after();
        for (int mt = 0; mt < a.m_tiles; ++mt) {
            const int m = mt * UM + q * 32 + lane;  // (tx, c) = (m / Cin, m mod Cin)
            if (mt * UM + q * 32 >= mrows) continue;  // warp-uniform: no real row in this quarter
            const int tx = m / a.Cin, c = m - tx * a.Cin;
            for (int ty = 0; ty < 3; ++ty) {
#pragma unroll 1
                for (int c0 = 0; c0 < a.N; c0 += 16) {
                    uint32_t r[16];
                    tmem_ld16(tmem + ((uint32_t)(q * 32) << 16) +
                                  (uint32_t)(buf * a.acc_cols + (ty * a.m_tiles + mt) * a.N + c0),
                              r);
                    const int o0 = it.nt * a.N + c0;
                    if (m >= mrows) continue;
#pragma unroll
                    for (int e = 0; e < 16; ++e) {
                        if (o0 + e < a.Cout)
                            atomicAdd(a.dW + ((long)((o0 + e) * 3 + ty) * 3 + tx) * a.Cin + c, __uint_as_float(r[e]));
                    }
                }
            }
        }
        tc_fence_before();
        mbar_arrive(&tempty_bar[buf]);
        ++local;
    }
}

__global__ void __launch_bounds__(kWgThreads, 1) wgrad_ring_kernel(const WrArgs a) {
    extern __shared__ unsigned char smem_raw[];
    __shared__ __align__(8) uint64_t full_bar[kWgMaxStages], empty_bar[kWgMaxStages], xempty_bar[kWrMaxXr],
        tfull_bar[2], tempty_bar[2];
    __shared__ uint32_t tmem_slot;
    __shared__ int abort_word;
    volatile int *abort_flag = &abort_word;
    const int warp = threadIdx.x >> 5;
    const uint32_t sbase = (smem_addr(smem_raw) + 1023u) & ~1023u;
    const long long per_blk = (long long)a.n_tiles * a.lb;
    const long long f_total = ((long long)a.total + a.lb - 1) / a.lb * per_blk;
    const long long f0 = (long long)blockIdx.x * a.f_per_cta;
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
        for (int s = 0; s < a.xr; ++s) mbar_init(&xempty_bar[s], 1);
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
        wr_produce(a, sbase, full_bar, empty_bar, xempty_bar, abort_flag, f0, f1);
    } else if (warp == kWgMmaWarp) {
        if ((threadIdx.x & 31) == 0)
            wr_issue(a, sbase, tmem, full_bar, empty_bar, xempty_bar, tfull_bar, tempty_bar, abort_flag, f0, f1);
    } else if (warp >= kWgEpiWarp0) {
        wr_drain(a, tmem, tfull_bar, tempty_bar, abort_flag, f0, f1);
    }

    tc_fence_before();
    __syncthreads();
    if (warp == kWgMmaWarp)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(a.tmem_cols)
                     : "memory");
}

// ------------------------------------------------------------------ host side
struct WrPlan {
    WrArgs a;
    size_t smem;
    int grid;
};

// Plans the launch; false if the accumulators of one N tile of at least 16 columns do not
// fit in TMEM, or no ring fits in shared memory.
bool wr_plan(int B, int H, int W, int Cin, int Cout, int sms, WrPlan &pl) {
    WrArgs &a = pl.a;
    a = WrArgs{};
    a.H = H, a.W = W, a.Cin = Cin, a.Cout = Cout;
    a.ncc = Cin / 8;
    a.m_tiles = (3 * Cin + UM - 1) / UM;
    a.n_atoms = (3 * Cin + 63) / 64;
    int nmax = 512 / (3 * a.m_tiles) / 16 * 16;
    if (nmax > kWgMaxN) nmax = kWgMaxN;
    if (nmax < 16) return false;
    a.n_tiles = (Cout + nmax - 1) / nmax;
    a.N = ((Cout + a.n_tiles - 1) / a.n_tiles + 15) / 16 * 16;
    a.acc_cols = 3 * a.m_tiles * a.N;
    a.nbuf = 2 * a.acc_cols <= 512 ? 2 : 1;
    uint32_t tc = 32;
    while ((int)tc < a.nbuf * a.acc_cols) tc <<= 1;
    a.tmem_cols = tc;
    const int seg0 = W < 128 ? (W + 15) / 16 * 16 : 128;
    const int cands[4] = {seg0, 64, 32, 16};
    for (int ci = 0; ci < 8 && !a.seg; ++ci) {
        const int seg = cands[ci & 3];
        const int min_stages = ci < 4 ? kWgGoodStages : kWgMinStages;
        if ((ci & 3) > 0 && seg >= seg0) continue;
        const int nk = seg / 16;
        if (3 * a.ncc * seg > kWgMaxUnits * kWgProducers || a.N / 8 * seg > kWgMaxUnits * kWgProducers) continue;
        const uint32_t xs = (uint32_t)(seg / 8 * a.n_atoms) << 10, gs = (uint32_t)(a.N / 8 * seg * 16);
        for (int S = kWgMaxStages; S >= min_stages; --S) {
            const int xr = S + 2;
            const uint32_t rings = (uint32_t)xr * xs + (uint32_t)S * gs;
            // A reads: MN atoms up to 2 m_tiles - 1 of the last pixel group of the last slot
            const uint32_t a_reach = (uint32_t)(xr - 1) * xs +
                                     ((uint32_t)((2 * (nk - 1) + 1) * a.n_atoms + 2 * (a.m_tiles - 1) + 1) << 10) +
                                     1024u;
            const uint32_t total = rings > a_reach ? rings : a_reach;
            if (total <= kWgBudget) {
                a.seg = seg, a.nk = nk, a.x_slot = xs, a.g_slot = gs;
                a.g_ring = (uint32_t)xr * xs;
                a.stages = S, a.xr = xr;
                pl.smem = total + 1024;
                break;
            }
        }
    }
    if (!a.seg) return false;
    a.nseg = (W + a.seg - 1) / a.seg;
    const long long stages = (long long)B * a.nseg * H;
    if (stages >= (1LL << 31)) return false;
    a.total = (int)stages;
    // each CTA takes about one block of every N tile
    const long long work = stages * a.n_tiles;
    const long long per = (work + sms - 1) / sms;
    long long lb = (per + a.n_tiles - 1) / a.n_tiles;
    if (lb < 4) lb = 4;
    a.lb = (int)lb;
    const long long f_total = (stages + lb - 1) / lb * a.n_tiles * lb;
    a.f_per_cta = (f_total + sms - 1) / sms;
    pl.grid = (int)((f_total + a.f_per_cta - 1) / a.f_per_cta);
    return true;
}

rbgs_status wr_launch(const uint16_t *X, const uint16_t *G, float *dW, int B, int H, int W, int Cin, int Cout,
                      cudaStream_t s, bool *launched) {
    *launched = false;
    WrPlan pl;
    if (!wr_plan(B, H, W, Cin, Cout, sm_count(), pl)) return RBGS_OK;
    static const cudaError_t attr = cudaFuncSetAttribute(wgrad_ring_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                         (int)(kWgBudget + 1024));
    RBGS_CUDA(attr);
    pl.a.X = X, pl.a.G = G, pl.a.dW = dW;
    wgrad_ring_kernel<<<pl.grid, kWgThreads, pl.smem, s>>>(pl.a);
    RBGS_LAUNCH_CHECK();
    *launched = true;
    return RBGS_OK;
}
