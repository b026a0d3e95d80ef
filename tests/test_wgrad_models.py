"""CPU models of the two shared-memory-descriptor weight-gradient kernels (the tap-row kernel
of csrc/conv_wgrad.cuh and the ring kernel of csrc/conv_wgrad_ring.cuh), written from their
descriptions: the launch plan, the staging of each operand into shared memory, the MMA
descriptors' reading of it (the layouts the kernels use: MN-major without swizzle, 16-byte
rows, LBO = 128 B between K groups, SBO between channel groups; MN-major with the 128-byte
swizzle, 1024-byte atoms of 8 pixels x 64 rows, chunk ch of pixel row r at ch ^ r) and the
epilogue's scatter into dW.

Each model runs small problems of exact small integers through that data flow and must give
the direct sums exactly; every address a descriptor forms must lie inside the shared-memory
allocation the plan reserves (the A operand reads 128 rows even when fewer are real), and the
ring model runs its producer as far ahead as the kernel's barriers allow, so a slot is never
overwritten before its last reader and the producer never waits on a stage it has yet to
fill.  These check the index arithmetic and bookkeeping of the design, on the CPU; the GPU
tests (tests/test_gpu_unet.py) check the kernels themselves against the oracle.
"""
import numpy as np
import pytest

UM, MAX_N, MAX_STAGES, GOOD_STAGES, MIN_STAGES = 128, 160, 16, 6, 4
BUDGET = 210 * 1024
PRODUCERS, MAX_UNITS = 256, 8


def _direct(x, g):
    """dW[o][ty][tx][c] = sum over pixels of g[b,y,x,o] x[b,y+ty-1,x+tx-1,c], zero padding."""
    B, H, W, _ = x.shape
    xp = np.zeros((B, H + 2, W + 2, x.shape[3]))
    xp[:, 1:-1, 1:-1] = x
    out = np.zeros((g.shape[3], 3, 3, x.shape[3]))
    for ty in range(3):
        for tx in range(3):
            out[:, ty, tx, :] = np.einsum("bhwo,bhwc->oc", g, xp[:, ty:ty + H, tx:tx + W, :])
    return out


def _inputs(B, H, W, Cin, Cout, seed):
    rng = np.random.default_rng(seed)
    return (rng.integers(-3, 4, (B, H, W, Cin)).astype(float),
            rng.integers(-3, 4, (B, H, W, Cout)).astype(float))


def _tiles(ndim):
    pad = (ndim + 15) // 16 * 16
    nt = (pad + MAX_N - 1) // MAX_N
    return nt, ((ndim + nt - 1) // nt + 15) // 16 * 16


def _segs(W):
    seg0 = (W + 15) // 16 * 16 if W < 128 else 128
    for ci in range(8):
        seg = [seg0, 64, 32, 16][ci & 3]
        if (ci & 3) > 0 and seg >= seg0:
            continue
        yield seg, (GOOD_STAGES if ci < 4 else MIN_STAGES)


def _read_plain(smem, start, sbo, rows):
    """The 16 K columns (pixels) of `rows` MN rows from a descriptor without swizzle."""
    m = np.arange(rows)[:, None]
    k = np.arange(16)[None, :]
    addr = start + (m // 8) * sbo + (k // 8) * 128 + (k % 8) * 16 + (m % 8) * 2
    assert addr.min() >= 0 and addr.max() + 2 <= 2 * smem.size
    return smem[addr // 2]


def _read_sw128(smem, start, sbo, rows):
    """The same from an MN-major 128-byte-swizzled descriptor with LBO = 1024 (atom-aligned)."""
    assert start % 1024 == 0
    m = np.arange(rows)[:, None]
    k = np.arange(16)[None, :]
    addr = (start + (m // 64) * 1024 + (k // 8) * sbo + (k % 8) * 128 + ((((m % 64) // 8) ^ (k % 8)) * 16)
            + (m % 8) * 2)
    assert addr.min() >= 0 and addr.max() + 2 <= 2 * smem.size
    return smem[addr // 2]


# ---------------------------------------------------------------- tap-row kernel
def taprow_plan(B, H, W, Cin, Cout, sms=152):
    ntg, ng = _tiles(Cin)
    ntx, nx = _tiles(Cout)
    mtg, mtx = (Cout + 127) // 128, (Cin + 127) // 128
    xa = mtx * ntx * nx < mtg * ntg * ng
    a = dict(xa=xa, m_tiles=mtx if xa else mtg, n_tiles=ntx if xa else ntg, N=nx if xa else ng)
    mdim = Cin if xa else Cout
    a["ngA"], a["ngB"] = min(16, (mdim + 7) // 8), a["N"] // 8
    a["ncombo"] = 3 * a["m_tiles"] * a["n_tiles"]
    ngx, ngg = (a["ngA"], a["ngB"]) if xa else (a["ngB"], a["ngA"])
    for seg, mins in _segs(W):
        nk = seg // 16
        lenA, lenB = (seg + 8, seg) if xa else (seg, seg + 8)
        As, Bs = a["ngA"] * lenA * 16, a["ngB"] * lenB * 16
        if (16 * (nk - 1) + (0 if xa else 2)) * 16 + (a["ngB"] - 1) * lenB * 16 + 256 > Bs:
            continue
        if ngx * (seg + 2) > MAX_UNITS * PRODUCERS or ngg * seg > MAX_UNITS * PRODUCERS:
            continue
        for S in range(MAX_STAGES, mins - 1, -1):
            reach = (S - 1) * As + (16 * (nk - 1) + (2 if xa else 0)) * 16 + 15 * lenA * 16 + 256
            total = max(S * (As + Bs), reach)
            if total <= BUDGET:
                a.update(seg=seg, nk=nk, lenA=lenA, lenB=lenB, a_slot=As, b_slot=Bs, b_ring=S * As,
                         stages=S, smem=total)
                break
        if "seg" in a:
            break
    if "seg" not in a:
        return None
    a["nseg"] = (W + a["seg"] - 1) // a["seg"]
    a["total"] = B * H * a["nseg"]
    cols = 3 * a["N"]
    a["nbuf"] = 2 if 2 * cols <= 512 else 1
    per = (a["total"] * a["ncombo"] + sms - 1) // sms
    a["lb"] = min(256, max(8, per // 3))
    a["f_total"] = (a["total"] + a["lb"] - 1) // a["lb"] * a["ncombo"] * a["lb"]
    a["f_per_cta"] = (a["f_total"] + sms - 1) // sms
    a["grid"] = (a["f_total"] + a["f_per_cta"] - 1) // a["f_per_cta"]
    return a


def _taprow_items(a, f, fe):
    per = a["ncombo"] * a["lb"]
    while f < fe:
        blk, rem = divmod(f, per)
        combo, j0 = divmod(rem, a["lb"])
        s0 = blk * a["lb"] + j0
        n = min(a["lb"] - j0, fe - f)
        f += n
        if a["total"] - s0 > 0:
            yield combo, s0, min(n, a["total"] - s0)


def run_taprow(B, H, W, Cin, Cout, seed=0):
    a = taprow_plan(B, H, W, Cin, Cout)
    x, g = _inputs(B, H, W, Cin, Cout, seed)
    dW = np.zeros((Cout, 3, 3, Cin))
    xa, seg = a["xa"], a["seg"]
    mdim, ndim = (Cin, Cout) if xa else (Cout, Cin)
    seen = np.zeros(a["total"] * a["ncombo"], int)
    for cta in range(a["grid"]):
        f0 = cta * a["f_per_cta"]
        for combo, s0, n in _taprow_items(a, f0, min(f0 + a["f_per_cta"], a["f_total"])):
            ty, rest = divmod(combo, a["m_tiles"] * a["n_tiles"])
            mt, nt = divmod(rest, a["n_tiles"])
            xc0, gc0 = (mt * 128, nt * a["N"]) if xa else (nt * a["N"], mt * 128)
            D = np.zeros((3, 128, a["N"]))
            for j in range(n):
                stage = s0 + j
                seen[combo * a["total"] + stage] += 1
                r, sg = divmod(stage, a["nseg"])
                b, y = divmod(r, H)
                x0 = sg * seg
                smem = np.full(a["smem"] // 2, np.nan)   # NaN: never written
                s = a["stages"] - 1                      # the last slot reaches furthest
                sa, sb = s * a["a_slot"], a["b_ring"] + s * a["b_slot"]
                ngx, ngg = (a["ngA"], a["ngB"]) if xa else (a["ngB"], a["ngA"])
                lenx, leng = (a["lenA"], a["lenB"]) if xa else (a["lenB"], a["lenA"])

                def stage_row(T, C, yy, c0, ng, npix, ln, xs, slot):
                    for p in range(npix):
                        for gg in range(ng):
                            xx, c = xs + p, c0 + gg * 8
                            ok = 0 <= yy < H and 0 <= xx < W and c < C
                            addr = slot + (gg * ln + p) * 16
                            assert 0 <= addr and addr + 16 <= a["smem"]
                            smem[addr // 2:addr // 2 + 8] = T[b, yy, xx, c:c + 8] if ok else 0.0

                stage_row(x, Cin, y + ty - 1, xc0, ngx, seg + 2, lenx, x0 - 1, sa if xa else sb)
                stage_row(g, Cout, y, gc0, ngg, seg, leng, x0, sb if xa else sa)
                real = min(128, mdim - mt * 128)
                for kk in range(a["nk"]):
                    for tx in range(3):
                        A = _read_plain(smem, sa + (16 * kk + (tx if xa else 0)) * 16, a["lenA"] * 16, 128)
                        Bm = _read_plain(smem, sb + (16 * kk + (0 if xa else tx)) * 16, a["lenB"] * 16, a["N"])
                        assert not np.isnan(A[:real]).any() and not np.isnan(Bm).any()
                        D[tx] += np.nan_to_num(A) @ Bm.T
            for tx in range(3):
                for m in range(min(128, mdim - mt * 128)):
                    for nn in range(min(a["N"], ndim - nt * a["N"])):
                        o, c = (nt * a["N"] + nn, mt * 128 + m) if xa else (mt * 128 + m, nt * a["N"] + nn)
                        dW[o, ty, tx, c] += D[tx, m, nn]
    assert (seen == 1).all()
    return a, dW, _direct(x, g)


# ---------------------------------------------------------------- ring kernel
def ring_plan(B, H, W, Cin, Cout, sms=152):
    a = dict(ncc=Cin // 8, m_tiles=(3 * Cin + 127) // 128, n_atoms=(3 * Cin + 63) // 64)
    nmax = min(MAX_N, 512 // (3 * a["m_tiles"]) // 16 * 16)
    if nmax < 16:
        return None
    a["n_tiles"] = (Cout + nmax - 1) // nmax
    a["N"] = ((Cout + a["n_tiles"] - 1) // a["n_tiles"] + 15) // 16 * 16
    acc = 3 * a["m_tiles"] * a["N"]
    a["nbuf"] = 2 if 2 * acc <= 512 else 1
    assert a["nbuf"] * acc <= 512
    for seg, mins in _segs(W):
        nk = seg // 16
        if 3 * a["ncc"] * seg > MAX_UNITS * PRODUCERS or a["N"] // 8 * seg > MAX_UNITS * PRODUCERS:
            continue
        xs, gs = seg // 8 * a["n_atoms"] * 1024, a["N"] // 8 * seg * 16
        for S in range(MAX_STAGES, mins - 1, -1):
            xr = S + 2
            reach = (xr - 1) * xs + ((2 * (nk - 1) + 1) * a["n_atoms"] + 2 * (a["m_tiles"] - 1) + 1) * 1024 + 1024
            total = max(xr * xs + S * gs, reach)
            if total <= BUDGET:
                a.update(seg=seg, nk=nk, x_slot=xs, g_slot=gs, g_ring=xr * xs, stages=S, xr=xr, smem=total)
                break
        if "seg" in a:
            break
    if "seg" not in a:
        return None
    a["nseg"] = (W + a["seg"] - 1) // a["seg"]
    a["total"] = B * a["nseg"] * H
    per = (a["total"] * a["n_tiles"] + sms - 1) // sms
    a["lb"] = max(4, (per + a["n_tiles"] - 1) // a["n_tiles"])
    a["f_total"] = (a["total"] + a["lb"] - 1) // a["lb"] * a["n_tiles"] * a["lb"]
    a["f_per_cta"] = (a["f_total"] + sms - 1) // sms
    a["grid"] = (a["f_total"] + a["f_per_cta"] - 1) // a["f_per_cta"]
    return a


def _ring_items(a, H, f, fe):
    per = a["n_tiles"] * a["lb"]
    while f < fe:
        blk, rem = divmod(f, per)
        nt, j0 = divmod(rem, a["lb"])
        s0 = blk * a["lb"] + j0
        n = min(a["lb"] - j0, fe - f)
        if a["total"] - s0 <= 0:
            f += n
            continue
        n = min(n, a["total"] - s0, H - s0 % H)
        f += n
        yield nt, s0, n


def run_ring(B, H, W, Cin, Cout, seed=0, sms=152):
    a = ring_plan(B, H, W, Cin, Cout, sms)
    x, g = _inputs(B, H, W, Cin, Cout, seed)
    dW = np.zeros((Cout, 3, 3, Cin))
    seg, S, xr, n_atoms = a["seg"], a["stages"], a["xr"], a["n_atoms"]
    seen = np.zeros(a["total"] * a["n_tiles"], int)
    for cta in range(a["grid"]):
        f0 = cta * a["f_per_cta"]
        items = list(_ring_items(a, H, f0, min(f0 + a["f_per_cta"], a["f_total"])))
        stages = [(k, j) for k, (_, _, n) in enumerate(items) for j in range(n)]
        # producer: rows loaded per stage, with their load counters
        loads, counter = [], 0
        for k, j in stages:
            nt, s0, n = items[k]
            strip, y = divmod(s0 + j, H)
            b, sc = divmod(strip, a["nseg"])
            rows = []
            for r in ([-1, 0, 1] if j == 0 else [1]):
                rows.append((counter, b, y + r, sc * seg))
                counter += 1
            loads.append(rows)
        # MMA side: the rows each stage reads, and those that die after it
        reads, dies, xc = [], [], 0
        for k, (nt, s0, n) in enumerate(items):
            for j in range(n):
                reads.append([xc + j + ty for ty in range(3)])
                dies.append([xc + j] + ([xc + j + 1, xc + j + 2] if j == n - 1 else []))
            xc += n + 2
        assert xc == counter
        smem = np.full(a["smem"] // 2, np.nan)
        slot_row, row_of, dead, gtag = {}, {}, set(), [None] * S
        P, done, D = 0, -1, {}

        def can_fill(p):  # the barriers: the stage slot freed, the activation slots' rows dead
            if p >= len(stages) or p - S > done:
                return False
            return all(c - xr < 0 or c - xr in dead for c, *_ in loads[p])

        for m in range(len(stages)):
            while can_fill(P):
                k, j = stages[P]
                nt, s0, n = items[k]
                strip, y = divmod(s0 + j, H)
                b, sc = divmod(strip, a["nseg"])
                x0 = sc * seg
                for c, bb, yy, xx0 in loads[P]:
                    slot = c % xr
                    slot_row[slot], row_of[c] = c, yy
                    for tx in range(3):
                        for gg in range(a["ncc"]):
                            for p in range(seg):
                                xx = xx0 - 1 + p + tx
                                mg, r8 = tx * a["ncc"] + gg, p & 7
                                addr = (slot * a["x_slot"] + ((p >> 3) * n_atoms + (mg >> 3)) * 1024 + r8 * 128
                                        + ((mg & 7) ^ r8) * 16)
                                assert addr + 16 <= a["smem"]
                                ok = 0 <= yy < H and 0 <= xx < W
                                smem[addr // 2:addr // 2 + 8] = x[bb, yy, xx, gg * 8:gg * 8 + 8] if ok else 0.0
                s = P % S
                gb, gc0 = a["g_ring"] + s * a["g_slot"], nt * a["N"]
                for gg in range(a["N"] // 8):
                    for p in range(seg):
                        xx, c = x0 + p, gc0 + gg * 8
                        addr = gb + (gg * seg + p) * 16
                        assert addr + 16 <= a["smem"]
                        smem[addr // 2:addr // 2 + 8] = g[b, y, xx, c:c + 8] if (xx < W and c < Cout) else 0.0
                gtag[s] = P
                P += 1
            assert P > m, "the producer cannot fill the stage the MMAs need"
            k, j = stages[m]
            nt, s0, n = items[k]
            s = m % S
            assert gtag[s] == m
            y = (s0 + j) % H
            if j == 0:
                D[k] = np.zeros((3, a["m_tiles"], 128, a["N"]))
            for ty in range(3):
                c = reads[m][ty]
                slot = c % xr
                assert slot_row[slot] == c and row_of[c] == y + ty - 1
                for mt in range(a["m_tiles"]):
                    real = min(128, 3 * Cin - mt * 128)
                    for kk in range(a["nk"]):
                        A = _read_sw128(smem, slot * a["x_slot"] + mt * 2048 + 2 * kk * n_atoms * 1024,
                                        n_atoms * 1024, 128)
                        Bm = _read_plain(smem, a["g_ring"] + s * a["g_slot"] + 16 * kk * 16, seg * 16, a["N"])
                        assert not np.isnan(A[:real]).any() and not np.isnan(Bm).any()
                        D[k][ty, mt] += np.nan_to_num(A) @ Bm.T
            done = m
            seen[nt * a["total"] + s0 + j] += 1
            dead.update(dies[m])
            if j == n - 1:
                for ty in range(3):
                    for mt in range(a["m_tiles"]):
                        for mm in range(min(128, 3 * Cin - mt * 128)):
                            tx, c = divmod(mt * 128 + mm, Cin)
                            for nn in range(min(a["N"], Cout - nt * a["N"])):
                                dW[nt * a["N"] + nn, ty, tx, c] += D[k][ty, mt, mm, nn]
    assert (seen == 1).all()
    return a, dW, _direct(x, g)


TAPROW_SHAPES = [(2, 8, 8, 16, 32), (1, 13, 11, 32, 64), (2, 16, 16, 96, 32), (1, 7, 5, 8, 48),
                 (2, 4, 20, 16, 256), (1, 3, 40, 384, 128), (1, 3, 200, 32, 32), (2, 5, 9, 32, 16)]
RING_SHAPES = [(2, 5, 8, 16, 32), (1, 7, 11, 32, 64), (2, 3, 16, 96, 32), (1, 4, 5, 8, 48), (2, 3, 20, 64, 64),
               (1, 2, 40, 48, 16), (1, 3, 200, 16, 16), (3, 1, 9, 32, 16), (1, 6, 12, 64, 128)]


@pytest.mark.parametrize("shape", TAPROW_SHAPES)
def test_taprow_model_gives_the_direct_sums(shape):
    a, got, want = run_taprow(*shape)
    assert a["stages"] >= MIN_STAGES and 3 * a["N"] * a["nbuf"] <= 512
    assert np.array_equal(got, want)


@pytest.mark.parametrize("shape", RING_SHAPES)
def test_ring_model_gives_the_direct_sums(shape):
    _, got, want = run_ring(*shape)
    assert np.array_equal(got, want)


@pytest.mark.parametrize("sms", [1, 3])
def test_ring_model_with_many_items_per_cta(sms):
    """Few CTAs: each walks several strips and N tiles, so items start and end inside its
    range and the activation ring carries over from one item to the next."""
    for shape in ((2, 5, 8, 16, 32), (1, 6, 12, 64, 128), (3, 2, 9, 32, 16)):
        _, got, want = run_ring(*shape, sms=sms)
        assert np.array_equal(got, want)


# the network's 3x3 layers at the training batch (16 x 256^2 at level 0): (W, Cin, Cout)
NETWORK = [(256, 16, 32), (256, 32, 32), (128, 32, 64), (128, 64, 64), (64, 64, 128), (64, 128, 128),
           (32, 128, 256), (32, 256, 256), (64, 384, 128), (64, 128, 128), (128, 192, 64), (128, 64, 64),
           (256, 96, 32), (256, 32, 32)]


def test_plans_fit_every_network_layer_and_the_automatic_choice():
    """Both plans fit every network layer they are chosen for within the shared-memory budget,
    TMEM and the producers' copy tables; and the automatic rule (ring for Cin <= 32, tap row
    where rows have >= 64 pixels and >= 40 stages fall to every SM, gather otherwise) picks,
    layer by layer, the kernel that measured fastest."""
    measured_best = ["ring", "ring", "ring", "taprow", "gather", "gather", "gather", "gather", "taprow",
                     "gather", "taprow", "taprow", "taprow", "ring"]
    for (W, Cin, Cout), best in zip(NETWORK, measured_best):
        r, t = ring_plan(16, W, W, Cin, Cout), taprow_plan(16, W, W, Cin, Cout)
        assert t is not None
        if Cin <= 32:
            choice = "ring" if r is not None else "taprow"
        elif W >= 64 and t["f_per_cta"] >= 40:
            choice = "taprow"
        else:
            choice = "gather"
        assert choice == best, (W, Cin, Cout, choice)
        if choice == "ring":
            assert r["smem"] <= BUDGET and 3 * r["m_tiles"] * r["N"] * r["nbuf"] <= 512
