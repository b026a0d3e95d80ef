"""GPU parity of the fused FP64 update (rbgs_opts.fma = 1) through the C ABI.

The fused update is exactly specified (Eq. (1)'s five terms on a 64-bit fixed-point grid,
summed exactly, rounded once; the grid chosen per block of sweeps from max |u| and
max |h2 f|), so the GPU iterate must equal oracle.sweeps_fused bit for bit.  It must also
stay within 1e-13 relative max-norm of the bit-exact iteration after the same sweeps (the
tolerance set for this mode).  Sizes span several blocks and ragged strips; both widths
per thread, several strip heights, the cached graphs of small grids, blocks of sweeps
longer than one scale block, solve loops, non-finite input and the full 16384^2 grid
(sampled windows) are covered.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2607_01735_gb300 as rb
import synth

from test_gpu_parity import RESID_RTOL, SIZES, _assert_bits, _problem, _window_inputs

pytestmark = pytest.mark.gpu

TOL = 1e-13  # relative max-norm against the bit-exact iterate


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_01735_gb300 import build
    build.build_library()
    rb.load_library()


def _run(n, h2, f, u0, sweep_calls, **opts):
    fd = torch.from_numpy(f).cuda()
    ud = torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, fma=1, **opts) as s:
        for k in sweep_calls:
            s.sweep(k)
        s.get_solution(out)
        rho = s.residual()
    return out.cpu().numpy(), rho


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


@pytest.mark.parametrize("values", [2, 4])
@pytest.mark.parametrize("n", SIZES)
def test_fused_bit_exact_against_fused_oracle(n, values):
    f, u0 = _problem(n, 311 + n)
    h2 = synth.h_squared(n)
    sweeps = 7 if n > 300 else 13
    got, rho = _run(n, h2, f, u0, [sweeps], sweep_values=values)
    ref = u0.copy()
    oracle.sweeps_fused(ref, f, h2, sweeps)
    _assert_bits(got, ref)
    # the residual walks both colours after a fused sweep
    rho_ref = oracle.residual(ref, f, h2)[0]
    assert abs(rho - rho_ref) <= RESID_RTOL * rho_ref
    plain = u0.copy()
    oracle.sweeps(plain, f, h2, sweeps)
    assert _relmax(got, plain) <= TOL


@pytest.mark.parametrize("rows", [1, 3, 16, 40])
def test_fused_strip_heights(rows):
    n = 257
    f, u0 = _problem(n, 17)
    h2 = synth.h_squared(n)
    got, _ = _run(n, h2, f, u0, [9], tile_rows=rows)
    ref = u0.copy()
    oracle.sweeps_fused(ref, f, h2, 9)
    _assert_bits(got, ref)


def test_fused_blocks_of_sweeps_and_cached_graphs():
    """One call of 1100 sweeps is a block of 1024 and one of 76 (graphs of 32 sweeps plus
    direct launches inside each), then calls of 40 and 5 sweeps are blocks of their own."""
    n = 63
    f, u0 = _problem(n, 23)
    h2 = synth.h_squared(n)
    got, _ = _run(n, h2, f, u0, [1100, 40, 5])
    ref = u0.copy()
    for k in (1100, 40, 5):
        oracle.sweeps_fused(ref, f, h2, k)
    _assert_bits(got, ref)
    plain = u0.copy()
    oracle.sweeps(plain, f, h2, 1145)
    assert _relmax(got, plain) <= TOL


def test_fused_solve_loop_matches_oracle_checks():
    """rbgs_solve with fma = 1: rho before the first sweep, then a block of check_every
    sweeps per check; the same checks replayed on the oracle give the same sweeps and bits."""
    n, every, tol = 47, 50, 1e-6
    f, u0 = _problem(n, 29, interior=False)
    h2 = synth.h_squared(n)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, fma=1, check_every=every) as s:
        done, rho, _ = s.solve(tol)
        s.get_solution(out)
    ref = u0.copy()
    ref_done, ref_rho = 0, oracle.residual(ref, f, h2)[0]
    while not ref_rho <= tol:
        oracle.sweeps_fused(ref, f, h2, every)
        ref_done += every
        ref_rho = oracle.residual(ref, f, h2)[0]
    assert done == ref_done
    _assert_bits(out.cpu().numpy(), ref)
    assert abs(rho - ref_rho) <= RESID_RTOL * ref_rho


def test_fused_set_problem_rescales():
    """A second problem loaded into the same context (a larger f) gets its own max |h2 f|."""
    n = 130
    h2 = synth.h_squared(n)
    f1, u1 = _problem(n, 41)
    f2, u2 = _problem(n, 42)
    f2 *= 1000.0
    fd, ud = torch.from_numpy(f1).cuda(), torch.from_numpy(u1).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, fma=1) as s:
        s.sweep(11)
        s.set_problem(torch.from_numpy(f2).cuda(), torch.from_numpy(u2).cuda())
        s.sweep(11)
        s.get_solution(out)
    ref = u2.copy()
    oracle.sweeps_fused(ref, f2, h2, 11)
    _assert_bits(out.cpu().numpy(), ref)


def test_fused_nonfinite_rhs_reports_status():
    n = 40
    f, u0 = _problem(n, 5)
    f[7, 9] = np.nan
    h2 = synth.h_squared(n)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, fma=1) as s:
        s.sweep(3)
        s.get_solution(out)
        with pytest.raises(rb.RbgsError) as e:
            s.residual()
        assert e.value.status == rb.RBGS_ENONFINITE
    got = out.cpu().numpy()
    assert np.all(np.isnan(got[1:-1, 1:-1])) and np.all(got[0] == u0[0])


def test_solve_stops_when_the_residual_stalls():
    """A tolerance below the rounding floor: the solve stops after stall_checks checks
    without a new minimum of rho, long before max_sweeps, with the iterate kept.  The fused
    iteration settles on a fixed point of its own rounding, where the residual (formed with
    four roundings) keeps a floor above zero.  (The bit-exact iteration on this grid instead
    reaches a point where every rt is exactly zero, rho = 0, as the oracle does.)"""
    n = 31
    f, u0 = _problem(n, 3)
    h2 = synth.h_squared(n)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    with rb.Solver(n, h2, fd, ud, fma=1, check_every=200, stall_checks=5, max_sweeps=10 ** 9) as s:
        with pytest.raises(rb.RbgsError) as e:
            s.solve(0.0)
        assert e.value.status == rb.RBGS_ENOTCONV and "stalled" in str(e.value)
        done, rho, st = s.solve(0.0, allow_not_converged=True)
        assert st == rb.RBGS_ENOTCONV and done == 5 * 200 and 0.0 < rho < 1e-12
    ref = u0.copy()
    done, rho = oracle.solve(ref, f, h2, 0.0, 200, 10 ** 6)
    assert rho == 0.0
    with rb.Solver(n, h2, fd, ud, check_every=200, stall_checks=-1) as s:
        assert s.solve(0.0) == (done, 0.0, rb.RBGS_OK)


@pytest.mark.slow
def test_fused_full_size_16384_sampled():
    """16384^2, f ~ U(-1,1) stream 1, zero ring, u0 = 0, 200 fused sweeps (one block); the
    sampled points recomputed by the fused oracle on their windows at the whole grid's
    scale, and within 1e-13 of the bit-exact iteration there."""
    n, sweeps, stream = 16384, 200, 1
    h2 = synth.h_squared(n)
    # max |h2 f| of the whole grid, from the generator on the CPU in slices
    fmax, step = 0.0, 1 << 24
    for start in range(0, n * n, step):
        cnt = min(step, n * n - start)
        fmax = max(fmax, float(torch.max(torch.abs(synth.uniform01(stream, cnt, start) * 2.0 - 1.0))))
    bound = (0.0, float(np.float64(h2) * np.float64(fmax)))
    fd = synth.uniform_pm1_grid(n, stream, device="cuda")
    ud = torch.zeros(n + 2, n + 2, dtype=torch.float64, device="cuda")
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, fma=1) as s:
        s.sweep(sweeps)
        s.get_solution(out)
    del ud, fd
    r = 2 * sweeps + 1
    for (i, j) in [(1, 1), (1, n), (n, 1), (n, n), (n // 2, n // 2 + 1), (777, 12345), (16000, 3)]:
        a, c, fw = _window_inputs(n, stream, i, j, r)
        parity = (a - 1 + c - 1) & 1
        uw = np.zeros((fw.shape[0] + 2, fw.shape[1] + 2))
        oracle.sweeps_fused(uw, fw, h2, sweeps, parity, bound)
        got = float(out[i, j].item())
        assert got == uw[i - a + 1, j - c + 1], (i, j)
        up = np.zeros_like(uw)
        oracle.sweeps(up, fw, h2, sweeps, parity)
        want = up[i - a + 1, j - c + 1]
        assert abs(got - want) <= TOL * float(np.max(np.abs(up))), (i, j, got, want)
