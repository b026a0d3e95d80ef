"""GPU parity: the CUDA path through the C ABI against the oracle.

The FP64 iterate must be bit-identical to the oracle after the same number of sweeps
(every update is the same sequence of correctly rounded operations); the residual
norm, whose summation order differs, must agree to 1e-12 relative.  Sizes span several
blocks and ragged row/strip tails; every FP64 add split (hardware, integer pipe, mixed)
and several strip heights are covered.  The full 16384^2 grid is checked on sampled
points, each recomputed by the oracle on its dependency window.
"""
import math
import os

import numpy as np
import pytest
import torch

import oracle
import paper_2607_01735_gb300 as rb
import synth

pytestmark = pytest.mark.gpu

RESID_RTOL = 1e-12
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_01735_gb300 import build
    build.build_library()
    rb.load_library()


def _problem(n, stream, ring=True, interior=True):
    f = synth.uniform_pm1_grid(n, stream).numpy().copy()
    u = np.zeros((n + 2, n + 2))
    if ring:
        r = synth.uniform01(stream + 7000, (n + 2) * (n + 2)).numpy().reshape(n + 2, n + 2) * 2 - 1
        u[0, :], u[-1, :], u[:, 0], u[:, -1] = r[0, :], r[-1, :], r[:, 0], r[:, -1]
    if interior:
        u[1:-1, 1:-1] = synth.uniform_pm1_grid(n, stream + 9000).numpy() * 0.5
    return f, u


def _run_gpu(n, h2, f, u0, sweeps, **opts):
    fd = torch.from_numpy(f).cuda()
    ud = torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, **opts) as s:
        s.sweep(sweeps)
        s.get_solution(out)
        rho = s.residual()
    return out.cpu().numpy(), rho


def _assert_bits(got, ref):
    if not np.array_equal(got.view(np.uint64), ref.view(np.uint64)):
        bad = np.argwhere(got.view(np.uint64) != ref.view(np.uint64))
        i, j = bad[0]
        raise AssertionError(f"{len(bad)} values differ; first at {(i, j)}: {got[i, j]!r} vs {ref[i, j]!r}")


SIZES = [1, 2, 3, 4, 5, 6, 7, 8, 9, 16, 31, 32, 33, 63, 64, 127, 255, 256, 257, 300, 509, 1000, 1030]


@pytest.mark.parametrize("values,step_rows,int_rows", [(2, 1, 0), (4, 1, 0), (2, 2, 0), (2, 1, 8)])
@pytest.mark.parametrize("n", SIZES)
def test_bit_exact_against_oracle(n, values, step_rows, int_rows):
    f, u0 = _problem(n, 11 + n)
    h2 = synth.h_squared(n)
    sweeps = 7 if n > 300 else 13
    got, rho = _run_gpu(n, h2, f, u0, sweeps, sweep_values=values, sweep_rows=step_rows, int_rows=int_rows)
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, sweeps)
    _assert_bits(got, ref)
    rho_ref = oracle.residual(ref, f, h2)[0]
    assert abs(rho - rho_ref) <= RESID_RTOL * rho_ref


@pytest.mark.parametrize("kernel", [rb.RBGS_KERNEL_COLOUR, rb.RBGS_KERNEL_PERSISTENT])
@pytest.mark.parametrize("n", SIZES)
def test_explicit_kernel_bit_exact(n, kernel):
    """One launch per colour and the cooperative launch on every size, whichever AUTO would
    pick there (it picks the cooperative launch from 416^2)."""
    f, u0 = _problem(n, 17 + n)
    h2 = synth.h_squared(n)
    sweeps = 7 if n > 300 else 13
    got, rho = _run_gpu(n, h2, f, u0, sweeps, kernel=kernel)
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, sweeps)
    _assert_bits(got, ref)
    rho_ref = oracle.residual(ref, f, h2)[0]
    assert abs(rho - rho_ref) <= RESID_RTOL * rho_ref


def test_cooperative_launch_in_solve_chunks():
    """rbgs_solve through the cooperative launch: one launch per check interval, the same
    sweep count and iterate as the oracle's solve."""
    n = 600
    f, u0 = _problem(n, 91, interior=False)
    h2 = synth.h_squared(n)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, kernel=rb.RBGS_KERNEL_PERSISTENT, check_every=37, max_sweeps=400) as s:
        done, rho, _ = s.solve(1e-30, allow_not_converged=True)
        s.get_solution(out)
    ref = u0.copy()
    ref_done, ref_rho = oracle.solve(ref, f, h2, 1e-30, 37, 400)
    assert done == ref_done == 400
    _assert_bits(out.cpu().numpy(), ref)
    assert abs(rho - ref_rho) <= RESID_RTOL * ref_rho


@pytest.mark.parametrize("values", [2, 4])
@pytest.mark.parametrize("emulate", [-2, 0x00, 0x08, 0x88, 0x8C, 0xCC, 0xFF])
@pytest.mark.parametrize("n", [33, 257])
def test_every_fp64_add_split_is_bit_exact(n, emulate, values):
    f, u0 = _problem(n, 100 + n)
    h2 = synth.h_squared(n)
    got, _ = _run_gpu(n, h2, f, u0, 9, fp64_emulate=emulate, sweep_values=values)
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, 9)
    _assert_bits(got, ref)


@pytest.mark.parametrize("int_rows", [0, 3])
@pytest.mark.parametrize("values,step_rows", [(2, 1), (4, 1), (2, 2), (4, 2)])
@pytest.mark.parametrize("rows", [1, 2, 7, 32, 64, 200])
def test_strip_heights(rows, values, step_rows, int_rows):
    n = 203
    f, u0 = _problem(n, 300 + rows)
    h2 = synth.h_squared(n)
    got, _ = _run_gpu(n, h2, f, u0, 5, tile_rows=rows, sweep_values=values, sweep_rows=step_rows,
                      int_rows=int_rows)
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, 5)
    _assert_bits(got, ref)


def test_zero_sweeps_and_ring_untouched():
    n = 40
    f, u0 = _problem(n, 5)
    got, _ = _run_gpu(n, synth.h_squared(n), f, u0, 0)
    _assert_bits(got, u0)
    got, _ = _run_gpu(n, synth.h_squared(n), f, u0, 3)
    _assert_bits(np.stack([got[0], got[-1]]), np.stack([u0[0], u0[-1]]))
    _assert_bits(np.stack([got[:, 0], got[:, -1]]), np.stack([u0[:, 0], u0[:, -1]]))


# ------------------------------------------------------------ 255^2, 1000 sweeps
def _golden_rho():
    rows = []
    with open(os.path.join(GOLDEN, "manufactured_rho_n255.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, r = line.split()
                rows.append((int(k), float(r)))
    return dict(rows)


@pytest.mark.parametrize("rhs", ["manufactured", "uniform"])
def test_plain_fp64_255_history(rhs):
    """-Lap u = f on 255^2 (h = 1/256), zero ring, u0 = 0, 1000 sweeps, rho every 100."""
    n = 255
    h2 = synth.h_squared(n)
    f = synth.manufactured_rhs(n) if rhs == "manufactured" else synth.uniform_pm1_grid(n, 0).numpy().copy()
    u0 = synth.ring_grid(n)
    ref = u0.copy()
    gold = _golden_rho()
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud) as s:
        done = 0
        for k in [1] + list(range(100, 1001, 100)):
            s.sweep(k - done)
            oracle.sweeps(ref, f, h2, k - done)
            done = k
            rho = s.residual()
            rho_ref = oracle.residual(ref, f, h2)[0]
            assert abs(rho - rho_ref) <= RESID_RTOL * rho_ref, (k, rho, rho_ref)
            if rhs == "manufactured":
                assert abs(rho - gold[k]) <= 1e-11 * gold[k]
        s.get_solution(out)
    _assert_bits(out.cpu().numpy(), ref)


# ------------------------------------------------------------ residual and solve
def test_residual_of_random_states():
    for n in (1, 2, 17, 128, 301):
        f, u = _problem(n, 900 + n)
        h2 = synth.h_squared(n)
        _, rho = _run_gpu(n, h2, f, u, 0)
        rho_ref = oracle.residual(u, f, h2)[0]
        assert abs(rho - rho_ref) <= RESID_RTOL * rho_ref


def test_residual_zero_rhs_is_absolute():
    n = 20
    f = np.zeros((n, n))
    u = np.zeros((n + 2, n + 2))
    u[1:-1, 1:-1] = 1.0
    _, rho = _run_gpu(n, synth.h_squared(n), f, u, 0)
    assert abs(rho - oracle.residual(u, f, synth.h_squared(n))[0]) <= 1e-12 * rho


@pytest.mark.parametrize("kernel", [rb.RBGS_KERNEL_COLOUR, rb.RBGS_KERNEL_PERSISTENT, rb.RBGS_KERNEL_TEMPORAL,
                                    rb.RBGS_KERNEL_WAVEFRONT])
@pytest.mark.parametrize("n", [1, 2, 5, 64, 257])
def test_residual_after_sweeps_walks_red_only_with_the_same_bits(kernel, n):
    """After a full sweep the library sums rt^2 over the red points only: the black rt is
    exactly zero there (the black values are s/4 of the very sums the residual forms).  The
    same iterate reloaded (so nothing is known of it) takes the walk over both colours; the
    two norms must agree bit for bit, and with the oracle's."""
    h2 = synth.h_squared(n)
    f, u0 = _problem(n, 85)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, kernel=kernel) as s:
        s.sweep(4)
        rho_red = s.residual()
        s.get_solution(out)
        s.set_solution(out)
        rho_full = s.residual()
        s.sweep(0)  # no sweep: the state stays unknown
        assert s.residual() == rho_full
    assert np.float64(rho_red).view(np.uint64) == np.float64(rho_full).view(np.uint64)
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, 4)
    _assert_bits(out.cpu().numpy(), ref)
    rho_ref = oracle.residual(ref, f, h2)[0]
    assert abs(rho_red - rho_ref) <= RESID_RTOL * rho_ref


def test_red_only_residual_with_subnormal_black_values():
    """A region of the grid where h^2 f and the iterate are subnormal: there the black
    values s * 0.25 are rounded, so the black rt is not exactly zero, but below 2^-1072, and
    its square adds nothing to the sum.  The red-only and two-colour norms agree bit for bit."""
    n = 64
    h2 = synth.h_squared(n)
    f = synth.uniform_pm1_grid(n, 86).numpy().copy()
    f[:, n // 2:] *= 1e-310   # right half: h^2 f and, after 3 sweeps, u on its far side subnormal
    u0 = np.zeros((n + 2, n + 2))
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, kernel=rb.RBGS_KERNEL_COLOUR) as s:
        s.sweep(3)
        rho_red = s.residual()
        s.get_solution(out)
        s.set_solution(out)
        rho_full = s.residual()
    got = out.cpu().numpy()
    tiny = got[1:-1, 1:-1][:, -16:]
    assert np.all(np.abs(tiny) < np.finfo(np.float64).tiny) and np.any(tiny != 0)
    # the premise: some black rt is not zero (s * 0.25 rounded), each far below 2^-1072
    s_ = h2 * f + got[:-2, 1:-1] + got[2:, 1:-1] + got[1:-1, :-2] + got[1:-1, 2:]
    rt = s_ - 4.0 * got[1:-1, 1:-1]
    i, j = np.indices((n, n)) + 1
    black = rt[(i + j) % 2 == 1]
    assert np.any(black != 0) and np.all(np.abs(black) < 2.0 ** -1072)
    assert np.float64(rho_red).view(np.uint64) == np.float64(rho_full).view(np.uint64)
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, 3)
    _assert_bits(got, ref)
    rho_ref = oracle.residual(ref, f, h2)[0]
    assert abs(rho_red - rho_ref) <= RESID_RTOL * rho_ref


def test_solve_matches_oracle_sweep_count():
    n = 63
    f, u0 = _problem(n, 77, interior=False)
    h2 = synth.h_squared(n)
    ref = u0.copy()
    done_ref, rho_ref = oracle.solve(ref, f, h2, 1e-8, 50, 10 ** 7)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, check_every=50) as s:
        done, rho, st = s.solve(1e-8)
        s.get_solution(out)
    assert st == rb.RBGS_OK and done == done_ref
    assert abs(rho - rho_ref) <= RESID_RTOL * rho_ref
    _assert_bits(out.cpu().numpy(), ref)


def test_solve_not_converged_keeps_state():
    n = 31
    f, u0 = _problem(n, 78)
    h2 = synth.h_squared(n)
    with rb.Solver(n, h2, torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda(),
                   check_every=10, max_sweeps=30) as s:
        done, rho, st = s.solve(1e-14, allow_not_converged=True)
        assert st == rb.RBGS_ENOTCONV and done == 30
        out = torch.empty(n + 2, n + 2, dtype=torch.float64, device="cuda")
        s.get_solution(out)
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, 30)
    _assert_bits(out.cpu().numpy(), ref)


def test_nonfinite_rhs_reports_status():
    n = 16
    f, u0 = _problem(n, 79)
    f[3, 4] = np.nan
    with rb.Solver(n, synth.h_squared(n), torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()) as s:
        s.sweep(2)
        with pytest.raises(rb.RbgsError) as e:
            s.residual()
        assert e.value.status == rb.RBGS_ENONFINITE


def test_host_buffers_match_device_buffers():
    n = 97
    f, u0 = _problem(n, 80)
    h2 = synth.h_squared(n)
    out_host = np.empty_like(u0)
    with rb.Solver(n, h2, f, u0) as s:  # numpy (pageable host) inputs and output
        s.sweep(11)
        s.get_solution(out_host)
    pinned_f = torch.from_numpy(f).pin_memory()
    pinned_u = torch.from_numpy(u0).pin_memory()
    out_pinned = torch.empty((n + 2, n + 2), dtype=torch.float64).pin_memory()
    with rb.Solver(n, h2, pinned_f, pinned_u) as s:
        s.sweep(11)
        s.get_solution(out_pinned)
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, 11)
    _assert_bits(out_host, ref)
    _assert_bits(out_pinned.numpy(), ref)


def test_set_solution_resumes():
    n = 50
    f, u0 = _problem(n, 81)
    h2 = synth.h_squared(n)
    mid = torch.empty(n + 2, n + 2, dtype=torch.float64, device="cuda")
    out = torch.empty_like(mid)
    fd = torch.from_numpy(f).cuda()
    with rb.Solver(n, h2, fd, torch.from_numpy(u0).cuda()) as s:
        s.sweep(4)
        s.get_solution(mid)
    with rb.Solver(n, h2, fd, torch.zeros_like(mid)) as s:
        s.set_solution(mid)
        s.sweep(6)
        s.get_solution(out)
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, 10)
    _assert_bits(out.cpu().numpy(), ref)


@pytest.mark.parametrize("kernel,precision", [(rb.RBGS_KERNEL_COLOUR, rb.RBGS_FP64),
                                              (rb.RBGS_KERNEL_WAVEFRONT, rb.RBGS_FP64),
                                              (rb.RBGS_KERNEL_TEMPORAL, rb.RBGS_FP64),
                                              (rb.RBGS_KERNEL_AUTO, rb.RBGS_FP32_REFINE)])
@pytest.mark.parametrize("host", [False, True])
def test_set_problem_reuses_the_context(kernel, precision, host):
    """A context reloaded with a second problem (host or device inputs) gives the oracle's
    iterate for that problem, as a freshly created one does; the first problem leaves no
    trace (graphs, partner buffers and the right-hand side norm are refreshed)."""
    n = 70
    h2 = synth.h_squared(n)
    fa, ua = _problem(n, 83)
    fb, ub = _problem(n, 84)
    conv = (lambda a: a) if host else (lambda a: torch.from_numpy(a).cuda())
    out = np.empty((n + 2, n + 2)) if host else torch.empty(n + 2, n + 2, dtype=torch.float64, device="cuda")
    refine = precision == rb.RBGS_FP32_REFINE
    with rb.Solver(n, h2, conv(fa), conv(ua), kernel=kernel, precision=precision, inner_sweeps=10,
                   max_sweeps=40, check_every=10) as s:
        for f, u0 in ((fa, ua), (fb, ub)):
            s.set_problem(conv(f), conv(u0))
            if refine:
                _, rho, _ = s.solve(0.0, allow_not_converged=True)
            else:
                s.sweep(40)
                rho = s.residual()
            s.get_solution(out)
            got = out if host else out.cpu().numpy()
            ref = u0.copy()
            if refine:
                _, ref_rho, _ = oracle.refine_solve(ref, f, h2, 0.0, 10, 40)
            else:
                oracle.sweeps(ref, f, h2, 40)
                ref_rho = oracle.residual(ref, f, h2)[0]
            _assert_bits(np.asarray(got), ref)
            assert abs(rho - ref_rho) <= RESID_RTOL * ref_rho


def test_graph_and_direct_launches_agree():
    # 70 sweeps = two cached 32-sweep graphs + 6 direct sweeps
    n = 130
    f, u0 = _problem(n, 82)
    h2 = synth.h_squared(n)
    got, _ = _run_gpu(n, h2, f, u0, 70)
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, 70)
    _assert_bits(got, ref)


def test_input_generator_same_bits_on_gpu():
    a = synth.uniform01(1, 100000, start=123456789, device="cuda").cpu()
    b = synth.uniform01(1, 100000, start=123456789, device="cpu")
    assert torch.equal(a, b)


# ------------------------------------------------------------ full-size grid, sampled
def _window_inputs(n, stream, i, j, r):
    """f on rows a..b, cols c..d around (i, j) drawn from the same counter stream."""
    a, b = max(1, i - r), min(n, i + r)
    c, d = max(1, j - r), min(n, j + r)
    rows = [synth.uniform01(stream, d - c + 1, (ii - 1) * n + (c - 1)).numpy() * 2 - 1 for ii in range(a, b + 1)]
    return a, c, np.ascontiguousarray(np.stack(rows))


@pytest.mark.slow
def test_full_size_16384_sampled():
    """16384^2, f ~ U(-1,1) stream 1, zero ring, u0 = 0, 200 sweeps (the benchmark's
    launch configuration); sampled points recomputed by the oracle on their windows, the
    residual of the GPU's final iterate recomputed by the oracle."""
    n, sweeps, stream = 16384, 200, 1
    h2 = synth.h_squared(n)
    fd = synth.uniform_pm1_grid(n, stream, device="cuda")
    ud = torch.zeros(n + 2, n + 2, dtype=torch.float64, device="cuda")
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud) as s:
        s.sweep(sweeps)
        s.get_solution(out)
        rho = s.residual()
    del ud
    r = 2 * sweeps + 1
    samples = [(1, 1), (1, n), (n, 1), (n, n), (n // 2, n // 2 + 1), (777, 12345), (16000, 3)]
    for (i, j) in samples:
        a, c, fw = _window_inputs(n, stream, i, j, r)
        uw = np.zeros((fw.shape[0] + 2, fw.shape[1] + 2))
        parity = (a - 1 + c - 1) & 1
        oracle.sweeps(uw, fw, h2, sweeps, parity)
        want = uw[i - a + 1, j - c + 1]
        got = float(out[i, j].item())
        assert got == want, (i, j, got, want)
    host = out.cpu().numpy()
    f_host = fd.cpu().numpy()
    rho_ref = oracle.residual(host, f_host, h2)[0]
    assert abs(rho - rho_ref) <= RESID_RTOL * rho_ref


@pytest.mark.slow
@pytest.mark.parametrize("n", [32768, 32769])
def test_largest_cooperative_size_and_the_one_past_it(n):
    """AUTO runs the cooperative launch up to n = 32768, where its flattened item index
    reaches 32768 * 16385 items, and one launch per colour from 32769 on.  Both sizes are
    checked on sampled points (oracle windows, corners and the last rows included) and on
    the residual of the final iterate."""
    sweeps, stream = 3, 5
    h2 = synth.h_squared(n)
    fd = synth.uniform_pm1_grid(n, stream, device="cuda")
    ud = torch.zeros(n + 2, n + 2, dtype=torch.float64, device="cuda")
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud) as s:
        s.sweep(sweeps)
        s.get_solution(out)
        rho = s.residual()
    del ud
    r = 2 * sweeps + 1
    samples = [(1, 1), (1, n), (n, 1), (n, n), (n - 1, n - 2), (n // 2, n // 2 + 1), (32000, 30001), (2, n - 1)]
    for (i, j) in samples:
        a, c, fw = _window_inputs(n, stream, i, j, r)
        uw = np.zeros((fw.shape[0] + 2, fw.shape[1] + 2))
        oracle.sweeps(uw, fw, h2, sweeps, (a - 1 + c - 1) & 1)
        assert float(out[i, j].item()) == uw[i - a + 1, j - c + 1], (i, j)
    host = out.cpu().numpy()
    del out
    f_host = fd.cpu().numpy()
    del fd
    rho_ref = oracle.residual(host, f_host, h2)[0]
    assert abs(rho - rho_ref) <= RESID_RTOL * rho_ref
