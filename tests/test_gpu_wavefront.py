"""GPU parity for the register-wavefront temporal kernel (RBGS_KERNEL_WAVEFRONT).

A pass performs K sweeps (2K half-sweeps of Eq. (1)) in one march down each strip, with
the iterate in registers, overlapping strips and row segments recomputed.  Every update
is the same correctly rounded sequence as the oracle's, so the iterate must match the
oracle bit for bit: FP64 sweeps for K = 2, 4, FP32 inner sweeps of the refinement for
K = 2, 4, 6.  Sizes cover one and many strips, one and many row segments, ragged edges,
and sweep counts that leave a remainder (run by the one-launch-per-colour kernel).
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2607_01735_gb300 as rb
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_01735_gb300 import build
    build.build_library()
    rb.load_library()


def _problem(n, stream, interior=True):
    f = synth.uniform_pm1_grid(n, stream).numpy().copy()
    u = np.zeros((n + 2, n + 2))
    r = synth.uniform01(stream + 7000, (n + 2) * (n + 2)).numpy().reshape(n + 2, n + 2) * 2 - 1
    u[0, :], u[-1, :], u[:, 0], u[:, -1] = r[0, :], r[-1, :], r[:, 0], r[:, -1]
    if interior:
        u[1:-1, 1:-1] = synth.uniform_pm1_grid(n, stream + 9000).numpy() * 0.5
    return f, u


def _assert_bits(got, ref):
    if not np.array_equal(got.view(np.uint64), ref.view(np.uint64)):
        bad = np.argwhere(got.view(np.uint64) != ref.view(np.uint64))
        i, j = bad[0]
        raise AssertionError(f"{len(bad)} values differ; first at {(i, j)}: {got[i, j]!r} vs {ref[i, j]!r}")


@pytest.mark.parametrize("k", [2, 4])
@pytest.mark.parametrize("n", [1, 2, 3, 5, 31, 64, 65, 119, 120, 121, 130, 257, 600, 1500])
def test_wavefront_fp64_bit_exact(n, k):
    f, u0 = _problem(n, 60 + n + k)
    h2 = synth.h_squared(n)
    sweeps = 2 * k + 1  # two passes and a remainder
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, kernel=rb.RBGS_KERNEL_WAVEFRONT, tblock_k=k) as s:
        s.sweep(sweeps)
        s.sweep(k)  # one more pass after the buffers have swapped
        s.get_solution(out)
        rho = s.residual()
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, sweeps + k)
    _assert_bits(out.cpu().numpy(), ref)
    rho_ref = oracle.residual(ref, f, h2)[0]
    # the norm sums n^2 squares: the oracle's sequential sum carries a relative error of up
    # to about n^2 u (u = 2^-53), the GPU's tree sum far less
    assert abs(rho - rho_ref) <= max(1e-12, n * n * 2.0 ** -53) * rho_ref


def test_wavefront_fp64_large_grid_bit_exact():
    """4097^2: many strips and segments in one launch, at a size where every block count
    and the segment height take their large-grid values."""
    n, k = 4097, 4
    f, u0 = _problem(n, 4242)
    h2 = synth.h_squared(n)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, kernel=rb.RBGS_KERNEL_WAVEFRONT, tblock_k=k) as s:
        s.sweep(2 * k)
        s.get_solution(out)
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, 2 * k)
    _assert_bits(out.cpu().numpy(), ref)


def test_wavefront_fp64_set_solution_and_solve():
    n = 300
    f, u0 = _problem(n, 91, interior=False)
    h2 = synth.h_squared(n)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    _, u1 = _problem(n, 92)
    with rb.Solver(n, h2, fd, ud, kernel=rb.RBGS_KERNEL_WAVEFRONT, tblock_k=2, check_every=7,
                   max_sweeps=50) as s:
        s.sweep(4)
        s.set_solution(torch.from_numpy(u1).cuda())  # replaces the iterate after a swap
        done, rho, st = s.solve(1e-30, allow_not_converged=True)
        s.get_solution(out)
    ref = u1.copy()
    oracle.sweeps(ref, f, h2, done)
    assert done == 50 and st == rb.RBGS_ENOTCONV
    _assert_bits(out.cpu().numpy(), ref)


@pytest.mark.parametrize("k", [2, 4, 6])
@pytest.mark.parametrize("n", [33, 150, 520, 1100])
def test_wavefront_refinement_bit_exact_against_oracle(n, k):
    f, u0 = _problem(n, 700 + n, interior=False)
    h2 = synth.h_squared(n)
    inner, max_sweeps = 23, 23 * 3 + 5  # inner counts that leave remainders
    ref = u0.copy()
    done_ref, rho_ref, outer = oracle.refine_solve(ref, f, h2, 1e-30, inner, max_sweeps)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, precision=rb.RBGS_FP32_REFINE, kernel=rb.RBGS_KERNEL_WAVEFRONT,
                   tblock_k=k, inner_sweeps=inner, max_sweeps=max_sweeps) as s:
        done, rho, st = s.solve(1e-30, allow_not_converged=True)
        s.get_solution(out)
    assert st == rb.RBGS_ENOTCONV and done == done_ref == max_sweeps and outer == 4
    _assert_bits(out.cpu().numpy(), ref)
    assert abs(rho - rho_ref) <= 1e-12 * rho_ref


def test_wavefront_refinement_reaches_tolerance_like_oracle():
    n = 127
    f, _ = synth.grf_rhs(n, 2)
    u0 = synth.ring_grid(n, synth.g_quadratic)
    h2 = synth.h_squared(n)
    ref = u0.copy()
    done_ref, rho_ref, _ = oracle.refine_solve(ref, f, h2, 1e-10, 200, 10 ** 6)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, precision=rb.RBGS_FP32_REFINE, kernel=rb.RBGS_KERNEL_WAVEFRONT,
                   tblock_k=4, inner_sweeps=200) as s:
        done, rho, st = s.solve(1e-10)
        s.get_solution(out)
    assert st == rb.RBGS_OK and done == done_ref
    _assert_bits(out.cpu().numpy(), ref)


def test_full_size_kernels_agree_bitwise():
    """16384^2 (the benchmark grid): the wavefront and one launch per colour give the same
    bits, for FP64 sweeps and for the refinement's FP32 inner sweeps.  Both are pinned to
    the oracle at smaller sizes; equality is what carries that pin to the full size."""
    n = 16384
    h2 = synth.h_squared(n)
    f = synth.uniform_pm1_grid(n, 1, device="cuda")
    u0 = torch.zeros(n + 2, n + 2, dtype=torch.float64, device="cuda")
    outs = []
    for kernel, k in ((rb.RBGS_KERNEL_COLOUR, 0), (rb.RBGS_KERNEL_WAVEFRONT, 2)):
        out = torch.empty_like(u0)
        with rb.Solver(n, h2, f, u0, kernel=kernel, tblock_k=k) as s:
            s.sweep(5)
            s.get_solution(out)
        outs.append(out)
    assert torch.equal(outs[0].view(torch.int64), outs[1].view(torch.int64))
    del outs
    outs = []
    for kernel, k in ((rb.RBGS_KERNEL_COLOUR, 0), (rb.RBGS_KERNEL_WAVEFRONT, 4)):
        out = torch.empty_like(u0)
        with rb.Solver(n, h2, f, u0, precision=rb.RBGS_FP32_REFINE, kernel=kernel, tblock_k=k,
                       inner_sweeps=10, max_sweeps=20) as s:
            done, rho, st = s.solve(1e-30, allow_not_converged=True)
            s.get_solution(out)
        assert done == 20
        outs.append(out)
    assert torch.equal(outs[0].view(torch.int64), outs[1].view(torch.int64))
