"""GPU parity for the temporally blocked (TMA) sweeps and the mixed-precision refinement.

- RBGS_KERNEL_TEMPORAL: K sweeps per shared-memory pass must give the oracle's FP64
  iterate bit for bit (same operations in the same order), for every depth, grid sizes
  with ragged tiles, and sweep counts that leave a remainder.
- RBGS_FP32_REFINE: binary32 inner sweeps (one launch per colour, or temporal tiles)
  with binary64 defect and correction must reproduce the oracle's refinement bit for bit
  (every step is a fixed sequence of correctly rounded operations; the scale exponent
  comes from an exact max), and must reach an FP64-level residual.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2607_01735_gb300 as rb
import synth
from oracle import direct

pytestmark = pytest.mark.gpu


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


def _assert_bits(got, ref):
    if not np.array_equal(got.view(np.uint64), ref.view(np.uint64)):
        bad = np.argwhere(got.view(np.uint64) != ref.view(np.uint64))
        i, j = bad[0]
        raise AssertionError(f"{len(bad)} values differ; first at {(i, j)}: {got[i, j]!r} vs {ref[i, j]!r}")


@pytest.mark.parametrize("k", [1, 2, 4])
@pytest.mark.parametrize("n", [1, 2, 5, 31, 64, 65, 130, 257, 600])
def test_temporal_fp64_bit_exact(n, k):
    f, u0 = _problem(n, 40 + n + k)
    h2 = synth.h_squared(n)
    sweeps = 2 * k + 1  # full passes plus a remainder
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, kernel=rb.RBGS_KERNEL_TEMPORAL, tblock_k=k) as s:
        s.sweep(sweeps)
        s.sweep(k)  # another pass after the buffers have swapped
        s.get_solution(out)
        rho = s.residual()
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, sweeps + k)
    _assert_bits(out.cpu().numpy(), ref)
    rho_ref = oracle.residual(ref, f, h2)[0]
    assert abs(rho - rho_ref) <= 1e-12 * rho_ref


def test_temporal_fp64_solve_and_resume():
    n = 200
    f, u0 = _problem(n, 77, interior=False)
    h2 = synth.h_squared(n)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, kernel=rb.RBGS_KERNEL_TEMPORAL, tblock_k=4, check_every=30,
                   max_sweeps=300) as s:
        done, rho, st = s.solve(1e-30, allow_not_converged=True)
        s.get_solution(out)
    ref = u0.copy()
    oracle.sweeps(ref, f, h2, done)
    assert done == 300 and st == rb.RBGS_ENOTCONV
    _assert_bits(out.cpu().numpy(), ref)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 16, 17, 64, 160, 161])
def test_refinement_small_grids_bit_exact(n):
    """Small grids run the FP32 inner sweeps in one launch of one thread-block cluster (up to
    160^2; most blocks hold one row or none at the smallest sizes), 161^2 the cached graphs."""
    f, u0 = _problem(n, 700 + n, interior=False)
    h2 = synth.h_squared(n)
    inner, max_sweeps = 17, 17 * 2 + 3
    ref = u0.copy()
    done_ref, rho_ref, outer = oracle.refine_solve(ref, f, h2, 1e-30, inner, max_sweeps)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, precision=rb.RBGS_FP32_REFINE, inner_sweeps=inner,
                   max_sweeps=max_sweeps) as s:
        done, rho, st = s.solve(1e-30, allow_not_converged=True)
        s.get_solution(out)
    # (the tiniest grids may reach rho = 0 before max_sweeps; the oracle then stops too)
    assert done == done_ref
    _assert_bits(out.cpu().numpy(), ref)
    assert abs(rho - rho_ref) <= 1e-12 * max(rho_ref, 1e-300) or rho == rho_ref


@pytest.mark.parametrize("kernel,k", [(rb.RBGS_KERNEL_COLOUR, 0), (rb.RBGS_KERNEL_TEMPORAL, 2),
                                      (rb.RBGS_KERNEL_TEMPORAL, 4), (rb.RBGS_KERNEL_TEMPORAL, 8)])
@pytest.mark.parametrize("n", [33, 150, 520])
def test_refinement_bit_exact_against_oracle(n, kernel, k):
    f, u0 = _problem(n, 500 + n, interior=False)
    h2 = synth.h_squared(n)
    inner, max_sweeps = 23, 23 * 3 + 5  # the last outer step is shortened
    ref = u0.copy()
    done_ref, rho_ref, outer = oracle.refine_solve(ref, f, h2, 1e-30, inner, max_sweeps)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, precision=rb.RBGS_FP32_REFINE, kernel=kernel, tblock_k=k,
                   inner_sweeps=inner, max_sweeps=max_sweeps) as s:
        done, rho, st = s.solve(1e-30, allow_not_converged=True)
        s.get_solution(out)
    assert st == rb.RBGS_ENOTCONV and done == done_ref == max_sweeps and outer == 4
    _assert_bits(out.cpu().numpy(), ref)
    assert abs(rho - rho_ref) <= 1e-12 * rho_ref


def test_refinement_reaches_fp64_residual_and_direct_solution():
    """GRF right-hand side, ring g = x^2 - y^2 (the mixed-precision workload at a size the
    oracle and the GPU finish quickly): tol 1e-10 reached, error vs the DST solution at FP64
    level, and the sweep count equals the oracle's."""
    n = 127
    f, _ = synth.grf_rhs(n, 2)
    u0 = synth.ring_grid(n, synth.g_quadratic)
    h2 = synth.h_squared(n)
    ref = u0.copy()
    done_ref, rho_ref, _ = oracle.refine_solve(ref, f, h2, 1e-10, 200, 10 ** 6)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, h2, fd, ud, precision=rb.RBGS_FP32_REFINE, inner_sweeps=200) as s:
        done, rho, st = s.solve(1e-10)
        s.get_solution(out)
    assert st == rb.RBGS_OK and rho <= 1e-10
    assert done == done_ref
    got = out.cpu().numpy()
    _assert_bits(got, ref)
    exact = direct.dst_solve(f, u0, h2)
    # relative error <= cond(A) * rho; binary32 sweeps alone would stall near 1e-4 here
    assert np.max(np.abs(got - exact)) / np.max(np.abs(exact)) <= 1e-6
