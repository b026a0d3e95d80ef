"""Pins for the oracle: facts fixed by the paper's method and by the mathematics,
independent of the oracle's own code (CPU only).

- closed-form residual history and rate on the manufactured problem (Section 2, Eq. (1));
- Gauss-Seidel on the red-black-permuted matrix equals one RBGS sweep (colouring, Section 2);
- convergence to the dense / sine-transform direct solution;
- exactness for quadratic (harmonic) Dirichlet data;
- exact rational brute force on tiny grids and a hand-worked N = 1 case;
- invariants: zero black residual after a sweep, the window (dependency-cone) evaluation.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import oracle
import synth
from oracle import direct

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _random_problem(n, stream, nj=None, ring=True):
    nj = n if nj is None else nj
    f = synth.uniform_pm1_grid(n, stream, nj=nj).numpy().copy()
    u = np.zeros((n + 2, nj + 2))
    if ring:
        r = synth.uniform01(stream + 1000, (n + 2) * (nj + 2)).numpy().reshape(n + 2, nj + 2) * 2 - 1
        u[0, :], u[-1, :], u[:, 0], u[:, -1] = r[0, :], r[-1, :], r[:, 0], r[:, -1]
    return f, u


def _relmax(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300))


# ---------------------------------------------------------------- closed forms (P1, P2)
def _golden_rho():
    rows = []
    with open(os.path.join(GOLDEN, "manufactured_rho_n255.txt")) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, r = line.split()
                rows.append((int(k), float(r)))
    return rows


def test_manufactured_residual_history_matches_closed_form():
    n = 255
    h2 = synth.h_squared(n)
    assert h2 == 2.0 ** -16
    f = synth.manufactured_rhs(n)
    u = synth.ring_grid(n)
    done = 0
    for k, rho_expected in _golden_rho():
        oracle.sweeps(u, f, h2, k - done)
        done = k
        rho, _, _ = oracle.residual(u, f, h2)
        assert abs(rho - rho_expected) <= 1e-11 * rho_expected, (k, rho, rho_expected)


def test_manufactured_rate_is_cos2_pi_h():
    n = 63
    h = 1.0 / (n + 1)
    h2 = synth.h_squared(n)
    f = synth.manufactured_rhs(n)
    u = synth.ring_grid(n)
    mu2 = math.cos(math.pi * h) ** 2
    oracle.sweeps(u, f, h2, 1)
    prev = oracle.residual(u, f, h2)[0]
    for _ in range(20):
        oracle.sweeps(u, f, h2, 5)
        rho = oracle.residual(u, f, h2)[0]
        assert abs(rho / prev - mu2 ** 5) <= 1e-10
        prev = rho


def test_manufactured_black_residual_vanishes_and_red_is_eigenvector():
    n = 31
    h2 = synth.h_squared(n)
    f = synth.manufactured_rhs(n)
    u = synth.ring_grid(n)
    oracle.sweeps(u, f, h2, 3)
    r = oracle.residual_field(u, f, h2)
    i, j = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    black = (i + j) % 2 == 1
    assert np.all(r[black] == 0.0)
    x, y, _ = synth.grid_coords(n)
    phi = (np.sin(math.pi * x) * np.sin(math.pi * y))[1:-1, 1:-1]
    ratio = r[~black] / phi[~black]
    assert np.ptp(ratio) <= 1e-9 * np.max(np.abs(ratio))


def test_discrete_solution_of_manufactured_problem():
    """c = (pi h/2)^2 / sin^2(pi h/2): the DST solve returns c phi; error vs sin sin is O(h^2)."""
    errs = []
    for n in (31, 63, 127):
        h = 1.0 / (n + 1)
        c = (math.pi * h / 2) ** 2 / math.sin(math.pi * h / 2) ** 2
        x, y, _ = synth.grid_coords(n)
        phi = np.sin(math.pi * x) * np.sin(math.pi * y)
        uh = direct.dst_solve(synth.manufactured_rhs(n), synth.ring_grid(n), synth.h_squared(n))
        assert _relmax(uh[1:-1, 1:-1], c * phi[1:-1, 1:-1]) <= 1e-12
        errs.append(np.max(np.abs(uh - phi)))
        assert abs(errs[-1] - (c - 1.0)) <= 1e-12
    # second order: halving h divides the error by ~4
    assert 3.9 < errs[0] / errs[1] < 4.1 and 3.9 < errs[1] / errs[2] < 4.1


# ---------------------------------------------------------------- permutation (P3)
@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8])
def test_red_black_is_gauss_seidel_in_permuted_order(n):
    f, u = _random_problem(n, 40 + n)
    interior = synth.uniform_pm1_grid(n, 80 + n).numpy()
    u[1:-1, 1:-1] = interior
    h2 = synth.h_squared(n)
    ref = u.copy()
    oracle.sweeps(ref, f, h2, 3)
    a = direct.dense_matrix(n, n)
    rhs = direct.scaled_rhs(f, u, h2).reshape(-1)
    x = direct.gauss_seidel_dense(a, rhs, interior.reshape(-1), direct.red_black_order(n, n), 3)
    assert _relmax(ref[1:-1, 1:-1].reshape(-1), x) <= 1e-14
    if n >= 3:
        lex = direct.gauss_seidel_dense(a, rhs, interior.reshape(-1), list(range(n * n)), 3)
        assert _relmax(lex, x) > 1e-6  # the ordering matters: natural order is a different method


def test_red_black_rectangular_and_parity_offset():
    ni, nj = 5, 7
    f, u = _random_problem(ni, 7, nj=nj)
    h2 = 0.01
    for parity in (0, 1):
        ref = u.copy()
        oracle.sweeps(ref, f, h2, 2, parity)
        a = direct.dense_matrix(ni, nj)
        rhs = direct.scaled_rhs(f, u, h2).reshape(-1)
        red = [(i - 1) * nj + (j - 1) for i in range(1, ni + 1) for j in range(1, nj + 1) if (i + j + parity) % 2 == 0]
        black = [(i - 1) * nj + (j - 1) for i in range(1, ni + 1) for j in range(1, nj + 1) if (i + j + parity) % 2 == 1]
        x = direct.gauss_seidel_dense(a, rhs, np.zeros(ni * nj), red + black, 2)
        assert _relmax(ref[1:-1, 1:-1].reshape(-1), x) <= 1e-14


# ---------------------------------------------------------------- direct solves (P4)
@pytest.mark.parametrize("n", [7, 16, 31])
def test_converges_to_dense_direct_solution(n):
    f, u = _random_problem(n, 100 + n)
    h2 = synth.h_squared(n)
    exact = direct.dense_solve(f, u, h2)
    mu2 = math.cos(math.pi / (n + 1)) ** 2
    sweeps = int(math.log(1e-16) / math.log(mu2)) + 50
    oracle.sweeps(u, f, h2, sweeps)
    assert _relmax(u, exact) <= 1e-12
    rho = oracle.residual(u, f, h2)[0]
    assert rho <= 1e-13


@pytest.mark.parametrize("n", [5, 16, 31])
def test_sine_transform_solve_matches_dense(n):
    f, u = _random_problem(n, 200 + n)
    h2 = synth.h_squared(n)
    assert _relmax(direct.dst_solve(f, u, h2), direct.dense_solve(f, u, h2)) <= 1e-12


def test_solve_stops_at_tolerance():
    n = 15
    f, u = _random_problem(n, 300)
    h2 = synth.h_squared(n)
    done, rho = oracle.solve(u, f, h2, 1e-8, 10, 100000)
    assert rho <= 1e-8 and done % 10 == 0 and done > 0
    u2 = _random_problem(n, 300)[1]
    oracle.sweeps(u2, f, h2, done - 10)
    assert oracle.residual(u2, f, h2)[0] > 1e-8  # not converged one check earlier


# ---------------------------------------------------------------- harmonic data (P5)
def test_quadratic_boundary_is_reproduced_exactly():
    n = 15
    h2 = synth.h_squared(n)
    u = synth.ring_grid(n, synth.g_quadratic)
    f = np.zeros((n, n))
    x, y, _ = synth.grid_coords(n)
    g = synth.g_quadratic(x, y)
    assert np.max(np.abs(direct.dst_solve(f, u, h2) - g)) <= 1e-14
    oracle.sweeps(u, f, h2, 2000)
    assert np.max(np.abs(u - g)) <= 1e-12


def test_constant_boundary_gives_constant_solution():
    n = 9
    u = synth.ring_grid(n, lambda x, y: 0.75 + 0 * x)
    f = np.zeros((n, n))
    u[1:-1, 1:-1] = 0.75  # 0.75 * k exact for k <= 4: every partial sum is exact
    oracle.sweeps(u, f, synth.h_squared(n), 7)
    assert np.all(u == 0.75)


# ---------------------------------------------------------------- tiny cases (P6)
def test_n1_hand_case():
    # h = 1/2, h^2 = 1/4, f = 3 -> h^2 f = 3/4; ring N, S, W, E = 1, 2, 3, 4:
    # u = (3/4 + 1 + 2 + 3 + 4) / 4 = 43/16 = 2.6875, exact in binary64; one sweep is exact.
    u = np.zeros((3, 3))
    u[0, 1], u[2, 1], u[1, 0], u[1, 2] = 1.0, 2.0, 3.0, 4.0
    f = np.array([[3.0]])
    oracle.sweeps(u, f, 0.25, 1)
    assert u[1, 1] == 2.6875
    oracle.sweeps(u, f, 0.25, 5)
    assert u[1, 1] == 2.6875


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_matches_exact_rational_brute_force(n):
    f, u = _random_problem(n, 500 + n)
    h2 = synth.h_squared(n)
    sweeps = 4
    exact = direct.exact_rbgs(f.tolist(), u.tolist(), h2, sweeps)
    ref = u.copy()
    oracle.sweeps(ref, f, h2, sweeps)
    ex = np.array([[float(v) for v in row] for row in exact])
    # each update rounds 6 times; errors are damped by the iteration
    assert np.max(np.abs(ref - ex)) <= 64 * np.finfo(np.float64).eps * np.max(np.abs(ex))


def test_n2_first_sweep_by_hand():
    # zero f, ring values chosen so every step is an exact binary fraction
    u = np.zeros((4, 4))
    u[0, 1], u[0, 2] = 8.0, 4.0      # north ring
    u[3, 1], u[3, 2] = 2.0, 1.0      # south ring
    u[1, 0], u[2, 0] = 16.0, 32.0    # west ring
    u[1, 3], u[2, 3] = 64.0, 128.0   # east ring
    f = np.zeros((2, 2))
    oracle.sweeps(u, f, 1.0 / 9.0, 1)
    # red (1,1): (8 + 0 + 16 + 0)/4 = 6 ; red (2,2): (0 + 1 + 0 + 128)/4 = 32.25
    # black (1,2): (4 + 32.25 + 6 + 64)/4 = 26.5625 ; black (2,1): (6 + 2 + 32 + 32.25)/4 = 18.0625
    assert u[1, 1] == 6.0 and u[2, 2] == 32.25
    assert u[1, 2] == 26.5625 and u[2, 1] == 18.0625


# ---------------------------------------------------------------- invariants (P7)
def test_black_residual_exactly_zero_after_full_sweep():
    n = 33
    f, u = _random_problem(n, 600)
    h2 = synth.h_squared(n)
    oracle.sweeps(u, f, h2, 2)
    r = oracle.residual_field(u, f, h2)
    i, j = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    assert np.all(r[(i + j) % 2 == 1] == 0.0)
    assert np.all(r[(i + j) % 2 == 0] != 0.0)


def test_red_points_alone_give_the_residual_sum_bit_for_bit():
    """After a full sweep the sum of rt^2 over the red points alone equals the oracle's sum
    over all points, bit for bit, also where the iterate is subnormal: there s * 0.25 is
    rounded, so a black rt need not be zero, but it stays below 2^-1072 and its square
    rounds to zero.  (The library's residual walks only the red points after a sweep.)"""
    n = 64
    h2 = synth.h_squared(n)
    f = synth.uniform_pm1_grid(n, 86).numpy().copy()
    f[:, n // 2:] *= 1e-310
    u = np.zeros((n + 2, n + 2))
    oracle.sweeps(u, f, h2, 3)
    r = oracle.residual_field(u, f, h2)
    i, j = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    black = r[(i + j) % 2 == 1]
    assert np.any(black != 0.0) and np.all(np.abs(black) < 2.0 ** -1072)
    _, r2_all, _ = oracle.residual(u, f, h2)
    acc = 0.0
    for ii in range(n):          # the oracle's i-major order, red points only
        for jj in range(n):
            if (ii + jj) % 2 == 0:
                acc = acc + float(r[ii, jj]) * float(r[ii, jj])
    assert acc == r2_all and acc > 0.0


def test_residual_of_zero_guess_is_one_and_of_exact_solution_tiny():
    n = 20
    f, _ = _random_problem(n, 700, ring=False)
    h2 = synth.h_squared(n)
    u = np.zeros((n + 2, n + 2))
    assert oracle.residual(u, f, h2)[0] == 1.0
    ex = direct.dense_solve(f, u, h2)
    assert oracle.residual(ex, f, h2)[0] <= 1e-14


def test_residual_definition_by_hand():
    # N = 1: rt = h2 f + N + S + W + E - 4u ; hb = h2 f + N + S + W + E
    u = np.array([[0.0, 1.0, 0.0], [3.0, 0.5, 4.0], [0.0, 2.0, 0.0]])
    f = np.array([[3.0]])
    rho, r2, b2 = oracle.residual(u, f, 0.25)
    assert r2 == (10.75 - 2.0) ** 2 and b2 == 10.75 ** 2
    assert rho == abs(10.75 - 2.0) / 10.75


def test_window_evaluation_matches_full_grid():
    n = 40
    f, u0 = _random_problem(n, 800)
    h2 = synth.h_squared(n)
    full = u0.copy()
    oracle.sweeps(full, f, h2, 3)
    for (i, j) in [(1, 1), (20, 21), (21, 21), (40, 40), (1, 40), (13, 2)]:
        assert oracle.window_value(f, u0, h2, 3, i, j) == full[i, j]


def test_float32_iteration_tracks_exact_arithmetic():
    n = 6
    f, u = _random_problem(n, 900)
    h2 = synth.h_squared(n)
    exact = direct.exact_rbgs(f.tolist(), u.tolist(), float(np.float32(h2)), 3)
    f32, u32 = f.astype(np.float32), u.astype(np.float32)
    # exact arithmetic on the float32-rounded inputs
    exact = direct.exact_rbgs(f32.astype(np.float64).tolist(), u32.astype(np.float64).tolist(),
                              float(np.float32(h2)), 3)
    oracle.sweeps_f32(u32, f32, h2, 3)
    ex = np.array([[float(v) for v in row] for row in exact])
    assert np.max(np.abs(u32 - ex)) <= 64 * np.finfo(np.float32).eps * np.max(np.abs(ex))
    assert np.max(np.abs(u32 - ex)) > 0  # really float32: not the float64 result


# ---------------------------------------------------------------- input generator
def test_splitmix64_published_vector():
    with open(os.path.join(GOLDEN, "splitmix64_seed0.txt")) as fh:
        vals = [int(l, 16) for l in fh if l.strip() and not l.startswith("#")]
    z = synth.splitmix64(0, len(vals))
    assert [int(v) & ((1 << 64) - 1) for v in z] == vals
    assert [synth.splitmix64_scalar(0, t) for t in range(len(vals))] == vals
    z = synth.splitmix64(5, 7, start=1 << 20)
    assert [int(v) & ((1 << 64) - 1) for v in z] == [synth.splitmix64_scalar(5, (1 << 20) + t) for t in range(7)]


def test_uniform_grid_properties():
    f = synth.uniform_pm1_grid(200, 1).numpy()
    assert f.min() >= -1.0 and f.max() < 1.0
    assert abs(f.mean()) < 0.01 and abs(f.var() - 1.0 / 3.0) < 0.01


# ---------------------------------------------------------------- mixed-precision refinement
def test_refinement_reaches_fp64_accuracy_with_fp32_sweeps():
    """FP32 sweeps alone stall near binary32 rounding; the FP64 defect/correction loop
    reaches the dense direct solution to FP64-level accuracy."""
    n = 31
    f, u0 = _random_problem(n, 1100)
    h2 = synth.h_squared(n)
    exact = direct.dense_solve(f, u0, h2)
    u = u0.copy()
    done, rho, outer = oracle.refine_solve(u, f, h2, 1e-13, 200, 10 ** 6)
    assert rho <= 1e-13 and outer >= 2
    assert _relmax(u, exact) <= 1e-12
    # plain binary32 RBGS with as many sweeps stalls at binary32 accuracy
    u32 = u0.astype(np.float32)
    oracle.sweeps_f32(u32, f.astype(np.float32), h2, done)
    err32 = _relmax(u32.astype(np.float64), exact)
    assert 1e-9 < err32 < 1e-4


def test_refinement_converges_like_plain_rbgs():
    """The defect equation is solved by the same iteration, so after the same number of
    sweeps the refined residual matches plain FP64 RBGS's up to binary32 noise."""
    n = 63
    f, u0 = _random_problem(n, 1200, ring=True)
    h2 = synth.h_squared(n)
    for total in (200, 600):
        u = u0.copy()
        oracle.refine_solve(u, f, h2, 0.0, 100, total)
        rho_ref, _, _ = oracle.residual(u, f, h2)
        p = u0.copy()
        oracle.sweeps(p, f, h2, total)
        rho_plain = oracle.residual(p, f, h2)[0]
        assert abs(rho_ref - rho_plain) <= 1e-5 * rho_plain


def test_refinement_first_step_by_definition():
    """One outer step with one inner sweep, recomputed from the definition in numpy."""
    n = 9
    f, u0 = _random_problem(n, 1300)
    h2 = synth.h_squared(n)
    u = u0.copy()
    oracle.refine_solve(u, f, h2, 0.0, 1, 1)
    rt = oracle.residual_field(u0, f, h2)
    mx = np.max(np.abs(rt))
    e = int(np.frexp(mx)[1])
    r32 = (rt * 2.0 ** -e).astype(np.float32)
    d = np.zeros((n + 2, n + 2), dtype=np.float32)
    oracle.sweeps_f32(d, r32, 1.0, 1)
    want = u0.copy()
    want[1:-1, 1:-1] = u0[1:-1, 1:-1] + d[1:-1, 1:-1].astype(np.float64) * 2.0 ** e
    assert np.array_equal(u, want)
