"""Pins for the oracle's fused update (oracle.sweeps_fused, the library's fma = 1 mode):
facts fixed by the mathematics, independent of the oracle's own code (CPU only).

The fused update evaluates Eq. (1) with one rounding: the five terms are put on a
fixed-point grid of step 2^-e (truncation), summed exactly, divided by 4 and rounded once
to binary64.  So
- after k sweeps it stays within a rigorous rounding bound of RBGS in exact rational
  arithmetic (each update errs by at most half an ulp of its result plus 5/4 of a grid
  step, and Gauss-Seidel passes earlier errors on without growth in the max-norm);
- where the exact quotient is a binary64 number the update returns it exactly, which the
  four-rounding form need not (a hand case below);
- exact data stay exact: quadratic and constant Dirichlet data, the N = 1 and N = 2 hand
  cases;
- the manufactured problem follows its closed-form residual history;
- it agrees with the bit-exact oracle to the tolerance set for this mode (1e-13 relative
  max-norm after the same sweeps) and a NaN poisons the block.
"""
import math

import numpy as np
import pytest

import oracle
import synth
from oracle import direct

from test_oracle_pins import _golden_rho, _random_problem, _relmax

EPS = np.finfo(np.float64).eps


def _scale(u, f, h2, m):
    """The block scale e of the fused update (for the error bound only)."""
    B = float(np.max(np.abs(u)))
    Q = float(np.max(np.abs(h2 * f))) if f.size else 0.0
    S = 4.0 * B + (2 * m + 1) * Q
    return 0 if S == 0 else min(61 - math.frexp(S)[1], 1020)


@pytest.mark.parametrize("n", [2, 3, 4, 6])
def test_within_rounding_bound_of_exact_rational_rbgs(n):
    f, u = _random_problem(n, 700 + n)
    h2 = synth.h_squared(n)
    sweeps = 4
    exact = np.array([[float(v) for v in row] for row in direct.exact_rbgs(f.tolist(), u.tolist(), h2, sweeps)])
    e = _scale(u, f, h2, sweeps)
    got = u.copy()
    oracle.sweeps_fused(got, f, h2, sweeps)
    vmax = np.max(np.abs(exact))
    # per update: half an ulp of a value <= vmax (<= eps/2 * vmax... times 2 for the ulp's
    # binade) plus 5 truncations of at most 2^-e each, divided by 4; 2 updates per sweep
    per_update = EPS * vmax + 1.25 * 2.0 ** -e
    bound = 2 * sweeps * per_update + EPS * vmax  # plus the final conversion of `exact`
    assert np.max(np.abs(got - exact)) <= bound
    # and tighter than the bit-exact iteration's bound (four roundings per update)
    plain = u.copy()
    oracle.sweeps(plain, f, h2, sweeps)
    assert np.max(np.abs(got - exact)) <= max(np.max(np.abs(plain - exact)), EPS * vmax) * 4


def test_single_rounding_by_hand():
    # N = 1, h2 f = 0, ring N, S, W, E = 1, 2^-53, 2^-53, 0.  Exact: (1 + 2^-52) / 4, a
    # binary64 number.  Four roundings: 1 + 2^-53 ties to 1, then + 2^-53 again to 1,
    # so 0.25; one rounding keeps the exact value.
    u = np.zeros((3, 3))
    u[0, 1], u[2, 1], u[1, 0] = 1.0, 2.0 ** -53, 2.0 ** -53
    f = np.zeros((1, 1))
    plain, fused = u.copy(), u.copy()
    oracle.sweeps(plain, f, 0.25, 1)
    oracle.sweeps_fused(fused, f, 0.25, 1)
    assert plain[1, 1] == 0.25
    assert fused[1, 1] == (1.0 + 2.0 ** -52) / 4


def test_n1_hand_case_and_first_sweep_of_n2():
    # (3/4 + 1 + 2 + 3 + 4) / 4 = 43/16, every step exact
    u = np.zeros((3, 3))
    u[0, 1], u[2, 1], u[1, 0], u[1, 2] = 1.0, 2.0, 3.0, 4.0
    oracle.sweeps_fused(u, np.array([[3.0]]), 0.25, 3)
    assert u[1, 1] == 2.6875
    u = np.zeros((4, 4))
    u[0, 1], u[0, 2], u[3, 1], u[3, 2] = 8.0, 4.0, 2.0, 1.0
    u[1, 0], u[2, 0], u[1, 3], u[2, 3] = 16.0, 32.0, 64.0, 128.0
    oracle.sweeps_fused(u, np.zeros((2, 2)), 1.0 / 9.0, 1)
    assert (u[1, 1], u[2, 2], u[1, 2], u[2, 1]) == (6.0, 32.25, 26.5625, 18.0625)


def test_quadratic_and_constant_boundaries_are_reproduced_exactly():
    n = 15
    h2 = synth.h_squared(n)
    u = synth.ring_grid(n, synth.g_quadratic)
    x, y, _ = synth.grid_coords(n)
    oracle.sweeps_fused(u, np.zeros((n, n)), h2, 2000)
    assert np.max(np.abs(u - synth.g_quadratic(x, y))) <= 1e-12
    n = 9
    u = synth.ring_grid(n, lambda x, y: 0.75 + 0 * x)
    u[1:-1, 1:-1] = 0.75
    oracle.sweeps_fused(u, np.zeros((n, n)), synth.h_squared(n), 7)
    assert np.all(u == 0.75)


def test_manufactured_residual_history_matches_closed_form():
    n = 255
    h2 = synth.h_squared(n)
    f = synth.manufactured_rhs(n)
    u = synth.ring_grid(n)
    done = 0
    for k, rho_expected in _golden_rho():
        oracle.sweeps_fused(u, f, h2, k - done)
        done = k
        rho = oracle.residual(u, f, h2)[0]
        assert abs(rho - rho_expected) <= 1e-11 * rho_expected, (k, rho, rho_expected)


@pytest.mark.parametrize("n,sweeps", [(63, 200), (100, 200), (255, 200), (31, 1500)])
def test_agrees_with_bit_exact_iteration_to_1e_13(n, sweeps):
    f, u = _random_problem(n, 800 + n)
    h2 = synth.h_squared(n)
    a, b = u.copy(), u.copy()
    oracle.sweeps(a, f, h2, sweeps)
    oracle.sweeps_fused(b, f, h2, sweeps)
    assert _relmax(b, a) <= 1e-13
    assert np.all(b[0] == u[0]) and np.all(b[:, 0] == u[:, 0])  # the ring never moves


def test_nan_poisons_the_block():
    n = 12
    f, u = _random_problem(n, 5)
    f[3, 4] = np.nan
    oracle.sweeps_fused(u, f, synth.h_squared(n), 2)
    assert np.all(np.isnan(u[1:-1, 1:-1]))
    assert np.all(np.isfinite(u[0]))


def test_window_at_the_whole_grid_scale_matches_full_grid():
    n, sweeps = 40, 6
    f, u0 = _random_problem(n, 9)
    h2 = synth.h_squared(n)
    full = u0.copy()
    oracle.sweeps_fused(full, f, h2, sweeps)
    bound = (float(np.max(np.abs(u0))), float(np.max(np.abs(h2 * f))))
    for i, j in ((1, 1), (20, 21), (40, 3), (17, 40)):
        assert oracle.window_value(f, u0, h2, sweeps, i, j, fused_bound=bound) == full[i, j]
