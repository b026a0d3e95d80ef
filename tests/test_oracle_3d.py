"""Pins for the oracle's 3D variant (oracle.sweeps3d, the 7-point red-black scheme the
paper's outlook names for 3D problems, Section 5): facts fixed by the mathematics,
independent of the oracle's own code (CPU only).

- the manufactured problem f = 3 pi^2 sin(pi x) sin(pi y) sin(pi z): its exact discrete
  solution is c phi with the same c as in 2D, and from u0 = 0 the iteration keeps its error
  in span{phi_red, phi_black}, with Jacobi factor mu = cos(pi h) per neighbour sum; so
  rho_k = 2 c mu^(2k-1) (1 - mu^2) ||phi_red|| / (pi^2 h^2 ||phi||) and the rate is mu^2;
- red-black ordering = Gauss-Seidel on the 7-point matrix in the red-then-black order;
- convergence to the dense direct solution; quadratic harmonic data reproduced;
  constant data constant; the N = 1 hand case.
"""
import math

import numpy as np
import pytest

import oracle
from oracle import direct


def _coords(n):
    h = 1.0 / (n + 1)
    x = np.arange(n + 2) * h
    return np.meshgrid(x, x, x, indexing="ij"), h


def _red(n):
    i, j, k = np.meshgrid(np.arange(n + 2), np.arange(n + 2), np.arange(n + 2), indexing="ij")
    return ((i + j + k) % 2 == 0)[1:-1, 1:-1, 1:-1]


def _manufactured(n):
    (x, y, z), h = _coords(n)
    phi = np.sin(np.pi * x) * np.sin(np.pi * y) * np.sin(np.pi * z)
    f = np.ascontiguousarray(3.0 * np.pi ** 2 * phi[1:-1, 1:-1, 1:-1])
    return f, phi[1:-1, 1:-1, 1:-1], h


def _closed_form_rho(n, k, phi_in, h):
    mu = math.cos(math.pi * h)
    c = (math.pi * h / 2) ** 2 / math.sin(math.pi * h / 2) ** 2
    red = _red(n)
    ratio = math.sqrt(float(np.sum(phi_in[red] ** 2)) / float(np.sum(phi_in ** 2)))
    return 2.0 * c * mu ** (2 * k - 1) * (1.0 - mu * mu) * ratio / (math.pi ** 2 * h * h)


@pytest.mark.parametrize("n", [7, 15])
def test_manufactured_history_and_rate(n):
    f, phi, h = _manufactured(n)
    h2 = h * h
    u = np.zeros((n + 2, n + 2, n + 2))
    done = 0
    for k in (1, 2, 5, 20, 60):
        oracle.sweeps3d(u, f, h2, k - done)
        done = k
        rho = oracle.residual3d(u, f, h2)[0]
        want = _closed_form_rho(n, k, phi, h)
        assert abs(rho - want) <= 1e-11 * want, (k, rho, want)
    # one more sweep multiplies rho by mu^2 = cos^2(pi h)
    oracle.sweeps3d(u, f, h2, 1)
    rho2 = oracle.residual3d(u, f, h2)[0]
    assert abs(rho2 / rho - math.cos(math.pi * h) ** 2) <= 1e-10


def _dense7(n):
    m = n ** 3
    a = np.zeros((m, m))
    idx = lambda i, j, k: (i * n + j) * n + k
    for i in range(n):
        for j in range(n):
            for k in range(n):
                p = idx(i, j, k)
                a[p, p] = 6.0
                for di, dj, dk in ((-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)):
                    ii, jj, kk = i + di, j + dj, k + dk
                    if 0 <= ii < n and 0 <= jj < n and 0 <= kk < n:
                        a[p, idx(ii, jj, kk)] = -1.0
    return a


def _rhs3(f, u, h2):
    """h^2 b: h^2 f plus the shell neighbours of each interior point."""
    n = f.shape[0]
    hb = h2 * f.copy()
    hb[0, :, :] += u[0, 1:-1, 1:-1]
    hb[-1, :, :] += u[-1, 1:-1, 1:-1]
    hb[:, 0, :] += u[1:-1, 0, 1:-1]
    hb[:, -1, :] += u[1:-1, -1, 1:-1]
    hb[:, :, 0] += u[1:-1, 1:-1, 0]
    hb[:, :, -1] += u[1:-1, 1:-1, -1]
    return hb.reshape(-1)


def _random3(n, seed):
    rng = np.random.default_rng(seed)
    f = rng.uniform(-1, 1, (n, n, n))
    u = np.zeros((n + 2, n + 2, n + 2))
    shell = rng.uniform(-1, 1, u.shape)
    u[0], u[-1], u[:, 0], u[:, -1], u[:, :, 0], u[:, :, -1] = (shell[0], shell[-1], shell[:, 0], shell[:, -1],
                                                             shell[:, :, 0], shell[:, :, -1])
    u[1:-1, 1:-1, 1:-1] = rng.uniform(-0.5, 0.5, (n, n, n))
    return f, u


@pytest.mark.parametrize("n", [1, 2, 3, 4])
def test_red_black_is_gauss_seidel_in_permuted_order(n):
    f, u = _random3(n, 10 + n)
    h2 = 1.0 / (n + 1) ** 2
    a = _dense7(n)
    rhs = _rhs3(f, u, h2)
    flat = np.arange(n ** 3)
    i, j, k = flat // (n * n), (flat // n) % n, flat % n
    parity = (i + j + k + 3) % 2  # interior indices are 1-based: colour of (i+1, j+1, k+1)
    order = [p for p in flat if parity[p] == 0] + [p for p in flat if parity[p] == 1]
    x = direct.gauss_seidel_dense(a, rhs, u[1:-1, 1:-1, 1:-1].reshape(-1).copy(), order, 3)
    got = u.copy()
    oracle.sweeps3d(got, f, h2, 3)
    scale = max(np.max(np.abs(x)), 1e-300)
    assert np.max(np.abs(got[1:-1, 1:-1, 1:-1].reshape(-1) - x)) <= 1e-13 * scale


def test_converges_to_the_dense_direct_solution():
    n = 5
    f, u = _random3(n, 3)
    h2 = 1.0 / (n + 1) ** 2
    x = np.linalg.solve(_dense7(n), _rhs3(f, u, h2))
    oracle.sweeps3d(u, f, h2, 400)
    assert np.max(np.abs(u[1:-1, 1:-1, 1:-1].reshape(-1) - x)) <= 1e-12 * np.max(np.abs(x))


def test_harmonic_quadratic_and_constant_data_are_reproduced():
    n = 15  # h = 1/16: the quadratic's node values are exact binary fractions
    (x, y, z), h = _coords(n)
    g = x * x + y * y - 2.0 * z * z  # Lap g = 0, and the 7-point stencil is exact for quadratics
    u = g.copy()
    u[1:-1, 1:-1, 1:-1] = 0.0
    oracle.sweeps3d(u, np.zeros((n, n, n)), h * h, 1500)
    assert np.max(np.abs(u - g)) <= 1e-12
    u = np.full((7, 7, 7), 0.75)  # 6 x 0.75 and its sixth are exact
    oracle.sweeps3d(u, np.zeros((5, 5, 5)), 1.0 / 36.0, 4)
    assert np.all(u == 0.75)


def test_n1_hand_case():
    # h = 1/2, h^2 f = 0.25 * 3 = 0.75; shell neighbours 1..6: (0.75 + 21) / 6 = 3.625
    u = np.zeros((3, 3, 3))
    u[0, 1, 1], u[2, 1, 1], u[1, 0, 1], u[1, 2, 1], u[1, 1, 0], u[1, 1, 2] = 1, 2, 3, 4, 5, 6
    oracle.sweeps3d(u, np.array([[[3.0]]]), 0.25, 2)
    assert u[1, 1, 1] == 3.625
    rho, r2, b2 = oracle.residual3d(u, np.array([[[3.0]]]), 0.25)
    assert r2 == 0.0 and b2 == 21.75 ** 2
