"""Direct solvers and a generic Gauss-Seidel that pin the oracle's iteration.

TEST INFRASTRUCTURE ONLY (see the package docstring).

The discrete problem of Section 2 (5-point stencil, Eq. (1), Dirichlet ring) is the
linear system  (4 I - Adj) u = h^2 b  on the N x N interior, where Adj couples the four
grid neighbours and h^2 b = h^2 f plus the ring values adjacent to each point.  This
module builds that system densely, solves it directly (numpy LAPACK for small N, the
type-I discrete sine transform for large N), and runs textbook Gauss-Seidel on the
matrix in an arbitrary point order.  RBGS is Gauss-Seidel in the order "all red
points, then all black points" (the colouring of Section 2); the tests use that fact.
"""
from __future__ import annotations

from fractions import Fraction

import numpy as np


def scaled_rhs(f: np.ndarray, u_ring: np.ndarray, h2: float) -> np.ndarray:
    """h^2 b: h^2 f_ij plus each neighbour of (i, j) that lies on the ring."""
    ni, nj = f.shape
    hb = h2 * f
    hb = hb.copy()
    hb[0, :] += u_ring[0, 1:nj + 1]
    hb[-1, :] += u_ring[ni + 1, 1:nj + 1]
    hb[:, 0] += u_ring[1:ni + 1, 0]
    hb[:, -1] += u_ring[1:ni + 1, nj + 1]
    return hb


def dense_matrix(ni: int, nj: int) -> np.ndarray:
    """h^2 A = 4 I - Adj over the interior, points numbered i-major (k = (i-1) nj + (j-1))."""
    m = ni * nj
    a = np.zeros((m, m), dtype=np.float64)
    for i in range(ni):
        for j in range(nj):
            k = i * nj + j
            a[k, k] = 4.0
            for di, dj in ((-1, 0), (1, 0), (0, -1), (0, 1)):
                ii, jj = i + di, j + dj
                if 0 <= ii < ni and 0 <= jj < nj:
                    a[k, ii * nj + jj] = -1.0
    return a


def dense_solve(f: np.ndarray, u_ring: np.ndarray, h2: float) -> np.ndarray:
    """Exact discrete solution by LU (numpy.linalg.solve); returns the full grid with ring."""
    ni, nj = f.shape
    x = np.linalg.solve(dense_matrix(ni, nj), scaled_rhs(f, u_ring, h2).reshape(-1))
    u = u_ring.copy()
    u[1:-1, 1:-1] = x.reshape(ni, nj)
    return u


def dst_solve(f: np.ndarray, u_ring: np.ndarray, h2: float) -> np.ndarray:
    """Exact discrete solution by diagonalising 4 I - Adj with the type-I sine transform.

    The orthonormal DST-I is symmetric and its own inverse; it diagonalises the 1D
    second difference with eigenvalues 4 sin^2(k pi / (2 (N + 1))), k = 1..N, so the 2D
    operator has eigenvalues lambda_kl = 4 sin^2(k pi h_i / 2) + 4 sin^2(l pi h_j / 2).
    """
    from scipy.fft import dst

    ni, nj = f.shape
    hb = scaled_rhs(f, u_ring, h2)
    k = np.arange(1, ni + 1, dtype=np.float64)[:, None]
    l = np.arange(1, nj + 1, dtype=np.float64)[None, :]
    lam = 4.0 * np.sin(k * np.pi / (2.0 * (ni + 1))) ** 2 + 4.0 * np.sin(l * np.pi / (2.0 * (nj + 1))) ** 2
    c = dst(dst(hb, type=1, axis=0, norm="ortho"), type=1, axis=1, norm="ortho")
    x = dst(dst(c / lam, type=1, axis=0, norm="ortho"), type=1, axis=1, norm="ortho")
    u = u_ring.copy()
    u[1:-1, 1:-1] = x
    return u


def red_black_order(ni: int, nj: int) -> list[int]:
    """Point numbers (i-major) of all red points (i + j even, 1-based), then all black."""
    red = [(i - 1) * nj + (j - 1) for i in range(1, ni + 1) for j in range(1, nj + 1) if (i + j) % 2 == 0]
    black = [(i - 1) * nj + (j - 1) for i in range(1, ni + 1) for j in range(1, nj + 1) if (i + j) % 2 == 1]
    return red + black


def gauss_seidel_dense(a: np.ndarray, rhs: np.ndarray, x: np.ndarray, order: list[int],
                       nsweeps: int) -> np.ndarray:
    """Textbook Gauss-Seidel on a dense matrix, visiting unknowns in `order`.

    x_k <- (rhs_k - sum_{m != k} a_km x_m) / a_kk, with the latest values of x; the
    off-diagonal sum runs over columns in increasing index.  Plain Python loops.
    """
    x = [float(v) for v in x]
    m = len(x)
    for _ in range(nsweeps):
        for k in order:
            s = 0.0
            for c in range(m):
                if c != k and a[k, c] != 0.0:
                    s += a[k, c] * x[c]
            x[k] = (rhs[k] - s) / a[k, k]
    return np.array(x)


def exact_rbgs(f, u_ring, h2, nsweeps: int):
    """RBGS in exact rational arithmetic (fractions.Fraction), for tiny grids.

    The same update as Eq. (1), red then black per sweep, with no rounding anywhere:
    the inputs are taken as the exact rationals their float64 values denote.
    """
    ni, nj = len(f), len(f[0])
    h2q = Fraction(h2)
    u = [[Fraction(float(v)) for v in row] for row in u_ring]
    fq = [[Fraction(float(v)) for v in row] for row in f]
    for _ in range(nsweeps):
        for colour in (0, 1):
            for i in range(1, ni + 1):
                for j in range(1, nj + 1):
                    if (i + j) % 2 == colour:
                        u[i][j] = (h2q * fq[i - 1][j - 1] + u[i - 1][j] + u[i + 1][j]
                                   + u[i][j - 1] + u[i][j + 1]) / 4
    return u
