"""Write manufactured_rho_n255.txt: the closed-form relative residual of RBGS on the
model problem, for the manufactured right-hand side f = 2 pi^2 sin(pi x) sin(pi y),
zero Dirichlet ring, u0 = 0, N = 255 (h = 1/256).

Derivation (Section 2, Eq. (1) and the red-black colouring).  phi = sin(pi x) sin(pi y)
is an eigenvector of the 5-point operator: Adj phi = 4 mu phi with mu = cos(pi h), so
the discrete solution is c phi with c = (pi h / 2)^2 / sin^2(pi h / 2).  Every neighbour
of a red point is black and vice versa, so with u0 = 0 the error after k sweeps is
-c mu^(2k-1) (phi_red, mu phi_black), the black residual vanishes, and

    rho_k = c mu^(2k-1) (1 - mu^2) (4 / h^2) ||phi_red|| / (2 pi^2 ||phi||).

This script uses no solver code: only the formula above.
"""
import math
import os

import numpy as np

N = 255
SWEEPS = [1] + list(range(100, 1001, 100))


def closed_form(n, sweeps):
    h = 1.0 / (n + 1)
    mu = math.cos(math.pi * h)
    c = (math.pi * h / 2) ** 2 / math.sin(math.pi * h / 2) ** 2
    s = np.sin(math.pi * np.arange(1, n + 1) * h)
    phi2 = np.outer(s, s) ** 2
    i, j = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    red = ((i + j) % 2) == 0
    nr, nphi = math.sqrt(phi2[red].sum()), math.sqrt(phi2.sum())
    return [c * mu ** (2 * k - 1) * (1 - mu * mu) * (4 / (h * h)) * nr / (2 * math.pi ** 2 * nphi)
            for k in sweeps]


if __name__ == "__main__":
    out = os.path.join(os.path.dirname(os.path.abspath(__file__)), "manufactured_rho_n255.txt")
    with open(out, "w") as fh:
        fh.write("# Closed-form RBGS relative residual rho_k, f = 2 pi^2 sin(pi x) sin(pi y), N = 255,\n")
        fh.write("# zero ring, u0 = 0 (Section 2, Eq. (1); derivation in make_manufactured_rho.py).\n")
        fh.write("# sweeps rho\n")
        for k, r in zip(SWEEPS, closed_form(N, SWEEPS)):
            fh.write(f"{k} {r:.15e}\n")
