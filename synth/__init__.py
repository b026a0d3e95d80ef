"""Seeded synthetic inputs for the red-black Gauss-Seidel (RBGS) Poisson workloads.

This module is the one piece shared by the CUDA path's tests/benchmarks and by the
oracle's tests. It holds no solver arithmetic: only random numbers, the right-hand
sides f and the Dirichlet boundary data g that the workloads are defined with.

Random numbers come from one counter-based generator, SplitMix64 (Steele, Lea and
Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014; the finaliser
constants are the published ones).  Element ``t`` (0-based) of stream ``s`` is

    x = (s * 2**32 + t + 1) * GAMMA  (mod 2**64),   out = mix64(x)

and a uniform double on [0, 1) is ``(out >> 11) * 2**-53``.  Grid values are drawn
in i-major order over the interior: point (i, j), 1 <= i, j <= N, takes element
``(i - 1) * N + (j - 1)``.  Coordinates follow the paper's grid (Section 2):
``x = i * h`` along rows (the slow index), ``y = j * h`` along columns, h = 1/(N+1).

The integer generator is written with torch int64 tensors so that it runs on the
CPU or on a GPU and gives the same bits on both (integer arithmetic only).  Anything
that goes through a transcendental function (Box-Muller, sines) is evaluated on the
CPU in float64 and then copied, so both sides of a comparison get identical arrays.
"""
from __future__ import annotations

import math

import numpy as np
import torch

GAMMA = 0x9E3779B97F4A7C15
MIX1 = 0xBF58476D1CE4E5B9
MIX2 = 0x94D049BB133111EB
_MASK64 = (1 << 64) - 1


def _signed(c: int) -> int:
    """The int64 value with the same 64-bit pattern as the unsigned constant c."""
    return c - (1 << 64) if c >= (1 << 63) else c


def _srl(z: torch.Tensor, k: int) -> torch.Tensor:
    """Logical right shift of int64 bit patterns."""
    return (z >> k) & ((1 << (64 - k)) - 1)


def _mix64(z: torch.Tensor) -> torch.Tensor:
    z = (z ^ _srl(z, 30)) * _signed(MIX1)
    z = (z ^ _srl(z, 27)) * _signed(MIX2)
    return z ^ _srl(z, 31)


def splitmix64_scalar(stream: int, t: int) -> int:
    """Element t of stream `stream`, in plain Python integers (the definition)."""
    x = ((stream * (1 << 32) + t + 1) * GAMMA) & _MASK64
    x = ((x ^ (x >> 30)) * MIX1) & _MASK64
    x = ((x ^ (x >> 27)) * MIX2) & _MASK64
    return x ^ (x >> 31)


def splitmix64(stream: int, count: int, start: int = 0, device="cpu") -> torch.Tensor:
    """Elements start .. start+count-1 of a stream as int64 bit patterns."""
    if stream < 0 or start < 0 or count < 0:
        raise ValueError("stream, start and count must be non-negative")
    base = (stream << 32) + start + 1
    t = torch.arange(count, dtype=torch.int64, device=device) + _signed(base & _MASK64)
    return _mix64(t * _signed(GAMMA))


def uniform01(stream: int, count: int, start: int = 0, device="cpu") -> torch.Tensor:
    """Uniform float64 on [0, 1): the top 53 bits of each draw times 2**-53 (exact)."""
    z = splitmix64(stream, count, start, device)
    return _srl(z, 11).to(torch.float64) * (2.0 ** -53)


def uniform_pm1_grid(n: int, stream: int, device="cpu", nj: int | None = None) -> torch.Tensor:
    """f ~ U(-1, 1) i.i.d. on an n x nj interior (i-major draw order); 2U - 1 is exact."""
    nj = n if nj is None else nj
    return (uniform01(stream, n * nj, 0, device) * 2.0 - 1.0).reshape(n, nj)


def normal_pairs(stream: int, count: int, start: int = 0) -> np.ndarray:
    """Standard normals by Box-Muller on consecutive uniform pairs (CPU, float64).

    Pair m uses uniforms (start + 2m, start + 2m + 1) = (U1, U2);
    z_{2m} = sqrt(-2 ln(1 - U1)) cos(2 pi U2),  z_{2m+1} = ... sin(2 pi U2).
    """
    m = (count + 1) // 2
    u = uniform01(stream, 2 * m, start, "cpu").numpy()
    u1, u2 = u[0::2], u[1::2]
    r = np.sqrt(-2.0 * np.log1p(-u1))
    out = np.empty(2 * m, dtype=np.float64)
    out[0::2] = r * np.cos(2.0 * math.pi * u2)
    out[1::2] = r * np.sin(2.0 * math.pi * u2)
    return out[:count]


def grid_coords(n: int) -> tuple[np.ndarray, np.ndarray, float]:
    """x = i h (rows) and y = j h (columns) over the (n+2) x (n+2) grid incl. the ring."""
    h = 1.0 / (n + 1)
    idx = np.arange(n + 2, dtype=np.float64) * h
    return idx[:, None], idx[None, :], h


def h_squared(n: int) -> float:
    """h*h with h = 1/(N+1), each rounded once in float64."""
    h = 1.0 / (n + 1)
    return h * h


def manufactured_rhs(n: int) -> np.ndarray:
    """f = 2 pi^2 sin(pi x) sin(pi y) on the interior; -Lap u = f has u = sin(pi x) sin(pi y)."""
    x, y, _ = grid_coords(n)
    f = 2.0 * math.pi ** 2 * np.sin(math.pi * x) * np.sin(math.pi * y)
    return np.ascontiguousarray(f[1:-1, 1:-1])


def grf_rhs(n: int, stream: int, nj: int | None = None) -> tuple[np.ndarray, int]:
    """Gaussian random field with power spectrum |k|^-3, unit RMS, zero on the ring.

    Sine-series synthesis f_ij = sum_{k,l} xi_kl (k^2 + l^2)^(-3/4) sin(k pi i h) sin(l pi j h)
    with xi_kl ~ N(0, 1) drawn i-major over (k, l) = 1..N, evaluated by a type-I DST.
    Returns the field and the number of uniforms consumed from the stream.
    """
    from scipy.fft import dst

    nj = n if nj is None else nj
    xi = normal_pairs(stream, n * nj).reshape(n, nj)
    k = np.arange(1, n + 1, dtype=np.float64)[:, None]
    l = np.arange(1, nj + 1, dtype=np.float64)[None, :]
    a = xi * (k * k + l * l) ** -0.75
    # DST-I: y_j = 2 sum_k x_k sin(pi (j+1)(k+1)/(N+1)); halve for the plain sine sum
    f = dst(dst(a, type=1, axis=0), type=1, axis=1) * 0.25
    f /= math.sqrt(float(np.mean(f * f)))
    used = 2 * ((n * nj + 1) // 2)
    return np.ascontiguousarray(f), used


def ring_grid(n: int, g=None, nj: int | None = None) -> np.ndarray:
    """(n+2) x (nj+2) float64 grid: ring = g(x, y) (zero if None), interior = 0 (u0 = 0)."""
    nj = n if nj is None else nj
    u = np.zeros((n + 2, nj + 2), dtype=np.float64)
    if g is not None:
        h = 1.0 / (n + 1)
        x = np.arange(n + 2, dtype=np.float64)[:, None] * h
        y = np.arange(nj + 2, dtype=np.float64)[None, :] * h
        gv = np.broadcast_to(g(x, y), u.shape)
        u[0, :], u[-1, :], u[:, 0], u[:, -1] = gv[0, :], gv[-1, :], gv[:, 0], gv[:, -1]
    return u


def g_quadratic(x, y):
    """Dirichlet data g = x^2 - y^2 (harmonic)."""
    return x * x - y * y


def batched_problem_table(count: int = 512, stream: int = 3,
                          sizes=(63, 127, 255, 511, 1023)) -> list[dict]:
    """Uneven batch: per problem p, size index floor(5 U_{2p}) and boundary c = 2 U_{2p+1} - 1.

    The right-hand side of problem p is U(-1, 1) from stream 3 * 2**16 + p.
    """
    u = uniform01(stream, 2 * count).numpy()
    out = []
    for p in range(count):
        k = min(int(u[2 * p] * len(sizes)), len(sizes) - 1)
        out.append({"n": sizes[k], "c": 2.0 * u[2 * p + 1] - 1.0,
                    "f_stream": stream * (1 << 16) + p})
    return out


def batched_problem(entry: dict) -> tuple[np.ndarray, np.ndarray, float]:
    """(f, u_init with constant ring c, h^2) for one entry of the batched table."""
    n = entry["n"]
    f = uniform_pm1_grid(n, entry["f_stream"]).numpy()
    u = np.zeros((n + 2, n + 2), dtype=np.float64)
    u[0, :] = u[-1, :] = u[:, 0] = u[:, -1] = entry["c"]
    return f, u, h_squared(n)


def learned_guess_sample(n: int, stream: int) -> tuple[np.ndarray, np.ndarray]:
    """GRF f from `stream`, then a, b, c ~ U(-1, 1) from the same stream after f;
    ring g = a + b x + c y, interior 0.  Returns (f, u_init)."""
    f, used = grf_rhs(n, stream)
    abc = (uniform01(stream, 3, used).numpy() * 2.0 - 1.0)
    a, b, c = (float(v) for v in abc)
    u = ring_grid(n, lambda x, y: a + b * x + c * y)
    return f, u
