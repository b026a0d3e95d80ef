"""Oracle for the red-black Gauss-Seidel Poisson solve.

TEST INFRASTRUCTURE ONLY: the test suite, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package; the library
(``paper_2607_01735_gb300``) never does, and the two share no code.

``rbgs_ref.c`` holds the iteration itself (plain single-threaded C, built with
``-O2 -ffp-contract=off``); this module loads it through ctypes and adds the direct
solvers the tests pin it with (``oracle.direct``).  Arrays are numpy float64 (float32
for the binary32 sweep), natural row-major layout with the Dirichlet ring:
``u`` is (ni+2) x (nj+2), ``f`` is ni x nj.

Each function cites the passage of the paper it follows (Section 2, Eq. (1) and the
red-black colouring; Algorithms 1 and 2 for the red-then-black sweep order).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "rbgs_ref.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "librbgs_ref.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile rbgs_ref.c into oracle/_build/librbgs_ref.so (IEEE, no FP contraction)."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-std=c99",
                               "-fPIC", "-shared", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp, fp = ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float)
        c_int, c_long, c_double, c_float = ctypes.c_int, ctypes.c_long, ctypes.c_double, ctypes.c_float
        lib.ref_sweeps_f64.argtypes = [c_int, c_int, c_double, dp, dp, c_long, c_int]
        lib.ref_sweeps_f64.restype = None
        lib.ref_half_sweep_f64.argtypes = [c_int, c_int, c_double, dp, dp, c_int, c_int]
        lib.ref_half_sweep_f64.restype = None
        lib.ref_sweeps_f32.argtypes = [c_int, c_int, c_float, fp, fp, c_long, c_int]
        lib.ref_sweeps_f32.restype = None
        lib.ref_residual_f64.argtypes = [c_int, c_int, c_double, dp, dp, dp, dp]
        lib.ref_residual_f64.restype = c_double
        lib.ref_residual_field_f64.argtypes = [c_int, c_int, c_double, dp, dp, dp]
        lib.ref_residual_field_f64.restype = None
        lib.ref_solve_f64.argtypes = [c_int, c_int, c_double, dp, dp, c_double, c_int, c_long, dp]
        lib.ref_solve_f64.restype = c_long
        lib.ref_refine_solve.argtypes = [c_int, c_int, c_double, dp, dp, c_double, c_long, c_long, dp,
                                         ctypes.POINTER(c_long)]
        lib.ref_refine_solve.restype = c_long
        lib.ref_sweeps_fused.argtypes = [c_int, c_int, c_double, dp, dp, c_long, c_int, dp]
        lib.ref_sweeps_fused.restype = None
        lib.ref_sweeps3d_f64.argtypes = [c_int, c_double, dp, dp, c_long]
        lib.ref_sweeps3d_f64.restype = None
        lib.ref_residual3d_f64.argtypes = [c_int, c_double, dp, dp, dp, dp]
        lib.ref_residual3d_f64.restype = c_double
        _lib = lib
    return _lib


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _fptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_float))


def _check(u, f, dtype):
    if u.dtype != dtype or f.dtype != dtype:
        raise TypeError(f"expected {dtype} arrays")
    if not (u.flags.c_contiguous and f.flags.c_contiguous):
        raise ValueError("arrays must be C-contiguous")
    ni, nj = f.shape
    if u.shape != (ni + 2, nj + 2):
        raise ValueError(f"u must be {(ni + 2, nj + 2)}, got {u.shape}")
    return ni, nj


def sweeps(u: np.ndarray, f: np.ndarray, h2: float, nsweeps: int, parity: int = 0) -> np.ndarray:
    """nsweeps red+black sweeps of Eq. (1) in float64, in place on u (Section 2)."""
    ni, nj = _check(u, f, np.float64)
    _load().ref_sweeps_f64(ni, nj, float(h2), _dptr(f), _dptr(u), int(nsweeps), int(parity))
    return u


def sweeps_fused(u: np.ndarray, f: np.ndarray, h2: float, nsweeps: int, parity: int = 0,
                 bound: tuple[float, float] | None = None) -> np.ndarray:
    """nsweeps sweeps of the fused update (the library's fma = 1 mode: Eq. (1)'s five terms
    summed exactly on a 64-bit fixed-point grid, rounded once), in place on u.  `bound`
    = (max |u|, max |h2 f|) of the whole grid, for a window cut out of it."""
    ni, nj = _check(u, f, np.float64)
    bq = None
    if bound is not None:
        bq_arr = np.array(bound, dtype=np.float64)
        bq = _dptr(bq_arr)
    _load().ref_sweeps_fused(ni, nj, float(h2), _dptr(f), _dptr(u), int(nsweeps), int(parity), bq)
    return u


def half_sweep(u, f, h2, colour: int, parity: int = 0):
    """One colour (0 red: i+j even; 1 black) of Eq. (1), in place."""
    ni, nj = _check(u, f, np.float64)
    _load().ref_half_sweep_f64(ni, nj, float(h2), _dptr(f), _dptr(u), int(parity), int(colour))
    return u


def sweeps_f32(u: np.ndarray, f: np.ndarray, h2: float, nsweeps: int, parity: int = 0) -> np.ndarray:
    """The same iteration in binary32 arithmetic, in place on a float32 u."""
    ni, nj = _check(u, f, np.float32)
    _load().ref_sweeps_f32(ni, nj, float(np.float32(h2)), _fptr(f), _fptr(u), int(nsweeps), int(parity))
    return u


def residual(u: np.ndarray, f: np.ndarray, h2: float) -> tuple[float, float, float]:
    """(rho, sum rt^2, sum hb^2): rho = ||b - A u||_2 / ||b||_2 with the ring folded into b."""
    ni, nj = _check(u, f, np.float64)
    r2, b2 = ctypes.c_double(), ctypes.c_double()
    rho = _load().ref_residual_f64(ni, nj, float(h2), _dptr(f), _dptr(u),
                                   ctypes.byref(r2), ctypes.byref(b2))
    return rho, r2.value, b2.value


def residual_field(u: np.ndarray, f: np.ndarray, h2: float) -> np.ndarray:
    """Pointwise scaled residual h^2 (b - A u) on the interior."""
    ni, nj = _check(u, f, np.float64)
    r = np.empty((ni, nj), dtype=np.float64)
    _load().ref_residual_field_f64(ni, nj, float(h2), _dptr(f), _dptr(u), _dptr(r))
    return r


def solve(u, f, h2, tol: float, check_every: int, max_sweeps: int) -> tuple[int, float]:
    """Sweep until rho <= tol, checking every `check_every` sweeps; returns (sweeps, rho)."""
    ni, nj = _check(u, f, np.float64)
    rho = ctypes.c_double()
    done = _load().ref_solve_f64(ni, nj, float(h2), _dptr(f), _dptr(u), float(tol),
                                 int(check_every), int(max_sweeps), ctypes.byref(rho))
    return int(done), rho.value


def refine_solve(u, f, h2, tol: float, inner: int, max_sweeps: int) -> tuple[int, float, int]:
    """Mixed-precision refinement (binary32 sweeps, binary64 defect and correction), in
    place on u; returns (inner sweeps done, rho, outer steps)."""
    ni, nj = _check(u, f, np.float64)
    rho, outer = ctypes.c_double(), ctypes.c_long()
    done = _load().ref_refine_solve(ni, nj, float(h2), _dptr(f), _dptr(u), float(tol), int(inner),
                                    int(max_sweeps), ctypes.byref(rho), ctypes.byref(outer))
    return int(done), rho.value, outer.value


def window_value(f_full: np.ndarray, u0_full: np.ndarray, h2: float, nsweeps: int,
                 i: int, j: int, fused_bound: tuple[float, float] | None = None) -> float:
    """u[i, j] after nsweeps, computed on a window around (i, j) only.

    One half-sweep moves information one grid step, so a point depends only on the
    points within Manhattan distance 2 * nsweeps of it.  The window reaches
    2 * nsweeps + 1 steps in each direction (clipped at the true boundary); its outer
    ring is held fixed, which is exact for the centre.  The window keeps the global
    colouring through the parity offset.  With `fused_bound` = (max |u0|, max |h2 f|) of
    the whole grid the window runs the fused update at the whole grid's scale (one block
    of sweeps, nsweeps <= 1024).
    """
    n_i, n_j = f_full.shape
    r = 2 * nsweeps + 1
    a, b = max(1, i - r), min(n_i, i + r)
    c, d = max(1, j - r), min(n_j, j + r)
    u = np.ascontiguousarray(u0_full[a - 1:b + 2, c - 1:d + 2], dtype=np.float64)
    f = np.ascontiguousarray(f_full[a - 1:b, c - 1:d], dtype=np.float64)
    parity = (a - 1 + c - 1) & 1
    if fused_bound is not None:
        if nsweeps > 1024:
            raise ValueError("a fused window covers one block of at most 1024 sweeps")
        sweeps_fused(u, f, h2, nsweeps, parity, fused_bound)
    else:
        sweeps(u, f, h2, nsweeps, parity)
    return float(u[i - a + 1, j - c + 1])


def _check3(u, f):
    if u.dtype != np.float64 or f.dtype != np.float64:
        raise TypeError("expected float64 arrays")
    if not (u.flags.c_contiguous and f.flags.c_contiguous):
        raise ValueError("arrays must be C-contiguous")
    n = f.shape[0]
    if f.shape != (n, n, n) or u.shape != (n + 2, n + 2, n + 2):
        raise ValueError(f"f must be n^3 and u (n+2)^3, got {f.shape} and {u.shape}")
    return n


def sweeps3d(u: np.ndarray, f: np.ndarray, h2: float, nsweeps: int) -> np.ndarray:
    """nsweeps red+black sweeps of the 7-point 3D update (the paper's 3D outlook, Section 5:
    Eq. (1) with six neighbours, divided by 6), in place on u ((n+2)^3 with the shell)."""
    n = _check3(u, f)
    _load().ref_sweeps3d_f64(n, float(h2), _dptr(f), _dptr(u), int(nsweeps))
    return u


def residual3d(u: np.ndarray, f: np.ndarray, h2: float) -> tuple[float, float, float]:
    """(rho, sum rt^2, sum hb^2) of the 3D system, the shell folded into b."""
    n = _check3(u, f)
    r2, b2 = ctypes.c_double(), ctypes.c_double()
    rho = _load().ref_residual3d_f64(n, float(h2), _dptr(f), _dptr(u), ctypes.byref(r2), ctypes.byref(b2))
    return rho, r2.value, b2.value
