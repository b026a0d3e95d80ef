"""GB300-native red-black Gauss-Seidel (RBGS) for the 2D Poisson equation.

A thin ctypes binding over ``librbgs.so`` (C ABI in ``include/rbgs.h``).  The names
match the C entry points; this module only marshals arguments (tensors -> pointers,
status codes -> exceptions).  Every step of the solve runs in the library's CUDA
kernels; there is no CPU fallback: importing works without a GPU, but any call that
needs the library raises if ``librbgs.so`` has not been built
(``python -m paper_2607_01735_gb300.build``).

Arrays: ``f`` is N x N and ``u`` is (N+2) x (N+2) (Dirichlet ring included), float64,
C-contiguous; torch tensors (CPU or CUDA) or numpy arrays.  h2 = h*h with h = 1/(N+1)
(Section 2 of the paper).
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "librbgs.so")

RBGS_OK, RBGS_EINVAL, RBGS_ENOMEM, RBGS_ECUDA, RBGS_ENOTCONV, RBGS_ENONFINITE, RBGS_ETIMEOUT = range(7)
STATUS_NAMES = {0: "RBGS_OK", 1: "RBGS_EINVAL", 2: "RBGS_ENOMEM", 3: "RBGS_ECUDA",
                4: "RBGS_ENOTCONV", 5: "RBGS_ENONFINITE", 6: "RBGS_ETIMEOUT"}
RBGS_FP64, RBGS_FP32_REFINE = 0, 1
RBGS_KERNEL_AUTO, RBGS_KERNEL_COLOUR, RBGS_KERNEL_TEMPORAL, RBGS_KERNEL_WAVEFRONT, RBGS_KERNEL_PERSISTENT = 0, 1, 2, 3, 4

# Every symbol include/rbgs.h declares.
EXPORTED = ("rbgs_default_opts", "rbgs_create", "rbgs_sweep", "rbgs_residual", "rbgs_solve",
            "rbgs_get_solution", "rbgs_set_solution", "rbgs_set_problem", "rbgs_solve_batched", "rbgs_destroy",
            "rbgs_last_error", "rbgs_residual_static", "rbgs_batched_last_shape", "rbgs_run_stream")


class RbgsError(RuntimeError):
    """A non-OK rbgs_status, with the library's message."""

    def __init__(self, status: int, message: str):
        super().__init__(f"{STATUS_NAMES.get(status, status)}: {message}")
        self.status = status


class Opts(ctypes.Structure):
    _fields_ = [("precision", ctypes.c_int), ("kernel", ctypes.c_int),
                ("check_every", ctypes.c_int), ("max_sweeps", ctypes.c_long),
                ("tblock_k", ctypes.c_int), ("tile_rows", ctypes.c_int),
                ("fp64_emulate", ctypes.c_int), ("inner_sweeps", ctypes.c_int),
                ("sweep_values", ctypes.c_int), ("sweep_rows", ctypes.c_int), ("int_rows", ctypes.c_int),
                ("team_size", ctypes.c_int), ("fma", ctypes.c_int), ("stall_checks", ctypes.c_int),
                ("max_seconds", ctypes.c_double)]


class Problem(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("h2", ctypes.c_double),
                ("f", ctypes.c_void_p), ("u_init", ctypes.c_void_p)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("sweeps", ctypes.c_long),
                ("rel", ctypes.c_double), ("latency_ms", ctypes.c_double)]


_lib = None


def load_library(path: str | None = None):
    """Load librbgs.so (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    path = path or LIB_PATH
    if not os.path.exists(path):
        raise RuntimeError(f"librbgs.so not found at {path}: build it with "
                           "`python -m paper_2607_01735_gb300.build` (needs nvcc)")
    lib = ctypes.CDLL(path)
    vp, c_int, c_long, c_double = ctypes.c_void_p, ctypes.c_int, ctypes.c_long, ctypes.c_double
    lib.rbgs_default_opts.argtypes = [ctypes.POINTER(Opts)]
    lib.rbgs_default_opts.restype = None
    lib.rbgs_create.argtypes = [c_int, c_double, vp, vp, ctypes.POINTER(Opts), vp, ctypes.POINTER(vp)]
    lib.rbgs_create.restype = c_int
    lib.rbgs_sweep.argtypes = [vp, c_long]
    lib.rbgs_sweep.restype = c_int
    lib.rbgs_residual.argtypes = [vp, ctypes.POINTER(c_double)]
    lib.rbgs_residual.restype = c_int
    lib.rbgs_solve.argtypes = [vp, c_double, ctypes.POINTER(c_long), ctypes.POINTER(c_double)]
    lib.rbgs_solve.restype = c_int
    lib.rbgs_get_solution.argtypes = [vp, vp]
    lib.rbgs_get_solution.restype = c_int
    lib.rbgs_set_solution.argtypes = [vp, vp]
    lib.rbgs_set_solution.restype = c_int
    lib.rbgs_set_problem.argtypes = [vp, vp, vp]
    lib.rbgs_set_problem.restype = c_int
    lib.rbgs_solve_batched.argtypes = [c_int, ctypes.POINTER(Problem), c_double, ctypes.POINTER(Opts),
                                       vp, ctypes.POINTER(vp), ctypes.POINTER(Result)]
    lib.rbgs_solve_batched.restype = c_int
    lib.rbgs_destroy.argtypes = [vp]
    lib.rbgs_destroy.restype = None
    lib.rbgs_residual_static.argtypes = [c_int, c_double, vp, vp, vp, vp]
    lib.rbgs_residual_static.restype = c_int
    lib.rbgs_last_error.argtypes = []
    lib.rbgs_last_error.restype = ctypes.c_char_p
    lib.rbgs_run_stream.argtypes = [vp, c_int, ctypes.POINTER(vp), ctypes.POINTER(vp), c_long, ctypes.POINTER(vp),
                                    ctypes.POINTER(c_double)]
    lib.rbgs_run_stream.restype = c_int
    lib.rbgs3d_create.argtypes = [c_int, c_double, vp, vp, vp, ctypes.POINTER(vp)]
    lib.rbgs3d_create.restype = c_int
    lib.rbgs3d_sweep.argtypes = [vp, c_long]
    lib.rbgs3d_sweep.restype = c_int
    lib.rbgs3d_residual.argtypes = [vp, ctypes.POINTER(c_double)]
    lib.rbgs3d_residual.restype = c_int
    lib.rbgs3d_get_solution.argtypes = [vp, vp]
    lib.rbgs3d_get_solution.restype = c_int
    lib.rbgs3d_destroy.argtypes = [vp]
    lib.rbgs3d_destroy.restype = None
    lib.rbgs_batched_last_shape.argtypes = [ctypes.POINTER(c_int)] * 5
    lib.rbgs_batched_last_shape.restype = None
    _lib = lib
    return lib


def rbgs_last_error() -> str:
    return load_library().rbgs_last_error().decode()


def _check(status: int, allowed=(RBGS_OK,)) -> int:
    if status not in allowed:
        raise RbgsError(status, rbgs_last_error())
    return status


def _ptr(a, dtype_name: str = "float64") -> int:
    """Address of a contiguous float64 torch tensor or numpy array."""
    if isinstance(a, np.ndarray):
        if a.dtype != np.dtype(dtype_name) or not a.flags.c_contiguous:
            raise TypeError(f"expected a C-contiguous {dtype_name} numpy array")
        return a.ctypes.data
    import torch
    if isinstance(a, torch.Tensor):
        if a.dtype != getattr(torch, dtype_name) or not a.is_contiguous():
            raise TypeError(f"expected a contiguous {dtype_name} tensor")
        return a.data_ptr()
    raise TypeError(f"unsupported array type {type(a)!r}")


def _stream_of(*arrays, stream=None) -> int | None:
    if stream is not None:
        return int(stream)
    import torch
    for a in arrays:
        if isinstance(a, torch.Tensor) and a.is_cuda:
            return torch.cuda.current_stream(a.device).cuda_stream
    return None


def default_opts(**kw) -> Opts:
    o = Opts()
    load_library().rbgs_default_opts(ctypes.byref(o))
    for k, v in kw.items():
        if not hasattr(o, k):
            raise KeyError(k)
        setattr(o, k, v)
    return o


def rbgs_create(n: int, h2: float, f, u_init, opts: Opts | None = None, stream=None) -> int:
    """rbgs_create: returns the context handle (an integer)."""
    lib = load_library()
    h = ctypes.c_void_p()
    s = _stream_of(f, u_init, stream=stream)
    _check(lib.rbgs_create(int(n), float(h2), _ptr(f), _ptr(u_init),
                           ctypes.byref(opts) if opts is not None else None, s, ctypes.byref(h)))
    return h.value


def rbgs_sweep(ctx: int, nsweeps: int) -> None:
    _check(load_library().rbgs_sweep(ctx, int(nsweeps)))


def rbgs_residual(ctx: int) -> float:
    rel = ctypes.c_double()
    _check(load_library().rbgs_residual(ctx, ctypes.byref(rel)))
    return rel.value


def rbgs_solve(ctx: int, tol: float, allow_not_converged: bool = False) -> tuple[int, float, int]:
    """rbgs_solve: returns (sweeps_done, rho, status)."""
    done, rel = ctypes.c_long(), ctypes.c_double()
    allowed = (RBGS_OK, RBGS_ENOTCONV) if allow_not_converged else (RBGS_OK,)
    st = _check(load_library().rbgs_solve(ctx, float(tol), ctypes.byref(done), ctypes.byref(rel)), allowed)
    return done.value, rel.value, st


def rbgs_get_solution(ctx: int, u_out) -> None:
    _check(load_library().rbgs_get_solution(ctx, _ptr(u_out)))


def rbgs_set_solution(ctx: int, u_in) -> None:
    _check(load_library().rbgs_set_solution(ctx, _ptr(u_in)))


def rbgs_set_problem(ctx: int, f, u_init) -> None:
    _check(load_library().rbgs_set_problem(ctx, _ptr(f), _ptr(u_init)))


def rbgs_run_stream(ctx: int, f_list, u_init_list, nsweeps: int, u_out_list,
                    allow_nonfinite: bool = False) -> list[float]:
    """rbgs_run_stream: a stream of problems of the context's size through one context,
    the host copies overlapping the neighbouring problems' sweeps; returns the rho values."""
    k = len(f_list)
    if not (len(u_init_list) == len(u_out_list) == k):
        raise ValueError("f, u_init and u_out lists must have the same length")
    arr = lambda xs: (ctypes.c_void_p * max(k, 1))(*[_ptr(x) for x in xs])
    rho = (ctypes.c_double * max(k, 1))()
    allowed = (RBGS_OK, RBGS_ENONFINITE) if allow_nonfinite else (RBGS_OK,)
    _check(load_library().rbgs_run_stream(ctx, k, arr(f_list), arr(u_init_list), int(nsweeps), arr(u_out_list),
                                          rho), allowed)
    return list(rho[:k])


def rbgs_destroy(ctx: int) -> None:
    if ctx:
        load_library().rbgs_destroy(ctx)


def rbgs_solve_batched(problems, tol: float, u_out: list, opts: Opts | None = None, stream=None,
                       allow_failures: bool = False) -> list[dict]:
    """problems: list of (n, h2, f, u_init); u_out: list of (n+2)^2 output arrays."""
    lib = load_library()
    k = len(problems)
    arr = (Problem * max(k, 1))()
    for p, (n, h2, f, u) in enumerate(problems):
        arr[p] = Problem(int(n), float(h2), _ptr(f), _ptr(u))
    outs = (ctypes.c_void_p * max(k, 1))(*[_ptr(u) for u in u_out])
    res = (Result * max(k, 1))()
    s = _stream_of(*(x for p in problems for x in p[2:]), stream=stream)
    st = lib.rbgs_solve_batched(k, arr, float(tol), ctypes.byref(opts) if opts is not None else None,
                                s, outs, res)
    if not allow_failures:
        _check(st)
    return [{"status": r.status, "sweeps": r.sweeps, "rel": r.rel, "latency_ms": r.latency_ms}
            for r in res[:k]]


def rbgs_batched_last_shape() -> dict:
    """rbgs_batched_last_shape: launch shape of this thread's last batched solve."""
    v = [ctypes.c_int(0) for _ in range(5)]
    load_library().rbgs_batched_last_shape(*[ctypes.byref(x) for x in v])
    return dict(zip(("threads", "blocks_per_sm", "team", "first", "nteam"), (x.value for x in v)))


def rbgs_residual_static(n: int, h2: float, f, u, rel_out, stream=None) -> None:
    """rbgs_residual_static: rho of a natural-layout device iterate into rel_out (device,
    one float64), allocating nothing (for callers that cannot allocate device memory)."""
    n = int(n)
    sizes = {"f": (f, n * n), "u": (u, (n + 2) * (n + 2)), "rel_out": (rel_out, 1)}
    for name, (a, need) in sizes.items():
        have = a.size if isinstance(a, np.ndarray) else a.numel()
        if (have < need) if name == "rel_out" else (have != need):
            raise RbgsError(RBGS_EINVAL, f"rbgs_residual_static: {name} holds {have} values, needs "
                                         f"{'at least ' if name == 'rel_out' else ''}{need} for n = {n}")
    import torch
    tensors = [a for a in (f, u, rel_out) if isinstance(a, torch.Tensor) and a.is_cuda]
    if len(tensors) != 3 or len({a.device for a in tensors}) != 1:
        raise RbgsError(RBGS_EINVAL, "rbgs_residual_static: f, u and rel_out must be CUDA tensors of one device")
    s = _stream_of(f, u, stream=stream)
    _check(load_library().rbgs_residual_static(n, float(h2), _ptr(f), _ptr(u), _ptr(rel_out), s))


class Solver:
    """Owning wrapper: ``with Solver(n, h2, f, u0) as s: s.sweep(10); s.residual()``."""

    def __init__(self, n, h2, f, u_init, opts: Opts | None = None, stream=None, **kw):
        if kw:
            opts = opts or default_opts()
            for key, v in kw.items():
                setattr(opts, key, v)
        self.n = n
        self.ctx = rbgs_create(n, h2, f, u_init, opts, stream)

    def sweep(self, nsweeps: int) -> None:
        rbgs_sweep(self.ctx, nsweeps)

    def residual(self) -> float:
        return rbgs_residual(self.ctx)

    def solve(self, tol: float, allow_not_converged: bool = False):
        return rbgs_solve(self.ctx, tol, allow_not_converged)

    def get_solution(self, u_out) -> None:
        rbgs_get_solution(self.ctx, u_out)

    def set_solution(self, u_in) -> None:
        rbgs_set_solution(self.ctx, u_in)

    def set_problem(self, f, u_init) -> None:
        rbgs_set_problem(self.ctx, f, u_init)

    def run_stream(self, f_list, u_init_list, nsweeps: int, u_out_list, allow_nonfinite: bool = False):
        return rbgs_run_stream(self.ctx, f_list, u_init_list, nsweeps, u_out_list, allow_nonfinite)

    def close(self) -> None:
        if self.ctx:
            rbgs_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Solver3D:
    """The 3D variant (include/rbgs3d.h): ``with Solver3D(n, h2, f, u0) as s: s.sweep(10)``.
    f is n^3, u (n+2)^3 with the boundary shell, float64, host or device."""

    def __init__(self, n, h2, f, u_init, stream=None):
        lib = load_library()
        h = ctypes.c_void_p()
        s = _stream_of(f, u_init, stream=stream)
        _check(lib.rbgs3d_create(int(n), float(h2), _ptr(f), _ptr(u_init), s, ctypes.byref(h)))
        self.n, self.ctx = n, h.value

    def sweep(self, nsweeps: int) -> None:
        _check(load_library().rbgs3d_sweep(self.ctx, int(nsweeps)))

    def residual(self) -> float:
        rel = ctypes.c_double()
        _check(load_library().rbgs3d_residual(self.ctx, ctypes.byref(rel)))
        return rel.value

    def get_solution(self, u_out) -> None:
        _check(load_library().rbgs3d_get_solution(self.ctx, _ptr(u_out)))

    def close(self) -> None:
        if self.ctx:
            load_library().rbgs3d_destroy(self.ctx)
            self.ctx = 0

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
