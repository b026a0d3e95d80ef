"""The fused update's fixed-point helpers (csrc/fixed64.cuh), compiled for the host from
the library's own header, against exact arithmetic:

* to_fixed(t, e) must be trunc(t * 2^e) (numpy's ldexp is exact here, and the cast to
  int64 truncates toward zero);
* fixed_quarter_to_double(s, e) must be s * 2^-(e+2) rounded once to the nearest binary64,
  ties to even (checked against Python's correctly rounded integer division, and on
  constructed ties);
* scale_exponent must bound every term and sum below 2^61.
CPU only."""
import ctypes
import os
import random
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "native", "fixed64_host_check.cpp")
OUT = os.path.join(HERE, "native", "_build", "libfixed64check.so")
HDRS = [os.path.join(os.path.dirname(HERE), "paper_2607_01735_gb300", "csrc", h) for h in ("fixed64.cuh", "fp64.cuh")]


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    pytest.skip("CUDA headers not found")


@pytest.fixture(scope="module")
def lib():
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    newest = max(os.path.getmtime(p) for p in [SRC] + HDRS)
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < newest:
        tmp = OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared",
                               "-I", _cuda_include(), SRC, "-o", tmp])
        os.replace(tmp, OUT)
    l = ctypes.CDLL(OUT)
    vp = ctypes.c_void_p
    l.check_to_fixed.argtypes = [ctypes.c_long, vp, vp, vp]
    l.check_fixed_quarter.argtypes = [ctypes.c_long, vp, vp, vp]
    l.check_scale_exponent.argtypes = [ctypes.c_long, vp, vp, vp, vp]
    return l


def _to_fixed(lib, t, e):
    t = np.ascontiguousarray(t, np.float64)
    e = np.ascontiguousarray(np.broadcast_to(e, t.shape), np.int32)
    out = np.empty(t.shape, np.int64)
    lib.check_to_fixed(t.size, t.ctypes.data, e.ctypes.data, out.ctypes.data)
    return out


def _quarter(lib, s, e):
    s = np.ascontiguousarray(s, np.int64)
    e = np.ascontiguousarray(np.broadcast_to(e, s.shape), np.int32)
    out = np.empty(s.shape, np.float64)
    lib.check_fixed_quarter(s.size, s.ctypes.data, e.ctypes.data, out.ctypes.data)
    return out


def _exact_quarter(s: int, e: int) -> float:
    """s * 2^-(e+2) correctly rounded (Python's int / int is correctly rounded)."""
    k = e + 2
    return s / (1 << k) if k >= 0 else float(s * (1 << -k))


def test_to_fixed_truncates_exactly():
    rng = np.random.default_rng(1)
    e = rng.integers(-900, 1021, 200000).astype(np.int32)
    # |t| 2^e < 2^61: draw the magnitude's exponent below 61 - e
    top = 61 - e.astype(np.float64)
    mag = np.ldexp(rng.random(e.size) * 0.999 + 0.0005, (top - rng.integers(0, 80, e.size)).astype(np.int32))
    t = np.where(rng.random(e.size) < 0.5, -mag, mag)
    t[:5] = [0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308]
    lib_ = pytest.lib_fixed
    got = _to_fixed(lib_, t, e)
    want = np.ldexp(t, e).astype(np.int64)          # ldexp exact (no overflow); cast truncates
    assert np.array_equal(got, want)


def test_fixed_quarter_rounds_once_to_nearest_even():
    lib_ = pytest.lib_fixed
    rnd = random.Random(2)
    s_list, e_list = [], []
    for _ in range(60000):
        bits = rnd.randint(0, 62)
        s = rnd.getrandbits(bits) if bits else 0
        s = -s if rnd.random() < 0.5 else s
        s_list.append(s)
        e_list.append(rnd.randint(-960, 1020))
    # constructed ties and near-ties at the rounding position (bit length L > 53: the 53rd
    # bit from the top is the last kept bit)
    for _ in range(20000):
        L = rnd.randint(54, 63)
        keep = rnd.getrandbits(53) | (1 << 52)
        drop = L - 53
        half = 1 << (drop - 1)
        low = rnd.choice([half, half - 1, half + 1, 0, (1 << drop) - 1])
        s = (keep << drop) | low
        if s >= 1 << 63:
            continue
        s_list.append(-s if rnd.random() < 0.5 else s)
        e_list.append(rnd.randint(-960, 1020))
    s = np.array(s_list, np.int64)
    e = np.array(e_list, np.int32)
    got = _quarter(lib_, s, e)
    want = np.array([_exact_quarter(int(a), int(b)) for a, b in zip(s_list, e_list)])
    bad = np.flatnonzero(got.view(np.uint64) != want.view(np.uint64))
    assert bad.size == 0, [(s_list[i], e_list[i], got[i], want[i]) for i in bad[:5]]
    # zero is +0, and no nonzero result is subnormal for e <= 1020
    assert _quarter(lib_, np.array([0], np.int64), 7)[0].hex() == "0x0.0p+0"
    assert np.all((got == 0) | (np.abs(got) >= 2.2250738585072014e-308))


def test_scale_exponent_bounds_every_sum_below_2_61():
    lib_ = pytest.lib_fixed
    rng = np.random.default_rng(3)
    B = np.ldexp(rng.random(20000), rng.integers(-1000, 1000, 20000).astype(np.int32))
    Q = np.ldexp(rng.random(20000), rng.integers(-1000, 1000, 20000).astype(np.int32))
    sw = rng.integers(1, 1025, 20000).astype(np.int64)
    B[:4] = [0.0, 0.0, np.inf, 1.0]
    Q[:4] = [0.0, 1.0, 1.0, np.nan]
    out = np.empty(B.size, np.int32)
    lib_.check_scale_exponent(B.size, B.ctypes.data, Q.ctypes.data, sw.ctypes.data, out.ctypes.data)
    assert out[0] == 0 and out[2] == -100000 and out[3] == -100000
    ok = out != -100000
    S = 4.0 * B[ok] + (2.0 * sw[ok] + 1.0) * Q[ok]
    e = out[ok]
    assert np.all(e <= 1020)
    # S 2^e < 2^61, and the bound is tight to a factor 2 unless the cap applies
    assert np.all(np.ldexp(S, e) < 2.0 ** 61)
    tight = (e != 1020) & (S > 0)
    assert np.all(np.ldexp(S[tight], e[tight]) >= 2.0 ** 59)


@pytest.fixture(autouse=True, scope="module")
def _bind(lib):
    pytest.lib_fixed = lib
    yield
