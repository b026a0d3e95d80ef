"""The library's integer-pipe binary64 add and exponent-decrement quarter must give the
same bits as IEEE 754 round-to-nearest-even hardware arithmetic (CPU only: the helpers
are compiled for the host from the library's own header and compared with numpy)."""
import ctypes
import os
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "native", "fp64_host_check.cpp")
OUT = os.path.join(HERE, "native", "_build", "libfp64check.so")
HDR = os.path.join(os.path.dirname(HERE), "paper_2607_01735_gb300", "csrc", "fp64.cuh")
HDR6 = os.path.join(os.path.dirname(HERE), "paper_2607_01735_gb300", "csrc", "div6.cuh")


def _cuda_include():
    for d in (os.environ.get("CUDA_HOME", ""), "/usr/local/cuda"):
        if d and os.path.exists(os.path.join(d, "include", "cuda_runtime.h")):
            return os.path.join(d, "include")
    pytest.skip("CUDA headers not found")


@pytest.fixture(scope="module")
def lib():
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    if not os.path.exists(OUT) or os.path.getmtime(OUT) < max(os.path.getmtime(SRC), os.path.getmtime(HDR), os.path.getmtime(HDR6)):
        tmp = OUT + f".tmp{os.getpid()}"
        subprocess.check_call(["g++", "-O2", "-ffp-contract=off", "-std=c++17", "-fPIC", "-shared",
                               "-I", _cuda_include(), SRC, "-o", tmp])
        os.replace(tmp, OUT)
    l = ctypes.CDLL(OUT)
    dp = ctypes.POINTER(ctypes.c_double)
    l.check_add_int.argtypes = [ctypes.c_long, dp, dp, dp]
    l.check_quarter.argtypes = [ctypes.c_long, dp, dp]
    l.check_div6.argtypes = [ctypes.c_long, dp, dp]
    l.check_add_core.argtypes = [ctypes.c_long, dp, dp, dp, ctypes.POINTER(ctypes.c_int)]
    return l


def _p(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _add(lib, a, b):
    a, b = np.ascontiguousarray(a, np.float64), np.ascontiguousarray(b, np.float64)
    out = np.empty_like(a)
    lib.check_add_int(a.size, _p(a), _p(b), _p(out))
    return out


def _core(lib, a, b):
    a, b = np.ascontiguousarray(a, np.float64), np.ascontiguousarray(b, np.float64)
    out = np.empty_like(a)
    ok = np.zeros(a.size, dtype=np.int32)
    lib.check_add_core(a.size, _p(a), _p(b), _p(out), ok.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out, ok.astype(bool)


def _same_bits(x, y):
    nan = np.isnan(x) & np.isnan(y)
    return np.all((x.view(np.uint64) == y.view(np.uint64)) | nan)


def _bits_to_f(u):
    return np.asarray(u, dtype=np.uint64).view(np.float64)


def test_add_random_bit_patterns(lib):
    rng = np.random.default_rng(1)
    a = _bits_to_f(rng.integers(0, 2 ** 64, 200000, dtype=np.uint64))
    b = _bits_to_f(rng.integers(0, 2 ** 64, 200000, dtype=np.uint64))
    with np.errstate(all="ignore"):
        assert _same_bits(_add(lib, a, b), a + b)


@pytest.mark.parametrize("spread", [0, 1, 2, 3, 8, 30, 53, 54, 60, 64, 70])
def test_add_close_exponents_both_signs(lib, spread):
    rng = np.random.default_rng(spread + 10)
    m = 300000
    e = rng.integers(-30, 30, m)
    a = np.ldexp(rng.uniform(1, 2, m), e) * rng.choice([-1.0, 1.0], m)
    b = np.ldexp(rng.uniform(1, 2, m), e - rng.integers(0, spread + 1, m)) * rng.choice([-1.0, 1.0], m)
    assert _same_bits(_add(lib, a, b), a + b)
    assert _same_bits(_add(lib, b, a), b + a)
    # the integer path itself takes (nearly) every one of these and is exact where it does
    r, ok = _core(lib, a, b)
    assert ok.mean() > 0.99
    assert _same_bits(r[ok], (a + b)[ok])


def test_add_near_cancellation_and_ties(lib):
    rng = np.random.default_rng(3)
    a = rng.uniform(-4, 4, 100000)
    ulps = rng.integers(-3, 4, a.size)
    b = -(a + ulps * np.spacing(a))
    assert _same_bits(_add(lib, a, b), a + b)
    # exact ties at every significand parity: 1 + k ulp plus half an ulp
    k = np.arange(0, 4096, dtype=np.float64)
    x = 1.0 + k * 2.0 ** -52
    for half in (2.0 ** -53, -(2.0 ** -53), 3 * 2.0 ** -54, 2.0 ** -54, 2.0 ** -53 + 2.0 ** -80):
        y = np.full_like(x, half)
        assert _same_bits(_add(lib, x, y), x + y)


def test_add_special_values(lib):
    tiny = np.finfo(np.float64).tiny
    big = np.finfo(np.float64).max
    vals = np.array([0.0, -0.0, 1.0, -1.0, tiny, -tiny, tiny / 2, 5e-324, -5e-324, big, -big,
                     np.inf, -np.inf, np.nan, 2.0 ** 1023, 1.5 * 2.0 ** 1023, 3 * tiny, 2 * tiny,
                     1.0 + 2.0 ** -52, 2.0 ** -1021, -(2.0 ** -1022) * 1.5])
    a, b = np.meshgrid(vals, vals)
    with np.errstate(all="ignore"):
        assert _same_bits(_add(lib, a.ravel(), b.ravel()), (a + b).ravel())


def test_add_solver_like_values(lib):
    # h2 f (tiny, either sign) plus neighbour values of O(1e-3 .. 1e-1)
    rng = np.random.default_rng(4)
    hf = rng.uniform(-1, 1, 400000) * 2.0 ** -28
    u = rng.normal(0, 0.05, 400000)
    assert _same_bits(_add(lib, hf, u), hf + u)
    assert _same_bits(_add(lib, u, -u * (1 + 1e-12)), u - u * (1 + 1e-12))
    r, ok = _core(lib, hf, u)
    assert ok.all() and _same_bits(r, hf + u)


def test_integer_path_domain(lib):
    # where the integer path declines: zero / subnormal / non-finite operands, exact
    # cancellation, subnormal sums
    tiny = np.finfo(np.float64).tiny
    a = np.array([0.0, 1.0, 5e-324, 1.0, np.inf, 1.0, 1.5 * tiny, 1.0])
    b = np.array([1.0, 0.0, 1.0, -1.0, 1.0, np.nan, -tiny, 2.0])
    _, ok = _core(lib, a, b)
    assert ok.tolist() == [False, False, False, False, False, False, False, True]


def test_quarter(lib):
    rng = np.random.default_rng(5)
    a = _bits_to_f(rng.integers(0, 2 ** 64, 200000, dtype=np.uint64))
    tiny = np.finfo(np.float64).tiny
    special = np.array([0.0, -0.0, tiny, 2 * tiny, 4 * tiny, 3 * tiny, 6 * tiny, 5e-324, np.inf,
                        -np.inf, np.nan, np.finfo(np.float64).max, 1.0, -3.0])
    # every rounding case of the integer path: biased exponents 0, 1, 2 (subnormal or zero
    # results, ties to even, carries into the smallest normal), 3 (the first exponent-
    # decrement case), both signs, random and extreme significands
    low = []
    for e in (0, 1, 2, 3):
        mant = np.concatenate([rng.integers(0, 2 ** 52, 20000, dtype=np.uint64),
                               np.arange(0, 16, dtype=np.uint64),
                               np.uint64(2 ** 52) - np.arange(1, 17, dtype=np.uint64)])
        for sgn in (0, 1):
            low.append((np.uint64(sgn) << np.uint64(63)) | (np.uint64(e) << np.uint64(52)) | mant)
    a = np.concatenate([a, special, _bits_to_f(np.concatenate(low))])
    out = np.empty_like(a)
    lib.check_quarter(a.size, _p(a), _p(out))
    with np.errstate(all="ignore"):
        assert _same_bits(out, a * 0.25)


def test_div6_is_the_correctly_rounded_quotient(lib):
    """div6 (Markstein's one-correction division by a constant) against IEEE division:
    random operands over the whole exponent range, exact multiples of 6 and their
    neighbours, contiguous significands, and the fallback's edge cases."""
    rng = np.random.default_rng(6)
    bits = rng.integers(0, 2 ** 63, 4_000_000, dtype=np.uint64) | (rng.integers(0, 2, 4_000_000, dtype=np.uint64) << 63)
    a = bits.view(np.float64)
    a = a[np.isfinite(a)]
    k = np.arange(1, 1_000_001, dtype=np.float64) * 6.0
    cont = (np.uint64(0x3FF0000000000000) + np.arange(2 ** 20, dtype=np.uint64)).view(np.float64)
    edge = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2250738585072014e-308, 1.7976931348623157e308, np.inf, -np.inf,
                     np.ldexp(1.0, -1016), np.ldexp(1.0, -1017), np.ldexp(1.0, 1020), np.ldexp(1.0, 1021)])
    a = np.concatenate([a, k, np.nextafter(k, 0), np.nextafter(k, np.inf), cont, cont * 3.0, edge])
    out = np.empty_like(a)
    lib.check_div6(a.size, _p(a), _p(out))
    want = a / 6.0
    assert np.array_equal(out.view(np.uint64), want.view(np.uint64))
    nan = np.array([np.nan])
    lib.check_div6(1, _p(nan), _p(out[:1]))
    assert np.isnan(out[0])
