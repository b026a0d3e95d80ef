"""Failure detection on the GPU without a fault.

* The bounded mbarrier wait that guards the temporally blocked kernel's TMA loads gives up
  on a barrier nothing completes, reports it through a status word, and the context stays
  usable (a control wait then completes).
* The grid barrier of the cooperative FP64 sweep launch: a block whose partner never
  arrives gives up after its poll limit and reports it; with both blocks present, both pass.
* The convolution kernels' abort protocol: a role whose wait runs out raises the block's
  abort flag and the failure word, and a role waiting on a hand-off from it leaves through
  the flag instead of waiting out its own (much longer) limit."""
import ctypes
import os
import shutil
import subprocess

import pytest
import torch

pytestmark = pytest.mark.gpu
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    out = os.path.join(HERE, "native", "_build", "libwaitcheck.so")
    os.makedirs(os.path.dirname(out), exist_ok=True)
    subprocess.check_call([nvcc, "-gencode", "arch=compute_103a,code=sm_103a", "-O2", "-std=c++17",
                           "-Xcompiler", "-fPIC", "-shared", os.path.join(HERE, "native", "wait_check.cu"),
                           "-o", out])
    l = ctypes.CDLL(out)
    l.run_wait_check.argtypes = [ctypes.c_uint, ctypes.c_int, ctypes.POINTER(ctypes.c_int)]
    l.run_wait_check.restype = ctypes.c_int
    l.run_abort_check.argtypes = [ctypes.c_uint, ctypes.c_uint, ctypes.POINTER(ctypes.c_int)]
    l.run_grid_barrier_check.argtypes = [ctypes.c_int, ctypes.c_uint, ctypes.POINTER(ctypes.c_int)]
    l.run_grid_barrier_check.restype = ctypes.c_int
    l.run_abort_check.restype = ctypes.c_int
    return l


def test_wait_that_never_completes_gives_up_and_reports(lib):
    st = ctypes.c_int(0)
    assert lib.run_wait_check(200, 0, ctypes.byref(st)) == 0
    assert st.value == 1  # every thread gave up, none saw completion
    # the context is still healthy: a barrier that is arrived on completes
    st = ctypes.c_int(0)
    assert lib.run_wait_check(200, 1, ctypes.byref(st)) == 0
    assert st.value == 2


@pytest.mark.parametrize("issuer_polls,waiter_polls,who_gives_up", [(1, 5000, "issuer"), (1 << 22, 1, "waiters")])
def test_abort_flag_releases_the_other_roles(lib, issuer_polls, waiter_polls, who_gives_up):
    # one side runs out after a single poll; the other side's limit is far longer (at most
    # 5000 suspending polls of up to 1 ms, or 2^22 spinning polls), so it can only leave
    # early through the abort flag
    out = (ctypes.c_int * 3)()
    assert lib.run_abort_check(issuer_polls, waiter_polls, out) == 0
    status, fail_issuer, fail_waiter = out[0], out[1], out[2]
    assert status == 1 | 2  # both roles returned without completion
    if who_gives_up == "issuer":
        assert (fail_issuer, fail_waiter) == (1, 0)
    else:
        assert (fail_issuer, fail_waiter) == (0, 1)


def test_grid_barrier_gives_up_when_a_block_never_arrives(lib):
    out = (ctypes.c_int * 2)()
    assert lib.run_grid_barrier_check(1, 1000, out) == 0
    assert (out[0], out[1]) == (2, 0)  # the waiting block gave up and said so
    out = (ctypes.c_int * 2)()
    assert lib.run_grid_barrier_check(0, 1 << 20, out) == 0
    assert (out[0], out[1]) == (0, 2)  # both present: both pass, no status
