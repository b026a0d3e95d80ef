"""Failure detection on the GPU without a fault: the bounded mbarrier wait that guards the
temporally blocked kernel's TMA loads gives up on a barrier nothing completes, reports
it through a status word, and the context stays usable (a control wait then completes)."""
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
    return l


def test_wait_that_never_completes_gives_up_and_reports(lib):
    st = ctypes.c_int(0)
    assert lib.run_wait_check(200, 0, ctypes.byref(st)) == 0
    assert st.value == 1  # every thread gave up, none saw completion
    # the context is still healthy: a barrier that is arrived on completes
    st = ctypes.c_int(0)
    assert lib.run_wait_check(200, 1, ctypes.byref(st)) == 0
    assert st.value == 2
