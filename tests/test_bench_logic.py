"""Host logic of bench.py that mirrors the library: the sizes at which the library picks
the cooperative FP64 launch, and the kernel each option resolves to.  No GPU needed."""
import argparse
import importlib.util
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_module", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _const(name):
    src = open(os.path.join(ROOT, "paper_2607_01735_gb300", "csrc", "api.cu")).read()
    m = re.search(rf"constexpr int {name} = (\d+)(?: << (\d+))?;", src)
    assert m, name
    return int(m.group(1)) << int(m.group(2) or 0)


def _args(**kw):
    base = dict(kernel=0, tile_rows=0, emulate=-1, values=0, rows=0, int_rows=0)
    base.update(kw)
    return argparse.Namespace(**base)


def test_persistent_size_range_matches_the_library():
    b = _bench()
    assert b.PERSIST_MIN_N == _const("kPersistMinN")
    assert b.PERSIST_MAX_N == _const("kPersistMaxN")


def test_kernel_resolution():
    b = _bench()
    assert b.uses_persistent(_args(), 16384, False)
    assert not b.uses_persistent(_args(), 255, False)          # graphs below the range
    assert not b.uses_persistent(_args(), 40000, False)        # above it
    assert not b.uses_persistent(_args(), 16384, True)         # FP32 inner sweeps
    assert not b.uses_persistent(_args(kernel=1), 16384, False)  # one launch per colour asked
    assert not b.uses_persistent(_args(tile_rows=16), 16384, False)
    assert b.uses_persistent(_args(kernel=4), 100, False)      # asked for explicitly
    assert b.resolved_kernel(16384, True, 0, 0) == (3, 4)       # FP32 wavefront above 2048
    assert b.resolved_kernel(1000, True, 0, 0) == (1, 1)
    assert b.resolved_kernel(16384, False, 4, 0) == (1, 1)
