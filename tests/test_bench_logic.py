"""Host logic of bench.py: the sizes at which the library picks the cooperative FP64 launch,
the kernel each option resolves to, the committed ncu summaries it reads traffic from, and
the clock-sample summary.  No GPU needed."""
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
    base = dict(kernel=0, tile_rows=0, emulate=-1, values=0, rows=0, int_rows=0, fma=0)
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
    assert not b.uses_persistent(_args(fma=1), 16384, False)   # the fused update: one launch per colour
    assert b.resolved_kernel(16384, True, 0, 0) == (3, 4)       # FP32 wavefront above 2048
    assert b.resolved_kernel(1000, True, 0, 0) == (1, 1)
    assert b.resolved_kernel(16384, False, 4, 0) == (1, 1)


def test_committed_profiles_match_the_kernel_sources():
    """bench.py reports a kernel's DRAM traffic only from an ncu summary taken of the current
    sources; each committed summary must match them and hold a plausible figure (at least the
    24 B per update that one half-sweep of 16384^2 must move, and not far above it)."""
    b = _bench()
    algorithmic = 24.0 * 16384 * 16384 / 2
    for kname in b.PROFILES:
        traffic = b.profiled_traffic(kname, -1)
        assert traffic is not None, kname
        assert 1.0 <= traffic / algorithmic < 1.1, (kname, traffic)
        assert b.profiled_traffic(kname, 0x11) is None  # another arithmetic form: not reported


def test_clock_summary_reads_throttle_reasons(tmp_path):
    b = _bench()
    rows = [
        "0, GPU-aaa, 2070, 2070, 900.1, 0x0, Not Active, Not Active, Not Active, Not Active",
        "0, GPU-aaa, 2040, 2070, 1390.0, 0x4, Not Active, Not Active, Not Active, Active",
        "0, GPU-aaa, 2055, 2070, 1000.0, 0x0, Not Active, Not Active, Not Active, Not Active",
        "1, GPU-bbb, 1200, 2070, 300.0, 0x40, Not Active, Active, Not Active, Not Active",  # other GPU
        "garbled line",
    ]
    path = tmp_path / "clocks.csv"
    path.write_text("\n".join(rows) + "\n")
    s = b.ClockSampler("GPU-aaa")
    s.path = str(path)
    s.proc = object()  # as if nvidia-smi had run
    got = s.summary()
    assert got["sm_mhz"] == 2055 and got["sm_max_mhz"] == 2070 and got["samples"] == 3
    assert got["reasons"] == ["sw_power_cap"]
    s.uuid = None  # every GPU's rows
    assert s.summary()["reasons"] == ["hw_thermal_slowdown", "sw_power_cap"]


def test_default_step_counts(monkeypatch):
    """The grid bench times 10 steps by default (the paper reports the median of 10 runs);
    the other modes 5; an explicit --steps wins."""
    b = _bench()
    for argv, want in ((["bench.py"], 10), (["bench.py", "--impl", "reference"], 10),
                       (["bench.py", "--mode", "batched"], 5), (["bench.py", "--steps", "3"], 3)):
        monkeypatch.setattr("sys.argv", argv)
        assert b.parse().steps == want
