"""Benchmark: plain FP64 red-black Gauss-Seidel on a 16384 x 16384 interior.

One step is one pass of the whole solver path over one synthetic problem, through the
C ABI: rbgs_set_problem (stage the natural-layout f and u0, split them into colours,
scale h^2 f, reduce ||h^2 b||), rbgs_sweep(200) (400 half-sweep launches, red then
black), rbgs_residual (the residual-norm reduction) and rbgs_get_solution (back to the
natural layout).  The solver context (its device buffers) is created once with
rbgs_create before timing.  Problem: -Lap u = f, zero Dirichlet ring, f ~ U(-1, 1)
i.i.d. from counter stream 1, u0 = 0, h = 1/16385.

`value` is whole-job GLUP/s (lattice-site updates, N^2 per sweep) with the inputs
resident in device memory; `e2e` is the same step with the inputs and the solution in
pinned host memory (copies inside the timed region), the copies of one step overlapping
the neighbouring steps' sweeps as a serving loop runs them (`e2e.serial`: host buffers
passed to the library, nothing overlapped).  With N > 1 processes (torchrun) every rank solves its own replica (the
single-grid path does not shard here) and the value is the sum over ranks over the
slowest rank's time.

--impl reference times the oracle (plain single-threaded C) on the host, one sweep of
the same grid per step.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "GLUP/s + HBM GB/s vs ~8 TB/s; time-to-residual 1e-8, plain vs chosen form"
UNIT = "GLUP/s"
BYTES_PER_LUP = 24  # FP64: read h2f and the other colour's value, write the own value
# committed ncu summaries with the DRAM traffic of the FP64 sweep kernels, and the sources
# each was captured from (the traffic is reported only while they are unchanged)
PROFILES = {
    "half_sweep_f64": ("profiles/half_sweep_f64_n16384.md",
                       ["paper_2607_01735_gb300/csrc/sweep.cu", "paper_2607_01735_gb300/csrc/sweep_impl.cuh",
                        "paper_2607_01735_gb300/csrc/fp64.cuh"]),
    "fused_half_sweep": ("profiles/fused_half_sweep_f64_n16384.md",
                         ["paper_2607_01735_gb300/csrc/fused.cu", "paper_2607_01735_gb300/csrc/fixed64.cuh",
                          "paper_2607_01735_gb300/csrc/fp64.cuh", "paper_2607_01735_gb300/csrc/sweep_impl.cuh"]),
    "persistent_sweeps<double>": ("profiles/persistent_sweeps_f64_n16384.md",
                                  ["paper_2607_01735_gb300/csrc/persistent.cu",
                                   "paper_2607_01735_gb300/csrc/grid_barrier.cuh",
                                   "paper_2607_01735_gb300/csrc/sweep_impl.cuh",
                                   "paper_2607_01735_gb300/csrc/fp64.cuh"]),
}
PERSIST_MIN_N, PERSIST_MAX_N = 416, 1 << 15
# side files of a run (nvidia-smi clock samples, trained U-Net parameters)
OUT_DIR = os.environ.get("RBGS_BENCH_OUT", os.path.join(ROOT, "bench_out"))

def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=None,
                   help="timed steps (default: 10 for the grid, as the median of 10 runs of the "
                        "paper's measurements; 5 for the other modes)")
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--n", type=int, default=16384)
    p.add_argument("--sweeps", type=int, default=200)
    p.add_argument("--emulate", type=int, default=-1, help="FP64 add split (-1: library default)")
    p.add_argument("--tile-rows", type=int, default=0)
    p.add_argument("--values", type=int, default=0, help="values per thread in a half-sweep (0 auto, 2, 4)")
    p.add_argument("--rows", type=int, default=0, help="rows per loop step in a half-sweep (0 auto, 1, 2)")
    p.add_argument("--int-rows", type=int, default=0, help="hybrid FP64: integer-pipe rows per strip pair")
    p.add_argument("--fma", type=int, default=-1, choices=[-1, 0, 1],
                   help="FP64 update: 0 bit-exact, 1 fused (exact fixed-point sum, one rounding); -1 (default): "
                        "both, the fused form as the headline")
    p.add_argument("--kernel", type=int, default=0,
                   help="0 auto, 1 one launch per colour, 2 temporal (TMA tiles), 3 register wavefront, "
                        "4 all sweeps in one cooperative launch (FP64)")
    p.add_argument("--tblock-k", type=int, default=0, help="sweeps per temporal or wavefront pass (0 auto)")
    p.add_argument("--precision", choices=["fp64", "refine"], default="fp64",
                   help="fp64: plain FP64 sweeps; refine: FP32 sweeps with FP64 defect correction")
    p.add_argument("--inner", type=int, default=0, help="FP32 sweeps per correction (refine)")
    p.add_argument("--train-samples", type=int, default=4096, help="learned: training problems (255^2)")
    p.add_argument("--train-steps", type=int, default=3000, help="learned: Adam steps")
    p.add_argument("--eval-sizes", default="1023,4095", help="learned: held-out grid sizes")
    p.add_argument("--eval-fields", type=int, default=8, help="learned: held-out fields per size")
    p.add_argument("--eval-first", type=int, default=0,
                   help="learned: index k of the first held-out field (stream 5000 + 100 k + N mod 97)")
    p.add_argument("--eval-cap", default="5000000,20000000", help="learned: sweep cap per solve, per size")
    p.add_argument("--eval-starts", default="zero,coarse,full;zero,full",
                   help="learned: guesses solved from, per size (';'-separated)")
    p.add_argument("--plain-fields", default="8,1",
                   help="learned: fields per size also solved from u0 = 0 by plain FP64 (fused update)")
    p.add_argument("--conv-batch", type=int, default=16, help="conv: batch of the layer inputs")
    p.add_argument("--conv-hw", type=int, default=256, help="conv: level-0 height = width")
    p.add_argument("--conv-layer", type=int, default=-1, help="conv: one layer index (-1: all 15)")
    p.add_argument("--conv-op", choices=["all", "fwd", "dgrad", "wgrad"], default="all")
    p.add_argument("--engine", choices=["tcgen05", "mma_sync", "tcgen05_gather", "tcgen05_ring", "tcgen05_taprow",
                                        "both", "all"], default="both",
                   help="conv: engine(s) to time (both: tcgen05 and mma_sync; all: every engine, and the "
                        "tcgen05 engine with each weight-gradient kernel forced)")
    p.add_argument("--mixed-n", type=int, default=8192, help="mixed: interior size")
    p.add_argument("--mixed-cap", type=int, default=20000, help="mixed: sweeps actually run per form")
    p.add_argument("--mixed-chunk", type=int, default=2000, help="mixed: sweeps between residual samples")
    p.add_argument("--mixed-tol", type=float, default=1e-10, help="mixed: relative residual target")
    p.add_argument("--n3", type=int, default=511, help="3d: interior size per side")
    p.add_argument("--mode", choices=["grid", "batched", "learned", "conv", "mixed", "3d"], default="grid",
                   help="grid: one large grid (default); batched: many uneven problems in one launch")
    p.add_argument("--nprob", type=int, default=512)
    p.add_argument("--sizes", default="63,127,255,511,1023", help="batched: allowed interior sizes")
    p.add_argument("--tol", type=float, default=1e-8, help="batched: relative residual target")
    p.add_argument("--sequential", action="store_true",
                   help="batched: also estimate the one-problem-at-a-time plain FP64 wall time")
    p.add_argument("--team", type=int, default=0,
                   help="batched: 0 autotuned, 1 one block per problem, 2/4 phased plan with clusters")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--no-ttr", action="store_true", help="skip the time-to-residual comparison")
    p.add_argument("--ttr-n", type=int, default=511, help="grid for the time-to-residual comparison")
    a = p.parse_args()
    if a.steps is None:
        a.steps = 10 if a.mode == "grid" else 5
    return a


def workload(n, sweeps, precision="fp64"):
    if precision == "refine":
        return (f"RBGS FP32 sweeps + FP64 defect correction, {n}x{n} interior, zero Dirichlet ring, "
                f"f~U(-1,1) seed 1, u0=0, {sweeps} sweeps + residual norm")
    return (f"plain RBGS FP64, {n}x{n} interior, zero Dirichlet ring, f~U(-1,1) seed 1, u0=0, "
            f"{sweeps} red+black sweeps + residual norm")


def kernel_hash(sources):
    h = hashlib.sha256()
    for rel in sources:
        with open(os.path.join(ROOT, rel), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profiled_traffic(kname, emulate):
    """Per-launch DRAM bytes from the committed ncu summary, if it matches this kernel."""
    if kname not in PROFILES:
        return None
    path, sources = PROFILES[kname]
    try:
        with open(os.path.join(ROOT, path)) as fh:
            text = fh.read()
    except OSError:
        return None
    vals = {}
    for line in text.splitlines():
        if line.startswith("- ") and ":" in line:
            k, v = line[2:].split(":", 1)
            vals[k.strip()] = v.strip().strip("`")
    if vals.get("kernel_sources_sha256_16") != kernel_hash(sources):
        return None
    if str(vals.get("fp64_emulate")) != str(emulate):
        return None
    try:
        return float(vals["traffic_bytes_per_launch"])
    except (KeyError, ValueError):
        return None


def uses_persistent(args, n, refine):
    """The FP64 sweeps run in one cooperative launch: RBGS_KERNEL_PERSISTENT, or AUTO with
    the default launch shape and PERSIST_MIN_N <= n <= PERSIST_MAX_N (the library's rule)."""
    if refine or args.fma:
        return False
    if args.kernel == 4:
        return True
    return (args.kernel == 0 and args.tile_rows == 0 and args.emulate == -1 and args.values in (0, 2)
            and args.rows in (0, 1) and args.int_rows <= 0 and PERSIST_MIN_N <= n <= PERSIST_MAX_N)


def resolved_kernel(n, refine, kernel, tblock_k):
    """The sweep kernel and depth the library runs (RBGS_KERNEL_AUTO as documented in
    include/rbgs.h): 1 one launch per colour, 2 TMA tiles, 3 register wavefront."""
    if kernel == 4:  # persistent FP64 sweeps; FP32 inner sweeps as one launch per colour
        return 1, 1
    if kernel:
        return kernel, (tblock_k or (4 if refine else 2))
    if tblock_k:
        return 1, 1
    if refine:
        return (3, 4) if n > 2048 else (1, 1)
    return 1, 1


def device_peaks(dev):
    """(FP64-pipe peak in T adds/s with its source, HBM GB/s with its source) for `dev`."""
    import torch
    peaks = measured_peaks()
    sms = torch.cuda.get_device_properties(dev).multi_processor_count
    mhz = float(peaks.get("sm_max_mhz", 2070.0)) if peaks else 2070.0
    alu = 2.0 * sms * mhz * 1e6 / 1e12
    alu_src = f"FP64 pipe: 2 instr/clk/SM x {sms} SMs x {mhz:.0f} MHz (one flop = one correctly rounded FP64 add)"
    hbm = peaks["hbm_gbs"] if peaks else 6800.0
    hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s"
    return alu, alu_src, hbm, hbm_src


def measured_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as fh:
            return json.load(fh)
    except OSError:
        return None


class ClockSampler:
    """nvidia-smi samples every 200 ms while the timed region runs."""

    FIELDS = ("index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid):
        self.uuid = uuid
        self.proc = None
        self.path = os.path.join(OUT_DIR, f"clocks_{os.getpid()}.csv")

    def __enter__(self):
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.fh = open(self.path, "w")
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                                          "-lms", "200"], stdout=self.fh, stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
            self.fh.close()

    def summary(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) < 10:
                    continue
                if self.uuid and self.uuid not in parts[1]:
                    continue
                try:
                    sm.append(float(parts[2]))
                    smax.append(float(parts[3]))
                except ValueError:
                    continue
                for name, val in zip(names, parts[6:10]):
                    if val.lower() == "active":
                        reasons.add(name)
        if not sm:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(smax), "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def cpu_oracle_rate(n, stream=1, target_s=10.0):
    """Oracle GLUP/s on the host: sweeps of the same n x n problem, ~target_s of work."""
    import numpy as np

    import oracle
    import synth
    oracle.build()
    f = synth.uniform_pm1_grid(n, stream).numpy()
    u = np.zeros((n + 2, n + 2))
    h2 = synth.h_squared(n)
    t0 = time.perf_counter()
    oracle.sweeps(u, f, h2, 1)
    t1 = time.perf_counter()
    done, elapsed = 1, t1 - t0
    more = max(0, min(50, int(target_s / max(elapsed, 1e-9)) - 1))
    if more:
        t0 = time.perf_counter()
        oracle.sweeps(u, f, h2, more)
        elapsed += time.perf_counter() - t0
        done += more
    return {"value": n * n * done / elapsed / 1e9, "unit": UNIT, "cores": 1, "kind": "oracle",
            "sample": f"{done} sweep(s) of the {n}x{n} grid (plain single-threaded C, -O2 "
                      f"-ffp-contract=off), {elapsed:.1f} s"}


def time_to_residual(n, tol=1e-8, stream=0):
    """Wall time to relative residual `tol` from u0 = 0 (f ~ U(-1,1), zero ring): plain
    FP64 RBGS vs FP32 sweeps with FP64 defect correction, same GPU, same check interval."""
    import torch

    import paper_2607_01735_gb300 as rb
    import synth
    h2 = synth.h_squared(n)
    f = synth.uniform_pm1_grid(n, stream, device="cuda")
    u0 = torch.zeros(n + 2, n + 2, dtype=torch.float64, device="cuda")
    out = {"n": n, "tol": tol, "workload": f"{n}x{n}, f~U(-1,1) stream {stream}, zero ring, u0=0"}
    for name, kw in (("plain_fp64", dict(check_every=100)),
                     ("fp32_refine", dict(precision=rb.RBGS_FP32_REFINE, inner_sweeps=100))):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with rb.Solver(n, h2, f, u0, **kw) as s:
            sweeps, rho, st = s.solve(tol, allow_not_converged=True)
        torch.cuda.synchronize()
        out[name] = {"seconds": time.perf_counter() - t0, "sweeps": sweeps, "rho": rho, "status": st}
    out["speedup"] = out["plain_fp64"]["seconds"] / out["fp32_refine"]["seconds"]
    return out


def small_grid_history(stream=0):
    """The small configuration: 255^2 interior (h = 1/256), zero ring, u0 = 0, 1000 FP64
    sweeps with the residual every 100, for f = 2 pi^2 sin(pi x) sin(pi y) and for f ~ U(-1,1);
    wall time of the whole loop (sweeps and residuals, one context per right-hand side)."""
    import torch

    import paper_2607_01735_gb300 as rb
    import synth
    n = 255
    h2 = synth.h_squared(n)
    out = {"n": n, "sweeps": 1000, "check_every": 100}
    for name, f in (("manufactured", torch.from_numpy(synth.manufactured_rhs(n)).cuda()),
                    ("uniform", synth.uniform_pm1_grid(n, stream, device="cuda"))):
        u0 = torch.from_numpy(synth.ring_grid(n)).cuda()
        with rb.Solver(n, h2, f, u0) as s:  # warm the graph and the kernels
            s.sweep(100)
            s.residual()
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        with rb.Solver(n, h2, f, u0) as s:
            hist = []
            for _ in range(10):
                s.sweep(100)
                hist.append(s.residual())
        torch.cuda.synchronize()
        dt = time.perf_counter() - t0
        out[name] = {"seconds": dt, "us_per_sweep": 1e6 * dt / 1000, "rho_every_100": hist}
    return out


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return 0
    import numpy as np

    import oracle
    import synth
    oracle.build()
    n = args.n
    f = synth.uniform_pm1_grid(n, 1).numpy()
    u = np.zeros((n + 2, n + 2))
    h2 = synth.h_squared(n)
    for _ in range(args.warmup):
        oracle.sweeps(u, f, h2, 1)
    times = []
    for _ in range(args.steps):
        t0 = time.perf_counter()
        oracle.sweeps(u, f, h2, 1)
        times.append(time.perf_counter() - t0)
    t = sum(times)
    value = n * n * args.steps / t / 1e9
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic",
            "config": {"workload": workload(n, args.sweeps), "n": n,
                       "reference_step": "one sweep of the same grid by the oracle (the step is "
                                         "bounded; the GPU arm's step is the full sweep count)"},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": f"{args.steps} timed sweep(s) of the {n}x{n} grid, one per step"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
            "gpu_launches": 0}
    print(json.dumps(line))
    return 0


def run_batched(args):
    """Uneven batch (size index and boundary constant from stream 3, f from stream
    3*2^16+p) solved to args.tol in one persistent launch per rank; problems shard across
    ranks by estimated work.  Reports problems/s and per-problem latency percentiles."""
    import numpy as np
    import torch
    import torch.distributed as dist

    import paper_2607_01735_gb300 as rb
    import synth
    from paper_2607_01735_gb300 import sharding

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    sizes_allowed = tuple(int(x) for x in args.sizes.split(","))
    table = synth.batched_problem_table(args.nprob, 3, sizes=sizes_allowed)
    mine = sharding.shard([e["n"] for e in table], world, args.tol)[rank]
    probs, outs = [], []
    for p in mine:
        f, u, h2 = synth.batched_problem(table[p])
        probs.append((table[p]["n"], h2, torch.from_numpy(f).to(dev), torch.from_numpy(u).to(dev)))
        outs.append(torch.empty_like(probs[-1][3]))
    refine = args.precision == "refine"
    opts = rb.default_opts(precision=rb.RBGS_FP32_REFINE if refine else rb.RBGS_FP64,
                           inner_sweeps=args.inner, check_every=100, team_size=args.team)
    stream = torch.cuda.current_stream(dev)
    # the launch-shape autotuner runs on the first call for a size mix and caches its choice;
    # a call capped at one sweep triggers it without a full solve
    warm = rb.default_opts(precision=opts.precision, inner_sweeps=args.inner, check_every=100,
                           team_size=args.team, max_sweeps=1)
    rb.rbgs_solve_batched(probs, args.tol, outs, warm, allow_failures=True)
    for _ in range(args.warmup):  # full warm-up solves
        rb.rbgs_solve_batched(probs, args.tol, outs, opts, allow_failures=True)
    torch.cuda.synchronize(dev)
    if world > 1:
        dist.barrier()
    times, res = [], None
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = rb.rbgs_solve_batched(probs, args.tol, outs, opts, allow_failures=True)
        e1.record(stream)
        torch.cuda.synchronize(dev)
        times.append(e0.elapsed_time(e1) / 1e3)
    t = sharding.max_over_ranks(sum(times) / len(times), world, dev)
    local_res = {p: r for p, r in zip(mine, res)}
    allres = sharding.gather_results(local_res, world)
    if rank == 0:
        lat = np.array([allres[p]["latency_ms"] for p in sorted(allres)])
        ok = sum(1 for r in allres.values() if r["status"] == 0)
        lups = sum(float(table[p]["n"]) ** 2 * allres[p]["sweeps"] for p in allres)
        line = {"metric": "problems/s (batched, each to relative residual %.0e)" % args.tol,
                "value": args.nprob / t, "unit": "problems/s", "n_gpus": world, "steps": args.steps,
                "warmup": args.warmup, "ms_per_step": 1e3 * t, "higher_is_better": True,
                "scaling": "weak" if world > 1 else "strong", "vs_baseline": None,
                "dtype": "f32+f64" if refine else "f64", "data": "synthetic",
                "config": {"workload": f"{args.nprob} problems, sizes {list(sizes_allowed)}, "
                                       f"constant boundary, f~U(-1,1); tol {args.tol:g}; "
                                       f"{'FP32+refinement' if refine else 'FP64'}",
                           "parallelism": f"problems sharded x{world}"},
                "converged": ok, "latency_ms": {"p50": float(np.percentile(lat, 50)),
                                                 "p99": float(np.percentile(lat, 99)),
                                                 "max": float(lat.max())},
                "glups": lups / t / 1e9, "total_sweeps": int(sum(r["sweeps"] for r in allres.values())),
                "launch_shape": rb.rbgs_batched_last_shape(),
                "step_s": [round(x, 4) for x in times]}
        if args.sequential and world == 1:
            line["sequential_plain_fp64"] = sequential_estimate(rb, torch, table, allres, args.tol, dev, stream)
            line["sequential_plain_fp64"]["batched_speedup"] = line["sequential_plain_fp64"]["seconds"] / t
        alu, alu_src, hbm, hbm_src = device_peaks(dev)
        if refine:  # FP32 sweeps dominate; the problems are L2-resident, so this is a floor
            achieved = 12.0 * lups / t / 1e9
            line["roofline"] = {"bound": "hbm", "achieved": achieved, "peak": hbm * world, "unit": "GB/s",
                                "frac": achieved / (hbm * world), "traffic": None,
                                "kernel": "batched_persistent_kernel (FP32 inner sweeps)", "peak_source": hbm_src,
                                "note": "algorithmic FP32 sweep bytes (12 B per update) over the batch time; "
                                        "the problems are L2-resident"}
        else:
            achieved = 4.0 * lups / t / 1e12
            line["roofline"] = {"bound": "alu", "achieved": achieved, "peak": alu * world, "unit": "TFLOP/s",
                                "frac": achieved / (alu * world), "traffic": None,
                                "kernel": "batched_persistent_kernel (FP64 sweeps)", "peak_source": alu_src,
                                "note": "4 FP64 adds per update of every problem over the batch time, "
                                        "residual checks and load imbalance included"}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


def sequential_estimate(rb, torch, table, res, tol, dev, stream, probe_sweeps=2000):
    """Wall time of solving the batch's problems one after another with plain FP64 rbgs_solve
    (bit-exact, check every 100 sweeps, each problem on the whole GPU).  The batched FP64
    iterate equals the single-problem solve bit for bit, so each problem's sweep count is the
    batch's; per size, the cost of a sweep (check included) and of loading a problem are
    measured on one context, and the time is the sum of count x cost.  An estimate from
    measured costs, labelled as such (it avoids re-running the whole batch serially)."""
    import synth
    per_size = {}
    for n in sorted({table[p]["n"] for p in res}):
        p0 = next(p for p in res if table[p]["n"] == n)
        f, u, h2 = synth.batched_problem(table[p0])
        fd, ud = torch.from_numpy(f).to(dev), torch.from_numpy(u).to(dev)
        with rb.Solver(n, h2, fd, ud, check_every=100, max_sweeps=probe_sweeps, stall_checks=-1) as s:
            s.solve(0.0, allow_not_converged=True)  # warm: graphs, caches
            e = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
            e[0].record(stream)
            s.set_problem(fd, ud)
            e[1].record(stream)
            s.solve(0.0, allow_not_converged=True)
            e[2].record(stream)
            torch.cuda.synchronize(dev)
            per_size[n] = {"load_s": e[0].elapsed_time(e[1]) / 1e3,
                           "s_per_sweep": e[1].elapsed_time(e[2]) / 1e3 / probe_sweeps}
    total = sum(per_size[table[p]["n"]]["load_s"] + res[p]["sweeps"] * per_size[table[p]["n"]]["s_per_sweep"]
                for p in res)
    return {"seconds": total, "problems_per_s": len(res) / total, "per_size": per_size,
            "how": f"estimate: per problem, its sweep count x the measured cost per sweep of rbgs_solve at its "
                   f"size (check every 100, measured over {probe_sweeps} sweeps) + the measured load time"}


def run_3d(args):
    """The 3D variant (the paper's 3D outlook): n^3 interior, zero boundary shell,
    f ~ U(-1,1) from stream 1, u0 = 0, `sweeps` 7-point red-black sweeps + the residual per
    step, on one context (the problem reloaded each step from device memory)."""
    import torch

    import paper_2607_01735_gb300 as rb
    import synth

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, sweeps = args.n3, args.sweeps
    h2 = 1.0 / float(n + 1) ** 2
    f = synth.uniform_pm1_grid(n * n, 1, device=dev, nj=n).reshape(n, n, n).contiguous()
    u0 = torch.zeros(n + 2, n + 2, n + 2, dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream(dev)
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    with rb.Solver3D(n, h2, f, u0) as s:
        for _ in range(args.warmup):
            s.sweep(sweeps)
        torch.cuda.synchronize(dev)
        with ClockSampler(str(uuid) if uuid else None) as clocks:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(args.steps):
                s.sweep(sweeps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        rho = s.residual()
    secs = e0.elapsed_time(e1) / 1e3
    lups = float(n) ** 3 * sweeps * args.steps
    alu, alu_src, hbm, hbm_src = device_peaks(dev)
    per_half = secs / (2 * sweeps * args.steps)
    alg = 24.0 * n ** 3 / 2
    line = {"metric": "GLUP/s (3D 7-point red-black sweeps)", "value": lups / secs / 1e9, "unit": "GLUP/s",
            "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 f ~ U(-1,1))",
            "config": {"workload": f"3D RBGS, {n}^3 interior, zero shell, f~U(-1,1) seed 1, u0=0, {sweeps} sweeps",
                       "update": "six correctly rounded adds + one correctly rounded division by 6 (bit-exact)"},
            "final_rho": rho,
            "roofline": {"bound": "alu", "kernel": "half_sweep3_kernel", "launch_ms": 1e3 * per_half,
                         "hbm": {"achieved": alg / per_half / 1e9, "peak": hbm, "unit": "GB/s",
                                 "frac": alg / per_half / 1e9 / hbm, "peak_source": hbm_src},
                         "achieved": 6.0 * n ** 3 / 2 / per_half / 1e12, "peak": alu, "unit": "TFLOP/s",
                         "frac": 6.0 * n ** 3 / 2 / per_half / 1e12 / alu, "peak_source": alu_src,
                         "note": "achieved counts the six adds per update only; the division by 6 runs on "
                                 "the FP64 pipe too, so the pipe's true load is higher"},
            "clocks": clocks.summary(), "gpu_launches": 2 * sweeps * args.steps}
    print(json.dumps(line))
    return 0


def run_mixed(args):
    """The mixed-precision workload: N^2 interior (default 8192), f = the |k|^-3 Gaussian
    random field from stream 2 (unit RMS), ring g = x^2 - y^2, u0 = 0, target rho <= tol
    (default 1e-10).  Reaching it takes ~1.6e8 sweeps at 8192^2, so both forms (plain FP64;
    FP32 sweeps + FP64 defect correction with 100 inner sweeps) run `mixed_cap` sweeps in
    chunks of `mixed_chunk` (rbgs_solve with max_sweeps = chunk, which includes its residual
    checks), timed with CUDA events; the time to tol is then extrapolated two ways from the
    measured cost per sweep: with the residual ratio of the last chunk, and with the
    asymptotic RBGS rate cos^2(pi h) (the slowest mode), which bounds the sweep count from
    above.  Both are labelled as extrapolations."""
    import math

    import torch

    import paper_2607_01735_gb300 as rb
    import synth

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    n, cap, chunk, tol = args.mixed_n, args.mixed_cap, args.mixed_chunk, args.mixed_tol
    h2 = synth.h_squared(n)
    f_np, _ = synth.grf_rhs(n, 2)
    f = torch.from_numpy(f_np).to(dev)
    u = torch.from_numpy(synth.ring_grid(n, synth.g_quadratic)).to(dev)
    del f_np
    mu2 = math.cos(math.pi / (n + 1)) ** 2
    stream = torch.cuda.current_stream(dev)
    forms = {}
    uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
    with ClockSampler(str(uuid) if uuid else None) as clocks:
        for name, kw in (("plain_fp64", dict(check_every=100)),
                         ("plain_fp64_fused", dict(check_every=100, fma=1)),
                         ("fp32_refine", dict(precision=rb.RBGS_FP32_REFINE, inner_sweeps=100))):
            with rb.Solver(n, h2, f, u, max_sweeps=chunk, **kw) as sol:
                rho0 = sol.residual()
                hist, secs, done = [(0, rho0)], 0.0, 0
                while done < cap:
                    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    sweeps, rho, st = sol.solve(tol, allow_not_converged=True)
                    e1.record(stream)
                    torch.cuda.synchronize(dev)
                    secs += e0.elapsed_time(e1) / 1e3
                    done += sweeps
                    hist.append((done, rho))
                    if st == rb.RBGS_OK or sweeps == 0:
                        break
            per = secs / max(done, 1)
            (s1, r1), (s2, r2) = hist[-2], hist[-1]
            tail = (r2 / r1) ** (1.0 / (s2 - s1)) if s2 > s1 and r1 > 0 and r2 > 0 else float("nan")
            est = {}
            for label, rate in (("tail_rate", tail), ("asymptotic_rate", mu2)):
                more = math.log(tol / r2) / math.log(rate) if r2 > tol and 0 < rate < 1 else 0.0
                est[label] = {"sweeps": done + more, "seconds": secs + more * per, "rate": rate}
            forms[name] = {"measured_sweeps": done, "measured_seconds": secs, "ms_per_sweep": 1e3 * per,
                           "glups": n * n / per / 1e9, "rho0": rho0, "rho": r2,
                           "history": [[a, b] for a, b in hist], "extrapolated": est}
    p_est = forms["plain_fp64"]["extrapolated"]["asymptotic_rate"]["seconds"]
    r_est = forms["fp32_refine"]["extrapolated"]["asymptotic_rate"]["seconds"]
    line = {"metric": f"seconds to relative residual {tol:g} (extrapolated from {cap} measured sweeps)",
            "value": r_est, "unit": "s", "n_gpus": 1, "steps": 1, "warmup": 0,
            "ms_per_step": 1e3 * forms["fp32_refine"]["measured_seconds"], "higher_is_better": False,
            "scaling": "strong", "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
            "config": {"workload": f"{n}x{n}, f = |k|^-3 GRF stream 2 (unit RMS), ring x^2-y^2, u0=0; "
                                   f"FP32 sweeps + FP64 refinement (100 inner) vs plain FP64",
                       "extrapolation": "measured cost per sweep x sweeps needed at the asymptotic "
                                        "rate cos^2(pi h) after the measured sweeps"},
            "speedup_vs_plain_fp64": p_est / r_est,
            "speedup_vs_plain_fp64_fused": forms["plain_fp64_fused"]["extrapolated"]["asymptotic_rate"]["seconds"] / r_est,
            "forms": forms, "clocks": clocks.summary()}
    alu, alu_src, hbm, hbm_src = device_peaks(dev)
    r_bytes = 3.0 * 1e9 * forms["fp32_refine"]["glups"] / 1e9  # 12 B per point per 4-sweep pass
    line["roofline"] = {"bound": "hbm", "achieved": r_bytes, "peak": hbm, "unit": "GB/s", "frac": r_bytes / hbm,
                        "traffic": None, "kernel": "wavefront_kernel<float, 4> (the refined form's inner sweeps)",
                        "peak_source": hbm_src,
                        "note": "algorithmic bytes of the FP32 passes (3 B per update) over the refined form's "
                                "whole time, FP64 defect and correction included",
                        "plain_fp64": {"bound": "alu", "achieved": 4.0 * forms["plain_fp64"]["glups"] / 1e3,
                                       "peak": alu, "unit": "TFLOP/s",
                                       "frac": 4.0 * forms["plain_fp64"]["glups"] / 1e3 / alu,
                                       "peak_source": alu_src}}
    print(json.dumps(line))
    return 0


# The learned guess's convolution layers: (Cin, Cout, ksize, level); level l runs at
# (H / 2^l) x (W / 2^l).  The same table as the network in csrc/unet.cu.
UNET_LAYERS = ((16, 32, 3, 0), (32, 32, 3, 0), (32, 64, 3, 1), (64, 64, 3, 1), (64, 128, 3, 2),
               (128, 128, 3, 2), (128, 256, 3, 3), (256, 256, 3, 3), (384, 128, 3, 2), (128, 128, 3, 2),
               (192, 64, 3, 1), (64, 64, 3, 1), (96, 32, 3, 0), (32, 32, 3, 0), (32, 8, 1, 0))


def run_conv(args):
    """The learned initial guess's convolutions on the tensor cores: for every layer of the
    U-Net at one training batch (conv_batch x conv_hw^2 at level 0), the forward product
    (bias, ReLU, bf16 out), the data gradient (not for the input layer) and the weight and
    bias gradients, through rbgs_conv_forward / rbgs_conv_backward.  A step is one pass over
    the selected layers and products; value = their FLOP / step time.  Each product is one
    tcgen05 kernel launch (the data gradient adds a small weight transpose; the bias
    gradient is a separate call), timed with events on the stream; the roofline entry is
    the product that takes the most time."""
    import torch

    import paper_2607_01735_gb300 as rb
    from paper_2607_01735_gb300 import unet as un

    rank, world, local = dist_env()
    if rank != 0:
        return 0
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rb.load_library()
    stream = torch.cuda.current_stream(dev)
    gen = torch.Generator(device=dev)
    gen.manual_seed(20260701)
    B, hw = args.conv_batch, args.conv_hw
    idx = range(len(UNET_LAYERS)) if args.conv_layer < 0 else [args.conv_layer]
    ops = ("fwd", "dgrad", "wgrad") if args.conv_op == "all" else (args.conv_op,)
    layers = []
    for i in idx:
        cin, cout, k, lev = UNET_LAYERS[i]
        H = W = hw >> lev
        x = (torch.randn(B, H, W, cin, generator=gen, device=dev) * 0.5).to(torch.bfloat16)
        w = (torch.randn(cout, k, k, cin, generator=gen, device=dev) / (k * k * cin) ** 0.5).to(torch.bfloat16)
        g = (torch.randn(B, H, W, cout, generator=gen, device=dev) * 0.1).to(torch.bfloat16)
        layers.append(dict(i=i, shape=(B, H, W, cin, cout, k), x=x, w=w, g=g,
                           bias=torch.zeros(cout, device=dev),
                           y=torch.empty(B, H, W, cout, dtype=torch.bfloat16, device=dev),
                           dx=torch.empty(B, H, W, cin, device=dev) if i > 0 else None,
                           dw=torch.zeros(cout, k, k, cin, device=dev), db=torch.zeros(cout, device=dev),
                           flop=2.0 * B * H * W * k * k * cin * cout))

    def timed(ev, key, li, flop, fn):
        if ev is None:
            fn()
            return
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        ev.append((key, li, flop, e0, e1))

    def step(ev=None):
        for L in layers:
            li = L["i"]
            if "fwd" in ops:
                timed(ev, "fwd", li, L["flop"],
                      lambda: un.rbgs_conv_forward(L["x"], L["w"], L["bias"], L["y"], relu=True))
            if "dgrad" in ops and L["dx"] is not None:
                timed(ev, "dgrad", li, L["flop"],
                      lambda: un.rbgs_conv_backward(L["x"], L["w"], L["g"], L["dx"], None, None))
            if "wgrad" in ops:
                timed(ev, "wgrad", li, L["flop"],
                      lambda: un.rbgs_conv_backward(L["x"], L["w"], L["g"], None, L["dw"], None, accumulate=True))
                un.rbgs_conv_backward(L["x"], L["w"], L["g"], None, None, L["db"], accumulate=True)

    flop = 0.0
    for L in layers:
        flop += L["flop"] * (("fwd" in ops) + ("dgrad" in ops and L["dx"] is not None) + ("wgrad" in ops))
    engines = {"both": ("tcgen05", "mma_sync"),
               "all": ("tcgen05", "mma_sync", "tcgen05_gather", "tcgen05_ring", "tcgen05_taprow")}.get(
        args.engine, (args.engine,))
    # engine, and the tcgen05 engine's 3x3 weight-gradient kernel (the last two force one)
    engine_ids = {"tcgen05": (un.RBGS_CONV_TCGEN05, un.RBGS_WGRAD_AUTO),
                  "mma_sync": (un.RBGS_CONV_MMA_SYNC, un.RBGS_WGRAD_AUTO),
                  "tcgen05_gather": (un.RBGS_CONV_TCGEN05_GATHER, un.RBGS_WGRAD_AUTO),
                  "tcgen05_ring": (un.RBGS_CONV_TCGEN05, un.RBGS_WGRAD_RING),
                  "tcgen05_taprow": (un.RBGS_CONV_TCGEN05, un.RBGS_WGRAD_TAPROW)}
    results = {}
    clocks = None
    peaks = measured_peaks() or {}
    peak = peaks.get("bf16_tflops", 1900.0)
    peak_src = "measured bf16 burst peak (MEASURED_PEAKS.json)" if "bf16_tflops" in peaks else \
        "fallback bf16 burst peak 1.9 PFLOP/s"
    for name in engines:
        un.rbgs_conv_set_engine(engine_ids[name][0])
        un.rbgs_conv_set_wgrad_kernel(engine_ids[name][1])
        for _ in range(args.warmup):
            step()
        un.rbgs_conv_check(dev)
        torch.cuda.synchronize(dev)
        uuid = getattr(torch.cuda.get_device_properties(dev), "uuid", None)
        sampler = ClockSampler(str(uuid) if uuid else None)
        ev = []
        with sampler:
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            torch.cuda.synchronize(dev)
            e0.record(stream)
            for _ in range(args.steps):
                step(ev)
            e1.record(stream)
            torch.cuda.synchronize(dev)
        un.rbgs_conv_check(dev)
        t = e0.elapsed_time(e1) / 1e3 / args.steps
        per, per_layer = {}, {}
        for key, li, fl, a, b in ev:
            dt = a.elapsed_time(b) / 1e3
            acc = per.setdefault(key, [0.0, 0.0])
            acc[0] += fl
            acc[1] += dt
            pl = per_layer.setdefault(f"{li}:{key}", [0.0, 0.0])
            pl[0] += fl
            pl[1] += dt
        results[name] = dict(tflops=flop / t / 1e12, ms_per_step=1e3 * t,
                             products={k: {"tflops": v[0] / v[1] / 1e12, "ms_per_step": 1e3 * v[1] / args.steps}
                                       for k, v in per.items() if v[1] > 0},
                             per_layer_tflops={k: v[0] / v[1] / 1e12 for k, v in per_layer.items() if v[1] > 0})
        if name == engines[0]:
            clocks = sampler.summary()
    un.rbgs_conv_set_engine(un.RBGS_CONV_TCGEN05)
    un.rbgs_conv_set_wgrad_kernel(un.RBGS_WGRAD_AUTO)
    main_e = engines[0]
    r = results[main_e]
    # dominant product: the one taking the most time per step
    dom = max(r["products"], key=lambda k: r["products"][k]["ms_per_step"])
    achieved = r["products"][dom]["tflops"]
    line = {"metric": "TFLOP/s (U-Net convolution products: forward, data and weight gradients)",
            "value": r["tflops"], "unit": "TFLOP/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": r["ms_per_step"], "higher_is_better": True, "scaling": "strong", "vs_baseline": None,
            "dtype": "bf16 (fp32 accumulate)", "data": "synthetic",
            "config": {"workload": f"U-Net layers {list(idx)} at batch {B}, level-0 {hw}x{hw}, ops {list(ops)}",
                       "engine": main_e, "l2": "per step all layers' operands, larger than L2 at the default size"},
            "roofline": {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                         "frac": achieved / peak, "traffic": None,
                         "kernel": f"{CONV_KERNELS.get((main_e, dom), 'conv_umma_kernel')} ({dom}: the product "
                                   "taking the most time)", "peak_source": peak_src},
            "engines": results, "clocks": clocks}
    print(json.dumps(line))
    return 0


# the kernel that runs each product under each engine (3x3 layers)
CONV_KERNELS = {("tcgen05", "fwd"): "conv_umma_kernel<0>", ("tcgen05", "dgrad"): "conv_tma_kernel<1>",
                ("tcgen05", "wgrad"): "wgrad_ring_kernel / wgrad_shift_kernel / conv_umma_kernel<2> (per layer)",
                ("tcgen05_gather", "fwd"): "conv_umma_kernel<0>",
                ("tcgen05_gather", "dgrad"): "conv_umma_kernel<1>", ("tcgen05_gather", "wgrad"): "conv_umma_kernel<2>",
                ("mma_sync", "fwd"): "conv_igemm_kernel<FWD>", ("mma_sync", "dgrad"): "conv_igemm_kernel<BWD_DATA>",
                ("mma_sync", "wgrad"): "conv_igemm_kernel<BWD_WEIGHT>"}


def _solve_from(rb, n, h2, f, u0, tol, cap, chunk):
    """Mixed-precision solve from u0 in chunks of `chunk` sweeps up to `cap`; returns
    (sweeps, rho, seconds, extrapolated sweeps to tol or None)."""
    import torch
    opts = rb.default_opts(precision=rb.RBGS_FP32_REFINE, inner_sweeps=200, max_sweeps=chunk)
    t0 = time.perf_counter()
    hist = []
    done, rho = 0, None
    with rb.Solver(n, h2, f, u0, opts) as s:
        while done < cap:
            d, rho, st = s.solve(tol, allow_not_converged=True)
            done += d
            hist.append((done, rho))
            if st == rb.RBGS_OK or d == 0:
                break
    torch.cuda.synchronize()
    secs = time.perf_counter() - t0
    extra = None
    if rho > tol and len(hist) >= 2 and hist[-1][1] < hist[-2][1]:
        (s0, r0), (s1, r1) = hist[-2], hist[-1]
        rate = math.log(r1 / r0) / (s1 - s0)
        extra = int(s1 + math.log(tol / r1) / rate)
    return done, rho, secs, extra


def run_learned(args):
    """Train the U-Net on solver-generated 255^2 solutions, then solve held-out GRF
    problems at larger sizes to args.tol from u0 = 0 and from the network's guess
    (predicted at the training resolution and interpolated, and predicted at full
    resolution); reports sweeps and wall time per start."""
    import torch

    import paper_2607_01735_gb300 as rb
    import synth
    from paper_2607_01735_gb300 import learned
    from paper_2607_01735_gb300.unet import UNet
    torch.cuda.set_device(0)
    t0 = time.perf_counter()
    x, y, m = learned.make_dataset(255, range(10, 10 + args.train_samples), tol=1e-12, refine=True)
    torch.cuda.synchronize()
    t_data = time.perf_counter() - t0
    net = UNet(seed=0)
    t0 = time.perf_counter()
    losses = learned.train(net, x, y, m, steps=args.train_steps, batch=16, lr=2e-3)
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    del x, y, m
    os.makedirs(OUT_DIR, exist_ok=True)
    torch.save(net.get_params().cpu(), os.path.join(OUT_DIR, "unet_params.pt"))
    results = []
    caps = [int(v) for v in args.eval_cap.split(",")]
    starts = [v.split(",") for v in args.eval_starts.split(";")]
    plain = [int(v) for v in args.plain_fields.split(",")]
    for si, n in enumerate(int(v) for v in args.eval_sizes.split(",")):
        cap = caps[min(si, len(caps) - 1)]
        h2 = synth.h_squared(n)
        for k in range(args.eval_first, args.eval_first + args.eval_fields):
            stream = 5000 + 100 * k + n % 97
            f, u = synth.learned_guess_sample(n, stream)
            fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u).cuda()
            row = {"n": n, "stream": stream}
            if k < plain[min(si, len(plain) - 1)]:
                # u0 = 0, plain FP64 sweeps (the fused update), to the same tolerance
                t1 = time.perf_counter()
                with rb.Solver(n, h2, fd, ud, fma=1, check_every=200, max_sweeps=cap) as s:
                    sw, rho, _ = s.solve(args.tol, allow_not_converged=True)
                torch.cuda.synchronize()
                row["zero_plain_fp64_fused"] = {"sweeps": sw, "rho": rho, "solve_s": time.perf_counter() - t1,
                                                "guess_s": 0.0, "sweeps_to_tol_extrapolated": None}
            for name in starts[min(si, len(starts) - 1)]:
                t1 = time.perf_counter()
                if name == "zero":
                    u0 = ud
                elif name == "coarse":
                    u0 = learned.initial_guess_coarse(net, fd, ud, 255).contiguous()
                else:
                    u0 = learned.initial_guess(net, fd, ud).contiguous()
                torch.cuda.synchronize()
                t_guess = time.perf_counter() - t1
                sweeps, rho, secs, extra = _solve_from(rb, n, h2, fd, u0, args.tol, cap, 20000)
                row[name] = {"sweeps": sweeps, "rho": rho, "solve_s": secs, "guess_s": t_guess,
                             "sweeps_to_tol_extrapolated": extra}
            results.append(row)
            # each field as it completes, so that a long evaluation leaves its partial results
            print(json.dumps({"learned_field": row}), file=sys.stderr, flush=True)
    line = {"metric": "sweeps and wall time to relative residual %.0e from the learned guess vs u0=0" % args.tol,
            "value": None, "unit": "sweeps", "n_gpus": 1, "higher_is_better": False, "data": "synthetic",
            "config": {"workload": f"U-Net (4 levels, 32 base channels, bf16 weights, fp32 accum) trained on "
                                   f"{args.train_samples} RBGS solutions at 255^2 (GRF |k|^-3, linear boundary), "
                                   f"{args.train_steps} Adam steps; held-out GRF fields at {args.eval_sizes}; "
                                   f"solver: FP32 sweeps + FP64 refinement"},
            "train": {"data_s": t_data, "train_s": t_train, "loss_first": losses[0], "loss_last": losses[-1],
                      "loss_min": min(losses)},
            "results": results}
    print(json.dumps(line))
    return 0


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    if args.mode == "batched":
        return run_batched(args)
    if args.mode == "learned":
        return run_learned(args)
    if args.mode == "conv":
        return run_conv(args)
    if args.mode == "mixed":
        return run_mixed(args)
    if args.mode == "3d":
        return run_3d(args)
    import torch
    import torch.distributed as dist

    import paper_2607_01735_gb300 as rb
    import synth

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    if world > 1:
        dist.init_process_group("nccl")
    dev = torch.device("cuda", local)
    n, sweeps = args.n, args.sweeps
    h2 = synth.h_squared(n)
    f = synth.uniform_pm1_grid(n, 1, device=dev)
    u0 = torch.zeros(n + 2, n + 2, dtype=torch.float64, device=dev)
    out = torch.empty_like(u0)
    refine = args.precision == "refine"
    # FP64 update forms to time: both by default (the fused form is the headline, the
    # bit-exact one beside it, measured in the same run), or the one --fma names
    modes = [0] if refine else ([args.fma] if args.fma >= 0 else [1, 0])
    lib = rb.load_library()
    stream = torch.cuda.current_stream(dev)
    props = torch.cuda.get_device_properties(dev)
    uuid = getattr(props, "uuid", None)

    def barrier():
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
            torch.cuda.synchronize(dev)

    def measure(fma):
        """Time args.steps whole steps of one FP64 update form on one context; returns the
        figures and the context (destroyed by the caller)."""
        margs = argparse.Namespace(**vars(args))
        margs.fma = fma
        opts = rb.default_opts(fp64_emulate=args.emulate, tile_rows=args.tile_rows, kernel=args.kernel,
                               sweep_values=args.values, sweep_rows=args.rows, int_rows=args.int_rows,
                               tblock_k=args.tblock_k,
                               precision=rb.RBGS_FP32_REFINE if refine else rb.RBGS_FP64,
                               inner_sweeps=args.inner, max_sweeps=sweeps, fma=fma)
        sweep_events = []

        # The solver context (device buffers) is allocated once, before timing; every step
        # loads its problem into it (the layout/staging step: copies and packing), sweeps,
        # computes the residual and reads the solution back.
        def run_sweeps(ctx, record=False):
            if record:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
            if refine:
                rb.rbgs_solve(ctx, 0.0, allow_not_converged=True)
            else:
                rb.rbgs_sweep(ctx, sweeps)
            if record:
                e1.record(stream)
                sweep_events.append((e0, e1))

        ctx = rb.rbgs_create(n, h2, f, u0, opts, stream=stream.cuda_stream)

        def step(fi, ui, uo, record=False):
            rb.rbgs_set_problem(ctx, fi, ui)
            run_sweeps(ctx, record)
            rho = rb.rbgs_residual(ctx)
            rb.rbgs_get_solution(ctx, uo)
            return rho

        kernel, kdepth = resolved_kernel(n, refine, args.kernel, args.tblock_k)
        if fma:
            kernel, kdepth = 1, 1
        blocked = kernel in (2, 3)  # several sweeps per launch (TMA tiles or register wavefront)
        persistent = uses_persistent(margs, n, refine)
        # pack f, pack u, ||b|| (2), the sweeps, residual, unpack.  The residual after
        # bit-exact FP64 sweeps walks the red points only (2 launches: the black rt is exactly
        # zero), else both colours (3)
        resid = 2 if sweeps > 0 and not fma else 3
        if fma:  # + max |h2 f| at load; per block of <= 1024 sweeps: max |u|, h2 f onto the grid
            launches_per_step = 4 + 1 + 2 * -(-sweeps // 1024) + 2 * sweeps + resid + 1
        elif refine:
            inner = args.inner or 100
            outer = -(-sweeps // inner)
            per_outer = 4 + 1 + 3 + (inner // kdepth + 2 * (inner % kdepth) if blocked else 2 * inner)
            launches_per_step = 4 + 4 + outer * per_outer + 3 + 1
        elif blocked:
            launches_per_step = 4 + sweeps // kdepth + 2 * (sweeps % kdepth) + resid + 1
        elif persistent:  # one cooperative launch runs all the sweeps (up to 2^20 per launch)
            launches_per_step = 4 + -(-sweeps // (1 << 20)) + resid + 1
        else:
            launches_per_step = 4 + 2 * sweeps + resid + 1

        for _ in range(args.warmup):
            step(f, u0, out)
        barrier()
        with ClockSampler(str(uuid) if uuid else None) as clocks:
            t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            t0.record(stream)
            marks = []
            for _ in range(args.steps):
                rho = step(f, u0, out, record=True)
                marks.append(torch.cuda.Event(enable_timing=True))
                marks[-1].record(stream)
            t1.record(stream)
            barrier()
        elapsed = t0.elapsed_time(t1) / 1e3
        step_ms = [a.elapsed_time(b) for a, b in zip([t0] + marks[:-1], marks)]
        sweep_ms = [a.elapsed_time(b) for a, b in sweep_events]
        if world > 1:
            tt = torch.tensor([elapsed], dtype=torch.float64, device=dev)
            dist.all_reduce(tt, op=dist.ReduceOp.MAX)
            elapsed = float(tt.item())
        lups = float(n) * n * sweeps * args.steps * world
        sweep_s = sum(a.elapsed_time(b) for a, b in sweep_events) / 1e3
        peaks = measured_peaks()
        peak_hbm = peaks["hbm_gbs"] if peaks else 6800.0
        hbm_src = "measured (MEASURED_PEAKS.json hbm_gbs)" if peaks else "fallback 6.8 TB/s"
        sm_count = props.multi_processor_count
        sm_mhz = float(peaks.get("sm_max_mhz", 2070.0)) if peaks else 2070.0
        names = {2: "temporal_tile", 3: "wavefront_kernel"}
        if refine:
            # dominant kernel: the FP32 inner sweeps (12 algorithmic bytes per update for one
            # launch per colour; a blocked pass moves the same bytes for kdepth sweeps)
            kname = f"{names[kernel]}<float, {kdepth}>" if blocked else "half_sweep_f32"
            if blocked:  # one pass: kdepth sweeps of every point, the iterate and h2f moved once
                launches = max(sweeps // kdepth, 1)
                alg_bytes = 12.0 * n * n
            else:  # one half-sweep: half the points
                launches = 2 * sweeps
                alg_bytes = 12 * n * n / 2.0
            launch_s = sweep_s / (launches * args.steps)
            achieved = alg_bytes / launch_s / 1e9
            roofline = {"bound": "hbm", "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
                        "frac": achieved / peak_hbm, "traffic": None, "kernel": kname, "peak_source": hbm_src,
                        "launch_ms": 1e3 * launch_s, "algorithmic_bytes_per_launch": alg_bytes,
                        "note": "per launch equivalent (a half-sweep, or a blocked pass), including the "
                                "FP64 defect/correction passes in the time"}
        elif fma:
            # dominant kernel: the fused half-sweep (integer arithmetic only), bound by HBM: 24
            # algorithmic bytes per update (h2 f on the fixed-point grid, the other colour, the
            # own colour written).  Per launch: half the points; the time includes the
            # rescaling passes of each block of sweeps (max |u|, h2 f onto the grid).
            launches = 2 * sweeps
            kname = "fused_half_sweep"
            launch_s = sweep_s / (launches * args.steps)
            alg_bytes = BYTES_PER_LUP * n * n / 2.0
            achieved = alg_bytes / launch_s / 1e9
            roofline = {"bound": "hbm", "achieved": achieved, "peak": peak_hbm, "unit": "GB/s",
                        "frac": achieved / peak_hbm, "traffic": profiled_traffic(kname, args.emulate),
                        "kernel": kname, "peak_source": hbm_src, "launch_ms": 1e3 * launch_s,
                        "algorithmic_bytes_per_launch": alg_bytes,
                        "note": "per half-sweep; the sweeps' device time includes the per-block rescaling "
                                "passes (max |u|, h2 f onto the fixed-point grid)"}
        else:
            # dominant kernel: the FP64 half-sweep, bound by the FP64 pipe: 4 correctly rounded
            # adds per update (the x0.25 runs on the integer pipe).  Peak: 2 FP64 instructions
            # per clock per SM (ncu's DFMA peak_sustained) x SMs x maximum SM clock.
            # (the persistent kernel: per half-sweep equivalent, its launch time / (2 sweeps))
            launches = (sweeps // kdepth) if blocked else 2 * sweeps
            kname = (f"{names[kernel]}<double, {kdepth}>" if blocked
                     else "persistent_sweeps<double>" if persistent else "half_sweep_f64")
            per_launch_lups = n * n * sweeps / launches
            launch_s = sweep_s / (launches * args.steps)
            achieved = 4 * per_launch_lups / launch_s / 1e12
            peak_alu = 2.0 * sm_count * sm_mhz * 1e6 / 1e12
            alg_bytes = BYTES_PER_LUP * per_launch_lups
            hbm_achieved = alg_bytes / launch_s / 1e9
            traffic = None if blocked else profiled_traffic(kname, args.emulate)
            roofline = {"bound": "alu", "achieved": achieved, "peak": peak_alu, "unit": "TFLOP/s",
                        "frac": achieved / peak_alu, "traffic": traffic, "kernel": kname,
                        "peak_source": f"FP64 pipe: 2 instr/clk/SM x {sm_count} SMs x {sm_mhz:.0f} MHz "
                                       "(one flop = one correctly rounded FP64 add)",
                        "launch_ms": 1e3 * launch_s, "algorithmic_bytes_per_launch": alg_bytes,
                        "hbm": {"achieved": hbm_achieved, "peak": peak_hbm, "unit": "GB/s",
                                "frac": hbm_achieved / peak_hbm, "peak_source": hbm_src}}
            if persistent:
                roofline["note"] = ("one cooperative launch runs all sweeps; launch_ms, traffic and the "
                                    "algorithmic bytes are per half-sweep equivalent (the launch / 2 sweeps)")
        kdesc = ("all sweeps in one cooperative launch (grid barrier between colours)" if persistent
                 else {1: "one launch per colour", 2: "temporal (TMA tiles)", 3: "register wavefront"}[kernel])
        return {"ctx": ctx, "step": step, "value": lups / elapsed / 1e9, "elapsed": elapsed, "lups": lups,
                "step_ms": step_ms, "sweep_ms": sweep_ms, "roofline": roofline, "clocks": clocks.summary(),
                "rho": rho, "launches": launches_per_step * args.steps, "kernel": kdesc,
                "blocked": blocked, "kdepth": kdepth}

    results = {}
    for fma in modes:
        results[fma] = measure(fma)
        if fma != modes[0]:
            rb.rbgs_destroy(results[fma].pop("ctx"))
    head = results[modes[0]]
    ctx_a, step, lups, elapsed = head["ctx"], head["step"], head["lups"], head["elapsed"]
    value = head["value"]

    e2e = None
    if not args.no_e2e:
        # End to end from pinned host memory through the library's host path: every step
        # copies its f and u0 in from page-locked host buffers, sweeps, and copies the
        # solution and rho out.  rbgs_run_stream runs the steps as a stream of problems, its
        # own copy streams moving the next step's inputs and the last step's solution while
        # the current step sweeps.  The serial figure beside it passes the host buffers to
        # rbgs_set_problem / rbgs_get_solution one step after another, nothing overlapped.
        # (The refinement runs the serial form only.)
        fh = f.cpu().pin_memory()
        uh = u0.cpu().pin_memory()
        oh = torch.empty(n + 2, n + 2, dtype=torch.float64).pin_memory()

        def streamed(k):
            rb.rbgs_run_stream(ctx_a, [fh] * k, [uh] * k, sweeps, [oh] * k)

        def timed(body):
            with ClockSampler(str(uuid) if uuid else None) as clk:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                body()
                e1.record(stream)
                barrier()
            et = e0.elapsed_time(e1) / 1e3
            if world > 1:
                tt = torch.tensor([et], dtype=torch.float64, device=dev)
                dist.all_reduce(tt, op=dist.ReduceOp.MAX)
                et = float(tt.item())
            return et, clk.summary()

        step(fh, uh, oh)  # warm the host path
        if not refine:
            streamed(2)
        barrier()
        et_serial, serial_clocks = timed(lambda: [step(fh, uh, oh) for _ in range(args.steps)])
        if refine:
            et, e2e_clocks, how = et_serial, serial_clocks, "serial host calls (the refinement)"
        else:
            et, e2e_clocks = timed(lambda: streamed(args.steps))
            how = ("rbgs_run_stream: the library's copy streams (one per direction) move the next step's "
                   "inputs and the last step's solution through double-buffered device staging while the "
                   "current step sweeps")
        e2e = {"value": lups / et / 1e9, "unit": UNIT,
               "h2d_bytes_per_step": 8 * (n * n + (n + 2) * (n + 2)),
               "d2h_bytes_per_step": 8 * (n + 2) * (n + 2) + 8,
               "ms_per_step": 1e3 * et / args.steps, "clocks": e2e_clocks, "api": how,
               "serial": {"value": lups / et_serial / 1e9, "ms_per_step": 1e3 * et_serial / args.steps}}
    rb.rbgs_destroy(ctx_a)

    if rank == 0:
        cpu = None
        if not args.no_cpu_baseline:
            cpu = cpu_oracle_rate(n)
        ttr = None if args.no_ttr else time_to_residual(args.ttr_n)
        small = None if args.no_ttr else small_grid_history()
        def update_desc(fma):
            return ("fused: the five binary64 terms summed exactly in 64-bit fixed point, one rounding to "
                    "binary64 per update (<= 1e-13 relative max-norm of the bit-exact iterate)" if fma else
                    "bit-exact: four correctly rounded FP64 adds per update, the bits of the plain sequential loop")

        def med(xs):
            return {"min": min(xs), "median": statistics.median(xs), "max": max(xs)}

        hm = modes[0]
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded SplitMix64 f ~ U(-1,1))",
            "config": {"workload": workload(n, sweeps, args.precision), "n": n, "sweeps": sweeps,
                       "kernel": head["kernel"], "update": update_desc(hm),
                       "tblock_k": head["kdepth"] if head["blocked"] else None, "precision": args.precision,
                       "fp64_emulate": args.emulate, "tile_rows": args.tile_rows or "auto",
                       "sweep_values": args.values or "auto", "sweep_rows": args.rows or "auto",
                       "int_rows": args.int_rows,
                       "l2": "inputs larger than L2 (4 colour arrays of 1.08 GB each)",
                       "parallelism": f"replicas x{world}"},
            "hbm_gbs_algorithmic": BYTES_PER_LUP * lups / elapsed / 1e9,
            "final_rho": head["rho"],
            "roofline": head["roofline"],
            "cpu_baseline": cpu,
            "e2e": e2e,
            "gpu_launches": head["launches"],
            "clocks": head["clocks"],
            "time_to_residual": ttr,
            "small_grid": small,
            "step_ms": med(head["step_ms"]),
            "sweeps_ms": dict(med(head["sweep_ms"]), note="device time of the sweeps alone in each step"),
        }
        for fma in modes[1:]:  # the other update form, same workload, same run
            r = results[fma]
            line["bit_exact" if fma == 0 else "fused"] = {
                "value": r["value"], "unit": UNIT, "ms_per_step": 1e3 * r["elapsed"] / args.steps,
                "update": update_desc(fma), "kernel": r["kernel"], "roofline": r["roofline"],
                "hbm_gbs_algorithmic": BYTES_PER_LUP * r["lups"] / r["elapsed"] / 1e9,
                "final_rho": r["rho"], "gpu_launches": r["launches"], "clocks": r["clocks"],
                "step_ms": med(r["step_ms"])}
        print(json.dumps(line))
    if world > 1:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
