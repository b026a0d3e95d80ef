"""Sharding of independent problems across ranks (one process per GPU).

Independent Poisson problems need no data exchange: each rank solves its own subset
with one rbgs_solve_batched call and only the per-problem results are gathered.  The
split balances estimated work.  The work of one problem to a relative residual tol is
about N^2 updates per sweep times the sweep count, and the sweep count follows from the
slowest mode's contraction per sweep, cos^2(pi h) (the model-problem rate of red-black
Gauss-Seidel): log(1/tol) / -log(cos^2(pi/(N+1))).  Problems are assigned
largest-first to the least-loaded rank (longest-processing-time order).
"""
from __future__ import annotations

import math


def estimated_work(n: int, tol: float = 1e-8) -> float:
    """Lattice-site updates to reach `tol` on an n x n interior (model-problem rate)."""
    h = 1.0 / (n + 1)
    rate = -math.log(math.cos(math.pi * h) ** 2)
    sweeps = math.log(1.0 / max(tol, 1e-300)) / rate if rate > 0 else 1.0
    return float(n) * n * max(sweeps, 1.0)


def shard(sizes: list[int], world: int, tol: float = 1e-8) -> list[list[int]]:
    """Problem indices per rank, balanced by estimated work (deterministic)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    order = sorted(range(len(sizes)), key=lambda p: (-sizes[p], p))
    load = [0.0] * world
    parts: list[list[int]] = [[] for _ in range(world)]
    for p in order:
        r = min(range(world), key=lambda k: (load[k], k))
        parts[r].append(p)
        load[r] += estimated_work(sizes[p], tol)
    for part in parts:
        part.sort()
    return parts


def gather_results(local: dict[int, dict], world: int, group=None) -> dict[int, dict]:
    """All-gather per-problem result dicts (keyed by global problem index) to every rank."""
    import torch.distributed as dist
    if world == 1:
        return dict(local)
    bucket: list = [None] * world
    dist.all_gather_object(bucket, local, group=group)
    merged: dict[int, dict] = {}
    for part in bucket:
        merged.update(part)
    return merged


def max_over_ranks(value: float, world: int, device=None, group=None) -> float:
    """The largest of one float per rank (the slowest rank's time)."""
    import torch
    import torch.distributed as dist
    if world == 1:
        return value
    t = torch.tensor([value], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX, group=group)
    return float(t.item())
