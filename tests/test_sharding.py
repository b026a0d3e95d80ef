"""The multi-process path on CPU: work-balanced sharding of independent problems and the
result gather / max-over-ranks timing with a world_size-2 gloo process group."""
import os
import socket

import pytest
import torch.multiprocessing as mp

from paper_2607_01735_gb300 import sharding


def test_estimated_work_follows_the_model_rate():
    # doubling N: 4x the points per sweep, ~4x the sweeps (rate ~ (pi h)^2)
    r = sharding.estimated_work(511) / sharding.estimated_work(255)
    assert 15.0 < r < 17.0


def test_shard_covers_every_problem_once_and_balances():
    sizes = [63, 127, 255, 511, 1023] * 20 + [1023, 63]
    for world in (1, 2, 3, 8):
        parts = sharding.shard(sizes, world)
        flat = sorted(p for part in parts for p in part)
        assert flat == list(range(len(sizes)))
        loads = [sum(sharding.estimated_work(sizes[p]) for p in part) for part in parts]
        biggest = max(sharding.estimated_work(n) for n in sizes)
        assert max(loads) - min(loads) <= biggest + 1e-6 * max(loads)
    assert sharding.shard(sizes, 4) == sharding.shard(sizes, 4)  # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, sizes, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    mine = sharding.shard(sizes, world)[rank]
    local = {p: {"rank": rank, "n": sizes[p]} for p in mine}
    merged = sharding.gather_results(local, world)
    slowest = sharding.max_over_ranks(float(rank + 1) * 0.5, world)
    out.put((rank, sorted(merged), {k: v["rank"] for k, v in merged.items()}, slowest))
    dist.barrier()
    dist.destroy_process_group()


def test_gloo_two_ranks_gather_and_max():
    sizes = [63, 127, 255, 511, 1023, 63, 127]
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, sizes, out)) for r in range(2)]
    for p in procs:
        p.start()
    got = [out.get(timeout=120) for _ in range(2)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    parts = sharding.shard(sizes, 2)
    for rank, keys, owner, slowest in got:
        assert keys == list(range(len(sizes)))
        assert all(owner[p] == r for r in range(2) for p in parts[r])
        assert slowest == 1.0
