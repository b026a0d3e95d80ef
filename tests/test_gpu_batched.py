"""GPU parity for rbgs_solve_batched: many uneven problems in one persistent launch.

Every problem's solution must equal the oracle's single-problem solve with the same
options bit for bit (FP64: residual check every check_every sweeps; FP32 refinement:
inner sweeps per correction), with the same sweep count, whatever launch shape the
autotuner or the caller picks.  Where the oracle's rho and the GPU's rho (different
summation order) straddle the tolerance the sweep counts may legitimately differ by one
check interval; the test inputs keep clear of that, and the check is still that the
rho values agree to 1e-12.
"""
import numpy as np
import pytest
import torch

import oracle
import paper_2607_01735_gb300 as rb
import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_01735_gb300 import build
    build.build_library()
    rb.load_library()


def _batch(sizes, seed):
    out = []
    for p, n in enumerate(sizes):
        f = synth.uniform_pm1_grid(n, seed * 1000 + p).numpy().copy()
        c = float(synth.uniform01(seed * 1000 + 500 + p, 1).numpy()[0] * 2 - 1)
        u = np.zeros((n + 2, n + 2))
        u[0, :] = u[-1, :] = u[:, 0] = u[:, -1] = c
        out.append((n, synth.h_squared(n), f, u))
    return out


def _assert_bits(got, ref):
    if not np.array_equal(got.view(np.uint64), ref.view(np.uint64)):
        bad = np.argwhere(got.view(np.uint64) != ref.view(np.uint64))
        raise AssertionError(f"{len(bad)} values differ; first at {tuple(bad[0])}")


def _run(batch, tol, device=True, **opts):
    o = rb.default_opts(**opts)
    if device:
        probs = [(n, h2, torch.from_numpy(f).cuda(), torch.from_numpy(u).cuda()) for n, h2, f, u in batch]
        outs = [torch.empty((n + 2, n + 2), dtype=torch.float64, device="cuda") for n, _, _, _ in batch]
    else:
        probs = [(n, h2, f, u) for n, h2, f, u in batch]
        outs = [np.empty((n + 2, n + 2)) for n, _, _, _ in batch]
    res = rb.rbgs_solve_batched(probs, tol, outs, o, allow_failures=True)
    outs = [x.cpu().numpy() if isinstance(x, torch.Tensor) else x for x in outs]
    return res, outs


SIZES = [1, 2, 5, 31, 33, 63, 64, 100, 127, 40, 7, 63]


@pytest.mark.parametrize("shape", [(0, 0), (256, 2), (512, 1), (1024, 1)])
def test_batched_fp64_matches_oracle(shape):
    batch = _batch(SIZES, 3)
    threads, per_sm = shape
    res, outs = _run(batch, 1e-8, check_every=25, tile_rows=threads, tblock_k=per_sm)
    for (n, h2, f, u0), r, got in zip(batch, res, outs):
        ref = u0.copy()
        done, rho = oracle.solve(ref, f, h2, 1e-8, 25, 10 ** 7)
        assert r["status"] == rb.RBGS_OK
        assert r["sweeps"] == done, (n, r["sweeps"], done)
        assert abs(r["rel"] - rho) <= 1e-12 * max(rho, 1e-300)
        _assert_bits(got, ref)
        assert r["latency_ms"] >= 0.0


def test_batched_refinement_matches_oracle():
    batch = _batch([63, 31, 100, 5, 127], 4)
    res, outs = _run(batch, 1e-9, precision=rb.RBGS_FP32_REFINE, inner_sweeps=40)
    for (n, h2, f, u0), r, got in zip(batch, res, outs):
        ref = u0.copy()
        done, rho, _ = oracle.refine_solve(ref, f, h2, 1e-9, 40, 10 ** 7)
        assert r["status"] == rb.RBGS_OK and r["sweeps"] == done
        assert abs(r["rel"] - rho) <= 1e-12 * rho
        _assert_bits(got, ref)


def test_batched_host_buffers_and_not_converged():
    batch = _batch([20, 9, 33], 5)
    res, outs = _run(batch, 1e-14, device=False, check_every=10, max_sweeps=30)
    for (n, h2, f, u0), r, got in zip(batch, res, outs):
        ref = u0.copy()
        oracle.sweeps(ref, f, h2, 30)
        assert r["status"] == rb.RBGS_ENOTCONV and r["sweeps"] == 30
        _assert_bits(got, ref)
    with pytest.raises(rb.RbgsError) as e:
        rb.rbgs_solve_batched([(p[0], p[1], p[2], p[3]) for p in batch], 1e-14,
                              [np.empty((p[0] + 2, p[0] + 2)) for p in batch],
                              rb.default_opts(check_every=10, max_sweeps=30))
    assert e.value.status == rb.RBGS_ENOTCONV


# several problems at the largest size, so that the phased plan gives them to clusters
TEAM_SIZES = [127, 63, 127, 1, 2, 100, 127, 5, 31, 127, 64, 33]


@pytest.mark.parametrize("team", [2, 4])
def test_batched_teams_match_oracle(team):
    batch = _batch(TEAM_SIZES, 6)
    res, outs = _run(batch, 1e-8, check_every=25, team_size=team)
    shape = rb.rbgs_batched_last_shape()
    assert shape["team"] == team and shape["first"] == 0 and shape["nteam"] == 4
    for (n, h2, f, u0), r, got in zip(batch, res, outs):
        ref = u0.copy()
        done, rho = oracle.solve(ref, f, h2, 1e-8, 25, 10 ** 7)
        assert r["status"] == rb.RBGS_OK
        assert r["sweeps"] == done, (n, r["sweeps"], done)
        assert abs(r["rel"] - rho) <= 1e-12 * rho
        _assert_bits(got, ref)


@pytest.mark.parametrize("team", [2, 4])
def test_batched_teams_refinement_matches_oracle(team):
    batch = _batch([100, 31, 100, 5, 100, 63], 7)
    res, outs = _run(batch, 1e-9, precision=rb.RBGS_FP32_REFINE, inner_sweeps=40, team_size=team)
    assert rb.rbgs_batched_last_shape()["nteam"] == 3
    for (n, h2, f, u0), r, got in zip(batch, res, outs):
        ref = u0.copy()
        done, rho, _ = oracle.refine_solve(ref, f, h2, 1e-9, 40, 10 ** 7)
        assert r["status"] == rb.RBGS_OK and r["sweeps"] == done
        assert abs(r["rel"] - rho) <= 1e-12 * rho
        _assert_bits(got, ref)


def test_batched_phased_plan_full_wave_then_teams():
    """More problems at the largest size than SMs: the first phase solves a full wave of
    them one block per SM, the second gives the rest to clusters of 4 blocks."""
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    sizes = [9] * (sms + 7) + [5, 3, 8]
    batch = _batch(sizes, 8)
    res, outs = _run(batch, 1e-8, check_every=10, team_size=4)
    shape = rb.rbgs_batched_last_shape()
    assert (shape["team"], shape["first"], shape["nteam"]) == (4, sms, 7)
    for (n, h2, f, u0), r, got in zip(batch, res, outs):
        ref = u0.copy()
        done, rho = oracle.solve(ref, f, h2, 1e-8, 10, 10 ** 7)
        assert r["status"] == rb.RBGS_OK and r["sweeps"] == done
        _assert_bits(got, ref)


def test_batched_autotuner_reports_its_shape_and_rejects_bad_team():
    batch = _batch([31, 31, 17], 9)
    res, outs = _run(batch, 1e-8, check_every=25)
    shape = rb.rbgs_batched_last_shape()
    assert shape["team"] in (1, 2, 4) and shape["threads"] in (256, 512, 1024)
    with pytest.raises(rb.RbgsError) as e:
        rb.rbgs_solve_batched([(p[0], p[1], p[2], p[3]) for p in batch], 1e-8,
                              [np.empty((p[0] + 2, p[0] + 2)) for p in batch],
                              rb.default_opts(team_size=3))
    assert e.value.status == rb.RBGS_EINVAL


@pytest.mark.slow
def test_batched_512_uneven_problems_sampled():
    """512 problems with the batched workload's recipe (size index and boundary constant
    from stream 3, f from stream 3*2^16+p), sizes restricted to {63, 127} so that the
    whole batch reaches 1e-8 in seconds; 8 problems re-solved by the oracle."""
    table = synth.batched_problem_table(512, 3, sizes=(63, 127))
    batch = []
    for e in table:
        f, u, h2 = synth.batched_problem(e)
        batch.append((e["n"], h2, f, u))
    res, outs = _run(batch, 1e-8, check_every=100)
    assert all(r["status"] == rb.RBGS_OK and r["rel"] <= 1e-8 for r in res)
    lat = np.array([r["latency_ms"] for r in res])
    assert np.all(lat > 0)
    for p in [0, 1, 100, 255, 256, 400, 510, 511]:
        n, h2, f, u0 = batch[p]
        ref = u0.copy()
        done, rho = oracle.solve(ref, f, h2, 1e-8, 100, 10 ** 7)
        assert res[p]["sweeps"] == done
        _assert_bits(outs[p], ref)


@pytest.mark.parametrize("team,precision", [(0, rb.RBGS_FP64), (4, rb.RBGS_FP64), (2, rb.RBGS_FP64),
                                            (4, rb.RBGS_FP32_REFINE)])
def test_batched_full_size_mix_capped_matches_oracle(team, precision):
    """The batched workload's size mix including 511^2 and 1023^2 (problems drawn with its
    recipe, stream 3), every problem capped at 200 sweeps so that the oracle finishes:
    each ends RBGS_ENOTCONV after exactly 200 sweeps with the oracle's bits.  With a team
    size the 1023^2 problems go to thread-block clusters (phased plan)."""
    table = synth.batched_problem_table(512, 3)
    pick = [e for e in table if e["n"] == 1023][:3] + [e for e in table if e["n"] == 511][:3] + \
        [e for e in table if e["n"] == 255][:2] + [e for e in table if e["n"] in (63, 127)][:4]
    batch = []
    for e in pick:
        f, u, h2 = synth.batched_problem(e)
        batch.append((e["n"], h2, f, u))
    refine = precision == rb.RBGS_FP32_REFINE
    res, outs = _run(batch, 1e-8, check_every=50, max_sweeps=200, team_size=team, precision=precision,
                     inner_sweeps=100)
    if team:
        shape = rb.rbgs_batched_last_shape()
        assert shape["team"] == team and shape["nteam"] == 3  # the three 1023^2 problems
    for (n, h2, f, u0), r, got in zip(batch, res, outs):
        ref = u0.copy()
        if refine:
            done, rho, _ = oracle.refine_solve(ref, f, h2, 1e-8, 100, 200)
        else:
            done, rho = oracle.solve(ref, f, h2, 1e-8, 50, 200)
        assert done == 200 and r["sweeps"] == 200 and r["status"] == rb.RBGS_ENOTCONV, (n, r)
        _assert_bits(got, ref)
        # rho: the oracle adds its n^2 squares one after another; recursive summation errs by
        # at most (count - 1) 2^-53 of the sum (Higham, Accuracy and Stability of Numerical
        # Algorithms, section 4.2), which at 1023^2 exceeds 1e-12 (interior squares far below
        # the running sum's last bit are absorbed); the GPU's tree sum errs far less
        assert abs(r["rel"] - rho) <= max(1e-12, n * n * 2.0 ** -53) * rho


def test_batched_stops_problems_whose_residual_stalls():
    """tol = 0 with the refinement, whose residual settles at a rounding floor near 5e-16
    on a 9^2 grid: each problem stops with RBGS_ENOTCONV once rho has gone stall_checks
    checks without a new minimum, after the same outer steps as the oracle's loop with
    that rule, with the oracle's bits."""
    batch = _batch([9, 9, 9], 12)
    res, outs = _run(batch, 0.0, precision=rb.RBGS_FP32_REFINE, inner_sweeps=40, stall_checks=3,
                     max_sweeps=10 ** 7)
    for (n, h2, f, u0), r, got in zip(batch, res, outs):
        ref = u0.copy()
        best, since, done = oracle.residual(ref, f, h2)[0], 0, 0
        while True:
            _, rho, _ = oracle.refine_solve(ref, f, h2, 0.0, 40, 40)  # one outer step
            done += 40
            if rho < best:
                best, since = rho, 0
            else:
                since += 1
                if since >= 3:
                    break
        assert r["status"] == rb.RBGS_ENOTCONV and r["sweeps"] == done, (r, done)
        _assert_bits(got, ref)


def test_batched_time_budget_ends_the_batch():
    """A batch that would run for minutes (160 problems of 511^2 to 1e-13) with a device-time
    budget of 0.3 s: every problem ends RBGS_ETIMEOUT; the first wave (one block per SM)
    after some sweeps, the problems that would have started after the budget with none,
    their output the initial guess.  The call returns within seconds."""
    import time
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    batch = _batch([511] * (sms + 8), 13)
    t = time.perf_counter()
    res, outs = _run(batch, 1e-13, check_every=20, max_seconds=0.3, tile_rows=1024, tblock_k=1)
    wall = time.perf_counter() - t
    assert wall < 10.0
    assert all(r["status"] == rb.RBGS_ETIMEOUT for r in res)
    started = [r["sweeps"] > 0 for r in res]
    assert sum(started) >= sms and sum(started) <= sms + 8
    late = [p for p, s in enumerate(started) if not s]
    assert len(late) >= 8 - 2  # a block that finishes its check early may claim one more
    for p in late:
        _assert_bits(outs[p], batch[p][3])
    assert max(r["latency_ms"] for r in res) < 2000.0
