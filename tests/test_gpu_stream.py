"""rbgs_run_stream through the C ABI: a stream of problems of one size through one context,
with host copies overlapped inside the library.  Every solution must equal the oracle's
after the same sweeps bit for bit (bit-exact mode; the fused oracle for fma = 1), whatever
memory each buffer lives in (pageable host, page-locked host, device), and each rho must
match the oracle's residual."""
import numpy as np
import pytest
import torch

import oracle
import paper_2607_01735_gb300 as rb
import synth

from test_gpu_parity import RESID_RTOL, _assert_bits, _problem

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_01735_gb300 import build
    build.build_library()
    rb.load_library()


def _place(a, kind):
    t = torch.from_numpy(a.copy())
    if kind == "device":
        return t.cuda()
    if kind == "pinned":
        return t.pin_memory()
    return a.copy()  # pageable numpy


def _as_np(x):
    return x.cpu().numpy() if isinstance(x, torch.Tensor) else x


@pytest.mark.parametrize("fma", [0, 1])
@pytest.mark.parametrize("n", [57, 600])
def test_stream_matches_oracle_in_every_memory_kind(n, fma):
    h2 = synth.h_squared(n)
    kinds = ["pageable", "pinned", "device", "pinned", "pageable"]
    probs = [_problem(n, 200 + q) for q in range(len(kinds))]
    sweeps = 9
    fs = [_place(f, k) for (f, _), k in zip(probs, kinds)]
    us = [_place(u, k) for (_, u), k in zip(probs, kinds)]
    outs = []
    for q, k in enumerate(reversed(kinds)):  # output kinds differ from the input kinds
        z = np.zeros((n + 2, n + 2))
        outs.append(_place(z, k))
    f0, u0 = probs[0]
    with rb.Solver(n, h2, torch.from_numpy(f0).cuda(), torch.from_numpy(u0).cuda(), fma=fma) as s:
        rho = s.run_stream(fs, us, sweeps, outs)
        rho_ctx = s.residual()  # the context holds the last problem
    assert rho_ctx == rho[-1]
    for q, (f, u) in enumerate(probs):
        ref = u.copy()
        (oracle.sweeps_fused if fma else oracle.sweeps)(ref, f, h2, sweeps)
        _assert_bits(_as_np(outs[q]), ref)
        want = oracle.residual(ref, f, h2)[0]
        assert abs(rho[q] - want) <= max(RESID_RTOL, n * n * 2.0 ** -53) * want


def test_stream_with_no_sweeps_and_a_nonfinite_problem():
    n = 33
    h2 = synth.h_squared(n)
    probs = [_problem(n, 300 + q) for q in range(3)]
    probs[1][0][4, 5] = np.nan
    outs = [np.zeros((n + 2, n + 2)) for _ in probs]
    with rb.Solver(n, h2, probs[0][0], probs[0][1]) as s:
        with pytest.raises(rb.RbgsError) as e:
            s.run_stream([p[0] for p in probs], [p[1] for p in probs], 3, outs)
        assert e.value.status == rb.RBGS_ENONFINITE
        rho = s.run_stream([p[0] for p in probs], [p[1] for p in probs], 3, outs, allow_nonfinite=True)
        assert np.isfinite(rho[0]) and not np.isfinite(rho[1]) and np.isfinite(rho[2])
        for q in (0, 2):
            ref = probs[q][1].copy()
            oracle.sweeps(ref, probs[q][0], h2, 3)
            _assert_bits(outs[q], ref)
        # zero sweeps: the solution is the initial guess, rho its residual
        rho = s.run_stream([probs[0][0]], [probs[0][1]], 0, outs[:1])
        _assert_bits(outs[0], probs[0][1])
        want = oracle.residual(probs[0][1], probs[0][0], h2)[0]
        assert abs(rho[0] - want) <= RESID_RTOL * want
        assert s.run_stream([], [], 5, []) == []
