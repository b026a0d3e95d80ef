"""GPU parity of the 3D variant (include/rbgs3d.h; the 7-point red-black scheme of the
paper's 3D outlook, Section 5) through the C ABI: the iterate bit for bit against
oracle.sweeps3d after the same sweeps (six correctly rounded adds and one correctly rounded
division per update, in the oracle's order), rho against the oracle's residual, and the
manufactured problem's closed-form residual history."""
import math

import numpy as np
import pytest
import torch

import oracle
import paper_2607_01735_gb300 as rb

from test_oracle_3d import _closed_form_rho, _manufactured, _random3

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_01735_gb300 import build
    build.build_library()
    rb.load_library()


def _bits(got, ref):
    bad = np.argwhere(got.view(np.uint64) != ref.view(np.uint64))
    assert bad.size == 0, f"{len(bad)} values differ; first at {tuple(bad[0])}: {got[tuple(bad[0])]} vs {ref[tuple(bad[0])]}"


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 8, 17, 31, 32, 33, 64, 100])
def test_3d_bit_exact_against_oracle(n):
    f, u0 = _random3(n, 40 + n)
    h2 = 1.0 / (n + 1) ** 2
    sweeps = 6
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver3D(n, h2, fd, ud) as s:
        s.sweep(sweeps)
        s.get_solution(out)
        rho = s.residual()
    ref = u0.copy()
    oracle.sweeps3d(ref, f, h2, sweeps)
    _bits(out.cpu().numpy(), ref)
    want = oracle.residual3d(ref, f, h2)[0]
    assert abs(rho - want) <= max(1e-12, n ** 3 * 2.0 ** -53) * want


def test_3d_host_buffers_and_manufactured_history():
    n = 31
    f, phi, h = _manufactured(n)
    h2 = h * h
    u0 = np.zeros((n + 2, n + 2, n + 2))
    out = np.empty_like(u0)
    with rb.Solver3D(n, h2, f, u0) as s:
        assert s.residual() == 1.0  # u0 = 0: rt = h^2 b at every point
        done = 0
        for k in (1, 5, 40):
            s.sweep(k - done)
            done = k
            rho = s.residual()
            want = _closed_form_rho(n, k, phi, h)
            assert abs(rho - want) <= 1e-11 * want, (k, rho, want)
        s.get_solution(out)
    ref = u0.copy()
    oracle.sweeps3d(ref, f, h2, 40)
    _bits(out, ref)
