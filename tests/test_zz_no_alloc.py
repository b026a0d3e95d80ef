"""rbgs_residual_static, the allocation-free residual, against rbgs_residual.

Some callers cannot allocate device memory (a fixed budget decided at start-up, code
running inside an allocator callback, code that must not trigger the synchronisation
that cudaMalloc/cudaFree can imply).  rbgs_residual_static serves them: it takes the
caller's device buffers and uses only a static scratch array inside the library.  This
file is collected last so that a run stopping at the first failure has run everything
else; it passes alone in a fresh process and after the other tests.
"""
import numpy as np
import pytest
import torch

import paper_2607_01735_gb300 as rb
import synth

pytestmark = pytest.mark.gpu

RTOL = 1e-12  # the residual tolerance of the other parity tests


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_01735_gb300 import build
    build.build_library()
    rb.load_library()


def _case(n, stream, sweeps):
    f = synth.uniform_pm1_grid(n, stream).numpy().copy()
    u0 = synth.ring_grid(n, synth.g_quadratic)
    fd, ud = torch.from_numpy(f).cuda(), torch.from_numpy(u0).cuda()
    out = torch.empty_like(ud)
    with rb.Solver(n, synth.h_squared(n), fd, ud) as s:
        s.sweep(sweeps)
        s.get_solution(out)
        rho = s.residual()
    return fd, out, rho


def test_static_residual_matches_context_residual_twice_in_a_row():
    h = torch.empty(2, dtype=torch.float64, device="cuda")
    cases = [(257, 5, 13), (1000, 6, 4)]
    expected = []
    for k, (n, stream, sweeps) in enumerate(cases):
        fd, ud, rho = _case(n, stream, sweeps)
        rb.rbgs_residual_static(n, synth.h_squared(n), fd, ud, h[k:k + 1])
        expected.append(rho)
    torch.cuda.synchronize()
    got = h.cpu().numpy()
    for g, e in zip(got, expected):
        assert abs(g - e) <= RTOL * e, (g, e)


def test_static_residual_rejects_oversize_and_host_memory():
    out = torch.empty(1, dtype=torch.float64, device="cuda")
    f = torch.zeros(4, 4, dtype=torch.float64, device="cuda")
    u = torch.zeros(6, 6, dtype=torch.float64, device="cuda")
    with pytest.raises(rb.RbgsError) as e:
        rb.rbgs_residual_static(32769, 1e-10, f, u, out)
    assert e.value.status == rb.RBGS_EINVAL and "32768" in str(e.value)
    with pytest.raises(rb.RbgsError) as e:
        rb.rbgs_residual_static(4, 0.04, np.zeros((4, 4)), u, out)
    assert e.value.status == rb.RBGS_EINVAL
