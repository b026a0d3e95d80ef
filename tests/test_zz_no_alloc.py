"""rbgs_residual_static, the allocation-free residual, against rbgs_residual.

Some callers cannot allocate device memory (a fixed budget decided at start-up, code
running inside an allocator callback, code that must not trigger the synchronisation
that cudaMalloc/cudaFree can imply).  rbgs_residual_static serves them: it takes the
caller's device buffers and uses only a static scratch array inside the library.  This
file is collected last so that a run stopping at the first failure has run everything
else; it passes alone in a fresh process and after the other tests.
"""
import math

import numpy as np
import pytest
import torch

import oracle
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
    # the C entry point's own limit (called directly: the binding would reject the sizes)
    lib = rb.load_library()
    st = lib.rbgs_residual_static(32769, 1e-10, f.data_ptr(), u.data_ptr(), out.data_ptr(), None)
    assert st == rb.RBGS_EINVAL and "32768" in rb.rbgs_last_error()
    # host memory is refused by the library too
    fh = np.zeros((4, 4))
    st = lib.rbgs_residual_static(4, 0.04, fh.ctypes.data, u.data_ptr(), out.data_ptr(), None)
    assert st == rb.RBGS_EINVAL
    with pytest.raises(rb.RbgsError) as e:
        rb.rbgs_residual_static(4, 0.04, fh, u, out)
    assert e.value.status == rb.RBGS_EINVAL


def _random_state(n, stream):
    """f ~ U(-1,1) and a random interior iterate with a zero ring, from the input generators
    (on the GPU for speed: the integer generator gives the same bits there).  A zero ring
    keeps the squares of each sum of similar size, so that the oracle's one-after-another
    summation stays accurate (large ring terms would absorb the small interior ones)."""
    f = synth.uniform_pm1_grid(n, stream, device="cuda")
    u = synth.uniform_pm1_grid(n + 2, stream + 1, device="cuda") * 0.5
    u[0, :] = 0.0
    u[-1, :] = 0.0
    u[:, 0] = 0.0
    u[:, -1] = 0.0
    return f, u


def _resid_tol(n):
    """The oracle's sums of n^2 squares, added one after another, err by at most
    (count - 1) 2^-53 of the sum (recursive summation bound); 1e-12 where that is smaller."""
    return max(RTOL, n * n * 2.0 ** -53)


@pytest.mark.parametrize("n", [2049, 4099])
def test_static_residual_against_oracle_on_a_side_stream(n):
    """More row blocks than the final kernel has threads (n > 1024: several passes over the
    partials; 4099 ends in a block of 3 rows), on a non-default stream, twice in a row."""
    f, u = _random_state(n, 60 + n)
    h2 = synth.h_squared(n)
    expected = oracle.residual(u.cpu().numpy(), f.cpu().numpy(), h2)[0]
    side = torch.cuda.Stream()
    side.wait_stream(torch.cuda.current_stream())
    out = torch.full((2,), -1.0, dtype=torch.float64, device="cuda")
    with torch.cuda.stream(side):
        for k in range(2):
            rb.rbgs_residual_static(n, h2, f, u, out[k:k + 1], stream=side.cuda_stream)
    side.synchronize()
    got = out.cpu().numpy()
    assert got[0] == got[1]
    assert abs(got[0] - expected) <= _resid_tol(n) * expected, (got[0], expected)


def test_static_residual_of_a_nonfinite_iterate_is_nonfinite():
    n = 300
    f, u = _random_state(n, 7)
    u[17, 33] = float("nan")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rb.rbgs_residual_static(n, synth.h_squared(n), f, u, out)
    assert math.isnan(out.item())
    u[17, 33] = float("inf")
    rb.rbgs_residual_static(n, synth.h_squared(n), f, u, out)
    assert not math.isfinite(out.item())


@pytest.mark.slow
def test_static_residual_against_oracle_at_the_largest_size():
    """n = 32768 fills all 8192 scratch slots.  The oracle adds 2^30 squares one after
    another: the recursive summation bound (count - 1) 2^-53 = 1.2e-7 is the rigorous
    tolerance here."""
    n = 32768
    f, u = _random_state(n, 90)
    h2 = synth.h_squared(n)
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    rb.rbgs_residual_static(n, h2, f, u, out)
    got = out.item()
    fh, uh = f.cpu().numpy(), u.cpu().numpy()
    del f, u
    torch.cuda.empty_cache()
    expected = oracle.residual(uh, fh, h2)[0]
    assert abs(got - expected) <= _resid_tol(n) * expected, (got, expected)
