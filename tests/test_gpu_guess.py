"""The grid kernels around the learned guess's network (rbgs_guess_*, include/rbgs_unet.h)
on the GPU: the boundary interpolation the network's correction is added to, the
network's input channels, the training target, the guess and the coarse-grid path.  The
network itself is replaced by a stand-in that predicts a zero correction and records its
inputs."""
import numpy as np
import pytest
import torch

import paper_2607_01735_gb300 as rb
from paper_2607_01735_gb300 import learned
from paper_2607_01735_gb300.unet import boundary_blend, guess_target, network_input

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2607_01735_gb300 import build
    build.build_library()
    rb.load_library()


def _ring_grid(n, fn):
    g = n + 2
    t = np.linspace(0.0, 1.0, g)
    x, y = np.meshgrid(t, t, indexing="ij")
    full = fn(x, y)
    u = np.zeros((g, g))
    u[0, :], u[-1, :], u[:, 0], u[:, -1] = full[0, :], full[-1, :], full[:, 0], full[:, -1]
    return torch.from_numpy(u).cuda(), torch.from_numpy(full)


class ZeroNet:
    """Predicts a zero correction; records the inputs it was given."""

    def __init__(self):
        self.inputs = []

    def forward(self, x):
        self.inputs.append(x)
        return torch.zeros(x.shape[:3], dtype=torch.float32, device=x.device)


@pytest.mark.parametrize("fn", [lambda x, y: 0.3 - 1.2 * x + 0.7 * y,
                                lambda x, y: -0.5 + 0.25 * x + 2.0 * y - 1.5 * x * y])
def test_boundary_blend_reproduces_bilinear_data(fn):
    """The Coons patch of data that is linear in x and in y separately is that function."""
    u, full = _ring_grid(37, fn)
    got = boundary_blend(u).cpu().numpy()
    np.testing.assert_allclose(got, full.numpy(), rtol=0, atol=1e-14)


def test_boundary_blend_keeps_the_ring():
    rng = np.random.default_rng(3)
    u = torch.from_numpy(rng.uniform(-1, 1, (20, 20))).cuda()
    got = boundary_blend(u).cpu()
    u = u.cpu()
    for a, b in ((got[0], u[0]), (got[-1], u[-1]), (got[:, 0], u[:, 0]), (got[:, -1], u[:, -1])):
        np.testing.assert_allclose(a.numpy(), b.numpy(), rtol=0, atol=1e-14)


def test_network_input_channels():
    n = 13
    g = n + 2
    rng = np.random.default_rng(4)
    f = torch.from_numpy(rng.uniform(-1, 1, (n, n))).cuda()
    u = torch.from_numpy(rng.uniform(-1, 1, (g, g))).cuda()
    x = network_input(f, u).cpu()
    blend = boundary_blend(u).cpu()
    f, u = f.cpu(), u.cpu()
    size = learned.grid_size(n)
    assert x.shape == (size, size, 4) and size % 8 == 0 and size >= g
    ring = np.ones((g, g), dtype=bool)
    ring[1:-1, 1:-1] = False
    assert np.array_equal(x[:g, :g, 1].numpy() == 1.0, ring)                 # mask
    np.testing.assert_array_equal(x[1:n + 1, 1:n + 1, 0].numpy(), f.numpy().astype(np.float32))
    assert np.all(x[:g, :g, 0].numpy()[ring] == 0)                          # f only inside
    np.testing.assert_array_equal(x[:g, :g, 2].numpy()[ring], u.numpy().astype(np.float32)[ring])
    assert np.all(x[:g, :g, 2].numpy()[~ring] == 0)                         # ring values only
    np.testing.assert_array_equal(x[:g, :g, 3].numpy(), blend.numpy().astype(np.float32))
    assert np.all(x[g:].numpy() == 0) and np.all(x[:, g:].numpy() == 0)     # zero padding


def test_initial_guess_with_zero_correction_is_the_blend_inside_the_given_ring():
    n = 21
    fn = lambda x, y: 0.1 + 0.9 * x - 0.4 * y  # noqa: E731
    u, full = _ring_grid(n, fn)
    f = torch.zeros((n, n), dtype=torch.float64, device="cuda")
    net = ZeroNet()
    u0 = learned.initial_guess(net, f, u)
    np.testing.assert_allclose(u0.cpu().numpy(), full.numpy(), rtol=0, atol=1e-14)
    assert torch.equal(u0[0], u[0]) and torch.equal(u0[:, -1], u[:, -1])    # ring kept bit for bit
    assert net.inputs[0].shape == (1, learned.grid_size(n), learned.grid_size(n), 4)


def test_coarse_guess_interpolates_and_keeps_the_fine_ring():
    """Predicting on a coarse grid whose nodes coincide with fine nodes: with a zero
    correction, linear boundary data comes back exactly on the fine grid, and the coarse
    network input holds the fine ring sampled at the coarse nodes and the fine f averaged
    around each coarse node."""
    n, nc = 47, 11                        # 48 = 4 * 12
    fn = lambda x, y: -0.2 + 0.6 * x + 1.1 * y  # noqa: E731
    u, full = _ring_grid(n, fn)
    i, j = np.meshgrid(np.arange(1, n + 1), np.arange(1, n + 1), indexing="ij")
    f = torch.from_numpy((i + 2 * j).astype(np.float64)).cuda()  # linear in the fine indices
    net = ZeroNet()
    u0 = learned.initial_guess_coarse(net, f, u, nc)
    np.testing.assert_allclose(u0.cpu().numpy(), full.numpy(), rtol=0, atol=1e-13)
    assert torch.equal(u0[0], u[0]) and torch.equal(u0[-1], u[-1])
    x = net.inputs[0][0].cpu()
    r = (n + 1) // (nc + 1)
    ring_c = u.cpu()[::r, ::r].numpy().astype(np.float32)
    np.testing.assert_array_equal(x[0, :nc + 2, 2].numpy(), ring_c[0])       # sampled ring
    # the symmetric window around coarse node (m, m') lies inside the fine interior, so the
    # average of the linear f is its value at the fine node (r m, r m')
    fc = x[1:nc + 1, 1:nc + 1, 0].numpy()
    m = np.arange(1, nc + 1)
    np.testing.assert_array_equal(fc, (r * m[:, None] + 2 * r * m[None, :]).astype(np.float32))
    with pytest.raises(ValueError):
        learned.initial_guess_coarse(net, f, u, 12)   # 48 is not a multiple of 13




def test_training_target_is_the_solution_minus_the_blend():
    n, size = 13, 16
    rng = np.random.default_rng(8)
    u = torch.from_numpy(rng.uniform(-1, 1, (n + 2, n + 2))).cuda()
    sol = torch.from_numpy(rng.uniform(-1, 1, (n + 2, n + 2))).cuda()
    t = guess_target(sol, u, size).cpu().numpy()
    want = (sol - boundary_blend(u)).cpu().numpy().astype(np.float32)
    np.testing.assert_array_equal(t[:n + 2, :n + 2], want)
    assert np.all(t[n + 2:] == 0) and np.all(t[:, n + 2:] == 0)


def test_grid_kernels_refuse_host_memory_and_bad_sizes():
    u = torch.zeros((10, 10), dtype=torch.float64)
    with pytest.raises(TypeError):
        boundary_blend(u)  # a CPU tensor
    ud = u.cuda()
    with pytest.raises(rb.RbgsError):
        network_input(torch.zeros((8, 8), dtype=torch.float64, device="cuda"), ud, size=12)  # not a multiple of 8
