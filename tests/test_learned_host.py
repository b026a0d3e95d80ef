"""Host-side logic of the learned initial guess, on the CPU: the boundary interpolation the
network's correction is added to, the network's input channels, the coarse-grid path and
the training schedule.  The network itself is replaced by a stand-in that predicts a zero
correction (or records its calls); its kernels are tested on the GPU."""
import numpy as np
import pytest
import torch

from paper_2607_01735_gb300 import learned
from paper_2607_01735_gb300.unet import boundary_blend, network_input


def _ring_grid(n, fn):
    g = n + 2
    t = np.linspace(0.0, 1.0, g)
    x, y = np.meshgrid(t, t, indexing="ij")
    full = fn(x, y)
    u = np.zeros((g, g))
    u[0, :], u[-1, :], u[:, 0], u[:, -1] = full[0, :], full[-1, :], full[:, 0], full[:, -1]
    return torch.from_numpy(u), torch.from_numpy(full)


class ZeroNet:
    """Predicts a zero correction; records the inputs it was given."""

    def __init__(self):
        self.inputs = []

    def forward(self, x):
        self.inputs.append(x)
        return torch.zeros(x.shape[:3], dtype=torch.float32)


@pytest.mark.parametrize("fn", [lambda x, y: 0.3 - 1.2 * x + 0.7 * y,
                                lambda x, y: -0.5 + 0.25 * x + 2.0 * y - 1.5 * x * y])
def test_boundary_blend_reproduces_bilinear_data(fn):
    """The Coons patch of data that is linear in x and in y separately is that function."""
    u, full = _ring_grid(37, fn)
    got = boundary_blend(u).numpy()
    np.testing.assert_allclose(got, full.numpy(), rtol=0, atol=1e-14)


def test_boundary_blend_keeps_the_ring():
    rng = np.random.default_rng(3)
    u = torch.from_numpy(rng.uniform(-1, 1, (20, 20)))
    got = boundary_blend(u)
    for a, b in ((got[0], u[0]), (got[-1], u[-1]), (got[:, 0], u[:, 0]), (got[:, -1], u[:, -1])):
        np.testing.assert_allclose(a.numpy(), b.numpy(), rtol=0, atol=1e-14)


def test_network_input_channels():
    n = 13
    g = n + 2
    rng = np.random.default_rng(4)
    f = torch.from_numpy(rng.uniform(-1, 1, (n, n)))
    u = torch.from_numpy(rng.uniform(-1, 1, (g, g)))
    x = network_input(f, u)
    size = learned.grid_size(n)
    assert x.shape == (size, size, 4) and size % 8 == 0 and size >= g
    ring = np.ones((g, g), dtype=bool)
    ring[1:-1, 1:-1] = False
    assert np.array_equal(x[:g, :g, 1].numpy() == 1.0, ring)                 # mask
    np.testing.assert_array_equal(x[1:n + 1, 1:n + 1, 0].numpy(), f.numpy().astype(np.float32))
    assert np.all(x[:g, :g, 0].numpy()[ring] == 0)                          # f only inside
    np.testing.assert_array_equal(x[:g, :g, 2].numpy()[ring], u.numpy().astype(np.float32)[ring])
    assert np.all(x[:g, :g, 2].numpy()[~ring] == 0)                         # ring values only
    np.testing.assert_array_equal(x[:g, :g, 3].numpy(), boundary_blend(u).numpy().astype(np.float32))
    assert np.all(x[g:].numpy() == 0) and np.all(x[:, g:].numpy() == 0)     # zero padding


def test_initial_guess_with_zero_correction_is_the_blend_inside_the_given_ring():
    n = 21
    fn = lambda x, y: 0.1 + 0.9 * x - 0.4 * y  # noqa: E731
    u, full = _ring_grid(n, fn)
    f = torch.zeros((n, n), dtype=torch.float64)
    net = ZeroNet()
    u0 = learned.initial_guess(net, f, u)
    np.testing.assert_allclose(u0.numpy(), full.numpy(), rtol=0, atol=1e-14)
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
    f = torch.from_numpy((i + 2 * j).astype(np.float64))  # linear in the fine indices
    net = ZeroNet()
    u0 = learned.initial_guess_coarse(net, f, u, nc)
    np.testing.assert_allclose(u0.numpy(), full.numpy(), rtol=0, atol=1e-13)
    assert torch.equal(u0[0], u[0]) and torch.equal(u0[-1], u[-1])
    x = net.inputs[0][0]
    r = (n + 1) // (nc + 1)
    ring_c = u[::r, ::r].numpy().astype(np.float32)
    np.testing.assert_array_equal(x[0, :nc + 2, 2].numpy(), ring_c[0])       # sampled ring
    # the symmetric window around coarse node (m, m') lies inside the fine interior, so the
    # average of the linear f is its value at the fine node (r m, r m')
    fc = x[1:nc + 1, 1:nc + 1, 0].numpy()
    m = np.arange(1, nc + 1)
    np.testing.assert_array_equal(fc, (r * m[:, None] + 2 * r * m[None, :]).astype(np.float32))
    with pytest.raises(ValueError):
        learned.initial_guess_coarse(net, f, u, 12)   # 48 is not a multiple of 13


def test_training_schedule_is_cosine_decay_over_the_steps():
    class Recorder:
        def __init__(self):
            self.lrs, self.batches = [], []

        def train_step(self, x, y, mask, lr):
            self.lrs.append(lr)
            self.batches.append(x.shape[0])
            return float(len(self.lrs))

    x = torch.zeros((10, 8, 8, 4))
    y = torch.zeros((10, 8, 8))
    mask = torch.ones((10, 8, 8))
    net = Recorder()
    losses = learned.train(net, x, y, mask, steps=8, batch=4, lr=2e-3)
    assert losses == [float(k) for k in range(1, 9)]
    assert net.batches == [4] * 8
    want = [2e-3 * 0.5 * (1 + np.cos(np.pi * k / 8)) for k in range(8)]
    np.testing.assert_allclose(net.lrs, want, rtol=1e-15)
    assert net.lrs[0] == 2e-3 and all(a > b for a, b in zip(net.lrs, net.lrs[1:]))
