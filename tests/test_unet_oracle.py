"""Pins for the U-Net oracle (CPU): the convolution against SciPy's textbook
cross-correlation, every backward formula against central finite differences, and the
full network's gradient against directional finite differences of its loss."""
import numpy as np
import pytest

from oracle import unet_ref as U

scipy_signal = pytest.importorskip("scipy.signal")


def test_conv_forward_matches_scipy_correlate():
    rng = np.random.default_rng(0)
    x = rng.normal(size=(2, 7, 9, 3))
    w = rng.normal(size=(4, 3, 3, 3))
    b = rng.normal(size=4)
    y = U.conv_forward(x, w, b)
    for bi in range(2):
        for o in range(4):
            ref = sum(scipy_signal.correlate2d(x[bi, :, :, c], w[o, :, :, c], mode="same", boundary="fill")
                      for c in range(3)) + b[o]
            assert np.allclose(y[bi, :, :, o], ref, rtol=1e-12, atol=1e-12)
    # 1x1 convolution is a per-pixel matrix product
    w1 = rng.normal(size=(5, 1, 1, 3))
    assert np.allclose(U.conv_forward(x, w1), np.einsum("bhwc,oc->bhwo", x, w1[:, 0, 0, :]))


@pytest.mark.parametrize("k", [1, 3])
def test_conv_backward_matches_finite_differences(k):
    rng = np.random.default_rng(1)
    x = rng.normal(size=(2, 5, 6, 3))
    w = rng.normal(size=(4, k, k, 3))
    g = rng.normal(size=(2, 5, 6, 4))
    dx, dw, db = U.conv_backward(x, w, g)
    f = lambda xx, ww, bb: float((U.conv_forward(xx, ww, bb) * g).sum())
    b0 = np.zeros(4)
    eps = 1e-6
    for idx in [(0, 0, 0, 0), (1, 4, 5, 2), (0, 2, 3, 1)]:
        e = np.zeros_like(x); e[idx] = eps
        assert abs((f(x + e, w, b0) - f(x - e, w, b0)) / (2 * eps) - dx[idx]) < 1e-6
    for idx in [(0, 0, 0, 0), (3, k - 1, k - 1, 2), (2, k // 2, 0, 1)]:
        e = np.zeros_like(w); e[idx] = eps
        assert abs((f(x, w + e, b0) - f(x, w - e, b0)) / (2 * eps) - dw[idx]) < 1e-6
    e = np.zeros(4); e[2] = eps
    assert abs((f(x, w, b0 + e) - f(x, w, b0 - e)) / (2 * eps) - db[2]) < 1e-6


def test_pool_and_upsample_adjoints():
    rng = np.random.default_rng(2)
    a = rng.normal(size=(1, 4, 6, 2))
    b = rng.normal(size=(1, 2, 3, 2))
    # <pool(a), b> = <a, pool^T(b)> and <up(b), a> = <b, up^T(a)>
    assert np.isclose((U.avgpool(a) * b).sum(), (a * U.avgpool_backward(b)).sum())
    assert np.isclose((U.upsample(b) * a).sum(), (b * U.upsample_backward(a)).sum())
    assert np.allclose(U.avgpool(U.upsample(b)), b)


def test_network_gradient_directional_derivatives():
    rng = np.random.default_rng(3)
    n = U.num_params()
    params = rng.normal(size=n) * 0.05
    x3 = rng.normal(size=(1, 8, 8, 3))
    target = rng.normal(size=(1, 8, 8))
    mask = (rng.uniform(size=(1, 8, 8)) > 0.3).astype(np.float64)
    L, grad = U.backward(params, x3, target, mask)
    assert np.isclose(L, U.loss(params, x3, target, mask))
    eps = 1e-7  # small enough that no ReLU switches under the perturbation
    for seed in range(3):
        v = np.random.default_rng(10 + seed).normal(size=n)
        fd = (U.loss(params + eps * v, x3, target, mask) - U.loss(params - eps * v, x3, target, mask)) / (2 * eps)
        assert abs(fd - grad @ v) <= 1e-6 * max(1.0, abs(fd))


def test_bf16_rounding_is_round_to_nearest_even():
    """unet_ref.bf16_round against torch's float32 -> bfloat16 conversion (round to nearest,
    ties to even) on float32 values, and on hand-made ties."""
    import torch
    rng = np.random.default_rng(0)
    a = (rng.normal(size=200000) * 10.0 ** rng.integers(-6, 6, 200000)).astype(np.float32).astype(np.float64)
    want = torch.from_numpy(a).float().to(torch.bfloat16).double().numpy()
    assert np.array_equal(U.bf16_round(a), want)
    one = 1.0
    ulp = 2.0 ** -7                      # spacing of bfloat16 in [1, 2)
    assert U.bf16_round(one + ulp / 2) == one                # tie to the even significand 1.0
    assert U.bf16_round(one + 3 * ulp / 2) == one + 2 * ulp  # tie up to the even one
    assert U.bf16_round(-(one + ulp / 2 + 2.0 ** -30)) == -(one + ulp)
    assert U.bf16_round(0.0) == 0.0


def test_bf16_network_stays_near_the_exact_one():
    """The bf16 storage statement perturbs the network by rounding-sized amounts only: the
    output within 3% of scale and the gradient's direction unchanged (cosine > 0.999)."""
    rng = np.random.default_rng(4)
    params = rng.normal(size=U.num_params()) * 0.05
    x = rng.normal(size=(1, 16, 16, 4))
    t = rng.normal(size=(1, 16, 16)) * 0.1
    m = np.ones((1, 16, 16))
    y0, y1 = U.forward(params, x)[..., 0], U.forward(params, x, bf16=True)[..., 0]
    assert np.max(np.abs(y1 - y0)) <= 3e-2 * np.max(np.abs(y0))
    assert not np.array_equal(y0, y1)
    _, g0 = U.backward(params, x, t, m)
    _, g1 = U.backward(params, x, t, m, bf16=True)
    assert g0 @ g1 / (np.linalg.norm(g0) * np.linalg.norm(g1)) > 0.999
