"""The seeded input recipes (synth/): Gaussian random fields, Box-Muller normals, the batched
problem table and the learned-guess samples, each checked against its stated definition on
the CPU.  (The SplitMix64 stream itself is pinned to its published outputs in
test_oracle_pins.py.)"""
import math

import numpy as np

import synth


def test_grf_is_the_stated_sine_series_with_unit_rms():
    """The DST synthesis equals the sine sum of its definition, evaluated term by term."""
    n, nj, stream = 6, 5, 12
    f, used = synth.grf_rhs(n, stream, nj)
    assert used == 2 * ((n * nj + 1) // 2)
    xi = synth.normal_pairs(stream, n * nj).reshape(n, nj)
    h_i, h_j = 1.0 / (n + 1), 1.0 / (nj + 1)
    direct = np.zeros((n, nj))
    for i in range(1, n + 1):
        for j in range(1, nj + 1):
            s = 0.0
            for k in range(1, n + 1):
                for l in range(1, nj + 1):
                    s += (xi[k - 1, l - 1] * (k * k + l * l) ** -0.75
                          * math.sin(k * math.pi * i * h_i) * math.sin(l * math.pi * j * h_j))
            direct[i - 1, j - 1] = s
    direct /= math.sqrt(np.mean(direct ** 2))
    np.testing.assert_allclose(f, direct, rtol=0, atol=1e-12)
    assert abs(np.mean(f * f) - 1.0) < 1e-14


def test_grf_spectrum_follows_the_power_law():
    """Projected back onto the sine modes, the field's coefficients are xi_kl (k^2+l^2)^(-3/4)
    times one normalising constant."""
    from scipy.fft import dst
    n, stream = 32, 2
    f, _ = synth.grf_rhs(n, stream)
    a = dst(dst(f, type=1, axis=0), type=1, axis=1) / (2 * (n + 1)) ** 2 * 4  # inverse of the synthesis
    xi = synth.normal_pairs(stream, n * n).reshape(n, n)
    k = np.arange(1, n + 1, dtype=np.float64)[:, None]
    want = xi * (k * k + k.T * k.T) ** -0.75
    ratio = a / want
    np.testing.assert_allclose(ratio, ratio[0, 0], rtol=1e-9)


def test_box_muller_normals():
    z = synth.normal_pairs(5, 200001)
    assert z.shape == (200001,)
    assert abs(z.mean()) < 0.01 and abs(z.var() - 1.0) < 0.01
    # pair m from uniforms (2m, 2m+1)
    u = synth.uniform01(5, 2).numpy()
    r = math.sqrt(-2.0 * math.log1p(-u[0]))
    assert z[0] == r * math.cos(2 * math.pi * u[1]) and z[1] == r * math.sin(2 * math.pi * u[1])
    # an odd count is the prefix of the next even one
    np.testing.assert_array_equal(synth.normal_pairs(5, 7), synth.normal_pairs(5, 8)[:7])


def test_batched_problem_table_recipe():
    sizes = (63, 127, 255, 511, 1023)
    table = synth.batched_problem_table(512, 3)
    u = synth.uniform01(3, 1024).numpy()
    for p, e in enumerate(table):
        assert e["n"] == sizes[int(u[2 * p] * 5)]
        assert e["c"] == 2.0 * u[2 * p + 1] - 1.0 and -1.0 <= e["c"] < 1.0
        assert e["f_stream"] == 3 * 2 ** 16 + p
    counts = np.bincount([sizes.index(e["n"]) for e in table], minlength=5)
    assert counts.sum() == 512 and counts.min() > 512 / 5 * 0.7   # every size well represented
    f, u0, h2 = synth.batched_problem(table[7])
    n = table[7]["n"]
    assert f.shape == (n, n) and u0.shape == (n + 2, n + 2) and h2 == synth.h_squared(n)
    np.testing.assert_array_equal(f, synth.uniform_pm1_grid(n, table[7]["f_stream"]).numpy())
    ring = np.ones((n + 2, n + 2), dtype=bool)
    ring[1:-1, 1:-1] = False
    assert np.all(u0[ring] == table[7]["c"]) and np.all(u0[~ring] == 0.0)


def test_learned_guess_sample_recipe():
    """GRF f from the stream, then a, b, c ~ U(-1, 1) from the same stream after f; the
    ring holds a + b x + c y and the interior is zero."""
    n, stream = 15, 10
    f, u = synth.learned_guess_sample(n, stream)
    f_ref, used = synth.grf_rhs(n, stream)
    np.testing.assert_array_equal(f, f_ref)
    a, b, c = synth.uniform01(stream, 3, used).numpy() * 2.0 - 1.0
    x, y, _ = synth.grid_coords(n)
    g = a + b * x + c * y
    ring = np.ones((n + 2, n + 2), dtype=bool)
    ring[1:-1, 1:-1] = False
    np.testing.assert_allclose(u[ring], np.broadcast_to(g, u.shape)[ring], rtol=0, atol=1e-15)
    assert np.all(u[~ring] == 0.0)


def test_manufactured_rhs_and_h_squared():
    n = 255
    assert synth.h_squared(n) == 2.0 ** -16           # h = 1/256 exactly
    f = synth.manufactured_rhs(n)
    x = np.arange(1, n + 1) / (n + 1)
    np.testing.assert_allclose(f, 2 * math.pi ** 2 * np.outer(np.sin(math.pi * x), np.sin(math.pi * x)),
                               rtol=1e-15, atol=1e-14)
