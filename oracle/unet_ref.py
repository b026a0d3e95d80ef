"""Oracle for the learned initial guess: the U-Net's forward and backward pass in plain
numpy float64.

TEST INFRASTRUCTURE ONLY (see the package docstring).  The paper has no network; this
is the plain definition of the one the library trains: 3x3 cross-correlations with zero
padding, ReLU, 2x2 average pooling, nearest-neighbour upsampling, channel concatenation
[upsampled, skip], a 1x1 output convolution, masked mean-squared error.  Tensors are
NHWC.  Parameters are one flat vector, per layer weights [Cout][k][k][Cin] then biases.
Backward is the chain rule written out layer by layer (no automatic differentiation).
"""
from __future__ import annotations

import numpy as np

# cin, cout, ksize, relu, level
LAYERS = [(16, 32, 3, 1, 0), (32, 32, 3, 1, 0), (32, 64, 3, 1, 1), (64, 64, 3, 1, 1),
          (64, 128, 3, 1, 2), (128, 128, 3, 1, 2), (128, 256, 3, 1, 3), (256, 256, 3, 1, 3),
          (384, 128, 3, 1, 2), (128, 128, 3, 1, 2), (192, 64, 3, 1, 1), (64, 64, 3, 1, 1),
          (96, 32, 3, 1, 0), (32, 32, 3, 1, 0), (32, 8, 1, 0, 0)]
IN_CH = 16


def param_slices():
    """(weight slice, bias slice, weight shape) per layer in the flat parameter vector."""
    out, off = [], 0
    for cin, cout, k, _, _ in LAYERS:
        nw = cout * k * k * cin
        out.append((slice(off, off + nw), slice(off + nw, off + nw + cout), (cout, k, k, cin)))
        off += nw + cout
    return out, off


def num_params() -> int:
    return param_slices()[1]


# ------------------------------------------------------------------ layer definitions
def conv_forward(x, w, b=None):
    """y[b,i,j,o] = bias[o] + sum_{di,dj,c} w[o,di,dj,c] x[b, i+di-p, j+dj-p, c], zero padding."""
    bsz, h, wd, cin = x.shape
    cout, k, _, _ = w.shape
    p = k // 2
    xp = np.zeros((bsz, h + 2 * p, wd + 2 * p, cin))
    xp[:, p:p + h, p:p + wd, :] = x
    y = np.zeros((bsz, h, wd, cout))
    for di in range(k):
        for dj in range(k):
            y += np.einsum("bhwc,oc->bhwo", xp[:, di:di + h, dj:dj + wd, :], w[:, di, dj, :])
    if b is not None:
        y += b
    return y


def conv_backward(x, w, g):
    """Gradients of conv_forward given g = dL/dy: (dx, dw, db)."""
    bsz, h, wd, cin = x.shape
    cout, k, _, _ = w.shape
    p = k // 2
    xp = np.zeros((bsz, h + 2 * p, wd + 2 * p, cin))
    xp[:, p:p + h, p:p + wd, :] = x
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for di in range(k):
        for dj in range(k):
            dw[:, di, dj, :] = np.einsum("bhwo,bhwc->oc", g, xp[:, di:di + h, dj:dj + wd, :])
            dxp[:, di:di + h, dj:dj + wd, :] += np.einsum("bhwo,oc->bhwc", g, w[:, di, dj, :])
    return dxp[:, p:p + h, p:p + wd, :], dw, g.sum(axis=(0, 1, 2))


def avgpool(x):
    b, h, w, c = x.shape
    return x.reshape(b, h // 2, 2, w // 2, 2, c).mean(axis=(2, 4))


def avgpool_backward(g):
    return np.repeat(np.repeat(g, 2, axis=1), 2, axis=2) * 0.25


def upsample(x):
    return np.repeat(np.repeat(x, 2, axis=1), 2, axis=2)


def upsample_backward(g):
    b, h, w, c = g.shape
    return g.reshape(b, h // 2, 2, w // 2, 2, c).sum(axis=(2, 4))


def relu(x):
    return np.maximum(x, 0.0)


def bf16_round(a):
    """Nearest bfloat16 value (ties to even) of each element, returned as float64.

    bfloat16 keeps binary32's sign and 8-bit exponent and the top 7 of its 23 fraction bits;
    rounding a binary64 value to it once: split off everything below the 8-bit significand
    with frexp, round that significand (an integer in [128, 256)) half to even, rescale.
    Zeros stay zeros; the values here never reach bfloat16's overflow or subnormal range.
    """
    a = np.asarray(a, dtype=np.float64)
    m, e = np.frexp(a)                  # a = m 2^e, 0.5 <= |m| < 1
    q = np.rint(m * 256.0)              # 8 significant bits; rint rounds half to even
    return np.ldexp(q, e - 8)


# ------------------------------------------------------------------ network
def forward(params, x3, keep=False, bf16=False):
    """x3: B x H x W x C input channels (C <= 16; the network reads 16, zero-padded).
    Returns the 8-channel output (channel 0 is the prediction) and, with keep=True, the
    cached tensors for backward.

    bf16=True states the library's storage precision: the weights (not the biases), the
    input channels and every stored activation (each hidden convolution's output after
    ReLU, each pooled map) are rounded to bfloat16; sums and the output layer stay exact.
    """
    sl, _ = param_slices()
    rnd = bf16_round if bf16 else (lambda a: a)
    W = [rnd(params[s]).reshape(shape) for s, _, shape in sl]
    Bv = [params[bs] for _, bs, _ in sl]
    b, h, w, _ = x3.shape
    x = np.zeros((b, h, w, IN_CH))
    x[..., :x3.shape[-1]] = rnd(x3)
    cache = {"in": x}

    def conv(li, inp, name):
        pre = conv_forward(inp, W[li], Bv[li])
        out = relu(pre) if LAYERS[li][3] else pre
        if li < len(LAYERS) - 1:
            out = rnd(out)
        cache[name] = out
        return out

    def pool(inp, name):
        cache[name] = rnd(avgpool(inp))
        return cache[name]

    e0a = conv(0, x, "e0a"); s0 = conv(1, e0a, "s0"); p0 = pool(s0, "p0")
    e1a = conv(2, p0, "e1a"); s1 = conv(3, e1a, "s1"); p1 = pool(s1, "p1")
    e2a = conv(4, p1, "e2a"); s2 = conv(5, e2a, "s2"); p2 = pool(s2, "p2")
    b3a = conv(6, p2, "b3a"); b3b = conv(7, b3a, "b3b")
    c2 = np.concatenate([upsample(b3b), s2], axis=-1); cache["c2"] = c2
    d2a = conv(8, c2, "d2a"); d2b = conv(9, d2a, "d2b")
    c1 = np.concatenate([upsample(d2b), s1], axis=-1); cache["c1"] = c1
    d1a = conv(10, c1, "d1a"); d1b = conv(11, d1a, "d1b")
    c0 = np.concatenate([upsample(d1b), s0], axis=-1); cache["c0"] = c0
    d0a = conv(12, c0, "d0a"); d0b = conv(13, d0a, "d0b")
    out = conv(14, d0b, "out")
    return (out, cache) if keep else out


def loss(params, x3, target, mask, bf16=False):
    out = forward(params, x3, bf16=bf16)
    d = out[..., 0] - target
    return float((mask * d * d).sum() / mask.sum())


def backward(params, x3, target, mask, bf16=False):
    """(loss, gradient vector) of the masked MSE, by the chain rule.  bf16=True: the forward
    as above, and each convolution's pre-activation gradient (what its weight, bias and input
    gradients are formed from) rounded to bfloat16, as the library stores it."""
    sl, n = param_slices()
    rnd = bf16_round if bf16 else (lambda a: a)
    W = [rnd(params[s]).reshape(shape) for s, _, shape in sl]
    out, c = forward(params, x3, keep=True, bf16=bf16)
    cnt = mask.sum()
    d = out[..., 0] - target
    L = float((mask * d * d).sum() / cnt)
    grad = np.zeros(n)
    gout = np.zeros_like(out)
    gout[..., 0] = 2.0 * mask * d / cnt

    def conv_b(li, inp_name, out_name, gpost):
        gpre = rnd(gpost * (c[out_name] > 0) if LAYERS[li][3] else gpost)
        dx, dw, db = conv_backward(c[inp_name], W[li], gpre)
        grad[sl[li][0]] += dw.reshape(-1)
        grad[sl[li][1]] += db
        return dx

    g = conv_b(14, "d0b", "out", gout)
    g = conv_b(13, "d0a", "d0b", g)
    g = conv_b(12, "c0", "d0a", g)
    g_d1b, g_s0 = upsample_backward(g[..., :64]), g[..., 64:]
    g = conv_b(11, "d1a", "d1b", g_d1b)
    g = conv_b(10, "c1", "d1a", g)
    g_d2b, g_s1 = upsample_backward(g[..., :128]), g[..., 128:]
    g = conv_b(9, "d2a", "d2b", g_d2b)
    g = conv_b(8, "c2", "d2a", g)
    g_b3b, g_s2 = upsample_backward(g[..., :256]), g[..., 256:]
    g = conv_b(7, "b3a", "b3b", g_b3b)
    g = conv_b(6, "p2", "b3a", g)
    g_s2 = g_s2 + avgpool_backward(g)
    g = conv_b(5, "e2a", "s2", g_s2)
    g = conv_b(4, "p1", "e2a", g)
    g_s1 = g_s1 + avgpool_backward(g)
    g = conv_b(3, "e1a", "s1", g_s1)
    g = conv_b(2, "p0", "e1a", g)
    g_s0 = g_s0 + avgpool_backward(g)
    g = conv_b(1, "e0a", "s0", g_s0)
    conv_b(0, "in", "e0a", g)
    return L, grad
