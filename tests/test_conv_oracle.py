"""Pins of the surrogate's FP64 CPU oracle: the convolution equals a library
2-D correlation, every gradient equals central finite differences of the
forward pass, Adam's first step has its closed form, and vertex-aligned
bilinear upsampling is exact on bilinear fields."""
import numpy as np
import pytest
from scipy.signal import correlate2d

import inputs
from oracle import conv_oracle as CO


def _rand(seed, shape, scale=1.0):
    return inputs.uniform_array(seed, shape, -scale, scale)


def test_conv_equals_library_correlation():
    x = _rand(1, (2, 3, 7, 5))
    w = _rand(2, (4, 3, 3, 3))
    b = _rand(3, (4,))
    y = CO.conv3x3(x, w, b)
    for bb in range(2):
        for o in range(4):
            ref = sum(correlate2d(x[bb, c], w[o, c], mode="same", boundary="fill") for c in range(3)) + b[o]
            assert np.abs(y[bb, o] - ref).max() < 1e-13


def _fd(f, x, eps=1e-6):
    g = np.zeros_like(x)
    it = np.nditer(x, flags=["multi_index"])
    for _ in it:
        i = it.multi_index
        xp = x.copy()
        xm = x.copy()
        xp[i] += eps
        xm[i] -= eps
        g[i] = (f(xp) - f(xm)) / (2 * eps)
    return g


def test_conv_gradients_match_finite_differences():
    x = _rand(4, (2, 2, 5, 4))
    w = _rand(5, (3, 2, 3, 3))
    b = _rand(6, (3,))
    dy = _rand(7, (2, 3, 5, 4))
    loss = lambda x_, w_, b_: float(np.sum(dy * CO.conv3x3(x_, w_, b_)))
    dx, dw, db = CO.conv3x3_backward(x, w, dy)
    assert np.abs(dx - _fd(lambda v: loss(v, w, b), x)).max() < 1e-8
    assert np.abs(dw - _fd(lambda v: loss(x, v, b), w)).max() < 1e-8
    assert np.abs(db - _fd(lambda v: loss(x, w, v), b)).max() < 1e-8


def test_network_gradient_matches_finite_differences():
    rng = inputs.rng(8)
    params = [(rng.normal(0, 0.5, (4, 3, 3, 3)), rng.normal(0, 0.1, 4)),
              (rng.normal(0, 0.5, (4, 4, 3, 3)), rng.normal(0, 0.1, 4)),
              (rng.normal(0, 0.5, (2, 4, 3, 3)), rng.normal(0, 0.1, 2))]
    x = rng.normal(0, 1, (2, 3, 6, 5))
    t = rng.normal(0, 1, (2, 2, 6, 5))

    def loss_of(ps):
        y, _ = CO.network_forward(x, ps)
        return CO.mse(y, t)[0]

    y, pre = CO.network_forward(x, params)
    _, dout = CO.mse(y, t)
    grads = CO.network_backward(params, pre, dout)
    for k in range(len(params)):
        w, b = params[k]
        fw = lambda v, k=k: loss_of([(v, params[j][1]) if j == k else params[j] for j in range(len(params))])
        fb = lambda v, k=k: loss_of([(params[j][0], v) if j == k else params[j] for j in range(len(params))])
        assert np.abs(grads[k][0] - _fd(fw, w)).max() < 1e-7
        assert np.abs(grads[k][1] - _fd(fb, b)).max() < 1e-7


def test_adam_first_step_closed_form():
    """After one step from m = v = 0 the bias-corrected update is
    -lr * g / (|g| + eps) (Kingma & Ba, 2015)."""
    w = _rand(9, (50,))
    g = _rand(10, (50,))
    w1, m1, v1 = CO.adam(w, g, np.zeros(50), np.zeros(50), 1, lr=1e-3)
    assert np.abs(w1 - (w - 1e-3 * g / (np.abs(g) + 1e-8))).max() < 1e-15
    assert np.allclose(m1, 0.1 * g) and np.allclose(v1, 0.001 * g * g)


def test_vertex_upsampling_is_exact_on_bilinear_fields():
    h, w, k = 5, 4, 8
    yy, xx = np.meshgrid(np.arange(h), np.arange(w), indexing="ij")
    f = 0.3 + 0.2 * xx - 0.7 * yy + 0.05 * xx * yy
    F = CO.upsample_bilinear_vertex(f, k)
    assert F.shape == ((h - 1) * k + 1, (w - 1) * k + 1)
    Y, X = np.meshgrid(np.arange(F.shape[0]) / k, np.arange(F.shape[1]) / k, indexing="ij")
    assert np.abs(F - (0.3 + 0.2 * X - 0.7 * Y + 0.05 * X * Y)).max() < 1e-14
    assert np.array_equal(F[::k, ::k], f)
