"""FP64 CPU oracle for the warm-start surrogate's layers.

TEST INFRASTRUCTURE ONLY (tests, smoke, benchmark baselines).  The CUDA
library never imports it.

The surrogate is a stack of 3x3 convolutions (stride 1, zero padding 1, NCHW
layout) with bias and ReLU between layers, trained on a mean-squared error.
Written out from the definition of a discrete correlation:

    y[b, o, i, j] = bias[o] + sum_{c, di, dj} w[o, c, di, dj] * x[b, c, i + di - 1, j + dj - 1]

with x = 0 outside the image.  The gradients follow from the same sum by the
chain rule:

    dx[b, c, i, j]  = sum_{o, di, dj} w[o, c, di, dj] * dy[b, o, i - di + 1, j - dj + 1]
    dw[o, c, di, dj] = sum_{b, i, j} dy[b, o, i, j] * x[b, c, i + di - 1, j + dj - 1]
    dbias[o]         = sum_{b, i, j} dy[b, o, i, j]
"""
import numpy as np


def _pad(x):
    return np.pad(x, ((0, 0), (0, 0), (1, 1), (1, 1)))


def conv3x3(x, w, bias=None):
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    B, C, H, W = x.shape
    O = w.shape[0]
    xp = _pad(x)
    y = np.zeros((B, O, H, W))
    for di in range(3):
        for dj in range(3):
            patch = xp[:, :, di:di + H, dj:dj + W]  # x[b, c, i + di - 1, j + dj - 1]
            y += np.einsum("oc,bchw->bohw", w[:, :, di, dj], patch)
    if bias is not None:
        y += np.asarray(bias, dtype=np.float64)[None, :, None, None]
    return y


def conv3x3_backward(x, w, dy):
    """Gradients (dx, dw, dbias) of sum(dy * conv3x3(x, w, bias))."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    dy = np.asarray(dy, dtype=np.float64)
    B, C, H, W = x.shape
    xp = _pad(x)
    dxp = np.zeros_like(xp)
    dw = np.zeros_like(w)
    for di in range(3):
        for dj in range(3):
            patch = xp[:, :, di:di + H, dj:dj + W]
            dw[:, :, di, dj] = np.einsum("bohw,bchw->oc", dy, patch)
            dxp[:, :, di:di + H, dj:dj + W] += np.einsum("oc,bohw->bchw", w[:, :, di, dj], dy)
    dx = dxp[:, :, 1:-1, 1:-1]
    db = dy.sum(axis=(0, 2, 3))
    return dx, dw, db


def relu(y):
    return np.maximum(y, 0.0)


def network_forward(x, params):
    """params: list of (w, b); ReLU after every layer but the last.
    Returns the output and the pre-activations of every layer."""
    pre = []
    a = np.asarray(x, dtype=np.float64)
    for k, (w, b) in enumerate(params):
        y = conv3x3(a, w, b)
        pre.append((a, y))
        a = relu(y) if k < len(params) - 1 else y
    return a, pre


def mse(y, t):
    d = np.asarray(y, dtype=np.float64) - np.asarray(t, dtype=np.float64)
    return float(np.mean(d * d)), 2.0 * d / d.size


def network_backward(params, pre, dout):
    """Gradients of the loss w.r.t. every (w, b), given dL/d(output)."""
    grads = [None] * len(params)
    g = np.asarray(dout, dtype=np.float64)
    for k in range(len(params) - 1, -1, -1):
        a_in, y = pre[k]
        if k < len(params) - 1:
            g = g * (y > 0.0)
        dx, dw, db = conv3x3_backward(a_in, params[k][0], g)
        grads[k] = (dw, db)
        g = dx
    return grads


def adam(w, g, m, v, t, lr, b1=0.9, b2=0.999, eps=1e-8):
    """One Adam update (Kingma & Ba 2015), bias-corrected, in place on copies."""
    m = b1 * m + (1.0 - b1) * g
    v = b2 * v + (1.0 - b2) * g * g
    mh = m / (1.0 - b1 ** t)
    vh = v / (1.0 - b2 ** t)
    return w - lr * mh / (np.sqrt(vh) + eps), m, v


def upsample_bilinear_vertex(f, factor):
    """Vertex-aligned bilinear upsampling of (..., h, w) to (..., (h-1)*factor+1,
    (w-1)*factor+1): coarse node (i, j) sits on fine node (factor*i, factor*j)."""
    f = np.asarray(f, dtype=np.float64)
    h, w = f.shape[-2:]
    H, W = (h - 1) * factor + 1, (w - 1) * factor + 1
    yi = np.arange(H) / factor
    xi = np.arange(W) / factor
    y0 = np.minimum(np.floor(yi).astype(int), h - 2)
    x0 = np.minimum(np.floor(xi).astype(int), w - 2)
    ty = (yi - y0)[:, None]
    tx = (xi - x0)[None, :]
    f00 = f[..., y0[:, None], x0[None, :]]
    f01 = f[..., y0[:, None], x0[None, :] + 1]
    f10 = f[..., y0[:, None] + 1, x0[None, :]]
    f11 = f[..., y0[:, None] + 1, x0[None, :] + 1]
    return (1 - ty) * ((1 - tx) * f00 + tx * f01) + ty * ((1 - tx) * f10 + tx * f11)
