"""FP64 reference of the learned Poisson-guess network -- TEST INFRASTRUCTURE ONLY.

The network (no counterpart in the paper; the paper cites data-driven multigrid,
Sec. 3, as the precedent of learned solver components) is a bias-free 3D
convolutional net on a coarse multigrid level:

    h1 = relu(conv(x, W1)),  h2 = relu(conv(h1, W2)),  y = conv(h2, W3)

with 3x3x3 kernels, zero padding, channels 1 -> C -> C -> 1. conv(x, W)[v, o] =
sum_{tap, i} x[v + tap, i] W[tap, i, o] (taps in z, y, x order, offsets -1..1),
arrays laid out as [z, y, x, channel]. The loss of a sample is
sum (y - t)^2 / sum t^2.

Written with plain numpy shifts (one multiply-add per tap); used only to check
the CUDA kernels and pinned by finite differences and closed forms in
tests/test_oracle_net.py. 2D grids are the nz = 1 case with the z taps reading
the zero padding.
"""
from __future__ import annotations

import numpy as np

TAPS = [(dz, dy, dx) for dz in (-1, 0, 1) for dy in (-1, 0, 1) for dx in (-1, 0, 1)]


def shift(x, dz, dy, dx):
    """s[z, y, x] = x[z + dz, y + dy, x + dx] with zeros outside."""
    nz, ny, nx = x.shape[:3]
    out = np.zeros_like(x)
    zs, ys, xs = slice(max(0, -dz), nz - max(0, dz)), slice(max(0, -dy), ny - max(0, dy)), slice(max(0, -dx), nx - max(0, dx))
    zt, yt, xt = slice(max(0, dz), nz - max(0, -dz)), slice(max(0, dy), ny - max(0, -dy)), slice(max(0, dx), nx - max(0, -dx))
    if zs.start < zs.stop and ys.start < ys.stop and xs.start < xs.stop:
        out[zs, ys, xs] = x[zt, yt, xt]
    return out


def conv(x, W):
    """x: [nz, ny, nx, Ci]; W: [27, Ci, Co] -> [nz, ny, nx, Co]."""
    y = np.zeros(x.shape[:3] + (W.shape[2],))
    for t, (dz, dy, dx) in enumerate(TAPS):
        y += shift(x, dz, dy, dx) @ W[t]
    return y


def conv_grads(x, W, dy):
    """Gradients of sum(conv(x, W) * dy) w.r.t. x and W."""
    dx = np.zeros_like(x)
    dW = np.zeros_like(W)
    for t, (dz, dyy, dxx) in enumerate(TAPS):
        xs = shift(x, dz, dyy, dxx)
        dW[t] = xs.reshape(-1, x.shape[3]).T @ dy.reshape(-1, dy.shape[3])
        dx += shift(dy @ W[t].T, -dz, -dyy, -dxx)
    return dx, dW


def forward(x, Ws):
    """x: [nz, ny, nx] input residual; Ws = (W1, W2, W3). Returns y and the
    intermediate pre-activations (for the backward pass)."""
    a0 = x[..., None]
    z1 = conv(a0, Ws[0])
    a1 = np.maximum(z1, 0.0)
    z2 = conv(a1, Ws[1])
    a2 = np.maximum(z2, 0.0)
    y = conv(a2, Ws[2])[..., 0]
    return y, (a0, z1, a1, z2, a2)


def loss(y, t):
    return float(np.sum((y - t) ** 2) / np.sum(t ** 2))


def backward(x, Ws, t):
    """Loss and its gradients w.r.t. the three weight tensors."""
    y, (a0, z1, a1, z2, a2) = forward(x, Ws)
    den = np.sum(t ** 2)
    L = float(np.sum((y - t) ** 2) / den)
    dy = (2.0 * (y - t) / den)[..., None]
    da2, dW3 = conv_grads(a2, Ws[2], dy)
    dz2 = da2 * (z2 > 0)
    da1, dW2 = conv_grads(a1, Ws[1], dz2)
    dz1 = da1 * (z1 > 0)
    _, dW1 = conv_grads(a0, Ws[0], dz1)
    return L, (dW1, dW2, dW3), y
