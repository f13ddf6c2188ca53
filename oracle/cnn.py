"""Oracle for the learned warm start: a small residual CNN, in FP64.

The paper has no network. This module is the reference for the library's
warm-start network, which maps an early split-SART image to an initial guess.

Network, on images x of shape [B][1][nz][nx]:
    a1 = relu(conv(x,  W1) + b1)     1 -> 32 channels
    a2 = relu(conv(a1, W2) + b2)    32 -> 32
    a3 = relu(conv(a2, W3) + b3)    32 -> 32
    n  = conv(a3, W4) + b4          32 -> 1
    y  = x + n                      (residual)
Details:
- conv is a 3x3 cross-correlation with zero padding 1 ("same").
- Weights are [out][in][3][3]; tap (dy, dx) reads input pixel
  (r + dy - 1, c + dx - 1).
- Loss: mean over all B nz nx pixels of (y - t)^2.
- Adam (Kingma and Ba, 2015): m <- b1 m + (1-b1) g, v <- b2 v + (1-b2) g^2,
  theta <- theta - lr (m / (1 - b1^k)) / (sqrt(v / (1 - b2^k)) + eps),
  for step k = 1, 2, ...

The parameters travel as one flat vector in the order W1, b1, W2, b2, W3, b3,
W4, b4 (19105 values for 32 channels).

This module is test infrastructure: see the package docstring.
"""
from __future__ import annotations

import numpy as np

C = 32
SHAPES = [("W1", (C, 1, 3, 3)), ("b1", (C,)), ("W2", (C, C, 3, 3)), ("b2", (C,)),
          ("W3", (C, C, 3, 3)), ("b3", (C,)), ("W4", (1, C, 3, 3)), ("b4", (1,))]
N_PARAMS = sum(int(np.prod(s)) for _, s in SHAPES)


def unpack(theta):
    out, k = {}, 0
    for name, shape in SHAPES:
        n = int(np.prod(shape))
        out[name] = np.asarray(theta[k:k + n], dtype=float).reshape(shape)
        k += n
    return out


def pack(d):
    return np.concatenate([np.asarray(d[name], dtype=float).ravel() for name, _ in SHAPES])


def conv(x, W, b):
    """Zero-padded 3x3 cross-correlation: x [B][Ci][H][W], W [Co][Ci][3][3] -> [B][Co][H][W]."""
    B, Ci, H, Wd = x.shape
    xp = np.zeros((B, Ci, H + 2, Wd + 2))
    xp[:, :, 1:H + 1, 1:Wd + 1] = x
    y = np.zeros((B, W.shape[0], H, Wd))
    for dy in range(3):
        for dx in range(3):
            y += np.einsum("bihw,oi->bohw", xp[:, :, dy:dy + H, dx:dx + Wd], W[:, :, dy, dx])
    return y + b[None, :, None, None]


def conv_backward(x, W, gy):
    """Gradients of conv(x, W, b) given dL/dy. Returns (gx, gW, gb)."""
    B, Ci, H, Wd = x.shape
    xp = np.zeros((B, Ci, H + 2, Wd + 2))
    xp[:, :, 1:H + 1, 1:Wd + 1] = x
    gxp = np.zeros_like(xp)
    gW = np.zeros_like(W)
    for dy in range(3):
        for dx in range(3):
            gW[:, :, dy, dx] = np.einsum("bohw,bihw->oi", gy, xp[:, :, dy:dy + H, dx:dx + Wd])
            gxp[:, :, dy:dy + H, dx:dx + Wd] += np.einsum("bohw,oi->bihw", gy, W[:, :, dy, dx])
    return gxp[:, :, 1:H + 1, 1:Wd + 1], gW, gy.sum(axis=(0, 2, 3))


def forward(theta, x):
    """Return (y, cache) for images x [B][nz][nx]."""
    p = unpack(theta)
    x4 = np.asarray(x, dtype=float)[:, None]
    z1 = conv(x4, p["W1"], p["b1"])
    a1 = np.maximum(z1, 0)
    z2 = conv(a1, p["W2"], p["b2"])
    a2 = np.maximum(z2, 0)
    z3 = conv(a2, p["W3"], p["b3"])
    a3 = np.maximum(z3, 0)
    n = conv(a3, p["W4"], p["b4"])
    y = x4 + n
    return y[:, 0], (x4, z1, a1, z2, a2, z3, a3)


def loss_and_grad(theta, x, t):
    """Return (MSE loss, gradient vector) for images x and targets t [B][nz][nx]."""
    p = unpack(theta)
    y, (x4, z1, a1, z2, a2, z3, a3) = forward(theta, x)
    d = y - np.asarray(t, dtype=float)
    loss = float(np.mean(d * d))
    gy = (2.0 / d.size) * d[:, None]
    ga3, gW4, gb4 = conv_backward(a3, p["W4"], gy)
    gz3 = ga3 * (z3 > 0)
    ga2, gW3, gb3 = conv_backward(a2, p["W3"], gz3)
    gz2 = ga2 * (z2 > 0)
    ga1, gW2, gb2 = conv_backward(a1, p["W2"], gz2)
    gz1 = ga1 * (z1 > 0)
    _, gW1, gb1 = conv_backward(x4, p["W1"], gz1)
    g = pack({"W1": gW1, "b1": gb1, "W2": gW2, "b2": gb2, "W3": gW3, "b3": gb3, "W4": gW4, "b4": gb4})
    return loss, g


def adam_step(theta, m, v, g, k, lr=1e-3, beta1=0.9, beta2=0.999, eps=1e-8):
    """One Adam update at step k (1-based). Returns (theta, m, v)."""
    m = beta1 * m + (1 - beta1) * g
    v = beta2 * v + (1 - beta2) * g * g
    mh = m / (1 - beta1 ** k)
    vh = v / (1 - beta2 ** k)
    return theta - lr * mh / (np.sqrt(vh) + eps), m, v
