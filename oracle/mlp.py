"""FP64 reference of the surrogate's network: 1 -> H -> H -> n_out, tanh hidden layers.

Parameter vector layout: W1[H], b1[H], W2[H][H], b2[H], W3[n_out][H], b3[n_out].
Loss: mean over all B x n_out outputs of (y - t)^2.  Backward pass by the chain rule, written
out layer by layer (no automatic differentiation).
"""
from __future__ import annotations

import numpy as np


def unpack(p, H, n_out):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H]; o += H
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + n_out * H].reshape(n_out, H); o += n_out * H
    b3 = p[o:o + n_out]; o += n_out
    assert o == len(p)
    return W1, b1, W2, b2, W3, b3


def forward(p, H, n_out, x):
    W1, b1, W2, b2, W3, b3 = unpack(p, H, n_out)
    x = np.asarray(x, dtype=np.float64)
    h1 = np.tanh(np.outer(x, W1) + b1)
    h2 = np.tanh(h1 @ W2.T + b2)
    return h2 @ W3.T + b3, (h1, h2)


def loss_grad(p, H, n_out, x, t):
    W1, b1, W2, b2, W3, b3 = unpack(p, H, n_out)
    x = np.asarray(x, dtype=np.float64)
    y, (h1, h2) = forward(p, H, n_out, x)
    n = y.size
    L = np.sum((y - t) ** 2) / n
    dy = 2.0 * (y - t) / n                     # (B, n_out)
    gW3 = dy.T @ h2
    gb3 = dy.sum(0)
    dz2 = (dy @ W3) * (1.0 - h2 ** 2)          # (B, H)
    gW2 = dz2.T @ h1
    gb2 = dz2.sum(0)
    dz1 = (dz2 @ W2) * (1.0 - h1 ** 2)
    gW1 = dz1.T @ x
    gb1 = dz1.sum(0)
    g = np.concatenate([gW1, gb1, gW2.ravel(), gb2, gW3.ravel(), gb3])
    return L, g


def n_params(H, n_out):
    return H + H + H * H + H + n_out * H + n_out
