"""Plain numpy reference of the screening network (test infrastructure only).

16 -> 64 -> 64 -> 1 multilayer perceptron with SiLU activations, evaluated in float64 with the
weights rounded to BF16 (round to nearest even) as the library's forward pass uses them.  Inputs
are standardised by (x - mean)/sd.  Loss: sum_s w_s (y_s - t_s)^2 / n, w_s = under_weight where
y_s < t_s.  The gradient is taken with respect to the weights as used (BF16-rounded values),
which is the gradient the library applies to its FP32 master weights.

Parameter layout: W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3[1].  Initial weights are a
seeded input drawn by the shared input generators (paper_2404_16245_gb300.workloads), not part of
this reference.
"""
from __future__ import annotations

import numpy as np

IN, H = 16, 64
NPARAM = H * IN + H + H * H + H + H + 1


def bf16_round(w) -> np.ndarray:
    """float32 values rounded to the nearest BF16 value (ties to even), returned as float64."""
    f = np.asarray(w, dtype=np.float32)
    bits = f.view(np.uint32).astype(np.uint64)
    lsb = (bits >> 16) & 1
    rounded = ((bits + 0x7FFF + lsb) >> 16) << 16
    return rounded.astype(np.uint32).view(np.float32).astype(np.float64)


def unpack(p):
    p = np.asarray(p, dtype=np.float64)
    o = 0
    W1 = p[o:o + H * IN].reshape(H, IN); o += H * IN
    b1 = p[o:o + H]; o += H
    W2 = p[o:o + H * H].reshape(H, H); o += H * H
    b2 = p[o:o + H]; o += H
    W3 = p[o:o + H]; o += H
    b3 = p[o]
    return W1, b1, W2, b2, W3, b3


def silu(z):
    return z / (1.0 + np.exp(-z))


def silu_grad(z):
    s = 1.0 / (1.0 + np.exp(-z))
    return s * (1.0 + z * (1.0 - s))


def forward(params, X, mean, sd, quantize=True):
    p = bf16_round(params) if quantize else np.asarray(params, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(p)
    x = (np.asarray(X, dtype=np.float64) - mean) / sd
    z1 = x @ W1.T + b1
    a1 = silu(z1)
    z2 = a1 @ W2.T + b2
    a2 = silu(z2)
    y = a2 @ W3 + b3
    return y, (x, z1, a1, z2, a2)


def loss_and_grad(params, X, T, mean, sd, under_weight=1.0, quantize=True):
    """(loss, gradient[NPARAM]) by backpropagation written out layer by layer."""
    p = bf16_round(params) if quantize else np.asarray(params, dtype=np.float64)
    W1, b1, W2, b2, W3, b3 = unpack(p)
    y, (x, z1, a1, z2, a2) = forward(p, X, mean, sd, quantize=False)
    n = len(y)
    r = y - np.asarray(T, dtype=np.float64)
    w = np.where(r < 0, under_weight, 1.0)
    loss = float(np.sum(w * r * r) / n)
    dy = 2.0 * w * r / n                       # d loss / d y
    gW3 = a2.T @ dy
    gb3 = np.sum(dy)
    dz2 = np.outer(dy, W3) * silu_grad(z2)     # d loss / d z2
    gW2 = dz2.T @ a1
    gb2 = dz2.sum(axis=0)
    dz1 = (dz2 @ W2) * silu_grad(z1)           # d loss / d z1
    gW1 = dz1.T @ x
    gb1 = dz1.sum(axis=0)
    g = np.concatenate([gW1.ravel(), gb1, gW2.ravel(), gb2, gW3, [gb3]])
    return loss, g
