"""Pins of the numpy screening-network reference (no GPU): its forward pass against a case
worked out by hand, its backward pass against central finite differences of its own forward pass,
and the BF16 rounding against known values."""
import math

import numpy as np

from oracle import mlp
from paper_2404_16245_gb300 import workloads as W


def test_bf16_rounding_known_values():
    vals = np.array([1.0, 1.00390625, 1.001953125, -3.14159265, 65504.0, 1e-3], dtype=np.float32)
    r = mlp.bf16_round(vals)
    assert r[0] == 1.0
    assert r[1] == 1.0  # 1 + 2^-8 is a tie between 1 and 1 + 2^-7: ties to even
    assert r[2] == 1.0  # below the tie
    assert abs(r[3] - (-3.140625)) < 1e-12
    assert r[4] == 65536.0
    assert abs(r[5] - 1e-3) / 1e-3 < 2 ** -8


def test_backward_matches_finite_differences():
    rng = np.random.default_rng(0)
    X = rng.normal(size=(23, 16))
    T = rng.normal(size=23)
    mean = rng.normal(size=16) * 0.1
    sd = rng.uniform(0.5, 2.0, 16)
    p = W.mlp_init_params(3).astype(np.float64)
    loss, g = mlp.loss_and_grad(p, X, T, mean, sd, under_weight=4.0, quantize=False)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X, T, mean, sd, 4.0, quantize=False)[0]
              - mlp.loss_and_grad(pm, X, T, mean, sd, 4.0, quantize=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])


def _silu_by_tanh(z):
    # z sigma(z) with sigma(z) = (1 + tanh(z / 2)) / 2: an identity independent of the reference's form
    return 0.5 * z * (1.0 + math.tanh(0.5 * z))


def test_forward_hand_computed_two_samples():
    """One path through the network with BF16-exact weights: x_5 -> hidden unit 3 -> hidden unit 7
    -> output.  W1[3][5] = 1, b1[3] = 1; W2[7][3] = 2, b2[7] = -0.5; W3[7] = 0.75, b3 = 0.25; every
    other weight zero.  Standardised sample 1 has x_5 = 2 (raw mean + 2 sd), sample 2 is at the
    mean.  Then z1_3 = 3 (sample 1) or 1 (sample 2), z2_7 = 2 silu(z1_3) - 0.5 and
    y = 0.25 + 0.75 silu(z2_7); silu(0) = 0 on every other unit.  A transposed weight matrix, a
    bias in the wrong slot or a wrong activation changes y."""
    H, IN = mlp.H, mlp.IN
    p = np.zeros(mlp.NPARAM)
    o_b1 = H * IN
    o_W2 = o_b1 + H
    o_b2 = o_W2 + H * H
    o_W3 = o_b2 + H
    o_b3 = o_W3 + H
    p[3 * IN + 5] = 1.0
    p[o_b1 + 3] = 1.0
    p[o_W2 + 7 * H + 3] = 2.0
    p[o_b2 + 7] = -0.5
    p[o_W3 + 7] = 0.75
    p[o_b3] = 0.25
    mean = np.linspace(-1.0, 1.0, IN)
    sd = np.full(IN, 0.5)
    X = np.stack([mean.copy(), mean.copy()])
    X[0, 5] = mean[5] + 2.0 * sd[5]
    y, _ = mlp.forward(p, X, mean, sd)
    want = [0.25 + 0.75 * _silu_by_tanh(2.0 * _silu_by_tanh(z1) - 0.5) for z1 in (3.0, 1.0)]
    assert abs(y[0] - want[0]) < 1e-14 and abs(y[1] - want[1]) < 1e-14, (y, want)
    # sample 1 by the closed form silu(3) = 3 / (1 + e^-3): y = 0.25 + 0.75 silu(5.357...)
    z2 = 6.0 / (1.0 + math.exp(-3.0)) - 0.5
    assert abs(y[0] - (0.25 + 0.75 * z2 / (1.0 + math.exp(-z2)))) < 1e-14
