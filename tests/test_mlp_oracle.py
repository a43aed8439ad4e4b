"""Pins of the numpy screening-network reference (no GPU): its backward pass against central
finite differences of its own forward pass, and the BF16 rounding against known values."""
import numpy as np

from oracle import mlp


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
    p = mlp.init_params(3).astype(np.float64)
    loss, g = mlp.loss_and_grad(p, X, T, mean, sd, under_weight=4.0, quantize=False)
    idx = rng.choice(mlp.NPARAM, 60, replace=False)
    h = 1e-6
    for i in idx:
        pp = p.copy(); pp[i] += h
        pm = p.copy(); pm[i] -= h
        fd = (mlp.loss_and_grad(pp, X, T, mean, sd, 4.0, quantize=False)[0]
              - mlp.loss_and_grad(pm, X, T, mean, sd, 4.0, quantize=False)[0]) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(g[i])) + 1e-9, (i, fd, g[i])
