"""The elementwise bound behind primitive-pair skipping, against the oracle (CPU).

For one primitive pair (normalised primitives of exponents alpha, beta, coefficients c_i, c_j) and any
nucleus C, every element of the pair's block satisfies
    |<a_i|1/|r - C||b_j>| <= |c_i c_j| K_AB 4 pi int_0^inf (r + |PA|)^la (r + |PB|)^lb e^{-p r^2} r dr
(|S_lm(r)| <= |r|^l, |r_A| <= r_P + |PA|, and the potential of a non-negative radial density peaks at
its centre), and every overlap element by the same integral with r^2 dr.  Here the oracle's values
for random pairs and nuclei must never exceed the bound."""
import math

import numpy as np
import pytest

import oracle
from paper_2404_16245_gb300 import workloads as W


def bound(la, lb, a, b, p, r_power):
    s = 0.0
    for i in range(la + 1):
        for j in range(lb + 1):
            n = i + j + r_power
            s += math.comb(la, i) * math.comb(lb, j) * a ** (la - i) * b ** (lb - j) * \
                math.gamma((n + 1) / 2) / (2 * p ** ((n + 1) / 2))
    return 4 * math.pi * s


@pytest.mark.parametrize("seed", range(6))
def test_bound_holds_for_random_primitive_pairs(seed):
    rng = np.random.default_rng(seed)
    for _ in range(12):
        la, lb = (int(x) for x in rng.integers(0, 5, 2))
        al, be = np.exp(rng.uniform(np.log(0.05), np.log(50.0), 2))
        A = rng.uniform(-1, 1, 3)
        Bc = A + rng.normal(size=3) * rng.uniform(0, 4)
        basis = W.make_basis([la, lb], [1, 1], [al, be], [1.0, 1.0], [A, Bc])
        C = A + rng.normal(size=(3, 3)) * rng.uniform(0, 5)
        p = al + be
        R = float(np.linalg.norm(Bc - A))
        K = math.exp(-al * be / p * R * R)
        # the oracle renormalises one-primitive shells to unit norm: c = N(l, alpha)
        c = oracle.prim_norm(la, al) * oracle.prim_norm(lb, be)
        na = 2 * la + 1
        bnuc = c * K * bound(la, lb, be / p * R, al / p * R, p, 1)
        bovl = c * K * bound(la, lb, be / p * R, al / p * R, p, 2)
        S = oracle.overlap(basis)[:na, na:]
        assert np.max(np.abs(S)) <= bovl * (1 + 1e-12)
        for Cc in C:
            V = oracle.nuclear_attraction(basis, Cc[None, :], np.ones(1))[:na, na:]
            assert np.max(np.abs(V)) <= bnuc * (1 + 1e-12), (la, lb, al, be, R)
