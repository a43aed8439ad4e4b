"""Seeded synthetic inputs shared by the tests and the benchmark.

This module only draws random numbers and lays them out; it holds none of the integral
arithmetic.  A basis is a dict of numpy arrays:

    l      int32[n_shells]        angular momentum of each shell
    nprim  int32[n_shells]        primitives per shell
    exps   float64[sum(nprim)]    Gaussian exponents, shell after shell
    coefs  float64[sum(nprim)]    contraction coefficients of normalised primitives
    xyz    float64[n_shells, 3]   shell centres (bohr)

Nuclei are ``centers`` float64[n, 3] (bohr) and ``charges`` float64[n].

The paper measures on no public benchmark; every workload below is synthetic with the
shapes and distributions of the five named configurations.  Seeds follow
``seed = 1000 * config + replica``.
"""
from __future__ import annotations

import numpy as np


def _rng(seed: int) -> np.random.Generator:
    return np.random.Generator(np.random.PCG64(seed))


def _log_uniform(rng, lo, hi, size):
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size))


def make_basis(l_list, nprim_list, exps, coefs, xyz) -> dict:
    return {
        "l": np.asarray(l_list, dtype=np.int32),
        "nprim": np.asarray(nprim_list, dtype=np.int32),
        "exps": np.asarray(exps, dtype=np.float64),
        "coefs": np.asarray(coefs, dtype=np.float64),
        "xyz": np.asarray(xyz, dtype=np.float64).reshape(-1, 3),
    }


def nbf(basis) -> int:
    return int(np.sum(2 * basis["l"] + 1))


def shell_pairs(basis) -> int:
    n = len(basis["l"])
    return n * (n + 1) // 2


def molecule(rng, n_atoms, box, z_lo, z_hi, shells_per_atom, nprim_of, exp_lo, exp_hi, coef_lo=0.1, coef_hi=1.0):
    """Atoms uniform in [0, box]^3; each atom carries the shells `shells_per_atom(Z)` (list of l);
    `nprim_of(rng)` draws the primitive count of one shell."""
    pos = rng.uniform(0.0, box, (n_atoms, 3))
    Z = rng.integers(z_lo, z_hi + 1, n_atoms).astype(np.float64)
    ls, nps, ex, co, xyz = [], [], [], [], []
    for a in range(n_atoms):
        for l in shells_per_atom(int(Z[a])):
            k = int(nprim_of(rng))
            ls.append(l)
            nps.append(k)
            ex.extend(_log_uniform(rng, exp_lo, exp_hi, k))
            co.extend(rng.uniform(coef_lo, coef_hi, k) if k > 1 else [1.0])
            xyz.append(pos[a])
    return make_basis(ls, nps, ex, co, xyz), pos, Z


def config1(replica: int = 0):
    """Plain FP64: 4 atoms uniform in a 6 bohr cube, Z ~ U{1..8}; every atom carries l = 0, 1, 2
    shells of 3 primitives, exponents log-uniform [0.1, 100], coefficients U[0.1, 1]."""
    rng = _rng(1000 * 1 + replica)
    pos = rng.uniform(0.0, 6.0, (4, 3))
    Z = rng.integers(1, 9, 4).astype(np.float64)
    ls, nps, ex, co, xyz = [], [], [], [], []
    for a in range(4):
        for l in (0, 1, 2):
            ls.append(l)
            nps.append(3)
            ex.extend(_log_uniform(rng, 0.1, 100.0, 3))
            co.extend(rng.uniform(0.1, 1.0, 3))
            xyz.append(pos[a])
    return make_basis(ls, nps, ex, co, xyz), pos, Z


def config2(replica: int = 0, n_atoms: int = 32, lmax: int = 6):
    """High l, FP64: 32 atoms in a 20 bohr cube, Z ~ U{1..10}; every atom carries one
    uncontracted shell per l = 0..6, exponents log-uniform [0.05, 50]."""
    rng = _rng(1000 * 2 + replica)
    pos = rng.uniform(0.0, 20.0, (n_atoms, 3))
    Z = rng.integers(1, 11, n_atoms).astype(np.float64)
    ls, nps, ex, co, xyz = [], [], [], [], []
    for a in range(n_atoms):
        for l in range(lmax + 1):
            ls.append(l)
            nps.append(1)
            ex.append(float(_log_uniform(rng, 0.05, 50.0, 1)[0]))
            co.append(1.0)
            xyz.append(pos[a])
    return make_basis(ls, nps, ex, co, xyz), pos, Z


H_SHELLS = [0, 0, 0, 1, 1, 2]                                   # 3s2p1d
HEAVY_SHELLS = [0] * 5 + [1] * 4 + [2] * 3 + [3] * 2 + [4]      # 5s4p3d2f1g


def config3_molecule(rng):
    """One molecule of the batched workload: N = clip(round(30 exp(0.5 z)), 8, 200) atoms at
    0.05 atoms/bohr^3; 40% H (Z=1, 3s2p1d), the rest Z ~ U{6..9} with 5s4p3d2f1g; 1..8
    primitives per shell, exponents log-uniform [0.05, 5000]."""
    n = int(np.clip(np.round(30.0 * np.exp(0.5 * rng.standard_normal())), 8, 200))
    box = (n / 0.05) ** (1.0 / 3.0)
    pos = rng.uniform(0.0, box, (n, 3))
    is_h = rng.uniform(size=n) < 0.4
    Z = np.where(is_h, 1, rng.integers(6, 10, n)).astype(np.float64)
    ls, nps, ex, co, xyz = [], [], [], [], []
    for a in range(n):
        for l in (H_SHELLS if Z[a] == 1 else HEAVY_SHELLS):
            k = int(rng.integers(1, 9))
            ls.append(l)
            nps.append(k)
            ex.extend(_log_uniform(rng, 0.05, 5000.0, k))
            co.extend(rng.uniform(0.1, 1.0, k) if k > 1 else [1.0])
            xyz.append(pos[a])
    return make_basis(ls, nps, ex, co, xyz), pos, Z


def config3(n_molecules: int = 2000, replica: int = 0):
    """The batched workload: a list of (basis, centers, charges), one per molecule."""
    rng = _rng(1000 * 3 + replica)
    return [config3_molecule(rng) for _ in range(n_molecules)]


def config4(replica: int = 0, n_atoms: int = 5000):
    """Learned screening: n_atoms uniform in a cube at 0.1 atoms/bohr^3, Z ~ U{1..9}; every
    atom carries 4s3p2d1f with 1..6 primitives, exponents log-uniform [0.05, 5000]."""
    rng = _rng(1000 * 4 + replica)
    box = (n_atoms / 0.1) ** (1.0 / 3.0)
    shells = [0] * 4 + [1] * 3 + [2] * 2 + [3]
    return molecule(rng, n_atoms, box, 1, 9, lambda Z: shells, lambda r: r.integers(1, 7), 0.05, 5000.0)


def config5_arrays(n_triples: int, replica: int = 0, lmax: int = 8):
    """Precision sweep as arrays: independent primitive triples.  la, lb ~ U{0..lmax}; exponents
    log-uniform [0.01, 1000]; A = 0, B = |AB| u, |AB| ~ U[0, 15]; the nucleus sits at distance
    |PC| ~ U[0, 15] in a uniform direction v from the exponent-weighted centre of A and B;
    Z ~ U{1..20}.  Returns (la, lb, alpha, beta, B [n, 3], C [n, 3], Z)."""
    rng = _rng(1000 * 5 + replica)
    n = int(n_triples)
    la = rng.integers(0, lmax + 1, n)
    lb = rng.integers(0, lmax + 1, n)
    lo, hi = np.log(0.01), np.log(1000.0)
    alpha = np.exp(rng.uniform(lo, hi, n))
    beta = np.exp(rng.uniform(lo, hi, n))
    u = rng.standard_normal((n, 3))
    u /= np.linalg.norm(u, axis=1, keepdims=True)
    v = rng.standard_normal((n, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    B = rng.uniform(0.0, 15.0, n)[:, None] * u
    centre = (beta / (alpha + beta))[:, None] * B
    C = centre + rng.uniform(0.0, 15.0, n)[:, None] * v
    Z = rng.integers(1, 21, n).astype(np.float64)
    return la, lb, alpha, beta, B, C, Z


def config5(n_triples: int, replica: int = 0, lmax: int = 8):
    """The precision-sweep triples of config5_arrays as a list of (basis with two one-primitive shells,
    centers [1, 3], charges [1])."""
    la, lb, alpha, beta, B, C, Z = config5_arrays(n_triples, replica, lmax)
    return [(make_basis([int(la[t]), int(lb[t])], [1, 1], [alpha[t], beta[t]], [1.0, 1.0], [np.zeros(3), B[t]]),
             C[t].reshape(1, 3), np.array([Z[t]])) for t in range(len(la))]


def random_basis(seed: int, n_shells: int, lmax: int, max_prim: int = 4, box: float = 4.0,
                 exp_lo: float = 0.1, exp_hi: float = 20.0, n_sites: int | None = None):
    """Small mixed basis for parity tests: shells on a few sites, l ~ U{0..lmax}, 1..max_prim
    primitives each."""
    rng = _rng(seed)
    n_sites = n_sites or max(1, n_shells // 3)
    sites = rng.uniform(0.0, box, (n_sites, 3))
    ls, nps, ex, co, xyz = [], [], [], [], []
    for s in range(n_shells):
        k = int(rng.integers(1, max_prim + 1))
        ls.append(int(rng.integers(0, lmax + 1)))
        nps.append(k)
        ex.extend(_log_uniform(rng, exp_lo, exp_hi, k))
        co.extend(rng.uniform(0.1, 1.0, k) if k > 1 else [1.0])
        xyz.append(sites[s % n_sites])
    return make_basis(ls, nps, ex, co, xyz)


def random_nuclei(seed: int, n: int, box: float = 4.0, z_lo: int = 1, z_hi: int = 10):
    rng = _rng(seed)
    return rng.uniform(0.0, box, (n, 3)), rng.integers(z_lo, z_hi + 1, n).astype(np.float64)


MLP_IN, MLP_H = 16, 64


def mlp_init_params(seed: int) -> np.ndarray:
    """Seeded initial weights of the 16-64-64-1 screening network (float32, the layout of
    include/shgo_mlp.h: W1[64][16], b1[64], W2[64][64], b2[64], W3[64], b3): He-style normal draws
    with standard deviation sqrt(2 / fan_in) for the two SiLU layers, sqrt(1 / fan_in) for the
    linear output, zero biases."""
    rng = np.random.default_rng(seed)
    W1 = rng.normal(0, np.sqrt(2.0 / MLP_IN), (MLP_H, MLP_IN))
    W2 = rng.normal(0, np.sqrt(2.0 / MLP_H), (MLP_H, MLP_H))
    W3 = rng.normal(0, np.sqrt(1.0 / MLP_H), MLP_H)
    p = np.concatenate([W1.ravel(), np.zeros(MLP_H), W2.ravel(), np.zeros(MLP_H), W3, [0.0]])
    return p.astype(np.float32)
