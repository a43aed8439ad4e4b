"""Electrostatic potential of a density at arbitrary points, against the oracle.

phi[k] = sum_ab D_ab <a|1/|r - x_k||b>: the oracle evaluates the attraction matrix of a unit charge
at each point (extended-precision build) and contracts it with D.  Bar per point:
|phi - phi_ref| <= 1e-11 sum_ab |D_ab V_ab(x_k)| + 1e-13 (the natural scale of the contraction)."""
import os

import numpy as np
import pytest

import oracle
from paper_2404_16245_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def shgo():
    from paper_2404_16245_gb300 import shgo as mod
    return mod


def density(n, seed):
    rng = np.random.default_rng(seed)
    d = rng.normal(size=(n, n))
    return (d + d.T) / 2


def check(shgo, basis, D, X):
    B = shgo.Basis(basis)
    phi = shgo.esp(B, torch.tensor(D, device="cuda"), torch.tensor(X, device="cuda")).cpu().numpy()
    B.close()
    for k, x in enumerate(X):
        V = oracle.nuclear_attraction(basis, x[None, :], np.ones(1), threads=THREADS, precision="ld")
        ref = float(np.sum(D * V))
        scale = float(np.sum(np.abs(D * V)))
        assert abs(phi[k] - ref) <= 1e-11 * scale + 1e-13, (k, phi[k], ref, scale)
    return phi


def test_small_contracted_basis(shgo):
    basis = W.random_basis(51, 12, 4, max_prim=3, box=3.0, exp_lo=0.1, exp_hi=30.0)
    rng = np.random.default_rng(52)
    X = np.vstack([rng.uniform(-1.0, 4.0, (20, 3)), basis["xyz"][:3]])  # three points on shell centres
    check(shgo, basis, density(W.nbf(basis), 53), X)


def test_every_class_up_to_l8(shgo):
    ls = list(range(9)) * 2
    rng = np.random.default_rng(54)
    sites = rng.uniform(0, 2.5, (3, 3))
    exps = np.exp(rng.uniform(np.log(0.2), np.log(8.0), len(ls) * 2))
    basis = W.make_basis(ls, [2] * len(ls), exps, rng.uniform(0.2, 1, len(ls) * 2),
                         [sites[i % 3] for i in range(len(ls))])
    X = rng.uniform(-1.0, 3.5, (9, 3))
    check(shgo, basis, density(W.nbf(basis), 55), X)


def test_ragged_point_chunks_and_far_points(shgo):
    basis = W.random_basis(56, 8, 3, max_prim=2)
    rng = np.random.default_rng(57)
    X = np.vstack([rng.uniform(0, 4, (33, 3)), [[40.0, -3.0, 2.0], [1.0, 30.0, -25.0]]])
    check(shgo, basis, density(W.nbf(basis), 58), X)


def test_potential_is_the_charge_derivative_of_V(shgo):
    # sum_ab D_ab V_ab(charges q) = sum_k q_k phi_k, with V from the library's own attraction kernels
    basis, C, Z = W.config2(n_atoms=8)
    D = density(W.nbf(basis), 59)
    B = shgo.Basis(basis)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    V = shgo.nuclear_attraction(B, Cd, Zd).cpu().numpy()
    phi = shgo.esp(B, torch.tensor(D, device="cuda"), Cd).cpu().numpy()
    B.close()
    lhs, rhs = float(np.sum(D * V)), float(np.dot(Z, phi))
    assert abs(lhs - rhs) <= 1e-11 * float(np.sum(np.abs(D * V))), (lhs, rhs)


def test_no_points(shgo):
    basis = W.random_basis(60, 4, 2)
    B = shgo.Basis(basis)
    phi = shgo.esp(B, torch.zeros((B.nbf, B.nbf), dtype=torch.float64, device="cuda"),
                   torch.zeros((0, 3), dtype=torch.float64, device="cuda"))
    assert phi.numel() == 0
    B.close()


def check_gradient(shgo, basis, D, X):
    B = shgo.Basis(basis)
    g = shgo.esp_gradient(B, torch.tensor(D, device="cuda"), torch.tensor(X, device="cuda")).cpu().numpy()
    B.close()
    for k, x in enumerate(X):
        F = oracle.nuclear_field(basis, x[None, :], np.ones(1), threads=THREADS, precision="ld")
        for c in range(3):
            ref = float(np.sum(D * F[c]))
            scale = float(np.sum(np.abs(D * F[c])))
            assert abs(g[k, c] - ref) <= 1e-11 * scale + 1e-13, (k, c, g[k, c], ref, scale)


def test_gradient_small_contracted_basis(shgo):
    basis = W.random_basis(61, 10, 4, max_prim=3, box=3.0, exp_lo=0.1, exp_hi=30.0)
    rng = np.random.default_rng(62)
    X = np.vstack([rng.uniform(-1.0, 4.0, (18, 3)), basis["xyz"][:2]])
    check_gradient(shgo, basis, density(W.nbf(basis), 63), X)


def test_gradient_every_class_up_to_l8(shgo):
    ls = list(range(9)) * 2
    rng = np.random.default_rng(64)
    sites = rng.uniform(0, 2.5, (3, 3))
    exps = np.exp(rng.uniform(np.log(0.2), np.log(8.0), len(ls) * 2))
    basis = W.make_basis(ls, [2] * len(ls), exps, rng.uniform(0.2, 1, len(ls) * 2),
                         [sites[i % 3] for i in range(len(ls))])
    X = rng.uniform(-1.0, 3.5, (5, 3))
    check_gradient(shgo, basis, density(W.nbf(basis), 65), X)


def test_gradient_ragged_chunks(shgo):
    basis = W.random_basis(66, 8, 3, max_prim=2)
    rng = np.random.default_rng(67)
    X = np.vstack([rng.uniform(0, 4, (17, 3)), [[25.0, -3.0, 2.0]]])
    check_gradient(shgo, basis, density(W.nbf(basis), 68), X)
