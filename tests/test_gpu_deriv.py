"""Derivative integrals against the oracle: dV/d(basis-function centre) and the field integrals of the nuclei.

The oracle differentiates Cartesian Gaussians directly (raised and lowered exponents, McMurchie-Davidson);
the library differentiates the Gaussian product and raises the one-centre integral of Eq. 12 by one order
(Eq. 3's l +- 1).  Bar per element: |got - ref| <= 1e-11 |ref| + 1e-13 max|ref| over the component's matrix
(derivative elements mix terms of opposite sign whose size is set by the largest elements, so the absolute
part scales with the matrix)."""
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


def check(got, ref, what):
    for X in range(3):
        scale = max(float(np.max(np.abs(ref[X]))), 1e-300)
        excess = np.abs(got[X] - ref[X]) - (1e-11 * np.abs(ref[X]) + 1e-13 * scale)
        if np.any(excess > 0):
            i = np.unravel_index(np.argmax(excess), excess.shape)
            raise AssertionError(f"{what}[{X}]: {int(np.sum(excess > 0))} out of tolerance; worst at {i}: "
                                 f"got {got[X][i]!r} ref {ref[X][i]!r} (scale {scale:.3e})")


def run(shgo, basis, C, Z, field=False):
    B = shgo.Basis(basis)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    fn = shgo.nuclear_field if field else shgo.nuclear_attraction_deriv
    out = fn(B, Cd, Zd).cpu().numpy()
    B.close()
    return out


def every_class_basis(seed, max_prim=2):
    ls = list(range(9)) * 2
    rng = np.random.default_rng(seed)
    sites = rng.uniform(0, 2.5, (3, 3))
    exps = np.exp(rng.uniform(np.log(0.2), np.log(8.0), len(ls) * max_prim))
    return W.make_basis(ls, [max_prim] * len(ls), exps, rng.uniform(0.2, 1, len(ls) * max_prim),
                        [sites[i % 3] for i in range(len(ls))]), sites


def test_deriv_small_contracted_basis(shgo):
    basis = W.random_basis(61, 12, 4, max_prim=3, box=3.0, exp_lo=0.1, exp_hi=30.0, n_sites=5)
    C, Z = W.random_nuclei(62, 7, box=3.0)
    C[0] = np.asarray(basis["xyz"]).reshape(-1, 3)[0]  # a nucleus on a basis centre
    got = run(shgo, basis, C, Z)
    check(got, oracle.nuclear_deriv(basis, C, Z, threads=THREADS, precision="ld"), "dV/dA")


def test_deriv_every_class_up_to_l8(shgo):
    basis, sites = every_class_basis(63)
    rng = np.random.default_rng(64)
    C = np.vstack([rng.uniform(-1.0, 3.5, (4, 3)), sites[1:2]])
    Z = rng.uniform(0.5, 8.0, len(C))
    got = run(shgo, basis, C, Z)
    check(got, oracle.nuclear_deriv(basis, C, Z, threads=THREADS, precision="ld"), "dV/dA (l <= 8)")


def test_field_every_class_up_to_l8(shgo):
    basis, sites = every_class_basis(65)
    rng = np.random.default_rng(66)
    C = np.vstack([rng.uniform(-1.0, 3.5, (4, 3)), sites[2:3]])
    Z = rng.uniform(0.5, 8.0, len(C))
    got = run(shgo, basis, C, Z, field=True)
    check(got, oracle.nuclear_field(basis, C, Z, threads=THREADS, precision="ld"), "field (l <= 8)")
    for X in range(3):
        assert np.array_equal(got[X], got[X].T)


def test_field_small_contracted_basis_and_per_nucleus(shgo):
    basis = W.random_basis(67, 10, 5, max_prim=3, box=3.0, exp_lo=0.1, exp_hi=40.0, n_sites=4)
    C, Z = W.random_nuclei(68, 5, box=3.0)
    got = run(shgo, basis, C, Z, field=True)
    check(got, oracle.nuclear_field(basis, C, Z, threads=THREADS, precision="ld"), "field")
    B = shgo.Basis(basis)
    per = shgo.field_matrices(B, torch.tensor(C, device="cuda")).cpu().numpy()
    B.close()
    for k in range(len(Z)):
        check(per[k], oracle.nuclear_field(basis, C[k:k + 1], np.ones(1), threads=THREADS, precision="ld"),
              f"field of nucleus {k}")
    total = np.einsum("k,kxab->xab", Z, per)
    assert np.max(np.abs(total - got)) <= 1e-12 * np.max(np.abs(got))


def test_translational_invariance_on_the_device(shgo):
    # moving the basis and the nuclei together leaves V unchanged: D + D^T + field = 0
    basis = W.random_basis(69, 14, 6, max_prim=2, box=4.0, exp_lo=0.1, exp_hi=20.0, n_sites=5)
    C, Z = W.random_nuclei(70, 9, box=4.0)
    D = run(shgo, basis, C, Z)
    F = run(shgo, basis, C, Z, field=True)
    for X in range(3):
        assert np.max(np.abs(D[X] + D[X].T + F[X])) <= 1e-12 * np.max(np.abs(D[X]))


def test_deriv_degenerate_inputs(shgo):
    basis = W.random_basis(71, 4, 2, max_prim=2, box=2.0)
    B = shgo.Basis(basis)
    none = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
    out = torch.full((3, B.nbf, B.nbf), float("nan"), dtype=torch.float64, device="cuda")
    shgo.nuclear_attraction_deriv(B, none, torch.zeros(0, dtype=torch.float64, device="cuda"), out=out)
    assert torch.count_nonzero(out).item() == 0
    shgo.nuclear_field(B, none, torch.zeros(0, dtype=torch.float64, device="cuda"), out=out)
    assert torch.count_nonzero(out).item() == 0
    B.close()
    # one s shell pair on one centre with the nucleus there: stationary by symmetry
    s = W.make_basis([0, 0], [1, 1], [0.8, 2.0], [1.0, 1.0], [np.zeros(3), np.zeros(3)])
    got = run(shgo, s, np.zeros((1, 3)), np.ones(1))
    assert np.max(np.abs(got)) <= 1e-14


def test_deriv_repeatable(shgo):
    # fixed summation order: two calls give the same bits
    basis = W.random_basis(72, 10, 5, max_prim=2, box=3.0, n_sites=4)
    C, Z = W.random_nuclei(73, 6, box=3.0)
    B = shgo.Basis(basis)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    a = shgo.nuclear_attraction_deriv(B, Cd, Zd).cpu().numpy()
    b = shgo.nuclear_attraction_deriv(B, Cd, Zd).cpu().numpy()
    B.close()
    assert np.array_equal(a, b)


def test_deriv_is_fp64_whatever_the_basis_precision(shgo):
    # the derivative path runs the FP64 coupling kernel for every basis: an FP32-bulk basis gives the same bits
    basis = W.random_basis(74, 8, 4, max_prim=2, box=3.0, n_sites=3)
    C, Z = W.random_nuclei(75, 5, box=3.0)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    B64 = shgo.Basis(basis)
    B32 = shgo.Basis(basis, precision=shgo.SHGO_PREC_FP32_BULK)
    for fn in (shgo.nuclear_attraction_deriv, shgo.nuclear_field):
        assert np.array_equal(fn(B64, Cd, Zd).cpu().numpy(), fn(B32, Cd, Zd).cpu().numpy())
    B64.close()
    B32.close()


def test_deriv_rejects_a_batch(shgo):
    mols = [(W.random_basis(76 + k, 3, 2, max_prim=2, box=2.0), 2) for k in range(2)]
    bt = shgo.Batch(mols)
    import ctypes
    c = shgo.shgo_centers(0, None)
    for fn in (shgo._lib.shgo_nuclear_attraction_deriv, shgo._lib.shgo_nuclear_field):
        assert fn(ctypes.c_void_p(bt.handle), ctypes.byref(c), None, None, None) == 1  # SHGO_ERR_INVALID_ARG
    bt.close()


def _shell_of_function(basis):
    l = np.asarray(basis["l"])
    return np.repeat(np.arange(len(l)), 2 * l + 1)


def test_gradient_contracts_the_oracle_derivative(shgo):
    # grad[s] = sum_{a in s} sum_b (P_ab + P_ba) dV_ab/dA against the oracle's derivative contracted on the host;
    # bar per component: 1e-11 of the contraction's absolute sum
    basis = W.random_basis(78, 12, 5, max_prim=3, box=3.0, exp_lo=0.1, exp_hi=30.0, n_sites=5)
    C, Z = W.random_nuclei(79, 6, box=3.0)
    n = W.nbf(basis)
    rng = np.random.default_rng(80)
    P = rng.normal(size=(n, n))  # not symmetric: the contraction takes P_ab + P_ba
    B = shgo.Basis(basis)
    g = shgo.nuclear_attraction_gradient(B, torch.tensor(P, device="cuda"), torch.tensor(C, device="cuda"),
                                         torch.tensor(Z, device="cuda")).cpu().numpy()
    B.close()
    D = oracle.nuclear_deriv(basis, C, Z, threads=THREADS, precision="ld")
    W2 = P + P.T
    sh = _shell_of_function(basis)
    for s in range(len(basis["l"])):
        rows = sh == s
        for X in range(3):
            terms = W2[rows, :] * D[X][rows, :]
            assert abs(g[s, X] - terms.sum()) <= 1e-11 * np.abs(terms).sum() + 1e-13, (s, X)


def test_gradient_and_nuclear_forces_sum_to_zero(shgo):
    # E = sum P_ab V_ab is unchanged when basis and nuclei move together: sum_s grad[s] + sum_C Z_C grad phi(C) = 0
    basis = W.random_basis(81, 14, 6, max_prim=2, box=4.0, exp_lo=0.1, exp_hi=20.0, n_sites=5)
    C, Z = W.random_nuclei(82, 8, box=4.0)
    n = W.nbf(basis)
    rng = np.random.default_rng(83)
    p = rng.normal(size=(n, n))
    P = (p + p.T) / 2
    B = shgo.Basis(basis)
    Pd, Cd, Zd = (torch.tensor(x, device="cuda") for x in (P, C, Z))
    g = shgo.nuclear_attraction_gradient(B, Pd, Cd, Zd).cpu().numpy()
    ge = shgo.esp_gradient(B, Pd, Cd).cpu().numpy()
    D = shgo.nuclear_attraction_deriv(B, Cd, Zd).cpu().numpy()
    B.close()
    total = g.sum(axis=0) + (Z[:, None] * ge).sum(axis=0)
    scale = np.abs(g).sum() + np.abs(Z[:, None] * ge).sum()
    assert np.max(np.abs(total)) <= 1e-11 * scale
    # the same as contracting the library's own derivative matrices
    sh = _shell_of_function(basis)
    for s in range(len(basis["l"])):
        rows = sh == s
        for X in range(3):
            terms = (2 * P)[rows, :] * D[X][rows, :]
            assert abs(g[s, X] - terms.sum()) <= 1e-12 * np.abs(terms).sum() + 1e-14


def test_gradient_repeatable_and_degenerate(shgo):
    basis = W.random_basis(84, 10, 4, max_prim=2, box=3.0, n_sites=4)
    C, Z = W.random_nuclei(85, 5, box=3.0)
    n = W.nbf(basis)
    P = torch.tensor(np.random.default_rng(86).normal(size=(n, n)), device="cuda")
    B = shgo.Basis(basis)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    a = shgo.nuclear_attraction_gradient(B, P, Cd, Zd).cpu().numpy()
    b = shgo.nuclear_attraction_gradient(B, P, Cd, Zd).cpu().numpy()
    assert np.array_equal(a, b)
    z = shgo.nuclear_attraction_gradient(B, P, Cd[:0], Zd[:0]).cpu().numpy()
    assert np.count_nonzero(z) == 0
    B.close()


def test_deriv_field_and_gradient_at_benchmark_size(shgo):
    # the benchmark molecule in full (1568 functions, 32 nuclei), in the launch configuration the bench times
    basis, C, Z = W.config2()
    B = shgo.Basis(basis)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    D = shgo.nuclear_attraction_deriv(B, Cd, Zd).cpu().numpy()
    F = shgo.nuclear_field(B, Cd, Zd).cpu().numpy()
    n = B.nbf
    rng = np.random.default_rng(87)
    p = rng.normal(size=(n, n))
    P = (p + p.T) / 2
    g = shgo.nuclear_attraction_gradient(B, torch.tensor(P, device="cuda"), Cd, Zd).cpu().numpy()
    B.close()
    Dref = oracle.nuclear_deriv(basis, C, Z, threads=THREADS)
    check(D, Dref, "dV/dA, benchmark molecule")
    check(F, oracle.nuclear_field(basis, C, Z, threads=THREADS), "field, benchmark molecule")
    sh = _shell_of_function(basis)
    for s in range(len(basis["l"])):
        rows = sh == s
        for X in range(3):
            terms = (2 * P)[rows, :] * Dref[X][rows, :]
            assert abs(g[s, X] - terms.sum()) <= 1e-11 * np.abs(terms).sum() + 1e-13, (s, X)
