"""Four-centre electron-repulsion integrals (ab|cd) (Eqs. 13-15) on the GPU against the CPU oracle, element
by element.

Same bar as the attraction integrals: |x - y| <= 1e-13 + 1e-11 |y| per element, judged by the oracle
(McMurchie-Davidson over four centres, pinned in test_oracle_eri_pins.py; its double build is certified
against the extended-precision build there).  At any size the tensor has the eight-fold permutational
symmetry exactly (each unique quartet is computed once) and is a positive semi-definite metric over
orbital pairs."""
import os

import numpy as np
import pytest

import oracle
from paper_2404_16245_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")

THREADS = os.cpu_count() or 1


@pytest.fixture(scope="module")
def shgo():
    from paper_2404_16245_gb300 import shgo as mod
    return mod


def gpu_E(shgo, basis):
    B = shgo.Basis(basis)
    E = shgo.eri(B)
    torch.cuda.synchronize()
    out = E.cpu().numpy()
    B.close()
    return out


def ref_E(basis, precision="f64"):
    return oracle.eri(basis, threads=THREADS, precision=precision)


def assert_eightfold(E):
    assert np.array_equal(E, E.transpose(1, 0, 2, 3))
    assert np.array_equal(E, E.transpose(0, 1, 3, 2))
    assert np.array_equal(E, E.transpose(2, 3, 0, 1))


def test_config1(shgo):
    basis, _, _ = W.config1()
    E = gpu_E(shgo, basis)
    parity.check(E, ref_E(basis), what="eri config1")
    assert_eightfold(E)


@pytest.mark.parametrize("seed,lmax,nshell", [(11, 4, 6), (12, 3, 9), (13, 2, 14)])
def test_mixed_classes_contracted(shgo, seed, lmax, nshell):
    basis = W.random_basis(seed, nshell, lmax, max_prim=3, box=3.0, exp_lo=0.1, exp_hi=30.0, n_sites=nshell)
    parity.check(gpu_E(shgo, basis), ref_E(basis), what=f"eri seed {seed}")


@pytest.mark.parametrize("n_sites", [1, 2, 3])
def test_every_class_up_to_l4_shared_centres(shgo, n_sites):
    """Shells l = 0..4 on one, two or three centres: every class (ab|cd) up to (gg|gg), including the
    degenerate geometries A = B, C = D and P = Q (S_LM(0) = delta_L0, u = 0)."""
    ls = [4, 3, 2, 1, 0]
    rng = np.random.default_rng(90 + n_sites)
    sites = rng.uniform(0, 2.0, (n_sites, 3))
    exps = np.exp(rng.uniform(np.log(0.3), np.log(6.0), len(ls)))
    basis = W.make_basis(ls, [1] * len(ls), exps, [1.0] * len(ls), [sites[i % n_sites] for i in range(len(ls))])
    parity.check(gpu_E(shgo, basis), ref_E(basis), what=f"eri l<=4 on {n_sites} centres")


def test_single_s_shell_and_a_distant_pair(shgo):
    one = W.make_basis([0], [2], [0.5, 3.0], [0.6, 0.4], [np.zeros(3)])
    parity.check(gpu_E(shgo, one), ref_E(one, "ld"), what="eri one s shell")
    far = W.make_basis([2, 1, 1], [1, 2, 1], [0.7, 1.5, 0.4, 0.9], [1.0, 0.5, 0.5, 1.0],
                       [np.zeros(3), np.array([0.5, 0.2, -0.3]), np.array([120.0, -80.0, 60.0])])
    parity.check(gpu_E(shgo, far), ref_E(far, "ld"), what="eri distant pair")


def test_rejects_l_above_4_and_batches(shgo):
    with pytest.raises(Exception):
        B = shgo.Basis(W.make_basis([5], [1], [1.0], [1.0], [np.zeros(3)]))
        try:
            shgo.eri(B)
        finally:
            B.close()
    rng = np.random.Generator(np.random.PCG64(3))
    mols = [W.config3_molecule(rng) for _ in range(2)]
    batch = shgo.Batch([(b, len(Z)) for b, _, Z in mols])
    with pytest.raises(Exception):
        shgo.eri(batch)
    with pytest.raises(shgo.ShgoError):  # the C entry point itself rejects a batch handle
        shgo.shgo_eri(batch.handle, torch.empty(1, dtype=torch.float64, device="cuda").data_ptr())
    batch.close()


def test_metric_positive_semidefinite_and_eightfold(shgo):
    basis, _, _ = W.config1(replica=2)
    E = gpu_E(shgo, basis)
    assert_eightfold(E)
    n = E.shape[0]
    ev = np.linalg.eigvalsh(E.reshape(n * n, n * n))
    assert ev.min() > -1e-11 * ev.max()


@pytest.mark.parametrize("cap", ["700", "20000"])
def test_scratch_split_into_rectangles(shgo, monkeypatch, cap):
    """A small per-stream scratch region (SHGO_ERI_SCRATCH_DOUBLES) cuts every class pair into several
    rectangles of quartets, down to single bra pairs against part of the ket range; the result is the same."""
    monkeypatch.setenv("SHGO_ERI_SCRATCH_DOUBLES", cap)
    basis = W.random_basis(12, 9, 3, max_prim=3, box=3.0, exp_lo=0.1, exp_hi=30.0, n_sites=9)
    E = gpu_E(shgo, basis)
    parity.check(E, ref_E(basis), what=f"eri scratch cap {cap}")
    assert_eightfold(E)


@pytest.mark.parametrize("which", ["config1", "mixed"])
def test_coulomb_and_exchange_matrices(shgo, which):
    """J[p,q] = sum_rs (pq|rs) D[r,s] and K[p,r] = sum_qs (pq|rs) D[q,s] without the tensor, against the oracle's
    tensor contracted with D (a symmetric density for config 1, a general matrix for the mixed basis).  Bar: the
    elementwise bar carried through the contraction, 1e-11 sum |(pq|rs)| |D| + 1e-13 sum |D|."""
    if which == "config1":
        basis = W.config1()[0]
    else:
        basis = W.random_basis(12, 9, 3, max_prim=3, box=3.0, exp_lo=0.1, exp_hi=30.0, n_sites=9)
    E = ref_E(basis)
    n = E.shape[0]
    d = np.random.default_rng(5).normal(size=(n, n))
    D = (d + d.T) / 2 if which == "config1" else d
    B = shgo.Basis(basis)
    Dt = torch.tensor(D, device="cuda")
    J, K = shgo.eri_jk(B, Dt)
    J1, none1 = shgo.eri_jk(B, Dt, exchange=False)
    none2, K1 = shgo.eri_jk(B, Dt, coulomb=False)
    torch.cuda.synchronize()
    B.close()
    assert none1 is None and none2 is None
    aE, aD = np.abs(E), np.abs(D)
    refs = [(J, np.einsum("pqrs,rs->pq", E, D), np.einsum("pqrs,rs->pq", aE, aD)),
            (J1, np.einsum("pqrs,rs->pq", E, D), np.einsum("pqrs,rs->pq", aE, aD)),
            (K, np.einsum("pqrs,qs->pr", E, D), np.einsum("pqrs,qs->pr", aE, aD)),
            (K1, np.einsum("pqrs,qs->pr", E, D), np.einsum("pqrs,qs->pr", aE, aD))]
    for got, ref, scale in refs:
        got = got.cpu().numpy()
        assert np.all(np.abs(got - ref) <= 1e-11 * scale + 1e-13 * aD.sum())
