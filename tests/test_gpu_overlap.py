"""Overlap matrix (Eqs. 9-10) on the GPU against the CPU oracle, element by element.

Same bar as the attraction integrals: |x - y| <= 1e-13 + 1e-11 |y|, judged by the oracle built in
extended precision.  At any size the diagonal of a normalised basis is 1 and S is symmetric."""
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


def gpu_S(shgo, basis):
    B = shgo.Basis(basis)
    S = shgo.overlap(B)
    torch.cuda.synchronize()
    out = S.cpu().numpy()
    B.close()
    return out


def ref_S(basis):
    return oracle.overlap(basis, threads=THREADS, precision="ld")


def test_config1(shgo):
    basis, _, _ = W.config1()
    parity.check(gpu_S(shgo, basis), ref_S(basis), what="overlap config1")


def test_config2_full_size(shgo):
    basis, _, _ = W.config2()
    got = gpu_S(shgo, basis)
    parity.check(got, ref_S(basis), what="overlap config2")
    assert np.array_equal(got, got.T)


@pytest.mark.parametrize("seed,lmax,nshell", [(1, 8, 14), (2, 6, 24), (4, 4, 30)])
def test_mixed_classes_ragged(shgo, seed, lmax, nshell):
    basis = W.random_basis(seed, nshell, lmax, max_prim=3, box=3.0, exp_lo=0.1, exp_hi=30.0)
    parity.check(gpu_S(shgo, basis), ref_S(basis), what=f"overlap seed {seed}")


def test_every_class_up_to_l8_and_coincident_centres(shgo):
    ls = list(range(9)) * 2
    rng = np.random.default_rng(77)
    sites = rng.uniform(0, 2.5, (3, 3))
    exps = np.exp(rng.uniform(np.log(0.2), np.log(8.0), len(ls) * 2))
    basis = W.make_basis(ls, [2] * len(ls), exps, rng.uniform(0.2, 1, len(ls) * 2),
                         [sites[i % 3] for i in range(len(ls))])
    S = gpu_S(shgo, basis)
    parity.check(S, ref_S(basis), what="overlap l<=8")
    # every function is normalised
    assert np.max(np.abs(np.diag(S) - 1.0)) < 1e-12


def test_diagonal_is_one_at_benchmark_size(shgo):
    basis, _, _ = W.config2(replica=3)
    S = gpu_S(shgo, basis)
    assert np.max(np.abs(np.diag(S) - 1.0)) < 1e-12
    assert np.array_equal(S, S.T)
    # Cauchy-Schwarz for normalised functions
    assert np.max(np.abs(S)) <= 1.0 + 1e-12


def test_batched_overlap_matches_single(shgo):
    rng = np.random.Generator(np.random.PCG64(5))
    mols = [W.config3_molecule(rng) for _ in range(5)]
    batch = shgo.Batch([(b, len(Z)) for b, _, Z in mols])
    S = shgo.overlap(batch)
    torch.cuda.synchronize()
    Sh = S.cpu().numpy()
    for m, (b, _, _) in enumerate(mols):
        parity.check(batch.block(Sh, m), ref_S(b), what=f"overlap molecule {m}")
    batch.close()


def test_repeat_is_bitwise_and_empty_classes_skip(shgo):
    # one launch over every class: two calls give the same bits; a basis with s and g shells only (classes
    # (0, 0), (4, 0), (4, 4)) covers the classes that hold no pairs being left out of the launch
    basis, _, _ = W.config2()
    B = shgo.Basis(basis)
    s1 = shgo.overlap(B).cpu().numpy()
    s2 = shgo.overlap(B).cpu().numpy()
    B.close()
    assert np.array_equal(s1, s2)
    rng = np.random.default_rng(12)
    ls = [0, 4, 0, 4, 4]
    b2 = W.make_basis(ls, [2] * len(ls), np.exp(rng.uniform(np.log(0.3), np.log(5.0), 2 * len(ls))),
                      rng.uniform(0.2, 1, 2 * len(ls)), list(rng.uniform(0, 3.0, (len(ls), 3))))
    parity.check(gpu_S(shgo, b2), ref_S(b2), what="overlap s and g shells")
