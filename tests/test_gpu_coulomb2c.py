"""Two-centre Coulomb integrals (a|b) (the two-centre case of Eqs. 13-15) on the GPU against the CPU oracle,
element by element.

Same bar as the attraction integrals: |x - y| <= 1e-13 + 1e-11 |y|, judged by the oracle built in extended
precision (McMurchie-Davidson, pinned by the s-s closed form, the dipole-dipole far field and rotation
covariance in test_oracle_pins.py).  At any size the matrix is symmetric and positive definite."""
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


def gpu_J(shgo, basis, precision=None):
    B = shgo.Basis(basis) if precision is None else shgo.Basis(basis, precision=precision)
    J = shgo.coulomb_2c(B)
    torch.cuda.synchronize()
    out = J.cpu().numpy()
    B.close()
    return out


def ref_J(basis):
    return oracle.coulomb_2c(basis, threads=THREADS, precision="ld")


def test_config1(shgo):
    basis, _, _ = W.config1()
    parity.check(gpu_J(shgo, basis), ref_J(basis), what="coulomb2c config1")


@pytest.mark.parametrize("seed,lmax,nshell", [(1, 8, 14), (2, 6, 24), (4, 4, 30)])
def test_mixed_classes_contracted(shgo, seed, lmax, nshell):
    basis = W.random_basis(seed, nshell, lmax, max_prim=3, box=3.0, exp_lo=0.1, exp_hi=30.0)
    parity.check(gpu_J(shgo, basis), ref_J(basis), what=f"coulomb2c seed {seed}")


def test_every_class_up_to_l8_coincident_and_distant_centres(shgo):
    ls = list(range(9)) * 2
    rng = np.random.default_rng(78)
    sites = np.vstack([rng.uniform(0, 2.5, (2, 3)), [[40.0, -25.0, 10.0]]])
    exps = np.exp(rng.uniform(np.log(0.2), np.log(8.0), len(ls) * 2))
    basis = W.make_basis(ls, [2] * len(ls), exps, rng.uniform(0.2, 1, len(ls) * 2),
                         [sites[i % 3] for i in range(len(ls))])
    parity.check(gpu_J(shgo, basis), ref_J(basis), what="coulomb2c l<=8")


def test_precision_option_is_ignored(shgo):
    basis = W.random_basis(9, 10, 3, max_prim=2)
    assert np.array_equal(gpu_J(shgo, basis), gpu_J(shgo, basis, precision=shgo.SHGO_PREC_FP32_BULK))


def test_batched_molecules(shgo):
    rng = np.random.Generator(np.random.PCG64(6))
    mols = [W.config3_molecule(rng) for _ in range(3)]
    batch = shgo.Batch([(b, len(Z)) for b, _, Z in mols])
    J = shgo.coulomb_2c(batch)
    torch.cuda.synchronize()
    Jh = J.cpu().numpy()
    for m, (b, _, _) in enumerate(mols):
        parity.check(batch.block(Jh, m), ref_J(b), what=f"coulomb2c molecule {m}")
    batch.close()


def test_symmetric_positive_definite_at_benchmark_size(shgo):
    basis, _, _ = W.config2()
    J = gpu_J(shgo, basis)
    assert np.array_equal(J, J.T)
    assert np.min(np.linalg.eigvalsh(J)) > 0
