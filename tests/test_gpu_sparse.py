"""Block-sparse output of V (SHGO_FLAG_BLOCK_SPARSE) and the method without the primitive-pair bound
(SHGO_FLAG_NO_PRIM_BOUND).

A spread-out contracted basis leaves many shell pairs with no primitive pair above the elementwise bound.
The block-sparse output must store exactly the other pairs, each block equal to the dense result (the same
kernels compute it) and to the extended-precision oracle at the parity bar; every omitted block is zero in
the oracle up to the bound (npp x 1e-20 x sum |Z|).  Without the bound, V matches the oracle at the same bar
and differs from the bounded V by at most that bound."""
import numpy as np
import pytest

import oracle
from oracle import mlp as ref
from paper_2404_16245_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def shgo():
    from paper_2404_16245_gb300 import shgo as mod
    return mod


def spread_basis():
    # 24 contracted shells (l <= 4) on 8 sites in a 40 bohr box, exponents 0.5..30: distant pairs drop out
    return W.random_basis(71, 24, 4, max_prim=3, box=40.0, exp_lo=0.5, exp_hi=30.0, n_sites=8)


def blocks_of_dense(V, basis, pa, pb):
    l = np.asarray(basis["l"])
    first = np.concatenate([[0], np.cumsum(2 * l + 1)[:-1]])
    return [V[first[a]:first[a] + 2 * l[a] + 1, first[b]:first[b] + 2 * l[b] + 1] for a, b in zip(pa, pb)]


def test_block_sparse_output_matches_dense_and_oracle(shgo):
    basis = spread_basis()
    C, Z = W.random_nuclei(72, 19, box=40.0)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    dense_B = shgo.Basis(basis)
    dense = shgo.nuclear_attraction(dense_B, Cd, Zd).cpu().numpy()
    S = shgo.Basis(basis, flags=shgo.SHGO_FLAG_BLOCK_SPARSE)
    assert S.out_shape() == (max(S.ndoubles, 1),)
    out = torch.full(S.out_shape(), float("nan"), dtype=torch.float64, device="cuda")
    shgo.nuclear_attraction(S, Cd, Zd, out=out)
    got = out.cpu().numpy()
    pa, pb = shgo.pair_shells(S.handle, S.npairs)
    nbl, nd, off = shgo.shgo_sparse_layout(S.handle)
    kept = off >= 0
    print(f"block-sparse: {nbl} of {S.npairs} shell pairs stored, {nd} doubles against {S.nbf ** 2} dense")
    assert nbl == int(kept.sum()) and 0 < nbl < S.npairs
    l = np.asarray(basis["l"])
    sizes = (2 * l[pa] + 1) * (2 * l[pb] + 1)
    assert nd == int(sizes[kept].sum())
    assert np.all(np.isfinite(got))  # every stored double written
    ref_V = oracle.nuclear_attraction(basis, C, Z, precision="ld")
    dblocks = blocks_of_dense(dense, basis, pa, pb)
    rblocks = blocks_of_dense(ref_V, basis, pa, pb)
    nprim = np.asarray(basis["nprim"])
    bound = 1e-20 * float(np.abs(Z).sum())
    for q in range(S.npairs):
        if kept[q]:
            blk = got[off[q]:off[q] + sizes[q]].reshape(2 * l[pa[q]] + 1, 2 * l[pb[q]] + 1)
            assert np.array_equal(blk, dblocks[q]), q
            parity.check(blk, rblocks[q], what=f"stored block {q}")
        else:
            assert np.max(np.abs(rblocks[q])) <= nprim[pa[q]] * nprim[pb[q]] * bound, q
    S.close()
    dense_B.close()


def test_block_sparse_screened_keep_all_equals_plain(shgo):
    basis = spread_basis()
    C, Z = W.random_nuclei(73, 11, box=40.0)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    S = shgo.Basis(basis, flags=shgo.SHGO_FLAG_BLOCK_SPARSE)
    plain = shgo.nuclear_attraction(S, Cd, Zd).cpu().numpy()
    p = np.zeros(ref.NPARAM, dtype=np.float32)
    p[-1] = 100.0
    keep = shgo.MLP(p, np.zeros(16), np.ones(16))
    kept, skipped = shgo.screen_build(S.handle, keep, Cd, Zd, len(Z), -12.0, 2.0)
    assert skipped == 0
    out = torch.full(S.out_shape(), float("nan"), dtype=torch.float64, device="cuda")
    shgo.nuclear_attraction_screened(S.handle, Cd, Zd, len(Z), out)
    assert np.array_equal(out.cpu().numpy(), plain)
    keep.close()
    S.close()


def test_no_primitive_pair_bound(shgo):
    basis = W.random_basis(74, 18, 4, max_prim=4, box=12.0, exp_lo=0.3, exp_hi=500.0, n_sites=6)
    C, Z = W.random_nuclei(75, 23, box=12.0)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    Bb = shgo.Basis(basis)
    Bn = shgo.Basis(basis, flags=shgo.SHGO_FLAG_NO_PRIM_BOUND)
    vb = shgo.nuclear_attraction(Bb, Cd, Zd).cpu().numpy()
    vn = shgo.nuclear_attraction(Bn, Cd, Zd).cpu().numpy()
    ref_V = oracle.nuclear_attraction(basis, C, Z, precision="ld")
    parity.check(vn, ref_V, what="no bound")
    npp = int(np.sum(np.asarray(basis["nprim"])) ** 2)
    assert np.max(np.abs(vn - vb)) <= npp * 1e-20 * float(np.abs(Z).sum()) + 1e-13
    # the bound skipped some primitive pairs here, so the two bases did different amounts of work
    fb, _ = shgo.shgo_basis_flops(Bb.handle, len(Z))
    fn, _ = shgo.shgo_basis_flops(Bn.handle, len(Z))
    assert fn[0] > fb[0]
    Bb.close()
    Bn.close()
