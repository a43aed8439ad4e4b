"""Batched launches: many molecules of uneven size and mixed angular momentum in one call.

Checks the batched output against the extended-precision oracle per molecule, against the
single-molecule entry point, and that the tuned first call, the captured graph and its replays
agree (replays bit for bit)."""
import numpy as np
import pytest

import oracle
from paper_2404_16245_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


def small_molecules(seed, n):
    """Contracted molecules like the batched workload, with few atoms (l <= 4, 1..8 primitives)."""
    rng = np.random.default_rng(seed)
    mols = []
    for _ in range(n):
        na = int(rng.integers(2, 6))
        box = (na / 0.05) ** (1 / 3)
        pos = rng.uniform(0, box, (na, 3))
        Z = np.where(rng.uniform(size=na) < 0.4, 1, rng.integers(6, 10, na)).astype(float)
        ls, nps, ex, co, xyz = [], [], [], [], []
        for a in range(na):
            for l in (W.H_SHELLS if Z[a] == 1 else W.HEAVY_SHELLS):
                k = int(rng.integers(1, 9))
                ls.append(l)
                nps.append(k)
                ex.extend(np.exp(rng.uniform(np.log(0.05), np.log(5000.0), k)))
                co.extend(rng.uniform(0.1, 1.0, k) if k > 1 else [1.0])
                xyz.append(pos[a])
        mols.append((W.make_basis(ls, nps, ex, co, xyz), pos, Z))
    return mols


def test_batched_matches_oracle_and_single_path():
    from paper_2404_16245_gb300 import shgo
    mols = small_molecules(5, 9)
    batch = shgo.Batch([(b, len(Z)) for b, _, Z in mols])
    C = torch.tensor(np.concatenate([C for _, C, _ in mols]), device="cuda")
    Zt = torch.tensor(np.concatenate([Z for _, _, Z in mols]), device="cuda")
    out = torch.full((batch.out_size,), float("nan"), dtype=torch.float64, device="cuda")
    runs = []
    for _ in range(4):  # tuned first call, capture + replay, replays
        shgo.nuclear_attraction_batched(batch, C, Zt, out=out)
        torch.cuda.synchronize()
        runs.append(out.cpu().numpy().copy())
    assert np.array_equal(runs[1], runs[2]) and np.array_equal(runs[2], runs[3])
    for m, (b, Cm, Zm) in enumerate(mols):
        ref = oracle.nuclear_attraction(b, Cm, Zm, precision="ld")
        for r in runs:
            parity.check(batch.block(r, m), ref, what=f"molecule {m}")
        B = shgo.Basis(b)
        single = shgo.nuclear_attraction(B, torch.tensor(Cm, device="cuda"), torch.tensor(Zm, device="cuda"))
        torch.cuda.synchronize()
        np.testing.assert_allclose(batch.block(runs[-1], m), single.cpu().numpy(), rtol=1e-12, atol=1e-14)
        B.close()
    batch.close()


def test_batched_new_output_pointer_recaptures():
    from paper_2404_16245_gb300 import shgo
    mols = small_molecules(8, 4)
    batch = shgo.Batch([(b, len(Z)) for b, _, Z in mols])
    C = torch.tensor(np.concatenate([C for _, C, _ in mols]), device="cuda")
    Zt = torch.tensor(np.concatenate([Z for _, _, Z in mols]), device="cuda")
    o1 = shgo.nuclear_attraction_batched(batch, C, Zt)
    o2 = shgo.nuclear_attraction_batched(batch, C, Zt)
    o3 = shgo.nuclear_attraction_batched(batch, C, Zt)  # a third buffer: a new graph
    torch.cuda.synchronize()
    assert np.array_equal(o2.cpu().numpy(), o3.cpu().numpy())
    np.testing.assert_allclose(o1.cpu().numpy(), o3.cpu().numpy(), rtol=1e-12, atol=1e-14)
    batch.close()


def test_batched_molecule_without_nuclei_and_mixed_sizes():
    from paper_2404_16245_gb300 import shgo
    mols = small_molecules(11, 3)
    b0, C0, Z0 = mols[0]
    entries = [(b0, 0)] + [(b, len(Z)) for b, _, Z in mols[1:]]
    batch = shgo.Batch(entries)
    C = torch.tensor(np.concatenate([C for _, C, _ in mols[1:]]), device="cuda")
    Zt = torch.tensor(np.concatenate([Z for _, _, Z in mols[1:]]), device="cuda")
    out = shgo.nuclear_attraction_batched(batch, C, Zt)
    torch.cuda.synchronize()
    o = out.cpu().numpy()
    assert np.array_equal(batch.block(o, 0), np.zeros_like(batch.block(o, 0)))
    for m in (1, 2):
        b, Cm, Zm = mols[m]
        parity.check(batch.block(o, m), oracle.nuclear_attraction(b, Cm, Zm, precision="ld"), what=f"mol {m}")
    batch.close()


def test_bounded_coupling_buffer_chunks_match(monkeypatch):
    # a tiny cap forces per-stream regions and many chunks per class; results must not change
    from paper_2404_16245_gb300 import shgo
    basis, C, Z = W.config2(n_atoms=10)
    Cd = torch.tensor(C, device="cuda")
    Zd = torch.tensor(Z, device="cuda")
    B = shgo.Basis(basis)
    ref = shgo.nuclear_attraction(B, Cd, Zd).cpu().numpy()
    B.close()
    monkeypatch.setenv("SHGO_RBUF_CAP_DOUBLES", "20000")
    B2 = shgo.Basis(basis)
    got = shgo.nuclear_attraction(B2, Cd, Zd).cpu().numpy()
    B2.close()
    assert np.array_equal(got, ref)
    mols = small_molecules(21, 5)
    batch = shgo.Batch([(b, len(Zm)) for b, _, Zm in mols])
    Cb = torch.tensor(np.concatenate([c for _, c, _ in mols]), device="cuda")
    Zb = torch.tensor(np.concatenate([z for _, _, z in mols]), device="cuda")
    outs = [shgo.nuclear_attraction_batched(batch, Cb, Zb).cpu().numpy() for _ in range(3)]
    for m, (b, Cm, Zm) in enumerate(mols):
        parity.check(batch.block(outs[-1], m), oracle.nuclear_attraction(b, Cm, Zm, precision="ld"), what=f"m{m}")
    assert np.array_equal(outs[1], outs[2])
    batch.close()


@pytest.mark.parametrize("cap", [None, "20000"])
def test_fp32_bulk_batched_matches_fp64(monkeypatch, cap):
    """FP32-bulk through the batched entry point (tuned first call, graph capture, replays) and, with a
    tiny cap, through per-stream regions of the coupling buffer: every molecule within 1e-10 of the FP64
    batched result relative to its largest element, replays bit for bit, and the bounded buffer equal
    to the unbounded one."""
    from paper_2404_16245_gb300 import shgo
    mols = small_molecules(33, 6)
    entries = [(b, len(Z)) for b, _, Z in mols]
    C = torch.tensor(np.concatenate([c for _, c, _ in mols]), device="cuda")
    Zt = torch.tensor(np.concatenate([z for _, _, z in mols]), device="cuda")
    b64 = shgo.Batch(entries)
    ref = shgo.nuclear_attraction_batched(b64, C, Zt).cpu().numpy()
    b64.close()
    unbounded = None
    if cap:
        b0 = shgo.Batch(entries, precision=shgo.SHGO_PREC_FP32_BULK)
        unbounded = [shgo.nuclear_attraction_batched(b0, C, Zt).cpu().numpy() for _ in range(2)][-1]
        b0.close()
        monkeypatch.setenv("SHGO_RBUF_CAP_DOUBLES", cap)
    b32 = shgo.Batch(entries, precision=shgo.SHGO_PREC_FP32_BULK)
    runs = [shgo.nuclear_attraction_batched(b32, C, Zt).cpu().numpy() for _ in range(4)]
    assert np.array_equal(runs[1], runs[2]) and np.array_equal(runs[2], runs[3])
    for m in range(len(mols)):
        r = b32.block(ref, m)
        for g in runs:
            assert np.max(np.abs(b32.block(g, m) - r)) <= 1e-10 * max(1.0, float(np.max(np.abs(r)))), m
    if unbounded is not None:
        assert np.array_equal(runs[-1], unbounded)
    b32.close()
