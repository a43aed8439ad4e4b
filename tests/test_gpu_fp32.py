"""FP32-bulk and FP32-plain precision modes against the FP64 GPU path and the oracle.

The FP64 path is itself parity-checked against the oracle (test_gpu_parity.py); here it is the
reference for the workloads, and the oracle for the edge cases.  Error measure (per shell-pair
block, the reading of the 1e-7 target): the block's max abs error over the block's max abs value.
FP32-bulk carries every per-nucleus factor as a pair of FP32 numbers (48 significant bits) with
error-free sums, so its bar is 1e-10, far inside 1e-7; FP32-plain (single FP32 numbers) is held to
1e-4.  The measured values are written to the test log."""
import os

import numpy as np
import pytest

import oracle
from paper_2404_16245_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def shgo():
    from paper_2404_16245_gb300 import shgo as mod
    return mod


def run(shgo, basis, C, Z, precision):
    B = shgo.Basis(basis, precision=precision)
    V = shgo.nuclear_attraction(B, torch.tensor(np.asarray(C).reshape(-1, 3), device="cuda"),
                                torch.tensor(np.asarray(Z, dtype=np.float64).reshape(-1), device="cuda"))
    torch.cuda.synchronize()
    out = V.cpu().numpy()
    B.close()
    return out


def block_errors(basis, got, ref):
    off = np.concatenate([[0], np.cumsum(2 * basis["l"] + 1)])
    errs = []
    n = len(basis["l"])
    for a in range(n):
        for b in range(a + 1):
            r = ref[off[a]:off[a + 1], off[b]:off[b + 1]]
            g = got[off[a]:off[a + 1], off[b]:off[b + 1]]
            scale = np.max(np.abs(r))
            if scale > 0:
                errs.append(np.max(np.abs(g - r)) / scale)
    return np.array(errs)


@pytest.mark.parametrize("name,factory", [("config1", W.config1), ("config2", W.config2)])
def test_fp32_bulk_blockwise_error(shgo, name, factory, capsys):
    basis, C, Z = factory()
    ref = run(shgo, basis, C, Z, shgo.SHGO_PREC_FP64)
    bulk = run(shgo, basis, C, Z, shgo.SHGO_PREC_FP32_BULK)
    plain = run(shgo, basis, C, Z, shgo.SHGO_PREC_FP32_PLAIN)
    eb = block_errors(basis, bulk, ref)
    ep = block_errors(basis, plain, ref)
    with capsys.disabled():
        print(f"\n{name}: FP32-bulk block error max {eb.max():.2e} median {np.median(eb):.2e}; "
              f"FP32-plain max {ep.max():.2e} median {np.median(ep):.2e}; "
              f"max abs difference FP32-bulk {np.max(np.abs(bulk - ref)):.2e} (max |V| {np.max(np.abs(ref)):.2e})")
    assert np.all(np.isfinite(bulk)) and np.all(np.isfinite(plain))
    assert eb.max() < 1e-10
    assert ep.max() < 1e-4


def test_fp32_bulk_high_l_triples(shgo, capsys):
    worst_b = worst_p = 0.0
    for basis, C, Z in W.config5(40, replica=3):
        ref = run(shgo, basis, C, Z, shgo.SHGO_PREC_FP64)
        bulk = run(shgo, basis, C, Z, shgo.SHGO_PREC_FP32_BULK)
        plain = run(shgo, basis, C, Z, shgo.SHGO_PREC_FP32_PLAIN)
        worst_b = max(worst_b, block_errors(basis, bulk, ref).max())
        worst_p = max(worst_p, block_errors(basis, plain, ref).max())
    with capsys.disabled():
        print(f"\nl<=8 triples: FP32-bulk worst block error {worst_b:.2e}; FP32-plain {worst_p:.2e}")
    assert worst_b < 1e-10
    assert worst_p < 1e-4


def test_fp32_bulk_edge_cases_against_oracle(shgo, capsys):
    """Nuclei on shell centres (d = 0 and C = A), far away (T past the exp table), near T = 40 where
    the Boys evaluation changes form, non-integer charges, 37 nuclei (a partial chunk of 32), and
    classes up to (8, 8), against the extended-precision oracle."""
    rng = np.random.default_rng(404)
    ls = [0, 1, 2, 3, 4, 5, 6, 7, 8, 8, 6, 3]
    sites = np.array([[0.0, 0.0, 0.0], [1.3, -0.4, 0.7], [-0.9, 1.1, -0.2]])
    exps = np.exp(rng.uniform(np.log(0.05), np.log(80.0), len(ls)))
    basis = W.make_basis(ls, [1] * len(ls), exps, np.ones(len(ls)), [sites[i % 3] for i in range(len(ls))])
    far = rng.standard_normal((8, 3))
    far = 60.0 * far / np.linalg.norm(far, axis=1, keepdims=True)
    # nuclei at distance sqrt(40 / p) from a shell centre put T near the switch for that shell's pairs
    near40 = sites[0] + np.outer(np.sqrt(40.0 / (2.0 * exps[:6])), [0.6, 0.0, 0.8])
    C = np.vstack([sites, far, near40, rng.uniform(-3.0, 3.0, (20, 3))])
    Z = np.round(rng.uniform(0.3, 9.0, len(C)), 3)
    assert len(C) == 37
    bulk = run(shgo, basis, C, Z, shgo.SHGO_PREC_FP32_BULK)
    ref = oracle.nuclear_attraction(basis, C, Z, threads=os.cpu_count() or 1, precision="ld")
    eb = block_errors(basis, bulk, ref)
    with capsys.disabled():
        print(f"\nedge cases: FP32-bulk vs oracle block error max {eb.max():.2e} median {np.median(eb):.2e}")
    assert np.all(np.isfinite(bulk))
    assert eb.max() < 1e-10


def block_errors_vs_oracle(basis, got, ref, Z):
    """Per shell-pair block against the oracle: (max abs error, block max) of the blocks above the library's
    elementwise bound (n_prim_a n_prim_b x 1e-20 x sum |Z|); a block below it, which the library skips, must
    match to that bound."""
    off = np.concatenate([[0], np.cumsum(2 * basis["l"] + 1)])
    nprim = np.asarray(basis["nprim"])
    zsum = float(np.sum(np.abs(Z)))
    errs, scales = [], []
    for a in range(len(basis["l"])):
        for b in range(a + 1):
            r = ref[off[a]:off[a + 1], off[b]:off[b + 1]]
            g = got[off[a]:off[a + 1], off[b]:off[b + 1]]
            bound = nprim[a] * nprim[b] * 1e-20 * zsum
            scale = np.max(np.abs(r))
            if scale <= bound:
                assert np.max(np.abs(g - r)) <= bound, (a, b)
                continue
            errs.append(np.max(np.abs(g - r)))
            scales.append(scale)
    return np.array(errs), np.array(scales)


def check_vs_oracle(name, e, sc, capsys):
    # blocks: |error| <= 1e-8 x block max + 1e-13, the relative measure of reading C9 (target 1e-7) on the blocks
    # above 1e-6 of the largest.  Against the oracle the bar is 1e-8 rather than the 1e-10 held against the FP64
    # path: at l = 6 the double oracle's own block error reaches ~1e-10 (the two GPU paths agree to ~3e-12)
    big = sc >= 1e-6 * sc.max()
    rel = e[big] / sc[big]
    with capsys.disabled():
        print(f"\n{name}: FP32-bulk vs oracle, {len(e)} blocks above the bound: block error max {rel.max():.2e} "
              f"median {np.median(rel):.2e} over the {int(big.sum())} blocks above 1e-6 of the largest; "
              f"max abs error {e.max():.2e}")
    assert np.all(e <= 1e-8 * sc + 1e-13)
    assert rel.max() <= 1e-8


@pytest.mark.parametrize("name,factory", [("config1", W.config1), ("config2", W.config2)])
def test_fp32_bulk_against_the_oracle_in_full(shgo, name, factory, capsys):
    # FP32-bulk checked directly against the oracle (not through the FP64 GPU path)
    basis, C, Z = factory()
    bulk = run(shgo, basis, C, Z, shgo.SHGO_PREC_FP32_BULK)
    ref = oracle.nuclear_attraction(basis, C, Z, threads=os.cpu_count() or 1)
    check_vs_oracle(name, *block_errors_vs_oracle(basis, bulk, ref, Z), capsys)


def test_fp32_bulk_every_class_to_l8_against_the_oracle(shgo, capsys):
    ls = list(range(9)) * 2
    rng = np.random.default_rng(97)
    sites = rng.uniform(0, 2.5, (3, 3))
    exps = np.exp(rng.uniform(np.log(0.1), np.log(30.0), len(ls) * 2))
    basis = W.make_basis(ls, [2] * len(ls), exps, rng.uniform(0.2, 1, len(ls) * 2), [sites[i % 3] for i in range(len(ls))])
    C = np.vstack([rng.uniform(-1.0, 3.5, (9, 3)), sites[:1]])
    Z = rng.uniform(0.5, 9.0, len(C))
    bulk = run(shgo, basis, C, Z, shgo.SHGO_PREC_FP32_BULK)
    ref = oracle.nuclear_attraction(basis, C, Z, threads=os.cpu_count() or 1, precision="ld")
    check_vs_oracle("every class to (8, 8)", *block_errors_vs_oracle(basis, bulk, ref, Z), capsys)
