"""The fused work-queue path of FP64 calls (one launch per Lambda; every step of a shell pair in one
block) against the two-kernel path, and its device-side time limit.

The allocation-free entry point still runs the two-kernel form (coupling blocks through a coupling
buffer, then the shell-pair kernel) and computes every entry with the same sequence of operations; only
the compiler's choice of which products it fuses into multiply-adds may differ between the two kernels,
so the outputs must agree to a few units in the last place (both are checked against the oracle
elsewhere).  The time limit is exercised without any fault: a limit of zero makes every launch stop
before taking work, the call's status reads SHGO_ERR_TIMEOUT, and the next call with no limit is exact."""
import numpy as np
import pytest

import oracle
from paper_2404_16245_gb300 import workloads as W
from tests import parity

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def shgo():
    from paper_2404_16245_gb300 import shgo as mod
    return mod


def _fused(shgo, basis, Cd, Zd):
    B = shgo.Basis(basis)
    V = shgo.nuclear_attraction(B, Cd, Zd)
    shgo.shgo_basis_sync(B.handle)
    out = V.cpu().numpy()
    B.close()
    return out


def _two_kernel(shgo, basis, Cd, Zd):
    n = W.nbf(basis)
    out = torch.full((n, n), float("nan"), dtype=torch.float64, device="cuda")
    shgo.shgo_nuclear_attraction_noalloc(len(basis["l"]), basis["l"], basis["nprim"], basis["exps"],
                                         basis["coefs"], basis["xyz"], Cd.shape[0], Cd.data_ptr(), Zd.data_ptr(),
                                         out.data_ptr(), torch.cuda.current_stream())
    torch.cuda.synchronize()
    return out.cpu().numpy()


@pytest.mark.parametrize("case", ["config1", "config2", "mixed_l8", "ragged_many_nuclei"])
def test_fused_matches_two_kernel_path_to_rounding(shgo, case):
    if case == "config1":
        basis, C, Z = W.config1()           # contracted: W in its own region, three primitive pairs each
    elif case == "config2":
        basis, C, Z = W.config2()           # uncontracted l <= 6: W shares the table region
    elif case == "mixed_l8":
        basis = W.random_basis(11, 12, 8, max_prim=3)
        C, Z = W.random_nuclei(12, 37)      # a partial second nucleus chunk
    else:
        basis = W.random_basis(13, 20, 4, max_prim=4)
        C, Z = W.random_nuclei(14, 97)      # four chunks, the last with one nucleus
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    a = _fused(shgo, basis, Cd, Zd)
    b = _two_kernel(shgo, basis, Cd, Zd)
    assert np.all(np.isfinite(a))
    diff = np.abs(a - b)
    # a few ulps of the matrix's scale: far below the 1e-13 + 1e-11 |y| parity bar
    bound = 64 * np.finfo(np.float64).eps * max(1.0, float(np.abs(b).max()))
    print(f"{case}: max |fused - two-kernel| = {diff.max():.3e} (bound {bound:.1e}), "
          f"identical elements {np.mean(a == b):.4f}")
    assert diff.max() <= bound, np.unravel_index(diff.argmax(), diff.shape)


def test_fused_launches_one_per_lambda(shgo):
    basis, C, Z = W.config2()
    B = shgo.Basis(basis)
    assert shgo.shgo_basis_launches(B.handle) == 13  # Lambda = 0..12
    B.close()


def test_time_limit_zero_reports_timeout_then_exact_without_limit(shgo):
    basis, C, Z = W.config1()
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    B = shgo.Basis(basis)
    shgo.shgo_basis_sync(B.handle)  # nothing run yet: OK
    shgo.shgo_basis_set_time_limit(B.handle, 0.0)
    shgo.nuclear_attraction(B, Cd, Zd)
    with pytest.raises(shgo.ShgoError) as e:
        shgo.shgo_basis_sync(B.handle)
    assert e.value.status == 5  # SHGO_ERR_TIMEOUT
    shgo.shgo_basis_sync(B.handle)  # reading the status cleared it
    shgo.shgo_basis_set_time_limit(B.handle, float("inf"))
    V = shgo.nuclear_attraction(B, Cd, Zd)
    shgo.shgo_basis_sync(B.handle)
    ref = oracle.nuclear_attraction(basis, C, Z, precision="ld")
    parity.check(V.cpu().numpy(), ref, what="after a timed-out call")
    # a generous limit does not trigger
    shgo.shgo_basis_set_time_limit(B.handle, 30.0)
    V = shgo.nuclear_attraction(B, Cd, Zd)
    shgo.shgo_basis_sync(B.handle)
    parity.check(V.cpu().numpy(), ref, what="within a 30 s limit")
    with pytest.raises(shgo.ShgoError):
        shgo.shgo_basis_set_time_limit(B.handle, -1.0)
    B.close()


def test_batch_time_limit_and_graph_replays(shgo):
    mols = [W.random_basis(20 + k, 6 + 2 * k, 4, max_prim=4) for k in range(3)]
    nucs = [W.random_nuclei(30 + k, 5 + 7 * k) for k in range(3)]
    batch = shgo.Batch([(b, len(z)) for b, (_, z) in zip(mols, nucs)])
    Cd = torch.tensor(np.concatenate([c for c, _ in nucs]), device="cuda")
    Zd = torch.tensor(np.concatenate([z for _, z in nucs]), device="cuda")
    out = torch.empty(batch.out_size, dtype=torch.float64, device="cuda")
    shgo.shgo_basis_set_time_limit(batch.handle, 0.0)
    shgo.nuclear_attraction_batched(batch, Cd, Zd, out=out)   # first call: direct launches
    with pytest.raises(shgo.ShgoError) as e:
        shgo.shgo_basis_sync(batch.handle)
    assert e.value.status == 5
    shgo.shgo_basis_set_time_limit(batch.handle, float("inf"))
    refs = [oracle.nuclear_attraction(b, c, z, precision="ld") for b, (c, z) in zip(mols, nucs)]
    outs = []
    for _ in range(3):                                          # capture, then two replays
        out.fill_(float("nan"))
        shgo.nuclear_attraction_batched(batch, Cd, Zd, out=out)
        shgo.shgo_basis_sync(batch.handle)
        outs.append(out.cpu().numpy().copy())
        for m, ref in enumerate(refs):
            parity.check(np.asarray(batch.block(outs[-1], m)), ref, what=f"molecule {m}")
    assert np.array_equal(outs[1], outs[2])
    batch.close()
