"""Work queues and the device-side time limit of the coupling and pair kernels.

The limit is exercised without any fault: a limit of zero makes every launch stop before taking work,
the call's status (shgo_basis_sync) reads SHGO_ERR_TIMEOUT, and the next call with no limit is exact.
Batches take their work in a cost order (molecules with more nuclei first); their output must not depend
on it, and graph replays must repeat the captured call bit for bit."""
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


@pytest.mark.parametrize("precision", [0, 1])
def test_time_limit_zero_reports_timeout_then_exact_without_limit(shgo, precision):
    basis, C, Z = W.config1()
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    B = shgo.Basis(basis, precision=precision)
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
    if precision == 0:
        parity.check(V.cpu().numpy(), ref, what="after a timed-out call")
    else:
        assert np.max(np.abs(V.cpu().numpy() - ref)) <= 1e-10 * max(1.0, np.max(np.abs(ref)))
    # a generous limit does not trigger
    shgo.shgo_basis_set_time_limit(B.handle, 30.0)
    V2 = shgo.nuclear_attraction(B, Cd, Zd)
    shgo.shgo_basis_sync(B.handle)
    assert np.array_equal(V2.cpu().numpy(), V.cpu().numpy())
    with pytest.raises(shgo.ShgoError):
        shgo.shgo_basis_set_time_limit(B.handle, -1.0)
    B.close()


def test_batch_time_limit_cost_order_and_graph_replays(shgo):
    mols = [W.random_basis(20 + k, 6 + 2 * k, 4, max_prim=4) for k in range(3)]
    nucs = [W.random_nuclei(30 + k, 5 + 7 * k) for k in range(3)]   # unequal molecules: a real cost order
    batch = shgo.Batch([(b, len(z)) for b, (_, z) in zip(mols, nucs)])
    Cd = torch.tensor(np.concatenate([c for c, _ in nucs]), device="cuda")
    Zd = torch.tensor(np.concatenate([z for _, z in nucs]), device="cuda")
    out = torch.empty(batch.out_size, dtype=torch.float64, device="cuda")
    refs = [oracle.nuclear_attraction(b, c, z, precision="ld") for b, (c, z) in zip(mols, nucs)]
    shgo.nuclear_attraction_batched(batch, Cd, Zd, out=out)     # tuning call (no limit)
    shgo.shgo_basis_sync(batch.handle)
    shgo.shgo_basis_set_time_limit(batch.handle, 0.0)
    shgo.nuclear_attraction_batched(batch, Cd, Zd, out=out)     # captured with a zero limit
    with pytest.raises(shgo.ShgoError) as e:
        shgo.shgo_basis_sync(batch.handle)
    assert e.value.status == 5
    shgo.shgo_basis_set_time_limit(batch.handle, float("inf"))
    outs = []
    for _ in range(3):                                           # re-capture for the new limit, two replays
        out.fill_(float("nan"))
        shgo.nuclear_attraction_batched(batch, Cd, Zd, out=out)
        shgo.shgo_basis_sync(batch.handle)
        outs.append(out.cpu().numpy().copy())
        for m, ref in enumerate(refs):
            parity.check(np.asarray(batch.block(outs[-1], m)), ref, what=f"molecule {m}")
    assert np.array_equal(outs[0], outs[1]) and np.array_equal(outs[1], outs[2])
    batch.close()


def test_repeated_single_basis_calls_replay_a_graph_that_reads_current_contents(shgo):
    """The second call with the same pointers captures the launches into a graph, later calls replay it;
    each replay reads what the arrays hold at that time (nuclei moved in place between calls), and a call
    with other pointers launches directly again.  Results equal a fresh basis's direct call bit for bit."""
    basis = W.random_basis(81, 16, 5, max_prim=3)
    C1, Z1 = W.random_nuclei(82, 21)
    C2, Z2 = W.random_nuclei(83, 21)
    B = shgo.Basis(basis)
    Cd, Zd = torch.tensor(C1, device="cuda"), torch.tensor(Z1, device="cuda")
    out = torch.empty((B.nbf, B.nbf), dtype=torch.float64, device="cuda")

    def fresh(C, Z):
        F = shgo.Basis(basis)
        v = shgo.nuclear_attraction(F, torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")).cpu().numpy()
        F.close()
        return v

    want1, want2 = fresh(C1, Z1), fresh(C2, Z2)
    for k in range(3):  # direct, capture + replay, replay
        out.fill_(float("nan"))
        shgo.nuclear_attraction(B, Cd, Zd, out=out)
        assert np.array_equal(out.cpu().numpy(), want1), k
    Cd.copy_(torch.tensor(C2))
    Zd.copy_(torch.tensor(Z2))
    shgo.nuclear_attraction(B, Cd, Zd, out=out)  # replay on the new contents
    assert np.array_equal(out.cpu().numpy(), want2)
    other = torch.empty_like(out)
    shgo.nuclear_attraction(B, Cd, Zd, out=other)  # new pointer: direct launch
    assert np.array_equal(other.cpu().numpy(), want2)
    B.close()
