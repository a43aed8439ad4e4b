"""One basis split over devices (shgo_basis_create_shard), run as CPU-simulated ranks: host threads on one GPU.

Every shard computes only its shell pairs' blocks; the shards' outputs, each into a zeroed matrix, add up to
the whole result.  V and the derivative matrices come from the same kernels on the same pairs, so the sum of
the shards equals the unsplit result bit for bit; the sums over pairs (potential, contracted gradient) agree
to rounding."""
import threading

import numpy as np
import pytest

from paper_2404_16245_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def shgo():
    from paper_2404_16245_gb300 import shgo as mod
    return mod


def run_ranks(shgo, basis, count, fn):
    """fn(Basis, stream) -> numpy result, once per shard, each in its own host thread and stream."""
    out = [None] * count
    errs = []

    def rank(k):
        try:
            s = torch.cuda.Stream()
            with torch.cuda.stream(s):
                B = shgo.Basis(basis, shard=(k, count))
                out[k] = (fn(B, s), shgo.pair_shells(B.handle, B.npairs))
                s.synchronize()
                B.close()
        except Exception as e:  # noqa: BLE001 (reported below)
            errs.append(e)

    th = [threading.Thread(target=rank, args=(k,)) for k in range(count)]
    for t in th:
        t.start()
    for t in th:
        t.join()
    if errs:
        raise errs[0]
    return out


def test_shards_add_up_to_v_bit_for_bit(shgo):
    for basis, C, Z, count in ((*W.config2(), 2),
                               (*W.config1(), 3),
                               (W.random_basis(91, 14, 5, max_prim=3, box=4.0, n_sites=5), *W.random_nuclei(92, 9, box=4.0), 3)):
        Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
        Bf = shgo.Basis(basis)
        full = shgo.nuclear_attraction(Bf, Cd, Zd).cpu().numpy()
        pa_f, pb_f = shgo.pair_shells(Bf.handle, Bf.npairs)
        Bf.close()

        def v(B, s):
            out = torch.zeros((B.nbf, B.nbf), dtype=torch.float64, device="cuda")
            shgo.nuclear_attraction(B, Cd, Zd, out=out, stream=s)
            return out.cpu().numpy()

        res = run_ranks(shgo, basis, count, v)
        assert np.array_equal(sum(r[0] for r in res), full)
        # the shards' pairs are the host split of the library's pair order
        split = shgo.host_shard_of_pairs(basis["l"], basis["nprim"], count)
        for k, (_, (pa, pb)) in enumerate(res):
            want = np.flatnonzero(split == k)
            assert np.array_equal(pa, pa_f[want]) and np.array_equal(pb, pb_f[want])


def test_shards_add_up_to_the_derivative_integrals_and_gradient(shgo):
    basis = W.random_basis(93, 12, 5, max_prim=2, box=3.5, n_sites=4)
    C, Z = W.random_nuclei(94, 7, box=3.5)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    n = W.nbf(basis)
    p = np.random.default_rng(95).normal(size=(n, n))
    Pd = torch.tensor((p + p.T) / 2, device="cuda")
    Bf = shgo.Basis(basis)
    D = shgo.nuclear_attraction_deriv(Bf, Cd, Zd).cpu().numpy()
    F = shgo.nuclear_field(Bf, Cd, Zd).cpu().numpy()
    g = shgo.nuclear_attraction_gradient(Bf, Pd, Cd, Zd).cpu().numpy()
    phi = shgo.esp(Bf, Pd, Cd).cpu().numpy()
    Bf.close()

    def all_of(B, s):
        d = torch.zeros((3, n, n), dtype=torch.float64, device="cuda")
        f = torch.zeros((3, n, n), dtype=torch.float64, device="cuda")
        shgo.nuclear_attraction_deriv(B, Cd, Zd, out=d, stream=s)
        shgo.nuclear_field(B, Cd, Zd, out=f, stream=s)
        gg = shgo.nuclear_attraction_gradient(B, Pd, Cd, Zd, stream=s)
        ph = shgo.esp(B, Pd, Cd, stream=s)
        return d.cpu().numpy(), f.cpu().numpy(), gg.cpu().numpy(), ph.cpu().numpy()

    res = [r[0] for r in run_ranks(shgo, basis, 2, all_of)]
    assert np.array_equal(res[0][0] + res[1][0], D)
    assert np.array_equal(res[0][1] + res[1][1], F)
    assert np.allclose(res[0][2] + res[1][2], g, rtol=1e-12, atol=1e-12 * np.max(np.abs(g)))
    assert np.allclose(res[0][3] + res[1][3], phi, rtol=1e-12, atol=1e-12 * np.max(np.abs(phi)))


def test_shard_arguments(shgo):
    basis = W.random_basis(96, 4, 2, max_prim=2, box=2.0)
    for bad in ((2, 2), (-1, 2), (0, 0)):
        with pytest.raises(shgo.ShgoError):
            shgo.Basis(basis, shard=bad)
    B = shgo.Basis(basis, shard=(0, 2))
    with pytest.raises(shgo.ShgoError):
        shgo.eri(B)
    B.close()
