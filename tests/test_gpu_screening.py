"""Screening network and learned screening on the GPU.

The network's forward pass and gradients (the library's own kernels) are checked against the numpy
reference in oracle/mlp.py; screening is checked through its limits (keep everything = the plain
method bit for bit, skip everything = zero), the features against an independent restatement, and
a trained network against the plain method on a small cluster with an exact audit."""
import math

import numpy as np
import pytest

from oracle import mlp as ref
from paper_2404_16245_gb300 import workloads as W

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")


@pytest.fixture(scope="module")
def shgo():
    from paper_2404_16245_gb300 import shgo as mod
    return mod


def test_mlp_gradients_match_reference(shgo):
    rng = np.random.default_rng(1)
    n = 333
    X = rng.normal(size=(n, 16)).astype(np.float32)
    T = rng.normal(size=n).astype(np.float32)
    mean = (rng.normal(size=16) * 0.1).astype(np.float32)
    sd = rng.uniform(0.5, 2.0, 16).astype(np.float32)
    p = W.mlp_init_params(7)
    net = shgo.MLP(p, mean, sd)
    g, loss = net.gradients(torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda"), under_weight=4.0)
    rloss, rg = ref.loss_and_grad(p, X, T, mean.astype(np.float64), sd.astype(np.float64), under_weight=4.0)
    assert loss == pytest.approx(rloss, rel=1e-4)
    scale = np.max(np.abs(rg))
    assert np.max(np.abs(g - rg)) <= 2e-4 * scale, np.max(np.abs(g - rg)) / scale
    y = net.forward(torch.tensor(X, device="cuda")).cpu().numpy()
    ry, _ = ref.forward(p, X, mean.astype(np.float64), sd.astype(np.float64))
    assert np.max(np.abs(y - ry)) <= 1e-4 * (1 + np.max(np.abs(ry)))
    net.close()


def test_mlp_training_reduces_loss(shgo):
    rng = np.random.default_rng(2)
    X = rng.normal(size=(8192, 16)).astype(np.float32)
    w = rng.normal(size=16)
    T = (X @ w + 0.5 * np.sin(X[:, 0])).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    net = shgo.MLP(W.mlp_init_params(0), np.zeros(16), np.ones(16))
    _, l0 = net.gradients(Xd, Td)
    for _ in range(300):
        net.train_step(Xd, Td, 1.0, 3e-3)
    _, l1 = net.gradients(Xd, Td)
    assert l1 < 0.05 * l0, (l0, l1)
    net.close()


def cluster(seed, n_atoms):
    rng = np.random.Generator(np.random.PCG64(seed))
    box = (n_atoms / 0.1) ** (1 / 3)
    return W.molecule(rng, n_atoms, box, 1, 9, lambda Z: [0] * 4 + [1] * 3 + [2] * 2 + [3],
                      lambda r: r.integers(1, 7), 0.05, 5000.0)


def const_net(shgo, bias):
    p = np.zeros(ref.NPARAM, dtype=np.float32)
    p[-1] = bias
    return shgo.MLP(p, np.zeros(16), np.ones(16))


def test_keep_all_equals_plain_and_skip_all_is_zero(shgo):
    basis, C, Z = cluster(41, 8)
    B = shgo.Basis(basis)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    plain = shgo.nuclear_attraction(B, Cd, Zd).cpu().numpy()
    keep = const_net(shgo, 100.0)
    kept, skipped = shgo.screen_build(B.handle, keep, Cd, Zd, len(Z), -12.0, 2.0)
    assert skipped == 0 and kept == B.npairs * len(Z)
    out = torch.empty_like(torch.tensor(plain, device="cuda"))
    shgo.nuclear_attraction_screened(B.handle, Cd, Zd, len(Z), out)
    assert np.array_equal(out.cpu().numpy(), plain)
    drop = const_net(shgo, -100.0)
    kept, skipped = shgo.screen_build(B.handle, drop, Cd, Zd, len(Z), -12.0, 2.0)
    assert kept == 0
    shgo.nuclear_attraction_screened(B.handle, Cd, Zd, len(Z), out)
    assert np.array_equal(out.cpu().numpy(), np.zeros_like(plain))
    B.close()


def test_features_match_definitions(shgo):
    basis, C, Z = cluster(43, 6)
    B = shgo.Basis(basis)
    a, b = shgo.pair_shells(B.handle, B.npairs)
    rng = np.random.default_rng(0)
    tr = np.stack([rng.integers(0, B.npairs, 50), rng.integers(0, len(Z), 50)], axis=1).astype(np.int32)
    X = shgo.screen_features(B.handle, torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda"),
                             torch.tensor(tr, device="cuda")).cpu().numpy()
    poff = np.concatenate([[0], np.cumsum(basis["nprim"])])
    for t, (q, c) in enumerate(tr):
        sa, sb = a[q], b[q]
        ea = basis["exps"][poff[sa]:poff[sa + 1]]
        eb = basis["exps"][poff[sb]:poff[sb + 1]]
        A, Bc, Cc = basis["xyz"][sa], basis["xyz"][sb], C[c]
        amin, bmin = ea.min(), eb.min()
        P = (amin * A + bmin * Bc) / (amin + bmin)
        assert X[t, 0] == basis["l"][sa] and X[t, 1] == basis["l"][sb]
        assert X[t, 2] == pytest.approx(math.log10(amin), abs=1e-5)
        assert X[t, 5] == pytest.approx(math.log10(eb.max()), abs=1e-5)
        assert X[t, 6] == pytest.approx(np.linalg.norm(Bc - A), abs=1e-4)
        assert X[t, 7] == pytest.approx(-amin * bmin / (amin + bmin) * np.sum((Bc - A) ** 2) / math.log(10), rel=1e-5,
                                        abs=1e-4)
        assert X[t, 8] == pytest.approx(np.linalg.norm(P - Cc), abs=1e-4)
        assert X[t, 10] == pytest.approx(math.log10(Z[c]), abs=1e-6)
        assert X[t, 13] == pytest.approx(np.linalg.norm(A - Cc), abs=1e-4)
    B.close()


def test_trained_screening_error_and_audit(shgo):
    # the rule the library documents: per-triple threshold = target / number of nuclei, margin
    # calibrated on held-out labelled triples
    from paper_2404_16245_gb300 import screening as S
    train_basis, Ct, Zt = cluster(44, 14)
    Bt = shgo.Basis(train_basis)
    a, b = shgo.pair_shells(Bt.handle, Bt.npairs)
    rng = np.random.default_rng(5)
    dist = np.linalg.norm(train_basis["xyz"][a] - train_basis["xyz"][b], axis=1)
    tr = S.sample_triples(rng, Bt.npairs, len(Zt), 60000, pair_dist=dist)
    T = S.plain_labels(train_basis, a, b, Ct, Zt, tr)
    X = shgo.screen_features(Bt.handle, torch.tensor(Ct, device="cuda"), torch.tensor(Zt, device="cuda"),
                             torch.tensor(tr, device="cuda"))
    nval = 6000
    Tt = torch.tensor(T, dtype=torch.float32, device="cuda")
    net, losses = S.train(X[nval:].contiguous(), Tt[nval:].contiguous(), epochs=8, batch=2048)
    assert losses[-1] < losses[0]
    Bt.close()
    basis, C, Z = cluster(45, 12)
    target = 1e-10
    cut = math.log10(target / len(Z))
    margin = S.calibrate_margin(net, X[:nval].contiguous(), T[:nval], cut)
    B = shgo.Basis(basis)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    plain = shgo.nuclear_attraction(B, Cd, Zd).cpu().numpy()
    kept, skipped = shgo.screen_build(B.handle, net, Cd, Zd, len(Z), cut, margin)
    out = torch.empty((B.nbf, B.nbf), dtype=torch.float64, device="cuda")
    shgo.nuclear_attraction_screened(B.handle, Cd, Zd, len(Z), out)
    err = np.max(np.abs(out.cpu().numpy() - plain))
    a, b = shgo.pair_shells(B.handle, B.npairs)
    mask = shgo.screen_mask(B.handle, kept + skipped)
    rep = S.audit(basis, a, b, C, Z, mask, np.full(B.npairs, len(Z)), 0.05, np.random.default_rng(1), 10 ** cut)
    print(f"\nscreening: margin {margin:.2f}; kept {kept} skipped {skipped}; max |V - V_plain| {err:.2e}; audit {rep}")
    assert skipped > 0
    assert err < target
    assert rep["false_skip_rate"] < 0.01
    B.close()
    net.close()


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_repeated_screened_calls_keep_all(shgo, precision):
    """Every call of the screened entry point (the tuning call, the graph capture and the replays) gives
    the plain result when the network keeps every triple: bit for bit in FP64, and to the FP32-bulk
    block accuracy otherwise."""
    prec = shgo.SHGO_PREC_FP64 if precision == "fp64" else shgo.SHGO_PREC_FP32_BULK
    basis, C, Z = cluster(46, 30)
    B = shgo.Basis(basis, precision=prec)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    plain = shgo.nuclear_attraction(B, Cd, Zd).cpu().numpy()
    keep = const_net(shgo, 100.0)
    kept, skipped = shgo.screen_build(B.handle, keep, Cd, Zd, len(Z), -12.0, 2.0)
    assert skipped == 0
    out = torch.empty((B.nbf, B.nbf), dtype=torch.float64, device="cuda")
    for call in range(4):
        out.fill_(float("nan"))
        shgo.nuclear_attraction_screened(B.handle, Cd, Zd, len(Z), out)
        got = out.cpu().numpy()
        diff = float(np.max(np.abs(got - plain)))
        if precision == "fp64":
            assert np.array_equal(got, plain), (call, diff)
        else:
            assert diff <= 1e-10 * max(1.0, float(np.max(np.abs(plain)))), (call, diff)
    B.close()
    keep.close()


def charge_net(shgo):
    """A hand-set network whose prediction falls with the nucleus charge (feature 10 is log10 Z):
    y = 10 - silu(silu(10 log10 Z + 5)), at or above 0 exactly for Z <= 3."""
    H, IN = 64, 16
    W1 = np.zeros((H, IN))
    b1 = np.zeros(H)
    W2 = np.zeros((H, H))
    W3 = np.zeros(H)
    W1[0, 10], b1[0], W2[0, 0], W3[0] = 10.0, 5.0, 1.0, -1.0
    p = np.concatenate([W1.ravel(), b1, W2.ravel(), np.zeros(H), W3, [10.0]]).astype(np.float32)
    assert p.size == ref.NPARAM
    return shgo.MLP(p, np.zeros(16), np.ones(16))


def test_ragged_nucleus_lists_equal_plain_over_the_kept_nuclei(shgo):
    """A mask that keeps, for every pair, the nuclei with Z <= 3 gives each pair a nucleus list
    shorter than the molecule's (a partial chunk): the screened V equals the plain V over those
    nuclei bit for bit, on every call (tuning, capture, replays)."""
    basis, C, Z = cluster(47, 30)
    keep_z = Z <= 3
    assert 0 < keep_z.sum() < len(Z)
    B = shgo.Basis(basis)
    Cd, Zd = torch.tensor(C, device="cuda"), torch.tensor(Z, device="cuda")
    expect = shgo.nuclear_attraction(B, torch.tensor(C[keep_z], device="cuda"),
                                     torch.tensor(Z[keep_z], device="cuda")).cpu().numpy()
    net = charge_net(shgo)
    kept, skipped = shgo.screen_build(B.handle, net, Cd, Zd, len(Z), 0.0, 0.0)
    assert kept == B.npairs * int(keep_z.sum()) and skipped == B.npairs * int((~keep_z).sum())
    out = torch.empty((B.nbf, B.nbf), dtype=torch.float64, device="cuda")
    for call in range(3):
        out.fill_(float("nan"))
        shgo.nuclear_attraction_screened(B.handle, Cd, Zd, len(Z), out)
        assert np.array_equal(out.cpu().numpy(), expect), call
    B.close()
    net.close()


def test_training_repeats_and_resumes_bit_for_bit(shgo):
    """Training sums in a fixed order: two runs from one initial state over the same batches give the
    same parameters bit for bit, and stopping after 7 steps, saving the state (parameters, Adam moments,
    step count), loading it into a fresh network and running the remaining steps gives them too.  The
    sample count is not a multiple of the 32-sample tile."""
    rng = np.random.default_rng(5)
    X = rng.normal(size=(5000, 16)).astype(np.float32)
    T = (X @ rng.normal(size=16) + np.sin(X[:, 1])).astype(np.float32)
    Xd, Td = torch.tensor(X, device="cuda"), torch.tensor(T, device="cuda")
    batches = [(int(s), int(s) + 1500) for s in rng.integers(0, 5000 - 1500, 18)]
    mean, sd = X.mean(axis=0), X.std(axis=0)

    def run(steps, state=None):
        net = shgo.MLP(W.mlp_init_params(3), mean, sd)
        if state is not None:
            net.load_state(state)
        done = state["step"] if state is not None else 0
        for k in range(done, steps):
            a, b = batches[k]
            net.train_step(Xd[a:b].contiguous(), Td[a:b].contiguous(), 4.0, 2e-3)
        torch.cuda.synchronize()
        st = net.state()
        net.close()
        return st

    full1 = run(18)
    full2 = run(18)
    assert np.array_equal(full1["params"], full2["params"])
    assert np.array_equal(full1["adam_v"], full2["adam_v"]) and full1["step"] == 18
    part = run(7)
    resumed = run(18, part)
    assert np.array_equal(resumed["params"], full1["params"])
    assert np.array_equal(resumed["adam_m"], full1["adam_m"])
    # training moved the parameters
    assert not np.array_equal(full1["params"], W.mlp_init_params(3))
