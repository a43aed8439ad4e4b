"""The N > 1 benchmark path on the CPU: world size 2 over gloo.

The path shards into independent replicas (no data exchange), so what several ranks add is host
logic: disjoint seeded replicas per rank, the step time taken as the maximum over ranks, and the
reference arm printing one line from rank 0 while the other ranks exit without work."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, totals, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        q.put((rank, bench.max_over_ranks(totals[rank], ws), bench.replica_seeds(rank, 4)))
    finally:
        dist.destroy_process_group()


def test_step_time_is_max_over_ranks_and_replicas_are_disjoint():
    ws, totals = 2, [3.5, 7.25]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, ws, port, totals, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = [q.get(timeout=120) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    by_rank = {r: (m, seeds) for r, m, seeds in got}
    assert by_rank[0][0] == by_rank[1][0] == max(totals)
    assert set(by_rank[0][1]).isdisjoint(by_rank[1][1])
    assert sorted(by_rank[0][1] + by_rank[1][1]) == list(range(8))


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(2.5, 1) == 2.5
    assert bench.replica_seeds(0, 3) == [0, 1, 2]


def test_reference_arm_under_torchrun_prints_once_from_rank_zero():
    port = free_port()
    env = dict(os.environ, OMP_NUM_THREADS="1")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0"]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["e2e"]["h2d_bytes_per_step"] == 0


# ---- one basis split over ranks (shgo_basis_create_shard): the host split, checked across gloo ranks ----

def _library_pair_order(l, nprim):
    """(a, b, primitive pairs) of every shell pair in the library's documented order: classes (la >= lb) in
    increasing la then lb, inside a class a over the shells of l = la, b over those of l = lb (b <= a when
    la = lb), each in shell-index order."""
    import numpy as np
    l = np.asarray(l)
    pairs = []
    for la in range(9):
        A = [int(s) for s in np.flatnonzero(l == la)]
        for lb in range(la + 1):
            B = [int(s) for s in np.flatnonzero(l == lb)]
            for x, a in enumerate(A):
                for b in (A[:x + 1] if la == lb else B):
                    pairs.append((la, lb, a, b, int(nprim[a] * nprim[b])))
    return pairs


def _shard_worker(rank, ws, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        from paper_2404_16245_gb300 import shgo
        from paper_2404_16245_gb300 import workloads as W
        import numpy as np
        b = W.config3_molecule(np.random.Generator(np.random.PCG64(3000)))[0]
        mine = [int(x) for x in np.flatnonzero(shgo.host_shard_of_pairs(b["l"], b["nprim"], ws) == rank)]
        allsets = [None] * ws
        dist.all_gather_object(allsets, mine)
        q.put((rank, allsets, np.asarray(b["l"]).tolist(), np.asarray(b["nprim"]).tolist()))
    finally:
        dist.destroy_process_group()


def test_one_basis_split_over_ranks_is_a_balanced_partition():
    pytest.importorskip("paper_2404_16245_gb300.shgo", reason="libshgo.so not built")
    ws = 2
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_shard_worker, args=(r, ws, port, q)) for r in range(ws)]
    for p in procs:
        p.start()
    got = [q.get(timeout=180) for _ in range(ws)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    _, sets, l, nprim = got[0]
    assert got[1][1] == sets  # both ranks see the same split
    pairs = _library_pair_order(l, nprim)
    owner = {}
    for r, s in enumerate(sets):
        for q_ in s:
            assert q_ not in owner
            owner[q_] = r
    assert sorted(owner) == list(range(len(pairs)))  # every pair on exactly one rank
    # per class, each rank's primitive pairs are within one pair's worth of an equal share
    classes = {}
    for q_, (la, lb, a, b, npp) in enumerate(pairs):
        c = classes.setdefault((la, lb), [[0] * ws, 0, 0])
        c[0][owner[q_]] += npp
        c[1] += npp
        c[2] = max(c[2], npp)
    for (la, lb), (per, tot, big) in classes.items():
        for r in range(ws):
            assert abs(per[r] - tot / ws) <= big, (la, lb, per, tot)
