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
