"""Host logic of the multi-GPU benchmark path, on CPU with world size 2 over
gloo: every rank runs its own filter (another seed), timings are reduced to
the maximum over ranks, and rank 0 alone prints the reference arm's line."""
import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _max_worker(rank, world, port, q):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    got = bench.max_over_ranks([10.0 + rank, 5.0 - rank, 7.5], dist)
    q.put((rank, got))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.SimpleQueue()
    port = _free_port()
    procs = [ctx.Process(target=_max_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    res = dict(q.get() for _ in range(2))
    for r in range(2):
        assert res[r] == [11.0, 5.0, 7.5]


def test_every_rank_runs_an_independent_filter():
    sys.path.insert(0, ROOT)
    import bench
    a, b = bench.make_problem("plain-64", 0), bench.make_problem("plain-64", 1)
    assert a.n == b.n and a.d == b.d and a.K == b.K
    assert a.seed != b.seed
    assert not np.array_equal(a.truth, b.truth) and not np.array_equal(a.prior, b.prior)
    np.testing.assert_array_equal(a.prior, bench.make_problem("plain-64", 0).prior)   # seeded


def test_reference_arm_prints_once_under_two_ranks():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--gpus", "2", "--impl", "reference", "--workload", "plain-64", "--steps", "1", "--warmup", "0",
           "--ref-step-s", "0.3"]
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["cpu_baseline"]["kind"] == "oracle"
