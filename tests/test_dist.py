"""The multi-GPU form is replicas only: every rank counts its own graph (or
serves its own request stream) and the job's figures are the max of the
ranks' times and the sum of their work.  That host-side logic runs here on
CPU processes over gloo, world size 2."""
from __future__ import annotations

import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")


def free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank: int, world: int, port: int, out):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mx, sm = bench.reduce_over_ranks([10.0 * (rank + 1), -rank], [rank + 1, 2.5], device="cpu")
        cat = bench.gather_over_ranks(np.arange(rank + 1, dtype=np.float64) + 100 * rank)
        dist.barrier()
        out.put((rank, mx, sm, cat.tolist()))
    finally:
        dist.destroy_process_group()


def test_reductions_over_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, mx, sm, cat in res:
        assert mx == [20.0, 0.0]            # max over ranks
        assert sm == [3.0, 5.0]             # sum over ranks
        assert cat == [0.0, 100.0, 101.0]   # rank 0's array, then rank 1's


def test_reductions_are_the_identity_on_one_rank():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks([1.5, 2.0], [3.0], device="cpu") == ([1.5, 2.0], [3.0])
    a = np.array([4.0, 5.0])
    assert bench.gather_over_ranks(a) is a


def test_reference_arm_prints_once_under_torchrun():
    """`bench.py --impl reference` launched like the multi-GPU bench: rank 0
    alone runs the oracle and prints one line; the other rank exits 0."""
    port = free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--workload", "rmat-s14"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, capture_output=True, text=True, timeout=600, cwd=ROOT, env=env)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "edges/s"
    assert d["cpu_baseline"]["kind"] == "oracle"
