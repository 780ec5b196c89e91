"""bench.py's multi-rank path on the CPU: world size 2 over gloo.  Each rank
reports its own timed span and units; the whole-job line uses the longest
span and the summed units.  The reference arm runs on rank 0 only."""
from __future__ import annotations

import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    spans, units = [12.5, 30.0], [1000, 3000]
    t, u = bench.whole_job(spans[rank], units[rank], dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()
    q.put((rank, t, u))


def test_whole_job_over_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    ps = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    got = sorted(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert got == [(0, 30.0, 4000.0), (1, 30.0, 4000.0)]


def test_single_rank_is_its_own_job():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.whole_job(7.0, 11, None, "cpu") == (7.0, 11.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    # a non-zero rank returns before reading its arguments, loading a
    # workload or printing
    assert bench.reference_arm(None, 1, 2) is None
    assert capsys.readouterr().out == ""
