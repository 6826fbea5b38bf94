"""The bench's multi-GPU mode is replicas (each rank runs the whole stage, no collective on the
data path): its host logic -- max over ranks of the timings, whole-job throughput, the reference
arm on rank 0 only -- on world_size-2 gloo process groups on CPU."""

import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        # rank r's two timings: 10 + r and 5 - r ms; the slowest rank sets each
        ms = bench.replica_max([10.0 + rank, 5.0 - rank], dist, "cpu")
        q.put((rank, ms, bench.job_value(world, 1000, ms[0])))
    finally:
        dist.destroy_process_group()


def test_replica_timing_takes_the_max_over_ranks():
    ctx = torch.multiprocessing.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    world = 2
    procs = [ctx.Process(target=_worker, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, ms, value in out:
        assert ms == [11.0, 5.0]
        assert value == pytest.approx(2 * 1000 / 11e-3)


def test_single_rank_needs_no_process_group():
    import bench

    assert bench.replica_max([3.0, 4.0]) == [3.0, 4.0]
    assert bench.job_value(1, 500, 2.0) == pytest.approx(250000.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    import argparse

    import bench

    args = argparse.Namespace(workload="vortex64", warmup=3, steps=1)
    assert bench.reference_arm(args, rank=1, world=2) is None
    assert capsys.readouterr().out == ""
