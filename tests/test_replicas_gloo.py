"""The multi-GPU form is replicas only: each rank runs its own requests, the
job time is the slowest rank's (all-reduce MAX) and the job rate counts every
rank's units.  Checked with two gloo ranks on the CPU."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [10.0 + 5.0 * rank, 20.0 - 3.0 * rank]          # rank 1 slower on the first, faster on the second
        got = bench.replica_times(mine, dist, torch.device("cpu"))
        q.put((rank, got, bench.job_rate(8192 * 5, world, got[0])))
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_rank():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    ps = [ctx.Process(target=_rank, args=(r, world, port, q)) for r in range(world)]
    for p in ps:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in ps:
        p.join(timeout=60)
        assert p.exitcode == 0
    for rank, got, rate in res:
        assert got == [15.0, 20.0]                             # element-wise max over ranks
        assert rate == pytest.approx(8192 * 5 * 2 / 0.015)     # both ranks' samples / slowest time


def test_single_process_needs_no_group():
    assert bench.replica_times([3.0, 4.0], None, torch.device("cpu")) == [3.0, 4.0]
    assert bench.job_rate(100, 1, 1000.0) == 100.0
