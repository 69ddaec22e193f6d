"""Multi-rank host logic of bench.py on CPU: two gloo ranks (replicas, no
collective on the data path) agree on the slowest rank's time, and the job's
rate counts every rank's operands."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch.distributed as dist
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(10.0 + 5.0 * rank, "cpu", world)
        q.put((rank, ms, bench.job_gbit_s(2 << 24, world, ms)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    assert [g[1] for g in got] == [15.0, 15.0]           # both ranks see the max
    assert got[0][2] == pytest.approx(2 * (2 << 24) / 15e-3 / 1e9)


def test_single_rank_is_its_own_time():
    import bench
    assert bench.max_over_ranks(3.5, "cpu", 1) == 3.5
    assert bench.job_gbit_s(2 << 24, 1, 1.0) == pytest.approx((2 << 24) / 1e-3 / 1e9)
