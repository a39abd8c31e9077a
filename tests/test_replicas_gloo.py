"""The N > 1 path of bench.py on the CPU: two gloo ranks run independent
replicas, the job time is the slowest rank's and the rate counts every
rank's particles.  (No GPU; the GPU path uses the same functions over NCCL.)"""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, l = bench.dist_env()
        # rank-dependent timings: rank 1 is the slow one
        ms = [10.0 + 5.0 * r, 3.0 + r]
        mx = bench.replica_aggregate(ms, dist, "cpu")
        out[r] = (w, l, mx, bench.replica_rate(w, 1000, 4, mx[0]))
    finally:
        dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank_and_count_all_particles():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        ctx = mp.get_context("spawn")
        procs = [ctx.Process(target=_rank, args=(r, world, PORT, out))
                 for r in range(world)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(60)
            assert p.exitcode == 0
        res = dict(out)
    assert set(res) == {0, 1}
    for r in (0, 1):
        w, l, mx, rate = res[r]
        assert w == 2 and l == r
        assert mx == [15.0, 4.0]                       # max over ranks, per quantity
        assert rate == pytest.approx(2 * 1000 * 4 / 0.015)  # all particles / slowest time


PORT = _free_port()


def test_single_process_aggregate_is_identity():
    import bench
    assert bench.replica_aggregate([1.5, 2.5]) == [1.5, 2.5]
    assert bench.replica_rate(1, 100, 2, 1000.0) == pytest.approx(200.0)
