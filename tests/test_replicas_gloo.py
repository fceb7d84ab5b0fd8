"""The multi-replica path of bench.py on the CPU: two gloo ranks (127.0.0.1).

Each GPU runs an independent replica of the solve (the path has no exchange
step); the job's time is the slowest rank's (all-reduce MAX) and its
throughput counts every rank's units.
"""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch.distributed as dist

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import bench

    w, r, local = bench.dist_setup()
    assert (w, r, local) == (world, rank, rank)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = 10.0 + 5.0 * rank  # rank 1 is the slow replica
        job_ms = bench.replica_max(mine, "cpu")
        out[rank] = (job_ms, bench.job_rate(w, 4, job_ms * 1e-3))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_gloo_replicas_take_the_slowest_time():
    world, port = 2, _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    assert res[0] == res[1]                   # every rank reports the same job time
    assert res[0][0] == pytest.approx(15.0)   # the slowest replica's
    assert res[0][1] == pytest.approx(2 * 4 / 15e-3)  # all ranks' units over that time


def test_single_process_needs_no_group():
    import bench

    assert bench.replica_max(3.5, "cpu") == 3.5
    assert bench.job_rate(1, 10, 2.0) == 5.0
