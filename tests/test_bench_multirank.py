"""The multi-GPU path of bench.py runs independent replicas (one cavity per
rank, no data-path collective); the only communication is the max over ranks
of the timed region.  Exercised here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks(100.0 + 10.0 * rank)
    out[rank] = got
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    assert out[0] == out[1] == 110.0


def test_job_value_is_weak_scaled():
    import bench
    one = bench.job_value(1, 10, 1000.0)
    two = bench.job_value(2, 10, 1000.0)
    assert one == bench.FIELDS * 10 / 1.0
    assert two == 2 * one
