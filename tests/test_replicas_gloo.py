"""Multi-replica bench logic on CPU: two gloo ranks on 127.0.0.1.

Each rank runs an independent replica (no data-path collective); the job
time is the maximum over ranks and the throughput is the aggregate."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", init_method="env://", rank=rank, world_size=world)
    import bench
    ms_local = [2.0, 5.0][rank]
    ms, value = bench.aggregate_over_ranks(ms_local, 1000, 10, world, dist)
    out[rank] = (ms, value)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_rank():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in range(2):
        ms, value = res[r]
        assert ms == 5.0
        assert abs(value - 1000 * 10 * 2 / 5e-3 / 1e9) < 1e-15


def test_single_rank_is_local():
    import bench
    ms, value = bench.aggregate_over_ranks(4.0, 100, 3, 1)
    assert ms == 4.0 and abs(value - 100 * 3 / 4e-3 / 1e9) < 1e-18
