"""The multi-GPU path of bench.py on CPU: two gloo ranks, each an independent replica (no
collective on the data path); the whole-job value is every rank's updates over the slowest
rank's timed region."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import sys

    import torch.distributed as dist

    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    ms_local = [12.0, 20.0][rank]  # rank 1 is the slowest
    units_local = [1000, 3000][rank]
    ms, units, value = bench.aggregate(ms_local, units_local, dist, "cpu")
    dist.barrier()
    out[rank] = (ms, units, value)
    dist.destroy_process_group()


def test_two_replicas_aggregate_over_the_slowest_rank():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    for r in range(2):
        ms, units, value = res[r]
        assert ms == 20.0 and units == 4000.0
        assert abs(value - 4000.0 / 0.020) < 1e-6


def test_single_process_aggregate_is_local():
    import bench

    assert bench.aggregate(10.0, 500) == (10.0, 500, 50000.0)
