"""The multi-process (N > 1) path of bench.py on CPU with gloo: independent
replicas, whole-job value = units of all ranks / max time over ranks."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    # rank r takes (r + 1) seconds for 1000 * (r + 1) units
    value, tmax = bench.aggregate_replicas(float(rank + 1), 1000.0 * (rank + 1), dist)
    out[rank] = (value, tmax)
    dist.barrier()
    dist.destroy_process_group()


def test_replica_aggregation_two_ranks():
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        value, tmax = out[r]
        assert tmax == 2.0 and value == (1000.0 + 2000.0) / 2.0


def test_single_process_aggregation():
    import bench
    assert bench.aggregate_replicas(2.0, 10.0) == (5.0, 2.0)
