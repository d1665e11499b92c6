"""Multi-rank logic of bench.py on CPU (gloo, world size 2): units are summed over ranks and the
time is the slowest rank's, so value = total snapshots / max time (weak scaling)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank)})
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    units, secs = bench.aggregate(100 * (rank + 1), 2.0 + rank)
    bench.barrier()
    out[rank] = (units, secs)
    assert bench.dist_env() == (world, rank, rank)
    dist.destroy_process_group()


def test_aggregate_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, port, out), nprocs=world, start_method="spawn")
    assert out[0] == out[1] == (300.0, 3.0)


def test_aggregate_single_process():
    import bench
    assert bench.aggregate(384, 1.5) == (384.0, 1.5)
