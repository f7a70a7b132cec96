"""The multi-rank path of bench.py on CPU: two gloo ranks reduce their timings and work counts
the way the GPU ranks do (max of the time, sum of the units) and get independent inputs."""
import os
import socket

import pytest
import torch
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
    elapsed, units = bench.reduce_over_ranks(dist, "cpu", 1.5 + rank, 100 * (rank + 1))
    out[rank] = (elapsed, units, bench.rank_seed(17, rank))
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_reduction_and_seeds():
    world = 2
    port = _free_port()
    manager = mp.Manager()
    out = manager.dict()
    mp.spawn(_worker, args=(world, port, out), nprocs=world, join=True)
    assert out[0][:2] == (2.5, 300) and out[1][:2] == (2.5, 300)
    assert out[0][2] != out[1][2]
    assert out[0][2] == 17
