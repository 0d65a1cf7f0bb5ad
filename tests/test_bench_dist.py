"""bench.py's multi-rank host logic on CPU: with world size 2 over gloo, every rank runs its
own replica and the reported time is the maximum over ranks (no collective on the data
path).  The GPU launch of the same path uses NCCL for the barrier and this reduction."""
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    got = bench.max_over_ranks(10.0 + rank * 5.0, dist, device="cpu")
    dist.barrier()
    out[rank] = got
    dist.destroy_process_group()


def test_max_over_ranks_world2():
    mgr = mp.Manager()
    out = mgr.dict()
    port = _free_port()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == 15.0


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(3.5, None) == 3.5
