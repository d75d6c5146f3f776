"""bench.py's replica aggregation over two gloo ranks on the CPU: the job's
time is the slowest rank's, its iterations the sum over ranks."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    ms, it = bench.aggregate_ranks(10.0 + 5.0 * rank, 100 + rank, world, torch.device("cpu"))
    out[rank] = (ms, it)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_aggregation():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    assert out[0] == out[1] == (15.0, 201)


def test_single_rank_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(3.5, 7, 1, None) == (3.5, 7)
