"""Multi-process (world size 2, gloo, CPU) coverage of the benchmark's replica
aggregation: the job time is the maximum over ranks and the work is summed."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms, work = bench.aggregate_ranks(10.0 * (rank + 1), 100.0 * (rank + 1))
    out[rank] = (ms, work)
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_max_time_and_summed_work():
    import socket

    import torch.multiprocessing as mp
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    mgr = mp.Manager()
    out = mgr.dict()
    mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
    assert out[0] == out[1] == (20.0, 300.0)


def test_single_process_passthrough():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate_ranks(3.5, 7.0) == (3.5, 7.0)
