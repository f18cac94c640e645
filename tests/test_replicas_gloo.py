"""The multi-GPU path is replicas only (independent scenarios per GPU, no
exchange step): two gloo ranks on the CPU check the bench's aggregation of
the ranks' timed regions and work."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t, w = bench.aggregate_over_ranks(1.5 + rank, 100.0 * (rank + 1), dist, torch.device("cpu"))
    out[rank] = (t, w)
    dist.destroy_process_group()


def test_two_replicas_take_the_slowest_time_and_the_total_work():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = _free_port()
        procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in procs:
            p.start()
        for p in procs:
            p.join(120)
        assert all(p.exitcode == 0 for p in procs)
        assert out[0] == out[1] == (2.5, 300.0)
