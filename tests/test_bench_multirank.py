"""The multi-rank timing reduction of bench.py (replicas: slowest rank's time,
units of all ranks) on two CPU ranks over gloo."""
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
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    tmax, value = bench.job_rate(1.0 + rank, 100, world)
    out[rank] = (tmax, value)
    dist.barrier()
    dist.destroy_process_group()


def test_two_rank_replica_rate():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    for r in range(2):
        tmax, value = out[r]
        assert tmax == 2.0            # the slower rank sets the job time
        assert value == 2 * 100 / 2.0  # all ranks' units over that time
