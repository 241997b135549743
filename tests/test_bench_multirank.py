"""The replicated (N > 1) timing path of bench.py on two gloo ranks (CPU):
the job time is the slowest rank's and the agent count the sum over ranks."""
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
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank,
                            world_size=world)
    t, a = bench.job_totals(10.0 + 5.0 * rank, 1000 * (rank + 1), world, "cpu")
    out[rank] = (t, a)
    dist.barrier()
    dist.destroy_process_group()


def test_job_totals_two_ranks():
    ctx = mp.get_context("spawn")
    mgr = ctx.Manager()
    out = mgr.dict()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    assert out[0] == out[1] == (15.0, 3000)


def test_job_totals_single_rank():
    import bench
    assert bench.job_totals(7.5, 42, 1, "cpu") == (7.5, 42)
