"""Multi-GPU runs are independent replicas (the step has no data exchange on
one GPU per rank); only the timing is reduced.  Checked here with two gloo
ranks on the CPU: the job time is the slowest rank's, the value counts every
rank's steps."""
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


def _rank(rank, world, port, out):
    import torch.distributed as dist
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms = 1000.0 * (rank + 1)                  # rank 1 is the slow one
    out[rank] = bench.reduce_timing(ms, steps=3, world=world, device="cpu")
    dist.destroy_process_group()


def test_timing_reduction_two_ranks():
    world = 2
    port = _free_port()
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    procs = [ctx.Process(target=_rank, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    for r in range(world):
        ms, value = out[r]
        assert ms == 2000.0                    # max over ranks
        assert abs(value - 3.0) < 1e-12        # 2 ranks x 3 steps / 2 s


def test_single_rank_needs_no_group():
    import bench
    assert bench.reduce_timing(500.0, 2, 1) == (500.0, 4.0)
