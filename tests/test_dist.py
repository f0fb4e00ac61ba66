"""Multi-process plumbing of bench.py on the CPU: two gloo ranks (127.0.0.1) set up
the process group the way bench.py does under torchrun, pass a barrier and agree on
the maximum step time (the slowest rank sets the job's time)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank), "CUDA_VISIBLE_DEVICES": ""})
    import bench
    dist, r, w = bench.dist_setup(None)
    assert (r, w) == (rank, world)
    bench.barrier(dist)
    t = bench.max_over_ranks(dist, 1.5 + rank)          # rank 1 is the slow one
    out[rank] = t
    dist.destroy_process_group()


def test_two_gloo_ranks_agree_on_the_slowest_time():
    ctx = mp.get_context("spawn")
    out = ctx.Manager().dict()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, out)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    assert dict(out) == {0: 2.5, 1: 2.5}


def test_reference_arm_runs_only_on_rank_zero():
    import bench
    class Args:
        steps, warmup = 1, 0
    assert bench.run_reference(Args, rank=1, world=2) is None
