"""The bench's multi-rank path on CPU: two gloo ranks, each with its own timed span, agree on
the slowest span (all-reduce MAX) and on the whole-job rate (all ranks' units over it)."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    span = 1.5 + rank            # rank 1 is the slower one
    slow = bench.max_over_ranks(span, dist)
    rate = bench.whole_job_rate(10, world, slow)
    out[rank] = (slow, rate)
    dist.destroy_process_group()


def test_max_over_ranks_and_rate_with_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
        res = dict(out)
    assert res[0] == res[1] == (2.5, 20 / 2.5)


def test_single_rank_has_no_collective():
    import bench
    assert bench.max_over_ranks(3.0, None) == 3.0
    assert bench.whole_job_rate(7, 1, 2.0) == 3.5
