"""The multi-rank path of bench.py on CPU: two gloo ranks, each with its own
(independent) problem; the job's step time is the slowest rank's and the
job rate adds the ranks' work (weak scaling).  No GPU."""
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


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    r, w, d = bench.dist_init("gloo")
    assert (r, w) == (rank, world)
    step_s = 0.5 + rank  # rank 1 is the slowest
    d.barrier()
    t = bench.max_over_ranks(step_s, d)
    out[rank] = (t, bench.job_rate(4.0e9, w, t))
    d.destroy_process_group()


@pytest.mark.parametrize("world", [2])
def test_two_gloo_ranks_take_the_max_and_add_the_work(world):
    out = mp.Manager().dict()
    mp.spawn(_rank, args=(world, _free_port(), out), nprocs=world, join=True)
    for rank in range(world):
        t, rate = out[rank]
        assert t == pytest.approx(0.5 + world - 1)
        assert rate == pytest.approx(world * 4.0e9 / t / 1e9)


def test_single_process_needs_no_group():
    import bench
    assert bench.max_over_ranks(1.25, None) == 1.25
    assert bench.job_rate(2e9, 1, 2.0) == pytest.approx(1.0)
