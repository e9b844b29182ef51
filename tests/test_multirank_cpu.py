"""The bench's N > 1 path on CPU: two gloo ranks, replicas, max-over-ranks timing.

With several GPUs every rank solves its own replica of the workload (the solve itself is
single-GPU); the only cross-rank steps are the barrier and the max-reduction of the timed
region, checked here with the gloo backend on CPU.
"""
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


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    import bench

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    slow = bench.max_over_ranks(1.0 + rank, world)  # rank 1 is the slower one
    rate = bench.whole_job_rate(100.0, world, slow)
    dist.barrier()
    out[rank] = (slow, rate)
    dist.destroy_process_group()


def test_two_rank_replicas_take_the_slowest_time():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank_main, args=(world, port, out), nprocs=world, start_method="spawn")
    assert out[0] == out[1] == (2.0, 100.0)


def test_single_rank_is_identity():
    import bench

    assert bench.max_over_ranks(3.5, 1) == 3.5
    assert bench.whole_job_rate(10.0, 1, 2.0) == 5.0
