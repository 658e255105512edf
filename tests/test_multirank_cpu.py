"""The multi-GPU bench path is replicas only: each rank runs its own system
and the whole-job rate is the summed simulated time over the slowest rank's
wall time. Checked here with two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    times = [1.0 + rank, 2.0 - rank, 0.5]           # rank 0: [1, 2, .5], rank 1: [2, 1, .5]
    got = bench.max_over_ranks(times, dist, "cpu")
    rate = bench.replica_ns_per_day(world, 100, 3.0, got[0])
    out[rank] = (got, rate)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_sum_replicas():
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    for rank in range(2):
        got, rate = out[rank]
        assert got == [2.0, 2.0, 0.5]
        # 2 replicas x 100 steps x 3 fs in 2 s
        assert rate == pytest.approx(2 * 100 * 3.0 / 1e6 / 2.0 * 86400.0)


def test_single_process_is_identity():
    assert bench.max_over_ranks([1.0, 2.0], None) == [1.0, 2.0]
