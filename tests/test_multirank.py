"""The benchmark's multi-rank path on CPU (gloo, world size 2): every rank
morphs its own batch (no data-path collective), and rank 0 reports the
whole-job rate from the slowest rank's time."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, times, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w, r, _ = bench.dist_setup()
        assert (w, r) == (world, rank)
        bench.barrier(world)
        t = bench.max_over_ranks(world, times[rank])
        out[rank] = (t, bench.whole_job_rate(world, 1.0e12, 5, t), bench.rank_sample_seed(rank))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_work():
    world, port = 2, _free_port()
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    times = [1.5, 2.0]
    mp.start_processes(_worker, args=(world, port, times, out), nprocs=world, start_method="spawn", join=True)
    for rank in range(world):
        t, rate, seed = out[rank]
        assert t == 2.0                                  # max over ranks
        assert rate == pytest.approx(2 * 1.0e12 * 5 / 2.0)
    assert out[0][2] != out[1][2]                        # each rank morphs its own samples


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(1, 3.25) == 3.25
    assert bench.whole_job_rate(1, 2.0, 4, 8.0) == 1.0
