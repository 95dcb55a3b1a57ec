"""Host logic of bench.py's multi-GPU replicas, on CPU with two gloo ranks
(no GPU): disjoint designs per rank and the whole-job time taken as the
slowest rank's timed region over all ranks' cells."""
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
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        mine = [40.0, 90.0][rank]          # rank 1 is the slower one
        total, per_cell = bench.job_ms_per_cell(mine, steps=5, world=world, dist=dist)
        out[rank] = (total, per_cell, bench.rank_seeds(rank, 8))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregation_and_disjoint_designs():
    world = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, start_method="spawn")
    assert out[0][0] == out[1][0] == 90.0
    assert out[0][1] == out[1][1] == pytest.approx(90.0 / (5 * 2))
    assert not set(out[0][2]) & set(out[1][2])


def test_single_rank_needs_no_collective():
    assert bench.job_ms_per_cell(30.0, steps=3, world=1) == (30.0, 10.0)
