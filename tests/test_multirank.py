"""The N > 1 path of bench.py (independent replicas, one per GPU): the job
time is the slowest rank's time and the value counts every rank's points.
Run as two gloo ranks on the CPU (no GPU, no data-path collective)."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    my_ms = [120.0, 95.5][rank]
    out[rank] = bench.max_over_ranks(my_ms, world, torch, dist, "cpu")
    dist.barrier()
    dist.destroy_process_group()


def test_max_over_ranks_gloo_world_2():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank, args=(2, port, out), nprocs=2, join=True)
        assert out[0] == 120.0 and out[1] == 120.0


def test_single_rank_and_job_value():
    assert bench.max_over_ranks(42.0, 1, torch, None, "cpu") == 42.0
    # 2 replicas x 1.31M points x 10 steps in 55 ms (slowest rank)
    v = bench.job_value(1_310_720, 10, 2, 55.0)
    assert v == pytest.approx(1_310_720 * 10 * 2 / 0.055 / 1e6)
