"""Replica timing over two ranks with the gloo backend on CPU."""
import os

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1711_10579_gb300 import replicas


def _rank(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        local_ms = [100.0, 250.0][rank]
        local_ok = [40, 38][rank]
        value, ms, total = replicas.aggregate(local_ms, local_ok, dist)
        out[rank] = (value, ms, total, replicas.scenario_seed(5, rank))
    finally:
        dist.destroy_process_group()


def test_two_rank_aggregate_is_max_time_and_total_count():
    port = 29500 + os.getpid() % 1000
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_rank, args=(2, port, out), nprocs=2, start_method="spawn")
        r0, r1 = out[0], out[1]
    assert r0[:3] == r1[:3]
    assert r0[1] == 250.0 and r0[2] == 78
    assert r0[0] == pytest.approx(78 / 0.25)
    assert r0[3] != r1[3]


def test_single_process_aggregate():
    value, ms, total = replicas.aggregate(50.0, 10, None)
    assert value == pytest.approx(200.0) and ms == 50.0 and total == 10
