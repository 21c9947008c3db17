"""Host logic of bench.py's multi-rank run (replicas), as two gloo ranks on the CPU:
the timed region's max over ranks, the whole-job throughput, and the reference arm's
rank filter (rank 0 alone runs the oracle)."""
import argparse
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


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = bench.max_over_ranks(torch, dist, 10.0 + 5.0 * rank, world, torch.device("cpu"))
        out[rank] = (ms, bench.job_throughput(1000, world, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_all_units():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    for r in range(world):
        ms, value = out[r]
        assert ms == 15.0                       # the slower rank's time on every rank
        assert value == pytest.approx(2000 / 15e-3)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks(torch, None, 3.5, 1, torch.device("cpu")) == 3.5
    assert bench.job_throughput(10, 1, 1000.0) == 10.0


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    monkeypatch.setenv("RANK", "1")
    args = argparse.Namespace(gpus=2, steps=1, warmup=3, impl="reference", no_e2e=False)
    assert bench.run_reference(args) is None
