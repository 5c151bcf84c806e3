"""The multi-rank bench path on CPU (gloo, world size 2): replicas only, no
data-path collective. Each rank times its own replica; the job's time is the
slowest rank's and every rank learns it; the reference arm runs on rank 0
alone (the others exit without work)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    sys.path.insert(0, ROOT)
    import bench

    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    try:
        seconds = 1.0 + 0.5 * rank  # rank 1 is the slow one
        out[rank] = bench.max_over_ranks(dist, seconds, "cpu")
    finally:
        dist.destroy_process_group()


def test_job_time_is_the_slowest_ranks_on_every_rank():
    world = 2
    out = mp.Manager().dict()
    mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
    assert dict(out) == {0: 1.5, 1: 1.5}


def test_single_rank_time_is_its_own():
    sys.path.insert(0, ROOT)
    import bench

    assert bench.max_over_ranks(None, 0.25, "cpu") == 0.25


def test_reference_arm_runs_on_rank_0_only(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "1")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--gpus", "2"])
    assert bench.main() == 0
    assert capsys.readouterr().out == ""
