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


def test_reference_arm_prints_one_contract_line(monkeypatch, capsys):
    # the reference arm (the FP64 oracle on the host) keeps the bench's JSON
    # contract: one line, the same metric and unit, its own cpu_baseline and
    # e2e, impl "reference"
    import json

    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "tiny", "--steps", "3",
                                      "--warmup", "1"])
    assert bench.main() == 0
    lines = [l for l in capsys.readouterr().out.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["steps"] == 3 and d["value"] > 0 and d["higher_is_better"] is True
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"] == {"value": d["value"], "unit": d["unit"], "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}


def test_reference_arm_serving_reports_oracle_solves_per_second(monkeypatch, capsys):
    import json

    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "serving", "--requests", "2",
                                      "--max-iters", "100", "--cpu-seconds", "30"])
    assert bench.main() == 0
    d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["unit"] == "solves/s" and d["steps"] == 2 and d["value"] > 0
    assert d["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_warmstart_reports_oracle_cold_iterations(monkeypatch, capsys):
    import json

    sys.path.insert(0, ROOT)
    import bench

    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(sys, "argv", ["bench.py", "--impl", "reference", "--workload", "warmstart", "--heldout", "1",
                                      "--max-iters", "100", "--cpu-seconds", "30"])
    assert bench.main() == 0
    d = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert d["impl"] == "reference" and d["steps"] == 1 and 50 <= d["value"] <= 100
    assert d["higher_is_better"] is False and d["cpu_baseline"]["kind"] == "oracle"
