"""The multi-rank path of bench.py on CPU: two gloo ranks on 127.0.0.1.

Each rank runs its own replica (seeds shifted by the rank), the timed region
is the slowest rank's, and the whole-job rate counts every rank's atoms; the
reference arm runs on rank 0 only."""
import json
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = 10.0 + 5.0 * rank                   # rank 1 is the slow one
        got = bench.max_over_ranks(ms, world, torch.device("cpu"))
        p, r, v, s, _ = bench.build_workload("fe_bcc_10x10x10_nve", rank)
        q.put((rank, got, bench.whole_job_rate(p["n_atoms"], world, 7, got * 1e-3), float(r[0, 0]),
               p["n_atoms"]))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_reduce_and_count():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(k, 2, port, q)) for k in range(2)]
    for pr in procs:
        pr.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    (r0, m0, v0, x0, n0), (r1, m1, v1, x1, n1) = res
    assert m0 == m1 == 15.0                      # both ranks see the slowest time
    assert v0 == v1 == pytest.approx(2 * n0 * 7 / 15e-3)
    assert n0 == n1 and x0 != x1                 # same size, different seeds


def test_reference_arm_runs_on_rank_zero_only(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    args = type("A", (), dict(steps=1, warmup=0, gpus=2, workload="fe_bcc_64x64x64_nve", full_workload=False))()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    bench.run_reference(args)
    assert capsys.readouterr().out == ""
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setattr(bench, "SAMPLE_CELLS", 6)
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_reference_arm_full_workload(capsys, monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "0")
    monkeypatch.setenv("WORLD_SIZE", "1")
    args = type("A", (), dict(steps=2, warmup=1, gpus=1, workload="fe_bcc_10x10x10_nve", full_workload=True))()
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["config"]["sample_atoms"] == 2000 and line["value"] > 0
    assert "whole workload" in line["cpu_baseline"]["sample"]
    args.workload = "fe_bcc_batch256"
    bench.run_reference(args)
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference" and "unavailable" in line
