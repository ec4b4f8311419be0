"""The benchmark's multi-rank logic on CPU ranks (gloo, world size 2): each
rank runs an independent replica, the job's step time is the slowest rank's
(max over ranks), the whole-job value counts every rank's units, and the
reference arm runs on rank 0 only."""
import importlib.util
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        w, r, _ = b.dist_env()
        ms = 10.0 + 5.0 * r                       # rank 1 is the slower one
        m = b.max_over_ranks(ms, w, "cpu")
        out[r] = (w, r, m, b.job_throughput(1000.0, w, m))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_job_value_on_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    with ctx.Manager() as mgr:
        out = mgr.dict()
        mp.start_processes(_worker, args=(world, port, out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert sorted(res) == [0, 1]
    for r in (0, 1):
        w, rr, m, v = res[r]
        assert w == 2 and rr == r
        assert m == 15.0                          # every rank sees the slowest rank's time
        assert v == pytest.approx(2 * 1000.0 / 15e-3)


def test_single_rank_helpers_need_no_process_group():
    b = _bench()
    assert b.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert b.job_throughput(100.0, 1, 2.0) == pytest.approx(50_000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch, capsys):
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    args = type("A", (), {"warmup": 0, "steps": 1, "gpus": 2, "workload": "rbf6"})()
    assert b.run_reference(args, b.WORKLOADS["rbf6"]) == 0
    assert capsys.readouterr().out == ""
