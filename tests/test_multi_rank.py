"""The N > 1 path of the benchmark on CPU ranks (gloo, world size 2).

The hot path runs as independent replicas, one per GPU, with no data-path
collective; what N > 1 adds is host logic: each rank times its own replica,
the job's time is the maximum over ranks and the reported value counts the
units of every rank over that time; the reference arm runs on rank 0 only.
"""
import io
import contextlib
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
        # rank r measured (push ms, step ms) = (1 + r, 5 - r)
        ms = bench.max_over_ranks([1.0 + rank, 5.0 - rank], dist, "cpu")
        rate = bench.whole_job_rate(world, 1000, ms[0])
        out[rank] = (ms, rate)
    finally:
        dist.destroy_process_group()


def test_max_over_ranks_and_whole_job_rate():
    world, port = 2, _free_port()
    with mp.Manager() as man:
        out = man.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    for rank in range(world):
        ms, rate = res[rank]
        assert ms == [2.0, 5.0]                     # element-wise maximum over the two ranks
        assert rate == pytest.approx(2 * 1000 / 2e-3)


def test_single_rank_needs_no_process_group():
    assert bench.max_over_ranks([3.0, 4.0], None, "cpu") == [3.0, 4.0]
    assert bench.whole_job_rate(1, 500, 250.0) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only(monkeypatch):
    class Args:
        workload, steps, warmup, gpus = "harris", 1, 0, 2
    monkeypatch.setenv("RANK", "1")
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        assert bench.run_reference(Args()) == 0
    assert buf.getvalue() == ""
