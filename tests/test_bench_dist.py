"""The benchmark's multi-rank host logic on two gloo ranks (CPU): every rank integrates its
own frames (disjoint seeds, no exchange on the data path), the job time is the slowest
rank's, and the rate counts every rank's frames.  The reference arm prints on rank 0 only."""
import importlib.util
import io
import os
import socket
import sys
from contextlib import redirect_stdout

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    mod = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(mod)
    return mod


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        b = _bench()
        assert b.dist_env() == (rank, world, rank)
        ms = b.max_over_ranks(10.0 * (rank + 1), world)
        seeds = b.frame_seeds(rank)
        gathered = [None] * world
        dist.all_gather_object(gathered, seeds)
        rate = b.whole_job_rate(128, world, 5, ms)
        out.put((rank, ms, gathered, rate))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=10) for _ in range(world))
    for rank, ms, gathered, rate in res:
        assert ms == 20.0                       # the slowest rank's time on every rank
        assert not set(gathered[0]) & set(gathered[1])  # disjoint frames
        assert rate == pytest.approx(2 * 128 * 5 / 0.020)


def test_reference_arm_prints_on_rank_zero_only(monkeypatch):
    b = _bench()
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("WORLD_SIZE", "2")
    buf = io.StringIO()
    with redirect_stdout(buf):
        b.run_reference(b.parse(["--impl", "reference", "--gpus", "2"]))
    assert buf.getvalue() == ""
