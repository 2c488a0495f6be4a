"""The benchmark's multi-rank host logic on CPU with the gloo backend at world size 2 (replicas only: the ranks
share nothing but the timing reduction): the barrier, the max-over-ranks step time, the whole-job rate, and the
reference arm leaving every rank but 0 without work."""
import importlib.util
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_under_test", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    b = _bench()
    r, w, local = b.dist_init(world, backend="gloo")
    b.barrier(w)
    t = b.max_over_ranks(10.0 + 5.0 * r, w)          # rank 1 is the slower one
    rate = b.whole_job_rate(32, w, t / 1e3)

    class A:
        steps, warmup = 1, 0

    ref = b.run_reference(A, r, w) if r != 0 else "skipped"
    q.put((r, w, t, rate, ref))
    b.barrier(w)
    dist.destroy_process_group()


def test_two_gloo_ranks():
    world = 2
    port = _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r, (rank, w, t, rate, ref) in enumerate(out):
        assert rank == r and w == world
        assert t == 15.0                               # the max over ranks, on every rank
        assert rate == pytest.approx(32 * 2 / 0.015)   # units of all ranks over the slowest rank's time
    assert out[1][4] is None                           # rank 1 did no reference work


def test_single_rank_needs_no_process_group(monkeypatch):
    b = _bench()
    monkeypatch.delenv("WORLD_SIZE", raising=False)
    monkeypatch.delenv("RANK", raising=False)
    assert b.dist_init(1) == (0, 1, 0)
    assert b.max_over_ranks(3.5, 1) == 3.5
    b.barrier(1)
