"""The bench's multi-rank path on the CPU: two gloo ranks (world size 2).

Every rank runs its own replica (the path does not shard); the timed total
is the slowest rank's, and the value counts every rank's right-hand sides.
The reference arm does its work on rank 0 only; the other ranks leave
without work."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, q):
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    try:
        mine = [2.0, 3.5][rank]            # each rank's own timed seconds
        slowest = bench.max_over_ranks(mine, world, dist, torch.device("cpu"))
        dist.barrier()
        q.put((rank, slowest, bench.whole_job_rate(16 * 10, world, slowest)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, slowest, rate in got:
        assert slowest == 3.5
        assert rate == pytest.approx(16 * 10 * 2 / 3.5)


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1.25, 1) == 1.25
    assert bench.whole_job_rate(160, 1, 2.0) == 80.0


def test_reference_arm_other_ranks_do_no_work(monkeypatch, capsys):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("RANK", "1")
    called = []
    monkeypatch.setattr(bench, "run_oracle", lambda *a, **k: called.append(1))

    class A:
        gpus, steps, warmup = 2, 3, 1
    assert bench.reference_arm(A()) == 0
    assert not called and capsys.readouterr().out == ""
