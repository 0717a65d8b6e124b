"""The N > 1 path of bench.py on the CPU: two gloo ranks.

Independent right-hand sides are the units the ranks share out (no data-path
collective); the only collectives are the barrier and the max-over-ranks of the
timings.  Each rank computes its incident directions and reduces a rank-dependent
time; the test checks the directions are disjoint between ranks and together are
the first ones on the circle, and that every rank sees the slowest rank's time.
"""
import math
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, steps, batch, q):
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        base = 0.25
        dirs = [bench.direction(base, k, rank, world) for k in range(steps * batch)]
        dist.barrier()
        ms = bench.max_over_ranks(100.0 + 7.0 * rank, world, "cpu")
        q.put((rank, dirs, ms, bench.job_seconds_per_rhs(ms, steps, batch, world)))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_directions_and_reduce_the_slowest_time():
    world, steps, batch = 2, 2, 8
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, world, port, steps, batch, q)) for r in range(world)]
    for p in procs:
        p.start()
    out = [q.get(timeout=120) for _ in range(world)]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    out.sort()
    d0, d1 = set(out[0][1]), set(out[1][1])
    assert len(d0) == len(d1) == steps * batch
    assert not d0 & d1
    expected = {0.25 + 2 * math.pi * i / 64 for i in range(world * steps * batch)}
    assert {round(x, 12) for x in d0 | d1} == {round(x, 12) for x in expected}
    assert out[0][2] == out[1][2] == 107.0
    assert out[0][3] == pytest.approx(107.0 / 1e3 / (steps * batch * world))


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.direction(0.0, 5, 0, 1) == pytest.approx(2 * math.pi * 5 / 64)
