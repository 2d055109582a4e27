"""The multi-rank path of bench.py on CPU: two gloo ranks (replicas).

Views are independent, so ranks shard the trajectory with no data exchange;
the only collective is the max over ranks of the timed region."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        sched = [bench.view_schedule(rank, step, 8, 16) for step in range(4)]
        slowest = bench.max_over_ranks(1.0 + 0.5 * rank, "cpu")
        value = bench.aggregate_views_per_s(4, 8, world, slowest)
        q.put((rank, sched, slowest, value))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_shard_views_and_take_the_max_time():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = {}
    for _ in procs:
        r, sched, slowest, value = q.get(timeout=120)
        res[r] = (sched, slowest, value)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # both ranks agree on the slowest time and on the whole-job throughput
    assert res[0][1] == res[1][1] == 1.5
    assert res[0][2] == res[1][2] == pytest.approx(4 * 8 * 2 / 1.5)
    # within every step the two replicas render different views
    for step in range(4):
        v0 = {v for v, _ in res[0][0][step]}
        v1 = {v for v, _ in res[1][0][step]}
        assert not (v0 & v1)
        # each view of a step reads its own frame tick
        assert len({t for _, t in res[0][0][step]}) == 8


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(2.5, "cpu") == 2.5
    assert bench.view_schedule(0, 1, 4, 16) == [(4, 4), (5, 5), (6, 6), (7, 7)]
