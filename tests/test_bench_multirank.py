"""bench.py's multi-GPU logic on CPU ranks (gloo, world size 2): every rank runs
an independent replica (its own seeds), the timed region is the slowest
rank's, and the reported value is all ranks' circuits over that time."""
import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, q):
    sys.path.insert(0, ROOT)
    import torch.distributed as dist

    import bench
    from paper_1809_11134_gb300 import workloads as W
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        searches = bench.replica_searches(W, 2, 512, rank)
        n = sum(s.P for s in searches)
        local_ms = 10.0 + 5.0 * rank
        total = bench.max_over_ranks(local_ms, ws, "cpu")
        q.put((rank, [s.seed for s in searches], n, total,
               bench.whole_job_rate(n, 7, ws, total)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_time_and_count_all_circuits():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, seeds0, n0, t0, v0), (r1, seeds1, n1, t1, v1) = out
    assert (r0, r1) == (0, 1)
    assert t0 == t1 == 15.0                      # max over ranks
    assert n0 == n1 == 3 * 512
    assert v0 == v1 == pytest.approx(2 * 3 * 512 * 7 / 0.015)
    assert set(seeds0).isdisjoint(seeds1)        # independent replicas


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, 1, "cpu") == 3.5
    assert bench.whole_job_rate(100, 10, 1, 1000.0) == 1000.0
