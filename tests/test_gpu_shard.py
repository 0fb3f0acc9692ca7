"""One search sharded over ranks, on one GPU: two ranks emulated in one process
(two library contexts, each evaluating its shard; the gather is a host-side
concatenation between the phases, so no kernel waits on another rank's).
Binary64: every generation's fitness and top-k and the final state equal the
oracle's single-rank trajectory bit for bit.  Binary32: equal to the
unsharded generation driver (qe_step) on one context."""
import numpy as np
import pytest

import oracle
from gpu_common import oracle_problem, state_equal
from paper_1809_11134_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as G
    G.build()
    from paper_1809_11134_gb300 import qe, shard
    assert torch.cuda.is_available()
    return qe, shard, torch


def _run_sharded(qe, shard, torch, s, ws, gens, own_streams=False):
    # own_streams: every context on a stream of its own, not torch's current
    # one (the device wrapper orders the two)
    ctxs = [qe.Context([s], stream=torch.cuda.Stream() if own_streams
                       else torch.cuda.current_stream()) for _ in range(ws)]
    runs = [shard.ShardedSearch(shard.QeShardDevice(c), rank=r, world=ws)
            for r, c in enumerate(ctxs)]
    traj = []
    for g in range(gens):
        parts = [run.evaluate_shard(g) for run in runs]
        F = torch.cat([f for f, _ in parts])
        C = torch.cat([c for _, c in parts])
        res = [run.finish(g, F, C) for run in runs]
        for r in res[1:]:
            assert r.topk == res[0].topk
        traj.append((F.cpu().numpy(), res[0].topk))
    states = [c.get_state(0) for c in ctxs]
    for c in ctxs:
        c.close()
    return traj, states


@pytest.mark.parametrize("ws,own", [(2, False), (3, False), (2, True)])
def test_sharded_binary64_search_is_the_oracles_trajectory(env, ws, own):
    qe, shard, torch = env
    s = W.Search(3, 16, 1000, W.LIB_NCV | W.LIB_HT | W.LIB_IDENTITY, W.cknot(3), seed=5,
                 precision=W.PREC_FP64, topk=16)
    gens = 5
    traj, states = _run_sharded(qe, shard, torch, s, ws, gens, own_streams=own)
    p = oracle_problem(s, 0)
    cur, best, bf = oracle.init_state(p)
    rep = oracle.new_report()
    for g in range(gens):
        gi, sid, F, cost, tk = oracle.step(p, cur, best, bf, g, s.topk, rep)
        assert np.array_equal(traj[g][0], F), g
        assert traj[g][1] == [(int(c), int(cost[c]), float(F[c])) for c in tk], g
    for c2, b2, f2 in states:
        assert state_equal(c2, cur) and state_equal(b2, best) and state_equal(f2, bf)


def test_sharded_binary32_search_is_the_unsharded_one(env):
    qe, shard, torch = env
    s = W.Search(4, 24, 3000, W.LIB_NCV | W.LIB_HT, W.cknot(4), seed=9,
                 precision=W.PREC_FP32, topk=32)
    gens = 4
    traj, states = _run_sharded(qe, shard, torch, s, 2, gens)
    with qe.Context([s], stream=torch.cuda.current_stream()) as ctx:
        for g in range(gens):
            ctx.step(1)
            last = ctx.last_generation(0)
            assert np.array_equal(traj[g][0], last["fitness"]), g
            top = [(int(t[0]), int(t[1]), float(t[2])) for t in last["topk"]]
            assert traj[g][1] == top, g
        ref = ctx.get_state(0)
    for st in states:
        assert all(state_equal(a, b) for a, b in zip(st, ref))
