"""qe_rank and the run-time check of the ranking's guard band.

A binary32 search's top-k is exact when every circuit's binary64 fitness lies in
the interval its binary32 fitness implies (|d32 - d64| <= eps_d, d = (1 - f)^2).
The rescoring checks that on every candidate it rescores; these tests feed
qe_rank binary32 fitness values that break it (a circuit's value raised beyond
the bound) and ones that keep it (real values, and a value moved by less than
the bound), against the oracle's ranking."""
import numpy as np
import pytest

import oracle
from gpu_common import eps_d, oracle_problem
from paper_1809_11134_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as G
    G.build()
    from paper_1809_11134_gb300 import qe
    assert torch.cuda.is_available()
    return qe, torch


def _setup(qe, torch, n=4, L=24, P=3000, seed=3, cost_weight=0.0):
    s = W.Search(n, L, P, W.LIB_NCV | W.LIB_HT, W.cknot(n), precision=W.PREC_FP32, topk=16,
                 cost_weight=cost_weight)
    G, _ = qe.qe_library_info(n, s.library)
    gates = W.random_gates(np.random.default_rng(seed), P, L, G)
    p = oracle_problem(s, 0)
    F64, cost = oracle.eval_circuits(p, gates)
    return s, gates, F64, cost


def _topk(F, cost, k):
    order = oracle.topk(F, cost, k)
    return [(int(c), int(cost[c]), float(F[c])) for c in order]


@pytest.mark.parametrize("cost_weight", [0.0, 0.05])
def test_rank_of_real_fitness_is_the_oracles_top_k(env, cost_weight):
    qe, torch = env
    s, gates, F64, cost = _setup(qe, torch, cost_weight=cost_weight)
    with qe.Context([s]) as ctx:
        g = torch.from_numpy(gates).cuda()
        fit = torch.zeros(s.P, dtype=torch.float32, device="cuda")
        c = torch.zeros(s.P, dtype=torch.int32, device="cuda")
        top_eval = ctx.eval(0, g, fit, cost=c, topk=True)
        top_rank = ctx.rank(0, g, fit, c)
        want = _topk(F64, cost, s.topk)
        assert top_rank == want
        assert top_eval == want
        assert np.array_equal(c.cpu().numpy().astype(np.uint32), cost)


def test_guard_band_violation_is_reported(env):
    qe, torch = env
    s, gates, F64, cost = _setup(qe, torch)
    e = eps_d(s.L)
    with qe.Context([s]) as ctx:
        g = torch.from_numpy(gates).cuda()
        fit = torch.zeros(s.P, dtype=torch.float32, device="cuda")
        c = torch.zeros(s.P, dtype=torch.int32, device="cuda")
        ctx.eval(0, g, fit, cost=c)
        f32 = fit.cpu().numpy()
        # a mediocre circuit given a binary32 fitness above the best: it becomes a
        # candidate, and its binary64 value is far outside its interval
        worst = int(np.argmin(F64))
        bad = f32.copy()
        bad[worst] = np.float32(F64.max() + 0.05)
        with pytest.raises(qe.QeError) as err:
            ctx.rank(0, g, torch.from_numpy(bad).cuda(), c)
        assert err.value.status == qe.QE_ENUMERIC and "guard band" in str(err.value)
        # the best circuit raised by 2.5 eps_d in d: still the best, outside the bound
        best = int(np.argmax(F64))
        d64 = (1.0 - F64[best]) ** 2
        assert d64 > 4 * e
        out = f32.copy()
        out[best] = np.float32(1.0 - np.sqrt(d64 - 2.5 * e))
        with pytest.raises(qe.QeError) as err:
            ctx.rank(0, g, torch.from_numpy(out).cuda(), c)
        assert "guard band" in str(err.value)
        # ... moved by half the bound: inside, no report, and the ranking still exact
        ok = f32.copy()
        ok[best] = np.float32(1.0 - np.sqrt(d64 - 0.5 * e))
        assert ctx.rank(0, g, torch.from_numpy(ok).cuda(), c) == _topk(F64, cost, s.topk)
        # the error word was cleared by the report: real values rank cleanly again
        assert ctx.rank(0, g, fit, c) == _topk(F64, cost, s.topk)


def test_real_generations_keep_the_guard_band(env):
    """Binary32 searches at every width: generations report no guard-band error
    (every rescored candidate's binary64 fitness inside its interval)."""
    qe, torch = env
    searches = [W.Search(n, L, 2048, W.LIB_NCV | W.LIB_HT | W.LIB_IDENTITY, W.cknot(n), seed=n,
                         precision=W.PREC_FP32, topk=64) for n, L in ((3, 16), (4, 32), (5, 64))]
    with qe.Context(searches) as ctx:
        for _ in range(4):
            reps = ctx.step(5)
            for r in reps:
                assert r["error_word"] == 0
