"""The launch-plan autotuner changes how a generation graph is launched, never
what it computes: a tuned context follows the untuned trajectory bit for bit,
and binary64 trajectories stay equal to the oracle's."""
import numpy as np
import pytest

from gpu_common import state_equal
from paper_1809_11134_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def qe():
    import __graft_entry__ as G
    G.build()
    from paper_1809_11134_gb300 import qe as Q
    return Q


@pytest.fixture(scope="module")
def torch():
    import torch as T
    assert T.cuda.is_available()
    return T


def _run(qe, searches, tune, gens_after):
    with qe.Context(searches) as ctx:
        ms = ctx.autotune(1) if tune else []
        done = ctx.generation()
        reps = ctx.step(gens_after)
        states = [ctx.get_state(r) for r in range(len(searches))]
        lasts = [ctx.last_generation(r) for r in range(len(searches))]
        return ms, done, reps, states, lasts, ctx.launch_plan()


@pytest.mark.parametrize("searches", [
    W.config(2, P=700),
    W.config(2, precision=W.PREC_FP64, P=200)
    + W.config(2, precision=W.PREC_FP64, P=90, encoding=W.ENC_GA)[:1],
    [W.Search(5, 20, 150, W.LIB_NCV | W.LIB_HT, W.cknot(5), seed=3, topk=7),
     W.Search(4, 9, 333, W.LIB_NCV | W.LIB_HT, W.cknot(4), seed=4, topk=5),
     W.Search(3, 30, 64, W.LIB_NCV | W.LIB_HT | W.LIB_IDENTITY, W.cknot(3), seed=5,
              encoding=W.ENC_GA)],
])
def test_autotuned_trajectory_is_unchanged(qe, torch, searches):
    ms, done, reps_t, st_t, last_t, plan = _run(qe, searches, True, 3)
    assert len(ms) >= 4 and all(m > 0 for m in ms)
    assert "autotuned" in plan
    assert done == len(ms) * 2  # one settling and one timed generation per plan
    _, done0, reps_u, st_u, last_u, plan0 = _run(qe, searches, False, done + 3)
    assert done0 == 0 and "default" in plan0
    for r, s in enumerate(searches):
        assert reps_t[r]["generation"] == reps_u[r]["generation"] == done + 3
        for key in ("best_fitness", "best_cost", "best_gates", "useful_flops", "mean_fitness"):
            assert reps_t[r][key] == reps_u[r][key], key
        assert np.array_equal(last_t[r]["gate_idx"], last_u[r]["gate_idx"])
        assert np.array_equal(last_t[r]["fitness"], last_u[r]["fitness"])
        assert last_t[r]["topk"] == last_u[r]["topk"]
        if s.encoding == W.ENC_GA:
            assert np.array_equal(st_t[r], st_u[r])
        else:
            assert all(state_equal(a, b) for a, b in zip(st_t[r], st_u[r]))


def test_autotune_needs_stage_timing_off(qe, torch):
    with qe.Context(W.config(1)) as ctx:
        ctx.stage_timing(True)
        with pytest.raises(qe.QeError):
            ctx.autotune(1)
        ctx.stage_timing(False)
        assert len(ctx.autotune(1)) >= 4
        with pytest.raises(qe.QeError):
            ctx.autotune(0)


@pytest.mark.parametrize("mode", [1, 2])
def test_stage_timing_leaves_the_trajectory_unchanged(qe, torch, mode):
    """stage timing (events inside the graph, mode 1; every kernel serialised on
    one stream, mode 2) changes only when the kernels run: the run follows the
    untimed trajectory bit for bit, and every stage interval is positive"""
    T = np.eye(8, dtype=np.complex128)[[1, 0, 2, 3, 4, 5, 7, 6]]  # a dense target
    searches = (W.config(2, P=300)
                + [W.Search(4, 9, 333, W.LIB_NCV | W.LIB_HT, W.cknot(4), seed=4, topk=5),
                   W.Search(3, 30, 64, W.LIB_NCV | W.LIB_HT | W.LIB_IDENTITY, W.cknot(3),
                            seed=5, encoding=W.ENC_GA),
                   W.Search(3, 10, 128, W.LIB_NCV | W.LIB_HT, W.cknot(3), seed=6, topk=4,
                            shots=6),
                   W.Search(3, 11, 96, W.LIB_NCV | W.LIB_HT, W.cknot(3), seed=7, topk=3,
                            target=T)])
    gens = 4
    with qe.Context(searches) as a, qe.Context(searches) as b:
        a.stage_timing(True, serial=(mode == 2))
        for _ in range(gens):
            a.step_raw(1, None)
            ms = a.stage_times()
            assert all(m > 0 for m in ms), ms
            assert ms[0] <= ms[5] and ms[4] <= ms[5]
        ra, rb = a.step(1), b.step(gens + 1)
        a.stage_timing(False)
        assert ra == rb
        for r, s in enumerate(searches):
            la, lb = a.last_generation(r), b.last_generation(r)
            assert np.array_equal(la["gate_idx"], lb["gate_idx"])
            assert np.array_equal(la["fitness"], lb["fitness"])
            assert la["topk"] == lb["topk"]
            sa, sb = a.get_state(r), b.get_state(r)
            if s.encoding == W.ENC_GA:
                assert np.array_equal(sa, sb)
            else:
                assert all(state_equal(x, y) for x, y in zip(sa, sb))
        with pytest.raises(qe.QeError):
            qe._check(a.h, qe.lib().qe_stage_timing(a.h, 3))
