"""The ranking's selection at both of its sizes: one CTA per search below
16384 circuits, a thread-block cluster of CTAs per search from 16384 up (the
population split into eight slices whose histograms are combined through
distributed shared memory).  Exact top-k (indices, costs, binary64 fitness)
against the CPU oracle on each side of the switch, with a ragged population,
many exact ties (a short circuit length: few distinct unitaries), NaN fitness
from invalid gate indices, and several searches of different sizes in one
batched call."""
import numpy as np
import pytest

import oracle
from gpu_common import oracle_problem
from paper_1809_11134_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NCV, HT, ID = W.LIB_NCV, W.LIB_HT, W.LIB_IDENTITY


@pytest.fixture(scope="module")
def qe():
    import __graft_entry__ as G
    G.build()
    from paper_1809_11134_gb300 import qe as Q
    return Q


def _expected(s, g):
    F, C = oracle.eval_circuits(oracle_problem(s, 0), g)
    k = min(max(s.topk, 1), len(g))
    order = oracle.topk(F, C, k)
    return F, [(int(c), int(C[c]), float(F[c])) for c in order]


def _check_top(top, want):
    assert [t[0] for t in top] == [w[0] for w in want]
    assert [t[1] for t in top] == [w[1] for w in want]
    for t, w in zip(top, want):
        assert (np.isnan(t[2]) and np.isnan(w[2])) or t[2] == w[2]


@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
@pytest.mark.parametrize("n", [16383, 16384, 20001])
def test_topk_on_both_sides_of_the_cluster_switch(qe, prec, n):
    rng = np.random.default_rng(n + 7 * prec)
    s = W.Search(3, 4, n, NCV | HT | ID, W.cknot(3), seed=3, precision=prec, topk=40)
    G = oracle.num_gates(s.n, s.library)
    g = W.random_gates(rng, n, s.L, G)
    g[rng.integers(0, n, size=25), 1] = 200  # invalid: NaN fitness, ranked last
    with qe.Context([s]) as ctx:
        with pytest.raises(qe.QeError) as e:
            ctx.eval_host(0, g, topk=True)
        assert e.value.status == qe.QE_ENUMERIC
        g[g >= G] = 0
        fit, top = ctx.eval_host(0, g, topk=True)
    F, want = _expected(s, g)
    if prec == W.PREC_FP64:
        assert np.array_equal(fit, F)
    _check_top(top, want)
    # L = 4 over a 28-gate library: many circuits share a fitness value
    assert len(np.unique(F)) < n // 4


@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
def test_batch_mixing_small_and_large_searches(qe, prec):
    """one batched call whose largest search takes the cluster selection: the
    small searches run on it too"""
    rng = np.random.default_rng(91 + prec)
    ss = [W.Search(3, 16, 24000, NCV | HT | ID, W.cknot(3), seed=1, precision=prec, topk=32),
          W.Search(4, 10, 500, NCV | HT, W.cknot(4), seed=2, precision=prec, topk=8),
          W.Search(2, 6, 37, NCV | ID, [0, 1, 3, 2], seed=3, precision=prec, topk=5)]
    plan = [(1, 500), (0, 24000), (2, 37)]
    items = [(q, W.random_gates(rng, n, ss[q].L, oracle.num_gates(ss[q].n, ss[q].library)))
             for q, n in plan]
    with qe.Context(ss) as ctx:
        fits, tops = ctx.eval_host_batch(items, topk=True)
    for (q, g), f, t in zip(items, fits, tops):
        F, want = _expected(ss[q], g)
        if prec == W.PREC_FP64:
            assert np.array_equal(f, F)
        _check_top(t, want)


@pytest.mark.parametrize("n", [3, 4, 5])
@pytest.mark.parametrize("form", ["trace", "prob", "dense"])
def test_split_rescoring_every_width_and_score(qe, n, form):
    """the binary64 rescoring splits a candidate's columns over 2 (n = 3) or 4
    (n = 4, 5) warps, each score form folding its column terms in the oracle's
    order: binary32 evaluation, top-k exact against the oracle"""
    from test_gpu_dense import near_target
    rng = np.random.default_rng(17 * n + len(form))
    lib = NCV | HT
    L = {3: 16, 4: 24, 5: 32}[n]
    kw = {}
    if form == "prob":
        kw["fitness_kind"] = W.FIT_PROB
    if form == "dense":
        kw["target"] = near_target(rng, n, lib, 8)
    s = W.Search(n, L, 600, lib, W.cknot(n), seed=n, precision=W.PREC_FP32, topk=24, **kw)
    g = W.random_gates(rng, 600, L, oracle.num_gates(n, lib))
    with qe.Context([s]) as ctx:
        fit, top = ctx.eval_host(0, g, topk=True)
    F, want = _expected(s, g)
    _check_top(top, want)
