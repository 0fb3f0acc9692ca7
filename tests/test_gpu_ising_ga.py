"""The paper's GA comparator on the Ising library (Sec. V-B) on the GPU against
the oracle: genes are (gate, angle) pairs, angles start on the 2 pi / Q lattice,
crossover takes two points, a gene not drawn fresh may have its angle turned by
a multiple of range / Q, and the elite keeps its angles.  Breeding is integer
work plus one binary32 rotation in a fixed order, so the next genome and its
angles are bit-exact given the same fitness; binary64 trajectories are
bit-exact end to end."""
import numpy as np
import pytest

import oracle
from gpu_common import assert_fp32_fitness, oracle_problem
from paper_1809_11134_gb300 import workloads as W

pytestmark = pytest.mark.gpu

ISING = W.LIB_ISING


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


def GA(n, L, P, perm=None, **kw):
    return W.Search(n, L, P, ISING, perm if perm is not None else W.cknot(n),
                    encoding=W.ENC_GA, **kw)


def _G(s):
    return oracle.num_gates(s.n, s.library)


def _oracle_run(searches, gens):
    """Per search: [(genome, angles, F, cost, topk, best_fitness, best_cost, best_gates,
    best_angles)] per generation, and the final (genome, angles)."""
    out = []
    for run, s in enumerate(searches):
        p = oracle_problem(s, run)
        genome, amps = oracle.ga_init_amp(p, _G(s))
        hist = []
        bfit, bcost, bgates, bamps = -np.inf, 2**32 - 1, None, None
        for gen in range(gens):
            F, C = oracle.eval_circuits(p, genome, amps)
            tk = oracle.topk(F, C, max(s.topk, 1))
            b = tk[0]
            if F[b] > bfit or (F[b] == bfit and C[b] < bcost):
                bfit, bcost = F[b], int(C[b])
                bgates, bamps = bytes(genome[b]), amps[b].ravel().tolist()
            hist.append((genome.copy(), amps.copy(), F, C, tk, bfit, bcost, bgates, bamps))
            genome, amps = oracle.ga_next_amp(p, _G(s), gen, s.ga_mutation_rate, genome, amps,
                                              F, C)
        out.append((hist, genome, amps))
    return out


@pytest.mark.parametrize("shape", [
    GA(2, 3, 64, seed=1, precision=W.PREC_FP64),
    GA(3, 16, 301, seed=2),
    GA(5, 64, 33, seed=5),
    GA(1, 1, 1, perm=[1, 0], seed=9),
])
def test_init_bit_exact(qe, torch, shape):
    with qe.Context([shape]) as ctx:
        g, a = ctx.get_state(0)
    eg, ea = oracle.ga_init_amp(oracle_problem(shape, 0), _G(shape))
    assert np.array_equal(g, eg) and np.array_equal(a, ea)


@pytest.mark.parametrize("searches,gens", [
    ([GA(2, 3, 64, seed=1, precision=W.PREC_FP64, topk=4)], 20),
    ([GA(3, 16, 200, seed=2, precision=W.PREC_FP64, topk=8, ga_mutation_rate=0.1),
      GA(4, 12, 81, seed=3, precision=W.PREC_FP64, topk=3, cost_weight=0.05),
      GA(3, 10, 150, W.peres(), seed=4, precision=W.PREC_FP64, topk=5,
         fitness_kind=W.FIT_PROB, ga_mutation_rate=0.3)], 8),
])
def test_trajectory_fp64_bit_exact(qe, torch, searches, gens):
    ref = _oracle_run(searches, gens)
    with qe.Context(searches) as ctx:
        for gen in range(gens):
            for run in range(len(searches)):
                g, a = ctx.get_state(run)
                assert np.array_equal(g, ref[run][0][gen][0]), (gen, run)
                assert np.array_equal(a, ref[run][0][gen][1]), (gen, run)
            reps = ctx.step(1)
            for run, s in enumerate(searches):
                genome, amps, F, C, tk, bfit, bcost, bgates, bamps = ref[run][0][gen]
                last = ctx.last_generation(run)
                assert np.array_equal(last["gate_idx"], genome)
                assert np.array_equal(last["fitness"], F)
                k = max(s.topk, 1)
                assert [t[0] for t in last["topk"][:k]] == list(tk[:k])
                r = reps[run]
                assert r["best_fitness"] == bfit and r["best_cost"] == bcost
                assert bytes(r["best_gates"]) == bgates[:s.L]
                assert r["best_amps"] == bamps
        for run in range(len(searches)):
            g, a = ctx.get_state(run)
            assert np.array_equal(g, ref[run][1]) and np.array_equal(a, ref[run][2])


def test_fp32_each_generation(qe, torch):
    """binary32: fitness within its bound; the next genome and angles bit-exact
    given the GPU's own binary32 fitness.  High mutation rates exercise both the
    fresh-gene and the angle-turn branches."""
    searches = [GA(3, 16, 1000, seed=1, topk=8),
                GA(5, 40, 63, seed=5, topk=3, ga_mutation_rate=0.4),
                GA(2, 1, 5, perm=[0, 1, 3, 2], seed=7, ga_mutation_rate=1.0),
                GA(4, 33, 129, seed=8, ga_mutation_rate=0.7, mutation_range=np.pi)]
    probs = [oracle_problem(s, r) for r, s in enumerate(searches)]
    with qe.Context(searches) as ctx:
        for gen in range(5):
            states = [ctx.get_state(r) for r in range(len(searches))]
            ctx.step(1)
            for run, s in enumerate(searches):
                p = probs[run]
                g, a = states[run]
                last = ctx.last_generation(run)
                assert np.array_equal(last["gate_idx"], g)
                F, C = oracle.eval_circuits(p, g, a)
                assert_fp32_fitness(last["fitness"], F, s, C)
                ng, na = oracle.ga_next_amp(p, _G(s), gen, s.ga_mutation_rate, g, a,
                                            last["fitness"], C)
                g2, a2 = ctx.get_state(run)
                assert np.array_equal(g2, ng) and np.array_equal(a2, na), (gen, run)


def test_shares_a_context_with_qeqea_and_discrete_ga(qe, torch):
    """Ising GA, Ising QEQEA and a discrete GA in one context (binary64): each
    follows its own oracle trajectory bit for bit."""
    ga_i = GA(3, 12, 90, seed=3, precision=W.PREC_FP64)
    qe_i = W.Search(3, 12, 70, ISING, W.cknot(3), seed=4, precision=W.PREC_FP64)
    ga_d = W.Search(3, 12, 60, W.LIB_NCV | W.LIB_HT, W.cknot(3), seed=5,
                    precision=W.PREC_FP64, encoding=W.ENC_GA)
    searches = [ga_i, qe_i, ga_d]
    gens = 5
    ref_i = _oracle_run([ga_i], gens)[0]
    p_q = oracle_problem(qe_i, 1)
    cur, best, bf = [x.copy() for x in oracle.init_state(p_q)]
    p_d = oracle_problem(ga_d, 2)
    gd = oracle.ga_init(p_d, _G(ga_d))
    with qe.Context(searches) as ctx:
        for gen in range(gens):
            ctx.step(1)
            last = ctx.last_generation(0)
            assert np.array_equal(last["gate_idx"], ref_i[0][gen][0])
            assert np.array_equal(last["fitness"], ref_i[0][gen][2])
            gi, sid, amps = oracle.sample(p_q, cur, gen, with_amps=True)
            F, C = oracle.eval_circuits(p_q, gi, amps)
            last = ctx.last_generation(1)
            assert np.array_equal(last["gate_idx"], gi) and np.array_equal(last["fitness"], F)
            oracle.update(p_q, cur, best, bf, gen, sid, F)
            F, C = oracle.eval_circuits(p_d, gd)
            last = ctx.last_generation(2)
            assert np.array_equal(last["gate_idx"], gd) and np.array_equal(last["fitness"], F)
            gd = oracle.ga_next(p_d, _G(ga_d), gen, ga_d.ga_mutation_rate, gd, F, C)
        g, a = ctx.get_state(0)
        assert np.array_equal(g, ref_i[1]) and np.array_equal(a, ref_i[2])
        assert np.array_equal(ctx.get_state(2), gd)


def test_set_state_round_trip_and_validation(qe, torch):
    s = GA(3, 9, 40, seed=2, precision=W.PREC_FP64)
    p = oracle_problem(s, 0)
    G = _G(s)
    rng = np.random.default_rng(5)
    mine = rng.integers(0, G, (s.P, s.L)).astype(np.uint8)
    t = rng.uniform(0, 2 * np.pi, (s.P, s.L))
    ang = np.stack([np.cos(t), np.sin(t)], -1).astype(np.float32)
    with qe.Context([s]) as ctx:
        ctx.step(2)
        ctx.set_state(0, mine, ang)
        g, a = ctx.get_state(0)
        assert np.array_equal(g, mine) and np.array_equal(a, ang)
        ctx.step(1)
        last = ctx.last_generation(0)
        F, C = oracle.eval_circuits(p, mine, ang)
        assert np.array_equal(last["gate_idx"], mine) and np.array_equal(last["fitness"], F)
        ng, na = oracle.ga_next_amp(p, G, 2, s.ga_mutation_rate, mine, ang, F, C)
        g, a = ctx.get_state(0)
        assert np.array_equal(g, ng) and np.array_equal(a, na)
        bad = mine.copy()
        bad[3, 4] = G
        with pytest.raises(qe.QeError):
            ctx.set_state(0, bad, ang)
        assert not np.array_equal(ctx.get_state(0)[0], bad)
