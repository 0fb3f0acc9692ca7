"""The classical GA (Sec. V-B comparison) on the GPU against the oracle.

The GA shares the circuit evaluation with QEQEA; its breeding (stochastic
universal sampling, one-point crossover, per-gene mutation, elitism) is integer
work and must match oracle.ga_next bit for bit given the same fitness.  In
binary64 whole trajectories are bit-exact; in binary32 each generation's
genome is bit-exact given the GPU's own working-precision fitness."""
import numpy as np
import pytest

import oracle
from gpu_common import assert_fp32_fitness, oracle_problem
from paper_1809_11134_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NCV, HT, ID = W.LIB_NCV, W.LIB_HT, W.LIB_IDENTITY


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


def GA(n, L, P, lib, perm=None, **kw):
    return W.Search(n, L, P, lib, perm if perm is not None else W.cknot(n),
                    encoding=W.ENC_GA, **kw)


def _G(s):
    return oracle.num_gates(s.n, s.library)


def _oracle_ga_run(searches, gens, runs=None):
    """Per search: [(genome, F, cost, topk, best_fitness, best_cost, best_gates)] per generation."""
    out = []
    for i, s in enumerate(searches):
        run = runs[i] if runs else i
        p = oracle_problem(s, run)
        genome = oracle.ga_init(p, _G(s))
        hist = []
        bfit, bcost, bgates = -np.inf, 2**32 - 1, None
        for gen in range(gens):
            F, C = oracle.eval_circuits(p, genome)
            tk = oracle.topk(F, C, max(s.topk, 1))
            b = tk[0]
            if F[b] > bfit or (F[b] == bfit and C[b] < bcost):
                bfit, bcost, bgates = F[b], int(C[b]), bytes(genome[b])
            hist.append((genome.copy(), F, C, tk, bfit, bcost, bgates))
            genome = oracle.ga_next(p, _G(s), gen, s.ga_mutation_rate, genome, F, C)
        out.append((hist, genome))
    return out


@pytest.mark.parametrize("shape", [
    GA(3, 5, 64, NCV | ID, seed=0, precision=W.PREC_FP64),
    GA(4, 32, 301, NCV | HT, seed=3),
    GA(5, 64, 77, NCV | HT, seed=5),
    GA(1, 1, 1, HT, perm=[1, 0], seed=9),
])
def test_ga_init_bit_exact(qe, torch, shape):
    with qe.Context([shape]) as ctx:
        g = ctx.get_state(0)
    assert np.array_equal(g, oracle.ga_init(oracle_problem(shape, 0), _G(shape)))


@pytest.mark.parametrize("searches,gens", [
    ([GA(3, 5, 64, NCV | ID, seed=0, precision=W.PREC_FP64)], 25),
    (W.config(2, precision=W.PREC_FP64, P=256, encoding=W.ENC_GA), 10),
    ([GA(4, 12, 129, NCV | HT, seed=4, precision=W.PREC_FP64, topk=5, ga_mutation_rate=0.1,
         cost_weight=0.05)], 8),
])
def test_ga_trajectory_fp64_bit_exact(qe, torch, searches, gens):
    ref = _oracle_ga_run(searches, gens)
    with qe.Context(searches) as ctx:
        for gen in range(gens):
            for run in range(len(searches)):
                assert np.array_equal(ctx.get_state(run), ref[run][0][gen][0]), (gen, run)
            reps = ctx.step(1)
            for run, s in enumerate(searches):
                genome, F, C, tk, bfit, bcost, bgates = ref[run][0][gen]
                last = ctx.last_generation(run)
                assert np.array_equal(last["gate_idx"], genome)
                assert np.array_equal(last["fitness"], F)
                k = max(s.topk, 1)
                assert [t[0] for t in last["topk"][:k]] == list(tk[:k])
                r = reps[run]
                assert r["generation"] == gen + 1
                assert r["best_fitness"] == bfit and r["best_cost"] == bcost
                assert bytes(r["best_gates"]) == bgates[:s.L]
        for run in range(len(searches)):
            assert np.array_equal(ctx.get_state(run), ref[run][1])


def test_ga_pipelined_generations_fp64(qe, torch):
    """Generations enqueued without reports give the same genome and record."""
    searches = W.config(2, precision=W.PREC_FP64, P=150, encoding=W.ENC_GA)
    ref = _oracle_ga_run(searches, 7)
    with qe.Context(searches) as ctx:
        ctx.step_raw(4, None)
        ctx.step_raw(2, None)
        reps = ctx.step(1)
        for run, s in enumerate(searches):
            genome, F, C, tk, bfit, bcost, bgates = ref[run][0][6]
            last = ctx.last_generation(run)
            assert np.array_equal(last["gate_idx"], genome) and np.array_equal(last["fitness"], F)
            assert reps[run]["best_fitness"] == bfit and reps[run]["best_cost"] == bcost
            assert np.array_equal(ctx.get_state(run), ref[run][1])


def test_ga_fp32_each_generation(qe, torch):
    """binary32 GA: fitness within its bound; the next genome bit-exact given
    the GPU's own binary32 fitness (the elite and the SUS weights are taken in
    the working precision on both sides)."""
    searches = [GA(3, 16, 1000, NCV | HT | ID, seed=1, topk=8),
                GA(4, 32, 257, NCV | HT, seed=3, topk=4),
                GA(5, 64, 63, NCV | HT, seed=5, topk=3),
                GA(5, 20, 2, NCV | HT | ID, seed=6, ga_mutation_rate=0.5),
                GA(2, 1, 5, NCV, perm=[0, 1, 3, 2], seed=7, ga_mutation_rate=1.0)]
    probs = [oracle_problem(s, r) for r, s in enumerate(searches)]
    with qe.Context(searches) as ctx:
        for gen in range(5):
            genomes = [ctx.get_state(r) for r in range(len(searches))]
            ctx.step(1)
            for run, s in enumerate(searches):
                p = probs[run]
                last = ctx.last_generation(run)
                assert np.array_equal(last["gate_idx"], genomes[run])
                F, C = oracle.eval_circuits(p, genomes[run])
                assert_fp32_fitness(last["fitness"], F, s, C)
                order = oracle.topk(F, C, max(s.topk, 1))
                assert [t[0] for t in last["topk"]][:len(order)] == list(order)
                nxt = oracle.ga_next(p, _G(s), gen, s.ga_mutation_rate, genomes[run],
                                     last["fitness"], C)
                assert np.array_equal(ctx.get_state(run), nxt), (gen, run)


def test_ga_and_qeqea_share_a_context(qe, torch):
    """QEQEA and GA searches of the same widths share the circuit launches; each
    follows its own oracle trajectory bit for bit (binary64)."""
    q = W.config(2, precision=W.PREC_FP64, P=128)[:2]
    g = W.config(2, precision=W.PREC_FP64, P=96, encoding=W.ENC_GA)[:2]
    searches = [q[0], g[0], q[1], g[1]]
    gens = 6
    ga_ref = _oracle_ga_run([g[0], g[1]], gens, runs=[1, 3])
    qe_probs = {0: oracle_problem(q[0], 0), 2: oracle_problem(q[1], 2)}
    qe_state = {r: [a.copy() for a in oracle.init_state(p)] for r, p in qe_probs.items()}
    with qe.Context(searches) as ctx:
        for gen in range(gens):
            ctx.step(1)
            for r, p in qe_probs.items():
                cur, best, bf = qe_state[r]
                gi, sid = oracle.sample(p, cur, gen)
                F, C = oracle.eval_circuits(p, gi)
                last = ctx.last_generation(r)
                assert np.array_equal(last["gate_idx"], gi) and np.array_equal(last["fitness"], F)
                oracle.update(p, cur, best, bf, gen, sid, F.astype(np.float64))
            for k, r in enumerate([1, 3]):
                last = ctx.last_generation(r)
                assert np.array_equal(last["gate_idx"], ga_ref[k][0][gen][0])
                assert np.array_equal(last["fitness"], ga_ref[k][0][gen][1])
        for k, r in enumerate([1, 3]):
            assert np.array_equal(ctx.get_state(r), ga_ref[k][1])


def test_ga_set_state_round_trip_and_validation(qe, torch):
    s = GA(3, 9, 40, NCV | HT | ID, seed=2, precision=W.PREC_FP64)
    p = oracle_problem(s, 0)
    G = _G(s)
    rng = np.random.default_rng(5)
    mine = rng.integers(0, G, (s.P, s.L)).astype(np.uint8)
    with qe.Context([s]) as ctx:
        ctx.step(2)
        ctx.set_state(0, mine)
        assert np.array_equal(ctx.get_state(0), mine)
        ctx.step(1)
        last = ctx.last_generation(0)
        F, C = oracle.eval_circuits(p, mine)
        assert np.array_equal(last["gate_idx"], mine) and np.array_equal(last["fitness"], F)
        assert np.array_equal(ctx.get_state(0), oracle.ga_next(p, G, 2, s.ga_mutation_rate,
                                                               mine, F, C))
        bad = mine.copy()
        bad[3, 4] = G
        with pytest.raises(qe.QeError):
            ctx.set_state(0, bad)
        assert not np.array_equal(ctx.get_state(0), bad)
