"""Benchmark workloads at their full sizes, through qe_step -- the generation
graph bench.py times -- against the oracle.

The 3-qubit workload (three searches of P = 4096) is checked completely, every
stage of every generation.  At the 4- and 5-qubit sizes (P = 65536 and 262144)
the oracle checks sampled outputs one by one: the generation-0 measurement in
full (4 qubits) or by its structure (5 qubits: the oracle's encoding state
would take 27 GB of host memory), binary32 fitness of a random subset of
circuits, the binary64 top-k values circuit by circuit, and the top-k property
(no sampled circuit outside it beats its last entry)."""
import numpy as np
import pytest

import oracle
from gpu_common import assert_fp32_fitness, oracle_problem, state_equal
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


def _G(s):
    return oracle.num_gates(s.n, s.library)


def _check_topk_sampled(p, s, last, rng, n_others):
    """Top-k of one generation: each entry's binary64 fitness and cost equal the
    oracle's for that circuit, the entries are in ranking order, and no circuit
    of a random sample outside the top-k ranks above the last entry."""
    gi = last["gate_idx"]
    tk = last["topk"][:s.topk]
    idx = np.array([t[0] for t in tk], np.int64)
    F, C = oracle.eval_circuits(p, gi[idx])
    assert [t[2] for t in tk] == list(F)
    assert [t[1] for t in tk] == list(C)
    keys = [(-f, c, i) for f, c, i in zip(F, C, idx)]
    assert keys == sorted(keys)
    others = np.setdiff1d(rng.choice(s.P, n_others, replace=False), idx)
    Fo, Co = oracle.eval_circuits(p, gi[others])
    for f, c, i in zip(Fo, Co, others):
        assert (-f, c, i) > keys[-1]


def test_bench_workload_every_stage(qe, torch):
    """Three 3-qubit searches of P = 4096 (binary32, top-32): sample bit-exact,
    fitness within its bound, top-32 bit-exact, update bit-exact given the
    step's own binary32 fitness, for each of four generations."""
    searches = W.config(2)
    probs = [oracle_problem(s, r) for r, s in enumerate(searches)]
    stream = torch.cuda.Stream()
    with qe.Context(searches, stream=stream) as ctx:
        for gen in range(4):
            before = [ctx.get_state(r) for r in range(len(searches))]
            ctx.step_raw(1, None)
            for run, s in enumerate(searches):
                p = probs[run]
                cur, best, bf = [a.copy() for a in before[run]]
                last = ctx.last_generation(run)
                gi, sid = oracle.sample(p, cur, gen)
                assert np.array_equal(last["gate_idx"], gi)
                assert np.array_equal(last["seg_id"], sid)
                F, C = oracle.eval_circuits(p, gi)
                assert_fp32_fitness(last["fitness"], F, s, C)
                order = oracle.topk(F, C, s.topk)
                assert [t[0] for t in last["topk"]] == list(order)
                assert [t[2] for t in last["topk"]] == list(F[order])
                oracle.update(p, cur, best, bf, gen, sid, last["fitness"])
                c2, b2, bf2 = ctx.get_state(run)
                assert state_equal(c2, cur) and state_equal(b2, best) and state_equal(bf2, bf)


def test_bench_workload_pipelined_record(qe, torch):
    """The same workload with generations enqueued back to back (each ranked
    while the next one runs): the best-so-far record after six generations is
    the oracle's best binary64 circuit over the six, and the last top-32 is the
    oracle's."""
    searches = W.config(2)
    probs = [oracle_problem(s, r) for r, s in enumerate(searches)]
    gens = 6
    with qe.Context(searches) as ctx:
        states = []
        for gen in range(gens):
            states.append([ctx.get_state(r) for r in range(len(searches))])
            if gen < gens - 1:
                ctx.step_raw(1, None)
        reps = ctx.step(1)
        for run, s in enumerate(searches):
            p = probs[run]
            bfit, bcost, bgates = -np.inf, 2**32 - 1, None
            for gen in range(gens):
                cur = states[gen][run][0].copy()
                gi, _ = oracle.sample(p, cur, gen)
                F, C = oracle.eval_circuits(p, gi)
                b = oracle.topk(F, C, 1)[0]
                if F[b] > bfit or (F[b] == bfit and C[b] < bcost):
                    bfit, bcost, bgates = F[b], int(C[b]), bytes(gi[b])
            r = reps[run]
            assert r["generation"] == gens
            assert r["best_fitness"] == bfit and r["best_cost"] == bcost
            assert bytes(r["best_gates"][:s.L]) == bgates
            last = ctx.last_generation(run)
            assert np.array_equal(last["gate_idx"], gi)
            order = oracle.topk(F, C, s.topk)
            assert [t[0] for t in last["topk"]] == list(order)


def test_4qubit_full_size_generation(qe, torch):
    """C3NOT search, P = 65536, L = 32, binary32 with binary64 top-64: the
    generation-0 sample bit-exact, the update bit-exact given the step's own
    fitness, and generation 1 checked on sampled circuits."""
    s = W.config(3)[0]
    p = oracle_problem(s, 0)
    rng = np.random.default_rng(3)
    with qe.Context([s]) as ctx:
        cur, best, bf = ctx.get_state(0)
        ctx.step_raw(1, None)
        last = ctx.last_generation(0)
        gi, sid = oracle.sample(p, cur, 0)
        assert np.array_equal(last["gate_idx"], gi)
        assert np.array_equal(last["seg_id"], sid)
        sub = rng.choice(s.P, 3000, replace=False)
        F, C = oracle.eval_circuits(p, gi[sub])
        assert_fp32_fitness(last["fitness"][sub], F, s, C)
        _check_topk_sampled(p, s, last, rng, 1500)
        oracle.update(p, cur, best, bf, 0, sid, last["fitness"])
        c2, b2, bf2 = ctx.get_state(0)
        assert state_equal(c2, cur) and state_equal(b2, best) and state_equal(bf2, bf)
        del best, b2
        ctx.step_raw(1, None)
        last = ctx.last_generation(0)
        gi, sid = oracle.sample(p, cur, 1)
        assert np.array_equal(last["gate_idx"], gi) and np.array_equal(last["seg_id"], sid)
        sub = rng.choice(s.P, 1000, replace=False)
        F, C = oracle.eval_circuits(p, gi[sub])
        assert_fp32_fitness(last["fitness"][sub], F, s, C)
        _check_topk_sampled(p, s, last, rng, 1000)


def test_5qubit_full_size_generation(qe, torch):
    """C4NOT search, P = 262144, L = 64, binary32 with binary64 top-128, first
    generation: every segment id is slot t of an individual of some region and
    its gate belongs to that region; from the uniform initial state the three
    outcomes of every region are equally likely (chi-square); fitness of a
    random subset within its bound; the top-128 circuit by circuit."""
    s = W.config(5)[0]
    p = oracle_problem(s, 0)
    rng = np.random.default_rng(5)
    R = oracle.num_regions(s.n, s.library)
    with qe.Context([s]) as ctx:
        ctx.step_raw(1, None)
        last = ctx.last_generation(0)
    gi = last["gate_idx"].astype(np.int64)
    sid = last["seg_id"].astype(np.int64)
    LP = s.L * s.P
    r, rem = sid // LP, sid % LP
    assert np.all(r < R)
    assert np.array_equal(rem % s.L, np.broadcast_to(np.arange(s.L), sid.shape))
    # outcome k of each slot: its gate's position among its region's three
    k = np.full(gi.shape, -1, np.int64)
    for rr in range(R):
        for kk in range(3):
            k[(r == rr) & (gi == oracle.region_gate(s.n, s.library, rr, kk))] = kk
    assert np.all(k >= 0)
    from scipy.stats import chisquare
    assert chisquare(np.bincount(k.ravel(), minlength=3)).pvalue > 1e-4
    assert chisquare(np.bincount(r.ravel(), minlength=R)).pvalue > 1e-4
    sub = rng.choice(s.P, 150, replace=False)
    F, C = oracle.eval_circuits(p, last["gate_idx"][sub])
    assert_fp32_fitness(last["fitness"][sub], F, s, C)
    _check_topk_sampled(p, s, last, rng, 150)


def test_5qubit_full_size_ga(qe, torch):
    """The GA run of the C4NOT search at P = 262144: the initial genome, the
    binary32 fitness of sampled circuits, and the next genome given the step's
    own fitness, bit for bit."""
    s = W.config(5, encoding=W.ENC_GA)[0]
    p = oracle_problem(s, 0)
    rng = np.random.default_rng(6)
    with qe.Context([s]) as ctx:
        g0 = ctx.get_state(0)
        assert np.array_equal(g0, oracle.ga_init(p, _G(s)))
        ctx.step_raw(1, None)
        last = ctx.last_generation(0)
        assert np.array_equal(last["gate_idx"], g0)
        sub = rng.choice(s.P, 150, replace=False)
        F, C = oracle.eval_circuits(p, g0[sub])
        assert_fp32_fitness(last["fitness"][sub], F, s, C)
        cost_all = np.array([oracle.cost(s.n, s.library, row) for row in g0], np.uint32)
        nxt = oracle.ga_next(p, _G(s), 0, s.ga_mutation_rate, g0, last["fitness"], cost_all)
        assert np.array_equal(ctx.get_state(0), nxt)



def test_maximum_sizes(qe, torch):
    """The largest search the ABI accepts: n = 5, L = 64, P = 2^20 (R*P*L =
    1.68e9 segments, 107 GB of encoding state), top-1024; plus 4096 searches
    in one context.  Checked on sampled outputs: the slot structure of the
    sample, binary32 fitness of a random subset, and the top-1024 (binary64
    values of a sample of its entries, ranking order, no sampled outsider above
    the last entry)."""
    s = W.Search(5, 64, 1 << 20, W.LIB_NCV | W.LIB_HT, W.cknot(5), seed=21, topk=1024)
    p = oracle_problem(s, 0)
    rng = np.random.default_rng(21)
    with qe.Context([s]) as ctx:
        ctx.step_raw(1, None)
        last = ctx.last_generation(0)
    sid = last["seg_id"].astype(np.int64)
    LP = s.L * s.P
    assert np.all(sid // LP < oracle.num_regions(s.n, s.library))
    assert np.array_equal(sid % s.L, np.broadcast_to(np.arange(s.L), sid.shape))
    sub = rng.choice(s.P, 100, replace=False)
    F, C = oracle.eval_circuits(p, last["gate_idx"][sub])
    assert_fp32_fitness(last["fitness"][sub], F, s, C)
    tk = last["topk"]
    assert len(tk) == 1024
    keys = [(-t[2], t[1], t[0]) for t in tk]
    assert keys == sorted(keys)
    pick = np.sort(rng.choice(1024, 64, replace=False))
    idx = np.array([tk[j][0] for j in pick], np.int64)
    Fk, Ck = oracle.eval_circuits(p, last["gate_idx"][idx])
    assert [tk[j][2] for j in pick] == list(Fk) and [tk[j][1] for j in pick] == list(Ck)
    others = np.setdiff1d(rng.choice(s.P, 100, replace=False), [t[0] for t in tk])
    Fo, Co = oracle.eval_circuits(p, last["gate_idx"][others])
    for f, c, i in zip(Fo, Co, others):
        assert (-f, c, i) > keys[-1]
    many = [W.Search(3, 4, 8, W.LIB_NCV | W.LIB_IDENTITY, W.cknot(3), seed=5, topk=2,
                     precision=W.PREC_FP64) for _ in range(4096)]
    with qe.Context(many) as ctx:
        reps = ctx.step(2)
    assert len(reps) == 4096 and all(r["generation"] == 2 for r in reps)
    for run in (0, 1234, 4095):
        ref = oracle_problem(many[run], run)
        cur, best, bf = oracle.init_state(ref)
        bfit = -np.inf
        for gen in range(2):
            gi, sid = oracle.sample(ref, cur, gen)
            Fg, Cg = oracle.eval_circuits(ref, gi)
            b = oracle.topk(Fg, Cg, 1)[0]
            bfit = max(bfit, Fg[b])
            oracle.update(ref, cur, best, bf, gen, sid, Fg)
        assert reps[run]["best_fitness"] == bfit
