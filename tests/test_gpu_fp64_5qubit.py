"""Whole binary64 generations at 5 qubits against the oracle.

At 5 qubits the binary64 circuit kernel spreads each circuit's 32 columns over
four warps (eight rows per lane); the warps of a group sample the same slots,
the first one writes them, lists the mutating individual and scatters the
segment fitness, and the score's terms meet in shared memory, summed in the
oracle's order (Eq. (11), columns ascending).  Every form the kernel is
compiled in runs here: one measurement per slot, K measurements per slot
(Sec. IV-A1), a dense target, the Ising library (Sec. III) and the GA's
genomes; sampled circuits, segment ids, fitness, top-k, the best-so-far record
and the state must equal the oracle's bit for bit.  One search holds more
circuits than the GPU has resident four-warp groups, so the groups' loop runs
more than once.
"""
import numpy as np
import pytest

import oracle
from gpu_common import oracle_problem, state_equal
from paper_1809_11134_gb300 import workloads as W

pytestmark = pytest.mark.gpu

NCV, HT, ID = W.LIB_NCV, W.LIB_HT, W.LIB_IDENTITY
FP64 = W.PREC_FP64


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


def _haar(rng, N):
    q, r = np.linalg.qr(rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def _near(rng, lib, L):
    """a reachable 5-qubit circuit's unitary times a random unitary, so that
    the fitness spreads instead of sitting near 0"""
    g = rng.integers(0, oracle.num_gates(5, lib), L).astype(np.uint8)
    re, im = oracle.compose(5, lib, g)
    return (re + 1j * im) @ _haar(rng, 32)


def _oracle_run(searches, gens):
    out = []
    for run, s in enumerate(searches):
        p = oracle_problem(s, run)
        cur, best, bf = oracle.init_state(p)
        rep = oracle.new_report()
        hist = []
        for gen in range(gens):
            gi, sid, F, cost, tk = oracle.step(p, cur, best, bf, gen, max(s.topk, 1), rep)
            hist.append((gi, sid, F, tk, rep.best_fitness, rep.best_cost, bytes(rep.best_gates)))
        out.append((hist, cur, best, bf))
    return out


def _searches():
    rng = np.random.default_rng(55)
    return [
        # one measurement per slot; P above the resident groups (152 SMs x 4)
        W.Search(5, 10, 700, NCV | HT, W.cknot(5), seed=51, precision=FP64, topk=7),
        # the identity in the library (the qubit decides "gate present"), the
        # probability reading of the fitness and a gate-cost penalty
        W.Search(5, 64, 40, NCV | HT | ID, W.cknot(5), seed=52, precision=FP64, topk=5,
                 fitness_kind=W.FIT_PROB, cost_weight=0.1),
        # K = 3 measurements per slot
        W.Search(5, 33, 45, NCV | HT, W.random_perm(rng, 5), seed=53, precision=FP64, topk=4,
                 shots=3),
        # dense target
        W.Search(5, 24, 50, NCV | HT, W.cknot(5), seed=54, precision=FP64, topk=6,
                 target=_near(rng, NCV | HT, 24)),
        # the paper's Ising library (rotation angles from the qubits)
        W.Search(5, 20, 60, W.LIB_ISING, W.cknot(5), seed=56, precision=FP64, topk=3),
    ]


def test_qeqea_generations_bit_exact(qe, torch):
    searches = _searches()
    gens = 4
    ref = _oracle_run(searches, gens)
    with qe.Context(searches) as ctx:
        for gen in range(gens):
            reps = ctx.step(1)
            for run, s in enumerate(searches):
                gi, sid, F, tk, bfit, bcost, bgates = ref[run][0][gen]
                last = ctx.last_generation(run)
                assert np.array_equal(last["gate_idx"], gi), (gen, run)
                assert np.array_equal(last["seg_id"], sid), (gen, run)
                assert np.array_equal(last["fitness"], F), (gen, run)
                assert [t[0] for t in last["topk"]] == list(tk[:s.topk]), (gen, run)
                assert reps[run]["best_fitness"] == bfit and reps[run]["best_cost"] == bcost
                assert bytes(reps[run]["best_gates"][:s.L]) == bgates[:s.L]
        for run in range(len(searches)):
            c, b, bf = ctx.get_state(run)
            assert state_equal(c, ref[run][1]) and state_equal(b, ref[run][2]), run
            assert state_equal(bf, ref[run][3]), run


def test_ga_generations_bit_exact(qe, torch):
    """the GA's genomes through the same kernel (no sampling, no scatter)"""
    s = W.Search(5, 40, 66, NCV | HT, W.cknot(5), seed=57, precision=FP64, topk=5,
                 encoding=W.ENC_GA, ga_mutation_rate=0.05)
    p = oracle_problem(s, 0)
    G = oracle.num_gates(5, s.library)
    genome = oracle.ga_init(p, G)
    with qe.Context([s]) as ctx:
        for gen in range(4):
            assert np.array_equal(ctx.get_state(0), genome), gen
            ctx.step(1)
            F, C = oracle.eval_circuits(p, genome)
            last = ctx.last_generation(0)
            assert np.array_equal(last["gate_idx"], genome)
            assert np.array_equal(last["fitness"], F), gen
            assert [t[0] for t in last["topk"]] == list(oracle.topk(F, C, s.topk)), gen
            genome = oracle.ga_next(p, G, gen, s.ga_mutation_rate, genome, F, C)
        assert np.array_equal(ctx.get_state(0), genome)


def test_4qubit_generations_bit_exact(qe, torch):
    """the same at 4 qubits, where binary64 circuits run on two warps each: one
    search with more circuits than the GPU has resident two-warp groups, one
    with a dense target (and K = 2 measurements), three generations"""
    rng = np.random.default_rng(44)
    T = _haar(rng, 16)
    searches = [W.Search(4, 8, 2000, NCV | HT, W.cknot(4), seed=41, precision=FP64, topk=6),
                W.Search(4, 21, 70, NCV | HT | ID, W.random_perm(rng, 4), seed=42,
                         precision=FP64, topk=4, shots=2, target=T)]
    gens = 3
    ref = _oracle_run(searches, gens)
    with qe.Context(searches) as ctx:
        for gen in range(gens):
            reps = ctx.step(1)
            for run, s in enumerate(searches):
                gi, sid, F, tk, bfit, bcost, bgates = ref[run][0][gen]
                last = ctx.last_generation(run)
                assert np.array_equal(last["gate_idx"], gi), (gen, run)
                assert np.array_equal(last["fitness"], F), (gen, run)
                assert [t[0] for t in last["topk"]] == list(tk[:s.topk]), (gen, run)
                assert reps[run]["best_fitness"] == bfit and reps[run]["best_cost"] == bcost
        for run in range(len(searches)):
            c, b, bf = ctx.get_state(run)
            assert state_equal(c, ref[run][1]) and state_equal(bf, ref[run][3]), run
