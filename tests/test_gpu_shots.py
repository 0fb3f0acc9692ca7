"""Repeated qutrit measurement (Sec. IV-A1) on the GPU against the oracle:
with K > 1 shots every slot's gate comes from the most frequent of K binary32
CDF comparisons (the lowest outcome on a tie), measured ahead of the circuit
kernel.  The decisions are integer work on the same binary32 numbers on both
sides, so samples are bit-exact, and so are binary64 trajectories."""
import numpy as np
import pytest

import oracle
from gpu_common import assert_fp32_fitness, oracle_problem, state_equal
from paper_1809_11134_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DISC = W.LIB_NCV | W.LIB_HT | W.LIB_IDENTITY


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


def random_state(rng, S):
    """normalised random qutrits (3 complex) and qubits (2 real) per segment"""
    q = rng.normal(size=(S, 6))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    b = rng.normal(size=(S, 2))
    b /= np.linalg.norm(b, axis=1, keepdims=True)
    cur = np.concatenate([q, b], 1).astype(np.float32)
    return cur.ravel(), cur.ravel().copy(), np.full(S, -1.0, np.float32)


@pytest.mark.parametrize("K", [2, 3, 4, 7, 8, 64])
@pytest.mark.parametrize("n,L,lib", [(3, 16, DISC), (4, 33, W.LIB_NCV | W.LIB_HT),
                                     (5, 64, DISC), (2, 5, W.LIB_ISING)])
def test_sample_bit_exact(qe, torch, K, n, L, lib):
    s = W.Search(n, L, 257, lib, W.cknot(n), seed=K, shots=K)
    p = oracle_problem(s, 0)
    rng = np.random.default_rng(K + n)
    S = oracle.num_regions(n, lib) * s.P * L
    cur, best, bf = random_state(rng, S)
    g = torch.zeros(s.P * L, dtype=torch.uint8, device="cuda")
    sid = torch.zeros(s.P * L, dtype=torch.int32, device="cuda")
    with qe.Context([s]) as ctx:
        ctx.set_state(0, cur, best, bf)
        for gen in (0, 5):
            ctx.sample(0, gen, g, sid)
            gi, si = oracle.sample(p, cur, gen)
            assert np.array_equal(g.cpu().numpy().reshape(s.P, L), gi)
            assert np.array_equal(sid.cpu().numpy().astype(np.uint32).reshape(s.P, L), si)


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


def test_trajectory_fp64_bit_exact(qe, torch):
    """K-shot searches (discrete and Ising) beside a one-shot search in one
    context, binary64, ten generations: everything bit-exact."""
    searches = [W.Search(3, 16, 200, DISC, W.cknot(3), seed=1, precision=W.PREC_FP64, topk=5,
                         shots=5),
                W.Search(3, 12, 150, DISC, W.peres(), seed=2, precision=W.PREC_FP64, topk=4),
                W.Search(2, 3, 64, W.LIB_ISING, W.cknot(2), seed=3, precision=W.PREC_FP64,
                         topk=3, shots=8),
                W.Search(4, 10, 90, W.LIB_NCV | W.LIB_HT, W.cknot(4), seed=4,
                         precision=W.PREC_FP64, topk=2, shots=2)]
    gens = 10
    ref = _oracle_run(searches, gens)
    with qe.Context(searches) as ctx:
        for gen in range(gens):
            reps = ctx.step(1)
            for run, s in enumerate(searches):
                gi, sid, F, tk, bfit, bcost, bgates = ref[run][0][gen]
                last = ctx.last_generation(run)
                assert np.array_equal(last["gate_idx"], gi), (gen, run)
                assert np.array_equal(last["seg_id"], sid)
                assert np.array_equal(last["fitness"], F)
                assert [t[0] for t in last["topk"]] == list(tk[:s.topk])
                assert reps[run]["best_fitness"] == bfit and reps[run]["best_cost"] == bcost
                assert bytes(reps[run]["best_gates"][:s.L]) == bgates[:s.L]
        for run in range(len(searches)):
            c, b, bf = ctx.get_state(run)
            assert state_equal(c, ref[run][1]) and state_equal(b, ref[run][2])
            assert state_equal(bf, ref[run][3])


def test_fp32_each_stage(qe, torch):
    """binary32 with K shots: the sample bit-exact, fitness within its bound, the
    update bit-exact given the step's own fitness."""
    searches = [W.Search(3, 16, 1000, DISC, W.cknot(3), seed=5, topk=16, shots=3),
                W.Search(5, 20, 120, W.LIB_NCV | W.LIB_HT, W.cknot(5), seed=6, topk=6, shots=15),
                W.Search(3, 9, 300, W.LIB_ISING, W.cknot(3), seed=7, topk=8, shots=4)]
    probs = [oracle_problem(s, r) for r, s in enumerate(searches)]
    with qe.Context(searches) as ctx:
        for gen in range(4):
            before = [ctx.get_state(r) for r in range(len(searches))]
            ctx.step(1)
            for run, s in enumerate(searches):
                p = probs[run]
                cur, best, bf = [x.copy() for x in before[run]]
                last = ctx.last_generation(run)
                if s.library == W.LIB_ISING:
                    gi, sid, amps = oracle.sample(p, cur, gen, with_amps=True)
                    F, C = oracle.eval_circuits(p, gi, amps)
                else:
                    gi, sid = oracle.sample(p, cur, gen)
                    F, C = oracle.eval_circuits(p, gi)
                assert np.array_equal(last["gate_idx"], gi) and np.array_equal(last["seg_id"], sid)
                assert_fp32_fitness(last["fitness"], F, s, C)
                oracle.update(p, cur, best, bf, gen, sid, last["fitness"])
                c2, b2, bf2 = ctx.get_state(run)
                assert state_equal(c2, cur) and state_equal(b2, best) and state_equal(bf2, bf)
