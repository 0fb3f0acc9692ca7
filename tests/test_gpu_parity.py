"""CUDA path vs the CPU oracle, element by element, through the C ABI.

Bit-exact: sampled gates and segment ids, binary64 fitness and unitaries,
top-k (indices, costs, binary64 fitness), the encoding state after an update,
whole binary64 trajectories.  Within the stated bound: binary32 fitness and
unitaries (1e-5 max-abs on unitary entries; the d-space bound on fitness)."""
import numpy as np
import pytest

import oracle
from gpu_common import assert_fp32_fitness, eps_d, oracle_problem, state_equal
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


def S(n, L, P, lib, perm=None, **kw):
    return W.Search(n, L, P, lib, perm if perm is not None else W.cknot(n), **kw)


SHAPES = [
    S(3, 16, 1000, NCV | HT | ID, seed=1),
    S(4, 32, 300, NCV | HT, seed=7),
    S(5, 64, 130, NCV | HT, seed=9),
    S(5, 33, 41, NCV | HT | ID, seed=2),
    S(1, 1, 1, HT, perm=[1, 0], seed=3),
    S(2, 7, 33, NCV | ID, perm=[0, 1, 3, 2], seed=4),
    S(3, 5, 64, NCV | ID, seed=0),
]


def _G(s):
    return oracle.num_gates(s.n, s.library)


# ------------------------------------------------------------------ sampling
@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
def test_sample_bit_exact(qe, torch, prec):
    searches = [W.Search(**{**s.__dict__, "precision": prec}) for s in SHAPES]
    rng = np.random.default_rng(5)
    with qe.Context(searches) as ctx:
        for run, s in enumerate(searches):
            p = oracle_problem(s, run)
            nseg = oracle.num_segments(p)
            cur, best, bf = W.random_state(rng, nseg)
            ctx.set_state(run, cur, best, bf)
            gi = torch.zeros(s.P * s.L, dtype=torch.uint8, device="cuda")
            sid = torch.zeros(s.P * s.L, dtype=torch.int32, device="cuda")
            for gen in (0, 1, 17, 4000000000):
                ctx.sample(run, gen, gi, sid)
                torch.cuda.synchronize()
                ogi, osid = oracle.sample(p, cur, gen)
                assert np.array_equal(gi.cpu().numpy().reshape(s.P, s.L), ogi)
                assert np.array_equal(sid.cpu().numpy().view(np.uint32).reshape(s.P, s.L), osid)


# ------------------------------------------------------------------ binary64 eval
EVAL_CASES = [
    (1, HT, 9), (2, NCV | ID, 12), (2, NCV | HT, 40), (3, NCV | ID, 5), (3, NCV | HT | ID, 16),
    (4, NCV | HT, 32), (5, NCV | HT, 64), (5, NCV | HT | ID, 1), (4, HT, 20),
]


@pytest.mark.parametrize("n,lib,L", EVAL_CASES)
@pytest.mark.parametrize("kind,lam", [(W.FIT_TRACE, 0.0), (W.FIT_PROB, 0.0), (W.FIT_TRACE, 0.3)])
def test_eval_fp64_bit_exact(qe, torch, n, lib, L, kind, lam):
    nc = 300 + 7 * n  # several warps per block plus a ragged tail
    rng = np.random.default_rng(n * 100 + L)
    s = S(n, L, nc, lib, perm=W.random_perm(rng, n), precision=W.PREC_FP64, fitness_kind=kind,
          cost_weight=lam)
    g = W.random_gates(rng, nc, L, _G(s))
    with qe.Context([s]) as ctx:
        fit = torch.zeros(nc, dtype=torch.float64, device="cuda")
        cost = torch.zeros(nc, dtype=torch.int32, device="cuda")
        ctx.eval(0, torch.from_numpy(g).cuda(), fit, cost=cost)
        torch.cuda.synchronize()
        F, C = oracle.eval_circuits(oracle_problem(s, 0), g)
        assert np.array_equal(fit.cpu().numpy(), F)
        assert np.array_equal(cost.cpu().numpy().astype(np.uint32), C)


@pytest.mark.parametrize("lib,Lmax", [(NCV | ID, 3), (NCV | HT | ID, 3)])
def test_bruteforce_short_circuits_fp64(qe, torch, lib, Lmax):
    """Every circuit of length <= 3 of the 19- and 28-gate 3-qubit libraries
    against the Toffoli: identical binary64 fitness for every circuit."""
    G = oracle.num_gates(3, lib)
    for L in range(1, Lmax + 1):
        idx = np.indices((G,) * L).reshape(L, -1).T.astype(np.uint8)
        nc = idx.shape[0]
        s = S(3, L, 64, lib, precision=W.PREC_FP64)
        with qe.Context([s]) as ctx:
            fit = torch.zeros(nc, dtype=torch.float64, device="cuda")
            ctx.eval(0, torch.from_numpy(np.ascontiguousarray(idx)).cuda(), fit, n_circuits=nc)
            torch.cuda.synchronize()
            p = oracle.make_problem(3, L, nc, lib, W.cknot(3))
            F, _ = oracle.eval_circuits(p, idx)
            assert np.array_equal(fit.cpu().numpy(), F)
            if lib == NCV | ID and L == 1:
                assert F.max() == 0.5


@pytest.mark.parametrize("n,lib,L", [(3, NCV | HT | ID, 16), (4, NCV | HT, 32), (5, NCV | HT, 64),
                                     (2, HT, 30), (1, HT, 3)])
def test_compose_matches_oracle(qe, torch, n, lib, L):
    nc = 40
    rng = np.random.default_rng(n + 50)
    N = 1 << n
    for prec in (W.PREC_FP64, W.PREC_FP32):
        s = S(n, L, nc, lib, precision=prec)
        g = W.random_gates(rng, nc, L, _G(s))
        dt = torch.float64 if prec == W.PREC_FP64 else torch.float32
        with qe.Context([s]) as ctx:
            U = torch.zeros(nc * N * N * 2, dtype=dt, device="cuda")
            ctx.compose(0, torch.from_numpy(g).cuda(), U)
            torch.cuda.synchronize()
            U = U.cpu().numpy().astype(np.float64).reshape(nc, N, N, 2)
        for c in range(nc):
            re, im = oracle.compose(n, lib, g[c])
            if prec == W.PREC_FP64:
                assert np.array_equal(U[c, :, :, 0], re) and np.array_equal(U[c, :, :, 1], im)
            else:
                assert np.abs(U[c, :, :, 0] - re).max() <= 1e-5
                assert np.abs(U[c, :, :, 1] - im).max() <= 1e-5


# ------------------------------------------------------------------ binary32 eval
@pytest.mark.parametrize("n,lib,L", [(3, NCV | HT | ID, 16), (4, NCV | HT, 32), (5, NCV | HT, 64),
                                     (5, NCV | HT, 7), (2, NCV | HT, 50)])
@pytest.mark.parametrize("kind", [W.FIT_TRACE, W.FIT_PROB])
def test_eval_fp32_within_bound(qe, torch, n, lib, L, kind):
    nc = 700
    rng = np.random.default_rng(n * 7 + L)
    s = S(n, L, nc, lib, precision=W.PREC_FP32, fitness_kind=kind)
    g = W.random_gates(rng, nc, L, _G(s))
    with qe.Context([s]) as ctx:
        fit = torch.zeros(nc, dtype=torch.float32, device="cuda")
        ctx.eval(0, torch.from_numpy(g).cuda(), fit)
        torch.cuda.synchronize()
        F, C = oracle.eval_circuits(oracle_problem(s, 0), g)
        assert_fp32_fitness(fit.cpu().numpy(), F, s)


def test_fp32_exact_on_textbook_circuits(qe, torch):
    """NCV products are dyadic: binary32 is exact, fitness exactly 1."""
    import test_oracle_pins as T
    lib = NCV | ID
    for spec, perm in [(T.TOFFOLI5, W.cknot(3)), (T.PERES4, W.peres()), (T.FREDKIN7, W.fredkin())]:
        g = T._circuit(3, lib, spec)
        g = np.array([g + [0] * (8 - len(g))], np.uint8)
        s = S(3, 8, 4, lib, perm=perm, precision=W.PREC_FP32)
        with qe.Context([s]) as ctx:
            fit = torch.zeros(1, dtype=torch.float32, device="cuda")
            ctx.eval(0, torch.from_numpy(g).cuda(), fit)
            assert fit.item() == 1.0


# ------------------------------------------------------------------ ranking
@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
@pytest.mark.parametrize("n,lib,L,P,k", [
    (3, NCV | ID, 3, 2000, 32),      # very many ties at the top
    (3, NCV | HT | ID, 16, 4096, 32),
    (4, NCV | HT, 32, 1500, 64),
    (5, NCV | HT, 64, 600, 128),
    (3, NCV | HT, 6, 50, 50),        # k = P
    (2, NCV, 2, 3000, 1),
    (4, NCV | HT, 12, 20000, 64),   # beyond the selection's shared-memory key cache
])
def test_topk_bit_exact(qe, torch, prec, n, lib, L, P, k):
    rng = np.random.default_rng(P + k)
    s = S(n, L, P, lib, precision=prec, topk=k, cost_weight=0.0 if n != 4 else 0.1)
    g = W.random_gates(rng, P, L, _G(s))
    with qe.Context([s]) as ctx:
        dt = torch.float64 if prec == W.PREC_FP64 else torch.float32
        fit = torch.zeros(P, dtype=dt, device="cuda")
        top = ctx.eval(0, torch.from_numpy(g).cuda(), fit, topk=True)
        F, C = oracle.eval_circuits(oracle_problem(s, 0), g)
        order = oracle.topk(F, C, k)
        assert [t[0] for t in top] == list(order)
        assert [t[1] for t in top] == list(C[order])
        assert [t[2] for t in top] == list(F[order])


@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
def test_topk_exact_whatever_the_previous_ranking(qe, torch, prec):
    """rankings in one context share their scratch (candidates, queue, top-k
    buffer): each top-k must depend on its own circuits only; the same
    population twice, a worse one after a better one, a better one after a
    worse one, and populations of other sizes in between"""
    s = S(3, 16, 4096, NCV | HT | ID, precision=prec, topk=32)
    rng = np.random.default_rng(77 + prec)
    g_good = W.random_gates(rng, 4096, 16, _G(s))
    g_bad = g_good.copy()
    g_bad[:, :] = 0  # all identities: every circuit scores f(I) (ties everywhere)
    g_bad[::7] = W.random_gates(rng, len(g_bad[::7]), 16, _G(s))
    dt = torch.float64 if prec == W.PREC_FP64 else torch.float32
    with qe.Context([s]) as ctx:
        for g in (g_good, g_good, g_bad, g_good, g_good[:100], g_good[:31], g_bad, g_bad):
            n = len(g)
            fit = torch.zeros(n, dtype=dt, device="cuda")
            top = ctx.eval(0, torch.from_numpy(np.ascontiguousarray(g)).cuda(), fit, topk=True)
            F, C = oracle.eval_circuits(oracle_problem(s, 0), g)
            order = oracle.topk(F, C, min(32, n))
            assert [t[0] for t in top] == list(order)
            assert [t[2] for t in top] == list(F[order])


def test_invalid_gate_index_is_reported(qe, torch):
    s = S(3, 4, 16, NCV | ID, precision=W.PREC_FP32, topk=4)
    g = np.zeros((16, 4), np.uint8)
    g[5, 2] = 200
    with qe.Context([s]) as ctx:
        fit = torch.zeros(16, dtype=torch.float32, device="cuda")
        with pytest.raises(qe.QeError) as e:
            ctx.eval(0, torch.from_numpy(g).cuda(), fit, topk=True)
        assert e.value.status == qe.QE_ENUMERIC
        f = fit.cpu().numpy()
        assert np.isnan(f[5]) and np.all(np.isfinite(np.delete(f, 5)))
        # the context stays usable
        g[5, 2] = 1
        top = ctx.eval(0, torch.from_numpy(g).cuda(), fit, topk=True)
        assert len(top) == 4


def test_empty_eval_is_a_no_op(qe, torch):
    s = S(3, 4, 16, NCV | ID, precision=W.PREC_FP32, topk=4)
    with qe.Context([s]) as ctx:
        fit = torch.zeros(1, dtype=torch.float32, device="cuda")
        assert ctx.eval(0, torch.zeros((0, 4), dtype=torch.uint8, device="cuda"), fit,
                        n_circuits=0, topk=True) == []


# ------------------------------------------------------------------ update
@pytest.mark.parametrize("pm", [0.0, 0.1, 1.0])
@pytest.mark.parametrize("si", [0, 1, 3, 5])
def test_update_bit_exact(qe, torch, pm, si):
    base = SHAPES[si]
    s = W.Search(**{**base.__dict__, "p_mutation": pm, "precision": W.PREC_FP64})
    rng = np.random.default_rng(si * 10 + int(pm * 10))
    with qe.Context([s]) as ctx:
        p = oracle_problem(s, 0)
        nseg = oracle.num_segments(p)
        cur, best, bf = W.random_state(rng, nseg, best_f_range=(-1.0, 0.9))
        ctx.set_state(0, cur, best, bf)
        for gen in (3, 4):
            gi, sid = oracle.sample(p, cur, gen)
            F = W.random_fitness(rng, s.P, discrete=gen == 3)
            ctx.update(0, gen, torch.from_numpy(sid.view(np.int32).ravel()).cuda(),
                       torch.from_numpy(F).cuda())
            oracle.update(p, cur, best, bf, gen, sid, F)
            c2, b2, bf2 = ctx.get_state(0)
            assert state_equal(c2, cur)
            assert state_equal(b2, best)
            assert state_equal(bf2, bf)


@pytest.mark.parametrize("P", [16383, 16384])
def test_update_bit_exact_many_slots(qe, torch, P):
    """2^20 circuit slots (L = 64, P = 16384) and one circuit fewer: the two
    sides of the size from which the elitism role runs four lanes per slot"""
    s = W.Search(2, 64, P, NCV, [0, 1, 3, 2], seed=6, precision=W.PREC_FP64, p_mutation=0.1)
    rng = np.random.default_rng(P)
    with qe.Context([s]) as ctx:
        p = oracle_problem(s, 0)
        cur, best, bf = W.random_state(rng, oracle.num_segments(p), best_f_range=(-1.0, 0.9))
        ctx.set_state(0, cur, best, bf)
        for gen in (0, 1):
            gi, sid = oracle.sample(p, cur, gen)
            F = W.random_fitness(rng, s.P, discrete=gen == 0)
            ctx.update(0, gen, torch.from_numpy(sid.view(np.int32).ravel()).cuda(),
                       torch.from_numpy(F).cuda())
            oracle.update(p, cur, best, bf, gen, sid, F)
            c2, b2, bf2 = ctx.get_state(0)
            assert state_equal(c2, cur)
            assert state_equal(b2, best)
            assert state_equal(bf2, bf)


# ------------------------------------------------------------------ whole generations
def _oracle_run(searches, gens):
    out = []
    for run, s in enumerate(searches):
        p = oracle_problem(s, run)
        cur, best, bf = oracle.init_state(p)
        rep = oracle.new_report()
        hist = []
        for gen in range(gens):
            gi, sid, F, cost, tk = oracle.step(p, cur, best, bf, gen, max(s.topk, 1), rep)
            hist.append((gi, sid, F, tk, rep.best_fitness, rep.best_cost, bytes(rep.best_gates),
                         rep.useful_flops, rep.mean_fitness))
        out.append((hist, cur, best, bf))
    return out


@pytest.mark.parametrize("cfg,P,gens", [(1, None, 20), (2, 256, 12), (0, 16384, 3)])
def test_step_trajectory_fp64_bit_exact(qe, torch, cfg, P, gens):
    if cfg == 0:  # 2^20 circuit slots per generation (L = 64): the four-lane elitism role
        searches = [W.Search(2, 64, P, NCV | HT, [0, 1, 3, 2], seed=6, precision=W.PREC_FP64,
                             topk=16)]
    else:
        searches = W.config(cfg, precision=W.PREC_FP64, P=P)
    ref = _oracle_run(searches, gens)
    with qe.Context(searches) as ctx:
        for gen in range(gens):
            reps = ctx.step(1)
            for run, s in enumerate(searches):
                gi, sid, F, tk, bfit, bcost, bgates, flops, mean = ref[run][0][gen]
                last = ctx.last_generation(run)
                assert np.array_equal(last["gate_idx"], gi)
                assert np.array_equal(last["seg_id"], sid)
                assert np.array_equal(last["fitness"], F)
                k = max(s.topk, 1)
                assert [t[0] for t in last["topk"][:k]] == list(tk[:k])
                r = reps[run]
                assert r["generation"] == gen + 1
                assert r["best_fitness"] == bfit and r["best_cost"] == bcost
                assert bytes(r["best_gates"]) == bgates[:s.L]
                assert r["useful_flops"] == flops
                assert abs(r["mean_fitness"] - mean) <= 1e-12
        for run in range(len(searches)):
            c, b, bf = ctx.get_state(run)
            assert state_equal(c, ref[run][1]) and state_equal(b, ref[run][2])
            assert state_equal(bf, ref[run][3])


@pytest.mark.parametrize("calls", [[5, 0], [3, 2], [1, 1, 1, 1]])
def test_pipelined_generations_fp64_bit_exact(qe, torch, calls):
    """Generations enqueued without reports rank the previous generation while
    the next one runs; the reports after draining equal the oracle's."""
    searches = W.config(2, precision=W.PREC_FP64, P=200)
    gens = sum(calls)
    ref = _oracle_run(searches, gens)
    with qe.Context(searches) as ctx:
        for n in calls[:-1]:
            ctx.step_raw(n, None)
        reps = ctx.step(calls[-1])
        for run, s in enumerate(searches):
            gi, sid, F, tk, bfit, bcost, bgates, flops, mean = ref[run][0][gens - 1]
            last = ctx.last_generation(run)
            assert np.array_equal(last["gate_idx"], gi) and np.array_equal(last["fitness"], F)
            assert [t[0] for t in last["topk"]] == list(tk[:s.topk])
            r = reps[run]
            assert r["generation"] == gens
            assert r["best_fitness"] == bfit and r["best_cost"] == bcost
            assert bytes(r["best_gates"]) == bgates[:s.L]
            c, b, bf = ctx.get_state(run)
            assert state_equal(c, ref[run][1]) and state_equal(bf, ref[run][3])


def test_step_fp32_each_stage_matches(qe, torch):
    """binary32 generations: the sample is bit-exact for the state the step
    started from, fitness within its bound, the rescored top-k bit-exact, and
    the update bit-exact given the step's own binary32 fitness."""
    searches = W.config(2, precision=W.PREC_FP32, P=512)
    searches.append(W.Search(5, 24, 200, NCV | HT, W.cknot(5), seed=11, topk=16))
    searches.append(W.Search(4, 9, 77, NCV | HT, W.random_perm(np.random.default_rng(1), 4),
                             seed=12, topk=8, cost_weight=0.05))
    probs = [oracle_problem(s, r) for r, s in enumerate(searches)]
    with qe.Context(searches) as ctx:
        for gen in range(6):
            before = [ctx.get_state(r) for r in range(len(searches))]
            ctx.step(1)
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


def test_uneven_batch_step(qe, torch):
    """Searches of 3, 4 and 5 qubits with uneven L and P in one context."""
    rng = np.random.default_rng(2)
    searches = []
    for run in range(9):
        n = 3 + run % 3
        searches.append(W.Search(n, int(rng.integers(8, 65)), int(rng.integers(40, 300)),
                                 NCV | HT, W.random_perm(rng, n), seed=2, topk=8))
    probs = [oracle_problem(s, r) for r, s in enumerate(searches)]
    with qe.Context(searches) as ctx:
        for gen in range(3):
            before = [ctx.get_state(r) for r in range(len(searches))]
            ctx.step(1)
            for run, s in enumerate(searches):
                last = ctx.last_generation(run)
                gi, sid = oracle.sample(probs[run], before[run][0], gen)
                assert np.array_equal(last["gate_idx"], gi)
                F, C = oracle.eval_circuits(probs[run], gi)
                assert_fp32_fitness(last["fitness"], F, s, C)
                order = oracle.topk(F, C, s.topk)
                assert [t[0] for t in last["topk"]] == list(order)


def test_degenerate_searches(qe, torch):
    searches = [W.Search(1, 1, 1, HT, [1, 0], seed=1, precision=W.PREC_FP64, topk=1),
                W.Search(2, 1, 3, NCV, [0, 1, 3, 2], seed=2, precision=W.PREC_FP64, topk=3,
                         p_mutation=1.0),
                W.Search(5, 64, 1, NCV | HT | ID, W.cknot(5), seed=3, precision=W.PREC_FP64)]
    ref = _oracle_run(searches, 5)
    with qe.Context(searches) as ctx:
        ctx.step(5)
        for run in range(len(searches)):
            c, b, bf = ctx.get_state(run)
            assert state_equal(c, ref[run][1]) and state_equal(bf, ref[run][3])


@pytest.mark.parametrize("kind,lam", [(W.FIT_PROB, 0.0), (W.FIT_TRACE, 0.2), (W.FIT_PROB, 0.1)])
def test_step_fitness_kinds_and_cost(qe, torch, kind, lam):
    """Whole generations with the probability reading of the fitness and with
    the gate-cost penalty: binary64 trajectories bit-exact (ranking, record,
    state), and binary32 generations with their top-k bit-exact."""
    s64 = [W.Search(3, 12, 300, NCV | HT | ID, W.peres(), seed=31, precision=W.PREC_FP64,
                    topk=9, fitness_kind=kind, cost_weight=lam),
           W.Search(4, 10, 120, NCV | HT, W.cknot(4), seed=32, precision=W.PREC_FP64,
                    topk=5, fitness_kind=kind, cost_weight=lam)]
    ref = _oracle_run(s64, 6)
    with qe.Context(s64) as ctx:
        for gen in range(6):
            reps = ctx.step(1)
            for run, s in enumerate(s64):
                gi, sid, F, tk, bfit, bcost, bgates, flops, mean = ref[run][0][gen]
                last = ctx.last_generation(run)
                assert np.array_equal(last["gate_idx"], gi) and np.array_equal(last["fitness"], F)
                assert [t[0] for t in last["topk"]] == list(tk[:s.topk])
                assert reps[run]["best_fitness"] == bfit and reps[run]["best_cost"] == bcost
        for run in range(len(s64)):
            c, b, bf = ctx.get_state(run)
            assert state_equal(c, ref[run][1]) and state_equal(bf, ref[run][3])
    s32 = [W.Search(3, 16, 700, NCV | HT | ID, W.fredkin(), seed=33, topk=16, fitness_kind=kind,
                    cost_weight=lam),
           W.Search(5, 20, 90, NCV | HT, W.cknot(5), seed=34, topk=6, fitness_kind=kind,
                    cost_weight=lam)]
    probs = [oracle_problem(s, r) for r, s in enumerate(s32)]
    with qe.Context(s32) as ctx:
        for gen in range(3):
            before = [ctx.get_state(r) for r in range(len(s32))]
            ctx.step_raw(1, None)
            for run, s in enumerate(s32):
                last = ctx.last_generation(run)
                gi, _ = oracle.sample(probs[run], before[run][0].copy(), gen)
                assert np.array_equal(last["gate_idx"], gi)
                F, C = oracle.eval_circuits(probs[run], gi)
                assert_fp32_fitness(last["fitness"], F, s, C)
                order = oracle.topk(F, C, s.topk)
                assert [t[0] for t in last["topk"]] == list(order)
                assert [t[2] for t in last["topk"]] == list(F[order])
