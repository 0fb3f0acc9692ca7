"""The paper's Ising library (R_x/R_y/R_z on each wire, interaction templates
J_ij on each pair) on the GPU against the oracle: binary64 fitness, unitaries
and whole trajectories bit-exact (the angles enter through half-angle square
roots, correctly rounded on both sides), binary32 within its bound."""
import numpy as np
import pytest

import oracle
from gpu_common import assert_fp32_fitness, oracle_problem, state_equal
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


def S(n, L, P, perm=None, **kw):
    return W.Search(n, L, P, ISING, perm if perm is not None else W.cknot(n), **kw)


def _G(s):
    return oracle.num_gates(s.n, s.library)


def random_amps(rng, shape):
    """qubit amplitudes (cos t, sin t), t uniform, with exact quadrant angles mixed in"""
    t = rng.uniform(0, 2 * np.pi, shape)
    a = np.stack([np.cos(t), np.sin(t)], -1).astype(np.float32)
    q = rng.random(shape) < 0.2
    quad = np.array([[1, 0], [0, 1], [-1, 0], [0, -1]], np.float32)
    a[q] = quad[rng.integers(0, 4, q.sum())]
    return a


@pytest.mark.parametrize("n,L,kind", [(1, 5, W.FIT_TRACE), (2, 9, W.FIT_TRACE), (3, 16, W.FIT_PROB),
                                      (4, 20, W.FIT_TRACE), (5, 33, W.FIT_TRACE),
                                      (5, 64, W.FIT_PROB)])
def test_eval_bit_exact_fp64_and_within_bound_fp32(qe, torch, n, L, kind):
    rng = np.random.default_rng(10 * n + L)
    nc = 300
    s64 = S(n, L, nc, seed=n, precision=W.PREC_FP64, fitness_kind=kind, cost_weight=0.1)
    s32 = S(n, L, nc, seed=n, precision=W.PREC_FP32, fitness_kind=kind, cost_weight=0.1)
    gates = rng.integers(0, _G(s64), (nc, L)).astype(np.uint8)
    amps = random_amps(rng, (nc, L))
    F, C = oracle.eval_circuits(oracle_problem(s64, 0), gates, amps)
    g = torch.from_numpy(gates).cuda()
    a = torch.from_numpy(amps).cuda()
    with qe.Context([s64, s32]) as ctx:
        f64 = torch.zeros(nc, dtype=torch.float64, device="cuda")
        cost = torch.zeros(nc, dtype=torch.int32, device="cuda")
        ctx.eval(0, g, f64, cost=cost, amps=a)
        assert np.array_equal(f64.cpu().numpy(), F)
        assert np.array_equal(cost.cpu().numpy(), C.astype(np.int32))
        f32 = torch.zeros(nc, dtype=torch.float32, device="cuda")
        ctx.eval(1, g, f32, amps=a)
        assert_fp32_fitness(f32.cpu().numpy().astype(np.float64), F, s32, C)


@pytest.mark.parametrize("n,L", [(2, 7), (3, 12), (4, 10), (5, 12)])
def test_compose_matches_oracle(qe, torch, n, L):
    rng = np.random.default_rng(n)
    nc = 24
    s64 = S(n, L, nc, precision=W.PREC_FP64)
    s32 = S(n, L, nc, precision=W.PREC_FP32)
    gates = rng.integers(0, _G(s64), (nc, L)).astype(np.uint8)
    amps = random_amps(rng, (nc, L))
    N = 1 << n
    g = torch.from_numpy(gates).cuda()
    a = torch.from_numpy(amps).cuda()
    with qe.Context([s64, s32]) as ctx:
        u64 = torch.zeros(nc * N * N * 2, dtype=torch.float64, device="cuda")
        u32 = torch.zeros(nc * N * N * 2, dtype=torch.float32, device="cuda")
        ctx.compose(0, g, u64, amps=a)
        ctx.compose(1, g, u32, amps=a)
    u64 = u64.cpu().numpy().reshape(nc, N, N, 2)
    u32 = u32.cpu().numpy().reshape(nc, N, N, 2)
    for c in range(nc):
        re, im = oracle.compose(n, ISING, gates[c], amps[c])
        assert np.array_equal(u64[c, ..., 0], re) and np.array_equal(u64[c, ..., 1], im)
        assert np.abs(u32[c, ..., 0] - re).max() < 1e-5 and np.abs(u32[c, ..., 1] - im).max() < 1e-5


def test_cnot_from_ising_gates(qe, torch):
    """The seven-gate Ising CNOT of the oracle pins scores 1 on the GPU in both precisions."""
    gates = np.array([[1, 0, 2, 5, 6, 1, 0]], np.uint8)
    half, pi, three = (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0)
    amps = np.array([[half, pi, half, half, three, half, pi]], np.float32)
    s64 = S(2, 7, 1, precision=W.PREC_FP64)
    s32 = S(2, 7, 1, precision=W.PREC_FP32)
    F, _ = oracle.eval_circuits(oracle_problem(s64, 0), gates, amps)
    with qe.Context([s64, s32]) as ctx:
        f64 = torch.zeros(1, dtype=torch.float64, device="cuda")
        f32 = torch.zeros(1, dtype=torch.float32, device="cuda")
        ctx.eval(0, torch.from_numpy(gates).cuda(), f64, amps=torch.from_numpy(amps).cuda())
        ctx.eval(1, torch.from_numpy(gates).cuda(), f32, amps=torch.from_numpy(amps).cuda())
    assert f64.item() == F[0] and F[0] > 1 - 1e-7
    assert f32.item() > 1 - 1e-3


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
                         list(rep.best_amps[:2 * s.L])))
        out.append((hist, cur, best, bf))
    return out


def test_step_trajectory_fp64_bit_exact(qe, torch):
    """Searches shaped like the paper's Table 3 runs (CNOT n=2 L=3, Toffoli L=16, C3NOT,
    Peres), ten generations: circuits, fitness, top-k, record and state bit-exact."""
    searches = [S(2, 3, 64, W.cknot(2), seed=1, precision=W.PREC_FP64, topk=4),
                S(3, 16, 200, W.cknot(3), seed=2, precision=W.PREC_FP64, topk=8),
                S(4, 12, 80, W.cknot(4), seed=3, precision=W.PREC_FP64, topk=3, cost_weight=0.05),
                S(3, 10, 150, W.peres(), seed=4, precision=W.PREC_FP64, topk=5,
                  fitness_kind=W.FIT_PROB)]
    gens = 10
    ref = _oracle_run(searches, gens)
    with qe.Context(searches) as ctx:
        for gen in range(gens):
            reps = ctx.step(1)
            for run, s in enumerate(searches):
                gi, sid, F, tk, bfit, bcost, bgates, bamps = ref[run][0][gen]
                last = ctx.last_generation(run)
                assert np.array_equal(last["gate_idx"], gi), (gen, run)
                assert np.array_equal(last["seg_id"], sid)
                assert np.array_equal(last["fitness"], F), (gen, run)
                assert [t[0] for t in last["topk"]] == list(tk[:s.topk])
                assert reps[run]["best_fitness"] == bfit and reps[run]["best_cost"] == bcost
                assert bytes(reps[run]["best_gates"][:s.L]) == bgates[:s.L]
                assert reps[run]["best_amps"] == bamps  # the best circuit's angles
        for run in range(len(searches)):
            c, b, bf = ctx.get_state(run)
            assert state_equal(c, ref[run][1]) and state_equal(b, ref[run][2])
            assert state_equal(bf, ref[run][3])


def test_step_fp32_each_stage(qe, torch):
    """binary32 Ising generations beside a discrete search: the sample bit-exact, fitness
    within its bound (oracle evaluated on the oracle's sampled angles), the binary64 top-k
    exact, the update bit-exact given the step's own fitness; the discrete search is
    unaffected by sharing the context."""
    searches = [S(3, 16, 1000, W.cknot(3), seed=5, topk=16),
                S(5, 20, 120, W.cknot(5), seed=6, topk=6),
                W.Search(3, 16, 300, W.LIB_NCV | W.LIB_HT | W.LIB_IDENTITY, W.fredkin(), seed=7,
                         topk=8)]
    probs = [oracle_problem(s, r) for r, s in enumerate(searches)]
    with qe.Context(searches) as ctx:
        for gen in range(4):
            before = [ctx.get_state(r) for r in range(len(searches))]
            ctx.step_raw(1, None)
            for run, s in enumerate(searches):
                p = probs[run]
                cur, best, bf = [x.copy() for x in before[run]]
                last = ctx.last_generation(run)
                if s.library == ISING:
                    gi, sid, amps = oracle.sample(p, cur, gen, with_amps=True)
                    F, C = oracle.eval_circuits(p, gi, amps)
                else:
                    gi, sid = oracle.sample(p, cur, gen)
                    F, C = oracle.eval_circuits(p, gi)
                assert np.array_equal(last["gate_idx"], gi) and np.array_equal(last["seg_id"], sid)
                assert_fp32_fitness(last["fitness"], F, s, C)
                order = oracle.topk(F, C, s.topk)
                assert [t[0] for t in last["topk"]] == list(order)
                assert [t[2] for t in last["topk"]] == list(F[order])
                oracle.update(p, cur, best, bf, gen, sid, last["fitness"])
                c2, b2, bf2 = ctx.get_state(run)
                assert state_equal(c2, cur) and state_equal(b2, best) and state_equal(bf2, bf)


def test_ising_calls_need_angles(qe, torch):
    s = S(3, 4, 16, precision=W.PREC_FP64)
    g = torch.zeros(16 * 4, dtype=torch.uint8, device="cuda")
    f = torch.zeros(16, dtype=torch.float64, device="cuda")
    with qe.Context([s]) as ctx:
        with pytest.raises(qe.QeError):
            ctx.eval(0, g.view(16, 4), f)
        with pytest.raises(qe.QeError):
            ctx.eval_host(0, np.zeros((16, 4), np.uint8))
        ctx.step(2)  # sampling supplies the angles itself


@pytest.mark.parametrize("n,L,kind", [(3, 16, W.FIT_TRACE), (4, 20, W.FIT_TRACE),
                                      (4, 20, W.FIT_PROB), (5, 33, W.FIT_TRACE)])
def test_fp32_topk_exact_every_split_width(qe, torch, n, L, kind):
    """binary32 Ising evaluation with the binary64 top-k: the rescoring splits
    each candidate over 2 (n = 3) or 4 (n = 4, 5) warps; indices, costs and
    binary64 fitness equal the oracle's"""
    rng = np.random.default_rng(1000 + 10 * n + L + kind)
    nc = 400
    s32 = S(n, L, nc, seed=n, precision=W.PREC_FP32, fitness_kind=kind, topk=20)
    gates = rng.integers(0, _G(s32), (nc, L)).astype(np.uint8)
    amps = random_amps(rng, (nc, L))
    F, C = oracle.eval_circuits(oracle_problem(s32, 0), gates, amps)
    g = torch.from_numpy(gates).cuda()
    a = torch.from_numpy(amps).cuda()
    with qe.Context([s32]) as ctx:
        f32 = torch.zeros(nc, dtype=torch.float32, device="cuda")
        top = ctx.eval(0, g, f32, topk=True, amps=a)
    order = oracle.topk(F, C, 20)
    assert [t[0] for t in top] == list(order)
    assert [t[1] for t in top] == list(C[order])
    assert [t[2] for t in top] == list(F[order])
