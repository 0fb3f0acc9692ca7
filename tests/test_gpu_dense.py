"""Dense target unitaries (Eq. (11) with a general T) on the GPU against the
oracle: binary64 fitness and trajectories bit-exact (the same order of
products and sums: each diagonal element of S^dag T over i ascending, then the
trace over j ascending), binary32 within its bound; a permutation matrix given
as a dense target reproduces the permutation search."""
import numpy as np
import pytest

import oracle
from gpu_common import assert_fp32_fitness, oracle_problem, state_equal
from paper_1809_11134_gb300 import workloads as W

pytestmark = pytest.mark.gpu

DISC = W.LIB_NCV | W.LIB_HT


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


def haar(rng, N):
    q, r = np.linalg.qr(rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N)))
    return q * (np.diag(r) / np.abs(np.diag(r)))


def near_target(rng, n, lib, L):
    """a reachable circuit's unitary times a small random perturbation, so that
    fitness values spread over [0, 1] instead of sitting near 0"""
    g = rng.integers(0, oracle.num_gates(n, lib), L).astype(np.uint8)
    re, im = oracle.compose(n, lib, g)
    return (re + 1j * im) @ haar(rng, 1 << n) if rng.random() < 0.5 else re + 1j * im


@pytest.mark.parametrize("n,L", [(1, 4), (2, 7), (3, 16), (4, 20), (5, 33), (5, 64)])
def test_eval_bit_exact_fp64_and_within_bound_fp32(qe, torch, n, L):
    rng = np.random.default_rng(n * 100 + L)
    T = near_target(rng, n, DISC, L)
    nc = 300
    s64 = W.Search(n, L, nc, DISC, W.cknot(n), precision=W.PREC_FP64, cost_weight=0.1, target=T)
    s32 = W.Search(n, L, nc, DISC, W.cknot(n), precision=W.PREC_FP32, target=T)
    gates = rng.integers(0, oracle.num_gates(n, DISC), (nc, L)).astype(np.uint8)
    F, C = oracle.eval_circuits(oracle_problem(s64, 0), gates)
    F32ref, _ = oracle.eval_circuits(oracle_problem(s32, 1), gates)
    g = torch.from_numpy(gates).cuda()
    with qe.Context([s64, s32]) as ctx:
        f64 = torch.zeros(nc, dtype=torch.float64, device="cuda")
        ctx.eval(0, g, f64)
        assert np.array_equal(f64.cpu().numpy(), F)
        f32 = torch.zeros(nc, dtype=torch.float32, device="cuda")
        ctx.eval(1, g, f32)
        assert_fp32_fitness(f32.cpu().numpy().astype(np.float64), F32ref, s32)


@pytest.mark.parametrize("n", [2, 3, 4, 5])
def test_permutation_matrix_as_dense_target(qe, torch, n):
    """binary64: identical fitness to the permutation path on the same circuits."""
    rng = np.random.default_rng(n)
    N = 1 << n
    perm = [int(x) for x in rng.permutation(N)]
    T = np.zeros((N, N))
    T[perm, np.arange(N)] = 1.0
    sp = W.Search(n, 12, 200, DISC, perm, precision=W.PREC_FP64)
    sd = W.Search(n, 12, 200, DISC, W.cknot(n), precision=W.PREC_FP64, target=T)
    gates = torch.from_numpy(rng.integers(0, oracle.num_gates(n, DISC), (200, 12))
                             .astype(np.uint8)).cuda()
    with qe.Context([sp, sd]) as ctx:
        a = torch.zeros(200, dtype=torch.float64, device="cuda")
        b = torch.zeros(200, dtype=torch.float64, device="cuda")
        ctx.eval(0, gates, a)
        ctx.eval(1, gates, b)
    assert np.array_equal(a.cpu().numpy(), b.cpu().numpy())


def _oracle_run(searches, gens):
    out = []
    for run, s in enumerate(searches):
        p = oracle_problem(s, run)
        cur, best, bf = oracle.init_state(p)
        rep = oracle.new_report()
        hist = []
        for gen in range(gens):
            gi, sid, F, cost, tk = oracle.step(p, cur, best, bf, gen, max(s.topk, 1), rep)
            hist.append((gi, F, tk, rep.best_fitness, rep.best_cost, rep.useful_flops))
        out.append((hist, cur, best, bf, p))
    return out


def test_trajectory_fp64_bit_exact(qe, torch):
    rng = np.random.default_rng(7)
    searches = [W.Search(3, 16, 200, DISC | W.LIB_IDENTITY, W.cknot(3), seed=1,
                         precision=W.PREC_FP64, topk=5, target=near_target(rng, 3, DISC, 6)),
                W.Search(3, 12, 150, DISC, W.peres(), seed=2, precision=W.PREC_FP64, topk=4),
                W.Search(2, 6, 64, W.LIB_ISING, W.cknot(2), seed=3, precision=W.PREC_FP64,
                         topk=3, target=haar(rng, 4)),
                W.Search(4, 10, 90, DISC, W.cknot(4), seed=4, precision=W.PREC_FP64, topk=2,
                         target=haar(rng, 16), shots=3)]
    gens = 8
    ref = _oracle_run(searches, gens)
    with qe.Context(searches) as ctx:
        for gen in range(gens):
            reps = ctx.step(1)
            for run, s in enumerate(searches):
                gi, F, tk, bfit, bcost, flops = ref[run][0][gen]
                last = ctx.last_generation(run)
                assert np.array_equal(last["gate_idx"], gi), (gen, run)
                assert np.array_equal(last["fitness"], F), (gen, run)
                assert [t[0] for t in last["topk"]] == list(tk[:s.topk])
                assert reps[run]["best_fitness"] == bfit and reps[run]["best_cost"] == bcost
                assert reps[run]["useful_flops"] == flops
        for run in range(len(searches)):
            c, b, bf = ctx.get_state(run)
            assert state_equal(c, ref[run][1]) and state_equal(b, ref[run][2])


def test_fp32_steps_rank_exactly(qe, torch):
    """binary32 dense searches: fitness within the widened bound and the binary64
    top-k exact (the guard band covers the dense score's rounding)."""
    rng = np.random.default_rng(9)
    searches = [W.Search(3, 16, 2000, DISC | W.LIB_IDENTITY, W.cknot(3), seed=5, topk=16,
                         target=near_target(rng, 3, DISC, 8)),
                W.Search(5, 24, 300, DISC, W.cknot(5), seed=6, topk=8,
                         target=near_target(rng, 5, DISC, 10))]
    probs = [oracle_problem(s, r) for r, s in enumerate(searches)]
    with qe.Context(searches) as ctx:
        for gen in range(3):
            before = [ctx.get_state(r) for r in range(len(searches))]
            ctx.step(1)
            for run, s in enumerate(searches):
                cur = before[run][0].copy()
                gi, sid = oracle.sample(probs[run], cur, gen)
                F, C = oracle.eval_circuits(probs[run], gi)
                last = ctx.last_generation(run)
                assert np.array_equal(last["gate_idx"], gi)
                assert_fp32_fitness(last["fitness"], F, s, C)
                order = oracle.topk(F, C, s.topk)
                assert [t[0] for t in last["topk"]] == list(order)
                assert [t[2] for t in last["topk"]] == list(F[order])


def test_target_validation_and_checkpoint(qe, torch, tmp_path):
    rng = np.random.default_rng(11)
    s = W.Search(3, 8, 64, DISC, W.cknot(3), seed=1, precision=W.PREC_FP64)
    sp = W.Search(3, 8, 64, DISC, W.cknot(3), seed=1, fitness_kind=W.FIT_PROB)
    T = haar(rng, 8)
    with qe.Context([s, sp]) as ctx:
        with pytest.raises(qe.QeError) as e:
            ctx.set_target(0, T * 1.01)  # not unitary
        assert e.value.status == qe.QE_EINVAL
        bad = T.copy()
        bad[2, 3] = np.nan
        with pytest.raises(qe.QeError):
            ctx.set_target(0, bad)
        with pytest.raises(qe.QeError) as e:
            ctx.set_target(1, T)
        assert e.value.status == qe.QE_EUNSUPPORTED
        ctx.set_target(0, T)
        ctx.step(2)
        path = str(tmp_path / "dense.qeckpt")
        ctx.save(path)
        reps_a = ctx.step(3)
    with qe.Context.from_checkpoint(path) as ctx:
        assert ctx.step(3) == reps_a  # the target travels with the checkpoint
    with qe.Context([s, sp]) as ctx:
        ctx.set_target(0, T)
        ctx.set_target(0, None)  # back to the permutation
        g = torch.from_numpy(rng.integers(0, oracle.num_gates(3, DISC), (64, 8))
                             .astype(np.uint8)).cuda()
        f = torch.zeros(64, dtype=torch.float64, device="cuda")
        ctx.eval(0, g, f)
        F, _ = oracle.eval_circuits(oracle_problem(s, 0), g.cpu().numpy())
        assert np.array_equal(f.cpu().numpy(), F)


@pytest.mark.parametrize("n,L", [(3, 16), (5, 24), (5, 64)])
def test_ising_dense_fp64_bit_exact_and_fp32_within_bound(qe, torch, n, L):
    """The paper's Ising library against a dense target: the 5-qubit binary32
    kernel defers its diagonal gates (R_z, J) and applies their phases when a
    rotation next reads the rows, or before the score; binary64 applies every
    gate in order and matches the oracle bit for bit."""
    rng = np.random.default_rng(700 + n * 10 + L)
    G = oracle.num_gates(n, W.LIB_ISING)
    g0 = rng.integers(0, G, L).astype(np.uint8)
    th0 = rng.uniform(0, 2 * np.pi, L)
    a0 = np.stack([np.cos(th0), np.sin(th0)], -1).astype(np.float32)
    re, im = oracle.compose(n, W.LIB_ISING, g0, a0)
    T = re + 1j * im
    nc = 300
    s64 = W.Search(n, L, nc, W.LIB_ISING, W.cknot(n), precision=W.PREC_FP64, target=T)
    s32 = W.Search(n, L, nc, W.LIB_ISING, W.cknot(n), precision=W.PREC_FP32, target=T)
    gates = rng.integers(0, G, (nc, L)).astype(np.uint8)
    gates[0] = g0  # one circuit that reaches the target exactly
    th = rng.uniform(0, 2 * np.pi, (nc, L))
    amps = np.stack([np.cos(th), np.sin(th)], -1).astype(np.float32)
    amps[0] = a0
    F, _ = oracle.eval_circuits(oracle_problem(s64, 0), gates, amps)
    assert F[0] > 1 - 1e-6
    g = torch.from_numpy(gates).cuda()
    a = torch.from_numpy(amps).cuda()
    with qe.Context([s64, s32]) as ctx:
        f64 = torch.zeros(nc, dtype=torch.float64, device="cuda")
        ctx.eval(0, g, f64, amps=a)
        assert np.array_equal(f64.cpu().numpy(), F)
        f32 = torch.zeros(nc, dtype=torch.float32, device="cuda")
        ctx.eval(1, g, f32, amps=a)
        assert_fp32_fitness(f32.cpu().numpy().astype(np.float64), F, s32)
