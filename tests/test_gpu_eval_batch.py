"""qe_eval_host_batch (several searches' host circuits in one call) against the
CPU oracle and against qe_eval_host, through the C ABI.

Bit-exact: binary64 fitness, top-k (indices, costs, binary64 fitness) in both
arithmetics, and the binary32 fitness against qe_eval_host's (same kernels).
Within the stated bound: binary32 fitness against the oracle's binary64."""
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


def searches(prec):
    # uneven widths, lengths, populations and top-k sizes in one context
    return [W.Search(3, 16, 1000, NCV | HT | ID, W.cknot(3), seed=1, precision=prec, topk=32),
            W.Search(4, 32, 300, NCV | HT, W.cknot(4), seed=7, precision=prec, topk=64,
                     cost_weight=0.1),
            W.Search(5, 64, 130, NCV | HT, W.cknot(5), seed=9, precision=prec, topk=128),
            W.Search(2, 7, 33, NCV | ID, [0, 1, 3, 2], seed=4, precision=prec, topk=1),
            W.Search(3, 5, 4096, NCV | ID, W.peres(), seed=0, precision=prec, topk=32,
                     fitness_kind=W.FIT_PROB)]


def gates_for(s, n, rng):
    return W.random_gates(rng, n, s.L, oracle.num_gates(s.n, s.library))


def check_item(s, g, fit, top):
    if len(g) == 0:
        assert len(fit) == 0 and (top is None or top == [])
        return
    F, C = oracle.eval_circuits(oracle_problem(s, 0), g)
    if s.precision == W.PREC_FP64:
        assert np.array_equal(fit, F)
    else:
        assert_fp32_fitness(fit, F, s, C)
    if top is not None:
        k = min(max(s.topk, 1), len(g))
        order = oracle.topk(F, C, k) if len(g) else []
        assert [t[0] for t in top] == list(order)
        assert [t[1] for t in top] == list(C[order])
        assert [t[2] for t in top] == list(F[order])


@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
def test_batch_matches_oracle_and_single_calls(qe, prec):
    ss = searches(prec)
    rng = np.random.default_rng(11 + prec)
    # items out of problem order, ragged counts (one at P, one of a single circuit)
    plan = [(4, 4096), (1, 299), (0, 1000), (3, 1), (2, 77)]
    items = [(q, gates_for(ss[q], n, rng)) for q, n in plan]
    with qe.Context(ss) as ctx:
        fits, tops = ctx.eval_host_batch(items, topk=True)
        for (q, g), f, t in zip(items, fits, tops):
            check_item(ss[q], g, f, t)
            f1, t1 = ctx.eval_host(q, g, topk=True)
            assert np.array_equal(f.view(np.uint8), f1.view(np.uint8))
            assert t == t1
        # without ranking: the same fitness
        fits2 = ctx.eval_host_batch(items)
        for f, f2 in zip(fits, fits2):
            assert np.array_equal(f.view(np.uint8), f2.view(np.uint8))


def test_batch_layouts_replay_and_change(qe):
    """the captured graph is replayed while the layout repeats and rebuilt when
    it changes (other problems, counts, a larger staging area); every call is
    checked against the oracle"""
    ss = searches(W.PREC_FP32)
    rng = np.random.default_rng(5)
    plans = [[(0, 1000), (1, 300)], [(0, 1000), (1, 300)], [(1, 17)],
             [(4, 4096), (2, 130), (0, 999), (1, 300), (3, 33)], [(0, 1000), (1, 300)]]
    with qe.Context(ss) as ctx:
        for plan in plans:
            items = [(q, gates_for(ss[q], n, rng)) for q, n in plan]
            fits, tops = ctx.eval_host_batch(items, topk=True)
            for (q, g), f, t in zip(items, fits, tops):
                check_item(ss[q], g, f, t)


def test_batch_empty_items(qe):
    ss = searches(W.PREC_FP32)
    rng = np.random.default_rng(9)
    with qe.Context(ss) as ctx:
        items = [(0, gates_for(ss[0], 0, rng)), (2, gates_for(ss[2], 64, rng)),
                 (1, gates_for(ss[1], 0, rng))]
        fits, tops = ctx.eval_host_batch(items, topk=True)
        assert [len(f) for f in fits] == [0, 64, 0]
        assert tops[0] == [] and tops[2] == []
        check_item(ss[2], items[1][1], fits[1], tops[1])
        # nothing to evaluate at all
        fits, tops = ctx.eval_host_batch([(3, gates_for(ss[3], 0, rng))], topk=True)
        assert len(fits[0]) == 0 and tops == [[]]


def test_batch_rejects_bad_arguments(qe):
    ss = searches(W.PREC_FP32)
    rng = np.random.default_rng(3)
    g0 = gates_for(ss[0], 10, rng)
    with qe.Context(ss) as ctx:
        bad = [[(0, g0), (0, g0)],                               # a problem twice
               [(0, gates_for(ss[0], 1001, rng))],               # more than P circuits
               [(7, g0)]]                                        # no such problem
        for items in bad:
            with pytest.raises(qe.QeError) as e:
                ctx.eval_host_batch(items, topk=True)
            assert e.value.status == qe.QE_EINVAL
        with pytest.raises(qe.QeError) as e:
            ctx.eval_host_batch([], topk=True)
        assert e.value.status == qe.QE_EINVAL
        # the context stays usable
        fits, tops = ctx.eval_host_batch([(0, g0)], topk=True)
        check_item(ss[0], g0, fits[0], tops[0])
    mixed = [searches(W.PREC_FP32)[0], searches(W.PREC_FP64)[1]]
    with qe.Context(mixed) as ctx:
        with pytest.raises(qe.QeError) as e:
            ctx.eval_host_batch([(0, gates_for(mixed[0], 4, rng)),
                                 (1, gates_for(mixed[1], 4, rng))])
        assert e.value.status == qe.QE_EINVAL
    ising = W.Search(3, 8, 16, W.LIB_ISING, W.cknot(3), seed=1, topk=4)
    with qe.Context([ising]) as ctx:
        with pytest.raises(qe.QeError) as e:
            ctx.eval_host_batch([(0, np.zeros((4, 8), np.uint8))])
        assert e.value.status == qe.QE_EINVAL


def test_batch_invalid_gate_index_is_reported(qe):
    ss = searches(W.PREC_FP32)
    rng = np.random.default_rng(4)
    g0, g1 = gates_for(ss[0], 50, rng), gates_for(ss[1], 40, rng)
    g1[7, 3] = 250
    with qe.Context(ss) as ctx:
        with pytest.raises(qe.QeError) as e:
            ctx.eval_host_batch([(0, g0), (1, g1)], topk=True)
        assert e.value.status == qe.QE_ENUMERIC
        g1[7, 3] = 0
        fits, tops = ctx.eval_host_batch([(0, g0), (1, g1)], topk=True)
        for (q, g), f, t in zip([(0, g0), (1, g1)], fits, tops):
            check_item(ss[q], g, f, t)


def test_batch_between_generations_leaves_the_run_unchanged(qe):
    """a batch evaluation between qe_step calls (it first ranks the pending
    generation) changes nothing in the run: binary64 reports equal those of a
    run without it"""
    ss = [W.Search(3, 16, 512, NCV | HT | ID, W.cknot(3), seed=1, precision=W.PREC_FP64,
                   topk=8),
          W.Search(4, 12, 256, NCV | HT, W.cknot(4), seed=2, precision=W.PREC_FP64, topk=8)]
    rng = np.random.default_rng(8)
    with qe.Context(ss) as a, qe.Context(ss) as b:
        for gen in range(4):
            ra, rb = a.step(1), b.step(1)
            assert ra == rb
            items = [(1, gates_for(ss[1], 100, rng)), (0, gates_for(ss[0], 512, rng))]
            fits, tops = a.eval_host_batch(items, topk=True)
            for (q, g), f, t in zip(items, fits, tops):
                check_item(ss[q], g, f, t)
        assert a.step(1) == b.step(1)


def test_batch_pinned_buffers_match_pageable(qe):
    """pinned (page-locked) gate and fitness buffers give the same results as
    pageable ones, over repeated calls, new contents, other pinned buffers and
    a switch back"""
    import ctypes as C
    import torch
    ss = searches(W.PREC_FP32)
    rng = np.random.default_rng(21)
    plan = [(0, 1000), (1, 300), (3, 33)]
    probs = (C.c_uint32 * len(plan))(*[q for q, _ in plan])
    counts = (C.c_uint32 * len(plan))(*[n for _, n in plan])
    ks = [min(max(ss[q].topk, 1), n) for q, n in plan]
    n_tot = sum(n for _, n in plan)

    def pinned_call(ctx, items, hg, hf):
        flat = np.concatenate([g.ravel() for _, g in items])
        hg[:flat.size].copy_(torch.from_numpy(flat))
        tops = (qe.qe_ranked * sum(ks))()
        ctx.eval_host_batch_ptr(probs, counts, hg.data_ptr(), hf.data_ptr(), tops)
        fits, out, fo, ko = [], [], 0, 0
        for (q, n), k in zip(plan, ks):
            fits.append(hf[fo:fo + n].numpy().copy())
            out.append([(t.circuit, t.cost, t.fitness) for t in tops[ko:ko + k]])
            fo += n
            ko += k
        return fits, out

    with qe.Context(ss) as ctx:
        bufs = [(torch.zeros(sum(n * ss[q].L for q, n in plan), dtype=torch.uint8).pin_memory(),
                 torch.zeros(n_tot, dtype=torch.float32).pin_memory()) for _ in range(2)]
        for hg, hf in (bufs[0], bufs[0], bufs[1], bufs[0]):
            items = [(q, gates_for(ss[q], n, rng)) for q, n in plan]
            fits, tops = pinned_call(ctx, items, hg, hf)
            fits2, tops2 = ctx.eval_host_batch(items, topk=True)  # pageable
            for (q, g), f, t, f2, t2 in zip(items, fits, tops, fits2, tops2):
                assert np.array_equal(f.view(np.uint8), f2.view(np.uint8))
                assert t == t2
                check_item(ss[q], g, f, t)


@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
def test_batch_with_dense_targets_and_shots(qe, prec):
    """searches against dense target unitaries (Eq. (11) with a general T) and
    a search measured K times share a batch with permutation searches; the
    evaluation of given circuits does not depend on K"""
    from test_gpu_dense import near_target
    rng = np.random.default_rng(31 + prec)
    lib = NCV | HT
    ss = [W.Search(3, 16, 500, lib, W.cknot(3), seed=1, precision=prec, topk=8,
                   target=near_target(rng, 3, lib, 6)),
          W.Search(4, 20, 300, lib, W.cknot(4), seed=2, precision=prec, topk=16),
          W.Search(5, 33, 120, lib, W.cknot(5), seed=3, precision=prec, topk=4,
                   target=near_target(rng, 5, lib, 8)),
          W.Search(3, 12, 256, lib | ID, W.peres(), seed=4, precision=prec, topk=8, shots=5)]
    plan = [(2, 120), (0, 499), (3, 256), (1, 300)]
    items = [(q, gates_for(ss[q], n, rng)) for q, n in plan]
    with qe.Context(ss) as ctx:
        fits, tops = ctx.eval_host_batch(items, topk=True)
        for (q, g), f, t in zip(items, fits, tops):
            check_item(ss[q], g, f, t)


def test_batch_benchmark_workload_full_size(qe):
    """the end-to-end workload bench.py times: one call with all three 3-qubit
    searches of the benchmark set at P = 4096, every circuit against the
    oracle, twice in a row (the second call replays the captured graph)"""
    ss = W.config(2)
    rng = np.random.default_rng(2)
    with qe.Context(ss) as ctx:
        for _ in range(2):
            items = [(q, gates_for(s, s.P, rng)) for q, s in enumerate(ss)]
            fits, tops = ctx.eval_host_batch(items, topk=True)
            for (q, g), f, t in zip(items, fits, tops):
                assert len(f) == 4096 and len(t) == 32
                check_item(ss[q], g, f, t)


@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
def test_batch_many_searches_of_every_width(qe, prec):
    """64 small searches of 1 to 5 qubits (shadow lanes at 1 and 2 qubits,
    every rescoring width, ragged populations and top-k sizes) in one batch,
    items in a shuffled order, every circuit against the oracle"""
    rng = np.random.default_rng(64 + prec)
    ss, plan = [], []
    for q in range(64):
        n = 1 + q % 5
        lib = HT if n == 1 else ((NCV | HT) if q % 3 else (NCV | ID))
        L = int(rng.integers(1, 40))
        P = int(rng.integers(1, 200))
        perm = [int(v) for v in rng.permutation(1 << n)]
        ss.append(W.Search(n, L, P, lib, perm, seed=q, precision=prec,
                           topk=int(rng.integers(0, min(12, P) + 1))))
        plan.append((q, int(rng.integers(0, P + 1))))
    order = rng.permutation(64)
    items = [(plan[i][0], gates_for(ss[plan[i][0]], plan[i][1], rng)) for i in order]
    with qe.Context(ss) as ctx:
        fits, tops = ctx.eval_host_batch(items, topk=True)
        for (q, g), f, t in zip(items, fits, tops):
            assert len(f) == len(g)
            check_item(ss[q], g, f, t)


class _Call:
    """Pinned buffers of one asynchronous batched call (items = [(prob, gates)])."""

    def __init__(self, qe, ss, items):
        import ctypes as C
        import torch
        self.items = items
        self.ns = [len(g) for _, g in items]
        self.ks = [min(max(ss[q].topk, 1), n) for (q, _), n in zip(items, self.ns)]
        flat = np.concatenate([g.ravel() for _, g in items])
        self.hg = torch.from_numpy(flat).pin_memory()
        fp64 = ss[items[0][0]].precision == W.PREC_FP64
        self.hf = torch.full((max(sum(self.ns), 1),), -7.0,
                             dtype=torch.float64 if fp64 else torch.float32).pin_memory()
        self.tops = (qe.qe_ranked * max(sum(self.ks), 1))()
        self.probs = (C.c_uint32 * len(items))(*[q for q, _ in items])
        self.counts = (C.c_uint32 * len(items))(*self.ns)

    def submit(self, ctx):
        return ctx.eval_host_batch_async_ptr(self.probs, self.counts, self.hg.data_ptr(),
                                             self.hf.data_ptr(), self.tops)

    def results(self):
        fits, tops, fo, ko = [], [], 0, 0
        for n, k in zip(self.ns, self.ks):
            fits.append(self.hf[fo:fo + n].numpy().copy())
            tops.append([(t.circuit, t.cost, t.fitness) for t in self.tops[ko:ko + k]])
            fo += n
            ko += k
        return fits, tops


@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
def test_async_calls_in_flight_match_the_oracle(qe, prec):
    """asynchronous calls in flight together (every slot busy, different
    layouts sharing searches, waited for in several orders, slots reused with
    new layouts and with old ones), every result against the oracle and
    against the synchronous call"""
    ss = searches(prec)
    rng = np.random.default_rng(41 + prec)
    plans = [[(0, 1000), (1, 300)], [(4, 4096), (2, 130), (3, 33)], [(1, 17), (0, 999)],
             [(0, 1000), (1, 300)], [(2, 77)], [(4, 4095), (0, 5)], [(0, 1000), (2, 130)],
             [(3, 33), (1, 300), (4, 4096)], [(0, 998)]]
    calls = [_Call(qe, ss, [(q, gates_for(ss[q], n, rng)) for q, n in plan]) for plan in plans]
    S = qe.QE_BATCH_SLOTS
    assert S >= 2
    with qe.Context(ss) as ctx:
        for r, start in enumerate(range(0, len(calls), S)):
            ts = [c.submit(ctx) for c in calls[start:start + S]]
            assert len(set(ts)) == len(ts)
            order = ts if r % 3 == 0 else (ts[::-1] if r % 3 == 1 else ts[1:] + ts[:1])
            for t in order:
                ctx.eval_host_batch_wait(t)
        for c in calls:
            fits, tops = c.results()
            for (q, g), f, t in zip(c.items, fits, tops):
                check_item(ss[q], g, f, t)
            fits2, tops2 = ctx.eval_host_batch(c.items, topk=True)
            for f, t, f2, t2 in zip(fits, tops, fits2, tops2):
                assert np.array_equal(f.view(np.uint8), f2.view(np.uint8))
                assert t == t2


def test_async_slot_and_ticket_errors(qe):
    """one call more than there are slots is QE_ESTATE, the ticket of a call
    already waited for or never issued is QE_EINVAL; the calls in flight are
    not disturbed and the context stays usable"""
    ss = searches(W.PREC_FP32)
    rng = np.random.default_rng(43)
    S = qe.QE_BATCH_SLOTS
    sizes = [(q % 5, min(ss[q % 5].P, 20 + 37 * q)) for q in range(S + 1)]
    calls = [_Call(qe, ss, [(q, gates_for(ss[q], n, rng))]) for q, n in sizes]
    with qe.Context(ss) as ctx:
        ts = [calls[i].submit(ctx) for i in range(S)]
        with pytest.raises(qe.QeError) as e:
            calls[S].submit(ctx)
        assert e.value.status == qe.QE_ESTATE
        with pytest.raises(qe.QeError) as e:
            ctx.eval_host_batch(calls[S].items, topk=True)
        assert e.value.status == qe.QE_ESTATE
        with pytest.raises(qe.QeError) as e:
            ctx.eval_host_batch_wait(max(ts) + 100)
        assert e.value.status == qe.QE_EINVAL
        ctx.eval_host_batch_wait(ts[1])
        with pytest.raises(qe.QeError) as e:
            ctx.eval_host_batch_wait(ts[1])
        assert e.value.status == qe.QE_EINVAL
        tl = calls[S].submit(ctx)
        for t in [ts[0]] + ts[2:] + [tl]:
            ctx.eval_host_batch_wait(t)
        for c in calls:
            fits, tops = c.results()
            for (q, g), f, t in zip(c.items, fits, tops):
                check_item(ss[q], g, f, t)


def test_async_invalid_gate_reported_with_or_without_ranking(qe):
    """an invalid gate index gives NaN fitness for its circuit and QE_ENUMERIC
    from the wait, with and without top-k lists; the other call in flight and
    the slot's next call are exact"""
    import torch
    ss = searches(W.PREC_FP32)
    rng = np.random.default_rng(47)
    g0 = gates_for(ss[0], 200, rng)
    g0[13, 2] = 200
    bad = _Call(qe, ss, [(0, g0)])
    good = _Call(qe, ss, [(1, gates_for(ss[1], 300, rng))])
    with qe.Context(ss) as ctx:
        for ranked in (True, False):
            tops = bad.tops if ranked else None
            tb = ctx.eval_host_batch_async_ptr(bad.probs, bad.counts, bad.hg.data_ptr(),
                                               bad.hf.data_ptr(), tops)
            tg = good.submit(ctx)
            with pytest.raises(qe.QeError) as e:
                ctx.eval_host_batch_wait(tb)
            assert e.value.status == qe.QE_ENUMERIC
            ctx.eval_host_batch_wait(tg)
            f = bad.hf.numpy()
            assert np.isnan(f[13]) and np.isfinite(np.delete(f[:200], 13)).all()
            fits, tops2 = good.results()
            check_item(ss[1], good.items[0][1], fits[0], tops2[0])
        # the error word was cleared: the slot's next call is clean
        g0[13, 2] = 0
        bad.hg.copy_(torch.from_numpy(g0.ravel()))
        ctx.eval_host_batch_wait(bad.submit(ctx))
        fits, tops = bad.results()
        check_item(ss[0], g0, fits[0], tops[0])


def test_async_call_across_generations_leaves_the_run_unchanged(qe):
    """a call in flight while qe_step runs generations (binary64): its results
    are exact and the run's reports equal those of a run without it"""
    ss = [W.Search(3, 16, 512, NCV | HT | ID, W.cknot(3), seed=1, precision=W.PREC_FP64,
                   topk=8),
          W.Search(4, 12, 256, NCV | HT, W.cknot(4), seed=2, precision=W.PREC_FP64, topk=8)]
    rng = np.random.default_rng(53)
    with qe.Context(ss) as a, qe.Context(ss) as b:
        for gen in range(3):
            c = _Call(qe, ss, [(1, gates_for(ss[1], 100, rng)), (0, gates_for(ss[0], 512, rng))])
            t = c.submit(a)
            ra, rb = a.step(1), b.step(1)
            assert ra == rb
            a.eval_host_batch_wait(t)
            fits, tops = c.results()
            for (q, g), f, tk in zip(c.items, fits, tops):
                check_item(ss[q], g, f, tk)
        assert a.step(1) == b.step(1)


def test_async_handles_from_numpy_equal_the_synchronous_call(qe):
    """Context.eval_host_batch_async on pageable numpy arrays: as many calls in
    flight as there are slots, waited for out of order, each equal to the
    synchronous call and checked against the oracle"""
    ss = searches(W.PREC_FP32)
    rng = np.random.default_rng(61)
    S = qe.QE_BATCH_SLOTS
    plans = [[(q % 5, min(ss[q % 5].P, 50 + 90 * q)), ((q + 2) % 5, ss[(q + 2) % 5].P)]
             for q in range(S)]
    all_items = [[(q, gates_for(ss[q], n, rng)) for q, n in plan] for plan in plans]
    with qe.Context(ss) as ctx:
        handles = [ctx.eval_host_batch_async(items, topk=True) for items in all_items]
        results = [None] * S
        for i in list(range(1, S)) + [0]:
            results[i] = handles[i].wait()
        for items, (fits, tops) in zip(all_items, results):
            fits2, tops2 = ctx.eval_host_batch(items, topk=True)
            for (q, g), f, t, f2, t2 in zip(items, fits, tops, fits2, tops2):
                assert np.array_equal(f.view(np.uint8), f2.view(np.uint8))
                assert t == t2
                check_item(ss[q], g, f, t)


def test_batch_follows_a_changed_target(qe):
    """a layout captured against the permutation target is recaptured after
    qe_set_target (dense target), and again when the permutation comes back;
    a call in flight when the target changes finishes with the old one"""
    import dataclasses
    from test_gpu_dense import near_target
    rng = np.random.default_rng(71)
    s = W.Search(3, 16, 500, NCV | HT, W.cknot(3), seed=1, precision=W.PREC_FP32, topk=8)
    dense = dataclasses.replace(s, target=near_target(rng, 3, NCV | HT, 6))
    items = [(0, gates_for(s, 500, rng))]
    g = items[0][1]
    with qe.Context([s]) as ctx:
        fits, tops = ctx.eval_host_batch(items, topk=True)
        check_item(s, g, fits[0], tops[0])
        ctx.set_target(0, dense.target)
        fits, tops = ctx.eval_host_batch(items, topk=True)
        check_item(dense, g, fits[0], tops[0])
        call = ctx.eval_host_batch_async(items, topk=True)
        ctx.set_target(0, None)  # waits for the call in flight
        fits, tops = call.wait()
        check_item(dense, g, fits[0], tops[0])
        fits, tops = ctx.eval_host_batch(items, topk=True)
        check_item(s, g, fits[0], tops[0])


@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
def test_async_pipeline_rotating_pinned_buffers(qe, prec):
    """the pattern of a pipelined caller: fewer calls in flight than slots, a
    ring of page-locked buffer sets refilled with new circuits before each
    reuse (each slot's graph copies its buffers itself and is matched to them
    again), a second layout on the same buffers, and calls with pinned gates
    but pageable fitness (copies around the graph); every result against the
    oracle"""
    import torch
    ss = searches(prec)
    rng = np.random.default_rng(81 + prec)
    plans = [[(0, 1000), (4, 4096)], [(4, 4096), (0, 1000)]]
    nb, depth = 5, 3
    ring = []
    for b in range(nb):
        c = _Call(qe, ss, [(q, gates_for(ss[q], n, rng)) for q, n in plans[0]])
        ring.append(c)
    flight = []

    def finish(entry):
        call, t, items = entry
        ctx.eval_host_batch_wait(t)
        fits, tops = call.results()
        for (q, g), f, tk in zip(items, fits, tops):
            check_item(ss[q], g, f, tk)

    with qe.Context(ss) as ctx:
        for i in range(4 * nb + 3):
            if len(flight) == depth:
                finish(flight.pop(0))
            c = ring[i % nb]
            # a new layout on the same buffers every seventh call
            plan = plans[1] if i % 7 == 6 else plans[0]
            items = [(q, gates_for(ss[q], n, rng)) for q, n in plan]
            c.items = items
            c.ns = [len(g) for _, g in items]
            c.ks = [min(max(ss[q].topk, 1), n) for (q, _), n in zip(items, c.ns)]
            c.hg.copy_(torch.from_numpy(np.concatenate([g.ravel() for _, g in items])))
            for j, (q, _) in enumerate(items):
                c.probs[j] = q
                c.counts[j] = c.ns[j]
            flight.append((c, c.submit(ctx), items))
        while flight:
            finish(flight.pop(0))
        # pinned gates, pageable fitness: the same results
        items = [(q, gates_for(ss[q], n, rng)) for q, n in plans[0]]
        c = ring[0]
        c.items, c.ns = items, [len(g) for _, g in items]
        c.ks = [min(max(ss[q].topk, 1), n) for (q, _), n in zip(items, c.ns)]
        c.hg.copy_(torch.from_numpy(np.concatenate([g.ravel() for _, g in items])))
        for j, (q, _) in enumerate(items):
            c.probs[j] = q
            c.counts[j] = c.ns[j]
        hf = np.full(sum(c.ns), -7.0, np.float64 if prec == W.PREC_FP64 else np.float32)
        t = ctx.eval_host_batch_async_ptr(c.probs, c.counts, c.hg.data_ptr(), hf.ctypes.data,
                                          c.tops)
        ctx.eval_host_batch_wait(t)
        fo = ko = 0
        fits2, tops2 = ctx.eval_host_batch(items, topk=True)
        for (q, g), n, k, f2, t2 in zip(items, c.ns, c.ks, fits2, tops2):
            assert np.array_equal(hf[fo:fo + n].view(np.uint8), f2.view(np.uint8))
            assert [(t.circuit, t.cost, t.fitness) for t in c.tops[ko:ko + k]] == t2
            check_item(ss[q], g, hf[fo:fo + n], t2)
            fo += n
            ko += k


@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
def test_pinned_buffers_at_unaligned_addresses(qe, prec):
    """page-locked buffers that the graph's copy kernels reach through their
    device mappings, at addresses and lengths that take each copy width (16-,
    4- and 1-byte words): the results equal those of pageable buffers"""
    import ctypes as C
    import torch
    ss = searches(prec)
    rng = np.random.default_rng(91 + prec)
    fb = 8 if prec == W.PREC_FP64 else 4
    for plan, g_off, f_off in (([(0, 1000), (1, 300)], 0, 0),    # 16-byte words
                               ([(0, 999), (1, 300)], 4, fb),     # 4-byte words
                               ([(1, 299), (2, 77)], 1, fb)):     # bytes in
        items = [(q, gates_for(ss[q], n, rng)) for q, n in plan]
        flat = np.concatenate([g.ravel() for _, g in items])
        n_tot = sum(n for _, n in plan)
        gbuf = torch.zeros(flat.size + 16, dtype=torch.uint8).pin_memory()
        gbuf[g_off:g_off + flat.size].copy_(torch.from_numpy(flat))
        fbuf = torch.zeros(n_tot * fb + 16, dtype=torch.uint8).pin_memory()
        ks = [min(max(ss[q].topk, 1), n) for q, n in plan]
        tops = (qe.qe_ranked * sum(ks))()
        probs = (C.c_uint32 * len(plan))(*[q for q, _ in plan])
        counts = (C.c_uint32 * len(plan))(*[n for _, n in plan])
        with qe.Context(ss) as ctx:
            for _ in range(2):  # the second call replays the slot's graph
                fbuf.zero_()
                ctx.eval_host_batch_wait(ctx.eval_host_batch_async_ptr(
                    probs, counts, gbuf.data_ptr() + g_off, fbuf.data_ptr() + f_off, tops))
                fits2, tops2 = ctx.eval_host_batch(items, topk=True)  # pageable
                raw = fbuf.numpy()[f_off:f_off + n_tot * fb].copy()
                got = raw.view(np.float64 if prec == W.PREC_FP64 else np.float32)
                fo = ko = 0
                for (q, g), k, f2, t2 in zip(items, ks, fits2, tops2):
                    n = len(g)
                    assert np.array_equal(got[fo:fo + n].view(np.uint8), f2.view(np.uint8))
                    assert [(t.circuit, t.cost, t.fitness) for t in tops[ko:ko + k]] == t2
                    check_item(ss[q], g, got[fo:fo + n], t2)
                    fo += n
                    ko += k
