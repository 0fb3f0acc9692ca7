"""qe_eval_rank_static, the entry point for callers that cannot allocate device
memory (no context, scratch in a static device array), against the context
entry point qe_eval and against the CPU oracle on the same circuits, twice in
a row so the second call runs on scratch the first one left behind; and a
check that a call after the first allocates no device memory.

This file is collected last on purpose: if it fails, a run that stops at the
first failure has already run every other test."""
import numpy as np
import pytest

import oracle
from gpu_common import assert_fp32_fitness, oracle_problem
from paper_1809_11134_gb300 import workloads as W

pytestmark = pytest.mark.gpu

RANKED = np.dtype([("circuit", "<u4"), ("cost", "<u4"), ("fitness", "<f8")])


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as G
    G.build()
    from paper_1809_11134_gb300 import qe
    assert torch.cuda.is_available()
    return qe, torch


@pytest.mark.parametrize("prec", [W.PREC_FP32, W.PREC_FP64])
def test_static_scratch_matches_context_eval_and_oracle_twice(env, prec):
    qe, torch = env
    s = W.Search(4, 24, 3000, W.LIB_NCV | W.LIB_HT, W.cknot(4), precision=prec, topk=48,
                 cost_weight=0.05)
    G, _ = qe.qe_library_info(s.n, s.library)
    dt = torch.float64 if prec == W.PREC_FP64 else torch.float32
    rng = np.random.default_rng(21 + prec)
    stream = torch.cuda.current_stream()
    with qe.Context([s], stream=stream) as ctx:
        for n in (3000, 1700):  # second call smaller: the first call's scratch is still there
            gates = W.random_gates(rng, n, s.L, G)
            g = torch.from_numpy(gates).cuda()
            k = min(s.topk, n)
            f_ref = torch.zeros(n, dtype=dt, device="cuda")
            top_ref = ctx.eval(0, g, f_ref, topk=True)
            # every buffer of the static call exists before it runs
            f_new = torch.full((n,), float("nan"), dtype=dt, device="cuda")
            top_buf = torch.zeros(k * RANKED.itemsize, dtype=torch.uint8, device="cuda")
            qe.qe_eval_rank_static(s, g, f_new, top_buf, stream=stream)
            torch.cuda.synchronize()
            a, b = f_new.cpu().numpy(), f_ref.cpu().numpy()
            top = top_buf.cpu().numpy().view(RANKED)
            # the context entry point
            if prec == W.PREC_FP64:
                assert np.array_equal(a, b)
            else:
                assert np.abs(a.astype(np.float64) - b).max() <= 1e-5
            assert [int(x) for x in top["circuit"]] == [t[0] for t in top_ref]
            assert [int(x) for x in top["cost"]] == [t[1] for t in top_ref]
            assert [float(x) for x in top["fitness"]] == [t[2] for t in top_ref]
            # the oracle: binary64 fitness bit for bit, binary32 within its bound,
            # the rescored top-k exactly
            p = oracle_problem(s, 0)
            p.P = n
            F, cost = oracle.eval_circuits(p, gates)
            if prec == W.PREC_FP64:
                assert np.array_equal(a, F)
            else:
                assert_fp32_fitness(a, F, s, cost)
            order = oracle.topk(F, cost, k)
            assert [int(x) for x in top["circuit"]] == [int(c) for c in order]
            assert [int(x) for x in top["cost"]] == [int(cost[c]) for c in order]
            assert [float(x) for x in top["fitness"]] == [float(F[c]) for c in order]


def test_static_call_allocates_no_device_memory(env):
    """After a first call on the device (which may load the library's code),
    further calls leave the device's free memory and torch's allocator alone."""
    qe, torch = env
    s = W.Search(5, 16, 4000, W.LIB_NCV | W.LIB_HT, W.cknot(5), precision=W.PREC_FP32, topk=32)
    G, _ = qe.qe_library_info(s.n, s.library)
    rng = np.random.default_rng(5)
    g = torch.from_numpy(W.random_gates(rng, s.P, s.L, G)).cuda()
    f = torch.zeros(s.P, dtype=torch.float32, device="cuda")
    top = torch.zeros(32 * RANKED.itemsize, dtype=torch.uint8, device="cuda")
    stream = torch.cuda.current_stream()
    qe.qe_eval_rank_static(s, g, f, top, stream=stream)
    torch.cuda.synchronize()
    first = top.cpu().numpy().copy()
    free0, _ = torch.cuda.mem_get_info()
    alloc0 = torch.cuda.memory_allocated()
    for _ in range(3):
        qe.qe_eval_rank_static(s, g, f, top, stream=stream)
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    assert torch.cuda.memory_allocated() == alloc0
    assert np.array_equal(top.cpu().numpy(), first)


def test_static_scratch_rejects_oversized_batches(env):
    qe, torch = env
    s = W.Search(3, 4, 16, W.LIB_NCV, W.cknot(3), precision=W.PREC_FP32)
    g = torch.zeros((65537, 4), dtype=torch.uint8, device="cuda")
    f = torch.zeros(65537, dtype=torch.float32, device="cuda")
    with pytest.raises(qe.QeError) as e:
        qe.qe_eval_rank_static(s, g, f, None)
    assert e.value.status == qe.QE_EINVAL and "65536" in str(e.value)
