"""Checkpoint / resume on the GPU: every random draw is a Philox function of
(seed, generation, ...), so a context that loads a checkpoint continues the
saved run bit for bit -- reports, circuits, fitness, top-k and encoding state --
for both encodings, both precisions and both gate libraries in one context."""
import os

import numpy as np
import pytest

from gpu_common import state_equal
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


def mixed():
    return [W.Search(3, 16, 500, W.LIB_NCV | W.LIB_HT | W.LIB_IDENTITY, W.cknot(3), seed=1,
                     topk=8),
            W.Search(4, 12, 200, W.LIB_NCV | W.LIB_HT, W.cknot(4), seed=2, topk=4,
                     precision=W.PREC_FP64),
            W.Search(3, 10, 150, W.LIB_NCV | W.LIB_HT, W.peres(), seed=3, topk=5,
                     encoding=W.ENC_GA),
            W.Search(2, 3, 64, W.LIB_ISING, W.cknot(2), seed=4, topk=4),
            W.Search(3, 16, 120, W.LIB_ISING, W.cknot(3), seed=5, topk=3, encoding=W.ENC_GA,
                     ga_mutation_rate=0.1),
            W.Search(5, 20, 64, W.LIB_NCV | W.LIB_HT, W.cknot(5), seed=6, topk=2)]


def _states_equal(a, b):
    if isinstance(a, tuple):
        return all(_states_equal(x, y) for x, y in zip(a, b))
    if a.dtype == np.uint8:
        return np.array_equal(a, b)
    return state_equal(a, b)


def _snapshot(ctx, n):
    last = [ctx.last_generation(r) for r in range(n)]
    states = [ctx.get_state(r) for r in range(n)]
    return last, states


def _assert_same(reps_a, snap_a, reps_b, snap_b):
    assert reps_a == reps_b
    for la, lb in zip(snap_a[0], snap_b[0]):
        assert np.array_equal(la["gate_idx"], lb["gate_idx"])
        assert np.array_equal(la["fitness"], lb["fitness"])
        assert la["topk"] == lb["topk"]
    for sa, sb in zip(snap_a[1], snap_b[1]):
        assert _states_equal(sa, sb)


def test_resume_continues_the_run_bit_for_bit(qe, torch, tmp_path):
    path = str(tmp_path / "run.qeckpt")
    ss = mixed()
    with qe.Context(ss) as ctx:
        ctx.step(3)
        ctx.step(2, reports=False)  # the last generation's ranking still pending
        ctx.save(path)
        assert ctx.generation() == 5
        reps_a = ctx.step(6)
        snap_a = _snapshot(ctx, len(ss))
    probs, gen = qe.checkpoint_info(path)
    assert gen == 5 and len(probs) == len(ss)
    with qe.Context.from_checkpoint(path) as ctx:
        assert ctx.generation() == 5
        with pytest.raises(qe.QeError):
            ctx.last_generation(0)  # not part of a checkpoint
        reps_b = ctx.step(6)
        snap_b = _snapshot(ctx, len(ss))
    _assert_same(reps_a, snap_a, reps_b, snap_b)


def test_load_rewinds_a_context_that_ran_on(qe, torch, tmp_path):
    """Loading into the same context after it ran further (with a pending
    ranking) discards the later generations and replays them identically."""
    path = str(tmp_path / "rew.qeckpt")
    ss = mixed()[:4]
    with qe.Context(ss) as ctx:
        ctx.step(4)
        ctx.save(path)
        reps_a = ctx.step(5)
        snap_a = _snapshot(ctx, len(ss))
        ctx.step(3, reports=False)
        ctx.load(path)
        assert ctx.generation() == 4
        reps_b = ctx.step(5)
        snap_b = _snapshot(ctx, len(ss))
    _assert_same(reps_a, snap_a, reps_b, snap_b)


def test_checkpoint_at_generation_zero_is_a_fresh_start(qe, torch, tmp_path):
    path = str(tmp_path / "zero.qeckpt")
    ss = mixed()[2:5]
    with qe.Context(ss) as ctx:
        ctx.save(path)
        reps_a = ctx.step(3)
        snap_a = _snapshot(ctx, len(ss))
    with qe.Context(ss) as ctx:
        ctx.step(2)
        ctx.load(path)
        reps_b = ctx.step(3)
        snap_b = _snapshot(ctx, len(ss))
    _assert_same(reps_a, snap_a, reps_b, snap_b)


def test_bad_checkpoints_change_nothing(qe, torch, tmp_path):
    path = str(tmp_path / "ok.qeckpt")
    ss = mixed()[:3]
    with qe.Context(ss) as ctx:
        ctx.step(2)
        ctx.save(path)
    raw = open(path, "rb").read()
    other = [W.Search(3, 16, 500, W.LIB_NCV | W.LIB_HT | W.LIB_IDENTITY, W.cknot(3), seed=99,
                      topk=8)] + ss[1:]
    with qe.Context(other) as ctx:
        ctx.step(1)
        before = [ctx.get_state(r) for r in range(3)]
        # other problems
        with pytest.raises(qe.QeError) as e:
            ctx.load(path)
        assert e.value.status == qe.QE_EINVAL
        # a flipped payload byte
        bad = str(tmp_path / "flip.qeckpt")
        open(bad, "wb").write(raw[:100] + bytes([raw[100] ^ 4]) + raw[101:])
        with pytest.raises(qe.QeError) as e:
            ctx.load(bad)
        assert e.value.status == qe.QE_EINVAL
        # truncated, missing
        open(bad, "wb").write(raw[:-7])
        with pytest.raises(qe.QeError):
            ctx.load(bad)
        with pytest.raises(qe.QeError) as e:
            ctx.load(str(tmp_path / "missing.qeckpt"))
        assert e.value.status == qe.QE_EIO
        assert ctx.generation() == 1
        after = [ctx.get_state(r) for r in range(3)]
        for a, b in zip(before, after):
            assert _states_equal(a, b)
        ctx.step(1)  # still usable
    # an unwritable path leaves no file and reports QE_EIO
    with qe.Context(ss) as ctx:
        with pytest.raises(qe.QeError) as e:
            ctx.save(str(tmp_path / "no_such_dir" / "x.qeckpt"))
        assert e.value.status == qe.QE_EIO
    assert not os.path.exists(str(tmp_path / "no_such_dir"))
