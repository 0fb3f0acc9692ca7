"""One search sharded over ranks, on CPU ranks (gloo): the exchange logic of
paper_1809_11134_gb300.shard with the CPU oracle standing in for each rank's
device.  Every rank samples the whole population, evaluates its shard, the
fitness and cost values are all-gathered, and every rank ranks and updates the
whole population: the trajectory (every generation's fitness and top-k, the
final encoding state) must equal the single-rank oracle's bit for bit, on
every rank, with shards of unequal size."""
import os
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HERE = os.path.dirname(os.path.abspath(__file__))


class OracleShardDevice:
    """The five device calls of ShardedSearch, computed by the oracle on the host."""

    def __init__(self, s):
        import oracle
        from gpu_common import oracle_problem
        self.oracle = oracle
        self.p = oracle_problem(s, 0)
        self.P, self.L, self.k = s.P, s.L, max(s.topk, 1)
        self.cur, self.best, self.bf = oracle.init_state(self.p)

    def sample(self, gen):
        import torch
        gi, sid = self.oracle.sample(self.p, self.cur, gen)
        return (torch.from_numpy(gi.ravel().copy()),
                torch.from_numpy(sid.ravel().view(np.int32).copy()))

    def evaluate(self, gates, lo, hi):
        import torch
        g = gates.numpy().reshape(self.P, self.L)[lo:hi]
        F, cost = self.oracle.eval_circuits(self.p, g)
        return torch.from_numpy(F.copy()), torch.from_numpy(cost.view(np.int32).copy())

    def rank(self, gates, fitness, cost):
        F = fitness.numpy()
        C = cost.numpy().view(np.uint32)
        order = self.oracle.topk(F, C, self.k)
        return [(int(c), int(C[c]), float(F[c])) for c in order]

    def update(self, gen, seg, fitness):
        self.oracle.update(self.p, self.cur, self.best, self.bf, gen,
                           seg.numpy().view(np.uint32), fitness.numpy().astype(np.float64))

    def state(self):
        return self.cur, self.best, self.bf


def _search(P):
    from paper_1809_11134_gb300 import workloads as W
    return W.Search(3, 6, P, W.LIB_NCV | W.LIB_HT | W.LIB_IDENTITY, W.cknot(3), seed=7,
                    precision=W.PREC_FP64, topk=8, p_mutation=0.3)


def _rank(rank, ws, port, P, gens, q):
    sys.path.insert(0, ROOT)
    sys.path.insert(0, HERE)
    import torch.distributed as dist

    from paper_1809_11134_gb300 import shard
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        dev = OracleShardDevice(_search(P))
        run = shard.ShardedSearch(dev, shard.TorchComm())
        out = []
        for g in range(gens):
            r = run.generation(g)
            out.append((r.fitness.numpy().copy(), r.topk))
        cur, best, bf = dev.state()
        q.put((rank, (run.lo, run.hi), out, cur.copy(), best.copy(), bf.copy()))
    finally:
        dist.destroy_process_group()


def _single_rank(P, gens):
    import oracle
    from gpu_common import oracle_problem
    s = _search(P)
    p = oracle_problem(s, 0)
    cur, best, bf = oracle.init_state(p)
    rep = oracle.new_report()
    traj = []
    for g in range(gens):
        gi, sid, F, cost, tk = oracle.step(p, cur, best, bf, g, s.topk, rep)
        traj.append((F.copy(), [(int(c), int(cost[c]), float(F[c])) for c in tk]))
    return traj, cur, best, bf


def test_shard_ranges_cover_the_population():
    sys.path.insert(0, ROOT)
    from paper_1809_11134_gb300.shard import shard_range
    for P in (1, 2, 7, 64, 1001):
        for ws in (1, 2, 3, 8):
            r = [shard_range(P, k, ws) for k in range(ws)]
            assert r[0][0] == 0 and r[-1][1] == P
            assert all(r[k][1] == r[k + 1][0] for k in range(ws - 1))
            sizes = [hi - lo for lo, hi in r]
            assert max(sizes) - min(sizes) <= 1


@pytest.mark.parametrize("ws,P", [(2, 301), (3, 128)])
def test_sharded_trajectory_equals_the_single_rank_one(ws, P):
    import torch.multiprocessing as mp
    gens = 6
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29700 + (os.getpid() + 37 * ws) % 1000
    procs = [ctx.Process(target=_rank, args=(r, ws, port, P, gens, q)) for r in range(ws)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda x: x[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    traj, cur, best, bf = _single_rank(P, gens)
    assert [r[1] for r in res] != [(0, P)] * ws  # the ranks really split the population
    for rank, span, out, c2, b2, f2 in res:
        for g in range(gens):
            assert np.array_equal(out[g][0], traj[g][0]), (rank, g)
            assert out[g][1] == traj[g][1], (rank, g)
        assert np.array_equal(c2.view(np.uint32), cur.view(np.uint32))
        assert np.array_equal(b2.view(np.uint32), best.view(np.uint32))
        assert np.array_equal(f2.view(np.uint32), bf.view(np.uint32))
