"""One search sharded over several GPUs: the population loop of Sec. IV-D
("repeat this process sizeOfPopulation times") split by circuit.

Every rank holds the whole encoding state and draws the same circuits (the
measurement of Sec. IV-D is a pure function of the state, the seed and the
generation).  Rank r evaluates the circuits [lo_r, hi_r) of the population
(Sec. IV-C composition, Eq. (11) score) and the ranks exchange one thing, an
all-gather of the working-precision fitness values and gate costs of their
shards (P values each per generation; the segment ids need no exchange, every
rank sampled the same ones).  Then every rank ranks the whole population
(the binary64-rescored top-k) and applies the same update (segment fitness as
the maximum over the circuits that used a segment, elitism, adaptive mutation
from the same counter-based draws, Sec. IV-E and IV-F).  No step depends on
the order in which the gathered values arrived, so all ranks keep identical
state, bit for bit, and the trajectory is the one a single GPU computes.

The arithmetic runs in the library (qe_sample, qe_eval, qe_rank, qe_update
through `QeShardDevice`); this module only splits the population, moves the
gathered values and sequences the calls.  `ShardedSearch` talks to its
device through five methods, so the exchange logic can be exercised on CPU
ranks with any object that provides them.
"""
from dataclasses import dataclass


def shard_range(P, rank, world):
    """Circuits [lo, hi) of rank `rank`: contiguous, sizes differing by at most one."""
    base, extra = divmod(P, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


class TorchComm:
    """All-gather over torch.distributed (NCCL for device tensors, gloo for host
    tensors); shards of unequal size are padded to the largest and trimmed."""

    def __init__(self, group=None):
        import torch.distributed as dist
        self.dist = dist
        self.group = group
        self.rank = dist.get_rank(group) if dist.is_initialized() else 0
        self.world = dist.get_world_size(group) if dist.is_initialized() else 1

    def all_gather(self, x, P):
        import torch
        if self.world == 1:
            return x
        m = (P + self.world - 1) // self.world
        dev = x.device
        if self.dist.get_backend(self.group) == "gloo" and dev.type != "cpu":
            x = x.cpu()
        buf = torch.zeros(m, dtype=x.dtype, device=x.device)
        buf[:x.numel()] = x
        parts = [torch.empty_like(buf) for _ in range(self.world)]
        self.dist.all_gather(parts, buf, group=self.group)
        sizes = [hi - lo for lo, hi in (shard_range(P, r, self.world) for r in range(self.world))]
        out = torch.cat([parts[r][:sizes[r]] for r in range(self.world)])
        return out.to(dev)


class QeShardDevice:
    """One search of a qe.Context on this rank's GPU (discrete libraries).

    The library runs on the context's stream, torch (allocations, the
    collectives) on its current stream: each call orders the two both ways."""

    def __init__(self, ctx, prob=0):
        import torch
        self.ctx, self.prob = ctx, prob
        s = ctx.searches[prob]
        self.P, self.L = s.P, s.L
        self.fp64 = s.precision == 0
        self.device = torch.device("cuda", torch.cuda.current_device())
        self.stream = ctx.stream if ctx.stream is not None else torch.cuda.current_stream()
        self.gates = torch.empty(self.P * self.L, dtype=torch.uint8, device=self.device)
        self.seg = torch.empty(self.P * self.L, dtype=torch.int32, device=self.device)

    def _enter(self):
        import torch
        self.stream.wait_stream(torch.cuda.current_stream())

    def _leave(self):
        import torch
        torch.cuda.current_stream().wait_stream(self.stream)

    def sample(self, gen):
        self._enter()
        self.ctx.sample(self.prob, gen, self.gates, self.seg)
        self._leave()
        return self.gates, self.seg

    def evaluate(self, gates, lo, hi):
        import torch
        n = hi - lo
        f = torch.empty(n, dtype=torch.float64 if self.fp64 else torch.float32, device=self.device)
        c = torch.empty(n, dtype=torch.int32, device=self.device)
        if n:
            g = gates[lo * self.L:hi * self.L]
            self._enter()
            self.ctx.eval(self.prob, g, f, n_circuits=n, cost=c)
            self._leave()
        return f, c

    def rank(self, gates, fitness, cost):
        self._enter()
        return self.ctx.rank(self.prob, gates, fitness, cost, n_circuits=self.P)

    def update(self, gen, seg, fitness):
        import torch
        f64 = fitness.to(torch.float64)
        self._enter()
        self.ctx.update(self.prob, gen, seg, f64)
        self._leave()

    def state(self):
        return self.ctx.get_state(self.prob)


@dataclass
class GenerationResult:
    generation: int
    topk: list            # [(circuit, cost, binary64 fitness)] of the whole population
    fitness: object       # the gathered working-precision fitness, all P circuits


class ShardedSearch:
    """Drives one search's generations on this rank's shard of the population."""

    def __init__(self, device, comm=None, rank=None, world=None):
        self.dev = device
        self.comm = comm
        self.rank = comm.rank if rank is None else rank
        self.world = comm.world if world is None else world
        self.lo, self.hi = shard_range(device.P, self.rank, self.world)
        self._gates = self._seg = None

    def evaluate_shard(self, gen):
        """Sample the whole population (identical on every rank) and evaluate
        this rank's circuits; returns (fitness, cost) of the shard."""
        self._gates, self._seg = self.dev.sample(gen)
        return self.dev.evaluate(self._gates, self.lo, self.hi)

    def finish(self, gen, fitness, cost):
        """Rank the whole population and update the state, given every rank's
        fitness and cost in rank order (the all-gather's result)."""
        top = self.dev.rank(self._gates, fitness, cost)
        self.dev.update(gen, self._seg, fitness)
        return GenerationResult(gen, top, fitness)

    def generation(self, gen):
        f, c = self.evaluate_shard(gen)
        F = self.comm.all_gather(f, self.dev.P)
        C = self.comm.all_gather(c, self.dev.P)
        return self.finish(gen, F, C)


def best_of(results):
    """The best circuit over generations as (fitness, cost, generation, circuit),
    by (fitness desc, cost asc, earlier generation)."""
    best = None
    for r in results:
        if not r.topk:
            continue
        c, cost, F = r.topk[0]
        key = (F, -cost, -r.generation)
        if best is None or key > best[0]:
            best = (key, (F, cost, r.generation, c))
    return None if best is None else best[1]


__all__ = ["shard_range", "TorchComm", "QeShardDevice", "ShardedSearch", "GenerationResult",
           "best_of"]
