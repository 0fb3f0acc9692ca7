#!/usr/bin/env python
"""Benchmark: candidate circuits evaluated per second, batched binary32 vs plain
binary64, on one GB300 per rank.

Workload (default): the 3-qubit search of the benchmark set -- Toffoli, Fredkin
and Peres targets, 28-gate NCV + H/T/T^dag + identity library, L = 16,
P = 4096 each, Philox seed 1, binary32 composition with binary64 top-32
rescoring.  One step = one whole generation of the three searches (sample ->
compose/score -> rank/rescore -> update), 12288 candidate circuits.  The L2 is
flushed (256 MB write) before every timed step; each step is timed with CUDA
events on the library's stream.

--impl reference times the CPU oracle (test infrastructure) on a bounded
sample of the same workload on the host cores.
"""
import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "candidate circuits evaluated/sec at n=3/4/5 qubits, FP32 batched vs FP64 plain"
WORKLOADS = {
    1: "3-qubit QEQEA: Toffoli, 19-gate NCV+I library, L=5, P=64, seed 0",
    2: "3-qubit QEQEA: Toffoli + Fredkin + Peres targets, 28-gate NCV+H/T/T^dag+I library, L=16, "
       "P=4096 each, Philox seed 1, top-32 per generation",
    3: "4-qubit QEQEA: C3NOT, 48-gate NCV+H/T/T^dag library, L=32, P=65536, top-64",
    4: "1024 uneven QEQEA searches, n in {3,4,5}, L in [8,64], P in [256,4096], random "
       "permutation targets, top-32",
    5: "5-qubit QEQEA: C4NOT, 75-gate NCV+H/T/T^dag library, L=64, P=262144, top-128",
}
UNIT = "circuits/s"


def dist_env():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return ws, rank, local


class ClockSampler:
    """nvidia-smi clocks/throttle reasons sampled every 200 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.out = None

    def __enter__(self):
        try:
            self.out = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.gpu), "--query-gpu=" + self.Q,
                 "--format=csv,noheader,nounits", "-lms", "200"],
                stdout=self.out, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.proc or not self.out:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.out.flush()
        rows = []
        for line in open(self.out.name):
            f = [x.strip() for x in line.split(",")]
            if len(f) < 9:
                continue
            try:
                rows.append((float(f[1]), float(f[2]), f[5:9], f[4]))
            except ValueError:
                continue
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"], "samples": 0}
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i, v in enumerate(r[2]) if v == "Active"})
        return {"sm_mhz": statistics.median(r[0] for r in rows), "sm_max_mhz": max(r[1] for r in rows),
                "reasons": reasons, "samples": len(rows)}


def peaks():
    try:
        return json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        return {}


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


def oracle_generation(oracle, p, state, gen, pool, k=32, chunk=64):
    """One whole generation of the oracle as it stands (sample, dense binary64
    compose/score, full sort, update) with its evaluation, nearly all of the
    time, split over `pool`'s threads in chunks of circuits (the oracle's calls
    release the interpreter lock); sampling and update run on one thread."""
    import numpy as np
    cur, best, bf = state
    gi, sid = oracle.sample(p, cur, gen)
    spans = [(lo, min(p.P, lo + chunk)) for lo in range(0, p.P, chunk)]
    parts = list(pool.map(lambda c: oracle.eval_circuits(p, gi[c[0]:c[1]]), spans))
    F = np.concatenate([f for f, _ in parts])
    cost = np.concatenate([c for _, c in parts])
    oracle.topk(F, cost, k)
    oracle.update(p, cur, best, bf, gen, sid, F)


# ---------------------------------------------------------------- reference arm
def run_reference(args):
    """The oracle as it stands, on a bounded sample of the same workload."""
    import numpy as np
    import oracle
    from paper_1809_11134_gb300 import workloads as W

    ws, rank, _ = dist_env()
    if rank != 0:
        return
    searches = W.config(args.config, P=args.population)
    P = min(args.ref_population, min(s.P for s in searches))
    probs = [oracle.make_problem(s.n, s.L, P, s.library, s.perm, seed=s.seed, run=r)
             for r, s in enumerate(searches)]
    states = [oracle.init_state(p) for p in probs]
    cores = host_cores()
    from concurrent.futures import ThreadPoolExecutor
    pool = ThreadPoolExecutor(cores)

    def one(step):
        j = step % len(probs)
        oracle_generation(oracle, probs[j], states[j], step // len(probs), pool)

    for w in range(args.warmup):
        one(w)
    t0 = time.perf_counter()
    for k in range(args.steps):
        one(args.warmup + k)
    dt = time.perf_counter() - t0
    pool.shutdown()
    value = P * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * dt / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
        "data": "synthetic",
        "config": {"workload": workload_name(args), "circuits_per_step": P,
                   "parallelism": "%d host threads (evaluation)" % cores, "l2": "host memory"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": "each step: one generation of one of the searches with its "
                                   "population capped at P=%d (sample, dense Kronecker compose, "
                                   "score, sort, update), the evaluation on %d threads"
                                   % (P, cores)},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


# ---------------------------------------------------------------- our arm
def cpu_baseline(seconds=10.0):
    """The oracle as it stands on the benchmark workload's Toffoli search
    (P=4096, L=16): whole generations repeated for `seconds`/2 on every host
    core (evaluation threaded, as oracle_generation) and for `seconds`/2 on
    one core (the oracle's own generation step)."""
    from concurrent.futures import ThreadPoolExecutor

    import oracle
    from paper_1809_11134_gb300 import workloads as W
    s = W.config(2)[0]
    cores = host_cores()

    def rate(secs, pool):
        p = oracle.make_problem(s.n, s.L, s.P, s.library, s.perm, seed=s.seed)
        state = oracle.init_state(p)
        rep = oracle.new_report()
        gen = 0
        t0 = time.perf_counter()
        while time.perf_counter() - t0 < secs:
            if pool is None:
                oracle.step(p, *state, gen, 32, rep)
            else:
                oracle_generation(oracle, p, state, gen, pool)
            gen += 1
        return s.P * gen / (time.perf_counter() - t0), gen

    v1, g1 = rate(seconds / 2, None)
    with ThreadPoolExecutor(cores) as pool:
        vn, gn = rate(seconds / 2, pool)
    return {"value": vn, "unit": UNIT, "cores": cores, "kind": "oracle",
            "one_core": {"value": v1, "unit": UNIT, "cores": 1},
            "sample": "whole generations of the Toffoli search (P=4096, L=16): sample, dense "
                      "binary64 compose/score, full sort, update; %d generations with the "
                      "evaluation on %d threads (chunks of 64 circuits), %d on one core; %.1f s "
                      "each" % (gn, cores, g1, seconds / 2)}


def workload_name(args):
    return (WORKLOADS.get(args.config, "benchmark search set %d" % args.config)
            + (" on the paper's Ising gate set" if getattr(args, "library", "discrete") == "ising"
               else "")
            + ("" if args.population is None else " (P capped at %d)" % args.population)
            + "; one step = one generation")


def replica_searches(W, config, population, rank, library=None):
    """The searches one rank runs: the benchmark set, seeds offset by rank so
    that every GPU runs an independent replica (weak scaling, no data-path
    collective); library=LIB_ISING: the same shapes on the paper's Ising set."""
    searches = W.config(config, P=population, library=library)
    for s in searches:
        s.seed = s.seed + 1000 * rank
    return searches


def max_over_ranks(total_ms, ws, device):
    """The timed region's length is the slowest rank's (all_reduce MAX)."""
    if ws <= 1:
        return total_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(n_circ_per_rank, steps, ws, total_ms):
    """Candidate circuits of all ranks per second of the slowest rank."""
    return ws * n_circ_per_rank * steps / (total_ms / 1e3)


def run_ours(args):
    import numpy as np
    import torch
    import torch.distributed as dist

    import __graft_entry__ as G
    ws, rank, local = dist_env()
    if ws > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    if rank == 0 or ws > 1:
        G.build()
    from paper_1809_11134_gb300 import qe
    from paper_1809_11134_gb300 import workloads as W

    searches = replica_searches(W, args.config, args.population, rank,
                                W.LIB_ISING if args.library == "ising" else None)
    n_circ = sum(s.P for s in searches)
    stream = torch.cuda.Stream()
    ctx = qe.Context(searches, stream=stream)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def do_flush():
        with torch.cuda.stream(stream):
            flush.zero_()

    # launch plan picked by timing real generations (results do not depend on it)
    tune_ms = ctx.autotune(3)
    plan = ctx.launch_plan()
    # the clock sampler starts before the warm-up, so that its own start-up
    # (nvidia-smi initialising NVML) does not fall into the timed region
    clk = ClockSampler(local).__enter__()
    time.sleep(0.5)
    for _ in range(args.warmup):
        ctx.step(1)
    # ---- timed region: K generations, L2 flushed before each
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    if ws > 1:
        dist.barrier()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for k in range(args.steps):
        do_flush()
        starts[k].record(stream)
        ctx.step_raw(1, None)
        ends[k].record(stream)
    stream.synchronize()
    wall = time.perf_counter() - t0
    torch.cuda.synchronize()
    clk.__exit__(None, None, None)
    step_ms = [starts[k].elapsed_time(ends[k]) for k in range(args.steps)]
    # host-driven rate: the same generations back to back, as a caller drives
    # them (no flush, no events), timed by the host clock
    stream.synchronize()
    h0 = time.perf_counter()
    for k in range(args.steps):
        ctx.step_raw(1, None)
    stream.synchronize()
    host_wall = time.perf_counter() - h0
    total_ms = max_over_ranks(sum(step_ms), ws, "cuda")
    if ws > 1:
        dist.barrier()
    value = whole_job_rate(n_circ, args.steps, ws, total_ms)
    clocks = clk.summary()

    # ---- per-stage times (events between the generation's kernels), L2
    # flushed before each generation: as the graph runs them (concurrent
    # stages, so the circuit and selection intervals include waiting on what
    # runs beside them), and serialised on one stream (each interval is that
    # kernel's own duration, the denominators of the rooflines)
    names = ["circuits", "rank_select", "rescore", "rank_sort", "update", "generation"]

    def stage_means(serial):
        ctx.stage_timing(True, serial=serial)
        rows = []
        for k in range(min(args.steps, 100)):
            do_flush()
            ctx.step_raw(1, None)
            rows.append(ctx.stage_times())
        ctx.stage_timing(False)
        return dict(zip(names, np.array(rows).mean(axis=0).tolist()))

    stage = stage_means(False)
    stage_serial = stage_means(True)

    # ---- roofline of the dominant kernel: the circuit kernel (sample +
    # compose + score + scatter), the largest kernel of a generation in the ncu
    # launch list of this workload (summarised under profiles/); its time is the event
    # interval around it in the serialised generation graph
    pk = peaks()
    alu32, alu64 = qe.measure_alu_peaks()
    last = [ctx.last_generation(r) for r in range(len(searches))]
    # useful flops of one more generation, counted by the library from the
    # sampled gates (qe_report.useful_flops); the gate mix drifts slowly
    reps = ctx.step(1)
    flops = sum(r["useful_flops"] for r in reps)
    roof = roofline("circuits", stage_serial["circuits"], flops, searches, pk,
                    traffic=TRAFFIC.get((args.config, args.population)))
    roof["timing"] = ("event interval around the circuit kernel in the serialised "
                      "generation graph (nothing runs beside it), L2 flushed before each "
                      "generation; mean of %d generations" % min(args.steps, 100))
    ub = update_bytes(searches, last)
    kernels = [
        {"kernel": "k_step (sample + compose + score + scatter)", "bound": "alu",
         "achieved_tflops": roof["achieved"], "frac_of_derived_fp32": roof["frac"],
         "frac_of_measured_fp32": roof["achieved"] / alu32},
        issue_roofline(roof, INSTR.get((args.config, args.population))),
        {"kernel": "k_update_elite + k_update_mutate_list", "bound": "hbm",
         "achieved_gbs": ub / (stage_serial["update"] / 1e3) / 1e9,
         "frac_of_measured_hbm": ub / (stage_serial["update"] / 1e3) / 1e9 / pk["hbm_gbs"]
         if pk.get("hbm_gbs") else None, "algorithmic_bytes": ub},
        {"kernel": "k_rank_select", "bound": "hbm",
         "achieved_gbs": n_circ * 8 / (stage_serial["rank_select"] / 1e3) / 1e9,
         "note": "reads each fitness and cost word once; one CTA per search, latency-bound"},
    ]

    # ---- end to end through the public API with host buffers
    e2e = end_to_end(qe, ctx, searches, last, args.steps)

    ctx.close()
    line = None
    if rank == 0:
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": ws, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": workload_name(args),
                       "arithmetic": "binary32 composition and scoring, top-k rescored in "
                                     "binary64 and ranked one generation behind (pipelined)",
                       "circuits_per_step": n_circ, "parallelism": "replica per GPU",
                       "l2": "flushed (256 MB write) before every timed step",
                       "launch_plan": plan, "autotune_ms_per_plan": [round(m, 5) for m in tune_ms],
                       "stage_ms": {k: round(v, 5) for k, v in stage.items()},
                       "stage_ms_serialised": {k: round(v, 5) for k, v in stage_serial.items()}},
            "roofline": roof,
            "kernel_rooflines": kernels,
            "alu_peaks_measured_tflops": {"fp32": alu32, "fp64": alu64,
                                          "how": "qe_measure_alu_peaks: FMA chains on every SM"},
            "e2e": e2e,
            "gpu_launches": launches_per_generation(searches) * args.steps,
            "clocks": clocks,
            "wall_s": wall,
            "host_driven": {"generations": args.steps, "wall_s": host_wall,
                            "circuits_per_s": n_circ * args.steps / host_wall,
                            "how": "generations launched back to back by the host (no L2 "
                                   "flush, no events), host clock around them"},
        }
        if not args.no_cpu:
            line["cpu_baseline"] = cpu_baseline(args.cpu_seconds)
        if not args.no_extra:
            line["per_config"] = per_config(qe, torch, args)
            line["by_qubits"] = by_qubits(line["per_config"])
        print(json.dumps(line), flush=True)
    if ws > 1:
        dist.barrier()
        dist.destroy_process_group()


# dram__bytes_read.sum + dram__bytes_write.sum of one k_step launch (a timed
# step, right after the L2 flush) from an ncu capture of this workload
# (summarised under profiles/): the reads include the update's L2 prefetch
TRAFFIC = {(2, None): 41.504e6}
# warp instructions of one k_step launch (smsp__inst_executed.sum) from the same
# capture: the circuit kernel at n = 3 is bound by instruction issue, not by
# the FP32 pipe, so its issue rate is reported beside the arithmetic roofline
INSTR = {(2, None): 9675705}


def issue_roofline(roof, instr):
    """Issue rate of the circuit kernel: warp instructions per second against
    152 SMs x 4 schedulers x one warp instruction per cycle at the maximum SM
    clock (null without a capture of this workload)."""
    pk = peaks()
    peak = 152 * 4 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e9  # G warp instructions/s
    if not instr:
        return {"kernel": roof["kernel"], "bound": "issue", "achieved_ginst_per_s": None,
                "peak": peak, "frac": None, "warp_instructions_per_launch": None}
    ach = instr / (roof["ms"] / 1e3) / 1e9
    return {"kernel": roof["kernel"], "bound": "issue", "achieved_ginst_per_s": ach,
            "peak": peak, "unit": "G warp instructions/s", "frac": ach / peak,
            "warp_instructions_per_launch": instr,
            "peak_source": "derived: 152 SMs x 4 schedulers x 1 warp instruction/cycle x %.0f MHz"
                           % pk.get("sm_max_mhz", 2070.0),
            "instructions_source": "smsp__inst_executed.sum of one launch, ncu capture of this "
                                   "workload (k_step summary under profiles/)"}


def roofline(dom, ms, flops, searches, pk, traffic=None):
    """Achieved algorithmic rate of the dominant kernel against its roofline."""
    hbm = pk.get("hbm_gbs")
    sm_max = pk.get("sm_max_mhz", 2070.0)
    fp32_peak = 152 * 128 * 2 * sm_max * 1e6 / 1e12  # TFLOP/s, FMA = 2 flops
    if dom == "circuits":
        # useful flops of a generation (gate-count model)
        ach = flops / (ms / 1e3) / 1e12
        return {"kernel": "k_step (sample + compose + score + scatter)", "bound": "alu",
                "achieved": ach, "peak": fp32_peak, "unit": "TFLOP/s", "frac": ach / fp32_peak,
                "traffic": traffic, "algorithmic_flops": flops, "ms": ms,
                "peak_source": "derived: 152 SMs x 128 FP32 lanes x 2 (FMA) x %.0f MHz" % sm_max}
    if dom == "update":
        b = flops  # algorithmic bytes of the update (update_bytes)
        ach = b / (ms / 1e3) / 1e9
        return {"kernel": "k_update (elitism + mutation)", "bound": "hbm", "achieved": ach,
                "peak": hbm, "unit": "GB/s", "frac": ach / hbm if hbm else None, "traffic": None,
                "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}
    # ranking kernels: bytes of the fitness arrays they read
    b = sum(s.P * 8 for s in searches)
    ach = b / (ms / 1e3) / 1e9
    return {"kernel": dom, "bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s",
            "frac": ach / hbm if hbm else None, "traffic": None,
            "peak_source": "MEASURED_PEAKS.json hbm_gbs (measured)"}


def launches_per_generation(searches):
    """Kernel nodes of one generation graph: one circuit kernel per (width,
    arithmetic) group, the two update kernels, selection, one rescoring kernel
    per width with binary32 searches, sort, finish."""
    groups = len(set((s.n, s.precision == 0) for s in searches))
    widths = len(set(s.n for s in searches if s.precision != 0))
    return groups + 2 + 1 + widths + 1 + 1


def update_bytes(searches, last):
    """Algorithmic bytes of one update launch: every (circuit, slot) reads its
    segment id and takes the segment key (4 + 4 B); every used segment moves its
    32 B record once (read cur or best, write the other) and reads best_f; every
    segment of a mutated individual reads and writes its 32 B record and reads
    best_f and its key."""
    import numpy as np
    total = 0
    for s, l in zip(searches, last):
        sid = l["seg_id"]
        used = len(np.unique(sid))
        if s.library == 8:  # Ising: the wires, then the wire pairs
            R = s.n + s.n * (s.n - 1) // 2
        else:
            R = (s.n * (s.n - 1) if s.library & 1 else 0) + (s.n if s.library & 2 else 0)
        mutated = s.p_mutation * s.P * R * s.L
        total += sid.size * 8 + used * (32 + 32 + 4) + mutated * (32 + 32 + 4 + 4)
    return total


def end_to_end(qe, ctx_unused, searches, last, steps):
    """qe_eval_host_batch per step: the step's candidate circuits (one generation
    of every search, host gate strings) go host -> device from pinned memory in
    one copy, binary32 evaluation and binary64 top-k ranking of every search run
    on the GPU, and the fitness and top-k lists come back to pinned host memory.
    Timed twice: through the asynchronous pair (as many calls in flight as the
    context has batch slots, each on its own set of pinned buffers, so that the
    copies, evaluations and rankings of consecutive steps overlap; the
    headline) and through the synchronous call (one synchronisation per
    step)."""
    import ctypes as C
    import numpy as np
    import torch
    from paper_1809_11134_gb300 import workloads as W
    if any(s.library & W.LIB_ISING for s in searches):
        return {"value": None, "unit": UNIT,
                "note": "the host batch call takes gate strings only; Ising circuits also "
                        "need their angles (qe_eval_amp, device buffers)"}
    ctx = qe.Context(searches)
    gates = np.concatenate([np.ascontiguousarray(l["gate_idx"]).ravel() for l in last])
    n = sum(s.P for s in searches)
    k_total = sum(min(max(s.topk, 1), s.P) for s in searches)
    depth = qe.QE_BATCH_SLOTS
    bufs = [(torch.from_numpy(gates.copy()).pin_memory(),
             torch.zeros(n, dtype=torch.float32).pin_memory(), (qe.qe_ranked * k_total)())
            for _ in range(depth)]
    probs = (C.c_uint32 * len(searches))(*range(len(searches)))
    counts = (C.c_uint32 * len(searches))(*[s.P for s in searches])

    def submit(i):
        hg, hf, tops = bufs[i % depth]
        return ctx.eval_host_batch_async_ptr(probs, counts, hg.data_ptr(), hf.data_ptr(), tops)

    def pipelined(k, d=depth):
        flight = []
        for i in range(k):
            if len(flight) == d:
                ctx.eval_host_batch_wait(flight.pop(0))
            flight.append(submit(i))
        for t in flight:
            ctx.eval_host_batch_wait(t)

    def synchronous(k):
        hg, hf, tops = bufs[0]
        for _ in range(k):
            ctx.eval_host_batch_ptr(probs, counts, hg.data_ptr(), hf.data_ptr(), tops)

    def timed(fn, d):
        # every slot in use warmed first (its first call allocates and
        # captures), then enough calls that filling and draining the pipeline
        # is a small part of the interval
        calls = max(steps, 16 * d)
        fn(2 * d + 2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        fn(calls)
        return n * calls / (time.perf_counter() - t0)

    out = {"sync": timed(synchronous, 1), "pipelined": timed(pipelined, depth)}
    by_depth = {}
    for d in sorted({1, 2, 4, 8, depth // 2} - {depth, 0}):
        if d < depth:
            by_depth[d] = timed(lambda k, d=d: pipelined(k, d), d)
    by_depth[depth] = out["pipelined"]
    # every buffer set holds the same circuits: the same results
    assert all(torch.equal(bufs[0][1], b[1]) for b in bufs[1:])
    ctx.close()
    return {"value": out["pipelined"], "unit": UNIT,
            "h2d_bytes_per_step": int(gates.size),
            "d2h_bytes_per_step": n * 4 + (k_total + 1) * 16,
            "sync_value": out["sync"],
            "by_calls_in_flight": {str(d): round(v) for d, v in by_depth.items()},
            "call": "qe_eval_host_batch_async / _wait: every search's circuits in one call "
                    "(binary32 eval + binary64 top-k), pinned host buffers (the gate strings "
                    "in and the fitness and top-k out are copied by the call's kernels "
                    "through the buffers' device mappings), %d calls in flight; sync_value: "
                    "qe_eval_host_batch, one synchronisation per step" % depth}


def _stage_rates(qe, torch, searches, gens):
    """Mean stage times of `gens` generations after one warm-up generation
    (binary32 searches first pick their launch plan with the autotuner)."""
    import numpy as np
    from paper_1809_11134_gb300 import workloads as W
    stream = torch.cuda.Stream()
    ctx = qe.Context(searches, stream=stream)
    if searches[0].precision != W.PREC_FP64:
        ctx.autotune(2)
    ctx.step(1)
    # whole generations as the graph runs them (no stage events), L2 flushed before each
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(gens)]
    for a, b in ev:
        with torch.cuda.stream(stream):
            flush.zero_()
        a.record(stream)
        ctx.step_raw(1, None)
        b.record(stream)
    stream.synchronize()
    gen_ms = float(np.mean([a.elapsed_time(b) for a, b in ev]))
    del flush
    # per-stage intervals (events between the kernels of the serialised graph:
    # each stage's own duration)
    ctx.stage_timing(True, serial=True)
    times = []
    for _ in range(gens):
        ctx.step_raw(1, None)
        times.append(ctx.stage_times())
    ctx.stage_timing(False)
    reps = ctx.step(1)
    t = np.array(times).mean(axis=0)
    t[5] = gen_ms
    n = sum(s.P for s in searches)
    flops = sum(r["useful_flops"] for r in reps)
    pk = peaks()
    fp32_peak = 152 * 128 * 2 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
    res = {"circuit_kernel_circuits_per_s": n / (t[0] / 1e3),
           "generation_circuits_per_s": n / (t[5] / 1e3),
           "circuit_kernel_ms": round(float(t[0]), 4), "generation_ms": round(float(t[5]), 4),
           "note": "generation: untimed graph, L2 flushed; circuit kernel and update: "
                   "event intervals in the serialised stage-timed graph",
           "circuit_kernel_useful_tflops": flops / (t[0] / 1e3) / 1e12,
           "launch_plan": ctx.launch_plan()}
    if searches[0].precision != W.PREC_FP64:
        res["circuit_kernel_alu_frac"] = res["circuit_kernel_useful_tflops"] / fp32_peak
        last = [ctx.last_generation(r) for r in range(len(searches))]
        if all(s.n == 5 and not (s.library & W.LIB_ISING) for s in searches):
            sb = sum(smem_bytes5(s, l["gate_idx"]) for s, l in zip(searches, last))
            peak = 152 * 128 * pk.get("sm_max_mhz", 2070.0) * 1e6 / 1e12
            res["circuit_kernel_smem"] = {
                "bound": "shared memory", "achieved_tbs": sb / (t[0] / 1e3) / 1e12,
                "peak_tbs": peak, "frac": sb / (t[0] / 1e3) / 1e12 / peak,
                "bytes_per_launch": sb,
                "model": "the kernel's own shared-memory traffic: 8 KB per CV (8 row pairs "
                         "read and written), 16 KB per H, 8 KB per T, none per CNOT, 8 KB "
                         "per circuit to set the identity; peak 152 SMs x 128 B/cycle x "
                         "the maximum SM clock (derived)"}
        if searches[0].encoding == W.ENC_QEQEA:
            ub = update_bytes(searches, last)
            res["update_ms"] = round(float(t[4]), 4)
            res["update_algorithmic_gbs"] = ub / (t[4] / 1e3) / 1e9
            res["update_hbm_frac"] = res["update_algorithmic_gbs"] / pk["hbm_gbs"] \
                if pk.get("hbm_gbs") else None
    return ctx, res


def _best_error(qe, torch, ctx32, searches, gens):
    """Run `gens` more generations, then evaluate every search's best-so-far
    circuit in binary32 (this context) and binary64: the error where the
    square root of Eq. (11) amplifies the rounding of d (f near 1)."""
    import numpy as np
    from paper_1809_11134_gb300 import workloads as W
    ctx32.step(gens, reports=False)
    reps = ctx32.step(1)
    s64 = [W.Search(**{**s.__dict__, "precision": W.PREC_FP64}) for s in searches]
    ctx64 = qe.Context(s64)
    out = []
    for r, (s, rep) in enumerate(zip(searches, reps)):
        g = torch.tensor([rep["best_gates"]], dtype=torch.uint8, device="cuda")
        f32 = torch.zeros(1, dtype=torch.float32, device="cuda")
        f64 = torch.zeros(1, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()
        ctx32.eval(r, g, f32)
        ctx64.eval(r, g, f64)
        torch.cuda.synchronize()
        a, b = float(f32.item()), float(f64.item())
        out.append({"fitness_fp64": b, "abs_err": abs(a - b),
                    "d_err": abs((1 - a) ** 2 - (1 - b) ** 2)})
    ctx64.close()
    return {"circuits": out, "max_abs_fitness_err_vs_fp64": max(o["abs_err"] for o in out),
            "d_space_bound": 8e-7 * searches[0].L + 2e-6}


def smem_bytes5(s, gate_idx):
    """Shared-memory bytes the 5-qubit binary32 circuit kernel moves for these
    circuits (library indices: [I], then CNOT, CV, CV^dag per ordered wire
    pair, then H, T, T^dag per wire)."""
    import numpy as np
    from paper_1809_11134_gb300 import workloads as W
    g = np.asarray(gate_idx, np.int64).ravel()
    base = 1 if s.library & W.LIB_IDENTITY else 0
    npair = 3 * s.n * (s.n - 1) if s.library & W.LIB_NCV else 0
    x = g - base
    pair = (x >= 0) & (x < npair)
    wire = x >= npair
    cv = int((pair & (x % 3 != 0)).sum())
    h = int((wire & ((x - npair) % 3 == 0)).sum())
    t = int((wire & ((x - npair) % 3 != 0)).sum())
    n_circ = np.asarray(gate_idx).shape[0]
    return 8192 * cv + 16384 * h + 8192 * t + (8192 + 256) * n_circ


def _fp32_error(qe, torch, ctx32, searches, n_unitary=256):
    """Max |F32 - F64| over the last binary32 generation's circuits and max
    elementwise |U32 - U64| over the first n_unitary of them; the binary64
    values come from the library's binary64 path, which the parity tests hold
    bit-exact with the oracle."""
    import numpy as np
    from paper_1809_11134_gb300 import workloads as W
    s64 = [W.Search(**{**s.__dict__, "precision": W.PREC_FP64}) for s in searches]
    ctx64 = qe.Context(s64)
    f_err, u_err, bad = 0.0, 0.0, 0
    hi_err, hi_n = 0.0, 0
    for r, s in enumerate(searches):
        last = ctx32.last_generation(r)
        g = torch.from_numpy(np.ascontiguousarray(last["gate_idx"])).cuda()
        f64 = torch.zeros(s.P, dtype=torch.float64, device="cuda")
        m = min(n_unitary, s.P)
        N = 1 << s.n
        u32 = torch.zeros(m * N * N * 2, dtype=torch.float32, device="cuda")
        u64 = torch.zeros(m * N * N * 2, dtype=torch.float64, device="cuda")
        torch.cuda.synchronize()  # the buffers are filled before either context's stream runs
        ctx64.eval(r, g, f64)
        ctx32.compose(r, g[:m], u32, n_circuits=m)
        ctx64.compose(r, g[:m], u64, n_circuits=m)
        torch.cuda.synchronize()
        df = np.abs(last["fitness"] - f64.cpu().numpy())
        du = (u32.double() - u64).abs().cpu().numpy()
        # a NaN would make max() skip it: count non-finite differences instead
        bad += int((~np.isfinite(df)).sum() + (~np.isfinite(du)).sum())
        f_err = max(f_err, float(np.nanmax(df)) if df.size else 0.0)
        u_err = max(u_err, float(np.nanmax(du)) if du.size else 0.0)
        # near f = 1 the square root of Eq. (11) amplifies the rounding of d
        hi = f64.cpu().numpy() > 0.99
        hi_n += int(hi.sum())
        if hi.any():
            hi_err = max(hi_err, float(np.nanmax(df[hi])))
    ctx64.close()
    if bad:
        raise RuntimeError("%d non-finite binary32/binary64 differences" % bad)
    return f_err, u_err, hi_err, hi_n


def by_qubits(pc):
    """The metric at n = 3/4/5 in one flat table: for each width's benchmark
    search (3: the three searches of P = 4096, 4: C3NOT at P = 65536, 5: C4NOT
    at P = 262144), circuits/s of the circuit kernel and of the whole
    generation, binary32 (binary64 top-k) against plain binary64."""
    out = {}
    for n, cfg in ((3, "config2"), (4, "config3"), (5, "config5")):
        res = pc.get(cfg, {})
        row = {}
        for prec in ("fp32", "fp64"):
            r = res.get(prec)
            if r:
                row[prec + "_circuit_kernel"] = r["circuit_kernel_circuits_per_s"]
                row[prec + "_generation"] = r["generation_circuits_per_s"]
        if "fp32_generation" in row and "fp64_generation" in row:
            row["fp32_over_fp64_generation"] = row["fp32_generation"] / row["fp64_generation"]
        out[str(n)] = row
    return out


def per_config(qe, torch, args):
    """Per benchmark search set: circuit-kernel rate (sample + compose + score)
    and generation rate, binary32 vs plain binary64, from the events inside the
    generation graph, with the binary32 path's largest error against binary64;
    the 1024 uneven searches (binary32); the GA run of the 5-qubit search on
    the same evaluation; the 3- and 5-qubit shapes on the paper's Ising gate
    set; and the 3-qubit set with repeated measurement and with dense targets
    (context next to the headline)."""
    import numpy as np
    from paper_1809_11134_gb300 import workloads as W
    out = {}
    for cfg, gens32, gens64 in ((2, 20, 5), (3, 6, 2), (5, 4, 1)):
        res = {}
        for prec, gens in ((W.PREC_FP32, gens32), (W.PREC_FP64, gens64)):
            searches = W.config(cfg, precision=prec)
            ctx, r = _stage_rates(qe, torch, searches, gens)
            if prec == W.PREC_FP32:
                fe, ue, he, hn = _fp32_error(qe, torch, ctx, searches)
                r["max_abs_fitness_err_vs_fp64"], r["max_abs_unitary_err_vs_fp64"] = fe, ue
                r["above_0.99"] = {"circuits": hn, "max_abs_fitness_err_vs_fp64": he}
                if cfg == 2:
                    # near f = 1: the searches' best circuits after 320 generations
                    # (the Toffoli and Peres searches reach exact circuits)
                    r["best_circuits_after_320_generations"] = _best_error(
                        qe, torch, ctx, searches, 300)
            ctx.close()
            res["fp32" if prec else "fp64"] = r
        res["fp32_over_fp64_circuit_kernel"] = (res["fp32"]["circuit_kernel_circuits_per_s"] /
                                                res["fp64"]["circuit_kernel_circuits_per_s"])
        res["fp32_over_fp64_generation"] = (res["fp32"]["generation_circuits_per_s"] /
                                            res["fp64"]["generation_circuits_per_s"])
        out["config%d" % cfg] = res
    searches = W.config(4)
    ctx, r = _stage_rates(qe, torch, searches, 3)
    ctx.close()
    r["searches"] = len(searches)
    r["circuits_per_generation"] = sum(s.P for s in searches)
    out["config4"] = {"fp32": r}
    searches = W.config(5, encoding=W.ENC_GA)
    ctx, r = _stage_rates(qe, torch, searches, 4)
    ctx.close()
    out["config5_ga"] = {"fp32": r}
    # the same shapes on the paper's Ising gate set (rotations and templates)
    for cfg, precs in ((2, (W.PREC_FP32, W.PREC_FP64)), (5, (W.PREC_FP32,))):
        res = {}
        for prec in precs:
            searches = W.config(cfg, precision=prec, library=W.LIB_ISING)
            ctx, r = _stage_rates(qe, torch, searches, 10 if cfg == 2 else 3)
            ctx.close()
            res["fp32" if prec else "fp64"] = r
        if "fp64" in res:
            res["fp32_over_fp64_generation"] = (res["fp32"]["generation_circuits_per_s"] /
                                                res["fp64"]["generation_circuits_per_s"])
        out["config%d_ising" % cfg] = res
    # the 3-qubit set with each slot's qutrit measured 8 times (majority outcome),
    # and against dense targets (the permutations as full complex matrices, so
    # the score is tr(S^dag T) over all N^2 entries)
    searches = W.config(2)
    for s in searches:
        s.shots = 8
    ctx, r = _stage_rates(qe, torch, searches, 10)
    ctx.close()
    out["config2_shots8"] = {"fp32": r}
    searches = W.config(2)
    for s in searches:
        N = 1 << s.n
        T = np.zeros((N, N), np.complex128)
        for j in range(N):
            T[s.perm[j], j] = 1.0
        s.target = T
    ctx, r = _stage_rates(qe, torch, searches, 10)
    ctx.close()
    out["config2_dense"] = {"fp32": r}
    return out


def launch_ranks(n):
    """Run this command as n ranks on this node (torch.distributed.run, one
    process per GPU, rendezvous on 127.0.0.1) and return their exit status."""
    import socket
    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node",
           str(n), "--master-addr", "127.0.0.1", "--master-port", str(port),
           os.path.abspath(__file__)] + sys.argv[1:]
    return subprocess.call(cmd)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10000)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-extra", action="store_true")
    ap.add_argument("--cpu-seconds", type=float, default=10.0)
    ap.add_argument("--ref-population", type=int, default=512)
    ap.add_argument("--config", type=int, default=2,
                    help="benchmark search set 1-5 (2 = the 3-qubit headline workload)")
    ap.add_argument("--library", default="discrete", choices=["discrete", "ising"],
                    help="the benchmark's gate library, or the paper's Ising set on the same "
                         "shapes (for profiling)")
    ap.add_argument("--population", type=int, default=None,
                    help="cap P (for profiling smaller cases of a configuration)")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3)
    if args.gpus > 1 and "WORLD_SIZE" not in os.environ:
        # not started by a launcher: start one process per GPU of this node
        sys.exit(launch_ranks(args.gpus))
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws != args.gpus:
        sys.exit("bench.py: --gpus %d, but the launcher started %d ranks" % (args.gpus, ws))
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
