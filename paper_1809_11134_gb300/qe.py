"""Thin ctypes binding of the C ABI in include/qe.h (libqe.so).

Every function marshals arguments and calls the library; all computation runs
in the library's CUDA kernels.  Device buffers are torch CUDA tensors (their
data_ptr() is passed), host buffers are numpy arrays.  There is no fallback:
importing the binding without a built libqe.so raises.
"""
import ctypes as C
import os
from typing import List, Optional, Sequence

import numpy as np

from . import workloads as W

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libqe.so")

(QE_OK, QE_EINVAL, QE_ENOMEM, QE_ECUDA, QE_ETIMEOUT, QE_ENUMERIC, QE_ESTATE, QE_EUNSUPPORTED,
 QE_EIO) = range(9)
STATUS_NAMES = ["QE_OK", "QE_EINVAL", "QE_ENOMEM", "QE_ECUDA", "QE_ETIMEOUT", "QE_ENUMERIC",
                "QE_ESTATE", "QE_EUNSUPPORTED", "QE_EIO"]
QE_LIB_NCV, QE_LIB_HT, QE_LIB_IDENTITY, QE_LIB_ISING = 1, 2, 4, 8
QE_PREC_FP64, QE_PREC_FP32, QE_PREC_SPLIT_TC = 0, 1, 2
QE_FIT_TRACE, QE_FIT_PROB = 0, 1
QE_ENC_QEQEA, QE_ENC_GA = 0, 1
QE_ERRW_BAD_GATE, QE_ERRW_NONFINITE, QE_ERRW_GUARD_BAND = 1, 2, 4
QE_BATCH_SLOTS = 16  # qe_eval_host_batch_async calls in flight at once

# every symbol include/qe.h declares
EXPORTS = ["qe_library_info", "qe_init", "qe_sample", "qe_eval", "qe_eval_amp", "qe_rank",
           "qe_eval_host",
           "qe_eval_host_batch", "qe_eval_host_batch_async", "qe_eval_host_batch_wait",
           "qe_compose", "qe_compose_amp",
           "qe_update", "qe_step", "qe_last_generation", "qe_state_bytes", "qe_get_state",
           "qe_set_state", "qe_generation", "qe_autotune", "qe_launch_plan", "qe_stage_timing",
           "qe_stage_times", "qe_measure_alu_peaks", "qe_save", "qe_load", "qe_checkpoint_info",
           "qe_set_target",
           "qe_eval_rank_static", "qe_last_error", "qe_destroy"]


class qe_problem(C.Structure):
    _fields_ = [("n_qubits", C.c_uint32), ("circuit_len", C.c_uint32),
                ("population", C.c_uint32), ("library", C.c_uint32), ("encoding", C.c_uint32),
                ("precision", C.c_uint32), ("fitness_kind", C.c_uint32), ("topk", C.c_uint32),
                ("seed", C.c_uint64), ("p_mutation", C.c_double), ("mutation_range", C.c_double),
                ("ga_mutation_rate", C.c_double), ("cost_weight", C.c_double),
                ("target_perm", C.c_uint8 * 32), ("shots", C.c_uint32), ("reserved", C.c_uint32)]


class qe_ranked(C.Structure):
    _fields_ = [("circuit", C.c_uint32), ("cost", C.c_uint32), ("fitness", C.c_double)]


class qe_report(C.Structure):
    _fields_ = [("generation", C.c_uint32), ("best_gen", C.c_uint32),
                ("best_fitness", C.c_double), ("gen_best_fitness", C.c_double),
                ("mean_fitness", C.c_double), ("useful_flops", C.c_uint64),
                ("best_cost", C.c_uint32), ("best_len", C.c_uint32), ("error_word", C.c_uint32),
                ("reserved", C.c_uint32), ("best_gates", C.c_uint8 * 64),
                ("best_amps", C.c_float * 128)]


class QeError(RuntimeError):
    def __init__(self, status, message):
        self.status = status
        super().__init__("%s: %s" % (STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES)
                                     else status, message))


_lib = None


def lib():
    """Load libqe.so (built by __graft_entry__.build() / _build.build())."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libqe.so is not built (run __graft_entry__.build()); "
                              "there is no CPU fallback")
        L = C.CDLL(LIB_PATH)
        vp, u32, u64, sz = C.c_void_p, C.c_uint32, C.c_uint64, C.c_size_t
        L.qe_library_info.argtypes = [u32, u32, C.POINTER(u32), C.POINTER(u32)]
        L.qe_init.argtypes = [C.POINTER(vp), C.POINTER(qe_problem), u32, vp]
        L.qe_sample.argtypes = [vp, u32, u32, vp, vp]
        L.qe_eval.argtypes = [vp, u32, vp, u32, vp, vp, C.POINTER(qe_ranked)]
        L.qe_eval_host.argtypes = [vp, u32, vp, u32, vp, C.POINTER(qe_ranked)]
        L.qe_eval_host_batch.argtypes = [vp, u32, C.POINTER(u32), C.POINTER(u32), vp, vp,
                                         C.POINTER(qe_ranked)]
        L.qe_eval_host_batch_async.argtypes = [vp, u32, C.POINTER(u32), C.POINTER(u32), vp, vp,
                                               C.POINTER(qe_ranked), C.POINTER(u64)]
        L.qe_eval_host_batch_wait.argtypes = [vp, u64]
        L.qe_compose.argtypes = [vp, u32, vp, u32, vp]
        L.qe_eval_amp.argtypes = [vp, u32, vp, vp, u32, vp, vp, C.POINTER(qe_ranked)]
        L.qe_compose_amp.argtypes = [vp, u32, vp, vp, u32, vp]
        L.qe_update.argtypes = [vp, u32, u32, vp, vp]
        L.qe_step.argtypes = [vp, u32, C.POINTER(qe_report)]
        L.qe_last_generation.argtypes = [vp, u32, vp, vp, vp, C.POINTER(qe_ranked)]
        L.qe_state_bytes.argtypes = [vp, u32, C.POINTER(sz)]
        L.qe_get_state.argtypes = [vp, u32, vp, sz]
        L.qe_set_state.argtypes = [vp, u32, vp, sz]
        L.qe_generation.argtypes = [vp, C.POINTER(u32)]
        L.qe_autotune.argtypes = [vp, u32, C.POINTER(C.c_float), C.POINTER(u32)]
        L.qe_launch_plan.argtypes = [vp, C.c_char_p, sz]
        L.qe_stage_timing.argtypes = [vp, C.c_int]
        L.qe_measure_alu_peaks.argtypes = [C.POINTER(C.c_double), C.POINTER(C.c_double)]
        L.qe_stage_times.argtypes = [vp, C.POINTER(C.c_float)]
        L.qe_eval_rank_static.argtypes = [C.POINTER(qe_problem), vp, u32, vp, vp, vp,
                                          C.c_char_p, sz]
        L.qe_set_target.argtypes = [vp, u32, vp]
        L.qe_save.argtypes = [vp, C.c_char_p]
        L.qe_load.argtypes = [vp, C.c_char_p]
        L.qe_checkpoint_info.argtypes = [C.c_char_p, C.POINTER(qe_problem), u32, C.POINTER(u32),
                                         C.POINTER(u32)]
        L.qe_last_error.argtypes = [vp]
        L.qe_last_error.restype = C.c_char_p
        L.qe_destroy.argtypes = [vp]
        L.qe_destroy.restype = None
        for name in EXPORTS:
            if name not in ("qe_last_error", "qe_destroy"):
                getattr(L, name).restype = C.c_int
        _lib = L
    return _lib


def _check(ctx_ptr, status):
    if status != QE_OK:
        msg = lib().qe_last_error(ctx_ptr)
        raise QeError(status, (msg or b"").decode())
    return status


def to_problem(s) -> qe_problem:
    """qe_problem from a workloads.Search (or pass a qe_problem through)."""
    if isinstance(s, qe_problem):
        return s
    p = qe_problem()
    p.n_qubits, p.circuit_len, p.population, p.library = s.n, s.L, s.P, s.library
    p.encoding = s.encoding
    p.precision, p.fitness_kind, p.topk = s.precision, s.fitness_kind, s.topk
    p.seed = s.seed
    p.p_mutation, p.mutation_range = s.p_mutation, s.mutation_range
    p.ga_mutation_rate, p.cost_weight = s.ga_mutation_rate, s.cost_weight
    p.shots = getattr(s, "shots", 1)
    for j in range(32):
        p.target_perm[j] = s.perm[j] if j < len(s.perm) else 0
    return p


def qe_library_info(n_qubits: int, library: int):
    g, r = C.c_uint32(), C.c_uint32()
    _check(None, lib().qe_library_info(n_qubits, library, C.byref(g), C.byref(r)))
    return g.value, r.value


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream_handle(stream):
    if stream is None:
        import torch
        stream = torch.cuda.current_stream()
    return C.c_void_p(stream.cuda_stream)


def _need(t, dtype, numel, name):
    import torch
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("%s must be a CUDA tensor" % name)
    if t.dtype != dtype or not t.is_contiguous() or t.numel() < numel:
        raise TypeError("%s must be a contiguous %s tensor with >= %d elements" % (name, dtype, numel))


class BatchCall:
    """A qe_eval_host_batch_async call in flight (see Context.eval_host_batch_async)."""

    def __init__(self, ctx, ticket, keep):
        self.ctx, self.ticket, self._keep = ctx, ticket, keep

    def wait(self):
        self.ctx.eval_host_batch_wait(self.ticket)
        return Context._batch_results(self._keep)


class Context:
    """One qe_ctx: n independent searches sharing every launch."""

    def __init__(self, searches: Sequence, stream=None):
        self.searches = list(searches)
        probs = (qe_problem * len(self.searches))(*[to_problem(s) for s in self.searches])
        self._probs = probs
        h = C.c_void_p()
        st = lib().qe_init(C.byref(h), probs, len(self.searches), _stream_handle(stream))
        if st != QE_OK:
            raise QeError(st, (lib().qe_last_error(None) or b"").decode())
        self.h = h
        self.stream = stream
        for i, s in enumerate(self.searches):
            if getattr(s, "target", None) is not None:
                self.set_target(i, s.target)

    def close(self):
        if getattr(self, "h", None):
            lib().qe_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def prob(self, i):
        return self._probs[i]

    # ------------------------------------------------------------ calls
    def sample(self, prob, gen, gate_idx, seg_id):
        import torch
        p = self._probs[prob]
        n = p.population * p.circuit_len
        _need(gate_idx, torch.uint8, n, "gate_idx")
        _need(seg_id, torch.int32, n, "seg_id")
        _check(self.h, lib().qe_sample(self.h, prob, gen, _ptr(gate_idx), _ptr(seg_id)))

    def eval(self, prob, gate_idx, fitness, n_circuits=None, cost=None, topk=False, amps=None):
        """amps: Ising searches, float32 [n, L, 2] device tensor of the slots' qubit
        amplitudes (their angles): calls qe_eval_amp"""
        import torch
        p = self._probs[prob]
        n = gate_idx.shape[0] if n_circuits is None else n_circuits
        _need(gate_idx, torch.uint8, n * p.circuit_len, "gate_idx")
        if amps is not None:
            _need(amps, torch.float32, n * p.circuit_len * 2, "amps")
        _need(fitness, torch.float64 if p.precision == QE_PREC_FP64 else torch.float32, n,
              "fitness")
        if cost is not None:
            _need(cost, torch.int32, n, "cost")
        out = None
        if topk:
            k = min(max(p.topk, 1), n)
            out = (qe_ranked * max(k, 1))()
        if amps is None:
            _check(self.h, lib().qe_eval(self.h, prob, _ptr(gate_idx), n, _ptr(fitness),
                                         _ptr(cost), out))
        else:
            _check(self.h, lib().qe_eval_amp(self.h, prob, _ptr(gate_idx), _ptr(amps), n,
                                             _ptr(fitness), _ptr(cost), out))
        if topk:
            return [(r.circuit, r.cost, r.fitness) for r in out[:k]]
        return None

    def rank(self, prob, gate_idx, fitness, cost, n_circuits=None, amps=None):
        """qe_rank: the top-k of given fitness values (device tensors), rescored in
        binary64 from the gates; returns [(circuit, cost, fitness)]"""
        import torch
        p = self._probs[prob]
        n = gate_idx.shape[0] if n_circuits is None else n_circuits
        _need(gate_idx, torch.uint8, n * p.circuit_len, "gate_idx")
        if amps is not None:
            _need(amps, torch.float32, n * p.circuit_len * 2, "amps")
        _need(fitness, torch.float64 if p.precision == QE_PREC_FP64 else torch.float32, n,
              "fitness")
        _need(cost, torch.int32, n, "cost")
        k = min(max(p.topk, 1), n)
        out = (qe_ranked * max(k, 1))()
        _check(self.h, lib().qe_rank(self.h, prob, _ptr(gate_idx), _ptr(amps), _ptr(fitness),
                                     _ptr(cost), n, out))
        return [(r.circuit, r.cost, r.fitness) for r in out[:k]]

    def eval_host(self, prob, gate_idx: np.ndarray, topk=False):
        p = self._probs[prob]
        g = np.ascontiguousarray(gate_idx, np.uint8)
        n = g.shape[0]
        fit = np.zeros(n, np.float64 if p.precision == QE_PREC_FP64 else np.float32)
        out = None
        if topk:
            k = min(max(p.topk, 1), n)
            out = (qe_ranked * max(k, 1))()
        _check(self.h, lib().qe_eval_host(self.h, prob, g.ctypes.data_as(C.c_void_p), n,
                                          fit.ctypes.data_as(C.c_void_p), out))
        if topk:
            return fit, [(r.circuit, r.cost, r.fitness) for r in out[:k]]
        return fit

    def eval_host_ptr(self, prob, h_gates_ptr, n, h_fit_ptr, topk_buf=None):
        """qe_eval_host on raw host pointers (pinned buffers, for timing)."""
        return _check(self.h, lib().qe_eval_host(self.h, prob, C.c_void_p(h_gates_ptr), n,
                                                 C.c_void_p(h_fit_ptr), topk_buf))

    def _batch_args(self, items, topk):
        probs = [int(q) for q, _ in items]
        known = [p if 0 <= p < len(self._probs) else None for p in probs]
        gs = [np.ascontiguousarray(g, np.uint8) for _, g in items]
        gs = [g.reshape(-1, self._probs[q].circuit_len) if q is not None else g
              for q, g in zip(known, gs)]
        ns = [g.shape[0] for g in gs]
        flat = np.concatenate([g.ravel() for g in gs]) if gs else np.zeros(0, np.uint8)
        fp64 = known and known[0] is not None and \
            self._probs[known[0]].precision == QE_PREC_FP64
        fit = np.zeros(max(sum(ns), 1), np.float64 if fp64 else np.float32)
        ks = [min(max(self._probs[q].topk, 1), n) if q is not None else 0
              for q, n in zip(known, ns)]
        out = (qe_ranked * max(sum(ks), 1))() if topk else None
        u32a = C.c_uint32 * max(len(probs), 1)
        args = (len(probs), u32a(*probs), u32a(*ns),
                flat.ctypes.data_as(C.c_void_p) if flat.size else None,
                fit.ctypes.data_as(C.c_void_p), out)
        return args, (ns, ks, flat, fit, out, topk)

    @staticmethod
    def _batch_results(keep):
        ns, ks, _, fit, out, topk = keep
        fits, tops, fo, ko = [], [], 0, 0
        for n, k in zip(ns, ks):
            fits.append(fit[fo:fo + n].copy())
            if topk:
                tops.append([(r.circuit, r.cost, r.fitness) for r in out[ko:ko + k]])
            fo += n
            ko += k
        return (fits, tops) if topk else fits

    def eval_host_batch(self, items, topk=False):
        """qe_eval_host_batch: items = [(prob, gate_idx ndarray [n, L]), ...]; returns
        one fitness array per item and, with topk, one ranked list per item"""
        args, keep = self._batch_args(items, topk)
        _check(self.h, lib().qe_eval_host_batch(self.h, *args))
        return self._batch_results(keep)

    def eval_host_batch_async(self, items, topk=False):
        """qe_eval_host_batch_async: enqueues the call and returns a handle whose
        wait() returns what eval_host_batch returns (up to QE_BATCH_SLOTS calls
        in flight; the handle keeps the call's host buffers alive)"""
        args, keep = self._batch_args(items, topk)
        t = C.c_uint64()
        _check(self.h, lib().qe_eval_host_batch_async(self.h, *args, C.byref(t)))
        return BatchCall(self, t.value, keep)

    def eval_host_batch_ptr(self, probs_arr, n_arr, h_gates_ptr, h_fit_ptr, topk_buf=None):
        """qe_eval_host_batch on raw host pointers (pinned buffers, for timing);
        probs_arr / n_arr are ctypes uint32 arrays"""
        return _check(self.h, lib().qe_eval_host_batch(self.h, len(probs_arr), probs_arr, n_arr,
                                                       C.c_void_p(h_gates_ptr),
                                                       C.c_void_p(h_fit_ptr), topk_buf))

    def eval_host_batch_async_ptr(self, probs_arr, n_arr, h_gates_ptr, h_fit_ptr,
                                  topk_buf=None):
        """qe_eval_host_batch_async on raw host pointers; returns the ticket.  The
        buffers must stay alive and untouched until eval_host_batch_wait(ticket)."""
        # (integers pass as void * through the declared argument types)
        t = C.c_uint64()
        st = _lib.qe_eval_host_batch_async(self.h, len(probs_arr), probs_arr, n_arr, h_gates_ptr,
                                           h_fit_ptr, topk_buf, C.byref(t))
        if st != QE_OK:
            _check(self.h, st)
        return t.value

    def eval_host_batch_wait(self, ticket):
        """qe_eval_host_batch_wait: the call's fitness and top-k buffers are filled."""
        st = _lib.qe_eval_host_batch_wait(self.h, ticket)
        return st if st == QE_OK else _check(self.h, st)

    def compose(self, prob, gate_idx, unitary, n_circuits=None, amps=None):
        import torch
        p = self._probs[prob]
        n = gate_idx.shape[0] if n_circuits is None else n_circuits
        N = 1 << p.n_qubits
        dt = torch.float64 if p.precision == QE_PREC_FP64 else torch.float32
        _need(unitary, dt, n * N * N * 2, "unitary")
        _need(gate_idx, torch.uint8, n * p.circuit_len, "gate_idx")
        if amps is None:
            _check(self.h, lib().qe_compose(self.h, prob, _ptr(gate_idx), n, _ptr(unitary)))
        else:
            _need(amps, torch.float32, n * p.circuit_len * 2, "amps")
            _check(self.h, lib().qe_compose_amp(self.h, prob, _ptr(gate_idx), _ptr(amps), n,
                                                _ptr(unitary)))

    def update(self, prob, gen, seg_id, fitness):
        import torch
        p = self._probs[prob]
        _need(seg_id, torch.int32, p.population * p.circuit_len, "seg_id")
        _need(fitness, torch.float64, p.population, "fitness")
        _check(self.h, lib().qe_update(self.h, prob, gen, _ptr(seg_id), _ptr(fitness)))

    def step(self, n_gen=1, reports=True):
        rep = (qe_report * len(self.searches))() if reports else None
        st = lib().qe_step(self.h, n_gen, rep)
        if st not in (QE_OK, QE_ENUMERIC):
            _check(self.h, st)
        if not reports:
            return st
        out = []
        for r in rep:
            out.append(dict(generation=r.generation, best_gen=r.best_gen,
                            best_fitness=r.best_fitness, gen_best_fitness=r.gen_best_fitness,
                            mean_fitness=r.mean_fitness, useful_flops=r.useful_flops,
                            best_cost=r.best_cost, best_len=r.best_len, error_word=r.error_word,
                            best_gates=list(r.best_gates[:r.best_len]),
                            best_amps=list(r.best_amps[:2 * r.best_len]), status=st))
        return out

    def step_raw(self, n_gen, rep_buf):
        """qe_step into a preallocated qe_report array (for timing)."""
        return lib().qe_step(self.h, n_gen, rep_buf)

    def last_generation(self, prob):
        p = self._probs[prob]
        PL = p.population * p.circuit_len
        gi = np.zeros(PL, np.uint8)
        sid = np.zeros(PL, np.uint32)
        fit = np.zeros(p.population, np.float64)
        k = max(p.topk, 1)
        tk = (qe_ranked * k)()
        _check(self.h, lib().qe_last_generation(self.h, prob, gi.ctypes.data_as(C.c_void_p),
                                                sid.ctypes.data_as(C.c_void_p),
                                                fit.ctypes.data_as(C.c_void_p), tk))
        return dict(gate_idx=gi.reshape(p.population, p.circuit_len),
                    seg_id=sid.reshape(p.population, p.circuit_len), fitness=fit,
                    topk=[(r.circuit, r.cost, r.fitness) for r in tk])

    def state_bytes(self, prob):
        n = C.c_size_t()
        _check(self.h, lib().qe_state_bytes(self.h, prob, C.byref(n)))
        return n.value

    def get_state(self, prob):
        """QEQEA: (cur[S*8] f32, best[S*8] f32, best_f[S] f32); GA: genome [P, L] u8,
        on the Ising library (genome, angles [P, L, 2] f32)."""
        nb = self.state_bytes(prob)
        buf = np.zeros(nb, np.uint8)
        _check(self.h, lib().qe_get_state(self.h, prob, buf.ctypes.data_as(C.c_void_p), nb))
        p = self._probs[prob]
        if p.encoding == QE_ENC_GA:
            PL = p.population * p.circuit_len
            genome = buf[:PL].reshape(p.population, p.circuit_len).copy()
            if p.library == QE_LIB_ISING:
                return genome, buf[PL:].view(np.float32).reshape(p.population, p.circuit_len, 2)
            return genome
        S = nb // 68
        cur = buf[:32 * S].view(np.float32).copy()
        best = buf[32 * S:64 * S].view(np.float32).copy()
        bf = buf[64 * S:].view(np.float32).copy()
        return cur, best, bf

    def set_state(self, prob, cur, best=None, best_f=None):
        """QEQEA: set_state(prob, cur, best, best_f); GA: set_state(prob, genome),
        on the Ising library set_state(prob, genome, angles)."""
        p = self._probs[prob]
        if p.encoding == QE_ENC_GA:
            buf = np.ascontiguousarray(cur, np.uint8).ravel()
            if p.library == QE_LIB_ISING:
                buf = np.concatenate([buf, np.ascontiguousarray(best, np.float32).view(np.uint8).ravel()])
        else:
            buf = np.concatenate([np.ascontiguousarray(cur, np.float32).view(np.uint8).ravel(),
                                  np.ascontiguousarray(best, np.float32).view(np.uint8).ravel(),
                                  np.ascontiguousarray(best_f, np.float32).view(np.uint8).ravel()])
        _check(self.h, lib().qe_set_state(self.h, prob, buf.ctypes.data_as(C.c_void_p), buf.size))

    def set_target(self, prob, T):
        """qe_set_target: a dense N x N complex target unitary (None: the permutation)."""
        if T is None:
            _check(self.h, lib().qe_set_target(self.h, prob, None))
            return
        N = 1 << self._probs[prob].n_qubits
        T = np.asarray(T, np.complex128)
        if T.shape != (N, N):
            raise ValueError("target must be %d x %d" % (N, N))
        buf = np.ascontiguousarray(np.stack([T.real, T.imag], -1), np.float64)
        _check(self.h, lib().qe_set_target(self.h, prob, buf.ctypes.data_as(C.c_void_p)))

    def save(self, path):
        """qe_save: checkpoint every search (state, records, generation) to path."""
        _check(self.h, lib().qe_save(self.h, os.fsencode(path)))

    def load(self, path):
        """qe_load: resume the run saved at path (same problems as this context)."""
        _check(self.h, lib().qe_load(self.h, os.fsencode(path)))

    @classmethod
    def from_checkpoint(cls, path, stream=None):
        """A new context for the searches saved at path, resumed where they stopped."""
        probs, _ = checkpoint_info(path)
        ctx = cls(probs, stream)
        try:
            ctx.load(path)
        except Exception:
            ctx.close()
            raise
        return ctx

    def autotune(self, gens_per_plan=2):
        """qe_autotune: time every launch plan on real generations, keep the
        fastest; returns the mean generation time (ms) of each plan tried."""
        ms = (C.c_float * 16)()
        n = C.c_uint32(16)
        _check(self.h, lib().qe_autotune(self.h, gens_per_plan, ms, C.byref(n)))
        return list(ms[:n.value])

    def launch_plan(self):
        b = C.create_string_buffer(256)
        _check(self.h, lib().qe_launch_plan(self.h, b, 256))
        return b.value.decode()

    def stage_timing(self, enable=True, serial=False):
        """events between the generation's kernels; serial=True runs them all on
        one stream (each interval is that stage's own duration)"""
        mode = 0 if not enable else (2 if serial else 1)
        _check(self.h, lib().qe_stage_timing(self.h, mode))

    def stage_times(self):
        """ms of the last generation: circuits, select, rescore, sort, update, whole"""
        ms = (C.c_float * 6)()
        _check(self.h, lib().qe_stage_times(self.h, ms))
        return list(ms)

    def generation(self):
        g = C.c_uint32()
        _check(self.h, lib().qe_generation(self.h, C.byref(g)))
        return g.value


def measure_alu_peaks():
    """(binary32, binary64) FMA throughput of the current GPU, TFLOP/s."""
    a, b = C.c_double(), C.c_double()
    _check(None, lib().qe_measure_alu_peaks(C.byref(a), C.byref(b)))
    return a.value, b.value


def qe_eval_rank_static(search, gate_idx, fitness, topk=None, n_circuits=None, stream=None):
    """Context-free evaluation + ranking that allocates no device memory.

    gate_idx, fitness and topk (a CUDA uint8 tensor of 16-byte qe_ranked
    records, or None) are device tensors; the call is asynchronous on `stream`.
    For callers that may not allocate while it runs, every buffer must exist
    beforehand; see include/qe.h for the limits and the race between
    overlapping calls."""
    import torch
    p = to_problem(search)
    n = gate_idx.shape[0] if n_circuits is None else n_circuits
    if n > 0:
        _need(gate_idx, torch.uint8, n * p.circuit_len, "gate_idx")
        _need(fitness, torch.float64 if p.precision == QE_PREC_FP64 else torch.float32, n,
              "fitness")
        if topk is not None:
            _need(topk, torch.uint8, 16 * min(max(p.topk, 1), n), "topk")
    msg = C.create_string_buffer(256)
    st = lib().qe_eval_rank_static(C.byref(p), _ptr(gate_idx), n, _ptr(fitness), _ptr(topk),
                                   _stream_handle(stream), msg, 256)
    if st != QE_OK:
        raise QeError(st, msg.value.decode())


# ABI-named entry points (same names as include/qe.h)
def qe_init(searches, stream=None) -> Context:
    return Context(searches, stream)


def qe_sample(ctx: Context, prob, gen, gate_idx, seg_id):
    return ctx.sample(prob, gen, gate_idx, seg_id)


def qe_eval(ctx: Context, prob, gate_idx, fitness, n_circuits=None, cost=None, topk=False):
    return ctx.eval(prob, gate_idx, fitness, n_circuits, cost, topk)


def qe_rank(ctx: Context, prob, gate_idx, fitness, cost, n_circuits=None, amps=None):
    return ctx.rank(prob, gate_idx, fitness, cost, n_circuits, amps)


def qe_eval_host(ctx: Context, prob, gate_idx, topk=False):
    return ctx.eval_host(prob, gate_idx, topk)


def qe_eval_host_batch(ctx: Context, items, topk=False):
    return ctx.eval_host_batch(items, topk)


def qe_compose(ctx: Context, prob, gate_idx, unitary, n_circuits=None):
    return ctx.compose(prob, gate_idx, unitary, n_circuits)


def qe_update(ctx: Context, prob, gen, seg_id, fitness):
    return ctx.update(prob, gen, seg_id, fitness)


def checkpoint_info(path):
    """qe_checkpoint_info: ([qe_problem], generation) of a checkpoint file; no GPU needed."""
    n, gen = C.c_uint32(), C.c_uint32()
    _check(None, lib().qe_checkpoint_info(os.fsencode(path), None, 0, C.byref(n), C.byref(gen)))
    arr = (qe_problem * n.value)()
    _check(None, lib().qe_checkpoint_info(os.fsencode(path), arr, n.value, C.byref(n), C.byref(gen)))
    return list(arr), gen.value


def qe_step(ctx: Context, n_gen=1):
    return ctx.step(n_gen)


def qe_last_generation(ctx: Context, prob):
    return ctx.last_generation(prob)


def qe_get_state(ctx: Context, prob):
    return ctx.get_state(prob)


def qe_set_state(ctx: Context, prob, cur, best=None, best_f=None):
    return ctx.set_state(prob, cur, best, best_f)


def qe_destroy(ctx: Context):
    ctx.close()
