"""ctypes front end of the FP64 CPU oracle (TEST INFRASTRUCTURE ONLY).

Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
reference legs import this package.  It never imports the CUDA library and
the CUDA library never imports it.  Arrays are numpy, on the host.
"""
import contextlib
import ctypes as C
import os

import numpy as np

from . import build as _build

LIB_NCV, LIB_HT, LIB_IDENTITY, LIB_ISING = 1, 2, 4, 8
I, CNOT, CV, CVDG, H, T, TDG, RX, RY, RZ, J = range(11)
FIT_TRACE, FIT_PROB = 0, 1
Q = 4096

_u8p = np.ctypeslib.ndpointer(np.uint8, flags="C_CONTIGUOUS")
_u32p = np.ctypeslib.ndpointer(np.uint32, flags="C_CONTIGUOUS")
_f32p = np.ctypeslib.ndpointer(np.float32, flags="C_CONTIGUOUS")
_f64p = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


class Problem(C.Structure):
    _fields_ = [("n", C.c_uint32), ("L", C.c_uint32), ("P", C.c_uint32), ("library", C.c_uint32),
                ("fitness_kind", C.c_uint32), ("run", C.c_uint32), ("seed", C.c_uint64),
                ("p_mutation", C.c_double), ("mutation_range", C.c_double),
                ("cost_weight", C.c_double), ("perm", C.c_uint8 * 32), ("shots", C.c_uint32),
                ("target", C.POINTER(C.c_double))]


class Report(C.Structure):
    _fields_ = [("generation", C.c_uint32), ("best_circuit", C.c_uint32),
                ("best_fitness", C.c_double), ("gen_best_fitness", C.c_double),
                ("mean_fitness", C.c_double), ("useful_flops", C.c_uint64),
                ("best_cost", C.c_uint32), ("best_gen", C.c_uint32),
                ("best_gates", C.c_uint8 * 64), ("best_amps", C.c_float * 128)]


_lib = None


def lib():
    global _lib
    if _lib is None:
        _lib = _configure(C.CDLL(_build.build()))
    return _lib


def load(path):
    """A handle of an oracle library built from another copy of the source
    (tests plant a mistake in a copy to check that the pins catch it)."""
    return _configure(C.CDLL(path))


@contextlib.contextmanager
def using(handle):
    """Route every function of this module through `handle` inside the block."""
    global _lib
    saved = lib()
    _lib = handle
    try:
        yield handle
    finally:
        _lib = saved


def _configure(L):
    L.oracle_philox4x32_10.argtypes = [_u32p, _u32p, _u32p]
    L.oracle_num_gates.argtypes = [C.c_uint32, C.c_uint32]
    L.oracle_num_gates.restype = C.c_uint32
    L.oracle_num_regions.argtypes = [C.c_uint32, C.c_uint32]
    L.oracle_num_regions.restype = C.c_uint32
    L.oracle_gate_desc.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.POINTER(C.c_int),
                                   C.POINTER(C.c_int), C.POINTER(C.c_int)]
    L.oracle_gate_desc.restype = C.c_int
    L.oracle_region_gate.argtypes = [C.c_uint32] * 4
    L.oracle_region_gate.restype = C.c_uint32
    L.oracle_segment_index.argtypes = [C.c_uint64] * 5
    L.oracle_segment_index.restype = C.c_uint64
    L.oracle_num_segments.argtypes = [C.POINTER(Problem)]
    L.oracle_num_segments.restype = C.c_uint64
    L.oracle_gate_matrix.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, _f64p, _f64p]
    L.oracle_half_angle.argtypes = [C.c_float, C.c_float, C.POINTER(C.c_double),
                                    C.POINTER(C.c_double)]
    L.oracle_gate_matrix_amp.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, C.c_float,
                                         C.c_float, _f64p, _f64p]
    L.oracle_compose_amp.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, _u8p, _f32p, _f64p,
                                     _f64p]
    L.oracle_eval_amp.argtypes = [C.POINTER(Problem), _u8p, _f32p, C.c_uint32, _f64p, _u32p]
    L.oracle_sample_amp.argtypes = [C.POINTER(Problem), _f32p, C.c_uint32, _u8p, _u32p,
                                    _f32p]
    L.oracle_compose.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, _u8p, _f64p, _f64p]
    L.oracle_score.argtypes = [C.c_uint32, _f64p, _f64p, _u8p, C.c_uint32]
    L.oracle_score_dense.argtypes = [C.c_uint32, _f64p, _f64p, _f64p]
    L.oracle_score_dense.restype = C.c_double
    L.oracle_score.restype = C.c_double
    L.oracle_cost.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, _u8p]
    L.oracle_cost.restype = C.c_uint32
    L.oracle_eval.argtypes = [C.POINTER(Problem), _u8p, C.c_uint32, _f64p, _u32p]
    L.oracle_useful_flops.argtypes = [C.c_uint32, C.c_uint32, C.c_uint32, _u8p]
    L.oracle_useful_flops.restype = C.c_uint64
    L.oracle_init_state.argtypes = [C.POINTER(Problem), _f32p, _f32p, _f32p]
    L.oracle_sample.argtypes = [C.POINTER(Problem), _f32p, C.c_uint32, _u8p, _u32p]
    L.oracle_update.argtypes = [C.POINTER(Problem), _f32p, _f32p, _f32p, C.c_uint32, _u32p,
                                _f64p]
    L.oracle_su3.argtypes = [_f64p, _f64p, _f64p, _f64p]
    L.oracle_su3_f32.argtypes = [_f32p, _f32p, _f32p, _f32p]
    L.oracle_su3_angles.argtypes = [_f64p, _f64p, _f64p]
    L.oracle_topk.argtypes = [_f64p, _u32p, C.c_uint32, C.c_uint32, _u32p]
    L.oracle_step.argtypes = [C.POINTER(Problem), _f32p, _f32p, _f32p, C.c_uint32,
                              C.c_uint32, _u8p, _u32p, _f64p, _u32p, _u32p,
                              C.POINTER(Report)]
    L.oracle_ga_init.argtypes = [C.POINTER(Problem), C.c_uint32, _u8p]
    L.oracle_ga_init_amp.argtypes = [C.POINTER(Problem), C.c_uint32, _u8p, _f32p]
    L.oracle_ga_next_amp.argtypes = [C.POINTER(Problem), C.c_uint32, C.c_uint32, C.c_double,
                                     _u8p, _f32p, _f64p, _u32p, _u8p, _f32p]
    L.oracle_ga_next.argtypes = [C.POINTER(Problem), C.c_uint32, C.c_uint32, C.c_double,
                                 _u8p, _f64p, _u32p, _u8p]
    return L


def make_problem(n, L, P, library, perm, seed=0, run=0, fitness_kind=FIT_TRACE, p_mutation=0.1,
                 mutation_range=np.pi / 4, cost_weight=0.0, shots=1, target=None):
    """target: a dense N x N complex target unitary (Eq. (11)), else the permutation perm"""
    p = Problem()
    p.shots = shots
    if target is not None:
        t = np.ascontiguousarray(np.stack([np.real(target), np.imag(target)], -1), np.float64)
        p._target = t  # kept alive with the problem
        p.target = t.ctypes.data_as(C.POINTER(C.c_double))
    p.n, p.L, p.P, p.library, p.fitness_kind, p.run = n, L, P, library, fitness_kind, run
    p.seed = seed
    p.p_mutation, p.mutation_range, p.cost_weight = p_mutation, mutation_range, cost_weight
    perm = list(perm)
    for j in range(32):
        p.perm[j] = perm[j] if j < len(perm) else 0
    return p


def philox(ctr, key):
    out = np.zeros(4, np.uint32)
    lib().oracle_philox4x32_10(np.asarray(ctr, np.uint32), np.asarray(key, np.uint32), out)
    return out


def num_gates(n, library):
    return lib().oracle_num_gates(n, library)


def num_regions(n, library):
    return lib().oracle_num_regions(n, library)


def gate_desc(n, library, g):
    k, c, t = C.c_int(), C.c_int(), C.c_int()
    rc = lib().oracle_gate_desc(n, library, g, C.byref(k), C.byref(c), C.byref(t))
    if rc != 0:
        raise IndexError(g)
    return k.value, c.value, t.value


def region_gate(n, library, r, k):
    return lib().oracle_region_gate(n, library, r, k)


def segment_index(r, i, t, L, P):
    return lib().oracle_segment_index(r, i, t, L, P)


def num_segments(p):
    return lib().oracle_num_segments(C.byref(p))


def gate_matrix(n, library, g):
    N = 1 << n
    re = np.zeros(N * N)
    im = np.zeros(N * N)
    lib().oracle_gate_matrix(n, library, g, re, im)
    return (re + 1j * im).reshape(N, N)


def half_angle(b0, b1):
    c, s = C.c_double(), C.c_double()
    lib().oracle_half_angle(b0, b1, C.byref(c), C.byref(s))
    return c.value, s.value


def gate_matrix_amp(n, library, g, b0, b1):
    N = 1 << n
    re = np.zeros(N * N)
    im = np.zeros(N * N)
    lib().oracle_gate_matrix_amp(n, library, g, b0, b1, re, im)
    return (re + 1j * im).reshape(N, N)


def compose(n, library, gates, amps=None):
    """amps: the slots' qubit amplitudes, shape [L, 2] float32 (Ising library)"""
    N = 1 << n
    g = np.ascontiguousarray(gates, np.uint8)
    re = np.zeros(N * N)
    im = np.zeros(N * N)
    if amps is None:
        lib().oracle_compose(n, library, len(g), g, re, im)
    else:
        a = np.ascontiguousarray(amps, np.float32).ravel()
        lib().oracle_compose_amp(n, library, len(g), g, a, re, im)
    return re.reshape(N, N), im.reshape(N, N)


def score(n, S, perm, kind=FIT_TRACE):
    S = np.asarray(S, np.complex128)
    re = np.ascontiguousarray(S.real.ravel())
    im = np.ascontiguousarray(S.imag.ravel())
    return lib().oracle_score(n, re, im, np.ascontiguousarray(perm, np.uint8), kind)


def score_dense(n, S, T):
    """Eq. (11) against a dense target T (N x N complex)"""
    S = np.asarray(S, np.complex128)
    t = np.ascontiguousarray(np.stack([np.real(T), np.imag(T)], -1), np.float64).ravel()
    return lib().oracle_score_dense(n, np.ascontiguousarray(S.real.ravel()),
                                    np.ascontiguousarray(S.imag.ravel()), t)


def cost(n, library, gates):
    g = np.ascontiguousarray(gates, np.uint8)
    return lib().oracle_cost(n, library, len(g), g)


def useful_flops(n, library, gates):
    g = np.ascontiguousarray(gates, np.uint8)
    return lib().oracle_useful_flops(n, library, len(g), g)


def eval_circuits(p, gates, amps=None):
    """amps: [n, L, 2] float32 slot amplitudes (Ising library), else None"""
    g = np.ascontiguousarray(gates, np.uint8).reshape(-1, p.L)
    nc = g.shape[0]
    F = np.zeros(max(nc, 1))
    cost_ = np.zeros(max(nc, 1), np.uint32)
    gp = g.ravel() if nc else np.zeros(1, np.uint8)
    if amps is None:
        lib().oracle_eval(C.byref(p), gp, nc, F, cost_)
    else:
        a = np.ascontiguousarray(amps, np.float32).ravel()
        lib().oracle_eval_amp(C.byref(p), gp, a if nc else np.zeros(2, np.float32), nc, F, cost_)
    return F[:nc], cost_[:nc]


def init_state(p):
    S = num_segments(p)
    cur = np.zeros(8 * max(S, 1), np.float32)
    best = np.zeros(8 * max(S, 1), np.float32)
    bf = np.zeros(max(S, 1), np.float32)
    lib().oracle_init_state(C.byref(p), cur, best, bf)
    return cur[:8 * S], best[:8 * S], bf[:S]


def sample(p, cur, gen, with_amps=False):
    gi = np.zeros(p.P * p.L, np.uint8)
    sid = np.zeros(p.P * p.L, np.uint32)
    if not with_amps:
        lib().oracle_sample(C.byref(p), np.ascontiguousarray(cur, np.float32), gen, gi, sid)
        return gi.reshape(p.P, p.L), sid.reshape(p.P, p.L)
    amps = np.zeros(2 * p.P * p.L, np.float32)
    lib().oracle_sample_amp(C.byref(p), np.ascontiguousarray(cur, np.float32), gen, gi, sid, amps)
    return gi.reshape(p.P, p.L), sid.reshape(p.P, p.L), amps.reshape(p.P, p.L, 2)


def update(p, cur, best, best_f, gen, seg_id, fitness):
    """In place on cur/best/best_f (numpy arrays)."""
    assert cur.dtype == np.float32 and best.dtype == np.float32 and best_f.dtype == np.float32
    lib().oracle_update(C.byref(p), cur, best, best_f, gen,
                        np.ascontiguousarray(seg_id, np.uint32).ravel(),
                        np.ascontiguousarray(fitness, np.float64))


def su3(cosv, sinv):
    Ur = np.zeros(9)
    Ui = np.zeros(9)
    lib().oracle_su3(np.ascontiguousarray(cosv, np.float64), np.ascontiguousarray(sinv, np.float64),
                     Ur, Ui)
    return (Ur + 1j * Ui).reshape(3, 3)


def su3_f32(cosv, sinv):
    Ur = np.zeros(9, np.float32)
    Ui = np.zeros(9, np.float32)
    lib().oracle_su3_f32(np.ascontiguousarray(cosv, np.float32),
                         np.ascontiguousarray(sinv, np.float32), Ur, Ui)
    return (Ur.astype(np.float64) + 1j * Ui).reshape(3, 3)


def su3_angles(params):
    Ur = np.zeros(9)
    Ui = np.zeros(9)
    lib().oracle_su3_angles(np.ascontiguousarray(params, np.float64), Ur, Ui)
    return (Ur + 1j * Ui).reshape(3, 3)


def topk(F, cost_, k):
    F = np.ascontiguousarray(F, np.float64)
    idx = np.zeros(max(k, 1), np.uint32)
    lib().oracle_topk(F, np.ascontiguousarray(cost_, np.uint32), len(F), k, idx)
    return idx[:min(k, len(F))]


def new_report():
    r = Report()
    r.best_fitness = -1e308
    r.best_cost = 0xFFFFFFFF
    return r


def step(p, cur, best, best_f, gen, k, rep):
    gi = np.zeros(p.P * p.L, np.uint8)
    sid = np.zeros(p.P * p.L, np.uint32)
    F = np.zeros(p.P)
    cost_ = np.zeros(p.P, np.uint32)
    tk = np.zeros(max(k, 1), np.uint32)
    lib().oracle_step(C.byref(p), cur, best, best_f, gen, k, gi, sid, F, cost_, tk, C.byref(rep))
    return gi.reshape(p.P, p.L), sid.reshape(p.P, p.L), F, cost_, tk[:max(k, 1)]


def ga_init(p, G):
    g = np.zeros(p.P * p.L, np.uint8)
    lib().oracle_ga_init(C.byref(p), G, g)
    return g.reshape(p.P, p.L)


def ga_init_amp(p, G):
    g = np.zeros(p.P * p.L, np.uint8)
    a = np.zeros(2 * p.P * p.L, np.float32)
    lib().oracle_ga_init_amp(C.byref(p), G, g, a)
    return g.reshape(p.P, p.L), a.reshape(p.P, p.L, 2)


def ga_next_amp(p, G, gen, rate, genome, amps, F, cost_):
    out = np.zeros(p.P * p.L, np.uint8)
    oa = np.zeros(2 * p.P * p.L, np.float32)
    lib().oracle_ga_next_amp(C.byref(p), G, gen, rate,
                             np.ascontiguousarray(genome, np.uint8).ravel(),
                             np.ascontiguousarray(amps, np.float32).ravel(),
                             np.ascontiguousarray(F, np.float64),
                             np.ascontiguousarray(cost_, np.uint32), out, oa)
    return out.reshape(p.P, p.L), oa.reshape(p.P, p.L, 2)


def ga_next(p, G, gen, rate, genome, F, cost_):
    out = np.zeros(p.P * p.L, np.uint8)
    lib().oracle_ga_next(C.byref(p), G, gen, rate, np.ascontiguousarray(genome, np.uint8).ravel(),
                         np.ascontiguousarray(F, np.float64), np.ascontiguousarray(cost_, np.uint32),
                         out)
    return out.reshape(p.P, p.L)
