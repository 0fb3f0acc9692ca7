"""Seeded synthetic inputs: targets, search shapes, gate strings and encoding states.

This module holds no arithmetic of the method itself.  It only builds the
inputs that both the CUDA path and the CPU oracle consume: target permutations
(T|j> = |perm[j]>), the parameters of the five benchmark searches, random gate
strings and random encoding states.  It imports neither torch nor the CUDA
library, so CPU-only tests can use it.

Wire w is bit (n-1-w) of a basis index (wire 0 = most significant bit).
"""
from dataclasses import dataclass, field
from typing import List, Optional

import numpy as np

LIB_NCV, LIB_HT, LIB_IDENTITY, LIB_ISING = 1, 2, 4, 8
PREC_FP64, PREC_FP32, PREC_SPLIT_TC = 0, 1, 2
FIT_TRACE, FIT_PROB = 0, 1
ENC_QEQEA, ENC_GA = 0, 1


def _bit(x, n, w):
    return (x >> (n - 1 - w)) & 1


def cknot(n: int) -> List[int]:
    """C^{n-1}NOT with the target on wire 0 and controls on wires 1..n-1.

    This is the orientation of the paper's Toffoli matrix (Table 2), whose
    only off-diagonal pair is basis states 3 and 7: the most significant bit
    flips when all lower bits are 1.
    """
    N = 1 << n
    perm = list(range(N))
    lo = (1 << (n - 1)) - 1
    hi = N - 1
    perm[lo], perm[hi] = hi, lo
    return perm


def peres() -> List[int]:
    """Peres gate on wires (a, b, c) = (0, 1, 2): (a, b, c) -> (a, a^b, c ^ ab)."""
    perm = []
    for x in range(8):
        a, b, c = _bit(x, 3, 0), _bit(x, 3, 1), _bit(x, 3, 2)
        b2, c2 = a ^ b, c ^ (a & b)
        perm.append((a << 2) | (b2 << 1) | c2)
    return perm


def fredkin() -> List[int]:
    """Fredkin gate: wire 0 controls a swap of wires 1 and 2."""
    perm = []
    for x in range(8):
        a, b, c = _bit(x, 3, 0), _bit(x, 3, 1), _bit(x, 3, 2)
        if a:
            b, c = c, b
        perm.append((a << 2) | (b << 1) | c)
    return perm


def random_perm(rng: np.random.Generator, n: int) -> List[int]:
    return [int(v) for v in rng.permutation(1 << n)]


@dataclass
class Search:
    """Parameters of one independent search (one entry of qe_problem)."""
    n: int
    L: int
    P: int
    library: int
    perm: List[int]
    seed: int = 0
    precision: int = PREC_FP32
    fitness_kind: int = FIT_TRACE
    topk: int = 0
    p_mutation: float = 0.1
    mutation_range: float = float(np.pi / 4)
    ga_mutation_rate: float = 0.02
    cost_weight: float = 0.0
    shots: int = 1  # qutrit measurements per slot, majority outcome taken
    target: Optional[np.ndarray] = None  # dense N x N target unitary instead of perm
    name: str = field(default="")
    encoding: int = ENC_QEQEA


def config(k: int, precision: int = None, P: int = None, seed: int = None,
           encoding: int = None, library: int = None) -> List[Search]:
    """The five benchmark searches (3-5 qubit permutation targets).

    1: 3-qubit Toffoli, NCV + identity (19 gates), L=5, P=64, FP64, seed 0
    2: 3-qubit Toffoli / Fredkin / Peres, NCV + H/T/T^dag + identity (28 gates),
       L=16, P=4096, Philox seed 1, FP32 with FP64 top-32
    3: 4-qubit C3NOT, NCV + H/T/T^dag (48 gates), L=32, P=65536, top-64
    4: 1024 uneven searches, n in {3,4,5}, L in [8,64], P in [256,4096],
       uniform random permutation targets (seed 2), top-32
    5: 5-qubit C4NOT, NCV + H/T/T^dag (75 gates), L=64, P=262144, top-128

    encoding=ENC_GA turns every search into the classical GA on the same
    shapes (integer genomes, per-gene mutation rate 0.02); library=LIB_ISING
    runs the same shapes on the paper's Ising gate set.
    """
    full = LIB_NCV | LIB_HT
    if k == 1:
        s = [Search(3, 5, 64, LIB_NCV | LIB_IDENTITY, cknot(3), seed=0, precision=PREC_FP64,
                    topk=0, name="toffoli")]
    elif k == 2:
        lib = full | LIB_IDENTITY
        s = [Search(3, 16, 4096, lib, cknot(3), seed=1, topk=32, name="toffoli"),
             Search(3, 16, 4096, lib, fredkin(), seed=1, topk=32, name="fredkin"),
             Search(3, 16, 4096, lib, peres(), seed=1, topk=32, name="peres")]
    elif k == 3:
        s = [Search(4, 32, 65536, full, cknot(4), seed=3, topk=64, name="c3not")]
    elif k == 4:
        rng = np.random.default_rng(2)
        s = []
        for run in range(1024):
            n = int(rng.integers(3, 6))
            L = int(rng.integers(8, 65))
            P = int(rng.integers(256, 4097))
            s.append(Search(n, L, P, full, random_perm(rng, n), seed=2, topk=32,
                            name="rand%d" % run))
    elif k == 5:
        s = [Search(5, 64, 262144, full, cknot(5), seed=5, topk=128, name="c4not")]
    else:
        raise ValueError("configs are 1..5")
    for x in s:
        if precision is not None:
            x.precision = precision
        if P is not None:
            x.P = min(x.P, P)
        if seed is not None:
            x.seed = seed
        if encoding is not None:
            x.encoding = encoding
        if library is not None:
            x.library = library
    return s


def random_gates(rng: np.random.Generator, n_circuits: int, L: int, G: int) -> np.ndarray:
    """Uniform gate strings, shape [n_circuits, L], uint8 library indices < G."""
    return rng.integers(0, G, size=(n_circuits, L), dtype=np.uint8)


def random_state(rng: np.random.Generator, n_segments: int, best_f_range=(-1.0, 1.0)):
    """Random encoding state: per segment 8 floats {q0re,q0im,q1re,q1im,q2re,q2im,b0,b1}.

    Qutrits are normalised complex Gaussian vectors, qubits random real unit
    vectors; best_f is uniform in best_f_range (float32)."""
    S = n_segments
    z = rng.standard_normal((S, 3, 2))
    z /= np.sqrt((z ** 2).sum(axis=(1, 2), keepdims=True))
    ang = rng.uniform(0, 2 * np.pi, S)
    cur = np.empty((S, 8), np.float32)
    cur[:, :6] = z.reshape(S, 6)
    cur[:, 6] = np.cos(ang)
    cur[:, 7] = np.sin(ang)
    z2 = rng.standard_normal((S, 3, 2))
    z2 /= np.sqrt((z2 ** 2).sum(axis=(1, 2), keepdims=True))
    best = np.empty((S, 8), np.float32)
    best[:, :6] = z2.reshape(S, 6)
    ang2 = rng.uniform(0, 2 * np.pi, S)
    best[:, 6] = np.cos(ang2)
    best[:, 7] = np.sin(ang2)
    best_f = rng.uniform(best_f_range[0], best_f_range[1], S).astype(np.float32)
    return cur.ravel(), best.ravel(), best_f


def random_fitness(rng: np.random.Generator, P: int, discrete: bool = True) -> np.ndarray:
    """Fitness arrays for update tests; discrete=True makes ties likely."""
    if discrete:
        return rng.integers(0, 17, P).astype(np.float64) / 16.0
    return rng.uniform(0.0, 1.0, P)
