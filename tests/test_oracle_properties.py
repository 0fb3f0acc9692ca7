"""Property-based pins of the oracle's composition (Sec. IV-C), over random
gate strings of every width and both discrete libraries (CPU only):

* composition order: the circuit g1 followed by g2 composes to S(g2) S(g1)
  (a later gate multiplies from the left; an implementation that multiplied
  in the other order, or transposed a gate, fails on non-commuting strings);
* every circuit followed by its gates' inverses in reverse order composes to
  the identity, whose fitness against the identity permutation is exactly 1
  (Eq. (11)); the inverse of each library gate is found by search, not from
  the oracle's own tables;
* a global phase of a dense target does not change Eq. (11)'s fitness.
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings
from hypothesis import strategies as st

import oracle
from paper_1809_11134_gb300 import workloads as W

LIBS = [W.LIB_NCV | W.LIB_HT, W.LIB_NCV | W.LIB_HT | W.LIB_IDENTITY]


def _S(n, lib, g):
    re, im = oracle.compose(n, lib, np.asarray(g, np.uint8))
    return re + 1j * im


_inv_cache = {}


def _inverses(n, lib):
    """gate index -> the library gate whose product with it is the identity"""
    key = (n, lib)
    if key not in _inv_cache:
        G = oracle.num_gates(n, lib)
        eye = np.eye(1 << n)
        inv = []
        for a in range(G):
            for b in range(G):
                if np.abs(_S(n, lib, [a, b]) - eye).max() < 1e-12:
                    inv.append(b)
                    break
            else:
                raise AssertionError("gate %d has no inverse in the library" % a)
        _inv_cache[key] = inv
    return _inv_cache[key]


circuits = st.tuples(st.integers(1, 5), st.sampled_from(LIBS), st.integers(0, 2 ** 31 - 1),
                     st.integers(0, 12), st.integers(0, 12))


@settings(max_examples=60, deadline=None, derandomize=True)
@given(circuits)
def test_composition_is_the_ordered_product(case):
    n, lib, seed, a, b = case
    rng = np.random.default_rng(seed)
    G = oracle.num_gates(n, lib)
    g1 = rng.integers(0, G, a).astype(np.uint8)
    g2 = rng.integers(0, G, b).astype(np.uint8)
    S12 = _S(n, lib, np.concatenate([g1, g2]))
    assert np.abs(S12 - _S(n, lib, g2) @ _S(n, lib, g1)).max() < 1e-12


@settings(max_examples=60, deadline=None, derandomize=True)
@given(circuits)
def test_circuit_then_its_inverse_is_the_identity(case):
    n, lib, seed, a, _ = case
    rng = np.random.default_rng(seed)
    G = oracle.num_gates(n, lib)
    inv = _inverses(n, lib)
    g = rng.integers(0, G, a).astype(np.uint8)
    back = np.array([inv[x] for x in g[::-1]], np.uint8)
    S = _S(n, lib, np.concatenate([g, back]))
    assert np.abs(S - np.eye(1 << n)).max() < 1e-12
    assert oracle.score(n, S, list(range(1 << n))) == pytest.approx(1.0, abs=1e-12)


@settings(max_examples=40, deadline=None, derandomize=True)
@given(circuits, st.floats(0.0, 2 * np.pi))
def test_dense_fitness_ignores_a_global_phase(case, alpha):
    n, lib, seed, a, b = case
    rng = np.random.default_rng(seed)
    G = oracle.num_gates(n, lib)
    S = _S(n, lib, rng.integers(0, G, a).astype(np.uint8))
    T = _S(n, lib, rng.integers(0, G, b).astype(np.uint8))
    f0 = oracle.score_dense(n, S, T)
    f1 = oracle.score_dense(n, S, T * np.exp(1j * alpha))
    # Eq. (11) takes 1 - sqrt(d) with d = (N - |tr|) / N: the phase moves |tr|
    # by a few rounding errors of an N-term sum, which the square root
    # magnifies to sqrt(|delta d|) near d = 0 (e.g. S = T = I gives 1.5e-8)
    N = 1 << n
    assert abs(f0 - f1) <= np.sqrt(16 * N * np.finfo(float).eps)
    assert 0.0 <= f0 <= 1.0 + 1e-12


def _order_holds(cases=40):
    rng = np.random.default_rng(3)
    for _ in range(cases):
        n = int(rng.integers(1, 6))
        lib = LIBS[int(rng.integers(0, 2))]
        G = oracle.num_gates(n, lib)
        g1 = rng.integers(0, G, int(rng.integers(1, 8))).astype(np.uint8)
        g2 = rng.integers(0, G, int(rng.integers(1, 8))).astype(np.uint8)
        S12 = _S(n, lib, np.concatenate([g1, g2]))
        if np.abs(S12 - _S(n, lib, g2) @ _S(n, lib, g1)).max() >= 1e-12:
            return False
    return True


def test_order_check_passes_on_the_oracle():
    assert _order_holds()


def test_order_check_catches_a_reversed_product(tmp_path):
    """the oracle compiled with S <- S G_t instead of S <- G_t S fails it"""
    import os
    from oracle import build as obuild
    src = open(os.path.join(os.path.dirname(oracle.__file__), "qe_oracle.c")).read()
    old = "matmul(N, G, S, T); /* S <- G_t S */"
    assert src.count(old) == 1, "the line to plant in is gone"
    path = obuild.build_variant(src.replace(old, "matmul(N, S, G, T);"),
                                str(tmp_path / "liboracle_planted.so"))
    with oracle.using(oracle.load(path)):
        assert not _order_holds()
