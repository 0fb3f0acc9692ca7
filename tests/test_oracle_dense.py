"""Pins of the oracle's dense-target fitness: Eq. (11) with a general unitary
T, f = 1 - sqrt((N - |tr(S^dag T)|) / N).  Closed forms: T = S and T = e^{ia} S
score 1; T = S Z_w (a Pauli Z on one wire) scores 0 because tr(Z_w) = 0;
T = S D with D diagonal scores through |tr D| alone; a permutation matrix as a
dense target gives exactly the permutation path's fitness."""
import numpy as np
import pytest

import oracle
from paper_1809_11134_gb300 import workloads as W

LIB = W.LIB_NCV | W.LIB_HT


def circuit(rng, n, L=12, lib=LIB):
    g = rng.integers(0, oracle.num_gates(n, lib), L).astype(np.uint8)
    re, im = oracle.compose(n, lib, g)
    return g, re + 1j * im


def f_of(tr_abs, N):
    return 1 - np.sqrt(max(0.0, (N - tr_abs) / N))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_self_and_global_phase_score_one(n):
    rng = np.random.default_rng(n)
    _, S = circuit(rng, n)
    assert oracle.score_dense(n, S, S) == pytest.approx(1.0, abs=1e-7)
    assert oracle.score_dense(n, S, np.exp(0.7j) * S) == pytest.approx(1.0, abs=1e-7)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_traceless_and_diagonal_factors(n):
    rng = np.random.default_rng(10 + n)
    _, S = circuit(rng, n)
    N = 1 << n
    for w in range(n):
        z = np.array([1 - 2 * ((j >> (n - 1 - w)) & 1) for j in range(N)], np.float64)
        assert oracle.score_dense(n, S, S @ np.diag(z)) == pytest.approx(0.0, abs=1e-7)
    ph = rng.uniform(0, 2 * np.pi, N)
    D = np.diag(np.exp(1j * ph))
    want = f_of(abs(np.exp(1j * ph).sum()), N)
    assert oracle.score_dense(n, S, S @ D) == pytest.approx(want, abs=1e-7)


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5])
def test_permutation_matrix_equals_the_permutation_path(n):
    rng = np.random.default_rng(20 + n)
    N = 1 << n
    for _ in range(5):
        perm = rng.permutation(N)
        T = np.zeros((N, N))
        T[perm, np.arange(N)] = 1.0  # T|j> = |perm[j]>
        _, S = circuit(rng, n, L=20)
        assert oracle.score_dense(n, S, T) == oracle.score(n, S, perm)


def test_eval_and_step_use_the_dense_target():
    """oracle_eval with a dense target = score_dense of each composed circuit; the
    permutation fields are then ignored; the reported flops count the dense score."""
    rng = np.random.default_rng(3)
    n, L, P = 3, 10, 40
    N = 1 << n
    q, _ = np.linalg.qr(rng.normal(size=(N, N)) + 1j * rng.normal(size=(N, N)))
    p = oracle.make_problem(n, L, P, LIB, W.cknot(n), seed=2, target=q)
    gates = rng.integers(0, oracle.num_gates(n, LIB), (P, L)).astype(np.uint8)
    F, C = oracle.eval_circuits(p, gates)
    for c in range(P):
        re, im = oracle.compose(n, LIB, gates[c])
        assert F[c] == oracle.score_dense(n, re + 1j * im, q)
    cur, best, bf = oracle.init_state(p)
    rep = oracle.new_report()
    gi, sid, F2, C2, tk = oracle.step(p, cur, best, bf, 0, 1, rep)
    flops = sum(oracle.useful_flops(n, LIB, gi[c]) for c in range(P)) + P * (8 * N * N - 2 * N)
    assert rep.useful_flops == flops
