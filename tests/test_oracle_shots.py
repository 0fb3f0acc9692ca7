"""Pins of the oracle's repeated qutrit measurement (Sec. IV-A1: the qutrit is
measured several times to approximate its state): with K shots the outcome is
the most frequent one, the lowest on a tie.  Its law has a closed form -- the
multinomial distribution of the K outcome counts pushed through that rule --
which the sampled gates must follow; K = 1 is the single-shot measurement."""
import itertools
import math

import numpy as np
import pytest
from scipy.stats import chisquare

import oracle
from paper_1809_11134_gb300 import workloads as W

LIB = W.LIB_NCV | W.LIB_HT  # no identity: gate = 3 r + k


def majority_law(p, K):
    """P(outcome k) for K independent shots with probabilities p, ties to the lowest k."""
    out = np.zeros(3)
    for n0 in range(K + 1):
        for n1 in range(K + 1 - n0):
            n2 = K - n0 - n1
            w = math.factorial(K) // (math.factorial(n0) * math.factorial(n1) * math.factorial(n2))
            pr = w * p[0] ** n0 * p[1] ** n1 * p[2] ** n2
            c = [n0, n1, n2]
            out[int(np.argmax(c))] += pr  # argmax returns the first maximum
    return out


def outcomes(p_state, K, P=2500, L=16, n=3, seed=3, gen=0):
    prob = oracle.make_problem(n, L, P, LIB, W.cknot(n), seed=seed, shots=K)
    R = oracle.num_regions(n, LIB)
    a = np.sqrt(np.asarray(p_state, np.float64))
    seg = np.array([a[0], 0, a[1], 0, a[2], 0, 2**-0.5, 2**-0.5], np.float32)
    cur = np.tile(seg, R * P * L)
    gi, sid = oracle.sample(prob, cur, gen)
    r = sid.ravel() // (L * P)
    k = gi.ravel().astype(np.int64) - 3 * r.astype(np.int64)
    assert np.all((k >= 0) & (k < 3))
    return k


def test_majority_law_by_hand():
    # two shots on a uniform qutrit: a tie goes to the lower outcome, so k = 2 needs
    # both shots on 2 and k = 1 needs no shot on 0 and not both on 2
    assert np.allclose(majority_law([1 / 3] * 3, 2), [5 / 9, 3 / 9, 1 / 9])
    assert np.allclose(majority_law([0.2, 0.5, 0.3], 1), [0.2, 0.5, 0.3])
    assert np.isclose(majority_law([0.2, 0.5, 0.3], 9).sum(), 1.0)


@pytest.mark.parametrize("K", [2, 3, 4, 5, 8, 15])
@pytest.mark.parametrize("p", [(0.3, 0.45, 0.25), (1 / 3, 1 / 3, 1 / 3), (0.5, 0.1, 0.4)])
def test_outcomes_follow_the_majority_law(K, p):
    k = outcomes(p, K, seed=K)
    obs = np.bincount(k, minlength=3)
    exp = majority_law(p, K) * len(k)
    keep = exp > 0
    assert chisquare(obs[keep], exp[keep] * obs[keep].sum() / exp[keep].sum()).pvalue > 1e-3


def test_more_shots_approach_the_most_probable_outcome():
    f = [np.mean(outcomes((0.3, 0.45, 0.25), K, P=1500) == 1) for K in (1, 5, 21, 63)]
    assert f[0] < f[1] < f[2] < f[3] and f[3] > 0.85
    assert abs(f[3] - majority_law((0.3, 0.45, 0.25), 63)[1]) < 0.01


def test_basis_states_are_certain_for_any_k():
    for K in (2, 7, 64):
        for b in range(3):
            p = [0.0, 0.0, 0.0]
            p[b] = 1.0
            assert np.all(outcomes(p, K, P=200, L=8) == b)


def test_one_shot_is_the_single_measurement():
    prob0 = oracle.make_problem(3, 16, 300, LIB | W.LIB_IDENTITY, W.cknot(3), seed=5, shots=0)
    prob1 = oracle.make_problem(3, 16, 300, LIB | W.LIB_IDENTITY, W.cknot(3), seed=5, shots=1)
    cur, _, _ = oracle.init_state(prob0)
    g0, s0 = oracle.sample(prob0, cur, 4)
    g1, s1 = oracle.sample(prob1, cur, 4)
    assert np.array_equal(g0, g1) and np.array_equal(s0, s1)
    # the individual, region and qubit draws do not depend on K
    probk = oracle.make_problem(3, 16, 300, LIB | W.LIB_IDENTITY, W.cknot(3), seed=5, shots=9)
    gk, sk = oracle.sample(probk, cur, 4)
    assert np.array_equal(sk, s0)
    assert np.array_equal(gk == 0, g0 == 0)  # identity decided by the qubit alone
