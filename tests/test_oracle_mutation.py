"""Pins of the oracle's adaptive mutation (Sec. IV-F, Eq. (12)), the magnitude
law included, and planted mistakes that each of them must catch.

What the paper fixes, and the readings these tests hold the oracle to:
  * an individual mutates with probabilityOfMutation; a mutation is a qubit
    or a qutrit mutation with equal probability;
  * qubit: the angle turns by +-(1 - segmentFitness) * mutationRange (read:
    quantised to the lattice range/Q, Q = 4096, m = floor((1 - f) Q); the
    segment fitness clamped to [0, 1]);
  * qutrit: one of Eq. (12)'s eight parameters (theta_1..3 with domain
    (0, pi/2), phi_1..5 with domain (0, 2 pi)) is drawn from its domain times
    (1 - segmentFitness), the others are zero (read: the value is
    m * domain / Q with m = floor(u (1 - f) Q), u uniform in (0, 1)).

The qubit turn is measured from the amplitudes before and after.  For the
qutrit, the same mutation (same seed, generation and segment) is applied to
the three basis states, which gives every segment's whole 3x3 operator; with
one parameter nonzero Eq. (12) reduces, by hand, to one of six forms --
a Givens rotation in the (0,1), (0,2) or (1,2) plane (theta_1, theta_2,
theta_3), diag(e^{i phi}, 1, e^{-i phi}) (phi_1), diag(1, e^{i phi}, e^{-i phi})
(phi_2), or the identity (phi_3, phi_4, phi_5, whose factors all meet a zero
sine) -- from which the parameter and its value are read back.

Each planted mistake is a one-line change to a copy of the oracle's source,
compiled with the oracle's flags; every one of them must fail at least one of
the checks that the oracle itself passes."""
import numpy as np
import pytest
from scipy.stats import binomtest, chisquare

import oracle
from oracle import build as obuild
from paper_1809_11134_gb300 import workloads as W

Q = oracle.Q
NCV, HT, IDENT, ISING = W.LIB_NCV, W.LIB_HT, W.LIB_IDENTITY, W.LIB_ISING
RANGE = np.pi / 4
N_SEG_L, N_SEG_P = 8, 400


def _problem(library, seed, gen_range=RANGE):
    return oracle.make_problem(3, N_SEG_L, N_SEG_P, library, W.cknot(3), seed=seed, p_mutation=1.0,
                               mutation_range=gen_range)


def _mutate(p, cur, best_f, gen):
    """One update in which elitism changes nothing and every individual
    mutates: every slot names segment 0, whose state equals its best, with a
    fitness below any best fitness (so segment 0 is reverted to itself)."""
    best = cur.copy()
    seg_id = np.zeros((p.P, p.L), np.uint32)
    fitness = np.full(p.P, -1e30)
    bf = best_f.copy()
    oracle.update(p, cur, best, bf, gen, seg_id, fitness)
    assert np.array_equal(bf, best_f)
    return cur


# ---------------------------------------------------------------- qubit mutation
# segment fitness values and the lattice step count the paper's law gives them:
# (2k+1)/8192 sits half a step between lattice points, so floor((1 - f) Q) = Q - k - 1
# has no rounding question; f < 0 and f > 1 are clamped to 0 and 1
QUBIT_F = [(-1.0, Q), (0.0, Q), (1.0, 0), (1.5, 0)] + \
          [((2 * k + 1) / 8192.0, Q - k - 1) for k in (0, 100, 1000, 2047, 2048, 3000, 4000, 4095)]


def check_qubit_law(library, seed=11, gen=3):
    p = _problem(library, seed)
    cur, _, bf = oracle.init_state(p)
    S = len(bf)
    rng = np.random.default_rng(seed)
    st = cur.reshape(S, 8)
    th0 = rng.uniform(0, 2 * np.pi, S)  # start from every direction on the circle
    st[:, 6] = np.cos(th0)
    st[:, 7] = np.sin(th0)
    pick = rng.integers(0, len(QUBIT_F), S)
    best_f = np.array([QUBIT_F[i][0] for i in pick], np.float32)
    m_law = np.array([QUBIT_F[i][1] for i in pick])
    before = st.copy()
    after = _mutate(p, cur, best_f, gen).reshape(S, 8)
    q_moved = np.any(after[:, :6] != before[:, :6], 1)
    b_moved = np.any(after[:, 6:] != before[:, 6:], 1)
    assert not np.any(q_moved & b_moved), "one mutation per segment, qubit or qutrit"
    assert not np.any((q_moved | b_moved) & (m_law == 0)), "fitness 1 must leave a segment alone"
    z0 = before[:, 6].astype(np.float64) + 1j * before[:, 7]
    z1 = after[:, 6].astype(np.float64) + 1j * after[:, 7]
    turn = np.angle(z1 / z0)
    step = RANGE / Q
    # the turn is +-(1 - f) range on the range/Q lattice, binary32 rounding aside
    err = np.abs(np.abs(turn[b_moved]) - m_law[b_moved] * step)
    assert err.max() < 1e-5, ("qubit turn off the law", err.max())
    assert np.all(np.abs(np.abs(z1) - 1) < 1e-6)
    live = m_law > 0
    # qubit and qutrit mutation are equiprobable (every live segment took one of the two;
    # the qubit one always moves the qubit)
    assert binomtest(int(b_moved[live].sum()), int(live.sum()), 0.5).pvalue > 1e-4
    # and the sign is + or - with equal probability
    assert binomtest(int((turn[b_moved] > 0).sum()), int(b_moved.sum()), 0.5).pvalue > 1e-4
    return b_moved.sum()


@pytest.mark.parametrize("library", [NCV | IDENT, NCV | HT | IDENT, ISING])
def test_qubit_turn_is_one_minus_f_times_range(library):
    assert check_qubit_law(library) > 1000


# ---------------------------------------------------------------- qutrit mutation
def _givens(c, s, a, b):
    U = np.zeros(c.shape + (3, 3), np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    U[..., a, a] = c
    U[..., b, b] = c
    U[..., a, b] = s
    U[..., b, a] = -s
    return U


def _phases(ph, k):
    U = np.zeros(ph.shape + (3, 3), np.complex128)
    U[..., 0, 0] = U[..., 1, 1] = U[..., 2, 2] = 1
    U[..., k, k] = np.exp(1j * ph)
    U[..., 2, 2] = np.exp(-1j * ph)
    return U


def _read_parameter(U):
    """(family, angle in [0, 2 pi)) of each operator: family 0..2 = theta_1..3,
    3..4 = phi_1..2, 5 = identity, -1 = none of the six forms."""
    S = U.shape[0]
    fam = np.full(S, -1)
    ang = np.zeros(S)
    ident = np.abs(U - np.eye(3)).max(axis=(1, 2)) < 1e-6
    fam[ident] = 5
    cands = []
    # the phase forms first: at phi = pi they coincide with a half turn of theta_2 or
    # theta_3, which lies outside theta's domain
    for f, k in ((3, 0), (4, 1)):
        t = np.angle(U[:, k, k])
        cands.append((f, t, _phases(t, k)))
    # theta_1: rotation in the (0,1) plane, theta_2 in (0,2), theta_3 in (1,2) with the
    # sine's sign on the (2,1) entry
    for f, (a, b, sgn) in enumerate([(0, 1, 1.0), (0, 2, 1.0), (1, 2, -1.0)]):
        t = np.arctan2(sgn * U[:, a, b].real, U[:, a, a].real)
        cands.append((f, t, _givens(np.cos(t), sgn * np.sin(t), a, b)))
    for f, t, V in cands:
        hit = (fam == -1) & (np.abs(U - V).max(axis=(1, 2)) < 1e-5)
        fam[hit] = f
        ang[hit] = np.mod(t[hit], 2 * np.pi)
    return fam, ang


# (segment fitness, 1 - f): e is exact in binary32 and u * e is exact, so the
# largest lattice index is e Q - 1
QUTRIT_F = [(-1.0, 1.0), (0.5, 0.5), (0.75, 0.25)]


def qutrit_operators(seed=5, gen=7):
    p = _problem(NCV | HT, seed)  # no qubit in this library: every mutation is a qutrit one
    cur0, _, bf = oracle.init_state(p)
    S = len(bf)
    rng = np.random.default_rng(seed)
    pick = rng.integers(0, len(QUTRIT_F), S)
    best_f = np.array([QUTRIT_F[i][0] for i in pick], np.float32)
    e = np.array([QUTRIT_F[i][1] for i in pick])
    cols = []
    for b in range(3):
        cur = cur0.copy()
        st = cur.reshape(S, 8)
        st[:, :6] = 0.0
        st[:, 2 * b] = 1.0
        out = _mutate(p, cur, best_f, gen).reshape(S, 8).astype(np.float64)
        cols.append(out[:, 0:6:2] + 1j * out[:, 1:6:2])
    return np.stack(cols, axis=2), e  # U[s, row, column]


def check_qutrit_law(seed=5, gen=7):
    U, e = qutrit_operators(seed, gen)
    S = len(e)
    UU = np.einsum("sij,skj->sik", U, U.conj())
    assert np.abs(UU - np.eye(3)).max() < 1e-5, "not unitary"
    fam, ang = _read_parameter(U)
    assert np.all(fam >= 0), ("operators outside the six one-parameter forms", np.sum(fam < 0))
    rot = fam <= 4
    domain = np.where(fam <= 2, np.pi / 2, 2 * np.pi)
    m = ang / (domain / Q)
    assert np.abs(m[rot] - np.round(m[rot])).max() < 2e-2, "value off the domain/Q lattice"
    mi = np.round(m).astype(np.int64)
    # theta in [0, (pi/2)(1 - f)), phi in [0, 2 pi (1 - f)): lattice index below e Q
    assert np.all(mi[rot] >= 1) and np.all(mi[rot] < np.round(e[rot] * Q)), "value outside its domain"
    # the parameter is one of eight, uniformly: five visible forms at 1/8 each, the
    # identity for phi_3, phi_4, phi_5 (3/8) and for a zero lattice index
    p0 = np.minimum(1.0, 1.0 / (e * Q))
    exp_rot = (1 - p0) / 8.0
    expected = [exp_rot.sum()] * 5 + [S - 5 * exp_rot.sum()]
    counts = np.bincount(fam, minlength=6)
    assert chisquare(counts, expected).pvalue > 1e-3, ("parameter choice", counts, expected)
    # the value is uniform over its range: m / (e Q) uniform in [0, 1), per kind
    for kind in (fam <= 2, (fam == 3) | (fam == 4)):
        for ev in {q[1] for q in QUTRIT_F}:
            sel = kind & (e == ev)
            v = mi[sel] / (ev * Q)
            h = np.bincount(np.minimum((v * 10).astype(int), 9), minlength=10)
            assert chisquare(h).pvalue > 1e-3, ("value not uniform", ev, h)
    return counts


def test_qutrit_mutation_sets_one_su3_parameter_from_its_shrunk_domain():
    counts = check_qutrit_law()
    assert counts.sum() == 9 * N_SEG_L * N_SEG_P
    assert counts[5] > 0.3 * counts.sum()  # phi_3..5 alone are the identity


def test_mutation_law_at_a_second_seed_and_generation():
    check_qubit_law(NCV | IDENT, seed=29, gen=0)
    check_qutrit_law(seed=31, gen=2)


# ---------------------------------------------------------------- planted mistakes
def _source():
    return open(obuild.SRC).read()


MISTAKES = {
    "(1 - f) squared": [("float e = 1.0f - fc;", "float e = (1.0f - fc) * (1.0f - fc);")],
    "fitness not clamped": [("float fc = bf < 0.0f ? 0.0f : (bf > 1.0f ? 1.0f : bf);",
                             "float fc = bf;")],
    "qubit sign always +": [("    if (w[1] & 1u) s = -s;\n", "")],
    "theta drawn over 2 pi": [("double domain = (j < 3) ? (ORC_PI / 2.0) : (2.0 * ORC_PI);",
                               "double domain = 2.0 * ORC_PI;")],
    "phi drawn over pi/2": [("double domain = (j < 3) ? (ORC_PI / 2.0) : (2.0 * ORC_PI);",
                             "double domain = ORC_PI / 2.0;")],
    "nine parameters": [("uint32_t j = below(w[1], 8);", "uint32_t j = below(w[1], 9);"),
                        ("float cv[8], sv[8];\n  for (int k = 0; k < 8; ++k) {",
                         "float cv[9], sv[9];\n  for (int k = 0; k < 9; ++k) {")],
    "no uniform draw in the value": [("floorf((unit32(w[2]) * e) * (float)ORC_Q)",
                                      "floorf(e * (float)ORC_Q)")],
    "qubit and qutrit not equiprobable": [("if (has_qubit && w[0] < 0x80000000u)",
                                           "if (has_qubit && w[0] < 0xC0000000u)")],
}


def _all_checks():
    check_qubit_law(NCV | IDENT)
    check_qubit_law(ISING)
    check_qutrit_law()


def test_the_checks_pass_on_the_oracle():
    _all_checks()


@pytest.mark.parametrize("name", sorted(MISTAKES))
def test_planted_mistake_fails_a_check(name, tmp_path):
    src = _source()
    for old, new in MISTAKES[name]:
        assert src.count(old) == 1, ("the line to plant in is gone", old)
        src = src.replace(old, new)
    path = obuild.build_variant(src, str(tmp_path / "liboracle_planted.so"))
    with oracle.using(oracle.load(path)):
        with pytest.raises(AssertionError):
            _all_checks()
