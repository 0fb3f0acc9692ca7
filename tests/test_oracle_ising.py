"""Pins of the oracle's Ising library (Sec. III Eqs. (3)-(5), the interaction
template, Sec. IV-A encoding) against definitions and identities that do not
reuse its own formulas: matrix exponentials of the Pauli generators, textbook
identities with the discrete library's CNOT/H/T, and an exact CNOT built from
Ising gates."""
import numpy as np
import pytest
from scipy.linalg import expm

import oracle
from paper_1809_11134_gb300 import workloads as W

ISING = oracle.LIB_ISING
X = np.array([[0, 1], [1, 0]], complex)
Y = np.array([[0, -1j], [1j, 0]])
Z = np.diag([1.0, -1.0]).astype(complex)
I2 = np.eye(2)


def amps_of(theta):
    return np.float32(np.cos(theta)), np.float32(np.sin(theta))


def theta_of(b0, b1):
    """the angle the encoding assigns: cos theta = b0, sin theta has b1's sign"""
    t = np.arccos(np.clip(np.float64(b0), -1.0, 1.0))
    return 2 * np.pi - t if b1 < 0 else t


def test_geometry():
    for n in range(1, 6):
        assert oracle.num_regions(n, ISING) == n + n * (n - 1) // 2
        assert oracle.num_gates(n, ISING) == 3 * n + n * (n - 1) // 2
    n = 4
    kinds = [oracle.gate_desc(n, ISING, g) for g in range(oracle.num_gates(n, ISING))]
    assert kinds[:12] == [(k, -1, w) for w in range(4) for k in (oracle.RX, oracle.RY, oracle.RZ)]
    pairs = [(i, j) for i in range(4) for j in range(i + 1, 4)]
    assert kinds[12:] == [(oracle.J, i, j) for i, j in pairs]
    # a rotation region's qutrit picks the axis, a template region is one gate
    assert [oracle.region_gate(n, ISING, 1, k) for k in range(3)] == [3, 4, 5]
    assert oracle.region_gate(n, ISING, 4 + 2, 0) == 12 + 2


def test_half_angle_quadrants_exact():
    h = np.sqrt(0.5)
    assert oracle.half_angle(1.0, 0.0) == (1.0, 0.0)          # theta = 0
    assert oracle.half_angle(0.0, 1.0) == (h, h)              # pi/2
    assert oracle.half_angle(-1.0, 0.0) == (0.0, 1.0)         # pi
    assert oracle.half_angle(0.0, -1.0) == (-h, h)            # 3 pi / 2
    rng = np.random.default_rng(0)
    for t in rng.uniform(0, 2 * np.pi, 200):
        b0, b1 = amps_of(t)
        c, s = oracle.half_angle(b0, b1)
        tt = theta_of(b0, b1)
        assert abs(c - np.cos(tt / 2)) < 1e-15 and abs(s - np.sin(tt / 2)) < 1e-15


@pytest.mark.parametrize("axis,P", [(0, X), (1, Y), (2, Z)])
def test_rotations_are_exponentials_of_paulis(axis, P):
    """Eqs. (3)-(5): R_a(theta) = exp(-i theta/2 sigma_a)."""
    rng = np.random.default_rng(axis)
    for t in rng.uniform(0, 2 * np.pi, 50):
        b0, b1 = amps_of(t)
        R = oracle.gate_matrix_amp(1, ISING, axis, b0, b1)
        ref = expm(-0.5j * theta_of(b0, b1) * P)
        assert np.abs(R - ref).max() < 1e-14
        assert np.abs(R @ R.conj().T - I2).max() < 1e-15


def test_interaction_template_is_exp_zz_and_cnot_conjugated_rz():
    """J_ij(theta) = exp(-i theta/2 Z_i Z_j) = CNOT_{i->j} R_z(theta)_j CNOT_{i->j}, on every
    pair of a 3-qubit register (CNOT from the discrete library, wire 0 = MSB)."""
    n = 3
    rng = np.random.default_rng(5)
    pairs = [(i, j) for i in range(n) for j in range(i + 1, n)]
    for q, (i, j) in enumerate(pairs):
        for t in rng.uniform(0, 2 * np.pi, 5):
            b0, b1 = amps_of(t)
            Jm = oracle.gate_matrix_amp(n, ISING, 3 * n + q, b0, b1)
            ops = [I2] * n
            ops[i], ops[j] = Z, Z
            ZZ = ops[0]
            for o in ops[1:]:
                ZZ = np.kron(ZZ, o)
            assert np.abs(Jm - expm(-0.5j * theta_of(b0, b1) * ZZ)).max() < 1e-14
            cnot = oracle.gate_matrix(n, W.LIB_NCV, 3 * (i * (n - 1) + (j - 1 if j > i else j)))
            assert oracle.gate_desc(n, W.LIB_NCV, 3 * (i * (n - 1) + (j - 1 if j > i else j))) == \
                (oracle.CNOT, i, j)
            Rz = oracle.gate_matrix_amp(n, ISING, 3 * j + 2, b0, b1)
            assert np.abs(Jm - cnot @ Rz @ cnot).max() < 1e-14


def test_rotations_against_the_discrete_library():
    """H R_z(theta) H = R_x(theta) and S R_x(theta) S^dag = R_y(theta), S = T^2, with H and T
    taken from the H/T library."""
    Hm = oracle.gate_matrix(1, W.LIB_HT, 0)
    Tm = oracle.gate_matrix(1, W.LIB_HT, 1)
    S = Tm @ Tm
    rng = np.random.default_rng(7)
    for t in rng.uniform(0, 2 * np.pi, 30):
        b0, b1 = amps_of(t)
        Rx, Ry, Rz = (oracle.gate_matrix_amp(1, ISING, k, b0, b1) for k in range(3))
        assert np.abs(Hm @ Rz @ Hm - Rx).max() < 1e-15
        assert np.abs(S @ Rx @ S.conj().T - Ry).max() < 1e-15


def test_rotation_angles_add():
    rng = np.random.default_rng(9)
    for axis in range(3):
        for t1, t2 in rng.uniform(0, 2 * np.pi, (20, 2)):
            a, b = amps_of(t1), amps_of(t2)
            S = oracle.compose(1, ISING, [axis, axis], np.array([a, b], np.float32))
            M = S[0] + 1j * S[1]
            P = (X, Y, Z)[axis]
            ref = expm(-0.5j * (theta_of(*a) + theta_of(*b)) * P)
            assert np.abs(M - ref).max() < 1e-14


def test_cnot_from_ising_gates_scores_one():
    """CNOT (control wire 1, target wire 0) = H_0 CZ H_0 with H = i R_x(pi) R_y(pi/2) and
    CZ = e^{i pi/4} R_z(pi/2)_0 R_z(pi/2)_1 J_01(-pi/2); J(3 pi/2) = -J(-pi/2), a global sign.
    Seven Ising gates at angles pi/2, pi, 3 pi/2 (exact amplitudes) reach fitness 1."""
    n = 2
    p = oracle.make_problem(n, 7, 1, ISING, W.cknot(2))
    ry0, rx0, rz0, rz1, j01 = 1, 0, 2, 5, 6
    gates = [ry0, rx0, rz0, rz1, j01, ry0, rx0]
    half, pi, three = (0.0, 1.0), (-1.0, 0.0), (0.0, -1.0)
    amps = np.array([half, pi, half, half, three, half, pi], np.float32)
    F, cost = oracle.eval_circuits(p, np.array([gates], np.uint8), amps[None])
    assert F[0] > 1 - 1e-7 and cost[0] == 7
    S = oracle.compose(n, ISING, gates, amps)
    M = S[0] + 1j * S[1]
    target = np.zeros((4, 4))
    for j, pj in enumerate(W.cknot(2)):
        target[pj, j] = 1
    phase = M[0, 0]
    assert abs(abs(phase) - 1) < 1e-14
    assert np.abs(M / phase - target).max() < 1e-14
    # a wrong axis anywhere breaks it
    bad = list(gates)
    bad[1] = 1
    assert oracle.eval_circuits(p, np.array([bad], np.uint8), amps[None])[0][0] < 0.9


def test_sampling_and_angles():
    """Rotation regions measure their qutrit for the axis, template regions always give their J;
    the qubit is not measured (never the identity) and its amplitudes are the slot's angle."""
    n, L, P = 3, 6, 200
    p = oracle.make_problem(n, L, P, ISING, W.cknot(3), seed=4)
    cur, best, bf = oracle.init_state(p)
    rng = np.random.default_rng(2)
    cur[:] = W.random_state(rng, len(bf))[0].ravel()
    gi, sid, amps = oracle.sample(p, cur, 0, with_amps=True)
    R = oracle.num_regions(n, ISING)
    r = sid.astype(np.int64) // (L * P)
    assert np.all(r < R)
    rot = r < n
    assert np.all(gi[rot] // 3 == r[rot])
    assert np.all(gi[~rot] == 3 * n + (r[~rot] - n))
    st = cur.reshape(-1, 8)
    assert np.array_equal(amps[..., 0], st[sid, 6]) and np.array_equal(amps[..., 1], st[sid, 7])
    g2, s2 = oracle.sample(p, cur, 0)
    assert np.array_equal(g2, gi) and np.array_equal(s2, sid)


def test_mutation_turns_the_angle():
    """In the Ising library the qubit mutation turns the slot's angle by +-m range/Q (the
    paper's theta <- theta +- (1 - f) range, mod 2 pi)."""
    n, L, P = 2, 3, 64
    p = oracle.make_problem(n, L, P, ISING, W.cknot(2), seed=8, p_mutation=1.0)
    cur, best, bf = oracle.init_state(p)
    before = cur.reshape(-1, 8)[:, 6:8].copy()
    gi, sid = oracle.sample(p, cur, 0)
    F = np.full(P, 0.25)
    oracle.update(p, cur, best, bf, 0, sid, F)
    after = cur.reshape(-1, 8)[:, 6:8]
    d = np.angle((after[:, 0] + 1j * after[:, 1]) / (before[:, 0] + 1j * before[:, 1]))
    moved = np.abs(d) > 1e-6
    assert moved.mean() > 0.3  # about half the segments take the qubit mutation
    step = p.mutation_range / oracle.Q
    m = np.abs(d[moved]) / step
    assert np.abs(m - np.round(m)).max() < 1e-3


# ---------------------------------------------------------------- the paper's GA on Ising genes
def _ga_problem(P=400, L=12, n=3, seed=3, rng_=0.3):
    return oracle.make_problem(n, L, P, ISING, W.cknot(n), seed=seed, mutation_range=rng_)


def test_ising_ga_init_is_uniform_on_the_angle_lattice():
    p = _ga_problem(P=2000, L=10)
    G = oracle.num_gates(3, ISING)
    g, a = oracle.ga_init_amp(p, G)
    from scipy.stats import chisquare
    assert chisquare(np.bincount(g.ravel(), minlength=G)).pvalue > 1e-3
    step = 2 * np.pi / oracle.Q
    th = np.mod(np.arctan2(a[..., 1].astype(np.float64), a[..., 0]), 2 * np.pi)
    m = np.round(th / step).astype(np.int64) % oracle.Q
    assert np.array_equal(a[..., 0], np.cos(m * step).astype(np.float32))
    assert np.array_equal(a[..., 1], np.sin(m * step).astype(np.float32))
    assert chisquare(np.bincount(m.ravel() * 8 // oracle.Q, minlength=8)).pvalue > 1e-3


def test_ising_ga_two_point_crossover_moves_genes_with_their_angles():
    p = _ga_problem()
    G = oracle.num_gates(3, ISING)
    rng = np.random.default_rng(1)
    g = rng.integers(0, G, (p.P, p.L)).astype(np.uint8)
    a = np.stack([np.cos(t := rng.uniform(0, 6.28, (p.P, p.L))), np.sin(t)], -1).astype(np.float32)
    F = rng.uniform(0, 1, p.P)
    out, oa = oracle.ga_next_amp(p, G, 0, 0.0, g, a, F, np.zeros(p.P, np.uint32))
    rows = {(bytes(g[c]), a[c].tobytes()): c for c in range(p.P)}
    seen_two = 0
    for m in range(2, 200, 2):
        x, y = out[m], out[m + 1]
        xa, ya = oa[m], oa[m + 1]
        ok = False
        for lo in range(1, p.L + 1):
            for hi in range(lo, p.L + 1):
                inner = slice(lo, hi)
                A = x.copy(); B = y.copy(); Aa = xa.copy(); Ba = ya.copy()
                A[inner], B[inner] = y[inner], x[inner]
                Aa[inner], Ba[inner] = ya[inner], xa[inner]
                if (bytes(A), Aa.tobytes()) in rows and (bytes(B), Ba.tobytes()) in rows:
                    ok = True
                    seen_two += hi < p.L and lo < hi
                    break
            if ok:
                break
        assert ok, m
    assert seen_two > 50  # genuinely two cuts, not one


def test_ising_ga_mutation_rates_and_angle_steps():
    p = _ga_problem(P=1500, L=16)
    G = oracle.num_gates(3, ISING)
    g, a = oracle.ga_init_amp(p, G)
    F = np.full(p.P, 0.5)
    cost = np.zeros(p.P, np.uint32)
    base, base_a = oracle.ga_next_amp(p, G, 4, 0.0, g, a, F, cost)
    rate = 0.1
    mut, mut_a = oracle.ga_next_amp(p, G, 4, rate, g, a, F, cost)
    gchg = (mut[1:] != base[1:]) | np.any(mut_a[1:] != base_a[1:], -1)
    assert abs(gchg.mean() - (rate + (1 - rate) * rate)) < 0.01
    # the angle-only mutations turn the amplitudes by a multiple of range/Q
    same_gate = mut[1:] == base[1:]
    turned = same_gate & np.any(mut_a[1:] != base_a[1:], -1)
    z0 = base_a[1:][turned, 0] + 1j * base_a[1:][turned, 1]
    z1 = mut_a[1:][turned, 0] + 1j * mut_a[1:][turned, 1]
    d = np.angle(z1 / z0)
    step = p.mutation_range / oracle.Q
    # all but the fresh genes that drew the same gate again (about rate/G of the genes)
    k = np.abs(d) / step
    small = (np.abs(d) <= p.mutation_range + 1e-6) & (np.abs(k - np.round(k)) < 1e-2)
    assert small.mean() > 1 - 2 * rate / G / ((1 - rate) * rate)
    assert out_elite_ok(p, G, g, a)


def out_elite_ok(p, G, g, a):
    F = np.linspace(0, 1, p.P)[::-1].copy()
    F[0] = 0.2  # the best is circuit 1
    out, oa = oracle.ga_next_amp(p, G, 1, 0.5, g, a, F, np.zeros(p.P, np.uint32))
    return np.array_equal(out[0], g[1]) and np.array_equal(oa[0], a[1])
