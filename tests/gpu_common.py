"""Shared helpers of the GPU parity tests (CUDA path vs the CPU oracle)."""
import numpy as np

import oracle
from paper_1809_11134_gb300 import workloads as W


def oracle_problem(s: W.Search, run: int):
    return oracle.make_problem(s.n, s.L, s.P, s.library, s.perm, seed=s.seed, run=run,
                               fitness_kind=s.fitness_kind, p_mutation=s.p_mutation,
                               mutation_range=s.mutation_range, cost_weight=s.cost_weight,
                               shots=s.shots, target=s.target)


def eps_d(L, dense_N=0):
    """Bound on |d32 - d64|, d = (N - |tr|)/N, that the ranking guard band uses
    (a dense N x N target adds the binary32 score's own rounding)."""
    return L * 8e-7 + 2e-6 + ((dense_N + 8) * 2.0**-23 if dense_N else 0.0)


def d_of(F, s: W.Search, cost=None):
    """d = (1 - f)^2 with f = F + penalty."""
    f = np.asarray(F, np.float64)
    if s.cost_weight and cost is not None:
        f = f + s.cost_weight * (np.asarray(cost, np.float64) / s.L)
    return (1.0 - f) ** 2


def assert_fp32_fitness(F32, F64, s: W.Search, cost=None):
    """binary32 fitness against binary64: within the d-space bound everywhere,
    and within 1e-5 absolute wherever d64 >= 1e-4 (f <= 0.99), where the square
    root of Eq. (11) no longer amplifies rounding."""
    d32, d64 = d_of(F32, s, cost), d_of(F64, s, cost)
    assert np.all(np.isfinite(F32))
    bound = eps_d(s.L, (1 << s.n) if s.target is not None else 0)
    assert np.abs(d32 - d64).max() <= bound, np.abs(d32 - d64).max()
    far = d64 >= 1e-4
    if far.any():
        err = np.abs(np.asarray(F32, np.float64)[far] - F64[far]).max()
        assert err <= 1e-5, err


def state_equal(a, b):
    """bitwise equality of float32 state arrays"""
    a = np.ascontiguousarray(a, np.float32).view(np.uint32)
    b = np.ascontiguousarray(b, np.float32).view(np.uint32)
    return np.array_equal(a, b)
