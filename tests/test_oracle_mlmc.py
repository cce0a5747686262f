"""Pins for the oracle's level pairs, statistics and Algorithm 1 (Sec. 2.2-2.3)."""
import math

import numpy as np
import pytest

from oracle import mlmc, rng
from workloads import STRIP_FP64_3LEVEL as C1


def test_pairs_share_xi_and_telescope():
    """Coarse solve of pair l+1 equals the fine solve of pair l on the same xi, so
    mean(Q_0) + sum_l mean(Y_l) = mean(Q_L) on identical samples (Eq. MLMC_expectation)."""
    b = mlmc.Basis(C1)
    xi = rng.kl_coefficients(11, 0, np.arange(6), C1["kl_terms"])
    pairs = [mlmc.level_pair_from_xi(C1, l, xi, b) for l in range(3)]
    for l in range(2):
        np.testing.assert_array_equal(pairs[l][0], pairs[l + 1][1])
    tel = pairs[0][0].mean(0) + sum((pairs[l][0] - pairs[l][1]).mean(0) for l in range(1, 3))
    np.testing.assert_allclose(tel, pairs[2][0].mean(0), rtol=1e-14)


def test_level_pair_uses_level_stream():
    b = mlmc.Basis(C1)
    qf, qc = mlmc.level_pair(C1, 1, [3, 4], b)
    xi = rng.kl_coefficients(C1["seed"], 1, [3, 4], C1["kl_terms"])
    qf2, qc2 = mlmc.level_pair_from_xi(C1, 1, xi, b)
    np.testing.assert_array_equal(qf, qf2)
    np.testing.assert_array_equal(qc, qc2)


def test_variance_of_level_differences_decays():
    b = mlmc.Basis(C1)
    V = []
    for l in range(1, 4):
        qf, qc = mlmc.level_pair(C1, l, np.arange(24), b)
        V.append(np.var(qf - qc, axis=0))
    V = np.array(V)
    assert np.all(V[1:, 0] < V[:-1, 0] / 4)       # reaction: fast decay
    assert np.all(V[1:, 1] < V[:-1, 1])           # stress: monotone decay


def test_moments_against_two_pass():
    y = np.random.default_rng(0).normal(1e7, 3.0, 5001)
    n, mean, s2 = mlmc.moments(y)
    assert n == 5001
    assert mean == pytest.approx(np.mean(y), rel=1e-15)
    # Eq. varianceestim evaluated in exact rational arithmetic
    from fractions import Fraction
    fy = [Fraction(float(v)) for v in y]
    m = sum(fy) / n
    exact = sum(v * v for v in fy) / n - m * m
    assert s2 == pytest.approx(float(exact), rel=1e-9)
    assert mlmc.moments([]) == (0, 0.0, 0.0)


def test_optimal_samples_meet_constraint_at_minimum_cost():
    V = np.array([4.0, 1.0, 0.2, 0.03])
    Cst = np.array([1.0, 4.0, 16.0, 64.0])
    es2 = 1e-3
    N = np.array(mlmc.optimal_samples(V, Cst, es2), dtype=float)
    assert np.sum(V / N) <= es2 * (1 + 1e-12)
    # the unrounded optimum is the Lagrange point: perturbing along the constraint raises cost
    Ns = (np.sum(np.sqrt(V * Cst)) / es2) * np.sqrt(V / Cst)
    assert np.sum(V / Ns) == pytest.approx(es2, rel=1e-12)
    base = np.sum(Ns * Cst)
    for k in range(4):
        for j in range(4):
            if j == k:
                continue
            t = Ns.copy()
            t[k] *= 1.05
            t[j] = V[j] / (es2 - np.sum(np.delete(V / t, j)))       # stay on the constraint
            assert np.sum(t * Cst) > base
    assert np.all(np.ceil(Ns) == N)


def test_bias_estimate():
    assert mlmc.bias_estimate(-3.0, 4, 1.0) == pytest.approx(1.0)
    assert mlmc.bias_estimate(15.0, 4, 2.0) == pytest.approx(1.0)


def test_algorithm1_on_a_synthetic_hierarchy():
    """Y_l ~ N(b 4^-l, v 4^-2l): Algorithm 1 must add levels until the bias test passes
    and size N_l so that the sampling error meets e_s."""
    bias0, v0 = 1.0, 1.0

    def sampler(level, ids):
        g = np.random.default_rng([level, int(ids[0]) if len(ids) else 0])
        if level == 0:
            return 10.0 + g.standard_normal(len(ids))
        return bias0 * 4.0 ** -level + math.sqrt(v0) * 4.0 ** -level * g.standard_normal(len(ids))

    e, theta = 0.02, 0.5
    est, Y, L, conv = mlmc.algorithm1(C1, e, theta, 100, 8, alpha=1.0, gamma=1.0, sampler=sampler)
    assert conv
    eb = math.sqrt(1 - theta) * e
    assert bias0 * 4.0 ** -L / 3.0 < 2 * eb                    # true bias near the tolerance
    assert abs(np.mean(Y[L])) / 3.0 < eb
    V = [mlmc.moments(y)[2] for y in Y]
    assert sum(v / len(y) for v, y in zip(V, Y)) <= theta * e * e * 1.3
    assert est == pytest.approx(10.0 + sum(bias0 * 4.0 ** -l for l in range(1, L + 1)), abs=3 * e)
    assert all(len(Y[l]) >= 100 for l in range(L + 1))
