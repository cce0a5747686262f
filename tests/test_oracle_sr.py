"""Pins of the oracle's selective refinement (Sec. 2.4, Algorithm 2) and estimators."""
import math

import numpy as np
import pytest

from oracle import mlmc as om
from workloads import STRIP_FP64_3LEVEL as C1


def geometric(lam_inf, c, ratio):
    """lambda_j = lambda_inf + c ratio^j: a sequence whose level differences shrink by
    `ratio` per level, for which |lambda_j - lambda_{j-1}| / (1/ratio - 1) is exactly
    |lambda_j - lambda_inf| (the sample bias estimate of Eq. sampleBias is exact)."""
    return lambda j: lam_inf + c * ratio ** j


@pytest.mark.parametrize("c", [3.0, -3.0])
def test_stopped_indicator_equals_the_fully_refined_one(c):
    # m^alpha = 4: the bias estimate is exact, so stopping when |lambda_j - lambda*|
    # exceeds it (times sr_factor >= 1) keeps lambda_j on lambda_inf's side of
    # lambda*; the indicator then agrees with the finest level's.
    level = 6
    solve = geometric(10.0, c, 0.25)
    stopped_early = 0
    for thr in np.linspace(6.0, 14.0, 161):
        J, lam, lf, lc, qf, qc = om.selective_refinement(None, level, 0, thr, m=4.0, alpha=1.0, sr_factor=1.0,
                                                          eps_rel=0.0, solve=solve)
        assert qf == (1 if solve(level) > thr else 0)
        assert qc == (1 if solve(level - 1) > thr else 0) or J == level
        assert lam == [solve(j) for j in range(J + 1)]
        stopped_early += J < level
    assert stopped_early > 100      # most thresholds are decided early


def test_stopping_rules():
    solve = geometric(10.0, 3.0, 0.25)
    # the threshold at the value itself: never decided before the sample's level
    J, lam, *_ = om.selective_refinement(None, 4, 0, solve(2), solve=solve)
    assert J >= 3
    # no test on mesh 0 (no bias estimate yet); a far threshold stops at mesh 1
    J, lam, *_ = om.selective_refinement(None, 4, 0, 1e6, solve=solve)
    assert J == 1 and len(lam) == 2
    # level 0 samples solve mesh 0 only, their coarse indicator is 0
    J, lam, lf, lc, qf, qc = om.selective_refinement(None, 0, 0, 0.0, solve=solve)
    assert (J, qf, qc, lc) == (0, 1, 0, 0.0)
    # a larger widening factor never stops earlier
    for thr in np.linspace(8.0, 13.0, 41):
        js = [om.selective_refinement(None, 5, 0, thr, sr_factor=f, solve=solve)[0] for f in (1.0, 2.0, 4.0, 8.0)]
        assert js == sorted(js)


def test_selective_refinement_solves_the_level_pair_meshes():
    # without early stopping the chain holds exactly the plain solves of the sample on
    # every mesh, and its fine / coarse values are those of the level pair
    level, sid = 2, 5
    basis = om.Basis(C1)
    J, lam, lf, lc, qf, qc = om.selective_refinement(C1, level, sid, 0.0, sr_factor=1e30, basis=basis)
    qf_pair, qc_pair = om.level_pair(C1, level, [sid], basis)
    assert J == level
    assert lam[level] == qf_pair[0, 1] and lam[level - 1] == qc_pair[0, 1]
    assert lf == qf_pair[0, 1] and lc == qc_pair[0, 1]
    xi = om.rng.kl_coefficients(C1["seed"], level, [sid], C1["kl_terms"])[0]
    assert lam[0] == om.solve_on_mesh(C1, basis, 0, xi)[1]


def test_trinomial_moments_reduce_to_sample_moments_at_k0():
    g = np.random.default_rng(4)
    y = g.choice([-1, 0, 0, 0, 1], size=997)
    mean, var = om.trinomial_moments(y, k=0)
    assert mean == pytest.approx(float(np.mean(y)), abs=1e-15)
    assert var == pytest.approx(float(np.var(y)), abs=1e-15)


@pytest.mark.parametrize("n,p,k", [(200, 0.01, 1), (1000, 0.002, 1), (50, 0.1, 3)])
def test_biased_estimator_relative_variance(n, p, k):
    # Eq. biased_estimator: Var[p~] / E[p~]^2 = N p (1 - p) / (N p + k)^2 < 1
    g = np.random.default_rng(11)
    x = g.binomial(n, p, size=400000)
    pt = om.biased_probability(x, n, k)
    rel = np.var(pt) / np.mean(pt) ** 2
    exact = n * p * (1 - p) / (n * p + k) ** 2
    assert rel == pytest.approx(exact, rel=0.02)
    assert exact < 1.0
    assert np.mean(pt) == pytest.approx((n * p + k) / (n + k), rel=2e-3)


def test_upper_quantile_order_statistic():
    v = np.arange(1, 4097)[::-1].astype(float)
    q = om.upper_quantile(v, 1.0 / 150.0)
    assert q == math.ceil(4096 * (1 - 1 / 150))
    assert np.sum(v > q) == 4096 - math.ceil(4096 * (1 - 1 / 150))


def synthetic_results(seed=5, n=3000, levels=4, p=0.05):
    g = np.random.default_rng(seed)
    lv = g.integers(0, levels, n)
    qm0 = (g.random(n) < p).astype(int)
    qf = np.where(g.random(n) < 0.1, 1 - qm0, qm0)
    qc = np.where(g.random(n) < 0.05, 1 - qf, qf)
    qc[lv == 0] = 0
    return lv, qf, qc, qm0


def test_failure_estimate_plain_means_at_k0():
    lv, qf, qc, qm0 = synthetic_results()
    est, terms = om.failure_estimate(lv, qf, qc, qm0, k=0)
    plain = sum(float(np.mean(np.where(lv[lv == l] == 0, qf[lv == l], qf[lv == l] - qc[lv == l])))
                for l in range(4))
    assert est == pytest.approx(plain, abs=1e-15)
    est2, terms2 = om.failure_estimate(lv, qf, qc, qm0, k=0, two_level=True)
    top = lv.max()
    assert est2 == pytest.approx(float(np.mean(qf[lv == 0])) + float(np.mean(qf[lv == top] - qm0[lv == top])),
                                 abs=1e-15)
    assert sorted(terms2) == [0, top]
