"""Pins for the oracle's KL basis (Nystrom eigenpairs of the covariance, Eq. inftyKL)."""
import math

import numpy as np
import pytest
from scipy import integrate

from oracle import kl
from workloads import STRIP_MIXED_5LEVEL as C2


@pytest.mark.parametrize("a", [1.0, 0.25])
def test_1d_eigenfunctions_orthonormal(a):
    x, w, mu, phi = kl.eig_1d(a, 0.2, 128)
    G = (phi[:, :20] * w[:, None]).T @ phi[:, :20]
    np.testing.assert_allclose(G, np.eye(20), atol=1e-12)
    used = mu > 1e-14 * mu[0]          # modes above rounding level (the only ones a basis can select)
    assert np.all(np.diff(mu[used]) < 0)
    assert np.all(phi[0, used] > 0.1)    # the sign rule acts on a value well away from zero


@pytest.mark.parametrize("a", [1.0, 0.25])
def test_eigen_equation_with_independent_quadrature(a):
    """int_0^a k(x, y) phi(y) dy = mu phi(x), checked by adaptive quadrature of the interpolant."""
    corr = 0.2
    x, w, mu, phi = kl.eig_1d(a, corr, 128)
    rng = np.random.default_rng(3)
    for i in range(6):
        f = lambda y: kl.eval_1d([y], x, w, mu, phi, corr, [i])[0, 0]
        for px in rng.uniform(0, a, 3):
            lhs, _ = integrate.quad(lambda y: math.exp(-(px - y) ** 2 / (2 * corr * corr)) * f(y),
                                    0.0, a, epsabs=1e-14, epsrel=1e-12, limit=200)
            rhs = mu[i] * f(px)
            assert abs(lhs - rhs) <= 1e-9 * mu[0]


def test_eigenvalues_converged_in_quadrature():
    _, _, m128, _ = kl.eig_1d(1.0, 0.2, 128)
    _, _, m256, _ = kl.eig_1d(1.0, 0.2, 256)
    np.testing.assert_allclose(m128[:12], m256[:12], rtol=1e-9)
    # trace = integral of k(x, x) = length of the interval (Mercer)
    assert abs(m128.sum() - 1.0) < 1e-12


def test_mercer_partial_sums_at_centroids():
    """sum_{n<=N} mu_n phi_n(x)^2 rises monotonically to k(x, x) = s^2 (Bessel/Mercer)."""
    s = np.deg2rad(2.0)
    cx, cy = kl.element_centroids(1.0, 0.25, 64, 16)
    B, modes, mu2 = kl.kl_basis(1.0, 0.25, 0.2, s, 128, 100, cx, cy)
    partial = np.cumsum(B ** 2, axis=1) / s ** 2
    assert np.all(np.diff(partial, axis=1) >= 0)
    assert np.all(partial[:, -1] <= 1.0 + 1e-10)
    assert np.all(partial[:, -1] >= 1.0 - 1e-6)
    assert np.all(np.diff(mu2) <= 0)
    assert len(set(modes)) == 100


def test_field_variance_matches_covariance():
    """Monte Carlo variance and correlation of theta against k(x, y)."""
    cfg = dict(C2)
    cfg["kl_terms"] = 60
    B = kl.basis_for_mesh(cfg, 16, 4)
    xi = np.random.default_rng(5).standard_normal((40000, 60))
    th = kl.theta_field(B, xi)
    s2 = np.deg2rad(2.0) ** 2
    cx, cy = kl.element_centroids(1.0, 0.25, 16, 4)
    cov = np.cov(th.T)
    d2 = (cx[:, None] - cx[None, :]) ** 2 + (cy[:, None] - cy[None, :]) ** 2
    exact = s2 * np.exp(-d2 / (2 * 0.2 ** 2))
    assert np.max(np.abs(cov - exact)) < 0.05 * s2
    # exact second moments of the truncated expansion: B B^T against k(x, y)
    assert np.max(np.abs(B @ B.T - exact)) < 1e-6 * s2
