"""Pins of the Cosserat oracle (the paper's first test problem) against what the
mathematics fixes (no GPU).

- mesh: 8 x 8 elements give M_0 = 243 DOFs (Sec. 3.2);
- rotation: C*(0) = C, period pi, frame-invariant energy, the quarter turn swaps the
  fibre-frame roles;
- element: symmetric, rank 9 (the two translations and the Cosserat rigid rotation
  u = w (-y, x), theta = w cost nothing), 2x2 = 3x3 Gauss;
- homogeneous block (phi constant 0 or pi/2): the uniform state u = eps x, v = 0,
  theta = 0 is exact under the boundary conditions, so the FE reproduces it on any mesh:
  reaction Q11 |Delta| and the closed-form strength R tau_y Q11 / Q12 (fibres along x),
  R tau_y (across);
- energy identity d^T K d = |Delta| R; dense and sparse solves agree;
- KL: the closed-form eigenpairs of the exponential kernel satisfy the eigen-equation
  under adaptive quadrature, are orthonormal, and match a Nystrom discretisation;
- telescoping on identical xi.
"""
import numpy as np
import pytest
import scipy.integrate as si

from oracle import cosserat as C
from oracle import rng
from workloads import COSSERAT_TEST1 as W


def test_level0_dof_count():
    K = C.assemble(W, 8, np.zeros(64))
    assert K.shape == (243, 243)
    assert C.dofs(W, 0) == 243 and C.dofs(W, 1) == C.assemble(W, 16, np.zeros(256)).shape[0]


def test_rotation_identities():
    Cf, Df = C.fibre_stiffness(W)
    C0, D0 = C.rotated_stiffness(Cf, Df, 0.0)
    np.testing.assert_allclose(C0, Cf, atol=1e-9 * np.abs(Cf).max())
    Cp, Dp = C.rotated_stiffness(Cf, Df, np.pi)
    np.testing.assert_allclose(Cp, Cf, atol=1e-9 * np.abs(Cf).max())
    np.testing.assert_allclose(Dp, Df, atol=1e-12)
    Cq, Dq = C.rotated_stiffness(Cf, Df, 0.5 * np.pi)
    assert Cq[0, 0] == pytest.approx(Cf[1, 1], rel=1e-12) and Cq[1, 1] == pytest.approx(Cf[0, 0], rel=1e-12)
    assert Dq[0, 0] == pytest.approx(Df[1, 1], rel=1e-12) and Dq[1, 1] == pytest.approx(Df[0, 0], rel=1e-12)
    # energy of a global strain equals the fibre-frame energy of its rotated form
    g = np.random.default_rng(1)
    for phi in (0.1, -0.7, 1.3):
        Cg, Dg = C.rotated_stiffness(Cf, Df, phi)
        R = C._rot(phi)
        for _ in range(3):
            E = g.normal(size=(2, 2))
            el = C._vec(R.T @ E @ R)
            assert C._vec(E) @ Cg @ C._vec(E) == pytest.approx(el @ Cf @ el, rel=1e-12)
            k = g.normal(size=2)
            assert k @ Dg @ k == pytest.approx((R.T @ k) @ Df @ (R.T @ k), rel=1e-12)
        np.testing.assert_allclose(Cg, Cg.T, atol=1e-9 * np.abs(Cf).max())


def test_element_rank_rigid_modes_and_quadrature():
    Cf, Df = C.fibre_stiffness(W)
    Cg, Dg = C.rotated_stiffness(Cf, Df, 0.3)
    h = 0.5
    K = C.element_matrix(Cg, Dg, h)
    np.testing.assert_allclose(K, K.T, atol=1e-9 * np.abs(K).max())
    ev = np.linalg.eigvalsh(K)
    assert np.sum(np.abs(ev) < 1e-10 * ev.max()) == 3
    X = (C._CORNERS + 1.0) * 0.5 * h
    d = np.zeros(12)
    d[0::3], d[1::3], d[2::3] = -X[:, 1], X[:, 0], 1.0          # rigid rotation, omega = 1
    assert np.abs(K @ d).max() < 1e-10 * np.abs(K).max() * h
    # 3x3 Gauss gives the same matrix (the integrands are at most cubic per variable)
    x, w = np.polynomial.legendre.leggauss(3)
    K3 = np.zeros((12, 12))
    for a in range(3):
        for b in range(3):
            Be, Bk = C.b_matrices(x[a], x[b], h)
            K3 += w[a] * w[b] * 0.25 * h * h * (Be.T @ Cg @ Be + Bk.T @ Dg @ Bk)
    np.testing.assert_allclose(K3, K, atol=1e-10 * np.abs(K).max())


@pytest.mark.parametrize("n", [8, 16])
def test_homogeneous_block_is_exact(n):
    Cf, _ = C.fibre_stiffness(W)
    Q11, Q12, Q22 = Cf[0, 0], Cf[0, 1], Cf[1, 1]
    eps = W["shortening"] / W["L"]
    s0, r0, d0 = C.solve_sample(W, n, np.zeros(n * n))
    k, j, i = 0, *np.meshgrid(np.arange(n + 1), np.arange(n + 1), indexing="ij")
    x = i.ravel() * (W["L"] / n)
    np.testing.assert_allclose(d0[0::3], eps * x, atol=1e-12 * abs(W["shortening"]))
    assert np.abs(d0[1::3]).max() < 1e-12 * abs(W["shortening"]) and np.abs(d0[2::3]).max() < 1e-12 * abs(eps)
    assert r0 == pytest.approx(Q11 * abs(W["shortening"]), rel=1e-11)
    assert s0 == pytest.approx(W["R_ratio"] * W["tau_y"] * Q11 / Q12, rel=1e-11)
    s9, r9, _ = C.solve_sample(W, n, np.full(n * n, 0.5 * np.pi))
    assert r9 == pytest.approx(Q22 * abs(W["shortening"]), rel=1e-10)
    assert s9 == pytest.approx(W["R_ratio"] * W["tau_y"], rel=1e-10)


def test_energy_identity_and_dense_solve():
    n = 4
    phi = np.random.default_rng(2).normal(scale=0.05, size=n * n)
    K = C.assemble(W, n, phi)
    dd, dv = C.dirichlet(n, W["shortening"])
    d = C.solve(K, dd, dv)
    R = C.reaction(K, d, n)
    assert d @ (K @ d) == pytest.approx(abs(W["shortening"]) * R, rel=1e-11)
    free = np.setdiff1d(np.arange(K.shape[0]), dd)
    Kd = K.toarray()
    dense = np.zeros_like(d)
    dense[dd] = dv
    dense[free] = np.linalg.solve(Kd[np.ix_(free, free)], -Kd[np.ix_(free, dd)] @ dv)
    np.testing.assert_allclose(dense, d, atol=1e-12 * np.abs(d).max())


@pytest.mark.parametrize("omega", [W["omega1"], W["omega2"]])
def test_exponential_kernel_eigenpairs(omega):
    a = W["L"]
    mu, w = C.exp_eig_1d(a, omega, 12)
    assert np.all(np.diff(mu) < 0)
    for i in (0, 1, 4, 11):
        for x0 in (0.0, 0.31 * a, 0.77 * a):
            lhs = si.quad(lambda y: np.exp(-abs(x0 - y) / omega) * C.exp_phi_1d(a, w[i], i, y), 0.0, a,
                          points=[x0], limit=400, epsabs=1e-13, epsrel=1e-12)[0]
            assert lhs == pytest.approx(mu[i] * C.exp_phi_1d(a, w[i], i, x0), rel=1e-9, abs=1e-12)
        assert C.exp_phi_1d(a, w[i], i, 0.0) > 0
    # orthonormal under quadrature
    xg, wg = np.polynomial.legendre.leggauss(400)
    xg, wg = (xg + 1) * 0.5 * a, wg * 0.5 * a
    Phi = np.array([C.exp_phi_1d(a, w[i], i, xg) for i in range(12)])
    np.testing.assert_allclose((Phi * wg) @ Phi.T, np.eye(12), atol=1e-10)
    # an independent discretisation: Nystrom on 800 Gauss points, leading eigenvalues
    xn, wn = np.polynomial.legendre.leggauss(800)
    xn, wn = (xn + 1) * 0.5 * a, wn * 0.5 * a
    A = np.sqrt(wn)[:, None] * np.exp(-np.abs(xn[:, None] - xn[None, :]) / omega) * np.sqrt(wn)[None, :]
    nys = np.sort(np.linalg.eigvalsh(A))[::-1][:6]
    np.testing.assert_allclose(nys, mu[:6], rtol=2e-4)


def test_telescoping_on_identical_xi():
    cfg = dict(W, kl_terms0=8, kl_terms_step=4)
    xi = rng.kl_coefficients(cfg["seed"], 2, [0, 1, 2], C.n_kl(cfg, 2))
    Q = {m: np.array([C.solve_on_mesh(cfg, m, x) for x in xi]) for m in range(3)}
    tel = Q[0].mean(0) + (Q[1] - Q[0]).mean(0) + (Q[2] - Q[1]).mean(0)
    np.testing.assert_allclose(tel, Q[2].mean(0), rtol=1e-13)
    # a level pair's coarse value is the sample's own solve on the coarser mesh
    qf, qc = C.level_pair(cfg, 2, [0])
    np.testing.assert_allclose(qf[0], Q[2][0], rtol=1e-13)
    np.testing.assert_allclose(qc[0], Q[1][0], rtol=1e-13)


def test_rotation_direction():
    # a uniform stretch along the fibre direction n = (cos phi, sin phi) is pure fibre strain,
    # so its energy is Q11; rotating by -phi instead gives a mixed strain for phi not k pi / 2
    Cf, Df = C.fibre_stiffness(W)
    for phi in (0.2, 0.9, -0.4):
        n = np.array([np.cos(phi), np.sin(phi)])
        Cg, Dg = C.rotated_stiffness(Cf, Df, phi)
        e = C._vec(np.outer(n, n))
        assert e @ Cg @ e == pytest.approx(Cf[0, 0], rel=1e-12)
        assert n @ Dg @ n == pytest.approx(Df[0, 0], rel=1e-12)   # fibre-direction curvature
        t = np.array([-n[1], n[0]])
        assert t @ Dg @ t == pytest.approx(Df[1, 1], rel=1e-12)


def test_kl_basis_correlations():
    # B B^T approaches the kernel s^2 exp(-|dx| / w1 - |dy| / w2) at the centroids: along x
    # (the fibre direction) the correlation length is omega1, across it omega2
    n = 4
    B, modes = C.kl_basis(W, n, 400)
    G = B @ B.T
    s2 = W["kl_std"] ** 2
    # the pointwise variance kept equals, up to the eigenfunctions' spatial variation, the
    # share of the Mercer trace (a^2) the kept products mu^x_i mu^y_j hold
    a = W["L"]
    mux, _ = C.exp_eig_1d(a, W["omega1"], 401)
    muy, _ = C.exp_eig_1d(a, W["omega2"], 401)
    kept = sum(mux[i] * muy[j] for i, j in modes) / (a * a)
    assert 0.9 < kept < 1.0
    np.testing.assert_allclose(np.diag(G) / s2, kept, atol=0.005)
    # the omitted short-scale modes raise the normalised correlations by a few hundredths;
    # swapping the axes would give exp(-h / omega2) = 0.10 where exp(-h / omega1) = 0.54 is due
    h = a / n
    cor = G / np.sqrt(np.outer(np.diag(G), np.diag(G)))
    assert cor[0, 1] == pytest.approx(np.exp(-h / W["omega1"]), abs=0.05)          # (0,0)-(1,0)
    assert cor[0, n] == pytest.approx(np.exp(-h / W["omega2"]), abs=0.05)          # (0,0)-(0,1)
    assert cor[0, n + 1] == pytest.approx(np.exp(-h / W["omega1"] - h / W["omega2"]), abs=0.05)
    # the 1D Mercer trace: the eigenvalues of exp(-|x - y| / w) on [0, a] sum to a
    mu, _ = C.exp_eig_1d(a, W["omega2"], 4000)
    # w_i ~ i pi / a, so mu_i ~ 2 c a^2 / (pi i)^2 and the terms past N hold 2 c a / (pi^2 N) of a
    tail = 2.0 * a / (np.pi ** 2 * 4000 * W["omega2"])
    assert mu.sum() / a == pytest.approx(1.0 - tail, abs=0.1 * tail)
