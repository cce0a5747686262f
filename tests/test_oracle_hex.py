"""Pins of the 3D Hex8 oracle against what the mathematics fixes (no GPU).

- rotation about y: the identity at 0, period pi, the inverse rotation, isotropy,
  frame-invariant strain energy, and the fibre-direction response of the rotated
  compliance (a uniaxial stress along the rotated fibre stretches it by sigma / E11),
  with the Voigt rotation rebuilt from the Bond stress-transformation matrix;
- element: six rigid-body modes (rank 18), 2x2x2 Gauss equal to 3x3x3 on a cube,
  the energy of a linear displacement field equal to volume * eps : C : eps;
- block: the homogeneous block under the roller conditions reproduces the uniform
  uniaxial stress state exactly (reaction A * shortening / (lx S'_11)); the clamped
  solve satisfies d^T K d = shortening * reaction; the 3D solve of a block one
  element thick with free faces is symmetric in the mesh numbering (refining y does
  not change the homogeneous response);
- telescoping: on identical xi the level pairs' differences sum to the finest mean.
"""
import numpy as np
import pytest

from oracle import hex as H
from oracle import kl, rng
from workloads import HEX8_MIXED_4LEVEL as W


def bond_stress(R):
    """6x6 Bond matrix of a rotation (sigma' = M sigma in Voigt 11, 22, 33, 23, 13, 12)."""
    M = np.zeros((6, 6))
    idx = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
    for I, (i, j) in enumerate(idx):
        for J, (k, l) in enumerate(idx):
            if J < 3:
                M[I, J] = R[i, k] * R[j, l]
            else:
                M[I, J] = R[i, k] * R[j, l] + R[i, l] * R[j, k]
    return M


@pytest.mark.parametrize("theta", [0.0, 0.05, -0.3, 1.1, np.pi / 2])
def test_rotation_matches_bond_matrix(theta):
    C = H.material_stiffness(W)
    M = bond_stress(H.rotation_y(theta))
    np.testing.assert_allclose(H.rotate(C, theta), M @ C @ M.T, rtol=1e-12, atol=1e-3)


def test_rotation_identities():
    C = H.material_stiffness(W)
    np.testing.assert_allclose(H.rotate(C, 0.0), C, rtol=1e-14)
    np.testing.assert_allclose(H.rotate(C, np.pi), C, rtol=1e-12, atol=1e-2)
    np.testing.assert_allclose(H.rotate(H.rotate(C, 0.4), -0.4), C, rtol=1e-12, atol=1e-2)
    lam, mu = 3e9, 2e9
    Ciso = np.zeros((6, 6))
    Ciso[:3, :3] = lam
    Ciso[range(3), range(3)] += 2 * mu
    Ciso[range(3, 6), range(3, 6)] = mu
    np.testing.assert_allclose(H.rotate(Ciso, 0.7), Ciso, rtol=1e-12, atol=1e-3)


def test_energy_invariance_and_fibre_modulus():
    C = H.material_stiffness(W)
    g = np.random.default_rng(1)
    theta = 0.37
    Cr = H.rotate(C, theta)
    R = H.rotation_y(theta)
    for _ in range(5):
        e_mat = g.normal(size=6)            # engineering strain in the material frame
        E = np.array([[e_mat[0], e_mat[5] / 2, e_mat[4] / 2], [e_mat[5] / 2, e_mat[1], e_mat[3] / 2],
                      [e_mat[4] / 2, e_mat[3] / 2, e_mat[2]]])
        Eg = R @ E @ R.T                    # the same strain in the global frame
        e_glob = np.array([Eg[0, 0], Eg[1, 1], Eg[2, 2], 2 * Eg[1, 2], 2 * Eg[0, 2], 2 * Eg[0, 1]])
        assert e_glob @ Cr @ e_glob == pytest.approx(e_mat @ C @ e_mat, rel=1e-12)
    # uniaxial stress along the rotated fibre: fibre strain sigma / E11
    a1 = H.fibre_direction(theta)
    sig = 1e8 * np.outer(a1, a1)
    s6 = np.array([sig[0, 0], sig[1, 1], sig[2, 2], sig[1, 2], sig[0, 2], sig[0, 1]])
    e6 = np.linalg.solve(Cr, s6)
    Eps = np.array([[e6[0], e6[5] / 2, e6[4] / 2], [e6[5] / 2, e6[1], e6[3] / 2], [e6[4] / 2, e6[3] / 2, e6[2]]])
    assert a1 @ Eps @ a1 == pytest.approx(1e8 / W["E11"], rel=1e-12)


def test_element_rigid_modes_and_quadrature():
    C = H.rotate(H.material_stiffness(W), 0.2)
    h = 0.03125
    K2 = H.element_matrix(C, h, order=2)
    K3 = H.element_matrix(C, h, order=3)
    np.testing.assert_allclose(K2, K3, rtol=1e-11, atol=1e-3 * np.abs(K2).max() * 1e-9)
    np.testing.assert_allclose(K2, K2.T, rtol=1e-13, atol=1e-6)
    ev = np.linalg.eigvalsh(K2)
    assert np.sum(np.abs(ev) < 1e-9 * ev.max()) == 6
    assert np.all(ev > -1e-9 * ev.max())
    # rigid rotation about z: u = -y, v = x
    X = H._CORNERS * h
    d = np.zeros(24)
    d[0::3], d[1::3] = -X[:, 1], X[:, 0]
    assert np.abs(K2 @ d).max() < 1e-9 * np.abs(K2).max() * h


def test_element_energy_of_linear_field():
    C = H.rotate(H.material_stiffness(W), -0.15)
    h = 0.5
    g = np.random.default_rng(2)
    G = g.normal(size=(3, 3)) * 1e-3       # displacement gradient
    X = H._CORNERS * h
    d = (X @ G.T).ravel()
    eps = 0.5 * (G + G.T)
    e6 = np.array([eps[0, 0], eps[1, 1], eps[2, 2], 2 * eps[1, 2], 2 * eps[0, 2], 2 * eps[0, 1]])
    K = H.element_matrix(C, h)
    assert d @ K @ d == pytest.approx(h ** 3 * e6 @ C @ e6, rel=1e-12)


@pytest.mark.parametrize("theta", [0.0, 0.06, -0.2])
def test_homogeneous_block_uniform_stress(theta):
    nx, ny, nz = 8, 2, 2
    cfg = dict(W)
    h = cfg["lx"] / nx
    ncol = nx * nz
    r, s, d = H.solve_sample(cfg, nx, ny, nz, np.full(ncol, theta), bc="roller")
    Sr = np.linalg.inv(H.rotate(H.material_stiffness(cfg), theta))
    area = (ny * h) * (nz * h)
    assert r == pytest.approx(area * cfg["shortening"] / (cfg["lx"] * Sr[0, 0]), rel=1e-10)
    # u is exactly linear in x
    u = d[0::3].reshape(nz + 1, ny + 1, nx + 1)
    np.testing.assert_allclose(u, np.broadcast_to(-cfg["shortening"] * np.arange(nx + 1) * h / cfg["lx"],
                                                  u.shape), atol=1e-15)


def test_energy_identity_clamped():
    nx, ny, nz = 8, 2, 2
    g = np.random.default_rng(3)
    theta = g.normal(scale=0.05, size=nx * nz)
    h = W["lx"] / nx
    C = H.material_stiffness(W)
    Cc = np.array([H.rotate(C, t) for t in theta])
    K = H.assemble(nx, ny, nz, h, Cc)
    dd, dv = H.dirichlet(nx, ny, nz, W["shortening"])
    d = H.solve(K, dd, dv)
    R = H.reaction(K, d, nx, ny, nz)
    assert d @ (K @ d) == pytest.approx(W["shortening"] * R, rel=1e-10)
    # equilibrium: reactions on the two end faces balance in x
    Kd = K @ d
    left = [3 * H.node_index(0, j, k, nx, ny) for k in range(nz + 1) for j in range(ny + 1)]
    assert np.sum(Kd[left]) == pytest.approx(R, rel=1e-10)


def test_telescoping_on_identical_xi():
    cfg = dict(W, nx0=8, ny0=2, nz0=1, kl_terms=12, levels=3)
    xi = rng.kl_coefficients(cfg["seed"], 2, list(range(3)), cfg["kl_terms"])
    Q = {}
    for lev in range(3):
        nx, ny, nz = cfg["nx0"] << lev, cfg["ny0"] << lev, cfg["nz0"] << lev
        cx, cz = H.column_centroids(cfg, nx, nz)
        B, _, _ = kl.kl_basis(cfg["lx"], cfg["lz"], cfg["kl_corr"], np.deg2rad(cfg["kl_std_deg"]), 64,
                              cfg["kl_terms"], cx, cz)
        th = xi @ B.T
        Q[lev] = np.array([H.solve_sample(cfg, nx, ny, nz, th[s])[:2] for s in range(3)])
    tel = Q[0].mean(0) + (Q[1] - Q[0]).mean(0) + (Q[2] - Q[1]).mean(0)
    np.testing.assert_allclose(tel, Q[2].mean(0), rtol=1e-13)
    # and refinement changes the reaction by a shrinking amount
    assert abs(Q[2][0, 0] - Q[1][0, 0]) < abs(Q[1][0, 0] - Q[0][0, 0])


@pytest.mark.parametrize("theta", [0.0, 0.06, -0.2, 0.7])
def test_fibre_stress_of_the_homogeneous_block(theta):
    """Under the roller conditions the stress is uniaxial, sigma_xx = -shortening /
    (lx S'_11), so the fibre-direction stress a1 . sigma a1 is sigma_xx cos^2 theta
    in every element (the 3D counterpart of the strip's c^2 sigma_xx pin)."""
    nx, ny, nz = 8, 2, 2
    cfg = dict(W)
    _, s, _ = H.solve_sample(cfg, nx, ny, nz, np.full(nx * nz, theta), bc="roller")
    Sr = np.linalg.inv(H.rotate(H.material_stiffness(cfg), theta))
    sxx = -cfg["shortening"] / (cfg["lx"] * Sr[0, 0])
    assert s == pytest.approx(max(0.0, -sxx * np.cos(theta) ** 2), rel=1e-10)


def test_fibre_stress_of_a_general_uniform_strain():
    """All six strain components at once, so that a misplaced shear slot or a wrong
    centroid strain shows: for a linear displacement field u = G x the centroid strain
    is sym(G) exactly, and the fibre stress equals the first material-frame stress
    component (C eps')_1, eps' = R^T eps R, computed without the rotated stiffness."""
    nx, ny, nz = 8, 2, 2
    cfg = dict(W)
    h = cfg["lx"] / nx
    g = np.random.default_rng(7)
    G = g.normal(size=(3, 3)) * 1e-3
    G[0, 0] = -2e-3                     # compressive along x
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    X = np.stack([i.ravel() * h, j.ravel() * h, k.ravel() * h], axis=1)   # node n = (k (ny+1) + j)(nx+1) + i
    d = (X @ G.T).ravel()
    theta = g.normal(scale=0.4, size=nx * nz)
    C = H.material_stiffness(cfg)
    C_col = np.array([H.rotate(C, t) for t in theta])
    eps = 0.5 * (G + G.T)
    expected = 0.0
    for col in range(nx * nz):
        xc = (col % nx + 0.5) * h
        if not (cfg["omega_x0"] <= xc <= cfg["omega_x1"]):
            continue
        R = H.rotation_y(theta[col])
        E = R.T @ eps @ R
        e_mat = np.array([E[0, 0], E[1, 1], E[2, 2], 2 * E[1, 2], 2 * E[0, 2], 2 * E[0, 1]])
        expected = max(expected, -(C @ e_mat)[0])
    got = H.max_fibre_compression(cfg, d, C_col, theta, nx, ny, nz, h)
    assert expected > 0
    assert got == pytest.approx(expected, rel=1e-10)


def test_fibre_stress_is_taken_at_the_centroid():
    """u = (a x y, 0, 0) is trilinear, so the element strain is exact: e_xx = a y. At
    theta = 0 the fibre stress is C_11 a y_c at the element centroid (y_c = (j + 1/2) h);
    with a < 0 the maximum compression sits in the top element row."""
    nx, ny, nz = 8, 2, 2
    cfg = dict(W)
    h = cfg["lx"] / nx
    a = -1e-2
    k, j, i = np.meshgrid(np.arange(nz + 1), np.arange(ny + 1), np.arange(nx + 1), indexing="ij")
    x, y = i.ravel() * h, j.ravel() * h
    d = np.zeros(3 * x.size)
    d[0::3] = a * x * y
    C = H.material_stiffness(cfg)
    theta = np.zeros(nx * nz)
    got = H.max_fibre_compression(cfg, d, np.array([C] * (nx * nz)), theta, nx, ny, nz, h)
    assert got == pytest.approx(-C[0, 0] * a * (ny - 0.5) * h, rel=1e-12)


def test_matrix_free_apply_equals_assembled_matrix():
    nx, ny, nz = 6, 2, 3
    h = W["lx"] / nx
    g = np.random.default_rng(11)
    C = H.material_stiffness(W)
    Cc = np.array([H.rotate(C, t) for t in g.normal(scale=0.2, size=nx * nz)])
    K = H.assemble(nx, ny, nz, h, Cc)
    x = g.normal(size=K.shape[0])
    np.testing.assert_allclose(H.apply(nx, ny, nz, h, Cc, x), K @ x, rtol=1e-12, atol=1e-12 * np.abs(K @ x).max())


def test_cg_solve_equals_direct_solve():
    nx, ny, nz = 8, 2, 2
    g = np.random.default_rng(12)
    theta = g.normal(scale=0.05, size=nx * nz)
    r1, s1, d1 = H.solve_sample(W, nx, ny, nz, theta)
    r2, s2, d2 = H.solve_sample(W, nx, ny, nz, theta, solver="cg")
    assert r2 == pytest.approx(r1, rel=1e-10)
    assert s2 == pytest.approx(s1, rel=1e-8)
    assert np.abs(d2 - d1).max() <= 1e-8 * np.abs(d1).max()
