"""Pins for the oracle's Q1 discretisation, boundary conditions and quantities of interest."""
import numpy as np
import pytest

from oracle import fem, material
from workloads import STRIP_FP64_3LEVEL as C1

C = material.material_from_cfg(C1)


@pytest.mark.parametrize("theta", [0.0, 0.035, -0.3, 1.0])
@pytest.mark.parametrize("mesh", [(4, 1), (16, 4), (7, 3), (32, 8)])
def test_homogeneous_block_closed_form(theta, mesh):
    """Uniform angle, roller ends: uniform stress s_xx = e_xx / S_bar_11 is the FE solution."""
    nx, ny = mesh
    qr, qs, d = fem.solve_sample(C1, nx, ny, np.full(nx * ny, theta), bc="roller")
    Sb = np.linalg.inv(material.rotate(C, theta))
    exx = -C1["shortening"] / C1["lx"]
    sxx = exx / Sb[0, 0]
    assert qr == pytest.approx(-sxx * C1["ly"], rel=1e-11)
    # displacement field u = exx x, v = S12 sxx y + S16 sxx x
    xs = np.tile(np.arange(nx + 1) / nx, ny + 1)
    ys = np.repeat(np.arange(ny + 1) * C1["ly"] / ny, nx + 1)
    np.testing.assert_allclose(d[0::2], exx * xs, atol=1e-15)
    np.testing.assert_allclose(d[1::2], Sb[0, 1] * sxx * ys + Sb[0, 2] * sxx * xs, atol=1e-15)
    # fibre-direction stress at every centroid: c^2 s_xx
    s11 = np.cos(theta) ** 2 * sxx
    assert qs == pytest.approx(max(0.0, -s11), rel=1e-10)


def test_element_matrix_properties():
    Cb = np.stack([material.rotate(C, t) for t in (0.0, 0.3, -1.1)])
    for hx, hy in ((1.0, 1.0), (0.25, 0.125)):
        K2 = fem.element_matrices(Cb, hx, hy, order=2)
        K3 = fem.element_matrices(Cb, hx, hy, order=3)   # 2x2 is exact for rectangles
        np.testing.assert_allclose(K2, K3, rtol=1e-12, atol=1e-12 * np.abs(K3).max())
        np.testing.assert_allclose(K2, np.transpose(K2, (0, 2, 1)), atol=1e-12 * np.abs(K2).max())
        xs = np.array([0, hx, hx, 0.0])
        ys = np.array([0, 0, hy, hy.__float__() if hasattr(hy, "__float__") else hy])
        rigid = [np.ravel(np.column_stack([np.ones(4), np.zeros(4)])),
                 np.ravel(np.column_stack([np.zeros(4), np.ones(4)])),
                 np.ravel(np.column_stack([-ys, xs]))]
        for Ke in K2:
            for r in rigid:
                assert np.abs(Ke @ r).max() < 1e-10 * np.abs(Ke).max()
            ev = np.linalg.eigvalsh(Ke)
            assert np.sum(ev > 1e-9 * ev.max()) == 5 and ev.min() > -1e-9 * ev.max()


def test_element_energy_by_brute_force_integration():
    """p^T K_e p against the strain energy of the interpolated field, integrated by a fine
    midpoint rule on derivatives taken by central differences of the bilinear interpolant."""
    hx, hy = 0.5, 0.25
    Cb = material.rotate(C, 0.4)
    Ke = fem.element_matrices(Cb[None], hx, hy)[0]
    p = np.random.default_rng(2).standard_normal(8)
    xs, ys = np.array([0, hx, hx, 0]), np.array([0, 0, hy, hy])

    def field(x, y):
        a, b = x / hx, y / hy
        N = np.array([(1 - a) * (1 - b), a * (1 - b), a * b, (1 - a) * b])
        return N @ p[0::2], N @ p[1::2]

    n, h = 200, 1e-6
    energy = 0.0
    for x in (np.arange(n) + 0.5) * hx / n:
        for y in (np.arange(n) + 0.5) * hy / n:
            ux = (field(x + h, y)[0] - field(x - h, y)[0]) / (2 * h)
            uy = (field(x, y + h)[0] - field(x, y - h)[0]) / (2 * h)
            vx = (field(x + h, y)[1] - field(x - h, y)[1]) / (2 * h)
            vy = (field(x, y + h)[1] - field(x, y - h)[1]) / (2 * h)
            e = np.array([ux, vy, uy + vx])
            energy += e @ Cb @ e
    energy *= hx * hy / n ** 2
    assert p @ Ke @ p == pytest.approx(energy, rel=1e-4)


@pytest.mark.parametrize("mesh", [(2, 1), (4, 1), (4, 2)])
def test_dense_brute_force_solve(mesh):
    nx, ny = mesh
    theta = np.random.default_rng(nx * 10 + ny).normal(0, 0.05, nx * ny)
    Cb = fem.rotated_stiffness(C, theta)
    K = fem.assemble(nx, ny, 1.0, 0.25, Cb).toarray()
    dd, dv = fem.dirichlet(nx, ny, 1e-3)
    n = K.shape[0]
    # brute force: enforce Dirichlet rows as identity in a dense system
    A = K.copy()
    b = np.zeros(n)
    A[dd, :] = 0.0
    A[dd, dd] = 1.0
    b[dd] = dv
    d_dense = np.linalg.solve(A, b)
    _, _, d = fem.solve_sample(C1, nx, ny, theta)
    np.testing.assert_allclose(d, d_dense, rtol=1e-10, atol=1e-12 * np.abs(d_dense).max())


def test_reaction_equilibrium_and_energy_identity():
    nx, ny = 16, 4
    theta = np.random.default_rng(9).normal(0, 0.035, nx * ny)
    Cb = fem.rotated_stiffness(C, theta)
    K = fem.assemble(nx, ny, 1.0, 0.25, Cb)
    dd, dv = fem.dirichlet(nx, ny, C1["shortening"])
    d = fem.solve(K, dd, dv)
    f = K @ d
    free = np.setdiff1d(np.arange(K.shape[0]), dd)
    assert np.abs(f[free]).max() < 1e-8 * np.abs(f).max()
    assert abs(np.sum(f[0::2])) < 1e-9 * np.abs(f).max()          # x-equilibrium of reactions
    assert abs(np.sum(f[1::2])) < 1e-9 * np.abs(f).max()          # y-equilibrium
    qr = fem.reaction(K, d, nx, ny)
    assert d @ (K @ d) == pytest.approx(C1["shortening"] * qr, rel=1e-12)   # d^T K d = delta R
    assert qr > 0


def test_patch_test_interior_forces_vanish():
    nx, ny = 6, 3
    Cb = fem.rotated_stiffness(C, np.random.default_rng(4).normal(0, 0.3, nx * ny))
    Cb[:] = Cb[0]                                   # one material, any orientation
    K = fem.assemble(nx, ny, 1.0, 0.25, Cb)
    xs = np.tile(np.arange(nx + 1) / nx, ny + 1)
    ys = np.repeat(np.arange(ny + 1) * 0.25 / ny, nx + 1)
    d = np.empty(2 * xs.size)
    d[0::2] = 1e-3 * xs + 2e-4 * ys
    d[1::2] = -3e-4 * ys + 5e-4 * xs
    f = K @ d
    interior = [(j * (nx + 1) + i) for j in range(1, ny) for i in range(1, nx)]
    idx = np.concatenate([2 * np.array(interior), 2 * np.array(interior) + 1])
    assert np.abs(f[idx]).max() < 1e-10 * np.abs(f).max()
