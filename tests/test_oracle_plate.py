"""Pins of the panel-buckling oracle against what the mathematics and the paper fix (no GPU).

- laminate: a single 0-degree ply gives A = Q t, B = 0, D = Q t^3 / 12 with the textbook
  plane-stress Q; the rotated stiffness at 90 degrees swaps the axes, keeps the two
  rotation invariants and matches the textbook Q_bar16 at 30 degrees; a symmetric
  laminate has B = 0 and D* = D; the knock-down D - D* is positive semi-definite;
- element: the three rigid plate modes (w = 1; w = x with theta_x = 1; w = y with
  theta_y = 1) carry no energy and the 1-point shear leaves rank 7; the geometric
  form integrates w = x exactly;
- closed forms: the Mindlin Fourier solution tends to the Kirchhoff one as the shear
  stiffness grows, and the Kirchhoff one gives k = 4 for a square isotropic plate; the
  FE load of a cross-ply plate converges to the Mindlin closed form at O(h^2);
- the paper's pristine panel (Sec. 4.2, tests/golden/panel_pristine_load.txt): closed
  form and FE within 0.5 % of the printed 278.59 kN; the FE load decreases with
  refinement (one-sided convergence, Sec. 4.2);
- symmetries: mirroring every ply angle, or reversing the stacking order, leaves the
  critical load unchanged; the dense and sparse eigensolvers agree;
- perturbations: the first n_plies normals of each sample's stream scaled by 3 degrees;
- the soft support never gives a higher load than the hard one (a larger admissible space).
"""
import os

import numpy as np
import pytest

from oracle import plate as P
from workloads import PANEL_C5_4LEVEL, PANEL_RM_4LEVEL as W

HERE = os.path.dirname(os.path.abspath(__file__))


def golden():
    vals = {}
    with open(os.path.join(HERE, "golden", "panel_pristine_load.txt")) as f:
        for line in f:
            if ":" in line and not line.startswith("#"):
                k, v = line.split(":")
                vals[k.strip()] = float(v)
    return vals


def textbook_q(E1, E2, G12, nu12):
    nu21 = nu12 * E2 / E1
    d = 1.0 - nu12 * nu21
    return np.array([[E1 / d, nu12 * E2 / d, 0.0], [nu12 * E2 / d, E2 / d, 0.0], [0.0, 0.0, G12]])


def test_single_ply_laminate():
    Q = P.lamina_q(W["E11"], W["E22"], W["G12"], W["nu12"])
    assert np.allclose(Q, textbook_q(W["E11"], W["E22"], W["G12"], W["nu12"]), rtol=1e-13)
    t = 0.8
    A, B, D = P.laminate_abd(Q, [0.0], t)
    assert np.allclose(A, Q * t, rtol=1e-13)
    assert np.abs(B).max() < 1e-9 * np.abs(Q).max()
    assert np.allclose(D, Q * t ** 3 / 12.0, rtol=1e-12)


def test_rotated_stiffness():
    Q = textbook_q(130e3, 9.25e3, 5.13e3, 0.36)
    Q90 = P.rotate_q(Q, np.pi / 2)
    assert np.isclose(Q90[0, 0], Q[1, 1]) and np.isclose(Q90[1, 1], Q[0, 0]) and np.isclose(Q90[0, 1], Q[0, 1])
    for a in np.linspace(0, np.pi, 7):
        Qb = P.rotate_q(Q, a)
        assert np.isclose(Qb[0, 0] + Qb[1, 1] + 2 * Qb[0, 1], Q[0, 0] + Q[1, 1] + 2 * Q[0, 1])
        assert np.isclose(Qb[2, 2] - Qb[0, 1], Q[2, 2] - Q[0, 1])
    a = np.radians(30.0)
    c, s = np.cos(a), np.sin(a)
    q11, q12, q22, q66 = Q[0, 0], Q[0, 1], Q[1, 1], Q[2, 2]
    q16 = (q11 - q12 - 2 * q66) * s * c ** 3 + (q12 - q22 + 2 * q66) * s ** 3 * c
    assert np.isclose(P.rotate_q(Q, a)[0, 2], q16, rtol=1e-12)


def test_symmetric_laminate_and_knockdown():
    Q = P.lamina_q(W["E11"], W["E22"], W["G12"], W["nu12"])
    ang = np.radians([0, 90, 90, 0])
    A, B, D = P.laminate_abd(Q, ang, 0.5)
    assert np.abs(B).max() < 1e-9 * np.abs(A).max()
    assert np.allclose(P.knocked_down_d(A, B, D), D)
    ang = np.radians([0, 45, 90, -30, 10])
    A, B, D = P.laminate_abd(Q, ang, 0.5)
    assert np.abs(B).max() > 1.0
    assert np.linalg.eigvalsh(D - P.knocked_down_d(A, B, D)).min() > -1e-9 * np.abs(D).max()


def test_element_rigid_modes_and_rank():
    Ds, kgt = P.panel_stiffness(W, np.zeros(8))
    hx, hy = 26.5, 26.5
    Ke, Ge = P.element_matrices(Ds, kgt, hx, hy)
    xy = np.array([(0, 0), (hx, 0), (hx, hy), (0, hy)], dtype=float)
    modes = []
    for w, tx, ty in [(lambda x, y: 1.0, 0.0, 0.0), (lambda x, y: x, 1.0, 0.0), (lambda x, y: y, 0.0, 1.0)]:
        v = np.zeros(12)
        for a in range(4):
            v[3 * a] = w(*xy[a])
            v[3 * a + 1] = tx
            v[3 * a + 2] = ty
        modes.append(v)
        assert np.abs(Ke @ v).max() < 1e-9 * np.abs(Ke).max()
    sv = np.linalg.svd(Ke, compute_uv=False)
    assert (sv > 1e-10 * sv[0]).sum() == 7
    v = np.zeros(12)
    v[0::3] = xy[:, 0]
    assert np.isclose(v @ Ge @ v, hx * hy, rtol=1e-13)
    assert np.allclose(Ke, Ke.T) and np.allclose(Ge, Ge.T)


def test_closed_forms():
    D = np.diag([3.0, 2.0, 0.7])
    D[0, 1] = D[1, 0] = 0.4
    assert np.isclose(P.mindlin_navier(D, 1e6, 500.0, 300.0), P.kirchhoff_navier(D, 500.0, 300.0), rtol=1e-6)
    assert P.mindlin_navier(D, 1.0, 500.0, 300.0) < P.kirchhoff_navier(D, 500.0, 300.0)
    Dm, nu, b = 1000.0, 0.3, 200.0
    Diso = np.array([[Dm, nu * Dm, 0.0], [nu * Dm, Dm, 0.0], [0.0, 0.0, (1 - nu) * Dm / 2]])
    assert np.isclose(P.kirchhoff_navier(Diso, b, b), 4.0 * np.pi ** 2 * Dm / b ** 2, rtol=1e-12)


def test_fe_converges_to_mindlin_closed_form():
    cfg = dict(W, lx=500.0, ly=500.0, plies_deg=(0, 90, 0, 90, 90, 0, 90, 0), t_ply=0.125)
    Ds, kgt = P.panel_stiffness(cfg, np.zeros(8))
    assert abs(Ds[0, 2]) < 1e-9 and abs(Ds[1, 2]) < 1e-9   # specially orthotropic
    ref = P.mindlin_navier(Ds, kgt, 500.0, 500.0)
    errs = [P.solve_sample(cfg, n, n, np.zeros(8), bc="hard") / ref - 1.0 for n in (16, 32, 64)]
    assert all(e > 0 for e in errs)
    assert 3.5 < errs[0] / errs[1] < 4.5 and 3.5 < errs[1] / errs[2] < 4.5
    assert errs[2] < 1e-3


def test_paper_pristine_panel():
    g = golden()
    Ds, kgt = P.panel_stiffness(W, np.zeros(8))
    closed = P.mindlin_navier(Ds, kgt, W["lx"], W["ly"]) * W["ly"] * 1e-3
    assert abs(closed / g["pristine_load_kN"] - 1.0) < 3e-3
    loads = [P.solve_sample(W, 12 * k, 4 * k, np.zeros(8), bc="hard") * W["ly"] * 1e-3 for k in (2, 4, 8)]
    assert loads[0] > loads[1] > loads[2] > closed
    assert abs(loads[2] / g["pristine_load_kN"] - 1.0) < 5e-3
    assert g["threshold_kN"] < g["pristine_load_kN"]


def test_mirror_and_reversal_symmetry():
    rng = np.random.default_rng(3)
    phi = np.radians(3.0) * rng.standard_normal(8)
    base = P.solve_sample(W, 24, 8, phi, bc="hard")
    mirrored = dict(W, plies_deg=tuple(-a for a in W["plies_deg"]))
    assert np.isclose(P.solve_sample(mirrored, 24, 8, -phi, bc="hard"), base, rtol=1e-10)
    reversed_ = dict(W, plies_deg=tuple(reversed(W["plies_deg"])))
    assert np.isclose(P.solve_sample(reversed_, 24, 8, phi[::-1], bc="hard"), base, rtol=1e-10)


def test_dense_and_sparse_eigensolvers_agree():
    rng = np.random.default_rng(4)
    phi = np.radians(3.0) * rng.standard_normal(8)
    for bc in ("hard", "soft"):
        a = P.solve_sample(W, 24, 8, phi, bc=bc, dense=True)
        b = P.solve_sample(W, 24, 8, phi, bc=bc, dense=False)
        assert np.isclose(a, b, rtol=1e-10)


def test_perturbations_and_level_pair():
    phi = P.sample_perturbations(W, 1, np.arange(4000))
    assert phi.shape == (4000, 8)
    sd = np.degrees(phi.std())
    assert abs(sd - 3.0) < 0.1 and abs(np.degrees(phi.mean())) < 0.1
    qf, qc = P.level_pair(W, 1, [5, 6])
    for k, sid in enumerate((5, 6)):
        p = P.sample_perturbations(W, 1, [sid])[0]
        assert np.allclose(qf[k], P.solve_mesh(W, 1, p)) and np.allclose(qc[k], P.solve_mesh(W, 0, p))
    assert qf[:, 1].tolist() == [1.0 if v < W["p_star"] else 0.0 for v in qf[:, 0]]


def test_soft_support_never_stiffer_than_hard():
    # the soft support frees the tangential rotation, so its admissible space contains the
    # hard one's and the smallest Rayleigh quotient can only fall
    rng = np.random.default_rng(7)
    for _ in range(3):
        phi = np.radians(3.0) * rng.standard_normal(8)
        for nx, ny in ((24, 8), (48, 16)):
            soft = P.solve_sample(W, nx, ny, phi, bc="soft")
            hard = P.solve_sample(W, nx, ny, phi, bc="hard")
            assert soft < hard


def test_thin_cross_ply_panel_converges_to_mindlin_closed_form():
    """b / t = 500: a 500 x 500 mm, 1 mm cross-ply [0/90]2s panel (D16 = D26 = 0, B = 0)
    with the hard support; the selectively integrated Q4 does not lock, so the FE load
    converges at O(h^2) to the Mindlin closed form (here within 1e-4 of Kirchhoff's)."""
    w = dict(PANEL_C5_4LEVEL, plies_deg=(0, 90, 0, 90, 90, 0, 90, 0))
    D, kgt = P.panel_stiffness(w, np.zeros(8))
    assert abs(D[0, 2]) < 1e-9 * D[0, 0] and abs(D[1, 2]) < 1e-9 * D[0, 0]
    ref = P.mindlin_navier(D, kgt, w["lx"], w["ly"])
    assert ref == pytest.approx(P.kirchhoff_navier(D, w["lx"], w["ly"]), rel=2e-4)
    err = [P.solve_sample(w, n, n, np.zeros(8), bc="hard") / ref - 1.0 for n in (16, 32, 64)]
    assert all(e > 0 for e in err) and err[0] < 0.01
    for a, b in zip(err, err[1:]):
        assert 3.8 < a / b < 4.2


def test_thin_panel_level_pair_uses_the_same_perturbations():
    """Config of the thin panel: a level pair's coarse value is the sample's own solve on
    the coarse mesh, and the two meshes' loads differ by little (h^2 convergence)."""
    w = PANEL_C5_4LEVEL
    qf, qc = P.level_pair(w, 1, [5, 6])
    phi = P.sample_perturbations(w, 1, [5, 6])
    for k in range(2):
        assert qc[k][0] == pytest.approx(P.solve_mesh(w, 0, phi[k])[0], rel=1e-12)
        assert abs(qf[k][0] / qc[k][0] - 1.0) < 0.01
