"""Pins for the plane-strain stiffness and its rotation (Sec. 3.1, C* = T^-1 C T)."""
import numpy as np
import pytest

from oracle import material
from workloads import STRIP_FP64_3LEVEL as C1

C = material.material_from_cfg(C1)


def test_identity_and_quarter_turn():
    np.testing.assert_allclose(material.rotate(C, 0.0), C, rtol=0, atol=1e-6)
    R = material.rotate(C, np.pi / 2)
    assert R[0, 0] == pytest.approx(C[1, 1], rel=1e-13)
    assert R[1, 1] == pytest.approx(C[0, 0], rel=1e-13)
    assert R[0, 1] == pytest.approx(C[0, 1], rel=1e-13)
    assert R[2, 2] == pytest.approx(C[2, 2], rel=1e-13)
    assert abs(R[0, 2]) < 1e-12 * C[0, 0] and abs(R[1, 2]) < 1e-12 * C[0, 0]


@pytest.mark.parametrize("theta", [0.03, -0.2, 0.7, 1.3, 2.9])
def test_invariants_period_and_symmetry(theta):
    R = material.rotate(C, theta)
    np.testing.assert_allclose(R, R.T, atol=1e-6)
    inv1 = lambda M: M[0, 0] + M[1, 1] + 2 * M[0, 1]      # Tsai-Pagano invariants
    inv2 = lambda M: M[2, 2] - M[0, 1]
    assert inv1(R) == pytest.approx(inv1(C), rel=1e-13)
    assert inv2(R) == pytest.approx(inv2(C), rel=1e-12)
    np.testing.assert_allclose(material.rotate(C, theta + np.pi), R, rtol=1e-12, atol=1e-3)
    M = material.rotate(C, -theta)
    np.testing.assert_allclose(M[[0, 0, 1, 2], [0, 1, 1, 2]], R[[0, 0, 1, 2], [0, 1, 1, 2]], rtol=1e-12)
    np.testing.assert_allclose(M[[0, 1], [2, 2]], -R[[0, 1], [2, 2]], rtol=1e-10)


@pytest.mark.parametrize("theta", [0.05, 0.6, 2.2])
def test_strain_energy_is_frame_invariant(theta):
    """e^T C_bar e equals the fibre-frame energy of the rotated strain."""
    R = material.rotate(C, theta)
    for e in np.random.default_rng(1).standard_normal((5, 3)):
        el = material.t_eps(theta) @ e
        assert e @ R @ e == pytest.approx(el @ C @ el, rel=1e-12)
        # and the fibre-frame stress of the global stress is C times the fibre-frame strain
        np.testing.assert_allclose(material.fibre_stress(R @ e, theta), C @ el, rtol=1e-10,
                                   atol=1e-12 * np.abs(C @ el).max())


def test_closed_form_transformed_stiffness():
    """Expanded trigonometric form of the transformed reduced stiffness."""
    Q11, Q12, Q22, Q66 = C[0, 0], C[0, 1], C[1, 1], C[2, 2]
    for t in (0.1, 0.45, 1.1):
        c, s = np.cos(t), np.sin(t)
        R = material.rotate(C, t)
        assert R[0, 0] == pytest.approx(Q11 * c**4 + 2 * (Q12 + 2 * Q66) * s**2 * c**2 + Q22 * s**4, rel=1e-12)
        assert R[1, 1] == pytest.approx(Q11 * s**4 + 2 * (Q12 + 2 * Q66) * s**2 * c**2 + Q22 * c**4, rel=1e-12)
        assert R[0, 1] == pytest.approx((Q11 + Q22 - 4 * Q66) * s**2 * c**2 + Q12 * (s**4 + c**4), rel=1e-12)
        assert R[2, 2] == pytest.approx((Q11 + Q22 - 2 * Q12 - 2 * Q66) * s**2 * c**2 + Q66 * (s**4 + c**4), rel=1e-12)
        assert R[0, 2] == pytest.approx((Q11 - Q12 - 2 * Q66) * s * c**3 + (Q12 - Q22 + 2 * Q66) * s**3 * c, rel=1e-10)


def test_isotropic_plane_strain_is_lame():
    E, nu = 70e9, 0.3
    M = material.plane_strain_stiffness(E, E, E / (2 * (1 + nu)), nu, E, nu, nu)
    lam = E * nu / ((1 + nu) * (1 - 2 * nu))
    mu = E / (2 * (1 + nu))
    np.testing.assert_allclose(M, [[lam + 2 * mu, lam, 0], [lam, lam + 2 * mu, 0], [0, 0, mu]], rtol=1e-13)
