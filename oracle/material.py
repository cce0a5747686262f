"""Orthotropic ply stiffness in plane strain and its rotation by the local angle.

Sec. 3.1 rotates the constitutive matrix to the global axes by the misalignment
angle, C* = (T)^-1 C T. With stresses (s_xx, s_yy, s_xy) and engineering strains
(e_xx, e_yy, g_xy) the rotation reads C_bar = T_sigma(theta)^-1 C T_eps(theta),
where T_sigma and T_eps map global to fibre-frame stress and strain (fibre
direction at +theta from the x axis). The paper's notation writes one matrix T
for both; with engineering shear the two differ by the factor 2 on the shear
entries, which is the reading taken here.

Plane strain (e_33 = 0): the in-plane stiffness is the (1, 2) block of the inverse
of the 3D normal compliance, with the in-plane shear modulus G12 on the shear
diagonal. The 3D constants not given for the strip (E33, nu13, nu23) close the
material as transversely isotropic.
"""
import numpy as np


def plane_strain_stiffness(E11, E22, G12, nu12, E33, nu13, nu23):
    """3x3 fibre-frame stiffness [C11 C12 0; C12 C22 0; 0 0 G12] in plane strain."""
    S = np.array([
        [1.0 / E11, -nu12 / E11, -nu13 / E11],
        [-nu12 / E11, 1.0 / E22, -nu23 / E22],
        [-nu13 / E11, -nu23 / E22, 1.0 / E33],
    ])
    C3 = np.linalg.inv(S)
    C = np.zeros((3, 3))
    C[:2, :2] = C3[:2, :2]
    C[2, 2] = G12
    return C


def material_from_cfg(cfg):
    return plane_strain_stiffness(cfg["E11"], cfg["E22"], cfg["G12"], cfg["nu12"],
                                  cfg["E33"], cfg["nu13"], cfg["nu23"])


def t_sigma(theta):
    c, s = np.cos(theta), np.sin(theta)
    return np.array([
        [c * c, s * s, 2.0 * c * s],
        [s * s, c * c, -2.0 * c * s],
        [-c * s, c * s, c * c - s * s],
    ])


def t_eps(theta):
    c, s = np.cos(theta), np.sin(theta)
    return np.array([
        [c * c, s * s, c * s],
        [s * s, c * c, -c * s],
        [-2.0 * c * s, 2.0 * c * s, c * c - s * s],
    ])


def rotate(C, theta):
    """C_bar(theta) = T_sigma(theta)^-1 C T_eps(theta)."""
    return np.linalg.solve(t_sigma(theta), C @ t_eps(theta))


def fibre_stress(sigma, theta):
    """Fibre-frame stress components T_sigma(theta) sigma."""
    return t_sigma(theta) @ sigma
