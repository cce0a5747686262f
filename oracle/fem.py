"""Bilinear Q1 finite elements for the strip: K d = f (Eq. matrixinplane).

The weak form (Eq. VarCosserat, here without the Cosserat rotation and couple
stress: classical anisotropic plane-strain elasticity, 2 DOF per node) is
discretised with 4-node bilinear quadrilaterals on the structured nx x ny grid of
[0, lx] x [0, ly]. Each element carries one angle (its centroid value) and so one
rotated stiffness C_bar_e. Element matrices use the 2x2 Gauss rule:

    K_e = sum_{g} w_g B_g^T C_bar_e B_g det J,     B = d(e_xx, e_yy, g_xy)/d(d_e).

Numbering: node n = j (nx + 1) + i at (i hx, j hy); DOFs 2n (u) and 2n + 1 (v);
element e = j nx + i with nodes (i, j), (i+1, j), (i+1, j+1), (i, j+1).

Boundary conditions (reading of "uniform end shortening with the other end
clamped"): u = v = 0 on x = 0; u = -shortening on x = lx, v free there; top and
bottom traction free. The 'roller' variant (u prescribed at both ends, v pinned at
the origin only) admits a uniform stress state and serves the closed-form check.
Dirichlet values are lifted to the right-hand side: K_FF d_F = -K_FD d_D.

Quantities of interest:
  reaction  Q_R = -sum over u-DOFs on x = lx of (K d)_i, the compressive end
            force per unit depth (positive in compression);
  stress    Q_S = max over elements with centroid x in [omega_x0, omega_x1] of
            max(0, -s_11^fibre), the fibre-direction compressive stress at the
            centroid (central region, by analogy with Omega' of Sec. 3.1).
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import material

_XI = np.array([-1.0, 1.0, 1.0, -1.0])
_ETA = np.array([-1.0, -1.0, 1.0, 1.0])


def shape_gradients(xi, eta, hx, hy):
    """dN_a/dx, dN_a/dy of the 4 bilinear shape functions at (xi, eta)."""
    dndxi = _XI * (1.0 + _ETA * eta) / 4.0
    dndeta = _ETA * (1.0 + _XI * xi) / 4.0
    return dndxi * (2.0 / hx), dndeta * (2.0 / hy)


def b_matrix(xi, eta, hx, hy):
    dx, dy = shape_gradients(xi, eta, hx, hy)
    B = np.zeros((3, 8))
    B[0, 0::2] = dx
    B[1, 1::2] = dy
    B[2, 0::2] = dy
    B[2, 1::2] = dx
    return B


def element_matrices(Cbar, hx, hy, order=2):
    """K_e[e, 8, 8] for per-element stiffness Cbar[e, 3, 3] by order x order Gauss."""
    g, w = np.polynomial.legendre.leggauss(order)
    det = hx * hy / 4.0
    Ke = np.zeros((Cbar.shape[0], 8, 8))
    for a, xi in enumerate(g):
        for b, eta in enumerate(g):
            B = b_matrix(xi, eta, hx, hy)
            Ke += w[a] * w[b] * det * np.einsum("ik,eij,jl->ekl", B, Cbar, B)
    return Ke


def element_dofs(nx, ny):
    i = np.tile(np.arange(nx), ny)
    j = np.repeat(np.arange(ny), nx)
    n0 = j * (nx + 1) + i
    nodes = np.stack([n0, n0 + 1, n0 + nx + 2, n0 + nx + 1], axis=1)
    dofs = np.empty((nx * ny, 8), dtype=np.int64)
    dofs[:, 0::2] = 2 * nodes
    dofs[:, 1::2] = 2 * nodes + 1
    return dofs


def assemble(nx, ny, lx, ly, Cbar):
    hx, hy = lx / nx, ly / ny
    Ke = element_matrices(Cbar, hx, hy)
    dofs = element_dofs(nx, ny)
    rows = np.repeat(dofs, 8, axis=1).reshape(-1)
    cols = np.tile(dofs, (1, 8)).reshape(-1)
    n = 2 * (nx + 1) * (ny + 1)
    return sp.csr_matrix((Ke.reshape(-1), (rows, cols)), shape=(n, n))


def dirichlet(nx, ny, shortening, bc="clamped"):
    """Prescribed DOFs and values."""
    left = np.arange(ny + 1) * (nx + 1)
    right = left + nx
    if bc == "clamped":
        dofs = np.concatenate([2 * left, 2 * left + 1, 2 * right])
        vals = np.concatenate([np.zeros(2 * (ny + 1)), np.full(ny + 1, -shortening)])
    elif bc == "roller":
        dofs = np.concatenate([2 * left, [1], 2 * right])
        vals = np.concatenate([np.zeros(ny + 1), [0.0], np.full(ny + 1, -shortening)])
    else:
        raise ValueError(bc)
    order = np.argsort(dofs)
    return dofs[order], vals[order]


def solve(K, ddofs, dvals):
    """d with d_D = dvals and K_FF d_F = -K_FD d_D (sparse LU, double precision)."""
    n = K.shape[0]
    free = np.setdiff1d(np.arange(n), ddofs)
    d = np.zeros(n)
    d[ddofs] = dvals
    rhs = -(K[free][:, ddofs] @ dvals)
    lu = spla.splu(K[free][:, free].tocsc())
    d[free] = lu.solve(rhs)
    return d


def reaction(K, d, nx, ny):
    right = np.arange(ny + 1) * (nx + 1) + nx
    return -float(np.sum((K @ d)[2 * right]))


def centroid_stress(d, Cbar, nx, ny, lx, ly):
    """Global stress (s_xx, s_yy, s_xy) at each element centroid."""
    B0 = b_matrix(0.0, 0.0, lx / nx, ly / ny)
    eps = d[element_dofs(nx, ny)] @ B0.T          # [e, 3]
    return np.einsum("eij,ej->ei", Cbar, eps)


def max_fibre_compression(d, Cbar, theta, nx, ny, lx, ly, x0, x1):
    sig = centroid_stress(d, Cbar, nx, ny, lx, ly)
    cx = np.tile((np.arange(nx) + 0.5) * (lx / nx), ny)
    inside = (cx >= x0) & (cx <= x1)
    c, s = np.cos(theta), np.sin(theta)
    s11 = c * c * sig[:, 0] + s * s * sig[:, 1] + 2.0 * c * s * sig[:, 2]
    return float(np.max(np.maximum(0.0, -s11[inside]))) if np.any(inside) else 0.0


def rotated_stiffness(C, theta):
    return np.stack([material.rotate(C, t) for t in np.asarray(theta).reshape(-1)])


def solve_sample(cfg, nx, ny, theta, bc="clamped"):
    """(Q_R, Q_S, d) for one realisation theta[e] on the nx x ny mesh."""
    C = material.material_from_cfg(cfg)
    Cbar = rotated_stiffness(C, theta)
    K = assemble(nx, ny, cfg["lx"], cfg["ly"], Cbar)
    ddofs, dvals = dirichlet(nx, ny, cfg["shortening"], bc)
    d = solve(K, ddofs, dvals)
    qr = reaction(K, d, nx, ny)
    qs = max_fibre_compression(d, Cbar, theta, nx, ny, cfg["lx"], cfg["ly"],
                               cfg["omega_x0"], cfg["omega_x1"])
    return qr, qs, d
