"""Trilinear Hex8 elements for the 3D fibre-waviness block (test infrastructure).

This is the oracle for the 3D generalisation of the strip problem: only tests/,
the smoke check and the benchmark's CPU baseline use it; the CUDA library never
does. Plain double precision, written from the mathematics, sharing no code with
the library.

The classical anisotropic elasticity weak form (Eq. VarCosserat without the
Cosserat rotation) is discretised with 8-node trilinear hexahedra on the structured
nx x ny x nz grid of cube elements of [0, lx] x [0, ly] x [0, lz]. Each element
column (i, k) carries one angle theta(x_i, z_k) of the out-of-plane waviness field;
the orthotropic ply stiffness (fibre axis 1) is rotated about the y axis by that
angle (Sec. 3.1's C* = T^-1 C T, here as the rotation of the fourth-order tensor,
C'_ijkl = R_ia R_jb R_kc R_ld C_abcd with R the rotation about y). Element matrices
use the 2x2x2 Gauss rule (exact for a cube with constant stiffness).

Voigt order (11, 22, 33, 23, 13, 12) with engineering shear strains.
Numbering: node n = (k (ny + 1) + j) (nx + 1) + i at (i h, j h, k h); DOFs 3n, 3n+1,
3n+2 (u, v, w); element (i, j, k) with corners (i+a, j+b, k+c) in the order
(0,0,0) (1,0,0) (1,1,0) (0,1,0) (0,0,1) (1,0,1) (1,1,1) (0,1,1).

Boundary conditions, as for the strip: u = v = w = 0 on x = 0; u = -shortening on
x = lx, v and w free there; all other faces traction free. The 'roller' variant
(u prescribed on both x faces, v = 0 on the y = 0 face, w = 0 at the origin node)
admits the uniform uniaxial stress state and serves the closed-form check.

Quantities of interest, as for the strip: the compressive end force
-sum over u-DOFs on x = lx of (K d)_i [N], and the maximum over elements with
centroid x in [omega_x0, omega_x1] of max(0, -sigma_fibre) at the centroid, with
sigma_fibre = a1 . sigma a1 and a1 the rotated fibre direction.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

# Voigt index pairs
_VOIGT = [(0, 0), (1, 1), (2, 2), (1, 2), (0, 2), (0, 1)]
_CORNERS = np.array([(0, 0, 0), (1, 0, 0), (1, 1, 0), (0, 1, 0),
                     (0, 0, 1), (1, 0, 1), (1, 1, 1), (0, 1, 1)])


def orthotropic_compliance(cfg):
    """6x6 compliance of the ply in its material axes (engineering shear)."""
    E1, E2, E3 = cfg["E11"], cfg["E22"], cfg["E33"]
    n12, n13, n23 = cfg["nu12"], cfg["nu13"], cfg["nu23"]
    S = np.zeros((6, 6))
    S[0, 0], S[1, 1], S[2, 2] = 1 / E1, 1 / E2, 1 / E3
    S[0, 1] = S[1, 0] = -n12 / E1
    S[0, 2] = S[2, 0] = -n13 / E1
    S[1, 2] = S[2, 1] = -n23 / E2
    S[3, 3], S[4, 4], S[5, 5] = 1 / cfg["G23"], 1 / cfg["G13"], 1 / cfg["G12"]
    return S


def material_stiffness(cfg):
    return np.linalg.inv(orthotropic_compliance(cfg))


def rotation_y(theta):
    """Rotation by theta about the y axis (right-handed)."""
    c, s = np.cos(theta), np.sin(theta)
    return np.array([[c, 0.0, s], [0.0, 1.0, 0.0], [-s, 0.0, c]])


def voigt_to_tensor(C6):
    C = np.zeros((3, 3, 3, 3))
    for I, (i, j) in enumerate(_VOIGT):
        for J, (k, l) in enumerate(_VOIGT):
            for (a, b) in {(i, j), (j, i)}:
                for (c, d) in {(k, l), (l, k)}:
                    C[a, b, c, d] = C6[I, J]
    return C


def tensor_to_voigt(C):
    C6 = np.zeros((6, 6))
    for I, (i, j) in enumerate(_VOIGT):
        for J, (k, l) in enumerate(_VOIGT):
            C6[I, J] = C[i, j, k, l]
    return C6


def rotate(C6, theta):
    """Stiffness in the global axes of a ply whose material frame is rotated by theta about y."""
    R = rotation_y(theta)
    C = voigt_to_tensor(C6)
    return tensor_to_voigt(np.einsum("ia,jb,kc,ld,abcd->ijkl", R, R, R, R, C))


def fibre_direction(theta):
    return rotation_y(theta)[:, 0]


def shape_derivatives(xi, eta, zeta, h):
    """dN_a/d(x, y, z) [8, 3] of the cube element of side h at the reference point."""
    a = _CORNERS * 2 - 1   # corner signs
    d = np.empty((8, 3))
    d[:, 0] = a[:, 0] * (1 + a[:, 1] * eta) * (1 + a[:, 2] * zeta) / 8
    d[:, 1] = a[:, 1] * (1 + a[:, 0] * xi) * (1 + a[:, 2] * zeta) / 8
    d[:, 2] = a[:, 2] * (1 + a[:, 0] * xi) * (1 + a[:, 1] * eta) / 8
    return d * (2.0 / h)


def b_matrix(xi, eta, zeta, h):
    """6 x 24 strain-displacement matrix (Voigt, engineering shear)."""
    d = shape_derivatives(xi, eta, zeta, h)
    B = np.zeros((6, 24))
    for a in range(8):
        dx, dy, dz = d[a]
        B[0, 3 * a] = dx
        B[1, 3 * a + 1] = dy
        B[2, 3 * a + 2] = dz
        B[3, 3 * a + 1], B[3, 3 * a + 2] = dz, dy
        B[4, 3 * a], B[4, 3 * a + 2] = dz, dx
        B[5, 3 * a], B[5, 3 * a + 1] = dy, dx
    return B


def element_matrix(C6, h, order=2):
    x, w = np.polynomial.legendre.leggauss(order)
    K = np.zeros((24, 24))
    det = (h / 2) ** 3
    for i in range(order):
        for j in range(order):
            for k in range(order):
                B = b_matrix(x[i], x[j], x[k], h)
                K += w[i] * w[j] * w[k] * det * B.T @ C6 @ B
    return K


def node_index(i, j, k, nx, ny):
    return (k * (ny + 1) + j) * (nx + 1) + i


def element_dofs(nx, ny, nz):
    """DOF indices [n_el, 24] of every element, element e = (k ny + j) nx + i."""
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    i, j, k = i.ravel(), j.ravel(), k.ravel()
    dofs = np.empty((i.size, 24), dtype=np.int64)
    for a, (ca, cb, cc) in enumerate(_CORNERS):
        n = node_index(i + ca, j + cb, k + cc, nx, ny)
        for c in range(3):
            dofs[:, 3 * a + c] = 3 * n + c
    return dofs


def assemble(nx, ny, nz, h, C_col):
    """Sparse K for per-column stiffness C_col[nx * nz, 6, 6] (column (i, k) -> k nx + i)."""
    dofs = element_dofs(nx, ny, nz)
    ke = {}
    n_el = nx * ny * nz
    vals = np.empty((n_el, 24, 24))
    e = 0
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                col = k * nx + i
                if col not in ke:
                    ke[col] = element_matrix(C_col[col], h)
                vals[e] = ke[col]
                e += 1
    rows = np.repeat(dofs, 24, axis=1).ravel()
    cols = np.tile(dofs, (1, 24)).ravel()
    n = 3 * (nx + 1) * (ny + 1) * (nz + 1)
    return sp.coo_matrix((vals.ravel(), (rows, cols)), shape=(n, n)).tocsr()


def dirichlet(nx, ny, nz, shortening, bc="clamped"):
    """Prescribed DOFs and values."""
    dd, dv = [], []
    for k in range(nz + 1):
        for j in range(ny + 1):
            n0 = node_index(0, j, k, nx, ny)
            n1 = node_index(nx, j, k, nx, ny)
            if bc == "clamped":
                dd += [3 * n0, 3 * n0 + 1, 3 * n0 + 2]
                dv += [0.0, 0.0, 0.0]
            else:
                dd.append(3 * n0)
                dv.append(0.0)
            dd.append(3 * n1)
            dv.append(-shortening)
    if bc == "roller":
        for k in range(nz + 1):
            for i in range(nx + 1):
                dd.append(3 * node_index(i, 0, k, nx, ny) + 1)
                dv.append(0.0)
        dd.append(3 * node_index(0, 0, 0, nx, ny) + 2)
        dv.append(0.0)
    return np.array(dd), np.array(dv)


def solve(K, ddofs, dvals):
    n = K.shape[0]
    free = np.setdiff1d(np.arange(n), ddofs)
    d = np.zeros(n)
    d[ddofs] = dvals
    rhs = -(K[free][:, ddofs] @ dvals)
    d[free] = spla.spsolve(K[free][:, free].tocsc(), rhs)
    return d


def apply(nx, ny, nz, h, C_col, x):
    """K x without assembling K: the sum over elements of the element matrix applied
    to the element's DOFs, scattered back (the definition of assembly, element by
    element column; column (i, k) -> k nx + i, all elements of a column alike)."""
    dofs = element_dofs(nx, ny, nz).reshape(nz, ny, nx, 24)
    contrib = np.empty((nz, ny, nx, 24))
    for k in range(nz):
        for i in range(nx):
            Ke = element_matrix(C_col[k * nx + i], h)
            contrib[k, :, i, :] = x[dofs[k, :, i, :]] @ Ke.T   # the column's ny elements
    return np.bincount(dofs.ravel(), weights=contrib.ravel(), minlength=3 * (nx + 1) * (ny + 1) * (nz + 1))


def solve_cg(K, ddofs, dvals, rtol=1e-12, maxiter=50000):
    """The same discrete solution as solve(), by conjugate gradients with the diagonal
    as preconditioner, to a relative residual of rtol on the free DOFs (for meshes on
    which the direct factorisation's fill-in is too large). Raises if CG stops short."""
    n = K.shape[0]
    free = np.setdiff1d(np.arange(n), ddofs)
    d = np.zeros(n)
    d[ddofs] = dvals
    Kff = K[free][:, free].tocsr()
    rhs = -(K[free][:, ddofs] @ dvals)
    dg = Kff.diagonal()
    M = spla.LinearOperator(Kff.shape, matvec=lambda v: v / dg)
    x, info = spla.cg(Kff, rhs, rtol=rtol, atol=0.0, maxiter=maxiter, M=M)
    if info != 0:
        raise RuntimeError(f"CG did not reach rtol {rtol} (info {info})")
    if np.linalg.norm(rhs - Kff @ x) > 10 * rtol * np.linalg.norm(rhs):
        raise RuntimeError("CG residual above its tolerance")
    d[free] = x
    return d


def reaction(K, d, nx, ny, nz):
    Kd = K @ d
    idx = [3 * node_index(nx, j, k, nx, ny) for k in range(nz + 1) for j in range(ny + 1)]
    return -float(np.sum(Kd[idx]))


def max_fibre_compression(cfg, d, C_col, theta_col, nx, ny, nz, h):
    """max over elements with centroid x in [omega_x0, omega_x1] of max(0, -a1 . sigma a1)."""
    dofs = element_dofs(nx, ny, nz)
    B0 = b_matrix(0.0, 0.0, 0.0, h)
    best = 0.0
    e = 0
    for k in range(nz):
        for j in range(ny):
            for i in range(nx):
                xc = (i + 0.5) * h
                if cfg["omega_x0"] <= xc <= cfg["omega_x1"]:
                    col = k * nx + i
                    s6 = C_col[col] @ (B0 @ d[dofs[e]])
                    sig = np.array([[s6[0], s6[5], s6[4]], [s6[5], s6[1], s6[3]], [s6[4], s6[3], s6[2]]])
                    a1 = fibre_direction(theta_col[col])
                    best = max(best, -float(a1 @ sig @ a1))
                e += 1
    return best


def solve_sample(cfg, nx, ny, nz, theta_col, bc="clamped", solver="direct"):
    """(reaction, stress, d) of one sample on the nx x ny x nz mesh; solver "direct"
    (sparse LU) or "cg" (solve_cg to a relative residual of 1e-12)."""
    h = cfg["lx"] / nx
    C = material_stiffness(cfg)
    C_col = np.array([rotate(C, t) for t in theta_col])
    K = assemble(nx, ny, nz, h, C_col)
    dd, dv = dirichlet(nx, ny, nz, cfg["shortening"], bc)
    d = solve(K, dd, dv) if solver == "direct" else solve_cg(K, dd, dv)
    return reaction(K, d, nx, ny, nz), max_fibre_compression(cfg, d, C_col, theta_col, nx, ny, nz, h), d


def column_centroids(cfg, nx, nz):
    """Centroids (x, z) of the element columns, column (i, k) -> k nx + i."""
    h = cfg["lx"] / nx
    cx = np.tile((np.arange(nx) + 0.5) * h, nz)
    cz = np.repeat((np.arange(nz) + 0.5) * h, nx)
    return cx, cz
