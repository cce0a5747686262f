"""Reissner-Mindlin Q4 panel buckling with uncertain ply angles (test infrastructure).

This is the oracle for the buckling test problem (Sec. 4): only tests/, the smoke
check and the benchmark's CPU baseline use it; the CUDA library never does. Plain
double precision, written from the mathematics, sharing no code with the library.

Laminate (Sec. 4.1): K plies of equal thickness t_ply, ply k at angle psi_k + phi_k
(pristine angle plus a random perturbation), stacked from z = -t/2 upwards. Each ply
has the plane-stress reduced stiffness Q of an orthotropic lamina (fibre axis 1),
rotated into panel axes (Q_bar). Classical laminate theory (Eq. CLTABD) gives
  A = sum Q_bar_k (z_k - z_{k-1}),  B = 1/2 sum Q_bar_k (z_k^2 - z_{k-1}^2),
  D = 1/3 sum Q_bar_k (z_k^3 - z_{k-1}^3),
and the bending stiffness is knocked down to D* = D - B^T A^-1 B (Sec. 4.1).

Plate (Eq. momentequil, Eq. MomentWeakForm): unknowns w (deflection) and
theta = (theta_x, theta_y) (rotations), curvature kappa = sym grad theta in Voigt form
(theta_x,x, theta_y,y, theta_x,y + theta_y,x), transverse shear strain
gamma = grad w - theta with shear stiffness k G t (k = 5/6). The prestress is a
uniform compressive line load N_x = 1 N/mm along x, so the geometric form is
int w_x w^_x and the eigenvalue lambda is the critical N_x in N/mm (the total load is
lambda * ly). Find the smallest lambda with
  int kappa : D* kappa^ + k G t int gamma . gamma^ = lambda int w_x w^_x.

Discretisation (Eq. matrixeig): bilinear Q4 for w, theta_x, theta_y on a uniform
nx x ny grid of [0, lx] x [0, ly]; bending by 2x2 Gauss, shear by 1-point (selective
reduced integration, free of shear locking), the geometric form by 1-point as well, so
that it has the same null space as the under-integrated shear (the w-hourglass mode
carries neither shear nor geometric energy; a 2x2 geometric form would give it a
spurious near-zero buckling load).

Boundary: simply supported, w = 0 on the whole boundary. Eq. momentequil states the
moment traction free ('soft' support, rotations free); the 'hard' variant also holds the
tangential rotation (theta_y = 0 on x = 0, lx; theta_x = 0 on y = 0, ly). With hard
support a single Fourier mode solves the continuous problem of a specially orthotropic
plate exactly (mindlin_navier below), and it is the hard support that reproduces the
pristine load printed in Sec. 4.2 (278.59 kN; the soft support gives about 6 % less), so
the workloads take it.

Units: N, mm, MPa. Numbering: node n = j (nx + 1) + i at (i hx, j hy), DOFs
3n + (0: w, 1: theta_x, 2: theta_y); element (i, j) with corners (i, j), (i+1, j),
(i+1, j+1), (i, j+1).
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import rng

_CORNERS = np.array([(-1.0, -1.0), (1.0, -1.0), (1.0, 1.0), (-1.0, 1.0)])
_G2 = 1.0 / np.sqrt(3.0)


# ---------------------------------------------------------------- laminate (Eq. CLTABD)

def lamina_q(E11, E22, G12, nu12):
    """Plane-stress reduced stiffness of an orthotropic lamina, Voigt (11, 22, 12)
    with engineering shear: the inverse of the in-plane compliance."""
    S = np.array([[1.0 / E11, -nu12 / E11, 0.0],
                  [-nu12 / E11, 1.0 / E22, 0.0],
                  [0.0, 0.0, 1.0 / G12]])
    return np.linalg.inv(S)


def rotate_q(Q, angle):
    """Q_bar = T^-1 Q T^-T with T the stress transformation for a ply whose fibre
    makes `angle` (radians, counter-clockwise) with the x axis (the in-plane form of
    Sec. 3.1's C* = T^-1 C T); strains engineering."""
    c, s = np.cos(angle), np.sin(angle)
    # stress transformation sigma_123 = T sigma_xyz
    T = np.array([[c * c, s * s, 2 * c * s],
                  [s * s, c * c, -2 * c * s],
                  [-c * s, c * s, c * c - s * s]])
    Ti = np.linalg.inv(T)
    # engineering strains: eps_123 = T^-T eps_xyz, so sigma_xyz = T^-1 Q T^-T eps_xyz
    return Ti @ Q @ Ti.T


def laminate_abd(Q, angles, t_ply):
    """A, B, D of plies at `angles` (radians, bottom ply first), each t_ply thick,
    stacked symmetrically about z = 0 (Eq. CLTABD)."""
    K = len(angles)
    z = -0.5 * K * t_ply + t_ply * np.arange(K + 1)
    A = np.zeros((3, 3))
    B = np.zeros((3, 3))
    D = np.zeros((3, 3))
    for k, a in enumerate(angles):
        Qb = rotate_q(Q, a)
        A += Qb * (z[k + 1] - z[k])
        B += 0.5 * Qb * (z[k + 1] ** 2 - z[k] ** 2)
        D += Qb * (z[k + 1] ** 3 - z[k] ** 3) / 3.0
    return A, B, D


def knocked_down_d(A, B, D):
    """D* = D - B^T A^-1 B (Sec. 4.1)."""
    return D - B.T @ np.linalg.solve(A, B)


def panel_stiffness(cfg, phi):
    """(D*, k G t) of a sample whose ply perturbations are phi (radians, one per ply)."""
    Q = lamina_q(cfg["E11"], cfg["E22"], cfg["G12"], cfg["nu12"])
    angles = np.radians(np.asarray(cfg["plies_deg"], dtype=float)) + np.asarray(phi, dtype=float)
    A, B, D = laminate_abd(Q, angles, cfg["t_ply"])
    t = cfg["t_ply"] * len(cfg["plies_deg"])
    return knocked_down_d(A, B, D), cfg["k_shear"] * cfg["G13"] * t


# ---------------------------------------------------------------- element (Eq. MomentWeakForm)

def _shape(xi, eta, hx, hy):
    """Q4 shape functions and their x, y derivatives at (xi, eta) in [-1, 1]^2."""
    N = 0.25 * (1 + _CORNERS[:, 0] * xi) * (1 + _CORNERS[:, 1] * eta)
    dx = 0.25 * _CORNERS[:, 0] * (1 + _CORNERS[:, 1] * eta) * (2.0 / hx)
    dy = 0.25 * _CORNERS[:, 1] * (1 + _CORNERS[:, 0] * xi) * (2.0 / hy)
    return N, dx, dy


def _b_bend(dx, dy):
    """kappa = (theta_x,x, theta_y,y, theta_x,y + theta_y,x) from the 12 element DOFs."""
    Bb = np.zeros((3, 12))
    Bb[0, 1::3] = dx
    Bb[1, 2::3] = dy
    Bb[2, 1::3] = dy
    Bb[2, 2::3] = dx
    return Bb


def _b_shear(N, dx, dy):
    """gamma = (w,x - theta_x, w,y - theta_y) from the 12 element DOFs."""
    Bs = np.zeros((2, 12))
    Bs[0, 0::3] = dx
    Bs[0, 1::3] = -N
    Bs[1, 0::3] = dy
    Bs[1, 2::3] = -N
    return Bs


def element_matrices(Dstar, kgt, hx, hy, geo_order=1):
    """(K_e, G_e), 12 x 12: bending by 2x2 Gauss with D*, shear by the 1-point rule
    with k G t, geometric int w_x w^_x by `geo_order` points per axis (1 or 2)."""
    det = 0.25 * hx * hy
    K = np.zeros((12, 12))
    for gx in (-_G2, _G2):
        for gy in (-_G2, _G2):
            _, dx, dy = _shape(gx, gy, hx, hy)
            Bb = _b_bend(dx, dy)
            K += Bb.T @ Dstar @ Bb * det
    N, dx, dy = _shape(0.0, 0.0, hx, hy)
    Bs = _b_shear(N, dx, dy)
    K += kgt * (Bs.T @ Bs) * (4.0 * det)
    G = np.zeros((12, 12))
    pts = [(0.0, 0.0, 4.0)] if geo_order == 1 else [(a, b, 1.0) for a in (-_G2, _G2) for b in (-_G2, _G2)]
    for gx, gy, wt in pts:
        _, dx, _ = _shape(gx, gy, hx, hy)
        g = np.zeros(12)
        g[0::3] = dx
        G += np.outer(g, g) * (wt * det)
    return K, G


# ---------------------------------------------------------------- assembly and boundary

def element_dofs(nx, ny):
    """[nx * ny, 12] global DOFs of each element (element e = j nx + i)."""
    out = np.zeros((nx * ny, 12), dtype=np.int64)
    for j in range(ny):
        for i in range(nx):
            nodes = [j * (nx + 1) + i, j * (nx + 1) + i + 1, (j + 1) * (nx + 1) + i + 1, (j + 1) * (nx + 1) + i]
            out[j * nx + i] = np.array([[3 * n, 3 * n + 1, 3 * n + 2] for n in nodes]).ravel()
    return out


def assemble(nx, ny, Ke, Ge):
    """Global sparse K and G of a uniform mesh whose elements all have K_e, G_e."""
    ed = element_dofs(nx, ny)
    n = 3 * (nx + 1) * (ny + 1)
    rows = np.repeat(ed, 12, axis=1).ravel()
    cols = np.tile(ed, (1, 12)).ravel()
    K = sp.csr_matrix((np.tile(Ke.ravel(), nx * ny), (rows, cols)), shape=(n, n))
    G = sp.csr_matrix((np.tile(Ge.ravel(), nx * ny), (rows, cols)), shape=(n, n))
    return K, G


def constrained_dofs(nx, ny, bc="soft"):
    """DOFs fixed to zero: w on the boundary; with bc='hard' also the tangential
    rotation (theta_y on x = 0, lx; theta_x on y = 0, ly)."""
    fixed = set()
    for j in range(ny + 1):
        for i in range(nx + 1):
            n = j * (nx + 1) + i
            on_x = i == 0 or i == nx
            on_y = j == 0 or j == ny
            if on_x or on_y:
                fixed.add(3 * n)
            if bc == "hard":
                if on_x:
                    fixed.add(3 * n + 2)
                if on_y:
                    fixed.add(3 * n + 1)
    return np.array(sorted(fixed), dtype=np.int64)


def free_dofs(nx, ny, bc="soft"):
    n = 3 * (nx + 1) * (ny + 1)
    mask = np.ones(n, dtype=bool)
    mask[constrained_dofs(nx, ny, bc)] = False
    return np.flatnonzero(mask)


# ---------------------------------------------------------------- eigenproblem (Eq. matrixeig)

def critical_load(K, G, free, dense=None):
    """(lambda, mode): the smallest lambda of K d = lambda G d on the free DOFs, as
    1 / mu for the largest mu of G d = mu K d (K is positive definite once w is held
    on the boundary; G is only semi-definite). mode is K-normalised (d^T K d = 1) with
    its largest-magnitude w entry positive, on all DOFs (zeros where constrained)."""
    Kf = K[free][:, free]
    Gf = G[free][:, free]
    nf = len(free)
    if dense is None:
        dense = nf <= 1500
    if dense:
        mu, V = sla.eigh(Gf.toarray(), Kf.toarray())
        m, v = mu[-1], V[:, -1]
    else:
        lu = spla.splu(Kf.tocsc())
        op = spla.LinearOperator((nf, nf), matvec=lambda x: lu.solve(Gf @ x), dtype=float)
        # K^-1 G is self-adjoint in the K inner product; its dominant eigenpair by
        # implicitly restarted Arnoldi on the operator itself
        mu, V = spla.eigs(op, k=1, which="LR", tol=1e-13, maxiter=10000)
        m, v = float(mu[0].real), V[:, 0].real
    v = v / np.sqrt(v @ (Kf @ v))
    d = np.zeros(K.shape[0])
    d[free] = v
    w = d[0::3]
    if w[np.argmax(np.abs(w))] < 0:
        d = -d
    return 1.0 / m, d


def solve_sample(cfg, nx, ny, phi, bc="soft", geo_order=1, dense=None):
    """Critical line load lambda (N/mm) of one sample on an nx x ny mesh."""
    Dstar, kgt = panel_stiffness(cfg, phi)
    hx, hy = cfg["lx"] / nx, cfg["ly"] / ny
    Ke, Ge = element_matrices(Dstar, kgt, hx, hy, geo_order)
    K, G = assemble(nx, ny, Ke, Ge)
    lam, _ = critical_load(K, G, free_dofs(nx, ny, bc), dense)
    return lam


# ---------------------------------------------------------------- closed forms

def mindlin_navier(D, kgt, lx, ly, modes=8):
    """Critical N_x of a simply supported ('hard') specially orthotropic Mindlin plate
    (D16 = D26 = 0): w = W sin(a x) sin(b y), theta_x = X cos(a x) sin(b y),
    theta_y = Y sin(a x) cos(b y), a = m pi / lx, b = n pi / ly, solves the continuous
    problem exactly; the energy of the mode is a quadratic form in (W, X, Y), and the
    rotations are eliminated (Schur complement). Minimum over m, n <= modes."""
    best = np.inf
    for m in range(1, modes + 1):
        for n in range(1, modes + 1):
            a, b = m * np.pi / lx, n * np.pi / ly
            S = np.array([
                [kgt * (a * a + b * b), -kgt * a, -kgt * b],
                [-kgt * a, D[0, 0] * a * a + D[2, 2] * b * b + kgt, (D[0, 1] + D[2, 2]) * a * b],
                [-kgt * b, (D[0, 1] + D[2, 2]) * a * b, D[1, 1] * b * b + D[2, 2] * a * a + kgt],
            ])
            schur = S[0, 0] - S[0, 1:] @ np.linalg.solve(S[1:, 1:], S[1:, 0])
            best = min(best, schur / (a * a))
    return best


def kirchhoff_navier(D, lx, ly, modes=8):
    """Critical N_x of a simply supported specially orthotropic Kirchhoff plate:
    min over (m, n) of (D11 a^4 + 2 (D12 + 2 D66) a^2 b^2 + D22 b^4) / a^2."""
    best = np.inf
    for m in range(1, modes + 1):
        for n in range(1, modes + 1):
            a, b = m * np.pi / lx, n * np.pi / ly
            best = min(best, (D[0, 0] * a ** 4 + 2 * (D[0, 1] + 2 * D[2, 2]) * a * a * b * b + D[1, 1] * b ** 4) / (a * a))
    return best


def ply_perturbations(cfg, xi):
    """phi (radians) from standard normals xi [n, plies]: phi = std * xi (Sec. 4.1)."""
    return np.radians(cfg["ply_std_deg"]) * np.asarray(xi, dtype=float)


# ---------------------------------------------------------------- MLMC level pairs (Sec. 2.2, Sec. 4.2)

def mesh_operators(cfg, mesh_level, phi):
    """Global K and G (no boundary conditions) of one sample on panel mesh `mesh_level`."""
    nx, ny = cfg["nx0"] << mesh_level, cfg["ny0"] << mesh_level
    Dstar, kgt = panel_stiffness(cfg, phi)
    Ke, Ge = element_matrices(Dstar, kgt, cfg["lx"] / nx, cfg["ly"] / ny)
    return assemble(nx, ny, Ke, Ge)


def quantities(cfg, lam):
    """(critical load P = lambda ly in kN, failure indicator P < p_star) (Sec. 4.2)."""
    P = lam * cfg["ly"] * 1e-3
    return np.array([P, 1.0 if P < cfg["p_star"] else 0.0])


def solve_mesh(cfg, mesh_level, phi):
    """Quantities of one sample (perturbations phi) on panel mesh `mesh_level`."""
    nx, ny = cfg["nx0"] << mesh_level, cfg["ny0"] << mesh_level
    return quantities(cfg, solve_sample(cfg, nx, ny, phi, bc=cfg.get("bc", "hard")))


def sample_perturbations(cfg, level, ids):
    """phi [n, plies] of samples `ids` of `level`: the first n_plies normals of each
    sample's counter stream, scaled by the ply angle deviation (Sec. 4.1)."""
    xi = rng.kl_coefficients(cfg["seed"], level, np.asarray(ids, dtype=np.uint64), len(cfg["plies_deg"]))
    return ply_perturbations(cfg, xi)


def level_pair(cfg, level, ids):
    """(q_fine [n, 2], q_coarse [n, 2]) of level-`level` samples `ids`: both meshes with
    the same perturbations (Eq. MLMC_defn); q_coarse is zero on level 0."""
    phi = sample_perturbations(cfg, level, ids)
    qf = np.array([solve_mesh(cfg, level, p) for p in phi])
    qc = np.array([solve_mesh(cfg, level - 1, p) for p in phi]) if level > 0 else np.zeros_like(qf)
    return qf, qc
