"""Two-dimensional Cosserat continuum for a composite with random fibre waviness: the
paper's first test problem as published (test infrastructure).

This is the oracle of the Cosserat engine: only tests/, the smoke check and the
benchmark's CPU baseline use it; the CUDA library never does. Plain double precision,
written from the mathematics, sharing no code with the library.

Model (Sec. 3.1, Eq. VarCosserat). Plane strain; each material point carries the
displacements u_1, u_2 (u, v) and an independent Cosserat rotation theta_3. Strains
and curvatures
    eps_ij = u_i,j + e_ij3 theta_3   ->  eps_11 = u_1,1, eps_22 = u_2,2,
                                          eps_12 = u_1,2 + theta_3, eps_21 = u_2,1 - theta_3,
    kappa_j = theta_3,j,
with the permutation symbol e_123 = 1, e_213 = -1 (a rigid rotation u = w (-y, x),
theta_3 = w strains nothing). Stresses sigma = C* eps on the vector
(11, 22, 12, 21) and couple stresses m = D* kappa on (1, 2), C* and D* the fibre-frame
C and D rotated by the local misalignment angle phi (Sec. 3.1, C* = T^-1 C T):
    sigma_g = R sigma_l R^T, eps_l = R^T eps_g R, kappa_l = R^T kappa_g, m_g = R m_l,
R = [[c, -s], [s, c]] turning the fibre direction e_1 onto (cos phi, sin phi).

Constitutive readings (the paper takes C and D from its micromechanics reference, Sec.
2.3 of [Dod15], which is not available): rule-of-mixtures values from the printed
AS4/8552 constants (v_f, E_f, E_m, G_f, G_m, d):
    E_11 = v_f E_f + (1 - v_f) E_m,           E_22 = E_33 = 1 / (v_f / E_f + (1 - v_f) / E_m),
    G_par = 1 / (v_f / G_f + (1 - v_f) / G_m) (sigma_12 = G_par eps_12: sliding of fibres
                                                along each other, matrix dominated),
    G_perp = v_f G_f + (1 - v_f) G_m          (sigma_21 = G_perp eps_21: fibre shear,
                                                fibre dominated, the stiffer of the two),
    nu_12 = nu_13 = 0.3, nu_23 = 0.45, the normal block the plane-strain part of the
    inverse 3D orthotropic compliance,
    D_1 = v_f E_f d^2 / 16 (fibre bending: the fibres' E I per unit area),
    D_2 = (1 - v_f) E_m d^2 / 16.
Failure (Sec. 3.1): effective stress tau_e = sqrt(sigma_12^2 + (sigma_22 / R)^2) in the
fibre frame, tau_y = tau_c, R = 2 (reading).

Quantities of interest: (0) the compressive strength: with f* the maximum of
tau_e / tau_y over the 2x2 Gauss points of the elements inside the central square
Omega', sigma = -(1 / |Omega'|) int_Omega' sigma_x / f* (Eq. failureCriterion read as
the applied mean stress scaled by 1 / f*: the printed f* / |Omega'| is garbled, the
problem is linear); (1) the end reaction -sum (K d)_u over the nodes on x = L [N per mm
of depth].

Discretisation (Eq. matrixinplane): bilinear Q1 for u, v, theta_3 on a uniform n x n
grid of the square [0, L]^2, 2x2 Gauss for both terms; node n = j (n + 1) + i, DOFs
3 n + (0: u, 1: v, 2: theta); element (i, j) with corners (i, j), (i+1, j), (i+1, j+1),
(i, j+1). Boundary: u = 0 on x = 0, u = shortening on x = L (negative), v = 0 on
y = 0 and y = L; theta free.
"""
import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

_G2 = 1.0 / np.sqrt(3.0)
_CORNERS = np.array([(-1.0, -1.0), (1.0, -1.0), (1.0, 1.0), (-1.0, 1.0)])


# ---------------------------------------------------------------- constitutive model

def micromechanics(cfg):
    """Fibre-frame constants (E11, E22, G_par, G_perp, D1, D2) from the constituents."""
    vf, Ef, Em, Gf, Gm, d = cfg["vf"], cfg["Ef"], cfg["Em"], cfg["Gf"], cfg["Gm"], cfg["d"]
    E11 = vf * Ef + (1 - vf) * Em
    E22 = 1.0 / (vf / Ef + (1 - vf) / Em)
    Gpar = 1.0 / (vf / Gf + (1 - vf) / Gm)
    Gperp = vf * Gf + (1 - vf) * Gm
    D1 = vf * Ef * d * d / 16.0
    D2 = (1 - vf) * Em * d * d / 16.0
    return E11, E22, Gpar, Gperp, D1, D2


def fibre_stiffness(cfg):
    """(C [4x4] on (11, 22, 12, 21), D [2x2]) in the fibre frame."""
    E11, E22, Gpar, Gperp, D1, D2 = micromechanics(cfg)
    n12, n23 = cfg["nu12"], cfg["nu23"]
    S = np.array([[1 / E11, -n12 / E11, -n12 / E11],
                  [-n12 / E11, 1 / E22, -n23 / E22],
                  [-n12 / E11, -n23 / E22, 1 / E22]])
    Q = np.linalg.inv(S)[:2, :2]   # plane strain: the (1, 2) block of the inverse compliance
    C = np.zeros((4, 4))
    C[:2, :2] = Q
    C[2, 2] = Gpar
    C[3, 3] = Gperp
    D = np.diag([D1, D2])
    return C, D


def _rot(phi):
    c, s = np.cos(phi), np.sin(phi)
    return np.array([[c, -s], [s, c]])


def _vec(T):
    return np.array([T[0, 0], T[1, 1], T[0, 1], T[1, 0]])


def _mat(v):
    return np.array([[v[0], v[2]], [v[3], v[1]]])


def rotated_stiffness(C, D, phi):
    """(C*, D*) in global axes at misalignment phi, built column by column from the
    tensor rotations: C* e = vec(R C(vec(R^T E R)) R^T)."""
    R = _rot(phi)
    Cg = np.zeros((4, 4))
    for k in range(4):
        e = np.zeros(4)
        e[k] = 1.0
        el = _vec(R.T @ _mat(e) @ R)
        Cg[:, k] = _vec(R @ _mat(C @ el) @ R.T)
    Dg = R @ D @ R.T
    return Cg, Dg


# ---------------------------------------------------------------- element (Eq. VarCosserat)

def _shape(xi, eta, h):
    N = 0.25 * (1 + _CORNERS[:, 0] * xi) * (1 + _CORNERS[:, 1] * eta)
    dx = 0.25 * _CORNERS[:, 0] * (1 + _CORNERS[:, 1] * eta) * (2.0 / h)
    dy = 0.25 * _CORNERS[:, 1] * (1 + _CORNERS[:, 0] * xi) * (2.0 / h)
    return N, dx, dy


def b_matrices(xi, eta, h):
    """(B_eps [4 x 12] on (eps_11, eps_22, eps_12, eps_21), B_kap [2 x 12]) at (xi, eta)."""
    N, dx, dy = _shape(xi, eta, h)
    Be = np.zeros((4, 12))
    Bk = np.zeros((2, 12))
    Be[0, 0::3] = dx            # u,x
    Be[1, 1::3] = dy            # v,y
    Be[2, 0::3] = dy            # u,y + theta
    Be[2, 2::3] = N
    Be[3, 1::3] = dx            # v,x - theta
    Be[3, 2::3] = -N
    Bk[0, 2::3] = dx
    Bk[1, 2::3] = dy
    return Be, Bk


def element_matrix(Cg, Dg, h):
    """12 x 12 element stiffness of a square element of side h, 2x2 Gauss."""
    K = np.zeros((12, 12))
    det = 0.25 * h * h
    for gx in (-_G2, _G2):
        for gy in (-_G2, _G2):
            Be, Bk = b_matrices(gx, gy, h)
            K += det * (Be.T @ Cg @ Be + Bk.T @ Dg @ Bk)
    return K


def element_dofs(n):
    out = np.zeros((n * n, 12), dtype=np.int64)
    for j in range(n):
        for i in range(n):
            nodes = [j * (n + 1) + i, j * (n + 1) + i + 1, (j + 1) * (n + 1) + i + 1, (j + 1) * (n + 1) + i]
            out[j * n + i] = np.array([[3 * a, 3 * a + 1, 3 * a + 2] for a in nodes]).ravel()
    return out


def assemble(cfg, n, phi):
    """Sparse K of the n x n mesh with one angle per element (phi[e], e = j n + i)."""
    C, D = fibre_stiffness(cfg)
    h = cfg["L"] / n
    ed = element_dofs(n)
    vals = np.empty((n * n, 12, 12))
    for e in range(n * n):
        Cg, Dg = rotated_stiffness(C, D, phi[e])
        vals[e] = element_matrix(Cg, Dg, h)
    m = 3 * (n + 1) ** 2
    rows = np.repeat(ed, 12, axis=1).ravel()
    cols = np.tile(ed, (1, 12)).ravel()
    return sp.coo_matrix((vals.ravel(), (rows, cols)), shape=(m, m)).tocsr()


def dirichlet(n, shortening):
    """Prescribed DOFs and values: u on x = 0 and x = L, v on y = 0 and y = L."""
    dd, dv = {}, {}
    for j in range(n + 1):
        dd[3 * (j * (n + 1))] = 0.0
        dd[3 * (j * (n + 1) + n)] = shortening
    for i in range(n + 1):
        dd[3 * i + 1] = 0.0
        dd[3 * (n * (n + 1) + i) + 1] = 0.0
    keys = np.array(sorted(dd))
    return keys, np.array([dd[k] for k in keys])


def solve(K, ddofs, dvals):
    m = K.shape[0]
    free = np.setdiff1d(np.arange(m), ddofs)
    d = np.zeros(m)
    d[ddofs] = dvals
    rhs = -(K[free][:, ddofs] @ dvals)
    d[free] = spla.spsolve(K[free][:, free].tocsc(), rhs)
    return d


# ---------------------------------------------------------------- quantities of interest

def centre_elements(cfg, n):
    """Elements lying inside the central square Omega' (side cfg['omega_side'])."""
    h = cfg["L"] / n
    lo, hi = 0.5 * (cfg["L"] - cfg["omega_side"]), 0.5 * (cfg["L"] + cfg["omega_side"])
    tol = 1e-9 * cfg["L"]
    inside = [k for k in range(n) if k * h >= lo - tol and (k + 1) * h <= hi + tol]
    return [j * n + i for j in inside for i in inside]


def strength(cfg, n, phi, d):
    """Compressive strength sigma = -(1/|Omega'|) int_Omega' sigma_x / f*, f* the largest
    tau_e / tau_y over the Gauss points of the elements inside Omega'."""
    C, D = fibre_stiffness(cfg)
    h = cfg["L"] / n
    ed = element_dofs(n)
    fmax, int_sx, area = 0.0, 0.0, 0.0
    for e in centre_elements(cfg, n):
        Cg, _ = rotated_stiffness(C, D, phi[e])
        R = _rot(phi[e])
        for gx in (-_G2, _G2):
            for gy in (-_G2, _G2):
                Be, _ = b_matrices(gx, gy, h)
                sg = Cg @ (Be @ d[ed[e]])
                sl = R.T @ _mat(sg) @ R            # fibre-frame stress tensor
                tau_e = np.hypot(sl[0, 1], sl[1, 1] / cfg["R_ratio"])
                fmax = max(fmax, tau_e / cfg["tau_y"])
                int_sx += 0.25 * h * h * sg[0]
                area += 0.25 * h * h
    return -(int_sx / area) / fmax


def reaction(K, d, n):
    Kd = K @ d
    return -float(np.sum(Kd[[3 * (j * (n + 1) + n) for j in range(n + 1)]]))


def solve_sample(cfg, n, phi):
    """(strength, reaction, d) of one sample (angles phi per element) on the n x n mesh."""
    K = assemble(cfg, n, phi)
    dd, dv = dirichlet(n, cfg["shortening"])
    d = solve(K, dd, dv)
    return strength(cfg, n, phi, d), reaction(K, d, n), d


# ---------------------------------------------------------------- KL of the exponential kernel

def exp_eig_1d(a, omega, n_modes):
    """The first n_modes eigenpairs of k(x, y) = exp(-|x - y| / omega) on [0, a], in closed
    form: with c = 1 / omega, A = a / 2 and x' = x - A, the i-th frequency w_i (i = 0, 1,
    ...) is the root in (i pi / (2 A), (i + 1) pi / (2 A)) of c - w tan(w A) (i even,
    phi = cos(w x') / sqrt(A + sin(2 w A) / (2 w))) or of w + c tan(w A) (i odd,
    phi = sin(w x') / sqrt(A - sin(2 w A) / (2 w))), and mu_i = 2 c / (w_i^2 + c^2).
    Returns (mu [n], w [n]); eigenfunctions from exp_phi_1d."""
    from scipy.optimize import brentq
    c, A = 1.0 / omega, 0.5 * a
    mu, w = np.empty(n_modes), np.empty(n_modes)
    for i in range(n_modes):
        lo, hi = i * np.pi / (2 * A), (i + 1) * np.pi / (2 * A)
        eps = 1e-12 * (hi - lo)
        f = (lambda x: c * np.cos(x * A) - x * np.sin(x * A)) if i % 2 == 0 else \
            (lambda x: x * np.cos(x * A) + c * np.sin(x * A))
        w[i] = brentq(f, lo + eps, hi - eps, xtol=1e-15, rtol=1e-15, maxiter=500)
        mu[i] = 2.0 * c / (w[i] ** 2 + c * c)
    return mu, w


def exp_phi_1d(a, w, i, x):
    """Eigenfunction i (frequency w) at points x, with the sign making phi(0) > 0."""
    A = 0.5 * a
    xp = np.asarray(x, dtype=np.float64) - A
    if i % 2 == 0:
        v = np.cos(w * xp) / np.sqrt(A + np.sin(2 * w * A) / (2 * w))
        sign = np.sign(np.cos(w * A))
    else:
        v = np.sin(w * xp) / np.sqrt(A - np.sin(2 * w * A) / (2 * w))
        sign = -np.sign(np.sin(w * A))
    return sign * v


def kl_basis(cfg, n, n_kl):
    """B[e, k] = s sqrt(mu_k) phi_k(centroid of e) for the first n_kl 2D modes of the
    separable exponential kernel (Eq. covarianceFunction) on [0, L]^2 at the centroids of
    the n x n mesh: products mu^x_i mu^y_j sorted descending, ties by (i + j, i)."""
    L, s = cfg["L"], cfg["kl_std"]
    mux, wx = exp_eig_1d(L, cfg["omega1"], n_kl + 1)
    muy, wy = exp_eig_1d(L, cfg["omega2"], n_kl + 1)
    cand = sorted((-(mux[i] * muy[j]), i + j, i, j) for i in range(n_kl + 1) for j in range(n_kl + 1))
    modes = [(i, j) for (_, _, i, j) in cand[:n_kl]]
    h = L / n
    cx = (np.arange(n) + 0.5) * h
    B = np.empty((n * n, n_kl))
    for k, (i, j) in enumerate(modes):
        fx = exp_phi_1d(L, wx[i], i, cx)
        fy = exp_phi_1d(L, wy[j], j, cx)
        B[:, k] = s * np.sqrt(mux[i] * muy[j]) * np.outer(fy, fx).ravel()   # e = j n + i
    return B, modes


# ---------------------------------------------------------------- level pairs (Sec. 2.2)

def dofs(cfg, mesh):
    """M of mesh `mesh`: 3 (n + 1)^2 with n = n0 2^mesh (Sec. 3.2: M_0 = 243 for n0 = 8)."""
    n = cfg["n0"] << mesh
    return 3 * (n + 1) ** 2


def n_kl(cfg, level):
    """N_KL of mesh `level`: 50 + 50 l (Sec. 3.2)."""
    return cfg["kl_terms0"] + cfg["kl_terms_step"] * level


def solve_on_mesh(cfg, mesh, xi):
    """(strength, reaction) of one sample on mesh `mesh` from the first n_kl(mesh) of its xi."""
    n = cfg["n0"] << mesh
    k = n_kl(cfg, mesh)
    B, _ = kl_basis(cfg, n, k)
    s, r, _ = solve_sample(cfg, n, B @ np.asarray(xi, dtype=np.float64)[:k])
    return np.array([s, r])


def level_pair(cfg, level, ids):
    """(q_fine [n, 2], q_coarse [n, 2]): level-`level` samples on meshes level and level-1
    with the same xi (the coarse mesh takes its first n_kl(level-1) terms); q_coarse zero
    on level 0."""
    from . import rng
    xi = rng.kl_coefficients(cfg["seed"], level, np.asarray(ids, dtype=np.uint64), n_kl(cfg, level))
    qf = np.array([solve_on_mesh(cfg, level, x) for x in xi])
    qc = np.array([solve_on_mesh(cfg, level - 1, x) for x in xi]) if level > 0 else np.zeros_like(qf)
    return qf, qc
