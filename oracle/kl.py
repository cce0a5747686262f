"""Truncated Karhunen-Loeve expansion of the misalignment field (Eq. inftyKL).

theta(x) = sum_{n=1}^{N_KL} sqrt(mu_n) phi_n(x) xi_n, where (mu_n, phi_n) are the
eigenpairs of the covariance operator (Eq. covarianceFunction gives the paper's
exponential kernel; the strip workloads use a squared-exponential kernel)

    k(x, y) = s^2 exp(-(x1 - y1)^2 / (2 l^2)) exp(-(x2 - y2)^2 / (2 l^2))

on the strip [0, lx] x [0, ly]. The kernel is separable, so the 2D eigenpairs are
products of the 1D eigenpairs of kx on [0, lx] and ky on [0, ly]:
mu_(i,j) = s^2 mu^x_i mu^y_j and phi_(i,j)(x) = phi^x_i(x1) phi^y_j(x2).

Each 1D operator is discretised by the Nystrom method on n_q Gauss-Legendre
points (x_q, w_q): the symmetric matrix A = W^1/2 K W^1/2 has eigenpairs
(mu, v) and phi(x_q) = v_q / sqrt(w_q), which makes sum_q w_q phi(x_q)^2 = 1.
The eigenfunctions are evaluated away from the nodes by the Nystrom
interpolant phi(x) = (1/mu) sum_q w_q k(x, x_q) phi(x_q).

Conventions this module fixes (the paper leaves them open):
  * sign: phi^x_i and phi^y_j are positive at the quadrature node nearest the
    origin of their interval;
  * order: the 2D modes are sorted by mu^x_i mu^y_j descending (ties broken by
    (i + j, i) ascending) and the first N_KL are kept;
  * the field is evaluated at element centroids (one angle per element).
"""
import numpy as np


def gauss_legendre(n, a):
    """n-point Gauss-Legendre nodes and weights on [0, a] (library primitive)."""
    x, w = np.polynomial.legendre.leggauss(n)
    return (x + 1.0) * (0.5 * a), w * (0.5 * a)


def se_kernel_1d(x, y, corr):
    return np.exp(-((x[:, None] - y[None, :]) ** 2) / (2.0 * corr * corr))


def eig_1d(a, corr, nq):
    """Nystrom eigenpairs of the 1D squared-exponential kernel on [0, a].

    Returns nodes, weights, eigenvalues (descending) and eigenfunction values at
    the nodes, phi[q, i], sign-fixed so that phi[0, i] > 0.
    """
    x, w = gauss_legendre(nq, a)
    sw = np.sqrt(w)
    A = sw[:, None] * se_kernel_1d(x, x, corr) * sw[None, :]
    mu, V = np.linalg.eigh(A)
    order = np.argsort(-mu, kind="stable")
    mu, V = mu[order], V[:, order]
    phi = V / sw[:, None]
    phi = phi * np.where(phi[0, :] < 0.0, -1.0, 1.0)[None, :]
    return x, w, mu, phi


def eval_1d(points, x, w, mu, phi, corr, modes):
    """Nystrom interpolant of eigenfunctions `modes` at `points` -> [len(points), len(modes)]."""
    Kp = se_kernel_1d(np.asarray(points, dtype=np.float64), x, corr)   # [p, q]
    return (Kp * w[None, :]) @ phi[:, modes] / mu[None, modes]


def select_modes(mux, muy, n_kl):
    """Index pairs (i, j) of the n_kl largest products mux[i] * muy[j]."""
    cand = [(-(mux[i] * muy[j]), i + j, i, j)
            for i in range(len(mux)) for j in range(len(muy))]
    cand.sort()
    return [(i, j) for (_, _, i, j) in cand[:n_kl]]


def kl_basis(lx, ly, corr, std_rad, nq, n_kl, px, py):
    """B[p, n] = sqrt(mu_n) phi_n(px[p], py[p]) for the first n_kl modes.

    Also returns the mode list [(i, j)] and the 2D eigenvalues mu_n (with s^2).
    """
    x, wx, mux, phx = eig_1d(lx, corr, nq)
    y, wy, muy, phy = eig_1d(ly, corr, nq)
    # only modes that can enter the top n_kl products matter
    modes = select_modes(mux[: n_kl + 1], muy[: n_kl + 1], n_kl)
    ii = sorted({i for i, _ in modes})
    jj = sorted({j for _, j in modes})
    fx = eval_1d(px, x, wx, mux, phx, corr, ii)
    fy = eval_1d(py, y, wy, muy, phy, corr, jj)
    col_x = {i: k for k, i in enumerate(ii)}
    col_y = {j: k for k, j in enumerate(jj)}
    mu2 = np.array([std_rad ** 2 * mux[i] * muy[j] for i, j in modes])
    B = np.empty((len(px), n_kl))
    for n, (i, j) in enumerate(modes):
        B[:, n] = np.sqrt(mu2[n]) * fx[:, col_x[i]] * fy[:, col_y[j]]
    return B, modes, mu2


def element_centroids(lx, ly, nx, ny):
    """Centroids of the nx x ny element grid, element e = j * nx + i."""
    hx, hy = lx / nx, ly / ny
    i = np.arange(nx)
    j = np.arange(ny)
    cx = np.tile((i + 0.5) * hx, ny)
    cy = np.repeat((j + 0.5) * hy, nx)
    return cx, cy


def basis_for_mesh(cfg, nx, ny):
    cx, cy = element_centroids(cfg["lx"], cfg["ly"], nx, ny)
    B, _, _ = kl_basis(cfg["lx"], cfg["ly"], cfg["kl_corr"], np.deg2rad(cfg["kl_std_deg"]),
                       cfg["kl_quad"], cfg["kl_terms"], cx, cy)
    return B


def theta_field(B, xi):
    """theta[s, e] = sum_n B[e, n] xi[s, n]   (Eq. inftyKL, truncated)."""
    return np.asarray(xi, dtype=np.float64) @ B.T
