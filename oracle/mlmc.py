"""Level differences, sample statistics and Algorithm 1 (Sec. 2.2-2.3).

Level pair (Eq. MLMC_defn): a level-l sample j draws xi^(j) from the level-l
stream, synthesises theta on the fine mesh l and on the coarse mesh l-1 from that
same xi, solves both, and returns Y_l = Q_l - Q_{l-1} (Y_0 = Q_0).

Statistics: the estimator sums the level means (Eq. MLMC_defn); the variance
estimate is Eq. varianceestim, s_l^2 = mean(Y^2) - mean(Y)^2, evaluated with
exactly rounded sums (math.fsum).

Algorithm 1 (reading where the printed listing is silent): L starts at -1 and is
incremented at the top of each pass, so the first pass computes level 0; the
sample ids of level l are 0, 1, 2, ... in order, a top-up continues from the
current count; N_hat_l is rounded up and never lowers N_l; the sampling/bias
split is e_s^2 = theta e^2 and e_b^2 = (1 - theta) e^2 (Eq. tausplit); the bias
is estimated on the finest level as |Y_hat_L| / (m^alpha - 1) (Eq. bias_estimate,
c = 1). The cost of one level-l sample is modelled as M_l^gamma + M_{l-1}^gamma
(DOFs of the solves it needs, Eq. gamma), M_{-1} = 0.
"""
import math

import numpy as np

from . import fem, kl, rng


def mesh_dims(cfg, level):
    return cfg["nx0"] << level, cfg["ny0"] << level


def dofs(cfg, level):
    nx, ny = mesh_dims(cfg, level)
    return 2 * (nx + 1) * (ny + 1)


class Basis:
    """KL basis rows at the element centroids of each mesh, computed on demand."""

    def __init__(self, cfg):
        self.cfg = cfg
        self._b = {}

    def __call__(self, mesh_level):
        if mesh_level not in self._b:
            nx, ny = mesh_dims(self.cfg, mesh_level)
            self._b[mesh_level] = kl.basis_for_mesh(self.cfg, nx, ny)
        return self._b[mesh_level]


def solve_on_mesh(cfg, basis, mesh_level, xi_row):
    nx, ny = mesh_dims(cfg, mesh_level)
    theta = kl.theta_field(basis(mesh_level), xi_row[None, :])[0]
    qr, qs, _ = fem.solve_sample(cfg, nx, ny, theta)
    return np.array([qr, qs])


def level_pair_from_xi(cfg, level, xi, basis=None):
    """Q_fine[n, 2], Q_coarse[n, 2] for level `level` and given xi[n, N_KL]."""
    basis = basis or Basis(cfg)
    xi = np.atleast_2d(xi)
    qf = np.zeros((xi.shape[0], 2))
    qc = np.zeros((xi.shape[0], 2))
    for s in range(xi.shape[0]):
        qf[s] = solve_on_mesh(cfg, basis, level, xi[s])
        if level > 0:
            qc[s] = solve_on_mesh(cfg, basis, level - 1, xi[s])
    return qf, qc


def level_pair(cfg, level, ids, basis=None):
    """Q_fine, Q_coarse for the level-`level` samples `ids` (same xi on both meshes)."""
    xi = rng.kl_coefficients(cfg["seed"], level, ids, cfg["kl_terms"])
    return level_pair_from_xi(cfg, level, xi, basis)


def _pair_worker(args):
    cfg, level, ids = args
    return level_pair(cfg, level, ids)


def level_pair_parallel(cfg, level, ids, workers):
    """level_pair over a 'spawn' process pool (one chunk of ids per task)."""
    import multiprocessing as mp
    ids = np.asarray(ids)
    chunks = [c for c in np.array_split(ids, max(1, min(len(ids), 4 * workers))) if c.size]
    ctx = mp.get_context("spawn")
    with ctx.Pool(workers) as pool:
        parts = pool.map(_pair_worker, [(cfg, level, c) for c in chunks])
    return (np.concatenate([p[0] for p in parts]), np.concatenate([p[1] for p in parts]))


def moments(y):
    """(n, mean, s^2 of Eq. varianceestim) with exactly rounded sums.

    Eq. varianceestim, mean(Y^2) - mean(Y)^2, is evaluated in the algebraically
    identical centred form mean((Y - mean(Y))^2): the printed form cancels
    catastrophically when |mean| >> std (e.g. Y_0 = Q_0).
    """
    y = [float(v) for v in np.asarray(y).reshape(-1)]
    n = len(y)
    if n == 0:
        return 0, 0.0, 0.0
    mean = math.fsum(y) / n
    return n, mean, math.fsum((v - mean) * (v - mean) for v in y) / n


def optimal_samples(V, C, es2):
    """N_l = ceil(e_s^-2 (sum_k sqrt(V_k C_k)) sqrt(V_l / C_l))  (Eq. optimal_Nl)."""
    V = np.asarray(V, dtype=np.float64)
    C = np.asarray(C, dtype=np.float64)
    total = math.fsum(np.sqrt(V * C))
    return [int(math.ceil(total * math.sqrt(v / c) / es2)) for v, c in zip(V, C)]


def bias_estimate(y_hat_L, m, alpha):
    """|Y_hat_L| / (m^alpha - 1)  (Eq. bias_estimate with c = 1)."""
    return abs(y_hat_L) / (m ** alpha - 1.0)


def level_cost(cfg, level, gamma):
    c = dofs(cfg, level) ** gamma
    if level > 0:
        c += dofs(cfg, level - 1) ** gamma
    return float(c)


def algorithm1(cfg, e, theta, n_star, max_level, qoi=0, alpha=1.0, gamma=1.0, m=4,
               sampler=None, cost=None):
    """Adaptive MLMC (Algorithm 1). Returns (estimate, per-level Y lists, L, converged).

    `sampler(level, ids) -> Y[len(ids)]` defaults to the FE level pair of this module;
    `cost(level)`, the cost of one level pair, defaults to level_cost(cfg, level, gamma).
    """
    if sampler is None:
        basis = Basis(cfg)

        def sampler(level, ids):
            qf, qc = level_pair(cfg, level, ids, basis)
            return qf[:, qoi] - qc[:, qoi]

    es2 = theta * e * e
    eb = math.sqrt(1.0 - theta) * e
    Y = []
    L = -1
    converged = False
    while not converged:
        if L + 1 > max_level:
            break
        L += 1
        Y.append(list(sampler(L, np.arange(n_star))))
        V = [moments(y)[2] for y in Y]
        C = [cost(l) if cost is not None else level_cost(cfg, l, gamma) for l in range(L + 1)]
        N_hat = optimal_samples(V, C, es2)
        for l in range(L + 1):
            if len(Y[l]) < N_hat[l]:
                Y[l].extend(sampler(l, np.arange(len(Y[l]), N_hat[l])))
        if bias_estimate(moments(Y[L])[1], m, alpha) < eb:
            converged = True
    estimate = math.fsum(moments(y)[1] for y in Y)
    return estimate, Y, L, converged


# ---------------------------------------------------------------- selective refinement
#
# Sec. 2.4 (Algorithm 2). For one sample (level l, id) the failure quantity lambda
# (quantity 1, the centroid fibre stress) is computed on meshes j = 0, 1, ... from the
# sample's own xi. From j >= 1 (reading: the printed "j > 1" contradicts the rare-event
# table, where most samples stop after level 1) the sample bias estimate of
# Eq. sampleBias, |lambda_j - lambda_{j-1}| / (m^alpha - 1), decides: once
# |lambda_j - lambda*| is at least that estimate (Eq. testFailure), widened by a solver
# error bound (reading of "within 2 solver-error bounds": factor sr_factor on
# max(eps_rel |lambda_j|, bias)), every finer level has the same failure indicator and
# refinement stops at J = j; otherwise it continues, up to J = l. The sample's level-l
# value is lambda_J and its level-(l-1) value lambda_min(J, l-1); the failure
# indicator is 1(lambda > lambda*) (reading of the garbled 1(lambda_l - lambda*)).

def sr_stops(lam, j, level, threshold, m, alpha, sr_factor, eps_rel):
    """Stopping test of Algorithm 2 after lambda_j (lam holds lambda_0 .. lambda_j)."""
    if j >= level:
        return True
    if j < 1:
        return False
    bias = abs(lam[j] - lam[j - 1]) / (m ** alpha - 1.0)
    return abs(lam[j] - threshold) >= sr_factor * max(eps_rel * abs(lam[j]), bias)


def selective_refinement(cfg, level, sample_id, threshold, m=4.0, alpha=1.0, sr_factor=2.0, eps_rel=1e-6,
                         basis=None, solve=None, below=False):
    """Algorithm 2 for one sample: (J, [lambda_0 .. lambda_J], lambda_l, lambda_{l-1}, Q_l, Q_{l-1}).

    `solve(mesh) -> lambda` defaults to the FE solve of this module on the sample's xi.
    Failure is lambda > threshold, or lambda < threshold with below (a buckling load
    under its threshold, Sec. 4.2's Q(lambda)); the stopping test is the same either way.
    """
    if solve is None:
        basis = basis or Basis(cfg)
        xi = rng.kl_coefficients(cfg["seed"], level, [sample_id], cfg["kl_terms"])[0]

        def solve(mesh):
            return solve_on_mesh(cfg, basis, mesh, xi)[1]

    lam = []
    j = 0
    while True:
        lam.append(float(solve(j)))
        if sr_stops(lam, j, level, threshold, m, alpha, sr_factor, eps_rel):
            break
        j += 1
    lam_fine = lam[j]
    lam_coarse = lam[min(j, level - 1)] if level >= 1 else 0.0
    fails = (lambda v: v < threshold) if below else (lambda v: v > threshold)
    q_fine = 1 if fails(lam_fine) else 0
    q_coarse = (1 if fails(lam_coarse) else 0) if level >= 1 else 0
    return j, lam, lam_fine, lam_coarse, q_fine, q_coarse


def biased_probability(x, n, k=1):
    """Eq. biased_estimator: (x + k) / (N + k) for x events in N samples (reading: k = 1)."""
    return (x + k) / (n + k)


def trinomial_moments(y, k=1):
    """Mean and variance of a level difference Y in {-1, 0, 1} from the biased estimates
    of p_{+1} and p_{-1}: E[Y] = p_{+1} - p_{-1}, V[Y] = p_{+1} + p_{-1} - (p_{+1} - p_{-1})^2
    (the trinomial moments; the printed forms are garbled)."""
    y = np.asarray(y)
    n = y.size
    pp = biased_probability(int(np.sum(y == 1)), n, k)
    pm = biased_probability(int(np.sum(y == -1)), n, k)
    return pp - pm, pp + pm - (pp - pm) ** 2


def upper_quantile(values, fraction):
    """The order statistic ceil(N (1 - fraction)) (1-based) of the sorted values: the
    threshold exceeded by about `fraction` of them (reading for the 1/150 quantile)."""
    v = np.sort(np.asarray(values, dtype=np.float64))
    k = int(math.ceil(v.size * (1.0 - fraction)))
    return float(v[min(max(k, 1), v.size) - 1])


def failure_estimate(levels, q_fine, q_coarse, q_mesh0, k=1, two_level=False):
    """Failure probability from selective-refinement samples (Sec. 2.4): per level l the
    indicators Q_l (q_fine), Q_{l-1} (q_coarse) and 1(lambda_0 > lambda*) (q_mesh0).

    Multilevel form: sum over levels of E[Y_l], Y_l = Q_l - Q_{l-1}, Y_0 = Q_0.
    Two-level form (the paper's E[Q] ~ Q_0 + Y_{L,0}): the level-0 samples' Q_0 plus
    the top level's Y_{L,0} = Q_L - Q_0 of the same sample. Each term's mean and
    variance come from the biased estimates (x + k)/(N + k) of P(Y = +1) and
    P(Y = -1) (trinomial moments; a level-0 term has no -1 outcome).
    Returns (estimate, {term level: (mean, var)})."""
    levels = np.asarray(levels)
    top = int(levels.max())
    terms = {}
    for l in sorted(set(levels.tolist())):
        idx = levels == l
        if l == 0:
            y = np.asarray(q_fine)[idx]
        elif not two_level:
            y = np.asarray(q_fine)[idx] - np.asarray(q_coarse)[idx]
        elif l == top:
            y = np.asarray(q_fine)[idx] - np.asarray(q_mesh0)[idx]
        else:
            continue
        n = y.size
        pp = biased_probability(int(np.sum(y == 1)), n, k)
        pm = 0.0 if l == 0 else biased_probability(int(np.sum(y == -1)), n, k)
        terms[l] = (pp - pm, pp + pm - (pp - pm) ** 2)
    return math.fsum(m for m, _ in terms.values()), terms
