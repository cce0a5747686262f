"""The smoother damping's bound (no GPU): the V-cycle preconditioner is SPD while
omega < 2 / lambda_max(B^-1 K), B the pair-block diagonal of the strip's stiffness
(u-DOFs of the node pairs {2m, 2m+1} of a row together, v-DOFs alone, Dirichlet DOFs
removed). These pins check the values the library's damping rests on, from the oracle's
own assembly (Eq. matrixinplane): every field stays under the colouring bound 4 (so
omega = 1/2 is always safe), fields of the benchmark workload (KL angles, 2 degrees
standard deviation) under 2 / 0.65, and fields turned far from the fibre axis above
2 / 0.6, which is why a larger damping needs the library's fall-back to 1/2. The last
test pins the same bound for the Cosserat engine's nodal block-Jacobi smoother."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import fem, kl, material
from workloads import STRIP_MIXED_5LEVEL as CFG

NX, NY = 32, 8


def pair_block_spectrum(theta):
    C = material.material_from_cfg(CFG)
    K = fem.assemble(NX, NY, CFG["lx"], CFG["ly"], fem.rotated_stiffness(C, theta)).toarray()
    n = K.shape[0]
    B = np.zeros_like(K)
    for j in range(NY + 1):
        for i in range(NX + 1):
            p = j * (NX + 1) + i
            B[2 * p, 2 * p] = K[2 * p, 2 * p]
            B[2 * p + 1, 2 * p + 1] = K[2 * p + 1, 2 * p + 1]
            if i % 2 == 0 and 0 < i and i + 1 < NX:   # both u of the pair free
                q = p + 1
                B[2 * p, 2 * q] = K[2 * p, 2 * q]
                B[2 * q, 2 * p] = K[2 * q, 2 * p]
    dd, _ = fem.dirichlet(NX, NY, CFG["shortening"])
    free = np.setdiff1d(np.arange(n), dd)
    return sla.eigh(K[np.ix_(free, free)], B[np.ix_(free, free)], eigvals_only=True)


@pytest.fixture(scope="module")
def basis():
    return kl.basis_for_mesh(CFG, NX, NY)


def test_workload_fields_allow_damping_065(basis):
    rng = np.random.default_rng(7)
    for _ in range(3):
        ev = pair_block_spectrum(kl.theta_field(basis, rng.standard_normal(basis.shape[1])))
        assert ev.min() > 0
        assert 2.5 < ev.max() < 2.0 / 0.65


def test_fibre_axis_field_and_colouring_bound():
    # uniform angles: 0 degrees is the workload's centre; 60 degrees is past 2 / 0.6
    ev0 = pair_block_spectrum(np.zeros(NX * NY))
    assert 2.6 < ev0.max() < 2.9
    ev60 = pair_block_spectrum(np.full(NX * NY, np.radians(60.0)))
    assert 2.0 / 0.6 < ev60.max() <= 4.0


def test_rough_fields_stay_under_the_colouring_bound(basis):
    rng = np.random.default_rng(11)
    for scale in (10.0, 45.0):   # standard deviations of 20 and 90 degrees
        ev = pair_block_spectrum(scale * kl.theta_field(basis, rng.standard_normal(basis.shape[1])))
        assert ev.max() <= 4.0


def test_cosserat_block_jacobi_allows_damping_065():
    """The Cosserat engine's nodal 3 x 3 block-Jacobi smoother (damping 0.65): on the
    paper's first test problem (Sec. 3.2 fields, and fields ten times rougher, and
    uniform angles) lambda_max(B^-1 A) of the oracle's assembly stays under 2 / 0.65."""
    from oracle import cosserat as O
    from workloads import COSSERAT_TEST1 as cfg
    n = 8
    dd, _ = O.dirichlet(n, cfg["shortening"])
    m = 3 * (n + 1) ** 2
    free = np.setdiff1d(np.arange(m), dd)

    def lam_max(phi):
        K = O.assemble(cfg, n, phi).toarray()
        Bd = np.zeros_like(K)
        for p in range((n + 1) ** 2):
            idx = [3 * p, 3 * p + 1, 3 * p + 2]
            Bd[np.ix_(idx, idx)] = K[np.ix_(idx, idx)]
        return sla.eigh(K[np.ix_(free, free)], Bd[np.ix_(free, free)], eigvals_only=True).max()

    Bk, _ = O.kl_basis(cfg, n, O.n_kl(cfg, 0))
    rng = np.random.default_rng(5)
    for scale in (1.0, 1.0, 10.0):
        assert lam_max(scale * (Bk @ rng.standard_normal(Bk.shape[1]))) < 2.0 / 0.65
    for deg in (0.0, 45.0, 90.0):
        assert lam_max(np.full(n * n, np.radians(deg))) < 2.0 / 0.65
