"""GPU parity of the Cosserat engine (the paper's first test problem) against the oracle,
through the C ABI.

- the misalignment fields equal the oracle's analytic exponential-kernel KL applied to the
  same xi (double synthesis: 1e-12 of s_Phi);
- K x with the boundary conditions applied equals the oracle's assembled matrix (identity
  on the prescribed DOFs) applied to the same vectors (1e-12 of max |K x|);
- solutions d equal the oracle's sparse direct solves on meshes 0 - 2 (rtol 1e-11 run:
  1e-8 of max |d|);
- level pairs (strength, reaction) on levels 0 - 3 equal the oracle's within 1e-8 at
  rtol 1e-11 and 1e-6 at the workload's rtol 1e-8;
- the homogeneous block (s_Phi = 0) gives the closed-form strength R tau_y Q11 / Q12 and
  reaction Q11 |Delta| on every mesh (rtol 1e-11 run: 1e-9);
- moments equal numpy's on the returned quantities; several levels in one call equal
  their separate calls and solve_batch; n = 0 is a no-op; bad arguments are refused;
  an iteration cap below need returns MLMC_ERR_NOT_CONVERGED without a fault.
"""
import numpy as np
import pytest

from oracle import cosserat as C
from oracle import rng
from workloads import COSSERAT_TEST1 as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_10271_gb300 import binding
    binding.libc()
    return binding


def make(B, **kw):
    return B.mlmcc_create(B.configc_from_workload(W, **kw))


@pytest.fixture(scope="module")
def ctx(B):
    h = make(B, levels=4)
    yield h
    B.mlmcc_destroy(h)


@pytest.fixture(scope="module")
def tight(B):
    h = make(B, levels=4, rtol=1e-11)
    yield h
    B.mlmcc_destroy(h)


def masked(K, n):
    dd, _ = C.dirichlet(n, 1.0)
    keep = np.ones(K.shape[0])
    keep[dd] = 0.0
    import scipy.sparse as sp
    return (sp.diags(keep) @ K @ sp.diags(keep) + sp.diags(1.0 - keep)).tocsr()


@pytest.mark.parametrize("level,mesh", [(0, 0), (2, 1), (3, 3)])
def test_field_matches_oracle(B, ctx, level, mesh):
    n_s, first = 3, 7
    n = W["n0"] << mesh
    phi = np.zeros(n_s * n * n)
    B.mlmcc_field(ctx, level, mesh, first, n_s, phi)
    xi = rng.kl_coefficients(W["seed"], level, np.arange(first, first + n_s, dtype=np.uint64), C.n_kl(W, mesh))
    Bm, _ = C.kl_basis(W, n, C.n_kl(W, mesh))
    ref = (xi @ Bm.T).ravel()
    assert np.abs(phi - ref).max() <= 1e-12 * W["kl_std"]


@pytest.mark.parametrize("level,mesh", [(0, 0), (1, 1), (2, 2)])
def test_operator_matches_oracle(B, ctx, level, mesh):
    n_s, first = 2, 3
    n = W["n0"] << mesh
    N = (n + 1) ** 2
    x = np.random.default_rng(5).normal(size=(n_s, N, 3))
    y = np.zeros_like(x)
    B.mlmcc_apply(ctx, level, mesh, first, n_s, np.ascontiguousarray(x), y)
    xi = rng.kl_coefficients(W["seed"], level, np.arange(first, first + n_s, dtype=np.uint64), C.n_kl(W, mesh))
    Bm, _ = C.kl_basis(W, n, C.n_kl(W, mesh))
    for s in range(n_s):
        K = masked(C.assemble(W, n, Bm @ xi[s]), n)
        ref = (K @ x[s].ravel()).reshape(N, 3)
        assert np.abs(y[s] - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("level,mesh", [(0, 0), (1, 1), (2, 2)])
def test_displacement_matches_oracle(B, tight, level, mesh):
    n_s, first = 2, 20
    n = W["n0"] << mesh
    d = np.zeros(n_s * (n + 1) ** 2 * 3)
    st = np.zeros(n_s, dtype=np.int32)
    B.mlmcc_displacement(tight, level, mesh, first, n_s, d, st)
    assert (st == 0).all()
    xi = rng.kl_coefficients(W["seed"], level, np.arange(first, first + n_s, dtype=np.uint64), C.n_kl(W, mesh))
    Bm, _ = C.kl_basis(W, n, C.n_kl(W, mesh))
    d = d.reshape(n_s, -1)
    for s in range(n_s):
        _, _, ref = C.solve_sample(W, n, Bm @ xi[s])
        assert np.abs(d[s] - ref).max() <= 1e-8 * np.abs(ref).max()


@pytest.mark.parametrize("level,n_s", [(0, 8), (1, 6), (2, 4), (3, 2)])
def test_level_pairs_match_oracle(B, tight, ctx, level, n_s):
    first = 100
    ref_f, ref_c = C.level_pair(W, level, np.arange(first, first + n_s))
    for h, tol in ((tight, 1e-8), (ctx, 1e-6)):
        qf, qc = np.zeros(2 * n_s), np.zeros(2 * n_s)
        st = np.zeros(n_s, dtype=np.int32)
        B.mlmcc_reset_stats(h)
        B.mlmcc_sample_level(h, level, first, n_s, qf, qc, st)
        assert (st == 0).all()
        np.testing.assert_allclose(qf.reshape(n_s, 2), ref_f, rtol=tol)
        if level > 0:
            np.testing.assert_allclose(qc.reshape(n_s, 2), ref_c, rtol=tol)
        else:
            assert not qc.any()


def test_homogeneous_block_closed_form(B):
    h = make(B, levels=4, kl_std=0.0, rtol=1e-11)
    try:
        Cf, _ = C.fibre_stiffness(W)
        for mesh in range(4):
            q = np.zeros(4)
            B.mlmcc_solve_batch(h, [(mesh, mesh, 0), (mesh, mesh, 1)], q)
            q = q.reshape(2, 2)
            np.testing.assert_allclose(q[:, 0], W["R_ratio"] * W["tau_y"] * Cf[0, 0] / Cf[0, 1], rtol=1e-9)
            np.testing.assert_allclose(q[:, 1], Cf[0, 0] * abs(W["shortening"]), rtol=1e-9)
    finally:
        B.mlmcc_destroy(h)


def test_moments_batching_and_solve_batch(B, ctx):
    levels, firsts, counts = [0, 1, 2, 3], [0, 5, 9, 2], [40, 12, 6, 3]
    tot = sum(counts)
    qf, qc = np.zeros(2 * tot), np.zeros(2 * tot)
    st = np.zeros(tot, dtype=np.int32)
    B.mlmcc_reset_stats(ctx)
    B.mlmcc_sample_levels(ctx, levels, firsts, counts, qf, qc, st)
    assert (st == 0).all()
    qf, qc = qf.reshape(tot, 2), qc.reshape(tot, 2)
    off = 0
    for lv, f0, n in zip(levels, firsts, counts):
        s = B.mlmcc_level_stats(ctx, lv)
        y = qf[off:off + n] - qc[off:off + n]
        assert s["n"] == n
        np.testing.assert_allclose(s["mean"], y.mean(0), rtol=1e-12)
        np.testing.assert_allclose(s["var"], y.var(0), rtol=1e-9)
        # the same level alone, and its fine / coarse solves through solve_batch
        af, ac = np.zeros(2 * n), np.zeros(2 * n)
        B.mlmcc_sample_level(ctx, lv, f0, n, af, ac)
        np.testing.assert_allclose(af.reshape(n, 2), qf[off:off + n], rtol=1e-9)
        np.testing.assert_allclose(ac.reshape(n, 2), qc[off:off + n], rtol=1e-9)
        items = [(lv, lv, f0 + k) for k in range(n)] + [(lv, max(lv - 1, 0), f0 + k) for k in range(n)]
        qb = np.zeros(2 * len(items))
        B.mlmcc_solve_batch(ctx, items, qb)
        qb = qb.reshape(-1, 2)
        np.testing.assert_allclose(qb[:n], qf[off:off + n], rtol=1e-9)
        if lv > 0:
            np.testing.assert_allclose(qb[n:], qc[off:off + n], rtol=1e-9)
        off += n
    it, rf = B.mlmcc_last_iters(ctx)
    assert 0 < it <= 400 and rf >= 1
    assert B.mlmcc_launch_count(ctx) > 0


def test_edge_cases(B, ctx):
    B.mlmcc_sample_level(ctx, 0, 0, 0, None, None)          # n = 0: no-op
    with pytest.raises(B.MLMCError):
        B.mlmcc_sample_level(ctx, 7, 0, 1, np.zeros(2), np.zeros(2))
    with pytest.raises(B.MLMCError):
        B.mlmcc_sample_levels(ctx, [1, 1], [0, 0], [1, 1], np.zeros(4), np.zeros(4))
    with pytest.raises(B.MLMCError):
        B.mlmcc_solve_batch(ctx, [(0, 5, 0)], np.zeros(2))
    for bad in (dict(n0=6), dict(levels=0), dict(shortening=1e-3), dict(vf=1.2), dict(omega_side=10.0)):
        with pytest.raises(B.MLMCError):
            make(B, **bad)


def test_iteration_cap_reports_not_converged(B):
    h = make(B, levels=3, max_iter=2)
    try:
        q = np.zeros(8)
        st = np.ones(4, dtype=np.int32)
        B.mlmcc_solve_batch(h, [(2, 2, k) for k in range(4)], q, st)
        assert (st == 4).all()
        # the context stays usable
        h2 = make(B, levels=2)
        q2 = np.zeros(2)
        B.mlmcc_solve_batch(h2, [(1, 1, 0)], q2)
        B.mlmcc_destroy(h2)
        assert np.isfinite(q2).all()
    finally:
        B.mlmcc_destroy(h)


def test_algorithm1_matches_oracle(B):
    """mlmcc_estimate (Algorithm 1 on the strength) against the oracle's Algorithm 1 driven
    by the oracle's level pairs on the same ids: the same levels, the same N_l and the
    same estimate (to the QoI tolerance)."""
    from oracle import mlmc as M
    cfg = dict(W, levels=3)
    kw = dict(e=80.0, theta=0.5, n_star=8, max_level=2, qoi=0, m=4.0, alpha=0.786, gamma=1.3)
    h = make(B, levels=3)
    try:
        B.mlmcc_reset_stats(h)
        est, stats, L, conv = B.mlmcc_estimate(h, **kw)
    finally:
        B.mlmcc_destroy(h)

    def sampler(level, ids):
        qf, qc = C.level_pair(cfg, level, np.asarray(ids))
        return qf[:, 0] - qc[:, 0]

    def cost(level):
        return C.dofs(cfg, level) ** 1.3 + (C.dofs(cfg, level - 1) ** 1.3 if level > 0 else 0.0)

    ref, Y, L_ref, conv_ref = M.algorithm1(cfg, kw["e"], kw["theta"], kw["n_star"], kw["max_level"], qoi=0,
                                           alpha=kw["alpha"], gamma=kw["gamma"], m=kw["m"], sampler=sampler,
                                           cost=cost)
    assert L == L_ref and conv == conv_ref
    assert [s["n"] for s in stats] == [len(y) for y in Y]
    assert abs(est / ref - 1.0) < 1e-6


def test_level4_pair_matches_oracle(B):
    """The largest mesh of the workload (128 x 128, 49,923 DOFs) against the oracle."""
    h = make(B, levels=5)
    try:
        qf, qc = np.zeros(2), np.zeros(2)
        st = np.ones(1, dtype=np.int32)
        B.mlmcc_sample_level(h, 4, 77, 1, qf, qc, st)
        assert st[0] == 0
        ref_f, ref_c = C.level_pair(W, 4, [77])
        np.testing.assert_allclose(qf, ref_f[0], rtol=1e-6)
        np.testing.assert_allclose(qc, ref_c[0], rtol=1e-6)
    finally:
        B.mlmcc_destroy(h)
