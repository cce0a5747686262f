"""GPU parity of the individual hot-path steps against the oracle (through the C ABI)."""
import math

import numpy as np
import pytest

from oracle import fem, kl, material, rng
from workloads import STRIP_FP64_3LEVEL, STRIP_MIXED_5LEVEL

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_10271_gb300 import binding
    binding.lib()
    return binding


def make(B, w, **kw):
    return B.mlmc_create(B.config_from_workload(w, **kw))


@pytest.mark.parametrize("w", [STRIP_FP64_3LEVEL, STRIP_MIXED_5LEVEL])
@pytest.mark.parametrize("level,first,n", [(0, 0, 37), (2, 1000, 5), (1, (7 << 32) + 123, 4)])
def test_kl_coefficients_bit_exact(B, w, level, first, n):
    ctx = make(B, w)
    try:
        xi = np.zeros(n * w["kl_terms"])
        B.mlmc_kl_coefficients(ctx, level, first, n, xi)
        ref = rng.kl_coefficients(w["seed"], level, np.arange(first, first + n, dtype=np.uint64), w["kl_terms"])
        np.testing.assert_array_equal(xi.reshape(n, -1), ref)
    finally:
        B.mlmc_destroy(ctx)


def test_kl_coefficients_odd_terms(B):
    ctx = make(B, STRIP_FP64_3LEVEL, kl_terms=7)
    try:
        xi = np.zeros(9 * 7)
        B.mlmc_kl_coefficients(ctx, 1, 3, 9, xi)
        np.testing.assert_array_equal(xi.reshape(9, 7), rng.kl_coefficients(0, 1, np.arange(3, 12), 7))
    finally:
        B.mlmc_destroy(ctx)


def synthesis_bound(Bm, xi, n_kl, mixed, s):
    """Per-value error bound of theta = Xi B^T against the oracle's, from the terms.

    Both sides build the KL basis independently (cyclic Jacobi in the library, LAPACK
    in the oracle); their retained modes agree to about 1e-15 s, and 1e-13 s (s the
    field's standard deviation) is allowed for that.
    Double path: plus 2 n_kl 2^-53 sum|terms| (worst-case accumulation error of both
    sums).
    Mixed path (tensor cores, 3xTF32): splitting each operand x = hi + lo with hi, lo
    rounded to TF32 (2^-11 relative) leaves |x - hi - lo| <= 2^-22 |x|, so dropping
    lo*lo and the two residuals costs <= 3 * 2^-22 |term|; the FP32 accumulation of
    3 n_kl products is taken at four standard deviations of a random walk of
    unit-roundoff steps, 4 sqrt(3 n_kl) 2^-24, relative to sum|terms|.
    """
    mag = np.abs(xi) @ np.abs(Bm).T
    basis = 1e-13 * s
    if not mixed:
        return 2 * n_kl * 2.0 ** -53 * mag + basis
    return (3 * 2.0 ** -22 + 4 * math.sqrt(3 * n_kl) * 2.0 ** -24) * mag + basis


@pytest.mark.parametrize("w", [STRIP_FP64_3LEVEL, STRIP_MIXED_5LEVEL])
def test_theta_synthesis(B, w):
    ctx = make(B, w)
    try:
        for mesh in (0, 1, 2):
            level = min(mesh + 1, w["levels"] - 1)
            nx, ny = w["nx0"] << mesh, w["ny0"] << mesh
            n = 70 if mesh < 2 else 130    # more than two 64-sample tiles, ragged tail
            th = np.zeros(n * nx * ny)
            B.mlmc_theta(ctx, level, mesh, 11, n, th)
            xi = rng.kl_coefficients(w["seed"], level, np.arange(11, 11 + n), w["kl_terms"])
            Bm = kl.basis_for_mesh(w, nx, ny)
            ref = kl.theta_field(Bm, xi)
            bound = synthesis_bound(Bm, xi, w["kl_terms"], w["precision"] == "mixed",
                                    np.deg2rad(w["kl_std_deg"]))
            err = np.abs(th.reshape(n, -1) - ref)
            assert np.all(err <= bound), float(np.max(err / bound))
    finally:
        B.mlmc_destroy(ctx)


@pytest.mark.parametrize("w,tol", [(STRIP_FP64_3LEVEL, 1e-13), (STRIP_MIXED_5LEVEL, 3e-6)])
@pytest.mark.parametrize("mesh", [0, 2])
def test_operator_apply(B, w, tol, mesh):
    ctx = make(B, w)
    try:
        nx, ny = w["nx0"] << mesh, w["ny0"] << mesh
        n = 3
        g = np.random.default_rng(mesh)
        theta = g.normal(0, 0.3, (n, nx * ny))
        p = g.standard_normal((n, 2 * (nx + 1) * (ny + 1)))
        q = np.zeros_like(p)
        B.mlmc_apply(ctx, mesh, n, np.ascontiguousarray(theta), p, q)
        C = material.material_from_cfg(w)
        for s in range(n):
            K = fem.assemble(nx, ny, w["lx"], w["ly"], fem.rotated_stiffness(C, theta[s]))
            ref = K @ p[s]
            assert np.max(np.abs(q[s] - ref)) <= tol * np.max(np.abs(ref))
    finally:
        B.mlmc_destroy(ctx)


@pytest.mark.parametrize("w,tol", [(STRIP_FP64_3LEVEL, 1e-9), (STRIP_MIXED_5LEVEL, 1e-6)])
def test_solve_given_theta(B, w, tol):
    ctx = make(B, w)
    try:
        for mesh in (0, 1, 2):
            nx, ny = w["nx0"] << mesh, w["ny0"] << mesh
            n = 3
            xi = rng.kl_coefficients(w["seed"], 2, np.arange(n), w["kl_terms"])
            theta = kl.theta_field(kl.basis_for_mesh(w, nx, ny), xi)
            q = np.zeros(2 * n)
            st = np.zeros(n, dtype=np.int32)
            it = np.zeros(n, dtype=np.int32)
            B.mlmc_solve_theta(ctx, mesh, n, np.ascontiguousarray(theta), q, st, it)
            assert np.all(st == 0)
            for s in range(n):
                qr, qs, _ = fem.solve_sample(w, nx, ny, theta[s])
                assert abs(q[2 * s] - qr) <= tol * abs(qr), (mesh, s, q[2 * s], qr)
                assert abs(q[2 * s + 1] - qs) <= tol * abs(qs), (mesh, s, q[2 * s + 1], qs)
    finally:
        B.mlmc_destroy(ctx)


@pytest.mark.parametrize("theta0", [0.0, 0.05, -0.4])
def test_homogeneous_block_clamped_vs_oracle(B, theta0):
    """Uniform angle field (std 0): the GPU solve against the oracle's direct solve."""
    w = STRIP_FP64_3LEVEL
    ctx = make(B, w)
    try:
        nx, ny = w["nx0"], w["ny0"]
        theta = np.full((1, nx * ny), theta0)
        q = np.zeros(2)
        B.mlmc_solve_theta(ctx, 0, 1, theta, q)
        qr, qs, _ = fem.solve_sample(w, nx, ny, theta[0])
        assert q[0] == pytest.approx(qr, rel=1e-9)
        assert q[1] == pytest.approx(qs, rel=1e-9)
    finally:
        B.mlmc_destroy(ctx)


def test_mixed_refinement_reaches_tight_tolerance(B):
    """The single-precision inner solve with the float-float refinement residual must
    reach a relative residual far below single precision (1e-11): only a residual
    evaluated to about double accuracy allows it."""
    w = STRIP_MIXED_5LEVEL
    ctx = make(B, w, rtol=1e-11)
    try:
        for mesh in (0, 2):
            nx, ny = w["nx0"] << mesh, w["ny0"] << mesh
            n = 2
            xi = rng.kl_coefficients(w["seed"], 3, np.arange(n), w["kl_terms"])
            theta = np.ascontiguousarray(kl.theta_field(kl.basis_for_mesh(w, nx, ny), xi))
            q = np.zeros(2 * n)
            st = np.ones(n, dtype=np.int32)
            B.mlmc_solve_theta(ctx, mesh, n, theta, q, st)
            assert np.all(st == 0)
            for s in range(n):
                # the field is rounded to single precision on the GPU: compare on that field
                th32 = theta[s].astype(np.float32).astype(np.float64)
                qr, qs, _ = fem.solve_sample(w, nx, ny, th32)
                assert abs(q[2 * s] / qr - 1) < 1e-6
                assert abs(q[2 * s + 1] / qs - 1) < 1e-6
    finally:
        B.mlmc_destroy(ctx)
