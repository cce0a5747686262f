"""The allocation-free entry point against the regular one (GPU, through the C ABI).

mlmc_solve_theta_static serves callers that cannot allocate device memory: its
workspace is a static device array. Here it must reproduce mlmc_solve_theta on the
same fields, on two calls in a row (the array keeps the previous call's contents,
which must not leak into the next result), and reject a request that does not fit.
This file sorts last so that a run stopping at the first failure has run every
other test already.
"""
import numpy as np
import pytest

from oracle import kl, rng
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


def fields(w, mesh, n, first):
    nx, ny = w["nx0"] << mesh, w["ny0"] << mesh
    xi = rng.kl_coefficients(w["seed"], mesh + 1, np.arange(first, first + n), w["kl_terms"])
    return np.ascontiguousarray(kl.theta_field(kl.basis_for_mesh(w, nx, ny), xi))


# the tolerances the other parity tests use for each precision
@pytest.mark.parametrize("w,mesh,tol", [(STRIP_FP64_3LEVEL, 2, 1e-9), (STRIP_MIXED_5LEVEL, 0, 1e-6),
                                        (STRIP_MIXED_5LEVEL, 1, 1e-6)])
def test_static_matches_regular_entry_point_twice(B, w, mesh, tol):
    import torch
    cfg = B.config_from_workload(w)
    ctx = B.mlmc_create(cfg)
    try:
        for call, (n, first) in enumerate([(6, 0), (4, 100)]):
            theta = fields(w, mesh, n, first)
            ref = np.zeros(2 * n)
            ref_st = np.zeros(n, dtype=np.int32)
            B.mlmc_solve_theta(ctx, mesh, n, theta, ref, ref_st)
            # device buffers for inputs and outputs (the caller's), host path covered below
            th_d = torch.from_numpy(theta).cuda()
            q_d = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
            st_d = torch.full((n,), -1, dtype=torch.int32, device="cuda")
            B.mlmc_solve_theta_static(cfg, mesh, n, th_d, q_d, st_d)
            torch.cuda.synchronize()
            got = q_d.cpu().numpy()
            assert np.all(st_d.cpu().numpy() == 0) and np.all(ref_st == 0), call
            np.testing.assert_allclose(got, ref, rtol=tol, atol=0)
            # host buffers through the same entry point
            q_h = np.zeros(2 * n)
            st_h = np.full(n, -1, dtype=np.int32)
            B.mlmc_solve_theta_static(cfg, mesh, n, theta, q_h, st_h)
            np.testing.assert_allclose(q_h, ref, rtol=tol, atol=0)
            assert np.all(st_h == 0)
    finally:
        B.mlmc_destroy(ctx)


def test_static_rejects_requests_beyond_its_scratch(B):
    cfg = B.config_from_workload(STRIP_MIXED_5LEVEL)
    nx, ny = 1024, 256
    n = 2
    theta = np.zeros(n * nx * ny)
    q = np.zeros(2 * n)
    with pytest.raises(B.MLMCError, match="static scratch"):
        B.mlmc_solve_theta_static(cfg, 4, n, theta, q)


def test_static_on_a_side_stream_matches_regular_entry_point(B):
    """On a caller's own (non-default) stream the call still runs directly, with no
    graph capture: the results match the regular entry point's, twice in a row."""
    import torch
    w, mesh, tol = STRIP_MIXED_5LEVEL, 1, 1e-6
    cfg = B.config_from_workload(w)
    ctx = B.mlmc_create(cfg)
    side = torch.cuda.Stream()
    try:
        for call, (n, first) in enumerate([(5, 7), (3, 300)]):
            theta = fields(w, mesh, n, first)
            ref = np.zeros(2 * n)
            ref_st = np.zeros(n, dtype=np.int32)
            B.mlmc_solve_theta(ctx, mesh, n, theta, ref, ref_st)
            with torch.cuda.stream(side):
                th_d = torch.from_numpy(theta).cuda()
                q_d = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
                st_d = torch.full((n,), -1, dtype=torch.int32, device="cuda")
                B.mlmc_solve_theta_static(cfg, mesh, n, th_d, q_d, st_d, stream=side.cuda_stream)
            side.synchronize()
            assert np.all(st_d.cpu().numpy() == 0) and np.all(ref_st == 0), call
            np.testing.assert_allclose(q_d.cpu().numpy(), ref, rtol=tol, atol=0)
    finally:
        B.mlmc_destroy(ctx)


@pytest.mark.parametrize("field,value,match", [("levels", 0, "levels"), ("nx0", 1, "nx0"), ("rtol", 1.5, "rtol"),
                                               ("E22", -1.0, "moduli"), ("nu23", 1.5, "positive definite")])
def test_static_rejects_the_configs_the_context_rejects(B, field, value, match):
    cfg = B.config_from_workload(STRIP_MIXED_5LEVEL)
    setattr(cfg, field, value)
    theta = np.zeros(64 * 16)
    q = np.zeros(2)
    with pytest.raises(B.MLMCError, match=match):
        B.mlmc_solve_theta_static(cfg, 0, 1, theta, q)
    with pytest.raises(B.MLMCError, match=match):
        B.mlmc_create(cfg)
