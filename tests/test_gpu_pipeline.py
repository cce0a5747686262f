"""GPU parity of whole level pairs, moments, Algorithm 1 and the batch entry points.

Everything goes through the C ABI; every expected value comes from the CPU oracle
on the same (seed, level, id) inputs. Tolerances: 1e-9 relative per quantity on the
double-precision path, 1e-6 on the mixed-precision path.
"""
import math

import numpy as np
import pytest

from oracle import mlmc as om
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


def oracle_pairs(w, level, ids, workers=None):
    import os
    ids = np.asarray(ids, dtype=np.uint64)
    workers = workers or min(16, os.cpu_count() or 1, len(ids))
    if workers <= 1 or len(ids) <= 2:
        return om.level_pair(w, level, ids)
    return om.level_pair_parallel(w, level, ids, workers)


def rel(a, b):
    return np.abs(a - b) / np.abs(b)


def test_fp64_three_levels_full_counts(B):
    """The 3-level double-precision strip at its full sample counts (200/100/50)."""
    w = STRIP_FP64_3LEVEL
    ctx = B.mlmc_create(B.config_from_workload(w))
    try:
        for level, n in enumerate(w["n_per_level"]):
            qf = np.zeros(2 * n)
            qc = np.zeros(2 * n)
            st = np.ones(n, dtype=np.int32)
            B.mlmc_sample_level(ctx, level, 0, n, qf, qc, st)
            assert np.all(st == 0)
            rf, rc = oracle_pairs(w, level, np.arange(n))
            assert rel(qf.reshape(n, 2), rf).max() < 1e-9
            if level > 0:
                assert rel(qc.reshape(n, 2), rc).max() < 1e-9
            else:
                assert np.all(qc == 0)
            # moments of the level against the oracle's exactly rounded sums on the oracle's values
            s = B.mlmc_level_stats_get(ctx, level)
            y = rf - rc
            assert s["n"] == n
            for k in range(2):
                n_, mean, var = om.moments(y[:, k])
                assert s["mean"][k] == pytest.approx(mean, rel=1e-9, abs=1e-9 * abs(rf[:, k]).max())
                # Y carries 1e-9 relative errors of Q ~ 1e7..1e8: compare var against its scale
                assert abs(s["var"][k] - var) <= 1e-6 * var + (1e-9 * abs(rf[:, k]).max()) ** 2 * 4
                assert s["sum_qf"][k] == pytest.approx(math.fsum(rf[:, k]), rel=1e-9)
    finally:
        B.mlmc_destroy(ctx)


def test_moment_accumulator_against_exact_sums(B):
    """The device accumulator on the values the GPU itself returned: Welford/Chan with
    compensated sums against exactly rounded two-pass sums, over two calls."""
    w = STRIP_FP64_3LEVEL
    ctx = B.mlmc_create(B.config_from_workload(w))
    try:
        n1, n2 = 37, 91
        q1, c1 = np.zeros(2 * n1), np.zeros(2 * n1)
        q2, c2 = np.zeros(2 * n2), np.zeros(2 * n2)
        B.mlmc_sample_level(ctx, 1, 5, n1, q1, c1)
        B.mlmc_sample_level(ctx, 1, 5 + n1, n2, q2, c2)
        s = B.mlmc_level_stats_get(ctx, 1)
        y = np.concatenate([(q1 - c1).reshape(n1, 2), (q2 - c2).reshape(n2, 2)])
        qf = np.concatenate([q1.reshape(n1, 2), q2.reshape(n2, 2)])
        assert s["n"] == n1 + n2
        for k in range(2):
            _, mean, var = om.moments(y[:, k])
            assert s["mean"][k] == pytest.approx(mean, rel=1e-13, abs=1e-12)
            assert s["var"][k] == pytest.approx(var, rel=1e-10)
            assert s["sum_qf"][k] == pytest.approx(math.fsum(qf[:, k]), rel=1e-15)
        B.mlmc_reset_stats(ctx)
        assert B.mlmc_level_stats_get(ctx, 1)["n"] == 0
    finally:
        B.mlmc_destroy(ctx)


def test_mixed_five_levels_reduced_counts(B):
    """Every level of the 5-level mixed-precision strip, a few samples each."""
    w = STRIP_MIXED_5LEVEL
    ctx = B.mlmc_create(B.config_from_workload(w))
    try:
        for level, ids in enumerate([np.arange(0, 9), np.arange(100, 105), np.arange(7, 10), [41], [3]]):
            ids = np.asarray(ids)
            n = len(ids)
            qf = np.zeros(2 * n)
            qc = np.zeros(2 * n)
            st = np.ones(n, dtype=np.int32)
            # non-contiguous ids: one call per contiguous run
            runs = np.split(ids, np.where(np.diff(ids) != 1)[0] + 1)
            off = 0
            for r in runs:
                B.mlmc_sample_level(ctx, level, int(r[0]), len(r), qf[2 * off:2 * (off + len(r))],
                                    qc[2 * off:2 * (off + len(r))], st[off:off + len(r)])
                off += len(r)
            assert np.all(st == 0)
            rf, rc = oracle_pairs(w, level, ids)
            assert rel(qf.reshape(n, 2), rf).max() < 1e-6, level
            if level > 0:
                assert rel(qc.reshape(n, 2), rc).max() < 1e-6, level
    finally:
        B.mlmc_destroy(ctx)


def test_full_size_launch_sampled_outputs(B):
    """The benchmark's launch (all five levels at N_l = 8192/2048/512/128/32 in one
    mlmc_sample_levels call, which the library solves by nested iteration along each
    sample's mesh chain); sampled outputs of every level, the 1024 x 256 / 512 x 128
    pairs included, checked one by one against the oracle."""
    import torch
    w = STRIP_MIXED_5LEVEL
    counts = list(w["n_per_level"])
    total = sum(counts)
    ctx = B.mlmc_create(B.config_from_workload(w))
    try:
        qf = torch.zeros(2 * total, dtype=torch.float64, device="cuda")
        qc = torch.zeros_like(qf)
        st = torch.ones(total, dtype=torch.int32, device="cuda")
        B.mlmc_sample_levels(ctx, list(range(5)), [0] * 5, counts, qf, qc, st)
        torch.cuda.synchronize()
        assert int((st != 0).sum()) == 0
        qf = qf.cpu().numpy().reshape(total, 2)
        qc = qc.cpu().numpy().reshape(total, 2)
        offs = np.concatenate([[0], np.cumsum(counts)])
        assert B.mlmc_get_tuning(ctx)["nested_min_nodes"] <= sum(
            n * ((w["nx0"] << l) + 1) * ((w["ny0"] << l) + 1) for l, n in enumerate(counts))
        picks = {0: [0, 4097, 8191], 1: [5, 2047], 2: [300], 3: [77], 4: [0, 31]}
        for level, ids in picks.items():
            rf, rc = oracle_pairs(w, level, ids)
            got_f = qf[offs[level] + np.array(ids)]
            got_c = qc[offs[level] + np.array(ids)]
            assert rel(got_f, rf).max() < 1e-6, level
            if level > 0:
                assert rel(got_c, rc).max() < 1e-6, level
        # every level's moments were folded in once
        for level, n in enumerate(counts):
            assert B.mlmc_level_stats_get(ctx, level)["n"] == n
        # properties at any size: quantities positive and finite, level differences
        # shrink with the level (variance decay of Y_l, reaction quantity)
        assert np.all(np.isfinite(qf)) and np.all(qf > 0)
        v = [np.var(qf[offs[l]:offs[l + 1], 0] - qc[offs[l]:offs[l + 1], 0]) for l in range(1, 5)]
        assert all(b < a for a, b in zip(v, v[1:]))
    finally:
        B.mlmc_destroy(ctx)


@pytest.mark.parametrize("nested_min_nodes", [0, 1 << 40])
def test_sample_levels_matches_single_level_calls_and_solve_batch(B, nested_min_nodes):
    """Same xi on both meshes of a pair; results independent of batch composition.

    With threshold 0 mlmc_sample_level(s) solve each sample's meshes by nested
    iteration (each mesh starts from the next coarser one's solution), with a huge
    one in one lock-stepped batch from the lifting like mlmc_solve_batch: all end at
    ||f - K d|| <= 1e-8 ||f||, possibly from different starting iterates, so they
    agree to the solver's accuracy on the quantities (the stated 1e-6), while calls
    running the same procedure agree to rounding."""
    w = STRIP_MIXED_5LEVEL
    ctx = B.mlmc_create(B.config_from_workload(w))
    try:
        B.mlmc_set_nested_threshold(ctx, nested_min_nodes)
        counts = [5, 4, 3]
        total = sum(counts)
        qf = np.zeros(2 * total)
        qc = np.zeros(2 * total)
        B.mlmc_sample_levels(ctx, [0, 1, 2], [10, 20, 30], counts, qf, qc)
        off = 0
        items = []
        for level, n, first in zip([0, 1, 2], counts, [10, 20, 30]):
            f1 = np.zeros(2 * n)
            c1 = np.zeros(2 * n)
            B.mlmc_sample_level(ctx, level, first, n, f1, c1)
            np.testing.assert_allclose(f1, qf[2 * off:2 * (off + n)], rtol=1e-8)
            np.testing.assert_allclose(c1, qc[2 * off:2 * (off + n)], rtol=1e-8)
            for j in range(n):
                items.append((level, level, first + j))
                if level > 0:
                    items.append((level, level - 1, first + j))
            off += n
        qb = np.zeros(2 * len(items))
        sb = np.ones(len(items), dtype=np.int32)
        B.mlmc_solve_batch(ctx, items, qb, sb)
        assert np.all(sb == 0)
        k = 0
        off = 0
        for level, n in zip([0, 1, 2], counts):
            for j in range(n):
                np.testing.assert_allclose(qb[2 * k:2 * k + 2], qf[2 * (off + j):2 * (off + j) + 2], rtol=1e-6)
                k += 1
                if level > 0:
                    np.testing.assert_allclose(qb[2 * k:2 * k + 2], qc[2 * (off + j):2 * (off + j) + 2], rtol=1e-6)
                    k += 1
            off += n
    finally:
        B.mlmc_destroy(ctx)


@pytest.mark.parametrize("nested_min_nodes", [0, 1 << 40])
def test_telescoping_on_identical_samples(B, nested_min_nodes):
    """mean(Q_0) + sum_l mean(Q_l - Q_{l-1}) = mean(Q_L) when every mesh solves the same
    xi (Eq. MLMC_expectation), with each mesh's values produced by separate solves."""
    w = STRIP_FP64_3LEVEL
    ctx = B.mlmc_create(B.config_from_workload(w))
    try:
        B.mlmc_set_nested_threshold(ctx, nested_min_nodes)
        ids = list(range(12))
        Q = {}
        for m in range(3):
            q = np.zeros(2 * len(ids))
            B.mlmc_solve_batch(ctx, [(2, m, i) for i in ids], q)
            Q[m] = q.reshape(-1, 2)
        tel = Q[0].mean(0) + (Q[1] - Q[0]).mean(0) + (Q[2] - Q[1]).mean(0)
        np.testing.assert_allclose(tel, Q[2].mean(0), rtol=1e-14)
        # and the coarse solve inside a level-2 pair equals the mesh-1 solve of the same xi
        # (nested iteration or a lock-stepped pair vs single-mesh solves from the
        # lifting: equal to the double path's 1e-9)
        qf, qc = np.zeros(2 * len(ids)), np.zeros(2 * len(ids))
        B.mlmc_sample_level(ctx, 2, 0, len(ids), qf, qc)
        np.testing.assert_allclose(qc.reshape(-1, 2), Q[1], rtol=1e-9)
        np.testing.assert_allclose(qf.reshape(-1, 2), Q[2], rtol=1e-9)
    finally:
        B.mlmc_destroy(ctx)


def test_algorithm1_against_oracle(B):
    w = dict(STRIP_FP64_3LEVEL)
    e, theta, n_star = 1.5e5, 0.5, 12
    ctx = B.mlmc_create(B.config_from_workload(w))
    try:
        status, est, stats, L = B.mlmc_estimate(ctx, e, theta, n_star, 2, qoi=0)
        ref_est, Y, ref_L, conv = om.algorithm1(w, e, theta, n_star, 2, qoi=0)
        assert conv and status == B.MLMC_OK
        assert L == ref_L
        assert [s["n"] for s in stats] == [len(y) for y in Y]
        assert est == pytest.approx(ref_est, rel=1e-9)
        for s, y in zip(stats, Y):
            assert s["mean"][0] == pytest.approx(np.mean(y), rel=1e-8, abs=1e-6 * abs(ref_est))
    finally:
        B.mlmc_destroy(ctx)


def test_edge_cases(B):
    import torch
    w = STRIP_FP64_3LEVEL
    ctx = B.mlmc_create(B.config_from_workload(w))
    try:
        B.mlmc_sample_level(ctx, 0, 0, 0)                      # empty request is a no-op
        assert B.mlmc_level_stats_get(ctx, 0)["n"] == 0
        with pytest.raises(B.MLMCError, match="INVALID_ARG"):
            B.mlmc_sample_level(ctx, 3, 0, 1, np.zeros(2))      # level out of range
        with pytest.raises(B.MLMCError, match="INVALID_ARG"):
            B.mlmc_solve_batch(ctx, [(0, 5, 0)], np.zeros(2))
        # device and host buffers give the same values; null coarse/status outputs allowed
        n = 3
        qh = np.zeros(2 * n)
        B.mlmc_sample_level(ctx, 1, 1 << 33, n, qh, None, None)
        qd = torch.zeros(2 * n, dtype=torch.float64, device="cuda")
        B.mlmc_sample_level(ctx, 1, 1 << 33, n, qd)
        np.testing.assert_allclose(qd.cpu().numpy(), qh, rtol=1e-12)
        rf, _ = om.level_pair(w, 1, np.arange(1 << 33, (1 << 33) + n, dtype=np.uint64))
        assert rel(qh.reshape(n, 2), rf).max() < 1e-9
    finally:
        B.mlmc_destroy(ctx)
    bad = B.config_from_workload(w)
    bad.nx0 = 3
    with pytest.raises(B.MLMCError, match="INVALID_ARG"):
        B.mlmc_create(bad)


def test_non_converged_samples_are_excluded(B):
    """An iteration cap too small to converge: status NOT_CONVERGED, moments skip them."""
    w = STRIP_FP64_3LEVEL
    ctx = B.mlmc_create(B.config_from_workload(w, max_iter=2, max_outer=1))
    try:
        n = 4
        st = np.zeros(n, dtype=np.int32)
        B.mlmc_sample_level(ctx, 1, 0, n, np.zeros(2 * n), np.zeros(2 * n), st)
        assert np.all(st == B.MLMC_ERR_NOT_CONVERGED)
        assert B.mlmc_level_stats_get(ctx, 1)["n"] == 0
    finally:
        B.mlmc_destroy(ctx)


def test_graph_replay_equals_direct_launches(B):
    """PCG batches replayed from a captured CUDA graph give the results of the same
    launches issued directly (the kernel timer forces direct launches); only the
    order in which warps add their partial dot products may differ."""
    import torch
    w = STRIP_MIXED_5LEVEL
    side = torch.cuda.Stream()   # capturable (the legacy default stream is not)
    ctx = B.mlmc_create(B.config_from_workload(w), side.cuda_stream)
    try:
        out = []
        for timer in (False, True):
            B.mlmc_profile_enable(ctx, timer)
            qf = np.zeros(2 * 40)
            qc = np.zeros(2 * 40)
            B.mlmc_sample_levels(ctx, [1, 2], [300, 300], [32, 8], qf, qc)
            out.append((qf.copy(), qc.copy()))
        B.mlmc_profile_enable(ctx, False)
        np.testing.assert_allclose(out[0][0], out[1][0], rtol=1e-12)
        np.testing.assert_allclose(out[0][1], out[1][1], rtol=1e-12)
    finally:
        B.mlmc_destroy(ctx)


def test_autotune_keeps_results_and_moments(B):
    """mlmc_autotune leaves the level moments as they were, returns values inside the
    candidate set, and solves after tuning agree with solves before it (the stated
    1e-6: tuning changes launch shapes and possibly nested iteration, not the method)."""
    w = STRIP_MIXED_5LEVEL
    ctx = B.mlmc_create(B.config_from_workload(w))
    try:
        qa = np.zeros(2 * 6)
        B.mlmc_sample_level(ctx, 2, 5, 6, qa, np.zeros(12))
        before = B.mlmc_level_stats_get(ctx, 2)
        t = B.mlmc_autotune(ctx, [0, 1, 2], [64, 16, 6], reps=1)
        assert t["max_rows"] in (32, 64) and t["min_rows"] in (4, 6, 8)
        assert t["target_waves"] in (0.75, 1.5, 3.0) and t["nested_min_nodes"] in (0, 1 << 22, 1 << 62)
        assert t["fused_bottom"] in (0, 1, 2) and t["pack_samples"] in (0, 1)
        assert t["step_ms"] > 0
        assert B.mlmc_level_stats_get(ctx, 2) == before
        assert B.mlmc_get_tuning(ctx)["max_rows"] == t["max_rows"]
        qb = np.zeros(2 * 6)
        B.mlmc_solve_batch(ctx, [(2, 2, 5 + k) for k in range(6)], qb)
        np.testing.assert_allclose(qb, qa, rtol=1e-6)
        with pytest.raises(B.MLMCError):
            B.mlmc_set_tuning(ctx, 65, 4, 1.5, 0)
    finally:
        B.mlmc_destroy(ctx)


@pytest.mark.parametrize("nested_min_nodes", [0, 1 << 40])
def test_fused_bottom_matches_separate_launches(B, nested_min_nodes):
    """The multigrid bottom in one launch (levels nl-4 .. nl-2 and the coarsest per
    sample in a thread block, or nl-3, nl-2 and the coarsest per sample in a warp) does
    the same operations as the separate PreR / coarsest / Post launches: the solves
    agree to rounding, checked at the stated 1e-6."""
    w = STRIP_MIXED_5LEVEL
    out = {}
    for fused in (2, 1, 0):
        ctx = B.mlmc_create(B.config_from_workload(w))
        try:
            B.mlmc_set_tuning(ctx, 64, 6, 1.5, nested_min_nodes, fused)
            qf, qc = np.zeros(2 * 20), np.zeros(2 * 20)
            st = np.ones(20, dtype=np.int32)
            B.mlmc_sample_levels(ctx, [0, 1, 2, 3], [0, 0, 0, 0], [8, 6, 4, 2], qf, qc, st)
            assert np.all(st == 0)
            out[fused] = (qf, qc)
        finally:
            B.mlmc_destroy(ctx)
    for fused in (2, 1):
        np.testing.assert_allclose(out[fused][0], out[0][0], rtol=1e-6)
        np.testing.assert_allclose(out[fused][1], out[0][1], rtol=1e-6, atol=0)


@pytest.mark.parametrize("nested_min_nodes", [0, 1 << 40])
def test_packed_strips_match_one_sample_per_strip(B, nested_min_nodes):
    """Strip kernels that tile the samples of a mesh side by side (a warp may hold the
    end of one sample and the start of the next) give the solves of one sample per
    strip: samples do not couple across the seam, and per-sample sums and the CG
    steps taken by each sample's last warp stay per sample. 13 samples of every level
    (an odd count, so that some warp strips straddle two samples on every mesh)."""
    w = STRIP_MIXED_5LEVEL
    out = {}
    for pack in (1, 0):
        ctx = B.mlmc_create(B.config_from_workload(w))
        try:
            B.mlmc_set_tuning(ctx, 64, 6, 1.5, nested_min_nodes, 2, pack)
            n = 13
            qf, qc = np.zeros(2 * 5 * n), np.zeros(2 * 5 * n)
            st = np.ones(5 * n, dtype=np.int32)
            B.mlmc_sample_levels(ctx, [0, 1, 2, 3, 4], [7] * 5, [n] * 5, qf, qc, st)
            assert np.all(st == 0)
            out[pack] = (qf, qc)
        finally:
            B.mlmc_destroy(ctx)
    np.testing.assert_allclose(out[1][0], out[0][0], rtol=1e-6)
    np.testing.assert_allclose(out[1][1], out[0][1], rtol=1e-6, atol=0)


def test_device_loop_matches_host_loop(B):
    """With CUDA graphs (a non-legacy stream), repeating the PCG batches and their
    convergence test on the device (tuning device_loop = 1: a conditional graph node)
    takes the same batches as the host loop and gives the same quantities, for the
    lock-stepped and the nested paths."""
    import torch
    w = STRIP_MIXED_5LEVEL
    stream = torch.cuda.Stream()
    for nested in (0, 1 << 40):
        out = {}
        with torch.cuda.stream(stream):
            for dl in (1, 0):
                ctx = B.mlmc_create(B.config_from_workload(w), stream.cuda_stream)
                try:
                    t = B.mlmc_get_tuning(ctx)
                    B.mlmc_set_tuning(ctx, t["max_rows"], t["min_rows"], t["target_waves"], nested, t["fused_bottom"],
                                      t["pack_samples"], dl)
                    assert B.mlmc_get_tuning(ctx)["device_loop"] == dl
                    counts = [64, 32, 16, 4, 2]
                    tot = sum(counts)
                    qf, qc = np.zeros(2 * tot), np.zeros(2 * tot)
                    st = np.ones(tot, dtype=np.int32)
                    B.mlmc_sample_levels(ctx, [0, 1, 2, 3, 4], [11] * 5, counts, qf, qc, st)
                    stream.synchronize()
                    assert np.all(st == 0)
                    out[dl] = (qf, qc)
                finally:
                    B.mlmc_destroy(ctx)
        np.testing.assert_allclose(out[1][0], out[0][0], rtol=1e-9)
        np.testing.assert_allclose(out[1][1], out[0][1], rtol=1e-9, atol=0)


@pytest.mark.parametrize("nested_min_nodes", [0, 1 << 40])
def test_wide_strips_match_one_column_strips(B, nested_min_nodes):
    """The node-pair strip kernels (bits of tuning wide_strips: a lane holds columns 2l
    and 2l + 1, 60 output columns per strip) do the operations of the one-column
    kernels: the solves agree to rounding (the dot products are summed in another
    order), checked at the stated 1e-6, with every kernel in pairs, with the default
    mask, with samples side by side at every mesh width and with one sample per strip.
    13 samples of every level, so that strips straddle samples."""
    w = STRIP_MIXED_5LEVEL
    out = {}
    keys = ((B.MLMC_WIDE_ALL, 1), (B.MLMC_WIDE_ALL, 0), (B.MLMC_WIDE_POST | B.MLMC_WIDE_POST_TOP, 1))
    for wide, pack in ((0, 1),) + keys:
        ctx = B.mlmc_create(B.config_from_workload(w))
        try:
            B.mlmc_set_tuning(ctx, 64, 6, 1.5, nested_min_nodes, 1, pack, 0, wide)
            assert B.mlmc_get_tuning(ctx)["wide_strips"] == wide
            n = 13
            qf, qc = np.zeros(2 * 5 * n), np.zeros(2 * 5 * n)
            st = np.ones(5 * n, dtype=np.int32)
            B.mlmc_sample_levels(ctx, [0, 1, 2, 3, 4], [7] * 5, [n] * 5, qf, qc, st)
            assert np.all(st == 0)
            out[(wide, pack)] = (qf, qc)
        finally:
            B.mlmc_destroy(ctx)
    for key in keys:
        np.testing.assert_allclose(out[key][0], out[(0, 1)][0], rtol=1e-6)
        np.testing.assert_allclose(out[key][1], out[(0, 1)][1], rtol=1e-6, atol=0)


def test_smoother_damping_and_its_retry(B):
    """The smoother's damping changes the preconditioner, not the solution: solves at
    omega = 0.65 (the V-cycle stays SPD while omega < 2 / lambda_max(B^-1 K), and
    lambda_max is about 2.75 on these fields) agree with omega = 1/2 at the stated 1e-6.
    A damping past that bound (0.95) makes the preconditioner indefinite: a call in
    which a sample does not converge is solved again at 1/2, so every sample converges,
    the results equal omega = 1/2's, and the retry counter moves."""
    w = STRIP_MIXED_5LEVEL
    counts = [8, 6, 4, 2]
    out = {}
    for om in (0.5, 0.65, 0.95):
        ctx = B.mlmc_create(B.config_from_workload(w))
        try:
            t = B.mlmc_get_tuning(ctx)
            assert t["omega"] == 0.6 and t["omega_retries"] == 0
            B.mlmc_set_tuning(ctx, t["max_rows"], t["min_rows"], t["target_waves"], t["nested_min_nodes"],
                              t["fused_bottom"], t["pack_samples"], 0, t["wide_strips"], om)
            tot = sum(counts)
            qf, qc = np.zeros(2 * tot), np.zeros(2 * tot)
            st = np.ones(tot, dtype=np.int32)
            B.mlmc_sample_levels(ctx, [0, 1, 2, 3], [3] * 4, counts, qf, qc, st)
            assert np.all(st == 0)
            t = B.mlmc_get_tuning(ctx)
            assert t["omega"] == om
            out[om] = (qf, qc, t["omega_retries"])
        finally:
            B.mlmc_destroy(ctx)
    assert out[0.5][2] == 0 and out[0.65][2] == 0 and out[0.95][2] > 0
    for om in (0.65, 0.95):
        np.testing.assert_allclose(out[om][0], out[0.5][0], rtol=1e-6)
        np.testing.assert_allclose(out[om][1], out[0.5][1], rtol=1e-6, atol=0)
    with pytest.raises(B.MLMCError):
        ctx = B.mlmc_create(B.config_from_workload(w))
        try:
            B.mlmc_set_tuning(ctx, 64, 6, 1.5, 0, omega=1.0)
        finally:
            B.mlmc_destroy(ctx)
