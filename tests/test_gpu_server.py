"""The request loop (continuous batching) and selective refinement, through the C ABI.

- a request's result is the same alone and in a mix of concurrent traffic (the stated
  1e-6 per quantity; nothing mixes samples, so the difference is summation order);
- served solves equal mlmc_solve_batch and the oracle;
- selective refinement follows the oracle's Algorithm 2 (same stopping meshes, same
  lambdas, same indicators);
- admission: a request that cannot fit a worker's share of the budget completes with
  MLMC_ERR_OOM, and the bytes admitted at once never exceed the budget.
"""
import time

import numpy as np
import pytest

from oracle import mlmc as om
from workloads import STRIP_FP64_3LEVEL, STRIP_MIXED_5LEVEL

pytestmark = pytest.mark.gpu

SOLVE, SEL = 0, 1


@pytest.fixture(scope="module")
def B():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_1907_10271_gb300 import binding
    binding.lib()
    return binding


def collect(B, srv, n, timeout_s=600):
    assert B.mlmc_server_drain(srv, timeout_s * 1e3), B.mlmc_server_last_error(srv)
    out = []
    while len(out) < n:
        got = B.mlmc_server_poll(srv, 4096)
        assert got, "drained server returned fewer results than submitted"
        out += got
    return {r["tag"]: r for r in out}


def rel(a, b):
    return abs(a - b) / max(abs(b), 1e-300)


def test_result_is_the_same_alone_and_in_the_mix(B):
    w = STRIP_MIXED_5LEVEL
    cfg = B.config_from_workload(w)
    cases = [(l, m, 1000 + 17 * k + l) for l in range(3) for m in sorted({l, max(l - 1, 0)}) for k in range(4)]
    probe = [(SOLVE, l, m, sid, tag) for tag, (l, m, sid) in enumerate(cases)]
    # alone: one worker, one request at a time
    srv = B.mlmc_server_create(cfg, workers=1, max_batch=64, hbm_budget_bytes=2e9)
    alone = {}
    try:
        for r in probe:
            B.mlmc_server_submit(srv, [r])
            alone.update(collect(B, srv, 1))
    finally:
        B.mlmc_server_destroy(srv)
    # in the mix: three workers, the probes interleaved with other traffic that keeps
    # arriving while earlier batches run
    g = np.random.default_rng(3)
    noise = [(SOLVE, int(l), int(l), 50000 + k, 10 ** 6 + k) for k, l in enumerate(g.integers(0, 3, 150))]
    traffic = probe + noise
    order = g.permutation(len(traffic))
    srv = B.mlmc_server_create(cfg, workers=3, max_batch=24, hbm_budget_bytes=3e9)
    try:
        for chunk in np.array_split(order, 6):
            B.mlmc_server_submit(srv, [traffic[i] for i in chunk])
            time.sleep(0.02)
        mix = collect(B, srv, len(traffic))
        counters = B.mlmc_server_counters(srv)
    finally:
        B.mlmc_server_destroy(srv)
    assert counters["batches"] > 6 and counters["solves"] == len(traffic)
    for r in probe:
        a, m = alone[r[4]], mix[r[4]]
        assert a["status"] == 0 and m["status"] == 0
        for k in range(2):
            assert rel(m["q"][k], a["q"][k]) < 1e-6, (r, a["q"], m["q"])
    # and both equal a plain batch solve of the same items
    ctx = B.mlmc_create(cfg)
    try:
        q = np.zeros(2 * len(probe))
        B.mlmc_solve_batch(ctx, [(r[1], r[2], r[3]) for r in probe], q)
    finally:
        B.mlmc_destroy(ctx)
    for k, r in enumerate(probe):
        for c in range(2):
            assert rel(alone[r[4]]["q"][c], q[2 * k + c]) < 1e-6


def test_served_solves_match_the_oracle(B):
    w = STRIP_FP64_3LEVEL
    srv = B.mlmc_server_create(B.config_from_workload(w), workers=2, max_batch=8, hbm_budget_bytes=1e9)
    cases = [(l, m, 7 + k) for l in range(3) for m in sorted({l, max(l - 1, 0)}) for k in range(3)]
    reqs = [(SOLVE, l, m, sid, tag) for tag, (l, m, sid) in enumerate(cases)]
    try:
        B.mlmc_server_submit(srv, reqs)
        res = collect(B, srv, len(reqs))
    finally:
        B.mlmc_server_destroy(srv)
    basis = om.Basis(w)
    for kind, l, m, sid, tag in reqs:
        xi = om.rng.kl_coefficients(w["seed"], l, [sid], w["kl_terms"])[0]
        ref = om.solve_on_mesh(w, basis, m, xi)
        for c in range(2):
            assert rel(res[tag]["q"][c], ref[c]) < 1e-9


def test_selective_refinement_matches_the_oracle(B):
    w = STRIP_FP64_3LEVEL
    basis = om.Basis(w)
    # threshold: an upper quantile of the level-1 stress from a seeded pilot on the
    # oracle, so that samples on both sides and near it occur
    pilot = [om.level_pair(w, 1, [k], basis)[0][0, 1] for k in range(40)]
    thr = om.upper_quantile(pilot, 0.3)
    srv = B.mlmc_server_create(B.config_from_workload(w), workers=2, max_batch=16, hbm_budget_bytes=1e9,
                               threshold=thr, sr_factor=2.0, eps_rel=1e-6)
    reqs = [(SEL, l, 0, sid, 1000 * l + sid) for l in range(3) for sid in range(12)]
    try:
        B.mlmc_server_submit(srv, reqs)
        res = collect(B, srv, len(reqs))
    finally:
        B.mlmc_server_destroy(srv)
    m, alpha = w.get("mlmc_m", 4.0), w.get("mlmc_alpha", 1.0)
    decided_early = 0
    for _, l, _, sid, tag in reqs:
        r = res[tag]
        assert r["status"] == 0
        J, lam, lf, lc, qf, qc = om.selective_refinement(w, l, sid, thr, m=m, alpha=alpha, sr_factor=2.0,
                                                          eps_rel=1e-6, basis=basis)
        assert r["stop_level"] == J and r["solves"] == J + 1
        assert all(rel(a, b) < 1e-9 for a, b in zip(r["lambdas"], lam))
        assert (r["q_fine"], r["q_coarse"]) == (qf, qc)
        assert rel(r["lambda_fine"], lf) < 1e-9
        decided_early += J < l
        assert r["latency_ms"] > 0
    assert decided_early > 0


def test_admission_by_memory_budget(B):
    w = STRIP_MIXED_5LEVEL
    cfg = B.config_from_workload(w)
    # a share (budget / workers) that holds level-2 meshes but not a 1024 x 256 solve
    srv = B.mlmc_server_create(cfg, workers=2, max_batch=1000, hbm_budget_bytes=2 * 20e6)
    reqs = [(SOLVE, 2, 2, k, k) for k in range(40)] + [(SOLVE, 4, 4, 0, 999)]
    try:
        B.mlmc_server_submit(srv, reqs)
        res = collect(B, srv, len(reqs))
        counters = B.mlmc_server_counters(srv)
    finally:
        B.mlmc_server_destroy(srv)
    assert res[999]["status"] == 2          # MLMC_ERR_OOM: larger than a worker's share
    assert all(res[k]["status"] == 0 for k in range(40))
    assert 0 < counters["peak_bytes"] <= 2 * 20e6
    assert counters["batches"] >= 4     # a 256 x 64 solve needs ~3.5 MB: the share splits the load


@pytest.mark.parametrize("k", [0, 1, 3])
@pytest.mark.parametrize("two_level", [False, True])
def test_failure_estimate_matches_the_oracle(B, k, two_level):
    # host arithmetic of the library on synthetic selective-refinement results
    g = np.random.default_rng(7 + k)
    n, thr = 2500, 1.0
    lv = g.integers(0, 4, n)
    lam0 = g.normal(0.0, 1.0, n) + 0.5
    qm0 = (lam0 > thr).astype(int)
    qf = np.where(g.random(n) < 0.1, 1 - qm0, qm0)
    qc = np.where(lv == 0, 0, np.where(g.random(n) < 0.05, 1 - qf, qf))
    res = [dict(tag=i, kind=SEL, level=int(lv[i]), mesh_level=0, sample_id=i, status=0, stop_level=0,
                lambdas=[float(lam0[i])], lambda_fine=0.0, lambda_coarse=0.0, q_fine=int(qf[i]), q_coarse=int(qc[i]))
           for i in range(n)]
    est, mean, var = B.mlmc_failure_estimate(res, thr, k=k, two_level=two_level)
    ref, terms = om.failure_estimate(lv, qf, qc, qm0, k=k, two_level=two_level)
    assert est == pytest.approx(ref, rel=1e-13, abs=1e-15)
    for l, (m, v) in terms.items():
        assert mean[l] == pytest.approx(m, rel=1e-13, abs=1e-15)
        assert var[l] == pytest.approx(v, rel=1e-13, abs=1e-15)


def _selective(B, w, thr, reqs, carry, workers, max_batch, chunks=1):
    srv = B.mlmc_server_create(B.config_from_workload(w), workers=workers, max_batch=max_batch,
                               hbm_budget_bytes=4e9, threshold=thr, sr_factor=2.0, eps_rel=1e-6,
                               carry_iterates=carry)
    try:
        for chunk in np.array_split(np.arange(len(reqs)), chunks):
            B.mlmc_server_submit(srv, [reqs[i] for i in chunk])
            if chunks > 1:
                time.sleep(0.02)
        return collect(B, srv, len(reqs))
    finally:
        B.mlmc_server_destroy(srv)


def test_carried_iterates_keep_results_and_save_iterations(B):
    """Selective refinement on the 5-level mixed strip with each sample's solution kept
    on the device between its solves (its next mesh starts from it) against every solve
    from the lifting: the same stopping meshes and lambdas (the stated 1e-6) and fewer
    PCG iterations per escalation solve."""
    w = STRIP_MIXED_5LEVEL
    ctx = B.mlmc_create(B.config_from_workload(w))
    try:
        n = 256
        qf, qc = np.zeros(2 * n), np.zeros(2 * n)
        B.mlmc_sample_level(ctx, 1, 0, n, qf, qc)
    finally:
        B.mlmc_destroy(ctx)
    thr = float(np.quantile(qf.reshape(n, 2)[:, 1], 0.6))
    reqs = [(SEL, l, 0, 300 + sid, 100 * l + sid) for l in range(1, 5) for sid in range(10)]
    on = _selective(B, w, thr, reqs, True, workers=2, max_batch=16)
    off = _selective(B, w, thr, reqs, False, workers=2, max_batch=16)
    esc_on, esc_off = [], []
    for r in reqs:
        a, b = on[r[4]], off[r[4]]
        assert a["status"] == 0 and b["status"] == 0
        assert a["stop_level"] == b["stop_level"] and a["solves"] == b["solves"]
        assert all(rel(x, y) < 1e-6 for x, y in zip(a["lambdas"], b["lambdas"]))
        assert a["pcg_iterations"][0] == b["pcg_iterations"][0]      # mesh 0: no coarser start either way
        esc_on += a["pcg_iterations"][1:]
        esc_off += b["pcg_iterations"][1:]
    assert len(esc_on) >= 20
    assert np.mean(esc_on) < 0.9 * np.mean(esc_off), (np.mean(esc_on), np.mean(esc_off))


def test_selective_result_is_the_same_alone_and_in_the_mix(B):
    """With carried iterates, a selective sample's escalations share batches with other
    requests (some starting from carried iterates, some from the lifting); each group of
    a batch keeps its own refinement sequence, so the lambdas equal the sample's alone."""
    w = STRIP_MIXED_5LEVEL
    thr = 1.3e8
    probe = [(SEL, l, 0, 700 + sid, 10 * l + sid) for l in range(1, 4) for sid in range(4)]
    alone = {}
    for r in probe:
        alone.update(_selective(B, w, thr, [r], True, workers=1, max_batch=8))
    g = np.random.default_rng(11)
    noise = [(SEL if k % 2 else SOLVE, int(l), int(l), 80000 + k, 10 ** 6 + k)
             for k, l in enumerate(g.integers(0, 4, 60))]
    traffic = probe + noise
    order = g.permutation(len(traffic))
    mix = _selective(B, w, thr, [traffic[i] for i in order], True, workers=3, max_batch=12, chunks=5)
    for r in probe:
        a, m = alone[r[4]], mix[r[4]]
        assert a["status"] == 0 and m["status"] == 0
        assert a["stop_level"] == m["stop_level"]
        assert all(rel(x, y) < 1e-6 for x, y in zip(a["lambdas"], m["lambdas"]))


# ---------------------------------------------------------------- panel requests
def _panel_oracle_sr(W, level, sid, thr):
    from oracle import plate as PL
    phi = PL.sample_perturbations(W, level, [sid])[0]
    return om.selective_refinement(W, level, sid, thr, m=4.0, alpha=1.0, sr_factor=2.0, eps_rel=1e-6,
                                   solve=lambda mesh: PL.solve_mesh(W, mesh, phi)[0], below=True)


def test_panel_selective_refinement_matches_the_oracle(B):
    """Panel requests through the same request loop: Algorithm 2 on the critical load
    P (failure below p*) gives the oracle's stopping meshes, loads (1e-6) and
    indicators, and SOLVE requests return the oracle's load."""
    from oracle import plate as PL
    from workloads import PANEL_RM_4LEVEL as W
    pilot = [PL.level_pair(W, 1, [k])[0][0, 0] for k in range(24)]
    thr = float(np.quantile(pilot, 0.4))
    W = dict(W, p_star=thr)
    srv = B.mlmcp_server_create(B.configp_from_workload(W), workers=2, max_batch=16, hbm_budget_bytes=2e9,
                                threshold=thr, sr_factor=2.0, eps_rel=1e-6)
    reqs = [(SEL, l, 0, 500 + sid, 100 * l + sid) for l in range(3) for sid in range(6)]
    reqs += [(SOLVE, 1, 1, 900 + k, 5000 + k) for k in range(3)]
    try:
        B.mlmc_server_submit(srv, reqs)
        res = collect(B, srv, len(reqs))
    finally:
        B.mlmc_server_destroy(srv)
    decided_early = 0
    for kind, l, m, sid, tag in reqs:
        r = res[tag]
        assert r["status"] == 0
        if kind == SOLVE:
            ref = PL.solve_mesh(W, m, PL.sample_perturbations(W, l, [sid])[0])
            assert rel(r["q"][0], ref[0]) < 1e-6
            continue
        J, lam, lf, lc, qf, qc = _panel_oracle_sr(W, l, sid, thr)
        assert r["stop_level"] == J and r["solves"] == J + 1
        assert all(rel(a, b) < 1e-6 for a, b in zip(r["lambdas"], lam))
        assert (r["q_fine"], r["q_coarse"]) == (qf, qc)
        assert r["q_mesh0"] == (1 if lam[0] < thr else 0)
        decided_early += J < l
    assert decided_early > 0


def test_panel_result_is_the_same_alone_and_in_the_mix(B):
    from workloads import PANEL_RM_4LEVEL as W
    cfg = B.configp_from_workload(W)
    probe = [(SOLVE, l, l, 60 + l, l) for l in range(3)] + [(SEL, 2, 0, 61, 10)]
    alone = {}
    srv = B.mlmcp_server_create(cfg, workers=1, max_batch=8, hbm_budget_bytes=1e9, threshold=272.47)
    try:
        for r in probe:
            B.mlmc_server_submit(srv, [r])
            alone.update(collect(B, srv, 1))
    finally:
        B.mlmc_server_destroy(srv)
    g = np.random.default_rng(5)
    noise = [(SOLVE, int(l), int(l), 7000 + k, 10 ** 6 + k) for k, l in enumerate(g.integers(0, 3, 40))]
    traffic = probe + noise
    order = g.permutation(len(traffic))
    srv = B.mlmcp_server_create(cfg, workers=3, max_batch=12, hbm_budget_bytes=2e9, threshold=272.47)
    try:
        for chunk in np.array_split(order, 4):
            B.mlmc_server_submit(srv, [traffic[i] for i in chunk])
            time.sleep(0.02)
        mix = collect(B, srv, len(traffic))
    finally:
        B.mlmc_server_destroy(srv)
    for r in probe:
        a, m = alone[r[4]], mix[r[4]]
        assert a["status"] == 0 and m["status"] == 0
        assert rel(m["q"][0], a["q"][0]) < 1e-6
        if r[0] == SEL:
            assert a["stop_level"] == m["stop_level"]
            assert all(rel(x, y) < 1e-6 for x, y in zip(a["lambdas"], m["lambdas"]))
