"""Multi-GPU layout of the hot path, exercised with CPU ranks (gloo, world size 2).

Samples are independent, so ranks take disjoint sample-id ranges and never
exchange field or solver data; the only exchange is the per-level moments, merged
with mlmc_merge_stats (a host function of the library, no GPU needed). Each rank
here evaluates its shard with the CPU oracle in place of its GPU.
"""
import os

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

from oracle import mlmc  # noqa: E402
from workloads import STRIP_FP64_3LEVEL  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def local_stats(y_pairs):
    """Stats dict (as the library reports them) of Y rows [n, 2] with Q rows."""
    qf, qc = y_pairs
    y = qf - qc
    n = y.shape[0]
    mean = y.mean(axis=0)
    m2 = ((y - mean) ** 2).sum(axis=0)
    return dict(n=n, mean=list(mean), m2=list(m2), var=list(m2 / n), sum_qf=list(qf.sum(0)),
                sum_qc=list(qc.sum(0)), cost=0.0)


def _rank(rank, world, port, level, per_rank, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import sys
    sys.path.insert(0, ROOT)
    import bench
    from paper_1907_10271_gb300 import binding as B
    first = bench.shard_first_ids(rank, 0, [per_rank])[0]
    ids = np.arange(first, first + per_rank, dtype=np.uint64)
    qf, qc = mlmc.level_pair(STRIP_FP64_3LEVEL, level, ids)
    mine = local_stats((qf, qc))
    gathered = [None] * world
    dist.all_gather_object(gathered, mine)
    ids_all = [None] * world
    dist.all_gather_object(ids_all, ids.tolist())
    merged = gathered[0]
    for s in gathered[1:]:
        merged = B.mlmc_merge_stats(merged, s)
    if rank == 0:
        out.put((merged, ids_all))
    dist.barrier()
    dist.destroy_process_group()


def test_two_ranks_disjoint_shards_and_merged_moments():
    from paper_1907_10271_gb300 import build
    build.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    level, per_rank = 1, 6
    procs = [ctx.Process(target=_rank, args=(r, 2, port, level, per_rank, q)) for r in range(2)]
    for p in procs:
        p.start()
    merged, ids_all = q.get(timeout=600)
    for p in procs:
        p.join(timeout=600)
        assert p.exitcode == 0
    # shards are disjoint and the union is what one rank would have sampled
    assert not set(ids_all[0]) & set(ids_all[1])
    all_ids = np.array(ids_all[0] + ids_all[1], dtype=np.uint64)
    qf, qc = mlmc.level_pair(STRIP_FP64_3LEVEL, level, all_ids)
    ref = local_stats((qf, qc))
    assert merged["n"] == ref["n"] == 2 * per_rank
    np.testing.assert_allclose(merged["mean"], ref["mean"], rtol=1e-12)
    np.testing.assert_allclose(merged["m2"], ref["m2"], rtol=1e-9)
    np.testing.assert_allclose(merged["sum_qf"], ref["sum_qf"], rtol=1e-13)


def test_shard_ids_disjoint_across_ranks_and_steps():
    import sys
    sys.path.insert(0, ROOT)
    import bench
    counts = [8192, 2048, 512, 128, 32]
    seen = {l: [] for l in range(5)}
    for r in range(8):
        for k in range(20):
            for l, f in enumerate(bench.shard_first_ids(r, k, counts)):
                seen[l].append((f, f + counts[l]))
    for l, ranges in seen.items():
        ranges.sort()
        assert all(a[1] <= b[0] for a, b in zip(ranges, ranges[1:]))


def test_merge_stats_closed_form():
    from paper_1907_10271_gb300 import binding as B
    from paper_1907_10271_gb300 import build
    build.build()
    g = np.random.default_rng(0)
    a, b = g.normal(5, 2, (37, 2)), g.normal(5.5, 1, (11, 2))
    sa = local_stats((a, np.zeros_like(a)))
    sb = local_stats((b, np.zeros_like(b)))
    m = B.mlmc_merge_stats(sa, sb)
    both = np.vstack([a, b])
    np.testing.assert_allclose(m["mean"], both.mean(0), rtol=1e-14)
    np.testing.assert_allclose(m["var"], both.var(0), rtol=1e-12)
    assert m["n"] == 48
