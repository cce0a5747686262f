"""Pins for the oracle's KL-coefficient generator (Philox4x32-10, ln, polar normals)."""
import math
import os
import subprocess
import sys

import numpy as np
import pytest

from oracle import rng

HERE = os.path.dirname(os.path.abspath(__file__))


def test_philox_matches_independent_implementation():
    """Triton ships its own Philox4x32-10; run it in interpreter mode on the CPU."""
    pytest.importorskip("triton")
    pytest.importorskip("torch")
    code = os.path.join(HERE, "philox_triton_ref.py")
    out = subprocess.run([sys.executable, code], capture_output=True, text=True, timeout=600,
                         env=dict(os.environ, TRITON_INTERPRET="1"))
    if out.returncode == 77:
        pytest.skip("triton interpreter unavailable: " + out.stdout[-200:])
    assert out.returncode == 0, out.stdout + out.stderr
    words = np.array([[int(v) for v in line.split()] for line in out.stdout.strip().splitlines()],
                     dtype=np.uint64)
    c0, c1, c2, c3, k0, k1 = words[:, :6].T
    mine = np.stack(rng.philox4x32_10(c0, c1, c2, c3, k0, k1), axis=1)
    np.testing.assert_array_equal(mine, words[:, 6:])


def test_philox_key_and_counter_sensitivity():
    # every output word changes when any single input bit changes (avalanche of a bijection)
    base = [np.uint64(x) for x in (1, 2, 3, 4)]
    k = (5, 6)
    ref = np.array(rng.philox4x32_10(*base, *k))
    for pos in range(4):
        for bit in (0, 13, 31):
            c = list(base)
            c[pos] = np.uint64(int(c[pos]) ^ (1 << bit))
            out = np.array(rng.philox4x32_10(*c, *k))
            assert np.all(out != ref)


def test_ln_accuracy_and_exact_points():
    x = np.concatenate([np.random.default_rng(0).uniform(1e-300, 1.0, 20000),
                        np.random.default_rng(1).uniform(0.5, 2.0, 20000),
                        np.ldexp(1.0, np.arange(-1000, 1000, 7)).astype(np.float64)])
    ref = np.log(x)
    got = rng.ln(x)
    ulp = np.abs(got - ref) / np.spacing(np.maximum(np.abs(ref), 1e-300))
    assert np.max(ulp[ref != 0]) <= 2.0
    assert rng.ln(1.0) == 0.0
    assert rng.LN2_HI + rng.LN2_LO == math.log(2.0)
    # the head has at most 24 significant bits so that e * ln2_hi is exact
    m, _ = math.frexp(rng.LN2_HI)
    assert (m * 2 ** 24) == int(m * 2 ** 24)


def test_uniform_pairs_are_exact_and_open():
    a = np.array([0, 0xFFFFFFFF, 0x12345678, 0xFFFFFFC0], dtype=np.uint64)
    b = np.array([0, 0xFFFFFFFF, 0x9ABCDEF0, 0x0000003F], dtype=np.uint64)
    v = rng._uniform_pm1(a, b)
    assert np.all(v > -1.0) and np.all(v < 1.0)
    x = ((a >> np.uint64(6)) << np.uint64(26)) | (b >> np.uint64(6))
    # v + 1 = (2x + 1) 2^-52 exactly
    np.testing.assert_array_equal((v + 1.0) * 2.0 ** 52, 2.0 * x.astype(np.float64) + 1.0)


def test_normals_are_standard_gaussian():
    from scipy import stats
    xi = rng.kl_coefficients(seed=0, level=0, ids=np.arange(4000), n_kl=50).reshape(-1)
    n = xi.size
    assert abs(xi.mean()) < 5.0 / math.sqrt(n)
    assert abs(xi.var() - 1.0) < 5.0 * math.sqrt(2.0 / n)
    assert abs(stats.kurtosis(xi, fisher=False) - 3.0) < 5.0 * math.sqrt(24.0 / n)
    assert stats.kstest(xi, "norm").pvalue > 1e-4


def test_polar_method_against_hand_evaluation():
    """First normals of one sample recomputed step by step from the Philox words."""
    seed, level, sid = 7, 2, 123456789012
    xi = rng.kl_coefficients(seed, level, [sid], 6)[0]
    k0, k1 = rng.stream_key(seed, level)
    got = []
    d = 0
    while len(got) < 6:
        w = rng.philox4x32_10(sid & 0xFFFFFFFF, sid >> 32, d, 0, k0, k1)
        w = [int(v) for v in w]
        v1 = (2.0 * (((w[0] >> 6) << 26) | (w[1] >> 6)) + 1.0) / 2.0 ** 52 - 1.0
        v2 = (2.0 * (((w[2] >> 6) << 26) | (w[3] >> 6)) + 1.0) / 2.0 ** 52 - 1.0
        s = v1 * v1 + v2 * v2
        if s < 1.0:
            f = math.sqrt(-2.0 * math.log(s) / s)
            got += [v1 * f, v2 * f]
        d += 1
    np.testing.assert_allclose(xi, got[:6], rtol=4e-16, atol=0)


def test_streams_levels_and_ids():
    a = rng.kl_coefficients(0, 1, np.arange(50), 20)
    b = rng.kl_coefficients(0, 2, np.arange(50), 20)
    c = rng.kl_coefficients(0, 1, np.arange(25, 75), 20)
    np.testing.assert_array_equal(a[25:], c[:25])     # a sample's xi depends on its id only
    assert not np.any(a == b)                          # levels draw from disjoint streams
    assert abs(np.corrcoef(a.reshape(-1), b.reshape(-1))[0, 1]) < 0.05
    odd = rng.kl_coefficients(0, 1, np.arange(50), 19)
    np.testing.assert_array_equal(odd, a[:, :19])      # odd N_KL drops the last partner
