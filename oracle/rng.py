"""KL coefficients xi for one (seed, level, sample id): Philox4x32-10 + polar normals.

The paper draws the KL coefficients xi_n as independent standard Gaussians
(Eq. inftyKL) and requires that both solves of a level pair use the same xi
(Sec. 2.2, Eq. MLMC_defn) while samples on different levels are independent
(Sec. 2.2, the MSE expansion). The generator below fixes how a counter-based
stream delivers that:

  key     = (lo32(seed), hi32(seed) XOR (level * 0x9E3779B9 mod 2^32))
  counter = (lo32(id), hi32(id), draw, 0),  draw = 0, 1, 2, ...

Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) maps each counter to four
32-bit words (a0, a1, a2, a3). Two uniforms on the open interval (-1, 1) are
formed exactly:  v = (2x + 1) 2^-52 - 1  with  x = (a >> 6) 2^26 + (b >> 6)
from the word pairs (a0, a1) and (a2, a3). Marsaglia's polar method accepts the
pair when s = v1^2 + v2^2 < 1 and returns v1 f, v2 f with f = sqrt(-2 ln(s) / s).
Normals are consumed in order until N_KL are collected (an odd N_KL discards the
last partner).

Every floating-point step is a single correctly rounded IEEE operation
(+, -, *, /, sqrt) with no fused multiply-add, and ln is computed here from
its series (below), so any implementation that follows these steps gets the same
bits. numpy ufuncs round each operation separately, which is what this needs.

Natural logarithm: write s = m 2^e with m in [sqrt(1/2), sqrt(2)); then
ln m = 2 atanh(t), t = (m - 1)/(m + 1), |t| <= 0.1716, summed as the odd
series 2 t (1 + t^2/3 + t^4/5 + ... + t^28/29) by Horner in t^2; and
ln s = e ln2_hi + (ln m + e ln2_lo), with ln2 split into a 24-bit head (so e ln2_hi
is exact) and the rounded remainder. ln 2 itself is evaluated in exact rational
arithmetic from ln 2 = 2 atanh(1/3).
"""
from fractions import Fraction
import math

import numpy as np

_M0 = np.uint64(0xD2511F53)
_M1 = np.uint64(0xCD9E8D57)
_W0 = 0x9E3779B9
_W1 = 0xBB67AE85
_MASK = np.uint64(0xFFFFFFFF)
_S32 = np.uint64(32)


def philox4x32_10(c0, c1, c2, c3, k0, k1):
    """Philox4x32 with 10 rounds on uint64 arrays holding 32-bit values.

    One round: (hi0, lo0) = M0 * c0 and (hi1, lo1) = M1 * c2 as full 64-bit
    products, then (c0, c1, c2, c3) <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0),
    and the key is bumped by the Weyl constants (W0, W1) between rounds.
    """
    c0, c1, c2, c3 = (np.asarray(c, dtype=np.uint64) & _MASK for c in (c0, c1, c2, c3))
    k0 = np.asarray(k0, dtype=np.uint64) & _MASK
    k1 = np.asarray(k1, dtype=np.uint64) & _MASK
    for r in range(10):
        p0 = _M0 * c0
        p1 = _M1 * c2
        hi0, lo0 = p0 >> _S32, p0 & _MASK
        hi1, lo1 = p1 >> _S32, p1 & _MASK
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & _MASK, lo1, (hi0 ^ c3 ^ k1) & _MASK, lo0
        if r < 9:
            k0 = (k0 + np.uint64(_W0)) & _MASK
            k1 = (k1 + np.uint64(_W1)) & _MASK
    return c0, c1, c2, c3


def stream_key(seed, level):
    """Philox key of the stream that serves every sample of `level`."""
    seed = int(seed) & 0xFFFFFFFFFFFFFFFF
    k0 = seed & 0xFFFFFFFF
    k1 = ((seed >> 32) ^ ((int(level) * _W0) & 0xFFFFFFFF)) & 0xFFFFFFFF
    return k0, k1


def _ln2_split():
    x = Fraction(1, 3)
    acc, power, k = Fraction(0), x, 0
    while power / (2 * k + 1) > Fraction(1, 10 ** 40):
        acc += power / (2 * k + 1)
        power *= x * x
        k += 1
    ln2 = 2 * acc
    f = float(ln2)
    _, e = math.frexp(f)
    hi = math.ldexp(float(round(ln2 * Fraction(2) ** (24 - e))), e - 24)
    lo = float(ln2 - Fraction(hi))
    return hi, lo


LN2_HI, LN2_LO = _ln2_split()
_ATANH_TERMS = 15                 # t^1 ... t^29
_ATANH_COEF = [1.0 / (2 * k + 1) for k in range(_ATANH_TERMS)]
_SQRT_HALF = math.sqrt(0.5)


def ln(x):
    """Natural log of positive normal doubles by the atanh series (module docstring)."""
    x = np.asarray(x, dtype=np.float64)
    m, e = np.frexp(x)                       # m in [0.5, 1)
    small = m < _SQRT_HALF
    m = np.where(small, m * 2.0, m)          # exact
    e = np.where(small, e - 1, e).astype(np.float64)
    t = (m - 1.0) / (m + 1.0)
    t2 = t * t
    p = np.full_like(t, _ATANH_COEF[-1])
    for c in reversed(_ATANH_COEF[:-1]):
        p = p * t2
        p = p + c
    lnm = (2.0 * t) * p
    return e * LN2_HI + (lnm + e * LN2_LO)


def _uniform_pm1(a, b):
    x = ((a >> np.uint64(6)) << np.uint64(26)) | (b >> np.uint64(6))
    return (2.0 * x.astype(np.float64) + 1.0) * 2.0 ** -52 - 1.0


def kl_coefficients(seed, level, ids, n_kl, chunk=None):
    """xi[len(ids), n_kl] (float64) for the samples `ids` of `level` (module docstring)."""
    ids = np.asarray(ids, dtype=np.uint64).reshape(-1)
    n = ids.size
    out = np.zeros((n, n_kl), dtype=np.float64)
    if n == 0 or n_kl == 0:
        return out
    k0, k1 = stream_key(seed, level)
    need_pairs = (n_kl + 1) // 2
    got = np.zeros(n, dtype=np.int64)
    draw = 0
    lo = ids & _MASK
    hi = ids >> _S32
    block = chunk or max(8, need_pairs + need_pairs // 2 + 4)
    while np.any(got < need_pairs):
        d = np.arange(draw, draw + block, dtype=np.uint64)
        c0 = np.broadcast_to(lo[:, None], (n, block))
        c1 = np.broadcast_to(hi[:, None], (n, block))
        c2 = np.broadcast_to(d[None, :], (n, block))
        a0, a1, a2, a3 = philox4x32_10(c0, c1, c2, 0, k0, k1)
        v1 = _uniform_pm1(a0, a1)
        v2 = _uniform_pm1(a2, a3)
        s = v1 * v1
        s = s + v2 * v2
        acc = s < 1.0
        s_safe = np.where(acc, s, 0.5)
        f = np.sqrt((-2.0 * ln(s_safe)) / s_safe)
        rank = np.cumsum(acc, axis=1) - 1 + got[:, None]      # pair index of each accepted draw
        take = acc & (rank < need_pairs)
        ii, jj = np.nonzero(take)
        kk = 2 * rank[ii, jj]
        out[ii, kk] = v1[ii, jj] * f[ii, jj]
        odd = kk + 1 < n_kl
        out[ii[odd], kk[odd] + 1] = v2[ii[odd], jj[odd]] * f[ii[odd], jj[odd]]
        got = np.minimum(got + acc.sum(axis=1), need_pairs)
        draw += block
    return out
