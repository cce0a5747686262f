// KL coefficients xi of (seed, level, sample id): Philox4x32-10 and polar normals.
//
// Both solves of a level pair must see the same xi (Sec. 2.2, Eq. MLMC_defn) and
// samples on different levels must be independent: the stream of level l uses
// key (lo32(seed), hi32(seed) ^ l * 0x9E3779B9) and sample id j uses counters
// (lo32(j), hi32(j), draw, 0). Philox4x32-10 is the counter-based generator of
// Salmon et al. (SC'11): ten rounds of two 32x32->64 multiplies and xors with a
// Weyl-sequence key schedule.
//
// Each counter yields two uniforms on (-1, 1), exactly v = (2x + 1) 2^-52 - 1 with
// x = (a >> 6) 2^26 + (b >> 6) from word pairs (a0, a1) and (a2, a3). Marsaglia's
// polar method accepts a pair when s = v1^2 + v2^2 < 1 and returns v f with
// f = sqrt(-2 ln s / s). All floating-point steps use explicitly rounded
// intrinsics (no contraction), and ln is the series below, so the values are
// reproducible bit for bit by any IEEE double implementation of the same steps.
//
// ln s: s = m 2^e with m in [sqrt(1/2), sqrt(2)); ln m = 2 atanh(t),
// t = (m - 1)/(m + 1), summed as 2t (1 + t^2/3 + ... + t^28/29) by Horner in t^2;
// ln s = e ln2_hi + (ln m + e ln2_lo) with ln 2 split into a 24-bit head and the
// rounded remainder.
#include "common.cuh"
#include "engine.h"

namespace mlmc {

namespace {

constexpr uint32_t kM0 = 0xD2511F53u, kM1 = 0xCD9E8D57u;
constexpr uint32_t kW0 = 0x9E3779B9u, kW1 = 0xBB67AE85u;
constexpr double kLn2Hi = 0x1.62e43p-1;
constexpr double kLn2Lo = -0x1.05c610ca86c39p-29;
constexpr double kSqrtHalf = 0x1.6a09e667f3bcdp-1;
constexpr int kAtanhTerms = 15;

__device__ __forceinline__ void philox(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t hi0 = __umulhi(kM0, c[0]), lo0 = kM0 * c[0];
    const uint32_t hi1 = __umulhi(kM1, c[2]), lo1 = kM1 * c[2];
    const uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
    k0 += kW0;
    k1 += kW1;
  }
}

__device__ __forceinline__ double series_ln(double x) {
  const long long bits = __double_as_longlong(x);
  int e = (int)((bits >> 52) & 0x7FF) - 1022;
  double m = __longlong_as_double((bits & 0x000FFFFFFFFFFFFFLL) | 0x3FE0000000000000LL);
  if (m < kSqrtHalf) {
    m = __dmul_rn(m, 2.0);
    e -= 1;
  }
  const double t = __ddiv_rn(__dsub_rn(m, 1.0), __dadd_rn(m, 1.0));
  const double t2 = __dmul_rn(t, t);
  // 1 / (2k + 1), correctly rounded (constant-folded at compile time)
  constexpr double kInvOdd[kAtanhTerms] = {1.0,        1.0 / 3.0,  1.0 / 5.0,  1.0 / 7.0,  1.0 / 9.0,
                                           1.0 / 11.0, 1.0 / 13.0, 1.0 / 15.0, 1.0 / 17.0, 1.0 / 19.0,
                                           1.0 / 21.0, 1.0 / 23.0, 1.0 / 25.0, 1.0 / 27.0, 1.0 / 29.0};
  double p = kInvOdd[kAtanhTerms - 1];
#pragma unroll
  for (int k = kAtanhTerms - 2; k >= 0; --k) {
    p = __dadd_rn(__dmul_rn(p, t2), kInvOdd[k]);
  }
  const double lnm = __dmul_rn(__dmul_rn(2.0, t), p);
  const double de = (double)e;
  return __dadd_rn(__dmul_rn(de, kLn2Hi), __dadd_rn(lnm, __dmul_rn(de, kLn2Lo)));
}

__device__ __forceinline__ double uniform_pm1(uint32_t a, uint32_t b) {
  const unsigned long long x = ((unsigned long long)(a >> 6) << 26) | (unsigned long long)(b >> 6);
  return __dsub_rn(__dmul_rn(__dadd_rn(__dmul_rn(2.0, (double)x), 1.0), 0x1p-52), 1.0);
}

// One warp per sample: xi[s * n_kl + n] (double), and optionally a float copy.
// With item arrays (levels, ids non-null) sample s uses (levels[s], ids[s]);
// otherwise (level, first_id + s). Draw d is a function of (key, id, d) alone, so
// the lanes evaluate draws d = 32 r + lane of round r together; an accepted draw's
// pair goes to position 2 * (accepted draws before it), found by a ballot prefix, which
// is the order of the one-draw-at-a-time definition (a then b, b dropped at n_kl).
__global__ void k_kl_coefficients(uint64_t seed, int level, uint64_t first_id, const int* __restrict__ levels,
                                  const uint64_t* __restrict__ ids, int64_t n, int n_kl, int max_draws,
                                  double* __restrict__ xi, float* __restrict__ xi32, int* __restrict__ fail) {
  const int64_t s = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (s >= n) return;   // whole warps
  const uint64_t id = ids ? ids[s] : first_id + (uint64_t)s;
  const int lv = levels ? levels[s] : level;
  const uint32_t key0 = (uint32_t)seed;
  const uint32_t key1 = (uint32_t)(seed >> 32) ^ ((uint32_t)lv * kW0);
  double* out = xi + s * n_kl;
  float* out32 = xi32 ? xi32 + s * n_kl : nullptr;
  int got = 0;
  for (int d0 = 0; d0 < max_draws && got < n_kl; d0 += 32) {
    const int d = d0 + lane;
    uint32_t c[4] = {(uint32_t)id, (uint32_t)(id >> 32), (uint32_t)d, 0u};
    philox(c, key0, key1);
    const double v1 = uniform_pm1(c[0], c[1]);
    const double v2 = uniform_pm1(c[2], c[3]);
    const double sq = __dadd_rn(__dmul_rn(v1, v1), __dmul_rn(v2, v2));
    const bool accept = sq < 1.0 && d < max_draws;
    const unsigned mask = __ballot_sync(0xffffffffu, accept);
    const int pos = got + 2 * __popc(mask & ((1u << lane) - 1u));
    if (accept && pos < n_kl) {
      const double f = __dsqrt_rn(__ddiv_rn(__dmul_rn(-2.0, series_ln(sq)), sq));
      const double a = __dmul_rn(v1, f), b = __dmul_rn(v2, f);
      out[pos] = a;
      if (out32) out32[pos] = (float)a;
      if (pos + 1 < n_kl) {
        out[pos + 1] = b;
        if (out32) out32[pos + 1] = (float)b;
      }
    }
    got = min(n_kl, got + 2 * __popc(mask));
  }
  if (got < n_kl && lane == 0) atomicExch(fail, 1);
}

}  // namespace

cudaError_t launch_kl_coefficients(uint64_t seed, int level, uint64_t first_id, const int* levels,
                                   const uint64_t* ids, int64_t n, int n_kl, double* xi, float* xi32, int* fail,
                                   cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int threads = 256;   // 8 samples per block
  const int64_t blocks = (n * 32 + threads - 1) / threads;
  // acceptance probability is pi/4 per draw; this cap is never reached in practice
  const int max_draws = 4 * ((n_kl + 1) / 2) + 256;
  k_kl_coefficients<<<(unsigned)blocks, threads, 0, st>>>(seed, level, first_id, levels, ids, n, n_kl,
                                                          max_draws, xi, xi32, fail);
  return cudaGetLastError();
}

}  // namespace mlmc
