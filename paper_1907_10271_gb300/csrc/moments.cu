// Level differences Y = Q_l - Q_{l-1} (Y_0 = Q_0, Eq. MLMC_defn) folded into the
// running per-level moments (Eq. varianceestim) in double precision.
//
// One 256-thread block: thread t takes a contiguous run of samples and runs
// Welford's update on Y (per quantity) and Kahan-compensated sums of Q_l, Q_{l-1};
// the 256 partial states are merged pairwise in a fixed tree with Chan's formula
// (M2 = M2a + M2b + delta^2 na nb / n), then merged into the level's running
// state. The summation order depends only on n, so results are reproducible.
// Samples whose status is non-zero are skipped.
#include "moments.cuh"

namespace mlmc {

namespace {

struct Part {
  double n;
  double mean[2], m2[2];
  double sqf[2], cqf[2], sqc[2], cqc[2];
};

__device__ __forceinline__ void kahan(double& s, double& c, double x) {
  const double y = x - c;
  const double t = s + y;
  c = (t - s) - y;
  s = t;
}

__device__ __forceinline__ void merge(Part& a, const Part& b) {
  const double n = a.n + b.n;
  if (b.n == 0.0) return;
  if (a.n == 0.0) {
    a = b;
    return;
  }
  for (int k = 0; k < 2; ++k) {
    const double d = b.mean[k] - a.mean[k];
    a.mean[k] += d * (b.n / n);
    a.m2[k] += b.m2[k] + d * d * (a.n * b.n / n);
    kahan(a.sqf[k], a.cqf[k], b.sqf[k]);
    a.cqf[k] += b.cqf[k];
    kahan(a.sqc[k], a.cqc[k], b.sqc[k]);
    a.cqc[k] += b.cqc[k];
  }
  a.n = n;
}

__global__ void __launch_bounds__(256) k_moments(const double* __restrict__ qf, const double* __restrict__ qc,
                                                 const int* __restrict__ status, int64_t n, LevelAcc* acc) {
  __shared__ Part parts[256];
  const int t = threadIdx.x;
  const int64_t per = (n + 255) / 256;
  const int64_t s0 = t * per, s1 = min(n, s0 + per);
  Part p;
  p.n = 0.0;
  for (int k = 0; k < 2; ++k) p.mean[k] = p.m2[k] = p.sqf[k] = p.cqf[k] = p.sqc[k] = p.cqc[k] = 0.0;
  for (int64_t s = s0; s < s1; ++s) {
    if (status && status[s] != 0) continue;
    p.n += 1.0;
    for (int k = 0; k < 2; ++k) {
      const double f = qf[2 * s + k];
      const double c = qc ? qc[2 * s + k] : 0.0;
      const double y = f - c;
      const double d = y - p.mean[k];
      p.mean[k] += d / p.n;
      p.m2[k] += d * (y - p.mean[k]);
      kahan(p.sqf[k], p.cqf[k], f);
      kahan(p.sqc[k], p.cqc[k], c);
    }
  }
  parts[t] = p;
  __syncthreads();
  for (int stride = 128; stride > 0; stride >>= 1) {
    if (t < stride) merge(parts[t], parts[t + stride]);
    __syncthreads();
  }
  if (t == 0) {
    Part a;
    a.n = (double)acc->n;
    for (int k = 0; k < 2; ++k) {
      a.mean[k] = acc->mean[k];
      a.m2[k] = acc->m2[k];
      a.sqf[k] = acc->sum_qf[k];
      a.cqf[k] = acc->comp_qf[k];
      a.sqc[k] = acc->sum_qc[k];
      a.cqc[k] = acc->comp_qc[k];
    }
    merge(a, parts[0]);
    acc->n = (long long)a.n;
    for (int k = 0; k < 2; ++k) {
      acc->mean[k] = a.mean[k];
      acc->m2[k] = a.m2[k];
      acc->sum_qf[k] = a.sqf[k];
      acc->comp_qf[k] = a.cqf[k];
      acc->sum_qc[k] = a.sqc[k];
      acc->comp_qc[k] = a.cqc[k];
    }
  }
}

}  // namespace

cudaError_t launch_moments(const double* qf, const double* qc, const int* status, int64_t n, LevelAcc* acc,
                           cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_moments<<<1, 256, 0, st>>>(qf, qc, status, n, acc);
  return cudaGetLastError();
}

}  // namespace mlmc
