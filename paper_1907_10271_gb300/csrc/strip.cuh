// Helpers shared by the strip kernels of fem.cu (one node column per lane) and
// strip_wide.cu (a node pair per lane): tile lookup, cp.async staging, per-lane sums and
// the PCG's per-sample scalar steps.
#pragma once
#include <cstdint>

#include "../../include/mlmc.h"
#include "fem.cuh"

namespace mlmc {
namespace {

// Per-lane sum of one chunk's row products: compensated in float for the FP32 kernels
// (at most 2 * 64 + 1 terms per lane, no double-precision arithmetic per node),
// plain double for the FP64 kernels. The warp and cross-warp sums are in double.
template <typename T>
struct LaneSum;
template <>
struct LaneSum<float> {
  float s = 0.f, c = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float y = x - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const { return (double)s - (double)c; }
};
template <>
struct LaneSum<double> {
  double s = 0.0;
  __device__ __forceinline__ void add(double x) { s += x; }
  __device__ __forceinline__ double value() const { return s; }
};

__device__ __forceinline__ double warp_sum(double x) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Locate the view, sample, strip and row chunk of this warp.
template <typename T>
__device__ __forceinline__ bool find_tile(const ViewList<T>& L, int gw, int& vi, int& s, int& strip, int& chunk) {
  vi = 0;
  while (vi < L.n && gw >= L.v[vi].work_begin + L.v[vi].nwork) ++vi;
  if (vi >= L.n || gw < L.v[vi].work_begin) return false;
  const View<T>& V = L.v[vi];
  const int tile = gw - V.work_begin;
  const int per_s = V.tiles_x * V.tiles_y;
  s = tile / per_s;
  const int r = tile - s * per_s;
  chunk = r / V.tiles_x;
  strip = r - chunk * V.tiles_x;
  return s < V.nsamp;
}

// Strips of a strip kernel that hold output columns of sample s.
template <typename T>
__device__ __forceinline__ int tiles_of_sample(const View<T>& V, int s, int cols) {
  if (!V.packed) return V.tiles_x * V.tiles_y;
  const int a = s * V.vw;
  return ((a + V.g.nx) / cols - a / cols + 1) * V.tiles_y;
}

// copy staging (cp.async, global to shared)
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
// copy `bytes` (4, 8 or 16) from global to shared; with `valid` false the slot entry
// is zero-filled and nothing is read
template <int kBytes>
__device__ __forceinline__ void cp_async(void* dst, const void* src, bool valid = true) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;" ::"r"(smem_u32(dst)), "l"(src), "n"(kBytes),
               "r"(valid ? kBytes : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory");
}

// ---------------------------------------------------------------- per-sample scalars
// The PCG's scalar steps run in the launch that completes their reduction: each live
// warp of a sample adds its partial sum and then counts itself in (lane 0); the warp
// whose count completes the sample's tiles sees every partial (fence before the count,
// fence after it, L2 reads) and takes the step. Nothing waits on another warp.

// True for the sample's last arriving warp, which also rearms the counter.
__device__ __forceinline__ bool last_tile(unsigned* arrive, int t, int tiles) {
  __threadfence();
  if (atomicAdd(&arrive[t], 1u) + 1u != (unsigned)tiles) return false;
  __threadfence();
  arrive[t] = 0u;
  return true;
}

// After b . z is complete (post-smoothing at the top level): convergence on the
// iteration's ||r||^2, then the conjugate-gradient beta = rz / rz_old. count[slot]
// receives the samples still active; batches start at even iterations, so slot and
// iteration have the same parity.
__device__ __forceinline__ void after_post(const SampleState& S, int t) {
  S.rpar[t] = (S.slot + 1) & 1;   // PreTop of this iteration wrote r' to buffer (iteration + 1) & 1
  const double rr = __ldcg(&S.red_rr[t]);
  if (rr <= S.tol2[t] * S.rr_ref[t]) {
    S.active[t] = 0;
    return;
  }
  const double rz = __ldcg(&S.red_rz[t]);
  if (!(rz > 0.0) || !isfinite(rz)) {   // preconditioned residual lost positivity
    S.active[t] = 0;
    S.status[t] = MLMC_ERR_NOT_CONVERGED;
    return;
  }
  const double old = S.rz_old[t];
  S.beta[t] = old > 0.0 ? rz / old : 0.0;
  S.rz_old[t] = rz;
  S.red_pq[t] = 0.0;
  S.iters[t] += 1;
  atomicAdd(&S.count[S.slot], 1);
}

// After p . q is complete: alpha = rz / pq, and the next iteration's sums start at 0.
__device__ __forceinline__ void after_p(const SampleState& S, int t) {
  const double pq = __ldcg(&S.red_pq[t]);
  if (!(pq > 0.0) || !isfinite(pq)) {
    S.active[t] = 0;
    S.status[t] = MLMC_ERR_NOT_CONVERGED;
    return;
  }
  S.alpha[t] = S.rz_old[t] / pq;
  S.red_rr[t] = 0.0;
  S.red_rz[t] = 0.0;
}

}  // namespace
}  // namespace mlmc
