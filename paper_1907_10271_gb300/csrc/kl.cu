// KL synthesis theta = Xi B^T (Eq. inftyKL truncated at N_KL terms).
//
// theta[s][e] = sum_n B[e][n] xi[s][n]: a dense contraction of the per-mesh basis
// (element rows, N_KL columns) with the per-sample coefficients. Register-tiled on
// the CUDA cores: each 256-thread block produces a 64 (elements) x 64 (samples)
// tile, each thread a 4 x 4 sub-tile, staging K-slices of both operands in shared
// memory; accumulation in the operand precision (FP32 in the mixed path, FP64 in
// the double path).
#include "engine.h"

namespace mlmc {

namespace {

constexpr int kTE = 64, kTS = 64, kTK = 16;

__device__ __forceinline__ void sincos_any(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_any(double x, double* s, double* c) { sincos(x, s, c); }

template <typename T>
__global__ void __launch_bounds__(256) k_kl_synthesis(const T* __restrict__ xi, const T* __restrict__ B,
                                                      int64_t nsamp, int n_el, int n_kl,
                                                      T* __restrict__ theta, bool trig2) {
  __shared__ T Bs[kTK][kTE + 1];
  __shared__ T Xs[kTK][kTS + 1];
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  const int e0 = blockIdx.x * kTE;
  const int64_t s0 = (int64_t)blockIdx.y * kTS;
  T acc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) acc[a][b] = (T)0;
  for (int k0 = 0; k0 < n_kl; k0 += kTK) {
    // 64 x 16 tiles of both operands: 1024 values, 4 per thread
#pragma unroll
    for (int r = 0; r < 4; ++r) {
      const int idx = threadIdx.x + r * 256;
      const int row = idx / kTK, kk = idx % kTK;
      const int e = e0 + row, k = k0 + kk;
      Bs[kk][row] = (e < n_el && k < n_kl) ? B[(int64_t)e * n_kl + k] : (T)0;
      const int64_t s = s0 + row;
      Xs[kk][row] = (s < nsamp && k < n_kl) ? xi[s * n_kl + k] : (T)0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < kTK; ++kk) {
      T bv[4], xv[4];
#pragma unroll
      for (int a = 0; a < 4; ++a) bv[a] = Bs[kk][tx + 16 * a];
#pragma unroll
      for (int b = 0; b < 4; ++b) xv[b] = Xs[kk][ty + 16 * b];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] += bv[a] * xv[b];
    }
    __syncthreads();
  }
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int64_t s = s0 + ty + 16 * b;
    if (s >= nsamp) continue;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int e = e0 + tx + 16 * a;
      if (e >= n_el) continue;
      if (trig2) {
        T sn, cs;
        sincos_any((T)2 * acc[a][b], &sn, &cs);
        theta[2 * (s * n_el + e)] = cs;
        theta[2 * (s * n_el + e) + 1] = sn;
      } else {
        theta[s * n_el + e] = acc[a][b];
      }
    }
  }
}

template <typename T>
__global__ void k_theta_to_trig2(const double* __restrict__ theta, int64_t n, T* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  T sn, cs;
  sincos_any((T)2 * (T)theta[i], &sn, &cs);
  out[2 * i] = cs;
  out[2 * i + 1] = sn;
}

}  // namespace

template <typename T>
cudaError_t launch_kl_synthesis(const T* xi, const T* basis, int64_t nsamp, int n_el, int n_kl,
                                T* out, bool trig2, cudaStream_t st) {
  if (nsamp <= 0) return cudaSuccess;
  dim3 grid((n_el + kTE - 1) / kTE, (unsigned)((nsamp + kTS - 1) / kTS));
  k_kl_synthesis<T><<<grid, 256, 0, st>>>(xi, basis, nsamp, n_el, n_kl, out, trig2);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_theta_to_trig2(const double* theta, int64_t n, T* trig2, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_theta_to_trig2<T><<<(unsigned)((n + 255) / 256), 256, 0, st>>>(theta, n, trig2);
  return cudaGetLastError();
}

template cudaError_t launch_kl_synthesis<float>(const float*, const float*, int64_t, int, int, float*, bool,
                                                cudaStream_t);
template cudaError_t launch_kl_synthesis<double>(const double*, const double*, int64_t, int, int,
                                                 double*, bool, cudaStream_t);
template cudaError_t launch_theta_to_trig2<float>(const double*, int64_t, float*, cudaStream_t);
template cudaError_t launch_theta_to_trig2<double>(const double*, int64_t, double*, cudaStream_t);

}  // namespace mlmc
