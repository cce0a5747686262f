// Kernels of the 3D Hex8 block engine: the matrix-free trilinear element operator on
// cube elements with the ply stiffness rotated about y (Sec. 3.1's C* = T^-1 C T for
// an out-of-plane waviness angle), a geometric-multigrid V(1,1) with damped Jacobi
// smoothing, full weighting and trilinear prolongation, rediscretised coarse operators
// and a dense coarsest solve, the batched PCG updates, and the double-precision
// refinement residual and quantities of interest.
//
// Element operator. For a cube of side h with the 2x2x2 Gauss rule, the derivative of
// the trilinear interpolant along x at a Gauss point does not depend on its x
// coordinate: it is the bilinear (in y, z) interpolation, at the point's (y, z), of the
// four edge differences u(1, b, c) - u(0, b, c), divided by h. So the 9 gradient
// entries at all 8 points come from three sets of four edge differences and two
// one-dimensional interpolation passes each; the nodal forces, B^T sigma summed over
// the points, are the transposed passes. About 600 flops per element instead of the
// 24 x 24 matrix's 1152 multiply-adds, in FP32 for the inner solve and FP64 for the
// refinement residual.
#include <cfloat>

#include "dfloat.cuh"
#include "hex3d.cuh"

namespace mlmc3 {

using mlmc::DF;

namespace {

__constant__ Harmonics g_harm;


template <typename T>
struct V3 {
  T x, y, z;
};
template <typename T>
__device__ __forceinline__ V3<T> operator+(V3<T> a, V3<T> b) {
  return V3<T>{a.x + b.x, a.y + b.y, a.z + b.z};
}
template <typename T>
__device__ __forceinline__ V3<T> operator-(V3<T> a, V3<T> b) {
  return V3<T>{a.x - b.x, a.y - b.y, a.z - b.z};
}
template <typename T, typename S>
__device__ __forceinline__ V3<T> operator*(S s, V3<T> a) {
  return V3<T>{s * a.x, s * a.y, s * a.z};
}
template <typename T>
__device__ __forceinline__ T zero_of() {
  return T{};
}

// A float-float value whose sums take the shorter form (mlmc::df_add_short): the
// refinement operator's element pass after its edge differences. There the operands are
// at the scale of the differences or of the element forces, so the shorter sum's error
// (relative to its operands) is no larger than the differences' own rounding; the
// differences themselves, where displacements cancel to a strain times h, keep the full
// float-float sum.
struct DFs {
  float hi, lo;
};
__device__ __forceinline__ DFs operator+(DFs a, DFs b) {
  const DF r = mlmc::df_add_short(DF{a.hi, a.lo}, DF{b.hi, b.lo});
  return DFs{r.hi, r.lo};
}
__device__ __forceinline__ DFs operator-(DFs a, DFs b) {
  const DF r = mlmc::df_sub_short(DF{a.hi, a.lo}, DF{b.hi, b.lo});
  return DFs{r.hi, r.lo};
}
__device__ __forceinline__ DFs operator*(float s, DFs a) {
  const DF r = DF{a.hi, a.lo} * s;
  return DFs{r.hi, r.lo};
}
__device__ __forceinline__ DFs operator*(DFs a, float s) { return s * a; }
__device__ __forceinline__ DFs to_arith(DF a, DFs) { return DFs{a.hi, a.lo}; }
__device__ __forceinline__ float to_arith(float a, float) { return a; }
__device__ __forceinline__ double to_arith(double a, double) { return a; }
// the element pass's arithmetic type for a value type
template <typename T>
struct Arith {
  using type = T;
};
template <>
struct Arith<DF> {
  using type = DFs;
};
template <typename T>
__device__ __forceinline__ V3<T> zero3() {
  return V3<T>{zero_of<T>(), zero_of<T>(), zero_of<T>()};
}

// The 13 monoclinic entries at one angle, from (c2, s2, c4, s4).
template <typename T>
struct Cm {
  T c11, c12, c13, c15, c22, c23, c25, c33, c35, c44, c46, c55, c66;
};
template <typename T>
__device__ __forceinline__ T harm(int e, T c2, T s2, T c4, T s4);
template <>
__device__ __forceinline__ float harm<float>(int e, float c2, float s2, float c4, float s4) {
  const float* h = g_harm.f[e];
  return h[0] + h[1] * c2 + h[2] * s2 + h[3] * c4 + h[4] * s4;
}
template <>
__device__ __forceinline__ double harm<double>(int e, double c2, double s2, double c4, double s4) {
  const double* h = g_harm.d[e];
  return h[0] + h[1] * c2 + h[2] * s2 + h[3] * c4 + h[4] * s4;
}
template <typename T>
__device__ __forceinline__ Cm<T> coef(const float4 t) {
  const T c2 = (T)t.x, s2 = (T)t.y, c4 = (T)t.z, s4 = (T)t.w;
  Cm<T> C;
  C.c11 = harm<T>(0, c2, s2, c4, s4);
  C.c12 = harm<T>(1, c2, s2, c4, s4);
  C.c13 = harm<T>(2, c2, s2, c4, s4);
  C.c15 = harm<T>(3, c2, s2, c4, s4);
  C.c22 = harm<T>(4, c2, s2, c4, s4);
  C.c23 = harm<T>(5, c2, s2, c4, s4);
  C.c25 = harm<T>(6, c2, s2, c4, s4);
  C.c33 = harm<T>(7, c2, s2, c4, s4);
  C.c35 = harm<T>(8, c2, s2, c4, s4);
  C.c44 = harm<T>(9, c2, s2, c4, s4);
  C.c46 = harm<T>(10, c2, s2, c4, s4);
  C.c55 = harm<T>(11, c2, s2, c4, s4);
  C.c66 = harm<T>(12, c2, s2, c4, s4);
  return C;
}

// One-dimensional Gauss weights of the trilinear interpolation at xi = -+1/sqrt(3):
// a corner on the same side as the point gets wp, the other wm.
template <typename T>
struct GW {
  static constexpr T wp = (T)0.78867513459481288225;   // (1 + 1/sqrt 3) / 2
  static constexpr T wm = (T)0.21132486540518711775;   // (1 - 1/sqrt 3) / 2
};

// out[g1][g2] = sum_{a1, a2} w(a1, g1) w(a2, g2) in[a1][a2] (and its transpose: the same)
template <typename T, typename S>
__device__ __forceinline__ void interp2(const V3<T> in[2][2], V3<T> out[2][2]) {
  const S wp = GW<S>::wp, wm = GW<S>::wm;
  V3<T> t[2][2];
#pragma unroll
  for (int g = 0; g < 2; ++g)
#pragma unroll
    for (int b = 0; b < 2; ++b) t[g][b] = wp * in[g][b] + wm * in[1 - g][b];
#pragma unroll
  for (int g1 = 0; g1 < 2; ++g1)
#pragma unroll
    for (int g2 = 0; g2 < 2; ++g2) out[g1][g2] = wp * t[g1][g2] + wm * t[g1][1 - g2];
}

// f = K_e u for the cube element of side h; u, f indexed [ax][ay][az]. T is the value
// type (float, float-float or double), S the scalar type of the stiffness and weights,
// TA the type of everything after the edge differences (Arith<T>).
template <typename T, typename TA>
__device__ __forceinline__ V3<TA> edge(V3<T> hi, V3<T> lo, float ih) {
  const V3<T> d = ih * (hi - lo);
  return V3<TA>{to_arith(d.x, TA{}), to_arith(d.y, TA{}), to_arith(d.z, TA{})};
}
template <typename T, typename TA>
__device__ __forceinline__ V3<TA> edge(V3<T> hi, V3<T> lo, double ih) {
  const V3<T> d = ih * (hi - lo);
  return V3<TA>{to_arith(d.x, TA{}), to_arith(d.y, TA{}), to_arith(d.z, TA{})};
}
template <typename T, typename S, typename TA = T>
__device__ __forceinline__ void element_apply(const Cm<S>& C, S h, const V3<T> u[2][2][2], V3<TA> f[2][2][2]) {
  using T_ = TA;
  V3<T_> D[2][2], Gx[2][2], Gy[2][2], Gz[2][2];
  const S ih = (S)1 / h;
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) D[a][b] = edge<T, T_>(u[1][a][b], u[0][a][b], ih);   // x edges, [ay][az]
  interp2<T_, S>(D, Gx);                                                              // Gx[gy][gz]
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) D[a][b] = edge<T, T_>(u[a][1][b], u[a][0][b], ih);   // y edges, [ax][az]
  interp2<T_, S>(D, Gy);                                                              // Gy[gx][gz]
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) D[a][b] = edge<T, T_>(u[a][b][1], u[a][b][0], ih);   // z edges, [ax][ay]
  interp2<T_, S>(D, Gz);                                                              // Gz[gx][gy]
  // stresses at the 8 points, summed into the fluxes of each derivative direction
  V3<T_> Sx[2][2], Sy[2][2], Sz[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) Sx[a][b] = Sy[a][b] = Sz[a][b] = zero3<T_>();
#pragma unroll
  for (int gx = 0; gx < 2; ++gx)
#pragma unroll
    for (int gy = 0; gy < 2; ++gy)
#pragma unroll
      for (int gz = 0; gz < 2; ++gz) {
        const V3<T_> dx = Gx[gy][gz], dy = Gy[gx][gz], dz = Gz[gx][gy];   // d(u,v,w)/dx, /dy, /dz
        const T_ e1 = dx.x, e2 = dy.y, e3 = dz.z;
        const T_ e4 = dz.y + dy.z, e5 = dz.x + dx.z, e6 = dy.x + dx.y;
        const T_ s1 = C.c11 * e1 + C.c12 * e2 + C.c13 * e3 + C.c15 * e5;
        const T_ s2 = C.c12 * e1 + C.c22 * e2 + C.c23 * e3 + C.c25 * e5;
        const T_ s3 = C.c13 * e1 + C.c23 * e2 + C.c33 * e3 + C.c35 * e5;
        const T_ s4 = C.c44 * e4 + C.c46 * e6;
        const T_ s5 = C.c15 * e1 + C.c25 * e2 + C.c35 * e3 + C.c55 * e5;
        const T_ s6 = C.c46 * e4 + C.c66 * e6;
        Sx[gy][gz] = Sx[gy][gz] + V3<T_>{s1, s6, s5};
        Sy[gx][gz] = Sy[gx][gz] + V3<T_>{s6, s2, s4};
        Sz[gx][gy] = Sz[gx][gy] + V3<T_>{s5, s4, s3};
      }
  // transposed passes; Gauss weights 1, det J = (h / 2)^3, dN/dx = sign / h: (h / 2)^3 / h
  const S wj = h * h / (S)8;
  V3<T_> A[2][2];
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b)
#pragma unroll
      for (int c = 0; c < 2; ++c) f[a][b][c] = zero3<T_>();
  interp2<T_, S>(Sx, A);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      f[1][a][b] = f[1][a][b] + wj * A[a][b];
      f[0][a][b] = f[0][a][b] - wj * A[a][b];
    }
  interp2<T_, S>(Sy, A);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      f[a][1][b] = f[a][1][b] + wj * A[a][b];
      f[a][0][b] = f[a][0][b] - wj * A[a][b];
    }
  interp2<T_, S>(Sz, A);
#pragma unroll
  for (int a = 0; a < 2; ++a)
#pragma unroll
    for (int b = 0; b < 2; ++b) {
      f[a][b][1] = f[a][b][1] + wj * A[a][b];
      f[a][b][0] = f[a][b][0] - wj * A[a][b];
    }
}

__device__ __forceinline__ int64_t node_of(const Grid3& g, int i, int j, int k) {
  return ((int64_t)k * (g.ny + 1) + j) * (g.nx + 1) + i;
}
// prescribed DOFs: u, v, w on x = 0; u on x = lx
__device__ __forceinline__ float4 mask4(const Grid3& g, int i, float4 a) {
  if (i == 0) a.x = a.y = a.z = 0.f;
  if (i == g.nx) a.x = 0.f;
  a.w = 0.f;
  return a;
}
__device__ __forceinline__ void node_ijk(const Grid3& g, int64_t n, int& i, int& j, int& k) {
  i = (int)(n % (g.nx + 1));
  const int64_t r = n / (g.nx + 1);
  j = (int)(r % (g.ny + 1));
  k = (int)(r / (g.ny + 1));
}

__device__ __forceinline__ double block_sum(double v) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (w == 0) {
    t = l < (int)(blockDim.x >> 5) ? red[l] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) t += __shfl_xor_sync(0xffffffffu, t, o);
  }
  return t;   // valid in thread 0
}

// ---------------------------------------------------------------- field and smoother setup

__global__ void k_expand_trig(const float* __restrict__ t2, int64_t n, float* __restrict__ t4) {
  const int64_t c = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (c >= n) return;
  const float a = t2[2 * c], b = t2[2 * c + 1];
  reinterpret_cast<float4*>(t4)[c] = make_float4(a, b, 2.f * a * a - 1.f, 2.f * a * b);
}

__global__ void k_average_trig(Grid3 f, const float4* __restrict__ tf, float4* __restrict__ tc) {
  const int s = blockIdx.y;
  const int ncx = f.nx / 2, ncz = f.nz / 2;
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncx * ncz) return;
  const int I = c % ncx, K = c / ncx;
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
  for (int dk = 0; dk < 2; ++dk)
#pragma unroll
    for (int di = 0; di < 2; ++di) {
      const float4 t = tf[(int64_t)s * f.cols() + (int64_t)(2 * K + dk) * f.nx + 2 * I + di];
      acc.x += t.x;
      acc.y += t.y;
      acc.z += t.z;
      acc.w += t.w;
    }
  tc[(int64_t)s * ncx * ncz + c] = make_float4(0.25f * acc.x, 0.25f * acc.y, 0.25f * acc.z, 0.25f * acc.w);
}

// diag(K_e) at corner (sx, sy, sz) (signs) for displacement component c: with the
// 2x2x2 rule on a cube, sum_g grad N grad N^T = h [1/9 on the diagonal, s_p s_q / 12
// off it], contracted with C[c p c q]; of the off-diagonal C[c p c q] only the x-z
// ones (C15, C46, C35) are non-zero for a rotation about y.
__device__ __forceinline__ float3 corner_diag(const Cm<float>& C, float h, float sx, float sy, float sz) {
  const float a = 1.f / 9.f, b = 2.f / 12.f;
  float3 d;
  // u: Q = C[(11,12,13)][(11,12,13)] in Voigt (1, 6, 5)
  d.x = h * (a * (C.c11 + C.c66 + C.c55) + b * (sx * sz * C.c15));
  // v: Voigt (6, 2, 4)
  d.y = h * (a * (C.c66 + C.c22 + C.c44) + b * (sx * sz * C.c46));
  // w: Voigt (5, 4, 3)
  d.z = h * (a * (C.c55 + C.c44 + C.c33) + b * (sx * sz * C.c35));
  return d;
}

__global__ void k_dinv(Grid3 g, const float4* __restrict__ trig4, float4* __restrict__ dinv) {
  const int s = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.nodes()) return;
  int i, j, k;
  node_ijk(g, n, i, j, k);
  float3 d = make_float3(0.f, 0.f, 0.f);
  for (int ek = k - 1; ek <= k; ++ek) {
    if (ek < 0 || ek >= g.nz) continue;
    for (int ei = i - 1; ei <= i; ++ei) {
      if (ei < 0 || ei >= g.nx) continue;
      const Cm<float> C = coef<float>(trig4[(int64_t)s * g.cols() + (int64_t)ek * g.nx + ei]);
      for (int ej = j - 1; ej <= j; ++ej) {
        if (ej < 0 || ej >= g.ny) continue;
        const float3 c = corner_diag(C, g.h, i > ei ? 1.f : -1.f, j > ej ? 1.f : -1.f, k > ek ? 1.f : -1.f);
        d.x += c.x;
        d.y += c.y;
        d.z += c.z;
      }
    }
  }
  float4 r = make_float4(kOmega3 / d.x, kOmega3 / d.y, kOmega3 / d.z, 0.f);
  dinv[(int64_t)s * g.nodes() + n] = mask4(g, i, r);
}

// ---------------------------------------------------------------- operator

// Node storage: the FP32 vectors hold one float4 (u, v, w, 0) per node; the refinement
// iterate d holds float-float pairs, 8 floats per node (u.hi, u.lo, v.hi, v.lo, w.hi,
// w.lo, 0, 0), so that updating and applying K to it needs no double arithmetic.
__device__ __forceinline__ V3<float> load_v(const float4* x, int64_t n) {
  const float4 a = x[n];
  return V3<float>{a.x, a.y, a.z};
}
__device__ __forceinline__ V3<DF> load_v(const float* d, int64_t n) {
  const float4 a = reinterpret_cast<const float4*>(d)[2 * n], b = reinterpret_cast<const float4*>(d)[2 * n + 1];
  return V3<DF>{DF{a.x, a.y}, DF{a.z, a.w}, DF{b.x, b.y}};
}
__device__ __forceinline__ V3<double> load_d(const float* d, int64_t n) {
  const V3<DF> v = load_v(d, n);
  return V3<double>{(double)v.x.hi + (double)v.x.lo, (double)v.y.hi + (double)v.y.lo,
                    (double)v.z.hi + (double)v.z.lo};
}
__device__ __forceinline__ void add_node(float4* y, int64_t n, V3<float> f) {
  atomicAdd(y + n, make_float4(f.x, f.y, f.z, 0.f));
}
// float-float contributions are summed in double (the nodes' totals cancel to a small
// residual; each contribution keeps about 48 bits)
__device__ __forceinline__ void add_node(double* y, int64_t n, V3<DF> f) {
  atomicAdd(y + 4 * n, (double)f.x.hi + (double)f.x.lo);
  atomicAdd(y + 4 * n + 1, (double)f.y.hi + (double)f.y.lo);
  atomicAdd(y + 4 * n + 2, (double)f.z.hi + (double)f.z.lo);
}

__device__ __forceinline__ void add_node(double* y, int64_t n, V3<DFs> f) {
  add_node(y, n, V3<DF>{DF{f.x.hi, f.x.lo}, DF{f.y.hi, f.y.lo}, DF{f.z.hi, f.z.lo}});
}

__device__ __forceinline__ float dot_part(V3<float> a, V3<float> b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
__device__ __forceinline__ float dot_part(V3<DF> a, V3<DFs> b) { return 0.f; }

// One thread per element; y (zeroed by the caller) += K x over all DOFs. T: value type
// (float, or float-float for the refinement residual: the same FP32 stiffness, every
// intermediate kept to about 48 bits). With `boundary` only the last element column
// (i = nx - 1), which alone reaches the nodes on x = lx. With `energy` set, also
// energy[s] += x . K x as the sum of the element energies x_e . K_e x_e (the PCG's
// p . q when x vanishes on the prescribed DOFs).
template <typename T, bool ENERGY, typename X, typename Y>
__global__ void __launch_bounds__(128, sizeof(T) == 4 ? 0 : 3) k_apply(Grid3 g, const float4* __restrict__ trig4, const X* __restrict__ x,
                                               Y* __restrict__ y, const int* __restrict__ active, int boundary,
                                               double* __restrict__ energy) {
  const int s = blockIdx.y;
  if (active && !active[s]) return;   // uniform over the block
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  int i = 0, j = 0, k = 0;
  bool valid;
  if (boundary) {
    valid = e < (int64_t)g.ny * g.nz;
    i = g.nx - 1;
    j = (int)(e % g.ny);
    k = (int)(e / g.ny);
  } else {
    valid = e < g.elems();
    i = (int)(e % g.nx);
    const int64_t r = e / g.nx;
    j = (int)(r % g.ny);
    k = (int)(r / g.ny);
  }
  float en = 0.f;
  // a warp covers one x-row of elements when rows are whole multiples of 32 elements (and
  // then every lane of a warp is valid or none is)
  const bool row_warps = !boundary && g.nx % 32 == 0;
  if (valid) {
    const Cm<float> C = coef<float>(trig4[(int64_t)s * g.cols() + (int64_t)k * g.nx + i]);
    const int64_t base = (int64_t)s * g.nodes();
    V3<T> u[2][2][2];
    V3<typename Arith<T>::type> f[2][2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c) u[a][b][c] = load_v(x, base + node_of(g, i + a, j + b, k + c));
    element_apply<T, float, typename Arith<T>::type>(C, g.h, u, f);
    if (ENERGY) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int c = 0; c < 2; ++c) en += dot_part(u[a][b][c], f[a][b][c]);
    }
    if constexpr (sizeof(T) == 4) {
      if (row_warps) {
        // the warp holds 32 consecutive elements of one x-row: node (i + 1, ., .) gets this
        // lane's right-face forces and the next lane's left-face forces in one atomic
        const int lane = threadIdx.x & 31;
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int c = 0; c < 2; ++c) {
            V3<T> nxt;
            nxt.x = __shfl_down_sync(0xffffffffu, f[0][b][c].x, 1);
            nxt.y = __shfl_down_sync(0xffffffffu, f[0][b][c].y, 1);
            nxt.z = __shfl_down_sync(0xffffffffu, f[0][b][c].z, 1);
            const V3<T> right = lane < 31 ? f[1][b][c] + nxt : f[1][b][c];
            add_node(y, base + node_of(g, i + 1, j + b, k + c), right);
            if (lane == 0) add_node(y, base + node_of(g, i, j + b, k + c), f[0][b][c]);
          }
        valid = false;   // scattered
      }
    }
    if (valid) {
#pragma unroll
      for (int a = 0; a < 2; ++a)
#pragma unroll
        for (int b = 0; b < 2; ++b)
#pragma unroll
          for (int c = 0; c < 2; ++c) add_node(y, base + node_of(g, i + a, j + b, k + c), f[a][b][c]);
    }
  }
  if (ENERGY) {   // every thread of the block reaches the reduction
    const double t = block_sum((double)en);
    if (threadIdx.x == 0) atomicAdd(&energy[s], t);
  }
}

// ---------------------------------------------------------------- coarsest mesh

// One block per sample: the dense matrix of the coarsest mesh (prescribed DOFs
// replaced by identity rows and columns), assembled from K_e applied to unit vectors,
// then inverted in place by Gauss-Jordan elimination (SPD: no pivoting).
__global__ void __launch_bounds__(256) k_coarsest_setup(Grid3 g, const float4* __restrict__ trig4, float* __restrict__ ainv) {
  extern __shared__ float A[];   // [n][n]
  const int s = blockIdx.x;
  const int nn = (int)g.nodes(), n = 3 * nn;
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) A[t] = 0.f;
  __syncthreads();
  // thread per (element, local DOF): column of K_e
  const int ne = (int)g.elems();
  for (int t = threadIdx.x; t < ne * 24; t += blockDim.x) {
    const int e = t / 24, q = t % 24;
    const int i = e % g.nx, j = (e / g.nx) % g.ny, k = e / (g.nx * g.ny);
    const Cm<float> C = coef<float>(trig4[(int64_t)s * g.cols() + (int64_t)k * g.nx + i]);
    V3<float> u[2][2][2], f[2][2][2];
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c) u[a][b][c] = V3<float>{0.f, 0.f, 0.f};
    const int qa = q / 3, qc = q % 3;
    {
      V3<float>& uq = u[qa & 1][(qa >> 1) & 1][qa >> 2];
      if (qc == 0) uq.x = 1.f;
      if (qc == 1) uq.y = 1.f;
      if (qc == 2) uq.z = 1.f;
    }
    element_apply<float, float>(C, g.h, u, f);
    const int col = 3 * (int)node_of(g, i + (qa & 1), j + ((qa >> 1) & 1), k + (qa >> 2)) + qc;
#pragma unroll
    for (int a = 0; a < 2; ++a)
#pragma unroll
      for (int b = 0; b < 2; ++b)
#pragma unroll
        for (int c = 0; c < 2; ++c) {
          const int row = 3 * (int)node_of(g, i + a, j + b, k + c);
          atomicAdd(&A[(row + 0) * n + col], f[a][b][c].x);
          atomicAdd(&A[(row + 1) * n + col], f[a][b][c].y);
          atomicAdd(&A[(row + 2) * n + col], f[a][b][c].z);
        }
  }
  __syncthreads();
  // prescribed DOFs -> identity (warps take rows, lanes columns: no division per entry)
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = blockDim.x >> 5;
  auto prescribed = [&](int dof) {
    const int i = (dof / 3) % (g.nx + 1);
    return i == 0 || (i == g.nx && dof % 3 == 0);
  };
  for (int r = warp; r < n; r += nw) {
    const bool pr = prescribed(r);
    for (int c = lane; c < n; c += 32)
      if (pr || prescribed(c)) A[r * n + c] = (r == c) ? 1.f : 0.f;
  }
  __syncthreads();
  // Gauss-Jordan inversion in place
  for (int p = 0; p < n; ++p) {
    const float piv = 1.f / A[p * n + p];
    __syncthreads();
    for (int c = threadIdx.x; c < n; c += blockDim.x) A[p * n + c] = (c == p) ? piv : A[p * n + c] * piv;
    __syncthreads();
    for (int r = warp; r < n; r += nw) {
      if (r == p) continue;
      const float m = A[r * n + p];
      for (int c = lane; c < n; c += 32)
        if (c != p) A[r * n + c] -= m * A[p * n + c];
    }
    __syncthreads();
    for (int r = threadIdx.x; r < n; r += blockDim.x)
      if (r != p) A[r * n + p] = -A[r * n + p] * A[p * n + p];
    __syncthreads();
  }
  for (int t = threadIdx.x; t < n * n; t += blockDim.x) ainv[(int64_t)s * n * n + t] = A[t];
}

__global__ void k_coarsest_solve(Grid3 g, const float* __restrict__ ainv, const float4* __restrict__ b,
                                 float4* __restrict__ x, const int* __restrict__ active) {
  const int s = blockIdx.x;
  if (active && !active[s]) return;
  const int nn = (int)g.nodes(), n = 3 * nn;
  __shared__ float bs[kMaxCoarse3];
  for (int t = threadIdx.x; t < nn; t += blockDim.x) {
    const float4 v = b[(int64_t)s * nn + t];
    bs[3 * t] = v.x;
    bs[3 * t + 1] = v.y;
    bs[3 * t + 2] = v.z;
  }
  __syncthreads();
  const float* A = ainv + (int64_t)s * n * n;
  for (int r = threadIdx.x; r < n; r += blockDim.x) {
    float acc = 0.f;
    for (int c = 0; c < n; ++c) acc += A[(int64_t)r * n + c] * bs[c];
    reinterpret_cast<float*>(x + (int64_t)s * nn)[4 * (r / 3) + r % 3] = acc;
  }
}

// ---------------------------------------------------------------- V-cycle pieces

__global__ void k_smooth_first(Grid3 g, const float4* __restrict__ dinv, const float4* __restrict__ b,
                               float4* __restrict__ x, float4* __restrict__ t, const int* __restrict__ active) {
  const int s = blockIdx.y;
  if (active && !active[s]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.nodes()) return;
  const int64_t q = (int64_t)s * g.nodes() + n;
  const float4 d = dinv[q], bb = b[q];
  x[q] = make_float4(d.x * bb.x, d.y * bb.y, d.z * bb.z, 0.f);
  t[q] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// coarse node (I, J, K) = sum over fine (2I+a, 2J+b, 2K+c), a, b, c in {-1, 0, 1}, of
// w(a) w(b) w(c) (b_f - t_f) with w(0) = 1, w(+-1) = 1/2 (the transpose of trilinear
// prolongation); then the coarse pre-smoothing from zero and the zeroed apply target
__global__ void k_restrict(Grid3 f, const float4* __restrict__ bf, const float4* __restrict__ tf, Grid3 c,
                           const float4* __restrict__ dinv_c, float4* __restrict__ bc, float4* __restrict__ xc,
                           float4* __restrict__ tc, const int* __restrict__ active) {
  const int s = blockIdx.y;
  if (active && !active[s]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= c.nodes()) return;
  int I, J, K;
  node_ijk(c, n, I, J, K);
  const int64_t fb = (int64_t)s * f.nodes();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  for (int dk = -1; dk <= 1; ++dk) {
    const int k = 2 * K + dk;
    if (k < 0 || k > f.nz) continue;
    const float wk = dk ? 0.5f : 1.f;
    for (int dj = -1; dj <= 1; ++dj) {
      const int j = 2 * J + dj;
      if (j < 0 || j > f.ny) continue;
      const float wjk = wk * (dj ? 0.5f : 1.f);
      for (int di = -1; di <= 1; ++di) {
        const int i = 2 * I + di;
        if (i < 0 || i > f.nx) continue;
        const float w = wjk * (di ? 0.5f : 1.f);
        const int64_t q = fb + node_of(f, i, j, k);
        const float4 bb = bf[q], tt = tf[q];
        const float4 r = mask4(f, i, make_float4(bb.x - tt.x, bb.y - tt.y, bb.z - tt.z, 0.f));
        acc.x += w * r.x;
        acc.y += w * r.y;
        acc.z += w * r.z;
      }
    }
  }
  const int64_t q = (int64_t)s * c.nodes() + n;
  acc = mask4(c, I, acc);
  bc[q] = acc;
  const float4 d = dinv_c[q];
  xc[q] = make_float4(d.x * acc.x, d.y * acc.y, d.z * acc.z, 0.f);
  tc[q] = make_float4(0.f, 0.f, 0.f, 0.f);
}

// fine node += trilinear interpolation of the coarse correction; zeroes the apply target
__global__ void k_prolong(Grid3 f, const float4* __restrict__ xc, float4* __restrict__ xf, float4* __restrict__ tf,
                          const int* __restrict__ active) {
  const int s = blockIdx.y;
  if (active && !active[s]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= f.nodes()) return;
  int i, j, k;
  node_ijk(f, n, i, j, k);
  Grid3 c{f.nx / 2, f.ny / 2, f.nz / 2, f.nsamp, 2.f * f.h};
  const int64_t cb = (int64_t)s * c.nodes();
  float4 acc = make_float4(0.f, 0.f, 0.f, 0.f);
  const int i0 = i >> 1, i1 = (i + 1) >> 1, j0 = j >> 1, j1 = (j + 1) >> 1, k0 = k >> 1, k1 = (k + 1) >> 1;
  for (int kk = k0; kk <= k1; ++kk) {
    const float wk = (k0 == k1) ? 1.f : 0.5f;
    for (int jj = j0; jj <= j1; ++jj) {
      const float wjk = wk * ((j0 == j1) ? 1.f : 0.5f);
      for (int ii = i0; ii <= i1; ++ii) {
        const float w = wjk * ((i0 == i1) ? 1.f : 0.5f);
        const float4 v = xc[cb + node_of(c, ii, jj, kk)];
        acc.x += w * v.x;
        acc.y += w * v.y;
        acc.z += w * v.z;
      }
    }
  }
  const int64_t q = (int64_t)s * f.nodes() + n;
  const float4 x = xf[q];
  xf[q] = mask4(f, i, make_float4(x.x + acc.x, x.y + acc.y, x.z + acc.z, 0.f));
  tf[q] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_post(Grid3 g, const float4* __restrict__ dinv, const float4* __restrict__ b,
                       const float4* __restrict__ t, float4* __restrict__ x, double* __restrict__ rz,
                       const int* __restrict__ active) {
  const int s = blockIdx.y;
  if (active && !active[s]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double v = 0.0;
  if (n < g.nodes()) {
    int i, j, k;
    node_ijk(g, n, i, j, k);
    const int64_t q = (int64_t)s * g.nodes() + n;
    const float4 d = dinv[q], bb = b[q], tt = t[q], xx = x[q];
    const float4 z = mask4(g, i, make_float4(xx.x + d.x * (bb.x - tt.x), xx.y + d.y * (bb.y - tt.y),
                                             xx.z + d.z * (bb.z - tt.z), 0.f));
    x[q] = z;
    v = (double)(bb.x * z.x + bb.y * z.y + bb.z * z.z);
  }
  if (rz) {
    const double t = block_sum(v);
    if (threadIdx.x == 0) atomicAdd(&rz[s], t);
  }
}

// ---------------------------------------------------------------- PCG

__global__ void k_beta(State3 S, int n, int first) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || !S.active[s]) return;
  const double rz = S.rz[s];
  S.beta[s] = first ? 0.0 : rz / S.rz_old[s];
  S.rz_old[s] = rz;
  S.pq[s] = 0.0;
}

__global__ void k_update_p(Grid3 g, State3 S, const float4* __restrict__ z, float4* __restrict__ p,
                           float4* __restrict__ q) {
  const int s = blockIdx.y;
  if (!S.active[s]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.nodes()) return;
  const float b = (float)S.beta[s];
  const int64_t t = (int64_t)s * g.nodes() + n;
  const float4 zz = z[t], pp = p[t];
  p[t] = make_float4(zz.x + b * pp.x, zz.y + b * pp.y, zz.z + b * pp.z, 0.f);
  q[t] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void k_dot_pq(Grid3 g, State3 S, const float4* __restrict__ p, const float4* __restrict__ q) {
  const int s = blockIdx.y;
  if (!S.active[s]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double v = 0.0;
  if (n < g.nodes()) {
    int i, j, k;
    node_ijk(g, n, i, j, k);
    const int64_t t = (int64_t)s * g.nodes() + n;
    const float4 pp = p[t], qq = mask4(g, i, q[t]);
    v = (double)(pp.x * qq.x + pp.y * qq.y + pp.z * qq.z);
  }
  const double t = block_sum(v);
  if (threadIdx.x == 0) atomicAdd(&S.pq[s], t);
}

__global__ void k_alpha(State3 S, int n) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || !S.active[s]) return;
  const double pq = S.pq[s], rz = S.rz_old[s];
  if (!(pq > 0.0) || !(rz > 0.0)) {   // breakdown
    S.active[s] = 0;
    S.alpha[s] = 0.0;
    return;
  }
  S.alpha[s] = rz / pq;
  S.rr[s] = 0.0;
  S.rz[s] = 0.0;
}

__global__ void k_update_xr(Grid3 g, State3 S, const float4* __restrict__ p, const float4* __restrict__ q,
                            float4* __restrict__ x, float4* __restrict__ r) {
  const int s = blockIdx.y;
  if (!S.active[s]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double v = 0.0;
  if (n < g.nodes()) {
    int i, j, k;
    node_ijk(g, n, i, j, k);
    const float a = (float)S.alpha[s];
    const int64_t t = (int64_t)s * g.nodes() + n;
    const float4 pp = p[t], qq = mask4(g, i, q[t]), xx = x[t], rr = r[t];
    x[t] = make_float4(xx.x + a * pp.x, xx.y + a * pp.y, xx.z + a * pp.z, 0.f);
    const float4 rn = make_float4(rr.x - a * qq.x, rr.y - a * qq.y, rr.z - a * qq.z, 0.f);
    r[t] = rn;
    v = (double)rn.x * rn.x + (double)rn.y * rn.y + (double)rn.z * rn.z;
  }
  const double t = block_sum(v);
  if (threadIdx.x == 0) atomicAdd(&S.rr[s], t);
}

__global__ void k_check(State3 S, int n, int it, int max_iter, int slot) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || !S.active[s]) return;
  S.iters[s] += 1;
  if (S.rr[s] <= S.tol2[s] * S.rr0[s]) {
    S.active[s] = 0;
    return;
  }
  if (it + 1 >= max_iter) {
    S.active[s] = 0;
    S.status[s] = 1;   // not converged
    return;
  }
  atomicAdd(&S.count[slot], 1);
}

// ---------------------------------------------------------------- refinement and outputs

// d = the lifting (u = -shortening on x = lx, as the float-float pair (hi, lo)); xl its FP32 copy
__global__ void k_lift(Grid3 g, float u_hi, float u_lo, float* __restrict__ d, float4* __restrict__ xl) {
  const int s = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.nodes()) return;
  const int i = (int)(n % (g.nx + 1));
  const int64_t q = (int64_t)s * g.nodes() + n;
  const bool end = i == g.nx;
  float4* d4 = reinterpret_cast<float4*>(d);
  d4[2 * q] = make_float4(end ? u_hi : 0.f, end ? u_lo : 0.f, 0.f, 0.f);
  d4[2 * q + 1] = make_float4(0.f, 0.f, 0.f, 0.f);
  xl[q] = make_float4(end ? u_hi : 0.f, 0.f, 0.f, 0.f);
}

// r = -(K x_lift) on free DOFs; ||r||^2 = ||f||^2
__global__ void k_lift_resid(Grid3 g, State3 S, const float4* __restrict__ t, float4* __restrict__ r) {
  const int s = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double v = 0.0;
  if (n < g.nodes()) {
    const int i = (int)(n % (g.nx + 1));
    const int64_t q = (int64_t)s * g.nodes() + n;
    const float4 tt = t[q];
    const float4 rr = mask4(g, i, make_float4(-tt.x, -tt.y, -tt.z, 0.f));
    r[q] = rr;
    v = (double)rr.x * rr.x + (double)rr.y * rr.y + (double)rr.z * rr.z;
  }
  const double tsum = block_sum(v);
  if (threadIdx.x == 0) {
    atomicAdd(&S.rrf[s], tsum);
    atomicAdd(&S.rr[s], tsum);
  }
}

// float-float d += float x (TwoSum of the heads, the tail added, renormalised)
__device__ __forceinline__ DF df_add(DF a, float x) {
  DF t = mlmc::two_sum(a.hi, x);
  t.lo = __fadd_rn(t.lo, a.lo);
  return mlmc::fast_two_sum(t.hi, t.lo);
}

__global__ void k_update_d(Grid3 g, State3 S, const float4* __restrict__ x, float* __restrict__ d) {
  const int s = blockIdx.y;
  if (!S.outer_active[s]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (n >= g.nodes()) return;
  const int64_t q = (int64_t)s * g.nodes() + n;
  const float4 xx = x[q];
  V3<DF> v = load_v(d, q);
  v.x = df_add(v.x, xx.x);
  v.y = df_add(v.y, xx.y);
  v.z = df_add(v.z, xx.z);
  float4* d4 = reinterpret_cast<float4*>(d);
  d4[2 * q] = make_float4(v.x.hi, v.x.lo, v.y.hi, v.y.lo);
  d4[2 * q + 1] = make_float4(v.z.hi, v.z.lo, 0.f, 0.f);
}

// kd = K d (double sums of float-float contributions): r = -(K d) on free DOFs
// (float), ||r||^2 (double)
__global__ void k_resid_exact(Grid3 g, State3 S, const double* __restrict__ kd, float4* __restrict__ r) {
  const int s = blockIdx.y;
  if (!S.outer_active[s]) return;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double rr = 0.0;
  if (n < g.nodes()) {
    const int i = (int)(n % (g.nx + 1));
    const int64_t q = (int64_t)s * g.nodes() + n;
    const double* k4 = kd + 4 * q;
    double rx = -k4[0], ry = -k4[1], rzv = -k4[2];
    if (i == 0) rx = ry = rzv = 0.0;
    if (i == g.nx) rx = 0.0;
    const float4 rf = make_float4((float)rx, (float)ry, (float)rzv, 0.f);
    r[q] = rf;
    rr = (double)rf.x * rf.x + (double)rf.y * rf.y + (double)rf.z * rf.z;
  }
  const double a = block_sum(rr);
  if (threadIdx.x == 0) atomicAdd(&S.rr[s], a);
}

// final pass: the reaction -sum over x = lx of (K d)_u (kd from the last element column
// only, complete on those nodes) and d_F . r_F with the latest residual r (zero on the
// prescribed DOFs)
__global__ void k_final(Grid3 g, State3 S, const double* __restrict__ kd, const float* __restrict__ d,
                        const float4* __restrict__ r) {
  const int s = blockIdx.y;
  const int64_t n = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double re = 0.0, dr = 0.0;
  if (n < g.nodes()) {
    const int i = (int)(n % (g.nx + 1));
    const int64_t q = (int64_t)s * g.nodes() + n;
    if (i == g.nx) re = -kd[4 * q];
    const float4 rr = r[q];
    const V3<double> dd = load_d(d, q);
    dr = dd.x * rr.x + dd.y * rr.y + dd.z * rr.z;
  }
  const double a = block_sum(re);
  if (threadIdx.x == 0) atomicAdd(&S.react[s], a);
  const double b = block_sum(dr);
  if (threadIdx.x == 0) atomicAdd(&S.dr[s], b);
}

// per sample: start an inner solve with tolerance max(floor, 0.5 rtol ||f|| / ||r||)
__global__ void k_inner_begin(State3 S, int n, double rtol, double floor_tol) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int on = S.outer_active[s];
  S.active[s] = on;
  if (!on) return;
  const double rr = S.rr[s];
  S.rr0[s] = rr;
  const double t = fmax(floor_tol, 0.5 * rtol * sqrt(S.rrf[s] / fmax(rr, 1e-300)));
  S.tol2[s] = fmin(t, 0.5) * fmin(t, 0.5);
  S.rz[s] = 0.0;
}

__global__ void k_outer_check(State3 S, int n, double rtol, int* outer_count) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || !S.outer_active[s]) return;
  if (S.status[s] != 0 || S.rr[s] <= rtol * rtol * S.rrf[s]) {
    S.outer_active[s] = 0;
    return;
  }
  atomicAdd(outer_count, 1);
}

// max over elements with centroid x in [x0, x1] of max(0, -a1 . sigma a1) at the
// centroid, a1 = (cos t, 0, -sin t) the rotated fibre direction
__global__ void k_stress(Grid3 g, State3 S, const float4* __restrict__ trig4, const float* __restrict__ d,
                         double x0, double x1) {
  const int s = blockIdx.y;
  const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  double best = 0.0;
  if (e < g.elems()) {
    const int i = (int)(e % g.nx);
    const int64_t r = e / g.nx;
    const int j = (int)(r % g.ny), k = (int)(r / g.ny);
    const double xc = (i + 0.5) * (double)g.h;
    if (xc >= x0 && xc <= x1) {
      const float4 t = trig4[(int64_t)s * g.cols() + (int64_t)k * g.nx + i];
      const Cm<double> C = coef<double>(t);
      const int64_t base = (int64_t)s * g.nodes();
      // centroid gradient: mean of the four edge differences per direction, / h
      V3<double> gx{0, 0, 0}, gy{0, 0, 0}, gz{0, 0, 0};
      for (int a = 0; a < 2; ++a)
        for (int b = 0; b < 2; ++b) {
          gx = gx + (load_d(d, base + node_of(g, i + 1, j + a, k + b)) -
                     load_d(d, base + node_of(g, i, j + a, k + b)));
          gy = gy + (load_d(d, base + node_of(g, i + a, j + 1, k + b)) -
                     load_d(d, base + node_of(g, i + a, j, k + b)));
          gz = gz + (load_d(d, base + node_of(g, i + a, j + b, k + 1)) -
                     load_d(d, base + node_of(g, i + a, j + b, k)));
        }
      const double f = 0.25 / (double)g.h;
      gx = f * gx;
      gy = f * gy;
      gz = f * gz;
      const double e1 = gx.x, e2 = gy.y, e3 = gz.z, e4 = gz.y + gy.z, e5 = gz.x + gx.z, e6 = gy.x + gx.y;
      const double s1 = C.c11 * e1 + C.c12 * e2 + C.c13 * e3 + C.c15 * e5;
      const double s3 = C.c13 * e1 + C.c23 * e2 + C.c33 * e3 + C.c35 * e5;
      const double s5 = C.c15 * e1 + C.c25 * e2 + C.c35 * e3 + C.c55 * e5;
      (void)e4;
      (void)e6;
      // cos t, sin t from (cos 2t, sin 2t), |t| < pi / 2
      const double ct = sqrt(fmax(0.5 * (1.0 + (double)t.x), 0.0));
      const double st = ct > 0.0 ? (double)t.y / (2.0 * ct) : 1.0;
      const double sf = ct * ct * s1 + st * st * s3 - 2.0 * ct * st * s5;
      best = fmax(0.0, -sf);
    }
  }
  // block max, then atomic max on the (non-negative) bit pattern
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) best = fmax(best, __shfl_xor_sync(0xffffffffu, best, o));
  if ((threadIdx.x & 31) == 0 && best > 0.0)
    atomicMax(reinterpret_cast<unsigned long long*>(&S.stress[s]), (unsigned long long)__double_as_longlong(best));
}

__global__ void k_qoi(State3 S, int n, double shortening, double* q, int* status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  q[2 * s] = S.react[s] - S.dr[s] / shortening;
  q[2 * s + 1] = S.stress[s];
  // MLMC_ERR_NOT_CONVERGED: an inner solve hit its cap, or refinement steps ran out
  status[s] = (S.status[s] || S.outer_active[s]) ? 4 : 0;
}

__global__ void k_combine_status(int* a, const int* b, int n) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n && b[s] != 0) a[s] = b[s];
}

__global__ void k_zero4(float4* v, int64_t n) {
  const int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (t < n) v[t] = make_float4(0.f, 0.f, 0.f, 0.f);
}

inline unsigned blocks(int64_t n, int bs) { return (unsigned)((n + bs - 1) / bs); }

}  // namespace

cudaError_t set_harmonics(const Harmonics& H) { return cudaMemcpyToSymbol(g_harm, &H, sizeof(H)); }

cudaError_t launch_expand_trig(const float* trig2, int64_t n, float* trig4, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_expand_trig<<<blocks(n, 256), 256, 0, st>>>(trig2, n, trig4);
  return cudaGetLastError();
}
cudaError_t launch_average_trig(const Grid3& f, const float* tf, float* tc, cudaStream_t st) {
  const int n = (f.nx / 2) * (f.nz / 2);
  k_average_trig<<<dim3(blocks(n, 128), f.nsamp), 128, 0, st>>>(f, reinterpret_cast<const float4*>(tf),
                                                                  reinterpret_cast<float4*>(tc));
  return cudaGetLastError();
}
cudaError_t launch_dinv(const Grid3& g, const float* trig4, float4* dinv, cudaStream_t st) {
  k_dinv<<<dim3(blocks(g.nodes(), 128), g.nsamp), 128, 0, st>>>(g, reinterpret_cast<const float4*>(trig4), dinv);
  return cudaGetLastError();
}
cudaError_t launch_apply(const Grid3& g, const float* trig4, const float4* x, float4* y, const int* active,
                         cudaStream_t st, double* energy) {
  const dim3 grid(blocks(g.elems(), 128), g.nsamp);
  if (energy)
    k_apply<float, true><<<grid, 128, 0, st>>>(g, reinterpret_cast<const float4*>(trig4), x, y, active, 0, energy);
  else
    k_apply<float, false><<<grid, 128, 0, st>>>(g, reinterpret_cast<const float4*>(trig4), x, y, active, 0, nullptr);
  return cudaGetLastError();
}
cudaError_t launch_apply_df(const Grid3& g, const float* trig4, const float* d, double* y, const int* active,
                            bool boundary, cudaStream_t st) {
  const int64_t n = boundary ? (int64_t)g.ny * g.nz : g.elems();
  k_apply<DF, false><<<dim3(blocks(n, 128), g.nsamp), 128, 0, st>>>(g, reinterpret_cast<const float4*>(trig4), d, y, active,
                                                             boundary ? 1 : 0, nullptr);
  return cudaGetLastError();
}
cudaError_t launch_coarsest_setup(const Grid3& g, const float* trig4, float* ainv, cudaStream_t st) {
  const int n = 3 * (int)g.nodes();
  if (n > kMaxCoarse3) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float) * n * n;
  cudaError_t e = cudaFuncSetAttribute(k_coarsest_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_coarsest_setup<<<g.nsamp, 256, smem, st>>>(g, reinterpret_cast<const float4*>(trig4), ainv);
  return cudaGetLastError();
}
cudaError_t launch_coarsest_solve(const Grid3& g, const float* ainv, const float4* b, float4* x, const int* active,
                                  cudaStream_t st) {
  k_coarsest_solve<<<g.nsamp, 192, 0, st>>>(g, ainv, b, x, active);
  return cudaGetLastError();
}
cudaError_t launch_smooth_first(const Grid3& g, const float4* dinv, const float4* b, float4* x, float4* t,
                                const int* active, cudaStream_t st) {
  k_smooth_first<<<dim3(blocks(g.nodes(), 256), g.nsamp), 256, 0, st>>>(g, dinv, b, x, t, active);
  return cudaGetLastError();
}
cudaError_t launch_restrict(const Grid3& f, const float4* bf, const float4* tf, const Grid3& c, const float4* dinv_c,
                            float4* bc, float4* xc, float4* tc, const int* active, cudaStream_t st) {
  k_restrict<<<dim3(blocks(c.nodes(), 128), c.nsamp), 128, 0, st>>>(f, bf, tf, c, dinv_c, bc, xc, tc, active);
  return cudaGetLastError();
}
cudaError_t launch_prolong(const Grid3& f, const float4* xc, float4* xf, float4* tf, const int* active,
                           cudaStream_t st) {
  k_prolong<<<dim3(blocks(f.nodes(), 128), f.nsamp), 128, 0, st>>>(f, xc, xf, tf, active);
  return cudaGetLastError();
}
cudaError_t launch_post(const Grid3& g, const float4* dinv, const float4* b, const float4* t, float4* x, double* rz,
                        const int* active, cudaStream_t st) {
  k_post<<<dim3(blocks(g.nodes(), 256), g.nsamp), 256, 0, st>>>(g, dinv, b, t, x, rz, active);
  return cudaGetLastError();
}
cudaError_t launch_beta(const State3& S, int n, int first, cudaStream_t st) {
  k_beta<<<blocks(n, 128), 128, 0, st>>>(S, n, first);
  return cudaGetLastError();
}
cudaError_t launch_update_p(const Grid3& g, const State3& S, const float4* z, float4* p, float4* q, cudaStream_t st) {
  k_update_p<<<dim3(blocks(g.nodes(), 256), g.nsamp), 256, 0, st>>>(g, S, z, p, q);
  return cudaGetLastError();
}
cudaError_t launch_dot_pq(const Grid3& g, const State3& S, const float4* p, const float4* q, cudaStream_t st) {
  k_dot_pq<<<dim3(blocks(g.nodes(), 256), g.nsamp), 256, 0, st>>>(g, S, p, q);
  return cudaGetLastError();
}
cudaError_t launch_alpha(const State3& S, int n, cudaStream_t st) {
  k_alpha<<<blocks(n, 128), 128, 0, st>>>(S, n);
  return cudaGetLastError();
}
cudaError_t launch_update_xr(const Grid3& g, const State3& S, const float4* p, const float4* q, float4* x, float4* r,
                             cudaStream_t st) {
  k_update_xr<<<dim3(blocks(g.nodes(), 256), g.nsamp), 256, 0, st>>>(g, S, p, q, x, r);
  return cudaGetLastError();
}
cudaError_t launch_check(const State3& S, int n, int it, int max_iter, int slot, cudaStream_t st) {
  k_check<<<blocks(n, 128), 128, 0, st>>>(S, n, it, max_iter, slot);
  return cudaGetLastError();
}
cudaError_t launch_lift(const Grid3& g, double shortening, float* d, float4* xl, cudaStream_t st) {
  const float hi = (float)(-shortening), lo = (float)(-shortening - (double)hi);
  k_lift<<<dim3(blocks(g.nodes(), 256), g.nsamp), 256, 0, st>>>(g, hi, lo, d, xl);
  return cudaGetLastError();
}
cudaError_t launch_lift_resid(const Grid3& g, const State3& S, const float4* t, float4* r, cudaStream_t st) {
  k_lift_resid<<<dim3(blocks(g.nodes(), 256), g.nsamp), 256, 0, st>>>(g, S, t, r);
  return cudaGetLastError();
}
cudaError_t launch_update_d(const Grid3& g, const State3& S, const float4* x, float* d, cudaStream_t st) {
  k_update_d<<<dim3(blocks(g.nodes(), 256), g.nsamp), 256, 0, st>>>(g, S, x, d);
  return cudaGetLastError();
}
cudaError_t launch_resid_exact(const Grid3& g, const State3& S, const double* kd, float4* r, cudaStream_t st) {
  k_resid_exact<<<dim3(blocks(g.nodes(), 256), g.nsamp), 256, 0, st>>>(g, S, kd, r);
  return cudaGetLastError();
}
cudaError_t launch_final(const Grid3& g, const State3& S, const double* kd, const float* d, const float4* r,
                         cudaStream_t st) {
  k_final<<<dim3(blocks(g.nodes(), 256), g.nsamp), 256, 0, st>>>(g, S, kd, d, r);
  return cudaGetLastError();
}
cudaError_t launch_inner_begin(const State3& S, int n, double rtol, double floor_tol, int, cudaStream_t st) {
  k_inner_begin<<<blocks(n, 128), 128, 0, st>>>(S, n, rtol, floor_tol);
  return cudaGetLastError();
}
cudaError_t launch_outer_check(const State3& S, int n, double rtol, int* outer_count, cudaStream_t st) {
  k_outer_check<<<blocks(n, 128), 128, 0, st>>>(S, n, rtol, outer_count);
  return cudaGetLastError();
}
cudaError_t launch_stress(const Grid3& g, const State3& S, const float* trig4, const float* d, double x0, double x1,
                          cudaStream_t st) {
  k_stress<<<dim3(blocks(g.elems(), 128), g.nsamp), 128, 0, st>>>(g, S, reinterpret_cast<const float4*>(trig4), d,
                                                                   x0, x1);
  return cudaGetLastError();
}
cudaError_t launch_qoi(const State3& S, int n, double shortening, double* q, int* status, cudaStream_t st) {
  k_qoi<<<blocks(n, 128), 128, 0, st>>>(S, n, shortening, q, status);
  return cudaGetLastError();
}
cudaError_t launch_combine_status(int* a, const int* b, int n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_combine_status<<<blocks(n, 128), 128, 0, st>>>(a, b, n);
  return cudaGetLastError();
}
cudaError_t launch_zero4(float4* v, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_zero4<<<blocks(n, 256), 256, 0, st>>>(v, n);
  return cudaGetLastError();
}

}  // namespace mlmc3
