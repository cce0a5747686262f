// Cosserat engine kernels (Sec. 3.1 - 3.2): stencil assembly from the per-element trig
// values, Galerkin coarse operators, the V(1,1) block-Jacobi multigrid cycle, the FP32
// correction CG, the FP64 refinement residual and the strength / reaction quantities.
//
// Every kernel takes a Views table: the batches of up to kMaxViews meshes of one call,
// each with its own first block, so that all meshes advance in one launch per step.
// Threads map to (sample, node) of the view's level in sample-major order.
#include <cuda_runtime.h>

#include <type_traits>

#include "cosserat.cuh"

namespace mlmcc {

namespace {

__device__ __forceinline__ int view_of(const Views& V) {
  int v = 0;
#pragma unroll 1
  for (int k = 1; k < V.nv; ++k)
    if ((int)blockIdx.x >= V.v[k].blk0) v = k;
  return v;
}

// bit 0: u prescribed (x = 0 or x = L), bit 1: v prescribed (y = 0 or y = L)
__device__ __forceinline__ int dmask(int i, int j, int n) {
  return ((i == 0 || i == n) ? 1 : 0) | ((j == 0 || j == n) ? 2 : 0);
}

// forward block offsets: E, N, NE, NW
constexpr int kE = 6, kN = 15, kNE = 24, kNW = 33;

// Coefficients K0 .. K0 + NK - 1 of node q from the float4 groups of one sample's
// stencil (group g of node q at A[g * N + q]); constant indices after unrolling.
template <int K0, int NK>
__device__ __forceinline__ void load_coef(const float4* __restrict__ A, int N, int q, float (&c)[NK]) {
  constexpr int g0 = K0 / 4, g1 = (K0 + NK - 1) / 4;
#pragma unroll
  for (int g = g0; g <= g1; ++g) {
    const float4 v = A[(size_t)g * N + q];
    const float e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int l = 0; l < 4; ++l) {
      const int k = 4 * g + l - K0;
      if (k >= 0 && k < NK) c[k] = e[l];
    }
  }
}

template <int K0>
__device__ __forceinline__ void fwd_blk(const float (&a)[kStencil], float4 v, float y[3]) {
#pragma unroll
  for (int r = 0; r < 3; ++r) y[r] += a[K0 + 3 * r] * v.x + a[K0 + 3 * r + 1] * v.y + a[K0 + 3 * r + 2] * v.z;
}
template <int K0>
__device__ __forceinline__ void bwd_blk(const float4* __restrict__ A, int N, int q, float4 v, float y[3]) {
  float b[9];
  load_coef<K0, 9>(A, N, q, b);
#pragma unroll
  for (int r = 0; r < 3; ++r) y[r] += b[r] * v.x + b[3 + r] * v.y + b[6 + r] * v.z;
}

// y += (stencil row of node (i, j)) * x, x per node as float4 (u, v, theta, -) from xf(q).
// A: one sample's float4 coefficient groups.
template <class XF>
__device__ __forceinline__ void apply_node(const float4* __restrict__ A, int N, int n, int i, int j, XF xf,
                                           float y[3]) {
  const int p = j * (n + 1) + i;
  const int w = n + 1;
  float a[kStencil];
  load_coef<0, kStencil>(A, N, p, a);
  {
    const float4 v = xf(p);
    y[0] += a[0] * v.x + a[1] * v.y + a[2] * v.z;
    y[1] += a[1] * v.x + a[3] * v.y + a[4] * v.z;
    y[2] += a[2] * v.x + a[4] * v.y + a[5] * v.z;
  }
  if (i < n) fwd_blk<kE>(a, xf(p + 1), y);
  if (j < n) {
    fwd_blk<kN>(a, xf(p + w), y);
    if (i < n) fwd_blk<kNE>(a, xf(p + w + 1), y);
    if (i > 0) fwd_blk<kNW>(a, xf(p + w - 1), y);
  }
  if (i > 0) bwd_blk<kE>(A, N, p - 1, xf(p - 1), y);
  if (j > 0) {
    bwd_blk<kN>(A, N, p - w, xf(p - w), y);
    if (i > 0) bwd_blk<kNE>(A, N, p - w - 1, xf(p - w - 1), y);
    if (i < n) bwd_blk<kNW>(A, N, p - w + 1, xf(p - w + 1), y);
  }
}

// 3 x 3 block from node (i, j) to (i + ox, j + oy) (both inside), [row][column]
__device__ __forceinline__ void block_of(const float4* __restrict__ A, int N, int n, int i, int j, int ox, int oy,
                                         float out[9]) {
  const int p = j * (n + 1) + i;
  const int w = n + 1;
  if (ox == 0 && oy == 0) {
    float c[6];
    load_coef<0, 6>(A, N, p, c);
    out[0] = c[0];
    out[1] = out[3] = c[1];
    out[2] = out[6] = c[2];
    out[4] = c[3];
    out[5] = out[7] = c[4];
    out[8] = c[5];
    return;
  }
  float b[9];
  bool tr;
  if (oy == 0) {
    tr = ox < 0;
    load_coef<kE, 9>(A, N, tr ? p - 1 : p, b);
  } else if (ox == 0) {
    tr = oy < 0;
    load_coef<kN, 9>(A, N, tr ? p - w : p, b);
  } else if (ox == oy) {
    tr = ox < 0;
    load_coef<kNE, 9>(A, N, tr ? p - w - 1 : p, b);
  } else {
    tr = oy < 0;   // (+1, -1): the NW block of the south-east node, transposed
    load_coef<kNW, 9>(A, N, tr ? p - w + 1 : p, b);
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int c = 0; c < 3; ++c) out[3 * a + c] = tr ? b[3 * c + a] : b[3 * a + c];
}

// coefficient k of node p in a sample's float4 groups, as a plain float address
__device__ __forceinline__ float* coef_at(float4* A, int N, int k, int p) {
  return reinterpret_cast<float*>(A + (size_t)(k >> 2) * N + p) + (k & 3);
}

// inverse of a symmetric 3 x 3 (upper triangle a00 a01 a02 a11 a12 a22), upper triangle out
template <typename T>
__device__ __forceinline__ void inv_sym3(const T m[6], T out[6]) {
  const T c00 = m[3] * m[5] - m[4] * m[4];
  const T c01 = m[2] * m[4] - m[1] * m[5];
  const T c02 = m[1] * m[4] - m[2] * m[3];
  const T det = m[0] * c00 + m[1] * c01 + m[2] * c02;
  const T id = (T)1 / det;
  out[0] = c00 * id;
  out[1] = c01 * id;
  out[2] = c02 * id;
  out[3] = (m[0] * m[5] - m[2] * m[2]) * id;
  out[4] = (m[1] * m[2] - m[0] * m[4]) * id;
  out[5] = (m[0] * m[3] - m[1] * m[1]) * id;
}

// Sum of v over the lanes of each sample (s < 0: no contribution) into *addr(s).
// Lanes of one sample are contiguous; all 32 lanes must call.
template <class Addr>
__device__ __forceinline__ void warp_add_by_sample(double v, int s, Addr addr) {
  const int lane = threadIdx.x & 31;
  const int s0 = __shfl_sync(0xffffffffu, s, 0);
  if (__all_sync(0xffffffffu, s == s0)) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0 && s0 >= 0) atomicAdd(addr(s0), v);
  } else if (s >= 0) {
    atomicAdd(addr(s), v);
  }
}

// max of v >= 0 per sample, as the ordered bit pattern of a non-negative double
template <class Addr>
__device__ __forceinline__ void warp_max_by_sample(double v, int s, Addr addr) {
  const int lane = threadIdx.x & 31;
  const int s0 = __shfl_sync(0xffffffffu, s, 0);
  if (__all_sync(0xffffffffu, s == s0)) {
#pragma unroll
    for (int o = 16; o; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
    if (lane == 0 && s0 >= 0)
      atomicMax((unsigned long long*)addr(s0), (unsigned long long)__double_as_longlong(v));
  } else if (s >= 0) {
    atomicMax((unsigned long long*)addr(s), (unsigned long long)__double_as_longlong(v));
  }
}

// (view, sample, node) of this thread; ok = false past the view's items
struct Item {
  int v, s, p;
  bool ok;
};
__device__ __forceinline__ Item item_of(const Views& V, int per_sample) {
  Item it;
  it.v = view_of(V);
  const View& W = V.v[it.v];
  const int k = (blockIdx.x - W.blk0) * blockDim.x + threadIdx.x;
  it.ok = k < W.items;
  it.s = it.ok ? k / per_sample : -1;
  it.p = it.ok ? k - it.s * per_sample : 0;
  return it;
}



// ---------------------------------------------------------------- float-float arithmetic
//
// A value is hi + lo with |lo| <= ulp(hi) / 2 (about 48 significant bits). GB300's FP64
// rate is a small fraction of its FP32 rate, so the parts that need more than FP32 (the
// stencil of the refinement residual, the residual itself, the KL synthesis) run on the
// FP32 pipes with the error-free transformations of Dekker and Knuth. Every operation
// uses explicitly rounded intrinsics, so no contraction changes them.
struct ff {
  float hi, lo;
};
__device__ __forceinline__ ff ff_of(double a) {
  const float h = __double2float_rn(a);
  return {h, __double2float_rn(a - (double)h)};
}
__device__ __forceinline__ double ff_dbl(ff a) { return (double)a.hi + (double)a.lo; }
// acc += a * b
__device__ __forceinline__ void ff_fma(ff& acc, ff a, ff b) {
  const float p = __fmul_rn(a.hi, b.hi);
  float e = __fmaf_rn(a.hi, b.hi, -p);          // exact error of the product
  e = __fmaf_rn(a.hi, b.lo, e);
  e = __fmaf_rn(a.lo, b.hi, e);
  const float s = __fadd_rn(acc.hi, p);          // two-sum of acc.hi and p
  const float bb = __fsub_rn(s, acc.hi);
  const float err = __fadd_rn(__fsub_rn(acc.hi, __fsub_rn(s, bb)), __fsub_rn(p, bb));
  const float t = __fadd_rn(err, __fadd_rn(e, acc.lo));
  const float hi = __fadd_rn(s, t);              // renormalise
  acc.lo = __fsub_rn(t, __fsub_rn(hi, s));
  acc.hi = hi;
}
// acc += a * b with b a plain float
__device__ __forceinline__ void ff_fma(ff& acc, ff a, float b) { ff_fma(acc, a, ff{b, 0.f}); }

// y += (stencil row of node (i, j)) * x in float-float; the stencil is (Ah, Al), both
// float4 coefficient groups of one sample; xf(q, v[3]) gives x at node q.
template <class XF>
__device__ __forceinline__ void apply_node_ff(const float4* __restrict__ Ah, const float4* __restrict__ Al, int N,
                                              int n, int i, int j, XF xf, ff y[3]) {
  const int p = j * (n + 1) + i;
  const int w = n + 1;
  {
    float h[kStencil], l[kStencil];
    load_coef<0, kStencil>(Ah, N, p, h);
    load_coef<0, kStencil>(Al, N, p, l);
    ff v[3];
    xf(p, v);
    const int sym[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) ff_fma(y[r], ff{h[sym[r][c]], l[sym[r][c]]}, v[c]);
    auto fwd = [&](int k0, int q) {
      ff u[3];
      xf(q, u);
#pragma unroll
      for (int r = 0; r < 3; ++r)
#pragma unroll
        for (int c = 0; c < 3; ++c) ff_fma(y[r], ff{h[k0 + 3 * r + c], l[k0 + 3 * r + c]}, u[c]);
    };
    if (i < n) fwd(kE, p + 1);
    if (j < n) {
      fwd(kN, p + w);
      if (i < n) fwd(kNE, p + w + 1);
      if (i > 0) fwd(kNW, p + w - 1);
    }
  }
  auto bwd = [&](auto K0, int q) {
    constexpr int k0 = decltype(K0)::value;
    float h[9], l[9];
    load_coef<k0, 9>(Ah, N, q, h);
    load_coef<k0, 9>(Al, N, q, l);
    ff u[3];
    xf(q, u);
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) ff_fma(y[r], ff{h[3 * c + r], l[3 * c + r]}, u[c]);
  };
  if (i > 0) bwd(std::integral_constant<int, kE>{}, p - 1);
  if (j > 0) {
    bwd(std::integral_constant<int, kN>{}, p - w);
    if (i > 0) bwd(std::integral_constant<int, kNE>{}, p - w - 1);
    if (i < n) bwd(std::integral_constant<int, kNW>{}, p - w + 1);
  }
}

// KL synthesis phi[s][e] = sum_k B[e][k] xi[s][k] in float-float: tiles of 128 elements
// x 16 samples, 16-term slices of both operands in shared memory; each thread 8
// elements (strided by 16) of one sample. Writes (cos 2 phi, sin 2 phi, cos 4 phi,
// sin 4 phi) as float-float pairs when trig, else phi in double.
constexpr int kSynE = 128, kSynS = 16, kSynK = 16;
__global__ void __launch_bounds__(256) k_synth_ff(const double* __restrict__ xi, const float* __restrict__ Bh,
                                                  const float* __restrict__ Bl, int S, int n_el, int K,
                                                  void* __restrict__ out, bool trig) {
  __shared__ float sBh[kSynK][kSynE], sBl[kSynK][kSynE];
  __shared__ float sXh[kSynK][kSynS + 1], sXl[kSynK][kSynS + 1];
  const int tid = threadIdx.x;
  const int ls = tid >> 4, le = tid & 15;
  const int e0 = blockIdx.x * kSynE, s0 = blockIdx.y * kSynS;
  ff acc[8];
#pragma unroll
  for (int a = 0; a < 8; ++a) acc[a] = ff{0.f, 0.f};
  for (int k0 = 0; k0 < K; k0 += kSynK) {
#pragma unroll
    for (int r = 0; r < (kSynE * kSynK) / 256; ++r) {
      const int idx = tid + 256 * r;
      const int row = idx / kSynK, kk = idx % kSynK;
      const int e = e0 + row, k = k0 + kk;
      const bool in = e < n_el && k < K;
      sBh[kk][row] = in ? Bh[(size_t)e * K + k] : 0.f;
      sBl[kk][row] = in ? Bl[(size_t)e * K + k] : 0.f;
    }
    {
      const int row = tid / kSynK, kk = tid % kSynK;   // 256 = 16 samples x 16 terms
      const int sm = s0 + row, k = k0 + kk;
      const ff x = (sm < S && k < K) ? ff_of(xi[(size_t)sm * K + k]) : ff{0.f, 0.f};
      sXh[kk][row] = x.hi;
      sXl[kk][row] = x.lo;
    }
    __syncthreads();
#pragma unroll 4
    for (int kk = 0; kk < kSynK; ++kk) {
      const ff x{sXh[kk][ls], sXl[kk][ls]};
#pragma unroll
      for (int a = 0; a < 8; ++a) ff_fma(acc[a], ff{sBh[kk][le + 16 * a], sBl[kk][le + 16 * a]}, x);
    }
    __syncthreads();
  }
  const int sm = s0 + ls;
  if (sm >= S) return;
#pragma unroll
  for (int a = 0; a < 8; ++a) {
    const int e = e0 + le + 16 * a;
    if (e >= n_el) continue;
    const double ph = ff_dbl(acc[a]);
    if (trig) {
      double sn, cs;
      sincos(2.0 * ph, &sn, &cs);
      const ff t[4] = {ff_of(cs), ff_of(sn), ff_of(cs * cs - sn * sn), ff_of(2.0 * sn * cs)};
      float* o = (float*)out + 8 * ((size_t)sm * n_el + e);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        o[2 * m] = t[m].hi;
        o[2 * m + 1] = t[m].lo;
      }
    } else {
      ((double*)out)[(size_t)sm * n_el + e] = ph;
    }
  }
}

// ---------------------------------------------------------------- setup

// Fine stencil of the solve mesh from the element matrices K_e = sum_m t_m(phi_e) Km[m]
// (t = 1, c2, s2, c4, s4), summed in float-float: the FP32 stencil A is its high part
// and Alo its low part (the refinement residual uses both). Five threads per node, one
// per stored block (self, E, N, NE, NW; items ordered sample, block, node so that the
// stores coalesce); the self-block thread also forms the damped block-Jacobi inverse,
// the lifting right-hand side b = -K d_prescribed (only u = shortening on x = L is
// non-zero), d = 0 and |b|^2 per sample.
__global__ void __launch_bounds__(kThreads) k_build_fine(const __grid_constant__ Views V) {
  const Item it = item_of(V, 5 * V.v[view_of(V)].f.N);
  const View& W = V.v[it.v];
  const int n = W.f.n, N = W.f.N, s = it.s;
  double bb = 0.0;
  if (it.ok) {
    const int slot = it.p / N, p = it.p - slot * N, i = p % (n + 1), j = p / (n + 1);
    const float* __restrict__ Kh = &V.cc->Kmh[W.F.mesh][0][0];
    const float* __restrict__ Kl = &V.cc->Kml[W.F.mesh][0][0];
    const int oxs[5] = {0, 1, 0, 1, -1}, oys[5] = {0, 0, 1, 1, 1};
    const int sx = oxs[slot], sy = oys[slot];
    const bool self = slot == 0;
    ff blk[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) blk[k] = ff{0.f, 0.f};
    ff rhs[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    const ff msh{V.cc->msh_hi, V.cc->msh_lo};
    // element q = (qx, qy) of the node's four lies at (i - 1 + qx, j - 1 + qy); the
    // node's local index a and each corner b's offset are constants after unrolling
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int qx = q & 1, qy = q >> 1;
      const int ie = i - 1 + qx, je = j - 1 + qy;
      if (ie < 0 || je < 0 || ie >= n || je >= n) continue;
      const int dx = 1 - qx, dy = 1 - qy;
      const int a = dy == 0 ? dx : 3 - dx;
      // the corner b of this element at offset (sx, sy) from the node, if any
      int bsel = -1;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        const int bx = (b == 1 || b == 2) ? 1 : 0, by = b >= 2 ? 1 : 0;
        if (bx - dx == sx && by - dy == sy) bsel = b;
      }
      const bool lift_any = self && ie + 1 == n;   // the element touches x = L
      if (bsel < 0 && !lift_any) continue;
      const float* tg = W.F.trig + 8 * ((size_t)s * n * n + (size_t)je * n + ie);
      const ff t[5] = {ff{1.f, 0.f}, ff{tg[0], tg[1]}, ff{tg[2], tg[3]}, ff{tg[4], tg[5]}, ff{tg[6], tg[7]}};
      auto entry = [&](int b, int r, int c) {
        const int off = (3 * a + r) * 12 + 3 * b + c;
        ff k{0.f, 0.f};
#pragma unroll
        for (int m = 0; m < kTerms; ++m) ff_fma(k, t[m], ff{Kh[m * 144 + off], Kl[m * 144 + off]});
        return k;
      };
      if (bsel >= 0) {
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
          for (int c = 0; c < 3; ++c) ff_fma(blk[3 * r + c], entry(bsel, r, c), 1.f);
      }
      if (lift_any) {
        // corners 1 and 2 lie on x = L: rhs -= shortening * K[a, b][:, u]
#pragma unroll
        for (int b = 1; b <= 2; ++b)
#pragma unroll
          for (int r = 0; r < 3; ++r) ff_fma(rhs[r], entry(b, r, 0), msh);
      }
    }
    // Dirichlet rows / columns -> identity
    const int dm = dmask(i, j, n);
    const int qi = i + sx, qj = j + sy;
    const bool in = qi >= 0 && qi <= n && qj <= n;
    const int dq = in ? dmask(qi, qj, n) : 0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const bool rowd = r < 2 && ((dm >> r) & 1), cold = c < 2 && ((dq >> c) & 1);
        if (!in || rowd || cold) blk[3 * r + c] = ff{0.f, 0.f};
      }
    float4* Ah = W.f.A + (size_t)s * kGroups * N;
    float4* Al = W.F.Alo + (size_t)s * kGroups * N;
    if (!self) {
      const int k0 = 6 + 9 * (slot - 1);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        *coef_at(Ah, N, k0 + k, p) = blk[k].hi;
        *coef_at(Al, N, k0 + k, p) = blk[k].lo;
      }
      if (slot == 4) {   // the two pad coefficients
        *coef_at(Ah, N, 42, p) = *coef_at(Ah, N, 43, p) = 0.f;
        *coef_at(Al, N, 42, p) = *coef_at(Al, N, 43, p) = 0.f;
      }
    } else {
#pragma unroll
      for (int r = 0; r < 2; ++r)
        if ((dm >> r) & 1) {
          blk[4 * r] = ff{1.f, 0.f};
          rhs[r] = ff{0.f, 0.f};
        }
      const ff sb[6] = {blk[0], blk[1], blk[2], blk[4], blk[5], blk[8]};
      float sf[6], inv[6];
#pragma unroll
      for (int k = 0; k < 6; ++k) {
        *coef_at(Ah, N, k, p) = sb[k].hi;
        *coef_at(Al, N, k, p) = sb[k].lo;
        sf[k] = sb[k].hi;
      }
      inv_sym3(sf, inv);   // the smoother's inverse needs no more than FP32
      float4* Di = W.f.Dinv + (size_t)s * kDinvGroups * N;
      Di[p] = make_float4(kOmega * inv[0], kOmega * inv[1], kOmega * inv[2], kOmega * inv[3]);
      Di[N + p] = make_float4(kOmega * inv[4], kOmega * inv[5], 0.f, 0.f);
      const size_t o = (size_t)s * N + p;
      W.F.bh[o] = make_float4(rhs[0].hi, rhs[1].hi, rhs[2].hi, 0.f);
      W.F.bl[o] = make_float4(rhs[0].lo, rhs[1].lo, rhs[2].lo, 0.f);
      W.F.dh[o] = make_float4(0.f, 0.f, 0.f, 0.f);
      W.F.dl[o] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int c = 0; c < 3; ++c) bb += (double)rhs[c].hi * (double)rhs[c].hi;
    }
  }
  SampleState* st = W.F.st;
  warp_add_by_sample(bb, s, [&](int k) { return &st[k].bnorm2; });
}

// Galerkin coarse operator P^T A P of the masked finer stencil (bilinear P), then the
// coarse Dirichlet rows / columns replaced by the identity. One thread per coarse node.
__global__ void __launch_bounds__(kThreads) k_rap(const __grid_constant__ Views V) {
  const Item it = item_of(V, V.v[view_of(V)].c.N);
  if (!it.ok) return;
  const View& W = V.v[it.v];
  const int nc = W.c.n, Nc = W.c.N, nf = W.f.n, Nf = W.f.N, s = it.s;
  const int P = it.p, I = P % (nc + 1), J = P / (nc + 1);
  const float4* Af = W.f.A + (size_t)s * kGroups * Nf;
  float acc[5][9];
#pragma unroll
  for (int b = 0; b < 5; ++b)
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[b][k] = 0.f;
  const int Dx[5] = {0, 1, 0, 1, -1}, Dy[5] = {0, 0, 1, 1, 1};
#pragma unroll 1
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll 1
    for (int dx = -1; dx <= 1; ++dx) {
      const int pi = 2 * I + dx, pj = 2 * J + dy;
      if (pi < 0 || pj < 0 || pi > nf || pj > nf) continue;
      const float wp = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f);
#pragma unroll 1
      for (int oy = -1; oy <= 1; ++oy)
#pragma unroll 1
        for (int ox = -1; ox <= 1; ++ox) {
          const int qi = pi + ox, qj = pj + oy;
          if (qi < 0 || qj < 0 || qi > nf || qj > nf) continue;
          float w[5];
          bool any = false;
#pragma unroll
          for (int b = 0; b < 5; ++b) {
            const int ex = qi - 2 * (I + Dx[b]), ey = qj - 2 * (J + Dy[b]);
            const bool in = I + Dx[b] >= 0 && I + Dx[b] <= nc && J + Dy[b] <= nc;
            w[b] = (in && ex >= -1 && ex <= 1 && ey >= -1 && ey <= 1) ? wp * (ex ? 0.5f : 1.f) * (ey ? 0.5f : 1.f)
                                                                      : 0.f;
            any |= w[b] != 0.f;
          }
          if (!any) continue;
          float B[9];
          block_of(Af, Nf, nf, pi, pj, ox, oy, B);
#pragma unroll
          for (int b = 0; b < 5; ++b)
            if (w[b] != 0.f)
#pragma unroll
              for (int k = 0; k < 9; ++k) acc[b][k] += w[b] * B[k];
        }
    }
  const int dm = dmask(I, J, nc);
#pragma unroll
  for (int b = 0; b < 5; ++b) {
    const int qi = I + Dx[b], qj = J + Dy[b];
    const bool in = qi >= 0 && qi <= nc && qj <= nc;
    const int dq = in ? dmask(qi, qj, nc) : 0;
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const bool rowd = r < 2 && ((dm >> r) & 1), cold = c < 2 && ((dq >> c) & 1);
        if (!in || rowd || cold) acc[b][3 * r + c] = 0.f;
      }
  }
#pragma unroll
  for (int r = 0; r < 2; ++r)
    if ((dm >> r) & 1) acc[0][4 * r] = 1.f;
  // the diagonal block is symmetric up to rounding: keep the mean of the two triangles
  float a[44];
  a[0] = acc[0][0];
  a[1] = 0.5f * (acc[0][1] + acc[0][3]);
  a[2] = 0.5f * (acc[0][2] + acc[0][6]);
  a[3] = acc[0][4];
  a[4] = 0.5f * (acc[0][5] + acc[0][7]);
  a[5] = acc[0][8];
#pragma unroll
  for (int b = 1; b < 5; ++b)
#pragma unroll
    for (int k = 0; k < 9; ++k) a[6 + 9 * (b - 1) + k] = acc[b][k];
  a[42] = a[43] = 0.f;
  float4* Ac = W.c.A + (size_t)s * kGroups * Nc;
#pragma unroll
  for (int g = 0; g < kGroups; ++g) Ac[(size_t)g * Nc + P] = make_float4(a[4 * g], a[4 * g + 1], a[4 * g + 2], a[4 * g + 3]);
  const float self[6] = {a[0], a[1], a[2], a[3], a[4], a[5]};
  float inv[6];
  inv_sym3(self, inv);
  float4* Di = W.c.Dinv + (size_t)s * kDinvGroups * Nc;
  Di[P] = make_float4(kOmega * inv[0], kOmega * inv[1], kOmega * inv[2], kOmega * inv[3]);
  Di[Nc + P] = make_float4(kOmega * inv[4], kOmega * inv[5], 0.f, 0.f);
}

// Dense inverse of the coarsest (2 x 2 elements, 27 DOFs, DOF 3 node + component)
// operator: one warp per sample, Gauss-Jordan on [M | I] in shared memory, FP32 (the
// inverse only serves the preconditioner; symmetric positive definite: no pivoting, a
// non-positive pivot leaves the inverse zero).
constexpr int kGJWarps = kInverseWarps;
__global__ void __launch_bounds__(32 * kGJWarps) k_coarsest_inverse(const __grid_constant__ Views V) {
  __shared__ float M[kGJWarps][kCoarseDofs][2 * kCoarseDofs + 1];
  const int v = view_of(V);
  const View& W = V.v[v];
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int s = (blockIdx.x - W.blk0) * kGJWarps + wid;
  if (s >= W.f.S) return;   // whole warps
  const int n = W.f.n, N = W.f.N;
  const float4* A = W.f.A + (size_t)s * kGroups * N;
  float(*m)[2 * kCoarseDofs + 1] = M[wid];
  for (int k = lane; k < kCoarseDofs * 2 * kCoarseDofs; k += 32) {
    const int r = k / (2 * kCoarseDofs), c = k % (2 * kCoarseDofs);
    m[r][c] = (c - kCoarseDofs == r) ? 1.f : 0.f;
  }
  __syncwarp();
  if (lane < N) {
    const int i = lane % (n + 1), j = lane / (n + 1);
    for (int oy = -1; oy <= 1; ++oy)
      for (int ox = -1; ox <= 1; ++ox) {
        const int qi = i + ox, qj = j + oy;
        if (qi < 0 || qj < 0 || qi > n || qj > n) continue;
        float B[9];
        block_of(A, N, n, i, j, ox, oy, B);
        const int q = qj * (n + 1) + qi;
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) m[3 * lane + a][3 * q + b] = B[3 * a + b];
      }
  }
  __syncwarp();
  bool ok = true;
  for (int k = 0; k < kCoarseDofs; ++k) {
    const float piv = m[k][k];
    ok = ok && piv > 0.f;
    const float ip = piv > 0.f ? 1.f / piv : 0.f;
    __syncwarp();
    for (int c = lane; c < 2 * kCoarseDofs; c += 32) m[k][c] *= ip;
    __syncwarp();
    if (lane < kCoarseDofs && lane != k) {
      const float f = m[lane][k];
      for (int c = 0; c < 2 * kCoarseDofs; ++c) m[lane][c] -= f * m[k][c];
    }
    __syncwarp();
  }
  float* out = W.Ainv + (size_t)s * kCoarseDofs * kCoarseDofs;
  for (int k = lane; k < kCoarseDofs * kCoarseDofs; k += 32) {
    const int r = k / kCoarseDofs, c = k % kCoarseDofs;
    out[k] = ok ? m[r][kCoarseDofs + c] : 0.f;
  }
}

// ---------------------------------------------------------------- V(1,1) cycle

__device__ __forceinline__ bool active(const View& W, int s) { return s >= 0 && W.F.st[s].act; }

__device__ __forceinline__ float4 f4(float a, float b, float c) { return make_float4(a, b, c, 0.f); }
// x = Dinv r with the block inverse's two groups (d0 = 00 01 02 11, d1 = 12 22 - -)
__device__ __forceinline__ float4 dmul(float4 d0, float4 d1, float4 r) {
  return f4(d0.x * r.x + d0.y * r.y + d0.z * r.z, d0.y * r.x + d0.w * r.y + d1.x * r.z,
            d0.z * r.x + d1.x * r.y + d1.y * r.z);
}

// Pre-smoothing from zero and the residual: x = Dinv r, t = r - A x (x of the
// neighbours recomputed from their r).
// four resident blocks per SM (at most 64 registers, no spills): the kernel is latency-bound
__global__ void __launch_bounds__(kThreads, 4) k_pre(const __grid_constant__ Views V) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  const View& W = V.v[it.v];
  if (!it.ok || !active(W, it.s)) return;
  const int n = W.f.n, N = W.f.N, p = it.p, i = p % (n + 1), j = p / (n + 1);
  const float4* __restrict__ A = W.f.A + (size_t)it.s * kGroups * N;
  const float4* __restrict__ D = W.f.Dinv + (size_t)it.s * kDinvGroups * N;
  const float4* __restrict__ r = W.f.r + (size_t)it.s * N;
  auto xf = [&](int q) { return dmul(D[q], D[N + q], r[q]); };
  float y[3] = {0.f, 0.f, 0.f};
  apply_node(A, N, n, i, j, xf, y);
  const float4 rp = r[p];
  W.f.x[(size_t)it.s * N + p] = xf(p);
  W.f.t[(size_t)it.s * N + p] = f4(rp.x - y[0], rp.y - y[1], rp.z - y[2]);
}

// Restriction c.r = P^T f.t, zero at the coarse Dirichlet DOFs.
__global__ void __launch_bounds__(kThreads) k_restrict(const __grid_constant__ Views V) {
  const Item it = item_of(V, V.v[view_of(V)].c.N);
  const View& W = V.v[it.v];
  if (!it.ok || !active(W, it.s)) return;
  const int nc = W.c.n, Nc = W.c.N, nf = W.f.n, Nf = W.f.N, P = it.p, I = P % (nc + 1), J = P / (nc + 1);
  const float4* __restrict__ t = W.f.t + (size_t)it.s * Nf;
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int pi = 2 * I + dx, pj = 2 * J + dy;
      if (pi < 0 || pj < 0 || pi > nf || pj > nf) continue;
      const float w = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f);
      const float4 v = t[pj * (nf + 1) + pi];
      acc[0] += w * v.x;
      acc[1] += w * v.y;
      acc[2] += w * v.z;
    }
  const int dm = dmask(I, J, nc);
  if (dm & 1) acc[0] = 0.f;
  if (dm & 2) acc[1] = 0.f;
  W.c.r[(size_t)it.s * Nc + P] = f4(acc[0], acc[1], acc[2]);
}

// Prolongation f.x += P c.t (bilinear).
__global__ void __launch_bounds__(kThreads) k_prolong(const __grid_constant__ Views V) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  const View& W = V.v[it.v];
  if (!it.ok || !active(W, it.s)) return;
  const int nf = W.f.n, Nf = W.f.N, nc = W.c.n, Nc = W.c.N, p = it.p, i = p % (nf + 1), j = p / (nf + 1);
  const float4* __restrict__ xc = W.c.t + (size_t)it.s * Nc;
  const int I0 = i >> 1, J0 = j >> 1;
  const bool ox = i & 1, oy = j & 1;
  const float w = (ox ? 0.5f : 1.f) * (oy ? 0.5f : 1.f);
  float4 x = W.f.x[(size_t)it.s * Nf + p];
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int di = b & 1, dj = b >> 1;
    if ((di && !ox) || (dj && !oy)) continue;
    const float4 v = xc[(J0 + dj) * (nc + 1) + I0 + di];
    x.x += w * v.x;
    x.y += w * v.y;
    x.z += w * v.z;
  }
  W.f.x[(size_t)it.s * Nf + p] = x;
}

// Post-smoothing: f.t = x + Dinv (r - A x). On the solve mesh (top) f.t is the
// preconditioned residual z and r . z is accumulated into rz_new.
// four resident blocks per SM (at most 64 registers, no spills)
__global__ void __launch_bounds__(kThreads, 4) k_post(const __grid_constant__ Views V, bool top) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  const View& W = V.v[it.v];
  const bool ok = it.ok && active(W, it.s);
  double rz = 0.0;
  if (ok) {
    const int n = W.f.n, N = W.f.N, p = it.p, i = p % (n + 1), j = p / (n + 1);
    const float4* __restrict__ A = W.f.A + (size_t)it.s * kGroups * N;
    const float4* __restrict__ D = W.f.Dinv + (size_t)it.s * kDinvGroups * N;
    const float4* __restrict__ x = W.f.x + (size_t)it.s * N;
    auto xf = [&](int q) { return x[q]; };
    float y[3] = {0.f, 0.f, 0.f};
    apply_node(A, N, n, i, j, xf, y);
    const float4 rp = W.f.r[(size_t)it.s * N + p], xp = x[p];
    const float4 e = dmul(D[p], D[N + p], f4(rp.x - y[0], rp.y - y[1], rp.z - y[2]));
    const float4 z = f4(xp.x + e.x, xp.y + e.y, xp.z + e.z);
    W.f.t[(size_t)it.s * N + p] = z;
    if (top) rz = (double)rp.x * z.x + (double)rp.y * z.y + (double)rp.z * z.z;
  }
  if (top) {
    SampleState* st = W.F.st;
    warp_add_by_sample(rz, ok ? it.s : -1, [&](int k) { return &st[k].rz_new; });
  }
}

// Fused multigrid bottom: one block per sample runs the part of the V(1,1) cycle on
// the meshes of at most kBottomN elements per side (entry mesh f, the next mesh c when
// the entry is 8 x 8, and the 2 x 2 coarsest through Ainv), with the vectors in shared
// memory and the stencils read from global memory: pre-smoothing and residual,
// restriction, the dense coarsest solve, prolongation and post-smoothing, level by
// level with a barrier between steps. Entry: f.r (written by the restriction from the
// mesh above, or the CG residual when f is the solve mesh); exit: f.t, and r . t into
// rz_new when f is the solve mesh (top). Replaces 4 launches per level and the coarse
// solve, whose tiny grids cost launch latency rather than bandwidth.
constexpr int kBotMaxN = (kBottomN + 1) * (kBottomN + 1);
__global__ void __launch_bounds__(kBottomThreads) k_bottom(const __grid_constant__ Views V, int top_mask) {
  __shared__ float4 sR[3][kBotMaxN], sX[3][kBotMaxN], sT[3][kBotMaxN];
  __shared__ double red[kBottomThreads / 32];
  const int v = view_of(V);
  const View& W = V.v[v];
  const int s = blockIdx.x - W.blk0;
  if (s >= W.f.S || !W.F.st[s].act) return;   // uniform over the block
  const int tid = threadIdx.x;
  const bool top = (top_mask >> v) & 1;
  // the chain of meshes: entry f (n = 8 or 4), then c when f is 8 x 8, then 2 x 2
  const int nl = W.f.n == 2 * kCoarsest ? 2 : 3;
  int nn[3], NN[3];
  nn[0] = W.f.n;
  for (int l = 1; l < nl; ++l) nn[l] = nn[l - 1] / 2;
  for (int l = 0; l < nl; ++l) NN[l] = (nn[l] + 1) * (nn[l] + 1);
  const float4* Al[2] = {W.f.A + (size_t)s * kGroups * NN[0], nl == 3 ? W.c.A + (size_t)s * kGroups * NN[1] : nullptr};
  const float4* Dl[2] = {W.f.Dinv + (size_t)s * kDinvGroups * NN[0],
                         nl == 3 ? W.c.Dinv + (size_t)s * kDinvGroups * NN[1] : nullptr};
  for (int p = tid; p < NN[0]; p += blockDim.x) sR[0][p] = W.f.r[(size_t)s * NN[0] + p];
  __syncthreads();
  // descend: pre-smoothing from zero, residual, restriction
  for (int l = 0; l + 1 < nl; ++l) {
    const int n = nn[l], N = NN[l];
    const float4* A = Al[l];
    const float4* D = Dl[l];
    for (int p = tid; p < N; p += blockDim.x) sX[l][p] = dmul(D[p], D[N + p], sR[l][p]);
    __syncthreads();
    for (int p = tid; p < N; p += blockDim.x) {
      const int i = p % (n + 1), j = p / (n + 1);
      float y[3] = {0.f, 0.f, 0.f};
      apply_node(A, N, n, i, j, [&](int q) { return sX[l][q]; }, y);
      const float4 r = sR[l][p];
      sT[l][p] = f4(r.x - y[0], r.y - y[1], r.z - y[2]);
    }
    __syncthreads();
    const int nc = nn[l + 1];
    for (int P = tid; P < NN[l + 1]; P += blockDim.x) {
      const int I = P % (nc + 1), J = P / (nc + 1);
      float acc[3] = {0.f, 0.f, 0.f};
      for (int dy = -1; dy <= 1; ++dy)
        for (int dx = -1; dx <= 1; ++dx) {
          const int pi = 2 * I + dx, pj = 2 * J + dy;
          if (pi < 0 || pj < 0 || pi > n || pj > n) continue;
          const float w = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f);
          const float4 t = sT[l][pj * (n + 1) + pi];
          acc[0] += w * t.x;
          acc[1] += w * t.y;
          acc[2] += w * t.z;
        }
      const int dm = dmask(I, J, nc);
      sR[l + 1][P] = f4((dm & 1) ? 0.f : acc[0], (dm & 2) ? 0.f : acc[1], acc[2]);
    }
    __syncthreads();
  }
  // coarsest: t = Ainv r, a thread per node
  {
    const int lc = nl - 1;
    const float* __restrict__ M = W.Ainv + (size_t)s * kCoarseDofs * kCoarseDofs;
    for (int node = tid; node < kCoarseDofs / 3; node += blockDim.x) {
      float o[3];
      for (int c = 0; c < 3; ++c) {
        const float* row = M + (3 * node + c) * kCoarseDofs;
        float acc = 0.f;
        for (int q = 0; q < kCoarseDofs / 3; ++q) {
          const float4 r = sR[lc][q];
          acc += row[3 * q] * r.x + row[3 * q + 1] * r.y + row[3 * q + 2] * r.z;
        }
        o[c] = acc;
      }
      sT[lc][node] = f4(o[0], o[1], o[2]);
    }
    __syncthreads();
  }
  // ascend: prolongation, post-smoothing (the result in sT of each level)
  double rz = 0.0;
  for (int l = nl - 2; l >= 0; --l) {
    const int n = nn[l], N = NN[l], nc = nn[l + 1];
    for (int p = tid; p < N; p += blockDim.x) {
      const int i = p % (n + 1), j = p / (n + 1);
      const int I0 = i >> 1, J0 = j >> 1;
      const bool ox = i & 1, oy = j & 1;
      const float w = (ox ? 0.5f : 1.f) * (oy ? 0.5f : 1.f);
      float4 x = sX[l][p];
      for (int b = 0; b < 4; ++b) {
        const int di = b & 1, dj = b >> 1;
        if ((di && !ox) || (dj && !oy)) continue;
        const float4 c = sT[l + 1][(J0 + dj) * (nc + 1) + I0 + di];
        x.x += w * c.x;
        x.y += w * c.y;
        x.z += w * c.z;
      }
      sX[l][p] = x;
    }
    __syncthreads();
    const float4* A = Al[l];
    const float4* D = Dl[l];
    for (int p = tid; p < N; p += blockDim.x) {
      const int i = p % (n + 1), j = p / (n + 1);
      float y[3] = {0.f, 0.f, 0.f};
      apply_node(A, N, n, i, j, [&](int q) { return sX[l][q]; }, y);
      const float4 r = sR[l][p], xp = sX[l][p];
      const float4 e = dmul(D[p], D[N + p], f4(r.x - y[0], r.y - y[1], r.z - y[2]));
      const float4 z = f4(xp.x + e.x, xp.y + e.y, xp.z + e.z);
      sT[l][p] = z;
      if (l == 0) {
        W.f.t[(size_t)s * N + p] = z;
        if (top) rz += (double)r.x * z.x + (double)r.y * z.y + (double)r.z * z.z;
      }
    }
    __syncthreads();
  }
  if (top) {
#pragma unroll
    for (int o = 16; o; o >>= 1) rz += __shfl_down_sync(0xffffffffu, rz, o);
    if ((tid & 31) == 0) red[tid >> 5] = rz;
    __syncthreads();
    if (tid == 0) {
      double t = 0.0;
      for (int k = 0; k < kBottomThreads / 32; ++k) t += red[k];
      atomicAdd(&W.F.st[s].rz_new, t);
    }
  }
}

// ---------------------------------------------------------------- correction CG

// p_out = z + beta p_in (z alone on a step's first direction), q = A p_out, p . q.
__global__ void __launch_bounds__(kThreads) k_cg_apply(const __grid_constant__ Views V, bool odd) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  const View& W = V.v[it.v];
  const bool ok = it.ok && active(W, it.s);
  double pq = 0.0;
  if (ok) {
    const int n = W.f.n, N = W.f.N, p = it.p, i = p % (n + 1), j = p / (n + 1);
    const size_t sN = (size_t)it.s * N;
    const float4* __restrict__ A = W.f.A + (size_t)it.s * kGroups * N;
    const float4* __restrict__ z = W.f.t + sN;
    const float4* __restrict__ pin = (odd ? W.F.p1 : W.F.p0) + sN;
    float4* pout = (odd ? W.F.p0 : W.F.p1) + sN;
    const float beta = (float)W.F.st[it.s].beta;
    auto pf = [&](int q) {
      const float4 a = z[q];
      if (beta == 0.f) return a;
      const float4 b = pin[q];
      return f4(a.x + beta * b.x, a.y + beta * b.y, a.z + beta * b.z);
    };
    float y[3] = {0.f, 0.f, 0.f};
    apply_node(A, N, n, i, j, pf, y);
    const float4 pv = pf(p);
    pout[p] = pv;
    W.F.q[sN + p] = f4(y[0], y[1], y[2]);
    pq = (double)pv.x * y[0] + (double)pv.y * y[1] + (double)pv.z * y[2];
  }
  SampleState* st = W.F.st;
  warp_add_by_sample(pq, ok ? it.s : -1, [&](int k) { return &st[k].pq; });
}

// c += alpha p_out, r -= alpha q, |r|^2.
__global__ void __launch_bounds__(kThreads) k_cg_update(const __grid_constant__ Views V, bool odd) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  const View& W = V.v[it.v];
  const bool ok = it.ok && active(W, it.s);
  double rr = 0.0;
  if (ok) {
    const size_t o = (size_t)it.s * W.f.N + it.p;
    const float a = (float)W.F.st[it.s].alpha;
    const float4 pv = (odd ? W.F.p0 : W.F.p1)[o], qv = W.F.q[o];
    float4 c = W.F.c[o], r = W.f.r[o];
    c = f4(c.x + a * pv.x, c.y + a * pv.y, c.z + a * pv.z);
    r = f4(r.x - a * qv.x, r.y - a * qv.y, r.z - a * qv.z);
    W.F.c[o] = c;
    W.f.r[o] = r;
    rr = (double)r.x * r.x + (double)r.y * r.y + (double)r.z * r.z;
  }
  SampleState* st = W.F.st;
  warp_add_by_sample(rr, ok ? it.s : -1, [&](int k) { return &st[k].rr; });
}

// one thread per sample of every view
__device__ __forceinline__ SampleState* sample_of(const Views& V, int* S_out) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  int base = 0;
  for (int v = 0; v < V.nv; ++v) {
    const int S = V.v[v].f.S;
    if (k < base + S) {
      *S_out = k - base;
      return V.v[v].F.st + (k - base);
    }
    base += S;
  }
  return nullptr;
}

__global__ void k_scal_a(const __grid_constant__ Views V) {
  int s;
  SampleState* st = sample_of(V, &s);
  if (!st || !st->act) return;
  if (st->pq > 0.0 && st->rz > 0.0) {
    st->alpha = st->rz / st->pq;
  } else {
    st->alpha = 0.0;
    st->act = 0;   // breakdown: the refinement takes over
  }
  st->rr = 0.0;
}

// After the preconditioner: convergence of the correction solve and the next beta.
__global__ void k_scal_b(const __grid_constant__ Views V, int max_iter) {
  int s;
  SampleState* st = sample_of(V, &s);
  if (!st || !st->act) return;
  if (st->first) {
    st->first = 0;
    st->beta = 0.0;
  } else {
    st->it += 1;
    st->it_total += 1;
    if (!(st->rr > st->tol2 * st->rr0) || st->it_total >= max_iter) st->act = 0;
    st->beta = st->rz > 0.0 ? st->rz_new / st->rz : 0.0;
  }
  if (!(st->rz_new > 0.0)) st->act = 0;
  st->rz = st->rz_new;
  st->rz_new = 0.0;
  st->pq = 0.0;
}

__global__ void k_count_active(const __grid_constant__ Views V, int* count) {
  int s;
  SampleState* st = sample_of(V, &s);
  const bool a = st && st->act;
  const unsigned m = __ballot_sync(0xffffffffu, a);
  if ((threadIdx.x & 31) == 0 && m) atomicAdd(count, __popc(m));
}

// ---------------------------------------------------------------- FP64 refinement

// r = b - A d with the float-float stencil and solution, in float-float; the FP32
// correction right-hand side r32 and |r|^2. With first (d = 0) r = b.
__global__ void __launch_bounds__(kThreads) k_resid64(const __grid_constant__ Views V, bool first) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  const View& W = V.v[it.v];
  const bool ok = it.ok && !W.F.st[it.s].done;
  double rr = 0.0;
  if (ok) {
    const int n = W.f.n, N = W.f.N, p = it.p, i = p % (n + 1), j = p / (n + 1);
    ff y[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    const size_t sN = (size_t)it.s * N;
    if (!first) {
      const float4* __restrict__ Ah = W.f.A + (size_t)it.s * kGroups * N;
      const float4* __restrict__ Al = W.F.Alo + (size_t)it.s * kGroups * N;
      const float4* __restrict__ dh = W.F.dh + sN;
      const float4* __restrict__ dl = W.F.dl + sN;
      auto xf = [&](int q, ff v[3]) {
        const float4 h = dh[q], l = dl[q];
        v[0] = ff{h.x, l.x};
        v[1] = ff{h.y, l.y};
        v[2] = ff{h.z, l.z};
      };
      apply_node_ff(Ah, Al, N, n, i, j, xf, y);
    }
    const float4 bh = W.F.bh[sN + p], bl = W.F.bl[sN + p];
    const ff b[3] = {ff{bh.x, bl.x}, ff{bh.y, bl.y}, ff{bh.z, bl.z}};
    float ev[3];
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // e = b - y: b + (-y) in float-float, then rounded
      ff e = b[c];
      ff_fma(e, y[c], -1.f);
      ev[c] = __fadd_rn(e.hi, e.lo);
      rr += (double)ev[c] * (double)ev[c];
    }
    W.f.r[sN + p] = f4(ev[0], ev[1], ev[2]);
  }
  SampleState* st = W.F.st;
  warp_add_by_sample(rr, ok ? it.s : -1, [&](int k) { return &st[k].r64n2; });
}

// Per sample: stop at rtol (or out of iterations), else start a correction solve whose
// target is |r| <= max(1e-4, rtol |b| / (2 |r64|)) |r64|.
__global__ void k_outer_check(const __grid_constant__ Views V, double rtol, int max_iter) {
  int s;
  SampleState* st = sample_of(V, &s);
  if (!st || st->done) return;
  st->refine += 1;
  const double r2 = st->r64n2;
  if (st->refine == 1) st->bnorm2 = r2;   // d = 0: r = b
  const bool conv = r2 <= rtol * rtol * st->bnorm2;
  if (conv || !(r2 == r2) || st->it_total >= max_iter) {
    st->done = 1;
    st->act = 0;
    st->conv = conv ? 1 : 0;
  } else {
    st->act = 1;
    st->it = 0;
    st->rr0 = r2;
    const double t2 = 0.25 * rtol * rtol * st->bnorm2 / r2;
    st->tol2 = fmin(0.25, fmax(1e-8, t2));
    st->first = 1;
    st->rz_new = 0.0;
  }
  st->r64n2 = 0.0;
}

// d += c in float-float, c = 0 (c is zero for samples that did not run).
__global__ void __launch_bounds__(kThreads) k_accumulate(const __grid_constant__ Views V) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  if (!it.ok) return;
  const View& W = V.v[it.v];
  const size_t o = (size_t)it.s * W.f.N + it.p;
  const float4 c = W.F.c[o], h = W.F.dh[o], l = W.F.dl[o];
  ff d[3] = {ff{h.x, l.x}, ff{h.y, l.y}, ff{h.z, l.z}};
  ff_fma(d[0], ff{c.x, 0.f}, 1.f);
  ff_fma(d[1], ff{c.y, 0.f}, 1.f);
  ff_fma(d[2], ff{c.z, 0.f}, 1.f);
  W.F.dh[o] = f4(d[0].hi, d[1].hi, d[2].hi);
  W.F.dl[o] = f4(d[0].lo, d[1].lo, d[2].lo);
  W.F.c[o] = f4(0.f, 0.f, 0.f);
}

// ---------------------------------------------------------------- quantities of interest

// Items per sample: the ncen^2 elements inside Omega' (strength), then the n elements of
// the last column (reaction). acc[s] = (f*, int_Omega' sigma_x, sum (K d)_u on x = L, -).
__global__ void __launch_bounds__(kThreads) k_qoi(const __grid_constant__ Views V) {
  const int v = view_of(V);
  const View& W = V.v[v];
  const int n = W.f.n, N = W.f.N;
  const int ncen = W.F.khi - W.F.klo + 1;
  const Item it = item_of(V, ncen * ncen + n);
  const Consts& K = *V.cc;
  const double h = K.h[W.F.mesh];
  double fmax_v = 0.0, sx = 0.0, rx = 0.0;
  int ie = 0, je = 0;
  bool cen = false;
  if (it.ok) {
    if (it.p < ncen * ncen) {
      cen = true;
      ie = W.F.klo + it.p % ncen;
      je = W.F.klo + it.p / ncen;
    } else {
      ie = n - 1;
      je = it.p - ncen * ncen;
    }
    const float4* __restrict__ dh = W.F.dh + (size_t)it.s * N;
    const float4* __restrict__ dl = W.F.dl + (size_t)it.s * N;
    double de[12];
    const int cx[4] = {0, 1, 1, 0}, cy[4] = {0, 0, 1, 1};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int q = (je + cy[a]) * (n + 1) + ie + cx[a];
#pragma unroll
      {
        const float4 h = dh[q], l = dl[q];
        de[3 * a] = (double)h.x + (double)l.x;
        de[3 * a + 1] = (double)h.y + (double)l.y;
        de[3 * a + 2] = (double)h.z + (double)l.z;
      }
      if (ie + cx[a] == n) de[3 * a] += K.shortening;
    }
    const float* tg = W.F.trig + 8 * ((size_t)it.s * n * n + (size_t)je * n + ie);
    const double c2 = (double)tg[0] + (double)tg[1], s2 = (double)tg[2] + (double)tg[3];
    const double t[5] = {1.0, c2, s2, (double)tg[4] + (double)tg[5], (double)tg[6] + (double)tg[7]};
    if (cen) {
      double Cg[16];
#pragma unroll
      for (int k = 0; k < 16; ++k) {
        double a = 0.0;
#pragma unroll
        for (int m = 0; m < kTerms; ++m) a += t[m] * K.Cm[m][k];
        Cg[k] = a;
      }
      // fibre direction from the double angle: cos phi >= 0 and phi = phi + pi give
      // the same fibre-frame stresses
      const double cf = sqrt(fmax(0.0, 0.5 * (1.0 + c2)));
      const double sf = cf > 0.0 ? 0.5 * s2 / cf : 1.0;
      const double g = 0.5773502691896257;   // 1 / sqrt(3)
#pragma unroll
      for (int gp = 0; gp < 4; ++gp) {
        const double xi = (gp & 1) ? g : -g, eta = (gp >> 1) ? g : -g;
        double e[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
        for (int a = 0; a < 4; ++a) {
          const double sx_ = (cx[a] ? 1.0 : -1.0), sy_ = (cy[a] ? 1.0 : -1.0);
          const double N_ = 0.25 * (1 + sx_ * xi) * (1 + sy_ * eta);
          const double dx = 0.5 * sx_ * (1 + sy_ * eta) / h, dy = 0.5 * sy_ * (1 + sx_ * xi) / h;
          e[0] += dx * de[3 * a];
          e[1] += dy * de[3 * a + 1];
          e[2] += dy * de[3 * a] + N_ * de[3 * a + 2];
          e[3] += dx * de[3 * a + 1] - N_ * de[3 * a + 2];
        }
        double sg[4];
#pragma unroll
        for (int r = 0; r < 4; ++r)
          sg[r] = Cg[4 * r] * e[0] + Cg[4 * r + 1] * e[1] + Cg[4 * r + 2] * e[2] + Cg[4 * r + 3] * e[3];
        // fibre frame: R^T S R, S = [[s11, s12], [s21, s22]], R = rotation by phi
        const double l12 = -cf * sf * sg[0] + cf * cf * sg[2] - sf * sf * sg[3] + cf * sf * sg[1];
        const double l22 = sf * sf * sg[0] - sf * cf * sg[2] - cf * sf * sg[3] + cf * cf * sg[1];
        const double tau = sqrt(l12 * l12 + (l22 / K.R) * (l22 / K.R));
        fmax_v = fmax(fmax_v, tau / K.tau_y);
        sx += 0.25 * h * h * sg[0];
      }
    } else {
      // rows of the prescribed u of local nodes 1 and 2 (on x = L)
      const double* __restrict__ Km = &K.Km[W.F.mesh][0][0];
#pragma unroll 1
      for (int rrow = 0; rrow < 2; ++rrow) {
        const int row = 3 * (1 + rrow);
        double acc = 0.0;
#pragma unroll
        for (int col = 0; col < 12; ++col) {
          double k = 0.0;
#pragma unroll
          for (int m = 0; m < kTerms; ++m) k += t[m] * Km[m * 144 + row * 12 + col];
          acc += k * de[col];
        }
        rx += acc;
      }
    }
  }
  double* acc = W.F.acc;
  warp_max_by_sample(fmax_v, (it.ok && cen) ? it.s : -1, [&](int k) { return &acc[4 * k]; });
  warp_add_by_sample(sx, (it.ok && cen) ? it.s : -1, [&](int k) { return &acc[4 * k + 1]; });
  warp_add_by_sample(rx, (it.ok && !cen) ? it.s : -1, [&](int k) { return &acc[4 * k + 2]; });
}

__global__ void k_qoi_final(const __grid_constant__ Views V) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  int base = 0;
  for (int v = 0; v < V.nv; ++v) {
    const View& W = V.v[v];
    if (k < base + W.f.S) {
      const int s = k - base;
      const double* a = W.F.acc + 4 * s;
      const int ncen = W.F.khi - W.F.klo + 1;
      const double h = V.cc->h[W.F.mesh];
      const double area = (double)ncen * ncen * h * h;
      W.F.q_out[2 * s] = a[0] > 0.0 ? -(a[1] / area) / a[0] : 0.0;
      W.F.q_out[2 * s + 1] = -a[2];
      const SampleState& st = W.F.st[s];
      W.F.stat_out[s] = st.conv ? 0 : 4;
      atomicMax(&W.F.iters[0], st.it_total);
      atomicMax(&W.F.iters[1], st.refine);
      return;
    }
    base += W.f.S;
  }
}

// y = A x with the float-float stencil; x, y [S][N][3] doubles (the C ABI's layout)
__global__ void __launch_bounds__(kThreads) k_apply64(const __grid_constant__ Views V, const double* __restrict__ x,
                                                      double* __restrict__ y) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  if (!it.ok) return;
  const View& W = V.v[it.v];
  const int n = W.f.n, N = W.f.N, p = it.p, i = p % (n + 1), j = p / (n + 1);
  const float4* Ah = W.f.A + (size_t)it.s * kGroups * N;
  const float4* Al = W.F.Alo + (size_t)it.s * kGroups * N;
  const double* xs = x + (size_t)it.s * N * 3;
  auto xf = [&](int q, ff v[3]) {
    v[0] = ff_of(xs[3 * q]);
    v[1] = ff_of(xs[3 * q + 1]);
    v[2] = ff_of(xs[3 * q + 2]);
  };
  ff o[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  apply_node_ff(Ah, Al, N, n, i, j, xf, o);
#pragma unroll
  for (int c = 0; c < 3; ++c) y[((size_t)it.s * N + p) * 3 + c] = ff_dbl(o[c]);
}

__global__ void k_ff_to_aos(const float4* __restrict__ hi, const float4* __restrict__ lo, double* __restrict__ out,
                            int S, int n, double sh) {
  const int N = (n + 1) * (n + 1);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)S * N) return;
  const int p = (int)(k % N);
  const float4 h = hi[k], l = lo[k];
  out[3 * k] = (double)h.x + (double)l.x + (p % (n + 1) == n ? sh : 0.0);
  out[3 * k + 1] = (double)h.y + (double)l.y;
  out[3 * k + 2] = (double)h.z + (double)l.z;
}

}  // namespace

// ---------------------------------------------------------------- launchers

namespace {
inline unsigned per_sample_blocks(const Views& V) {
  int S = 0;
  for (int v = 0; v < V.nv; ++v) S += V.v[v].f.S;
  return (unsigned)((S + kThreads - 1) / kThreads);
}
}  // namespace

#define MLMCC_LAUNCH(KERNEL, THREADS, ...)                        \
  do {                                                            \
    if (V.nv <= 0 || V.nblk <= 0) return cudaSuccess;             \
    KERNEL<<<(unsigned)V.nblk, (THREADS), 0, st>>>(__VA_ARGS__);  \
    return cudaGetLastError();                                    \
  } while (0)

cudaError_t launch_build_fine(const Views& V, cudaStream_t st) { MLMCC_LAUNCH(k_build_fine, kThreads, V); }
cudaError_t launch_rap(const Views& V, cudaStream_t st) { MLMCC_LAUNCH(k_rap, kThreads, V); }
cudaError_t launch_coarsest_inverse(const Views& V, cudaStream_t st) {
  MLMCC_LAUNCH(k_coarsest_inverse, 32 * kGJWarps, V);
}
cudaError_t launch_pre(const Views& V, cudaStream_t st) { MLMCC_LAUNCH(k_pre, kThreads, V); }
cudaError_t launch_restrict(const Views& V, cudaStream_t st) { MLMCC_LAUNCH(k_restrict, kThreads, V); }
cudaError_t launch_bottom(const Views& V, int top_mask, cudaStream_t st) {
  MLMCC_LAUNCH(k_bottom, kBottomThreads, V, top_mask);
}
cudaError_t launch_prolong(const Views& V, cudaStream_t st) { MLMCC_LAUNCH(k_prolong, kThreads, V); }
cudaError_t launch_post(const Views& V, bool top, cudaStream_t st) { MLMCC_LAUNCH(k_post, kThreads, V, top); }
cudaError_t launch_cg_apply(const Views& V, bool odd, cudaStream_t st) {
  MLMCC_LAUNCH(k_cg_apply, kThreads, V, odd);
}
cudaError_t launch_cg_update(const Views& V, bool odd, cudaStream_t st) {
  MLMCC_LAUNCH(k_cg_update, kThreads, V, odd);
}
cudaError_t launch_resid64(const Views& V, bool first, cudaStream_t st) {
  MLMCC_LAUNCH(k_resid64, kThreads, V, first);
}
cudaError_t launch_accumulate(const Views& V, cudaStream_t st) { MLMCC_LAUNCH(k_accumulate, kThreads, V); }
cudaError_t launch_qoi(const Views& V, cudaStream_t st) { MLMCC_LAUNCH(k_qoi, kThreads, V); }
cudaError_t launch_apply64(const Views& V, const double* x, double* y, cudaStream_t st) {
  MLMCC_LAUNCH(k_apply64, kThreads, V, x, y);
}
#undef MLMCC_LAUNCH

cudaError_t launch_scal_a(const Views& V, cudaStream_t st) {
  k_scal_a<<<per_sample_blocks(V), kThreads, 0, st>>>(V);
  return cudaGetLastError();
}
cudaError_t launch_scal_b(const Views& V, int max_iter, cudaStream_t st) {
  k_scal_b<<<per_sample_blocks(V), kThreads, 0, st>>>(V, max_iter);
  return cudaGetLastError();
}
cudaError_t launch_count_active(const Views& V, int* count, cudaStream_t st) {
  k_count_active<<<per_sample_blocks(V), kThreads, 0, st>>>(V, count);
  return cudaGetLastError();
}
cudaError_t launch_outer_check(const Views& V, double rtol, int max_iter, cudaStream_t st) {
  k_outer_check<<<per_sample_blocks(V), kThreads, 0, st>>>(V, rtol, max_iter);
  return cudaGetLastError();
}
cudaError_t launch_qoi_final(const Views& V, cudaStream_t st) {
  k_qoi_final<<<per_sample_blocks(V), kThreads, 0, st>>>(V);
  return cudaGetLastError();
}
cudaError_t launch_synth_ff(const double* xi, const float* Bh, const float* Bl, int S, int n_el, int K, void* out,
                            bool trig, cudaStream_t st) {
  if (S <= 0 || n_el <= 0) return cudaSuccess;
  dim3 grid((n_el + kSynE - 1) / kSynE, (S + kSynS - 1) / kSynS);
  k_synth_ff<<<grid, 256, 0, st>>>(xi, Bh, Bl, S, n_el, K, out, trig);
  return cudaGetLastError();
}

cudaError_t launch_ff_to_aos(const float4* hi, const float4* lo, double* out, int S, int n, double sh,
                             cudaStream_t st) {
  const int64_t cnt = (int64_t)S * (n + 1) * (n + 1);
  if (cnt <= 0) return cudaSuccess;
  k_ff_to_aos<<<(unsigned)((cnt + kThreads - 1) / kThreads), kThreads, 0, st>>>(hi, lo, out, S, n, sh);
  return cudaGetLastError();
}


}  // namespace mlmcc
