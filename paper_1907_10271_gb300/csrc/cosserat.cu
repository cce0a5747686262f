// Cosserat engine kernels (Sec. 3.1 - 3.2): stencil assembly from the per-element trig
// values, Galerkin coarse operators, the V(1,1) block-Jacobi multigrid cycle, the FP32
// correction CG, the FP64 refinement residual and the strength / reaction quantities.
//
// Every kernel takes a Views table: the batches of up to kMaxViews meshes of one call,
// each with its own first block, so that all meshes advance in one launch per step.
// Threads map to (sample, node) of the view's level in sample-major order.
#include <cuda_runtime.h>

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

// y += (stencil row of node (i, j)) * x, x given per node by xf(q, v[3])
template <typename T, typename Acc, class XF>
__device__ __forceinline__ void apply_node(const T* __restrict__ A, int N, int n, int i, int j, XF xf, Acc y[3]) {
  const int p = j * (n + 1) + i;
  const int w = n + 1;
  {
    Acc v[3];
    xf(p, v);
    const Acc a00 = A[p], a01 = A[N + p], a02 = A[2 * N + p], a11 = A[3 * N + p], a12 = A[4 * N + p],
              a22 = A[5 * N + p];
    y[0] += a00 * v[0] + a01 * v[1] + a02 * v[2];
    y[1] += a01 * v[0] + a11 * v[1] + a12 * v[2];
    y[2] += a02 * v[0] + a12 * v[1] + a22 * v[2];
  }
  auto fwd = [&](int k0, int q) {
    Acc v[3];
    xf(q, v);
#pragma unroll
    for (int a = 0; a < 3; ++a)
      y[a] += (Acc)A[(k0 + 3 * a) * N + p] * v[0] + (Acc)A[(k0 + 3 * a + 1) * N + p] * v[1] +
              (Acc)A[(k0 + 3 * a + 2) * N + p] * v[2];
  };
  auto bwd = [&](int k0, int q) {
    Acc v[3];
    xf(q, v);
#pragma unroll
    for (int a = 0; a < 3; ++a)
      y[a] += (Acc)A[(k0 + a) * N + q] * v[0] + (Acc)A[(k0 + 3 + a) * N + q] * v[1] +
              (Acc)A[(k0 + 6 + a) * N + q] * v[2];
  };
  if (i < n) fwd(kE, p + 1);
  if (j < n) {
    fwd(kN, p + w);
    if (i < n) fwd(kNE, p + w + 1);
    if (i > 0) fwd(kNW, p + w - 1);
  }
  if (i > 0) bwd(kE, p - 1);
  if (j > 0) {
    bwd(kN, p - w);
    if (i > 0) bwd(kNE, p - w - 1);
    if (i < n) bwd(kNW, p - w + 1);
  }
}

// 3 x 3 block from node (i, j) to (i + ox, j + oy) (both inside), [row][column]
template <typename T>
__device__ __forceinline__ void block_of(const T* __restrict__ A, int N, int n, int i, int j, int ox, int oy,
                                         T out[9]) {
  const int p = j * (n + 1) + i;
  const int w = n + 1;
  if (ox == 0 && oy == 0) {
    out[0] = A[p];
    out[1] = out[3] = A[N + p];
    out[2] = out[6] = A[2 * N + p];
    out[4] = A[3 * N + p];
    out[5] = out[7] = A[4 * N + p];
    out[8] = A[5 * N + p];
    return;
  }
  int k0, q;
  bool tr;
  if (oy == 0) {
    tr = ox < 0;
    k0 = kE;
    q = tr ? p - 1 : p;
  } else if (ox == 0) {
    tr = oy < 0;
    k0 = kN;
    q = tr ? p - w : p;
  } else if (ox == oy) {
    tr = ox < 0;
    k0 = kNE;
    q = tr ? p - w - 1 : p;
  } else {
    tr = oy < 0;   // (+1, -1): the NW block of the south-east node, transposed
    k0 = kNW;
    q = tr ? p - w + 1 : p;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) out[3 * a + b] = tr ? A[(k0 + 3 * b + a) * N + q] : A[(k0 + 3 * a + b) * N + q];
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

// y += (stencil row of node (i, j)) * x in float-float; the stencil is (Ah, Al).
template <class XF>
__device__ __forceinline__ void apply_node_ff(const float* __restrict__ Ah, const float* __restrict__ Al, int N, int n,
                                              int i, int j, XF xf, ff y[3]) {
  const int p = j * (n + 1) + i;
  const int w = n + 1;
  auto A = [&](int k, int q) { return ff{Ah[(size_t)k * N + q], Al[(size_t)k * N + q]}; };
  {
    ff v[3];
    xf(p, v);
    const ff a00 = A(0, p), a01 = A(1, p), a02 = A(2, p), a11 = A(3, p), a12 = A(4, p), a22 = A(5, p);
    ff_fma(y[0], a00, v[0]);
    ff_fma(y[0], a01, v[1]);
    ff_fma(y[0], a02, v[2]);
    ff_fma(y[1], a01, v[0]);
    ff_fma(y[1], a11, v[1]);
    ff_fma(y[1], a12, v[2]);
    ff_fma(y[2], a02, v[0]);
    ff_fma(y[2], a12, v[1]);
    ff_fma(y[2], a22, v[2]);
  }
  auto fwd = [&](int k0, int q) {
    ff v[3];
    xf(q, v);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) ff_fma(y[a], A(k0 + 3 * a + b, p), v[b]);
  };
  auto bwd = [&](int k0, int q) {
    ff v[3];
    xf(q, v);
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
      for (int b = 0; b < 3; ++b) ff_fma(y[a], A(k0 + 3 * b + a, q), v[b]);
  };
  if (i < n) fwd(kE, p + 1);
  if (j < n) {
    fwd(kN, p + w);
    if (i < n) fwd(kNE, p + w + 1);
    if (i > 0) fwd(kNW, p + w - 1);
  }
  if (i > 0) bwd(kE, p - 1);
  if (j > 0) {
    bwd(kN, p - w);
    if (i > 0) bwd(kNE, p - w - 1);
    if (i < n) bwd(kNW, p - w + 1);
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
    float* Ah = W.f.A + (size_t)s * kStencil * N;
    float* Al = W.F.Alo + (size_t)s * kStencil * N;
    if (!self) {
      const int k0 = 6 + 9 * (slot - 1);
#pragma unroll
      for (int k = 0; k < 9; ++k) {
        Ah[(size_t)(k0 + k) * N + p] = blk[k].hi;
        Al[(size_t)(k0 + k) * N + p] = blk[k].lo;
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
        Ah[(size_t)k * N + p] = sb[k].hi;
        Al[(size_t)k * N + p] = sb[k].lo;
        sf[k] = sb[k].hi;
      }
      inv_sym3(sf, inv);   // the smoother's inverse needs no more than FP32
      float* Di = W.f.Dinv + (size_t)s * kDinv * N;
#pragma unroll
      for (int k = 0; k < 6; ++k) Di[(size_t)k * N + p] = kOmega * inv[k];
      const size_t s3 = (size_t)s * 3 * N;
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        W.F.bh[s3 + (size_t)c * N + p] = rhs[c].hi;
        W.F.bl[s3 + (size_t)c * N + p] = rhs[c].lo;
        W.F.dh[s3 + (size_t)c * N + p] = 0.f;
        W.F.dl[s3 + (size_t)c * N + p] = 0.f;
        bb += (double)rhs[c].hi * (double)rhs[c].hi;
      }
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
  const float* Af = W.f.A + (size_t)s * kStencil * Nf;
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
  float* Ac = W.c.A + (size_t)s * kStencil * Nc;
  // the diagonal block is symmetric up to rounding: keep the mean of the two triangles
  const float self[6] = {acc[0][0], 0.5f * (acc[0][1] + acc[0][3]), 0.5f * (acc[0][2] + acc[0][6]), acc[0][4],
                         0.5f * (acc[0][5] + acc[0][7]), acc[0][8]};
#pragma unroll
  for (int k = 0; k < 6; ++k) Ac[(size_t)k * Nc + P] = self[k];
#pragma unroll
  for (int b = 1; b < 5; ++b)
#pragma unroll
    for (int k = 0; k < 9; ++k) Ac[(size_t)(6 + 9 * (b - 1) + k) * Nc + P] = acc[b][k];
  float inv[6];
  inv_sym3(self, inv);
  float* Di = W.c.Dinv + (size_t)s * kDinv * Nc;
#pragma unroll
  for (int k = 0; k < 6; ++k) Di[(size_t)k * Nc + P] = kOmega * inv[k];
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
  const float* A = W.f.A + (size_t)s * kStencil * N;
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

// Pre-smoothing from zero and the residual: x = Dinv r, t = r - A x (x of the
// neighbours recomputed from their r).
__global__ void __launch_bounds__(kThreads) k_pre(const __grid_constant__ Views V) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  const View& W = V.v[it.v];
  if (!it.ok || !active(W, it.s)) return;
  const int n = W.f.n, N = W.f.N, p = it.p, i = p % (n + 1), j = p / (n + 1);
  const size_t s3 = (size_t)it.s * 3 * N;
  const float* __restrict__ A = W.f.A + (size_t)it.s * kStencil * N;
  const float* __restrict__ D = W.f.Dinv + (size_t)it.s * kDinv * N;
  const float* __restrict__ r = W.f.r + s3;
  auto xf = [&](int q, float v[3]) {
    const float r0 = r[q], r1 = r[N + q], r2 = r[2 * N + q];
    const float d0 = D[q], d1 = D[N + q], d2 = D[2 * N + q], d3 = D[3 * N + q], d4 = D[4 * N + q],
                d5 = D[5 * N + q];
    v[0] = d0 * r0 + d1 * r1 + d2 * r2;
    v[1] = d1 * r0 + d3 * r1 + d4 * r2;
    v[2] = d2 * r0 + d4 * r1 + d5 * r2;
  };
  float x[3], y[3] = {0.f, 0.f, 0.f};
  xf(p, x);
  apply_node(A, N, n, i, j, xf, y);
  float* xo = W.f.x + s3;
  float* to = W.f.t + s3;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    xo[(size_t)c * N + p] = x[c];
    to[(size_t)c * N + p] = r[(size_t)c * N + p] - y[c];
  }
}

// Restriction c.r = P^T f.t, zero at the coarse Dirichlet DOFs.
__global__ void __launch_bounds__(kThreads) k_restrict(const __grid_constant__ Views V) {
  const Item it = item_of(V, V.v[view_of(V)].c.N);
  const View& W = V.v[it.v];
  if (!it.ok || !active(W, it.s)) return;
  const int nc = W.c.n, Nc = W.c.N, nf = W.f.n, Nf = W.f.N, P = it.p, I = P % (nc + 1), J = P / (nc + 1);
  const float* __restrict__ t = W.f.t + (size_t)it.s * 3 * Nf;
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int dy = -1; dy <= 1; ++dy)
#pragma unroll
    for (int dx = -1; dx <= 1; ++dx) {
      const int pi = 2 * I + dx, pj = 2 * J + dy;
      if (pi < 0 || pj < 0 || pi > nf || pj > nf) continue;
      const float w = (dx ? 0.5f : 1.f) * (dy ? 0.5f : 1.f);
      const int p = pj * (nf + 1) + pi;
#pragma unroll
      for (int c = 0; c < 3; ++c) acc[c] += w * t[(size_t)c * Nf + p];
    }
  const int dm = dmask(I, J, nc);
  if (dm & 1) acc[0] = 0.f;
  if (dm & 2) acc[1] = 0.f;
  float* rc = W.c.r + (size_t)it.s * 3 * Nc;
#pragma unroll
  for (int c = 0; c < 3; ++c) rc[(size_t)c * Nc + P] = acc[c];
}

// Coarsest level: f.t = Ainv f.r, one thread per (sample, DOF).
__global__ void __launch_bounds__(kThreads) k_coarse_solve(const __grid_constant__ Views V) {
  const Item it = item_of(V, kCoarseDofs);
  const View& W = V.v[it.v];
  if (!it.ok || !active(W, it.s)) return;
  const int N = W.f.N, row = it.p;
  const float* __restrict__ r = W.f.r + (size_t)it.s * 3 * N;
  const float* __restrict__ M = W.Ainv + ((size_t)it.s * kCoarseDofs + row) * kCoarseDofs;
  float acc = 0.f;
#pragma unroll
  for (int k = 0; k < kCoarseDofs; ++k) acc += M[k] * r[(size_t)(k % 3) * N + k / 3];
  W.f.t[(size_t)it.s * 3 * N + (size_t)(row % 3) * N + row / 3] = acc;
}

// Prolongation f.x += P c.t (bilinear).
__global__ void __launch_bounds__(kThreads) k_prolong(const __grid_constant__ Views V) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  const View& W = V.v[it.v];
  if (!it.ok || !active(W, it.s)) return;
  const int nf = W.f.n, Nf = W.f.N, nc = W.c.n, Nc = W.c.N, p = it.p, i = p % (nf + 1), j = p / (nf + 1);
  const float* __restrict__ xc = W.c.t + (size_t)it.s * 3 * Nc;
  const int I0 = i >> 1, J0 = j >> 1;
  const bool ox = i & 1, oy = j & 1;
  float acc[3] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int b = 0; b < 4; ++b) {
    const int di = b & 1, dj = b >> 1;
    if ((di && !ox) || (dj && !oy)) continue;
    const float w = (ox ? 0.5f : 1.f) * (oy ? 0.5f : 1.f);
    const int P = (J0 + dj) * (nc + 1) + I0 + di;
#pragma unroll
    for (int c = 0; c < 3; ++c) acc[c] += w * xc[(size_t)c * Nc + P];
  }
  float* x = W.f.x + (size_t)it.s * 3 * Nf;
#pragma unroll
  for (int c = 0; c < 3; ++c) x[(size_t)c * Nf + p] += acc[c];
}

// Post-smoothing: f.t = x + Dinv (r - A x). On the solve mesh (top) f.t is the
// preconditioned residual z and r . z is accumulated into rz_new.
__global__ void __launch_bounds__(kThreads) k_post(const __grid_constant__ Views V, bool top) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  const View& W = V.v[it.v];
  const bool ok = it.ok && active(W, it.s);
  double rz = 0.0;
  if (ok) {
    const int n = W.f.n, N = W.f.N, p = it.p, i = p % (n + 1), j = p / (n + 1);
    const size_t s3 = (size_t)it.s * 3 * N;
    const float* __restrict__ A = W.f.A + (size_t)it.s * kStencil * N;
    const float* __restrict__ D = W.f.Dinv + (size_t)it.s * kDinv * N;
    const float* __restrict__ r = W.f.r + s3;
    const float* __restrict__ x = W.f.x + s3;
    auto xf = [&](int q, float v[3]) {
      v[0] = x[q];
      v[1] = x[N + q];
      v[2] = x[2 * N + q];
    };
    float y[3] = {0.f, 0.f, 0.f};
    apply_node(A, N, n, i, j, xf, y);
    const float e0 = r[p] - y[0], e1 = r[N + p] - y[1], e2 = r[2 * N + p] - y[2];
    const float d0 = D[p], d1 = D[N + p], d2 = D[2 * N + p], d3 = D[3 * N + p], d4 = D[4 * N + p],
                d5 = D[5 * N + p];
    const float z0 = x[p] + d0 * e0 + d1 * e1 + d2 * e2;
    const float z1 = x[N + p] + d1 * e0 + d3 * e1 + d4 * e2;
    const float z2 = x[2 * N + p] + d2 * e0 + d4 * e1 + d5 * e2;
    float* t = W.f.t + s3;
    t[p] = z0;
    t[N + p] = z1;
    t[2 * N + p] = z2;
    if (top) rz = (double)r[p] * z0 + (double)r[N + p] * z1 + (double)r[2 * N + p] * z2;
  }
  if (top) {
    SampleState* st = W.F.st;
    warp_add_by_sample(rz, ok ? it.s : -1, [&](int k) { return &st[k].rz_new; });
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
    const size_t s3 = (size_t)it.s * 3 * N;
    const float* __restrict__ A = W.f.A + (size_t)it.s * kStencil * N;
    const float* __restrict__ z = W.f.t + s3;
    const float* __restrict__ pin = (odd ? W.F.p1 : W.F.p0) + s3;
    float* pout = (odd ? W.F.p0 : W.F.p1) + s3;
    const float beta = (float)W.F.st[it.s].beta;
    auto pf = [&](int q, float v[3]) {
      if (beta == 0.f) {
        v[0] = z[q];
        v[1] = z[N + q];
        v[2] = z[2 * N + q];
      } else {
        v[0] = z[q] + beta * pin[q];
        v[1] = z[N + q] + beta * pin[N + q];
        v[2] = z[2 * N + q] + beta * pin[2 * N + q];
      }
    };
    float pv[3], y[3] = {0.f, 0.f, 0.f};
    pf(p, pv);
    apply_node(A, N, n, i, j, pf, y);
    float* qv = W.F.q + s3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      pout[(size_t)c * N + p] = pv[c];
      qv[(size_t)c * N + p] = y[c];
      pq += (double)pv[c] * y[c];
    }
  }
  SampleState* st = W.F.st;
  warp_add_by_sample(pq, ok ? it.s : -1, [&](int k) { return &st[k].pq; });
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

// c += alpha p_out, r -= alpha q, |r|^2.
__global__ void __launch_bounds__(kThreads) k_cg_update(const __grid_constant__ Views V, bool odd) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  const View& W = V.v[it.v];
  const bool ok = it.ok && active(W, it.s);
  double rr = 0.0;
  if (ok) {
    const int N = W.f.N, p = it.p;
    const size_t s3 = (size_t)it.s * 3 * N;
    const float a = (float)W.F.st[it.s].alpha;
    const float* __restrict__ pv = (odd ? W.F.p0 : W.F.p1) + s3;
    const float* __restrict__ qv = W.F.q + s3;
    float* c = W.F.c + s3;
    float* r = W.f.r + s3;
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const size_t o = (size_t)k * N + p;
      c[o] += a * pv[o];
      const float rn = r[o] - a * qv[o];
      r[o] = rn;
      rr += (double)rn * rn;
    }
  }
  SampleState* st = W.F.st;
  warp_add_by_sample(rr, ok ? it.s : -1, [&](int k) { return &st[k].rr; });
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
    const size_t s3 = (size_t)it.s * 3 * N;
    ff y[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
    if (!first) {
      const float* __restrict__ Ah = W.f.A + (size_t)it.s * kStencil * N;
      const float* __restrict__ Al = W.F.Alo + (size_t)it.s * kStencil * N;
      const float* __restrict__ dh = W.F.dh + s3;
      const float* __restrict__ dl = W.F.dl + s3;
      auto xf = [&](int q, ff v[3]) {
        v[0] = ff{dh[q], dl[q]};
        v[1] = ff{dh[N + q], dl[N + q]};
        v[2] = ff{dh[2 * N + q], dl[2 * N + q]};
      };
      apply_node_ff(Ah, Al, N, n, i, j, xf, y);
    }
    float* r = W.f.r + s3;
#pragma unroll
    for (int c = 0; c < 3; ++c) {
      // e = b - y: b + (-y) in float-float, then rounded
      ff e{W.F.bh[s3 + (size_t)c * N + p], W.F.bl[s3 + (size_t)c * N + p]};
      ff_fma(e, y[c], -1.f);
      const float ev = __fadd_rn(e.hi, e.lo);
      r[(size_t)c * N + p] = ev;
      rr += (double)ev * (double)ev;
    }
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
  const int N = W.f.N;
  const size_t s3 = (size_t)it.s * 3 * N;
  float* c = W.F.c + s3;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const size_t o = (size_t)k * N + it.p;
    ff d{W.F.dh[s3 + o], W.F.dl[s3 + o]};
    ff_fma(d, ff{c[o], 0.f}, 1.f);
    W.F.dh[s3 + o] = d.hi;
    W.F.dl[s3 + o] = d.lo;
    c[o] = 0.f;
  }
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
    const float* __restrict__ dh = W.F.dh + (size_t)it.s * 3 * N;
    const float* __restrict__ dl = W.F.dl + (size_t)it.s * 3 * N;
    double de[12];
    const int cx[4] = {0, 1, 1, 0}, cy[4] = {0, 0, 1, 1};
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int q = (je + cy[a]) * (n + 1) + ie + cx[a];
#pragma unroll
      for (int c = 0; c < 3; ++c) de[3 * a + c] = (double)dh[(size_t)c * N + q] + (double)dl[(size_t)c * N + q];
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

__global__ void __launch_bounds__(kThreads) k_apply64(const __grid_constant__ Views V, const double* __restrict__ x,
                                                      double* __restrict__ y) {
  const Item it = item_of(V, V.v[view_of(V)].f.N);
  if (!it.ok) return;
  const View& W = V.v[it.v];
  const int n = W.f.n, N = W.f.N, p = it.p, i = p % (n + 1), j = p / (n + 1);
  const size_t s3 = (size_t)it.s * 3 * N;
  const float* Ah = W.f.A + (size_t)it.s * kStencil * N;
  const float* Al = W.F.Alo + (size_t)it.s * kStencil * N;
  const double* xs = x + s3;
  auto xf = [&](int q, ff v[3]) {
    v[0] = ff_of(xs[q]);
    v[1] = ff_of(xs[N + q]);
    v[2] = ff_of(xs[2 * N + q]);
  };
  ff o[3] = {{0.f, 0.f}, {0.f, 0.f}, {0.f, 0.f}};
  apply_node_ff(Ah, Al, N, n, i, j, xf, o);
#pragma unroll
  for (int c = 0; c < 3; ++c) y[s3 + (size_t)c * N + p] = ff_dbl(o[c]);
}

__global__ void k_aos_to_soa(const double* __restrict__ in, double* __restrict__ out, int S, int N) {
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)S * N * 3) return;
  const int64_t s = k / (3 * N), r = k % (3 * N), p = r / 3, c = r % 3;
  out[(s * 3 + c) * N + p] = in[k];
}

__global__ void k_soa_to_aos(const double* __restrict__ in, double* __restrict__ out, int S, int n, bool lift,
                             double sh) {
  const int N = (n + 1) * (n + 1);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)S * N * 3) return;
  const int64_t s = k / (3 * N), r = k % (3 * N), p = r / 3, c = r % 3;
  double v = in[(s * 3 + c) * N + p];
  if (lift && c == 0 && p % (n + 1) == n) v += sh;
  out[k] = v;
}

__global__ void k_ff_to_aos(const float* __restrict__ hi, const float* __restrict__ lo, double* __restrict__ out, int S,
                            int n, double sh) {
  const int N = (n + 1) * (n + 1);
  const int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= (int64_t)S * N * 3) return;
  const int64_t s = k / (3 * N), r = k % (3 * N), p = r / 3, c = r % 3;
  const int64_t o = (s * 3 + c) * N + p;
  double v = (double)hi[o] + (double)lo[o];
  if (c == 0 && p % (n + 1) == n) v += sh;
  out[k] = v;
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
cudaError_t launch_coarse_solve(const Views& V, cudaStream_t st) { MLMCC_LAUNCH(k_coarse_solve, kThreads, V); }
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

cudaError_t launch_ff_to_aos(const float* hi, const float* lo, double* out, int S, int n, double sh, cudaStream_t st) {
  const int64_t cnt = (int64_t)S * (n + 1) * (n + 1) * 3;
  if (cnt <= 0) return cudaSuccess;
  k_ff_to_aos<<<(unsigned)((cnt + kThreads - 1) / kThreads), kThreads, 0, st>>>(hi, lo, out, S, n, sh);
  return cudaGetLastError();
}

cudaError_t launch_aos_to_soa(const double* in, double* out, int S, int N, cudaStream_t st) {
  const int64_t n = (int64_t)S * N * 3;
  if (n <= 0) return cudaSuccess;
  k_aos_to_soa<<<(unsigned)((n + kThreads - 1) / kThreads), kThreads, 0, st>>>(in, out, S, N);
  return cudaGetLastError();
}
cudaError_t launch_soa_to_aos(const double* in, double* out, int S, int n, bool add_lift, double sh,
                              cudaStream_t st) {
  const int64_t cnt = (int64_t)S * (n + 1) * (n + 1) * 3;
  if (cnt <= 0) return cudaSuccess;
  k_soa_to_aos<<<(unsigned)((cnt + kThreads - 1) / kThreads), kThreads, 0, st>>>(in, out, S, n, add_lift, sh);
  return cudaGetLastError();
}

}  // namespace mlmcc
