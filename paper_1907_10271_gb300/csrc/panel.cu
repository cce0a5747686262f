// Panel-buckling kernels: laminate (Eq. CLTABD), Reissner-Mindlin Q4 operators
// (Eq. MomentWeakForm), the multigrid V-cycle on K, and the LOBPCG steps for the
// largest mu of G d = mu K d (Eq. matrixeig, lambda = 1 / mu).
//
// Every sample's plate has constant coefficients (its laminate is uniform over the
// panel), so one 12 x 12 element matrix per sample and mesh describes K entirely; the
// node-centric kernels keep it in shared memory and each node forms its own three rows
// from the (up to) four elements around it. The geometric form with the 1-point rule
// is sample-independent: G_e = hy / (4 hx) s s^T on the w-DOFs, s = (-1, 1, 1, -1).
#include "dfloat.cuh"
#include "panel.cuh"

#include <algorithm>
#include <cmath>

#include "../../include/mlmc.h"

namespace mlmcp {
namespace {

constexpr int kThreads = 128;
constexpr int kPatchesPerWarp = 3;   // patches of one colour per warp in the patch sweep (27 of 32 lanes)

// corner a of an element at offset (ox, oy) from its lower-left node
__device__ __forceinline__ int corner_of(int ox, int oy) { return oy == 0 ? ox : 3 - ox; }
__device__ __forceinline__ int corner_x(int a) { return (a == 1 || a == 2) ? 1 : 0; }
__device__ __forceinline__ int corner_y(int a) { return a >= 2 ? 1 : 0; }

// which DOFs of node (i, j) are free (w held on the boundary; with hard support the
// tangential rotation too)
struct Free {
  bool w, tx, ty;
};
__device__ __forceinline__ Free free_of(const PGrid& g, int i, int j) {
  const bool bx = i == 0 || i == g.nx, by = j == 0 || j == g.ny;
  return Free{!(bx || by), !(g.hard && by), !(g.hard && bx)};
}
__device__ __forceinline__ float4 masked(const Free& f, float4 v) {
  return make_float4(f.w ? v.x : 0.f, f.tx ? v.y : 0.f, f.ty ? v.z : 0.f, 0.f);
}

__device__ __forceinline__ double warp_sum_d(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

__global__ void k_laminate(Laminate lam, const double* __restrict__ xi, int n, double* __restrict__ dstar,
                           double* __restrict__ kgt) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  // lamina stiffness (plane stress)
  const double nu21 = lam.nu12 * lam.E22 / lam.E11;
  const double den = 1.0 - lam.nu12 * nu21;
  const double q11 = lam.E11 / den, q22 = lam.E22 / den, q12 = lam.nu12 * lam.E22 / den, q66 = lam.G12;
  double A[6] = {0, 0, 0, 0, 0, 0}, B[6] = {0, 0, 0, 0, 0, 0}, D[6] = {0, 0, 0, 0, 0, 0};   // 11 12 16 22 26 66
  const double t = lam.t_ply * lam.n_plies;
  for (int k = 0; k < lam.n_plies; ++k) {
    const double th = lam.psi[k] + lam.std_rad * xi[(size_t)s * lam.n_plies + k];
    const double c = cos(th), sn = sin(th);
    const double c2 = c * c, s2 = sn * sn, cs = c * sn;
    // transformed reduced stiffness, angle from the x axis to the fibre
    const double Qb[6] = {
        q11 * c2 * c2 + 2.0 * (q12 + 2.0 * q66) * s2 * c2 + q22 * s2 * s2,
        (q11 + q22 - 4.0 * q66) * s2 * c2 + q12 * (s2 * s2 + c2 * c2),
        (q11 - q12 - 2.0 * q66) * cs * c2 + (q12 - q22 + 2.0 * q66) * cs * s2,
        q11 * s2 * s2 + 2.0 * (q12 + 2.0 * q66) * s2 * c2 + q22 * c2 * c2,
        (q11 - q12 - 2.0 * q66) * cs * s2 + (q12 - q22 + 2.0 * q66) * cs * c2,
        (q11 + q22 - 2.0 * q12 - 2.0 * q66) * s2 * c2 + q66 * (s2 * s2 + c2 * c2)};
    const double z0 = -0.5 * t + k * lam.t_ply, z1 = z0 + lam.t_ply;
    for (int m = 0; m < 6; ++m) {
      A[m] += Qb[m] * (z1 - z0);
      B[m] += 0.5 * Qb[m] * (z1 * z1 - z0 * z0);
      D[m] += Qb[m] * (z1 * z1 * z1 - z0 * z0 * z0) / 3.0;
    }
  }
  // D* = D - B A^-1 B with symmetric 3x3 matrices stored as (11 12 16 22 26 66)
  const double a11 = A[0], a12 = A[1], a13 = A[2], a22 = A[3], a23 = A[4], a33 = A[5];
  const double c11 = a22 * a33 - a23 * a23, c12 = a13 * a23 - a12 * a33, c13 = a12 * a23 - a13 * a22;
  const double c22 = a11 * a33 - a13 * a13, c23 = a12 * a13 - a11 * a23, c33 = a11 * a22 - a12 * a12;
  const double det = a11 * c11 + a12 * c12 + a13 * c13;
  const double Ai[3][3] = {{c11 / det, c12 / det, c13 / det}, {c12 / det, c22 / det, c23 / det},
                           {c13 / det, c23 / det, c33 / det}};
  const double Bm[3][3] = {{B[0], B[1], B[2]}, {B[1], B[3], B[4]}, {B[2], B[4], B[5]}};
  double T[3][3];
  for (int r = 0; r < 3; ++r)
    for (int c = 0; c < 3; ++c) T[r][c] = Ai[r][0] * Bm[0][c] + Ai[r][1] * Bm[1][c] + Ai[r][2] * Bm[2][c];
  const int rr[6] = {0, 0, 0, 1, 1, 2}, cc[6] = {0, 1, 2, 1, 2, 2};
  for (int m = 0; m < 6; ++m) {
    const int r = rr[m], c = cc[m];
    dstar[(size_t)s * 6 + m] = D[m] - (Bm[r][0] * T[0][c] + Bm[r][1] * T[1][c] + Bm[r][2] * T[2][c]);
  }
  kgt[s] = lam.k_shear * lam.G13 * t;
}

// bending column (kappa_x, kappa_y, kappa_xy) and shear column (gamma_x, gamma_y) of
// local DOF q = 3 a + comp at (xi, eta)
__device__ void b_columns(int q, double xi, double eta, double hx, double hy, double bb[3], double bs[2]) {
  const int a = q / 3, comp = q - 3 * a;
  const double sx = corner_x(a) ? 1.0 : -1.0, sy = corner_y(a) ? 1.0 : -1.0;
  const double N = 0.25 * (1.0 + sx * xi) * (1.0 + sy * eta);
  const double dx = 0.25 * sx * (1.0 + sy * eta) * 2.0 / hx;
  const double dy = 0.25 * sy * (1.0 + sx * xi) * 2.0 / hy;
  bb[0] = bb[1] = bb[2] = 0.0;
  bs[0] = bs[1] = 0.0;
  if (comp == 0) {
    bs[0] = dx;
    bs[1] = dy;
  } else if (comp == 1) {
    bb[0] = dx;
    bb[2] = dy;
    bs[0] = -N;
  } else {
    bb[1] = dy;
    bb[2] = dx;
    bs[1] = -N;
  }
}

__global__ void k_element(const double* __restrict__ dstar, const double* __restrict__ kgt, int n, double hx,
                          double hy, float* __restrict__ k32, double* __restrict__ k64) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (int64_t)n * 144) return;
  const int s = (int)(t / 144), e = (int)(t - (int64_t)s * 144);
  const int p = e / 12, q = e - 12 * p;
  const double* d = dstar + (size_t)s * 6;
  const double D[3][3] = {{d[0], d[1], d[2]}, {d[1], d[3], d[4]}, {d[2], d[4], d[5]}};
  const double det = 0.25 * hx * hy, g = 0.577350269189625764509148780502;
  double v = 0.0;
  double bp[3], bq[3], sp[2], sq[2];
  for (int gy = 0; gy < 2; ++gy)
    for (int gx = 0; gx < 2; ++gx) {
      const double xi = gx ? g : -g, eta = gy ? g : -g;
      b_columns(p, xi, eta, hx, hy, bp, sp);
      b_columns(q, xi, eta, hx, hy, bq, sq);
      double m = 0.0;
      for (int r = 0; r < 3; ++r) m += bp[r] * (D[r][0] * bq[0] + D[r][1] * bq[1] + D[r][2] * bq[2]);
      v += det * m;
    }
  b_columns(p, 0.0, 0.0, hx, hy, bp, sp);
  b_columns(q, 0.0, 0.0, hx, hy, bq, sq);
  v += kgt[s] * 4.0 * det * (sp[0] * sq[0] + sp[1] * sq[1]);
  if (k32) k32[t] = (float)v;
  if (k64) k64[t] = v;
}

// K x (rows of node (i, j)) with the element matrix K in shared memory; the G x w-row
// in *gw; optionally the node's 3x3 diagonal block of K in diag (11 12 13 22 23 33)
template <bool DIAG>
__device__ __forceinline__ float4 node_kx(const PGrid& g, const float* K, const float4* xe, int i, int j, bool bc,
                                          float* gw, float* diag) {
  const int np = g.nx + 1;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f, gsum_all = 0.f;
  // both loops unroll, so the node's corner index a in each element is a constant; the
  // element matrix (16-byte aligned rows of 12) is read as float4s from shared memory
#pragma unroll
  for (int oy = 0; oy < 2; ++oy)
#pragma unroll
    for (int ox = 0; ox < 2; ++ox) {
      const int ei = i - ox, ej = j - oy;   // element whose corner (ox, oy) is this node
      if (ei < 0 || ej < 0 || ei >= g.nx || ej >= g.ny) continue;
      const int a = corner_of(ox, oy);
      const float* Ka = K + 36 * a;   // rows 3a .. 3a+2
      float gs = 0.f;
      if (xe) {
        float4 v[4];
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int ni = ei + corner_x(c), nj = ej + corner_y(c);
          v[c] = xe[nj * np + ni];
          if (bc) v[c] = masked(free_of(g, ni, nj), v[c]);
          gs += corner_x(c) ? v[c].x : -v[c].x;
        }
        float acc[3];
#pragma unroll
        for (int rr = 0; rr < 3; ++rr) {
          const float4* R = reinterpret_cast<const float4*>(Ka + 12 * rr);
          const float4 k0 = R[0], k1 = R[1], k2 = R[2];   // columns 0-3, 4-7, 8-11
          acc[rr] = k0.x * v[0].x + k0.y * v[0].y + k0.z * v[0].z + k0.w * v[1].x + k1.x * v[1].y +
                    k1.y * v[1].z + k1.z * v[2].x + k1.w * v[2].y + k2.x * v[2].z + k2.y * v[3].x + k2.z * v[3].y +
                    k2.w * v[3].z;
        }
        a0 += acc[0];
        a1 += acc[1];
        a2 += acc[2];
      }
      gsum_all += corner_x(a) ? gs : -gs;
      if (DIAG) {
        const float* r = Ka + 3 * a;
        diag[0] += r[0];
        diag[1] += r[1];
        diag[2] += r[2];
        diag[3] += r[13];
        diag[4] += r[14];
        diag[5] += r[26];
      }
    }
  if (gw) *gw = gsum_all * (g.hy / (4.f * g.hx));
  return make_float4(a0, a1, a2, 0.f);
}

__global__ void __launch_bounds__(kThreads) k_apply(PGrid g, const float* __restrict__ ke, const float4* __restrict__ x,
                                                    const float4* __restrict__ b, float4* __restrict__ out,
                                                    float4* __restrict__ gout, const int* __restrict__ active, int bc) {
  const int e = blockIdx.y, s = e >> g.cshift;
  if (active && !active[s]) return;
  __shared__ __align__(16) float K[144];
  for (int k = threadIdx.x; k < 144; k += blockDim.x) K[k] = ke[(size_t)s * 144 + k];
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nn = g.nodes();
  if (t >= nn) return;
  const int i = t % (g.nx + 1), j = t / (g.nx + 1);
  const size_t o = (size_t)e * nn;
  float gw = 0.f;
  float4 y = node_kx<false>(g, K, x + o, i, j, bc != 0, gout ? &gw : nullptr, nullptr);
  if (b) {
    const float4 bb = b[o + t];
    y = make_float4(bb.x - y.x, bb.y - y.y, bb.z - y.z, 0.f);
  }
  const Free f = free_of(g, i, j);
  if (bc) y = masked(f, y);
  out[o + t] = y;
  if (gout) gout[o + t] = make_float4((bc && !f.w) ? 0.f : gw, 0.f, 0.f, 0.f);
}

// K x with the element matrix of double accuracy and float-float sums (the vector itself
// single, w in two parts): for thin plates, whose transverse shear strain grad w - theta
// is a small difference of large terms, a single-precision sum keeps only a few digits
// of it. The double element matrix is split into float-float pairs in shared memory and
// every product and sum runs on the FP32 pipes (Knuth / Dekker transformations): GB300's
// FP64 rate is a small fraction of its FP32 rate. G x in single precision (no
// cancellation). Rounded to single at the end.
__global__ void __launch_bounds__(kThreads) k_apply64(PGrid g, const double* __restrict__ ke64,
                                                      const float4* __restrict__ x, float4* __restrict__ out,
                                                      float4* __restrict__ gout, float4* __restrict__ rout,
                                                      const double* __restrict__ mu, const int* __restrict__ active) {
  using mlmc::DF;
  const int e = blockIdx.y, s = e >> g.cshift;
  if (active && !active[s]) return;
  __shared__ float Kh[144], Kl[144];
  for (int k = threadIdx.x; k < 144; k += blockDim.x) {
    const DF v = mlmc::df_from_double(ke64[(size_t)s * 144 + k]);
    Kh[k] = v.hi;
    Kl[k] = v.lo;
  }
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nn = g.nodes();
  if (t >= nn) return;
  const int i = t % (g.nx + 1), j = t / (g.nx + 1), np = g.nx + 1;
  const float4* xe = x + (size_t)e * nn;
  DF a0{0.f, 0.f}, a1{0.f, 0.f}, a2{0.f, 0.f}, gsum{0.f, 0.f};
#pragma unroll
  for (int oy = 0; oy < 2; ++oy)
#pragma unroll
    for (int ox = 0; ox < 2; ++ox) {
      const int ei = i - ox, ej = j - oy;
      if (ei < 0 || ej < 0 || ei >= g.nx || ej >= g.ny) continue;
      const int a = corner_of(ox, oy);
      const float* Ha = Kh + 36 * a;
      const float* La = Kl + 36 * a;
      DF gs{0.f, 0.f};
#pragma unroll
      for (int c = 0; c < 4; ++c) {
        const int ni = ei + corner_x(c), nj = ej + corner_y(c);
        const Free fc = free_of(g, ni, nj);
        const float4 v = xe[nj * np + ni];
        // w in two parts (high in x, low in w; the low part is zero for vectors kept in
        // one float)
        const DF vw = fc.w ? DF{v.x, v.w} : DF{0.f, 0.f};
        const DF vx = mlmc::df(fc.tx ? v.y : 0.f), vy = mlmc::df(fc.ty ? v.z : 0.f);
        const int r = 3 * c;
        mlmc::df_fma(a0, DF{Ha[r], La[r]}, vw);
        mlmc::df_fma(a0, DF{Ha[r + 1], La[r + 1]}, vx);
        mlmc::df_fma(a0, DF{Ha[r + 2], La[r + 2]}, vy);
        mlmc::df_fma(a1, DF{Ha[r + 12], La[r + 12]}, vw);
        mlmc::df_fma(a1, DF{Ha[r + 13], La[r + 13]}, vx);
        mlmc::df_fma(a1, DF{Ha[r + 14], La[r + 14]}, vy);
        mlmc::df_fma(a2, DF{Ha[r + 24], La[r + 24]}, vw);
        mlmc::df_fma(a2, DF{Ha[r + 25], La[r + 25]}, vx);
        mlmc::df_fma(a2, DF{Ha[r + 26], La[r + 26]}, vy);
        gs = corner_x(c) ? gs + vw : gs - vw;
      }
      gsum = corner_x(a) ? gsum + gs : gsum - gs;
    }
  const Free f = free_of(g, i, j);
  const double d0 = mlmc::df_to_double(a0), d1 = mlmc::df_to_double(a1), d2 = mlmc::df_to_double(a2);
  const double gw = f.w ? mlmc::df_to_double(gsum) * ((double)g.hy / (4.0 * (double)g.hx)) : 0.0;
  const size_t o = (size_t)e * nn + t;
  out[o] = masked(f, make_float4((float)d0, (float)d1, (float)d2, 0.f));
  if (gout) gout[o] = make_float4((float)gw, 0.f, 0.f, 0.f);
  if (rout) {   // R = G x - mu K x of the entry's column
    const double m = mu[(size_t)s * kCols + (e & ((1 << g.cshift) - 1))];
    rout[o] = masked(f, make_float4((float)(gw - m * d0), (float)(-m * d1), (float)(-m * d2), 0.f));
  }
}

__global__ void __launch_bounds__(kThreads) k_smooth(PGrid g, const float* __restrict__ ke, const float4* __restrict__ b,
                                                     const float4* __restrict__ x, float4* __restrict__ out,
                                                     const int* __restrict__ active) {
  const int e = blockIdx.y, s = e >> g.cshift;
  if (active && !active[s]) return;
  __shared__ __align__(16) float K[144];
  for (int k = threadIdx.x; k < 144; k += blockDim.x) K[k] = ke[(size_t)s * 144 + k];
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nn = g.nodes();
  if (t >= nn) return;
  const int i = t % (g.nx + 1), j = t / (g.nx + 1);
  const size_t o = (size_t)e * nn;
  float d[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  const float4 kx = node_kx<true>(g, K, x ? x + o : nullptr, i, j, true, nullptr, d);
  const Free f = free_of(g, i, j);
  const float4 bb = b[o + t];
  float r0 = f.w ? bb.x - kx.x : 0.f, r1 = f.tx ? bb.y - kx.y : 0.f, r2 = f.ty ? bb.z - kx.z : 0.f;
  // restrict the block to the free DOFs (identity rows for the held ones)
  if (!f.w) {
    d[0] = 1.f;
    d[1] = d[2] = 0.f;
  }
  if (!f.tx) {
    d[3] = 1.f;
    d[1] = d[4] = 0.f;
  }
  if (!f.ty) {
    d[5] = 1.f;
    d[2] = d[4] = 0.f;
  }
  // inverse of the symmetric block by cofactors
  const float c00 = d[3] * d[5] - d[4] * d[4], c01 = d[2] * d[4] - d[1] * d[5], c02 = d[1] * d[4] - d[2] * d[3];
  const float c11 = d[0] * d[5] - d[2] * d[2], c12 = d[1] * d[2] - d[0] * d[4], c22 = d[0] * d[3] - d[1] * d[1];
  const float inv = kOmegaP / (d[0] * c00 + d[1] * c01 + d[2] * c02);
  const float u0 = inv * (c00 * r0 + c01 * r1 + c02 * r2);
  const float u1 = inv * (c01 * r0 + c11 * r1 + c12 * r2);
  const float u2 = inv * (c02 * r0 + c12 * r1 + c22 * r2);
  float4 xo = x ? x[o + t] : make_float4(0.f, 0.f, 0.f, 0.f);
  out[o + t] = masked(f, make_float4(xo.x + u0, xo.y + u1, xo.z + u2, 0.f));
}

__global__ void __launch_bounds__(kThreads) k_restrict(PGrid gf, PGrid gc, const float4* __restrict__ rf,
                                                       float4* __restrict__ bc, const int* __restrict__ active) {
  const int e = blockIdx.y, s = e >> gc.cshift;
  if (active && !active[s]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nc = gc.nodes(), nf = gf.nodes();
  if (t >= nc) return;
  const int I = t % (gc.nx + 1), J = t / (gc.nx + 1);
  const float4* r = rf + (size_t)e * nf;
  float a0 = 0.f, a1 = 0.f, a2 = 0.f;
  for (int dj = -1; dj <= 1; ++dj) {
    const int fj = 2 * J + dj;
    if (fj < 0 || fj > gf.ny) continue;
    for (int di = -1; di <= 1; ++di) {
      const int fi = 2 * I + di;
      if (fi < 0 || fi > gf.nx) continue;
      const float w = (di ? 0.5f : 1.f) * (dj ? 0.5f : 1.f);
      const float4 v = r[fj * (gf.nx + 1) + fi];
      a0 += w * v.x;
      a1 += w * v.y;
      a2 += w * v.z;
    }
  }
  bc[(size_t)e * nc + t] = masked(free_of(gc, I, J), make_float4(a0, a1, a2, 0.f));
}

__global__ void __launch_bounds__(kThreads) k_prolong(PGrid gf, PGrid gc, const float4* __restrict__ xc,
                                                      float4* __restrict__ xf, const int* __restrict__ active) {
  const int e = blockIdx.y, s = e >> gf.cshift;
  if (active && !active[s]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nf = gf.nodes(), nc = gc.nodes();
  if (t >= nf) return;
  const int i = t % (gf.nx + 1), j = t / (gf.nx + 1);
  const float4* c = xc + (size_t)e * nc;
  const int I0 = i >> 1, J0 = j >> 1, I1 = (i & 1) ? I0 + 1 : I0, J1 = (j & 1) ? J0 + 1 : J0;
  const int cp = gc.nx + 1;
  const float4 v00 = c[J0 * cp + I0], v10 = c[J0 * cp + I1], v01 = c[J1 * cp + I0], v11 = c[J1 * cp + I1];
  const float4 xo = xf[(size_t)e * nf + t];
  const float4 p = make_float4(0.25f * (v00.x + v10.x + v01.x + v11.x), 0.25f * (v00.y + v10.y + v01.y + v11.y),
                               0.25f * (v00.z + v10.z + v01.z + v11.z), 0.f);
  xf[(size_t)e * nf + t] = masked(free_of(gf, i, j), make_float4(xo.x + p.x, xo.y + p.y, xo.z + p.z, 0.f));
}

// ---------------------------------------------------------------- patch smoother
// boundary case of a patch centre c on an axis of n elements: -1, 0, 1 -> 0, 1, 2;
// interior -> 3; n - 1, n, n + 1 -> 4, 5, 6 (n >= 4: the cases are distinct)
__device__ __forceinline__ int patch_case(int c, int n) {
  if (c <= 1) return c + 1;
  if (c >= n - 1) return c - n + 5;
  return 3;
}
__device__ __forceinline__ int patch_centre(int t, int n) { return t <= 2 ? t - 1 : (t == 3 ? 2 : n - 5 + t); }
__device__ __forceinline__ bool free_comp(const Free& f, int c) { return c == 0 ? f.w : (c == 1 ? f.tx : f.ty); }

// one block per (case, sample): A_p from the element matrix, scaled to a unit diagonal,
// inverted by Gauss-Jordan in single precision (symmetric positive definite: no
// pivoting; scaled, the patches' condition numbers stay near 1e3 to 1e4), unscaled
__global__ void __launch_bounds__(kThreads) k_patch_setup(PGrid g, const float* __restrict__ ke,
                                                          float* __restrict__ pinv) {
  const int type = blockIdx.x, s = blockIdx.y;
  __shared__ __align__(16) float K[144];
  __shared__ float A[kPatchDofs][kPatchDofs + 1];
  __shared__ float dsc[kPatchDofs], fcol[kPatchDofs];
  for (int k = threadIdx.x; k < 144; k += blockDim.x) K[k] = ke[(size_t)s * 144 + k];
  __syncthreads();
  const int ci = patch_centre(type % 7, g.nx), cj = patch_centre(type / 7, g.ny);
  auto slot_dof = [&](int p, int& i, int& j, int& c) -> bool {
    const int a = p / 3;
    c = p - 3 * a;
    i = ci + a % 3 - 1;
    j = cj + a / 3 - 1;
    return i >= 0 && i <= g.nx && j >= 0 && j <= g.ny && free_comp(free_of(g, i, j), c);
  };
  for (int idx = threadIdx.x; idx < kPatchDofs * kPatchDofs; idx += blockDim.x) {
    const int p = idx / kPatchDofs, q = idx - kPatchDofs * p;
    int ia, ja, ca, ib, jb, cb;
    const bool fa = slot_dof(p, ia, ja, ca), fb = slot_dof(q, ib, jb, cb);
    float v = p == q ? 1.f : 0.f;
    if (fa && fb) {
      v = 0.f;
      // elements with both nodes as corners (lower-left node (ei, ej))
      for (int ej = max(ja, jb) - 1; ej <= min(ja, jb); ++ej)
        for (int ei = max(ia, ib) - 1; ei <= min(ia, ib); ++ei) {
          if (ei < 0 || ej < 0 || ei >= g.nx || ej >= g.ny) continue;
          const int la = corner_of(ia - ei, ja - ej), lb = corner_of(ib - ei, jb - ej);
          v += K[(3 * la + ca) * 12 + 3 * lb + cb];
        }
    }
    A[p][q] = v;
  }
  __syncthreads();
  for (int p = threadIdx.x; p < kPatchDofs; p += blockDim.x) dsc[p] = rsqrtf(A[p][p]);
  __syncthreads();
  for (int idx = threadIdx.x; idx < kPatchDofs * kPatchDofs; idx += blockDim.x) {
    const int p = idx / kPatchDofs, q = idx - kPatchDofs * p;
    A[p][q] *= dsc[p] * dsc[q];
  }
  __syncthreads();
  for (int k = 0; k < kPatchDofs; ++k) {
    const float piv = 1.f / A[k][k];
    __syncthreads();
    for (int q = threadIdx.x; q < kPatchDofs; q += blockDim.x) A[k][q] = (q == k ? 1.f : A[k][q]) * piv;
    for (int r = threadIdx.x; r < kPatchDofs; r += blockDim.x) fcol[r] = r == k ? 0.f : A[r][k];
    __syncthreads();
    for (int idx = threadIdx.x; idx < kPatchDofs * kPatchDofs; idx += blockDim.x) {
      const int r = idx / kPatchDofs, q = idx - kPatchDofs * r;
      if (r != k) A[r][q] = (q == k ? 0.f : A[r][q]) - fcol[r] * A[k][q];
    }
    __syncthreads();
  }
  float* out = pinv + ((size_t)s * kPatchTypes + type) * kPatchDofs * kPatchDofs;
  for (int idx = threadIdx.x; idx < kPatchDofs * kPatchDofs; idx += blockDim.x) {
    const int p = idx / kPatchDofs, q = idx - kPatchDofs * p;
    out[idx] = A[p][q] * dsc[p] * dsc[q];
  }
}

// kPatchesPerWarp consecutive patches of colour (sx, sy) per warp: the residual at each
// patch's 9 nodes (lanes 9 t .. 9 t + 8 for the warp's patch t, from `in`), then each
// patch's correction A_p^-1 r at its 27 slots (lanes 0..26 in turn; A_p^-1 is symmetric,
// so lane l reads column l, coalesced), out = in + correction on the patch. The patches
// of a colour tile the mesh, so every node is written.
__global__ void __launch_bounds__(kThreads, 8) k_patch_color(PGrid g, const float* __restrict__ ke,
                                                          const float* __restrict__ pinv, const float4* __restrict__ b,
                                                          const float4* __restrict__ xin, float4* __restrict__ xout,
                                                          int sx, int sy, int pinv_per_sample,
                                                          const int* __restrict__ active) {
  const int e = blockIdx.y, s = e >> g.cshift;
  if (active && !active[s]) return;
  __shared__ __align__(16) float K[144];
  __shared__ float rs[kThreads / 32][kPatchesPerWarp][kPatchDofs + 1], ds[kThreads / 32][kPatchesPerWarp][kPatchDofs + 1];
  for (int k = threadIdx.x; k < 144; k += blockDim.x) K[k] = ke[(size_t)s * 144 + k];
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int fx = sx == 2 ? -1 : sx, fy = sy == 2 ? -1 : sy;   // first centres of the colour
  const int px_n = (g.nx + 1 - fx) / 3 + 1, py_n = (g.ny + 1 - fy) / 3 + 1;
  const int npatch = px_n * py_n;
  const int pbase = (blockIdx.x * (kThreads / 32) + warp) * kPatchesPerWarp;
  if (pbase >= npatch) return;   // the whole warp
  // lanes 0 .. 26: node t % 9 of the warp's patch t / 9
  const int t = lane / 9, nidx = lane - 9 * t;
  const int pid = pbase + t;
  const bool patch_ok = lane < 9 * kPatchesPerWarp && pid < npatch;
  const int ci = fx + 3 * (pid % px_n), cj = fy + 3 * (pid / px_n);
  const int np = g.nx + 1;
  const size_t o = (size_t)e * g.nodes();
  const int li = ci + nidx % 3 - 1, lj = cj + nidx / 3 - 1;
  const bool node_in = patch_ok && li >= 0 && li <= g.nx && lj >= 0 && lj <= g.ny;
  float4 xo = make_float4(0.f, 0.f, 0.f, 0.f);
  if (node_in) {
    // K x rows of the node, one element at a time (a rolled loop keeps registers low)
    float4 kx = xo;
    if (xin) {
      const float4* xe = xin + o;
#pragma unroll 1
      for (int k = 0; k < 4; ++k) {
        const int ox = k & 1, oy = k >> 1;
        const int ei = li - ox, ej = lj - oy;
        if (ei < 0 || ej < 0 || ei >= g.nx || ej >= g.ny) continue;
        const float* Ka = K + 36 * corner_of(ox, oy);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
          const int ni = ei + corner_x(c), nj = ej + corner_y(c);
          const float4 v = masked(free_of(g, ni, nj), xe[nj * np + ni]);
          const float* r = Ka + 3 * c;
          kx.x += r[0] * v.x + r[1] * v.y + r[2] * v.z;
          kx.y += r[12] * v.x + r[13] * v.y + r[14] * v.z;
          kx.z += r[24] * v.x + r[25] * v.y + r[26] * v.z;
        }
      }
    }
    const float4 bb = b[o + lj * np + li];
    const Free f = free_of(g, li, lj);
    if (xin) xo = xin[o + lj * np + li];
    rs[warp][t][3 * nidx] = f.w ? bb.x - kx.x : 0.f;
    rs[warp][t][3 * nidx + 1] = f.tx ? bb.y - kx.y : 0.f;
    rs[warp][t][3 * nidx + 2] = f.ty ? bb.z - kx.z : 0.f;
  } else if (patch_ok) {
    rs[warp][t][3 * nidx] = rs[warp][t][3 * nidx + 1] = rs[warp][t][3 * nidx + 2] = 0.f;
  }
  __syncwarp();
  // the local solves: lane q forms DOF q of each patch's correction (the patches of a
  // warp are neighbours along x and mostly of one type, so M comes from L1)
#pragma unroll 1
  for (int u = 0; u < kPatchesPerWarp; ++u) {
    const int pu = pbase + u;
    if (pu >= npatch) break;   // the same on every lane
    if (lane < kPatchDofs) {
      const int type = patch_case(fx + 3 * (pu % px_n), g.nx) + 7 * patch_case(fy + 3 * (pu / px_n), g.ny);
      const float* M = pinv + ((size_t)(pinv_per_sample ? s : 0) * kPatchTypes + type) * kPatchDofs * kPatchDofs;
      float d = 0.f;
#pragma unroll 3
      for (int q = 0; q < kPatchDofs; ++q) d += M[q * kPatchDofs + lane] * rs[warp][u][q];
      ds[warp][u][lane] = d;
    }
  }
  __syncwarp();
  if (node_in) {
    const Free f = free_of(g, li, lj);
    xout[o + lj * np + li] = masked(f, make_float4(xo.x + ds[warp][t][3 * nidx], xo.y + ds[warp][t][3 * nidx + 1],
                                                  xo.z + ds[warp][t][3 * nidx + 2], 0.f));
  }
}

// one block per sample: assemble K on the free DOFs in shared memory, invert in place
// (Gauss-Jordan without pivoting: K is symmetric positive definite there)
__global__ void k_coarse_setup(PGrid g, const float* __restrict__ ke, const int* __restrict__ freedofs, int nf,
                               float* __restrict__ ainv) {
  extern __shared__ float smem[];
  float* A = smem;                  // nf * nf
  float* col = A + nf * nf;         // nf
  int* map = reinterpret_cast<int*>(col + nf);   // nodes * 4
  __shared__ __align__(16) float K[144];
  __shared__ float pinv;
  const int s = blockIdx.x;
  const int nn = g.nodes();
  for (int k = threadIdx.x; k < 144; k += blockDim.x) K[k] = ke[(size_t)s * 144 + k];
  for (int k = threadIdx.x; k < nf * nf; k += blockDim.x) A[k] = 0.f;
  for (int k = threadIdx.x; k < 4 * nn; k += blockDim.x) map[k] = -1;
  __syncthreads();
  for (int k = threadIdx.x; k < nf; k += blockDim.x) map[freedofs[k]] = k;
  __syncthreads();
  const int ne = g.nx * g.ny;
  for (int k = threadIdx.x; k < ne * 144; k += blockDim.x) {
    const int el = k / 144, pq = k - 144 * el, p = pq / 12, q = pq - 12 * p;
    const int ei = el % g.nx, ej = el / g.nx;
    const int ap = p / 3, aq = q / 3;
    const int np_ = (ej + corner_y(ap)) * (g.nx + 1) + ei + corner_x(ap);
    const int nq = (ej + corner_y(aq)) * (g.nx + 1) + ei + corner_x(aq);
    const int fp = map[4 * np_ + p - 3 * ap], fq = map[4 * nq + q - 3 * aq];
    if (fp >= 0 && fq >= 0) atomicAdd(&A[fp * nf + fq], K[pq]);
  }
  for (int k = 0; k < nf; ++k) {
    __syncthreads();
    if (threadIdx.x == 0) pinv = 1.f / A[k * nf + k];
    for (int r = threadIdx.x; r < nf; r += blockDim.x) col[r] = A[r * nf + k];
    __syncthreads();
    for (int c = threadIdx.x; c < nf; c += blockDim.x) A[k * nf + c] = (c == k ? 1.f : A[k * nf + c]) * pinv;
    __syncthreads();
    // a warp per row, lanes along the row (conflict-free, no index division)
    const int nw = blockDim.x >> 5, lane = threadIdx.x & 31;
    const float* Ak = A + k * nf;
    for (int r = threadIdx.x >> 5; r < nf; r += nw) {
      if (r == k) continue;
      const float f = col[r];
      float* Ar = A + r * nf;
      for (int c = lane; c < nf; c += 32) Ar[c] = (c == k ? 0.f : Ar[c]) - f * Ak[c];
    }
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nf * nf; k += blockDim.x) ainv[(size_t)s * nf * nf + k] = A[k];
}

__global__ void k_coarse_solve(PGrid g, const float* __restrict__ ainv, const int* __restrict__ freedofs, int nf,
                               const float4* __restrict__ b, float4* __restrict__ x, const int* __restrict__ active,
                               int shared) {
  const int e = blockIdx.x, s = e >> g.cshift;
  if (active && !active[s]) return;
  __shared__ float bl[kMaxCoarseFree];
  const int nn = g.nodes();
  const float* bf = reinterpret_cast<const float*>(b + (size_t)e * nn);
  float* xf = reinterpret_cast<float*>(x + (size_t)e * nn);
  for (int k = threadIdx.x; k < nf; k += blockDim.x) bl[k] = bf[freedofs[k]];
  for (int k = threadIdx.x; k < 4 * nn; k += blockDim.x) xf[k] = 0.f;
  __syncthreads();
  const float* A = ainv + (shared ? (size_t)0 : (size_t)s * nf * nf);
  for (int r = threadIdx.x; r < nf; r += blockDim.x) {
    float acc = 0.f;
    for (int c = 0; c < nf; ++c) acc += A[r * nf + c] * bl[c];
    xf[freedofs[r]] = acc;
  }
}

// ---------------------------------------------------------------- LOBPCG

__device__ __forceinline__ float hash_unit(uint32_t v) {
  v ^= v >> 16;
  v *= 0x7feb352dU;
  v ^= v >> 15;
  v *= 0x846ca68bU;
  v ^= v >> 16;
  return (float)(v >> 8) * (2.f / 16777216.f) - 1.f;
}

__global__ void k_init_start(PGrid g, float4* __restrict__ z) {
  const int e = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nn = g.nodes();
  if (t >= nn) return;
  const int i = t % (g.nx + 1), j = t / (g.nx + 1);
  const int c = e & ((1 << g.cshift) - 1);
  const float w = hash_unit((uint32_t)t * 2654435761U + (uint32_t)c * 40503U + 17U);
  z[(size_t)e * nn + t] = masked(free_of(g, i, j), make_float4(w, 0.f, 0.f, 0.f));
}

__global__ void __launch_bounds__(kThreads) k_residual(PGrid g, Eig E, const float4* __restrict__ kx,
                                                       const float4* __restrict__ gx, float4* __restrict__ r) {
  const int e = blockIdx.y, s = e >> g.cshift, c = e & ((1 << g.cshift) - 1);
  if (!E.active[s]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nn = g.nodes();
  if (t >= nn) return;
  const size_t o = (size_t)e * nn + t;
  const float mu = (float)E.mu[s * kCols + c];
  const float4 k = kx[o], q = gx[o];
  r[o] = make_float4(q.x - mu * k.x, q.y - mu * k.y, q.z - mu * k.z, 0.f);
}

// v: X, W, P, KX, KW, KP, GX, GW, GP, each [n][kCols][nodes]; one block row per sample.
// A thread sums the products of its few nodes in single precision; warps and the block
// add in double, and each block adds its 42 sums to the sample's Gram matrices.
__global__ void __launch_bounds__(kThreads) k_gram(PGrid g, Eig E, const __grid_constant__ Vecs V) {
  const float4* const* vp = V.v;
  const int s = blockIdx.y;
  if (!E.active[s]) return;
  const int nn = g.nodes();
  float acc[2 * kGram];
#pragma unroll
  for (int k = 0; k < 2 * kGram; ++k) acc[k] = 0.f;
  for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < nn; t += gridDim.x * blockDim.x) {
    float4 S[kSub], KS[kSub];
    float GS[kSub];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int c = 0; c < kCols; ++c) {
        const size_t o = ((size_t)s * kCols + c) * nn + t;
        S[b * kCols + c] = vp[b][o];
        KS[b * kCols + c] = vp[3 + b][o];
        GS[b * kCols + c] = vp[6 + b][o].x;
      }
    int m = 0;
#pragma unroll
    for (int p = 0; p < kSub; ++p)
#pragma unroll
      for (int q = p; q < kSub; ++q, ++m) {
        acc[m] += S[p].x * KS[q].x + S[p].y * KS[q].y + S[p].z * KS[q].z;
        acc[kGram + m] += S[p].x * GS[q];
      }
  }
  __shared__ double red[kThreads / 32][2 * kGram];
  const int warp = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 2 * kGram; ++k) {
    const double v = warp_sum_d((double)acc[k]);
    if ((threadIdx.x & 31) == 0) red[warp][k] = v;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < 2 * kGram; k += blockDim.x) {
    double v = 0.0;
#pragma unroll
    for (int w = 0; w < kThreads / 32; ++w) v += red[w][k];
    if (v != 0.0) atomicAdd(&E.gram[(size_t)s * 2 * kGram + k], v);
  }
}

// One Jacobi rotation of the symmetric kSub x kSub matrix A (both triangles kept)
// zeroing A[p][q], accumulated into V. p, q are compile-time after unrolling, so A and V
// stay in registers.
template <typename R>
__device__ __forceinline__ void jacobi_rotate(R (&A)[kSub][kSub], R (&V)[kSub][kSub], int p, int q) {
  const R apq = A[p][q];
  if (apq == R(0)) return;
  const R th = (A[q][q] - A[p][p]) / (R(2) * apq);
  // |th| beyond 1e18: the rotation is the identity to working precision (avoids th^2 overflow)
  const R t = fabs(th) > R(1e18) ? R(0) : (th >= R(0) ? R(1) : R(-1)) / (fabs(th) + sqrt(th * th + R(1)));
  const R c = R(1) / sqrt(t * t + R(1)), sn = t * c;
#pragma unroll
  for (int k = 0; k < kSub; ++k) {
    if (k == p || k == q) continue;
    const R akp = A[k][p], akq = A[k][q];
    A[k][p] = A[p][k] = c * akp - sn * akq;
    A[k][q] = A[q][k] = sn * akp + c * akq;
  }
  A[p][p] -= t * apq;
  A[q][q] += t * apq;
  A[p][q] = A[q][p] = R(0);
#pragma unroll
  for (int k = 0; k < kSub; ++k) {
    const R vkp = V[k][p], vkq = V[k][q];
    V[k][p] = c * vkp - sn * vkq;
    V[k][q] = sn * vkp + c * vkq;
  }
}

// Per-sample Rayleigh-Ritz on S = [X0 X1 W0 W1 P0 P1]: the K and G Gram matrices are
// scaled to unit K-diagonal, K is factored by Cholesky with dependent directions
// dropped (a dropped direction gets an identity row and eigenvalue -1, below every
// Ritz value mu > 0), A = L^-1 G L^-T is diagonalised by cyclic Jacobi, and the two
// largest eigenpairs give the coefficients C = D L^-T V. All loops have compile-time
// bounds so that the small matrices live in registers.
__global__ void __launch_bounds__(32) k_rayleigh_ritz(Eig E, int n, double tol2, int max_iter, int first) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n || !E.active[s]) return;
  double* gr = E.gram + (size_t)s * 2 * kGram;
  double A[kSub][kSub], L[kSub][kSub];   // A first holds the scaled G, L the scaled K
  double dsc[kSub];
  bool keep[kSub];
  {
    int m = 0;
#pragma unroll
    for (int p = 0; p < kSub; ++p)
#pragma unroll
      for (int q = p; q < kSub; ++q, ++m) {
        L[p][q] = L[q][p] = gr[m];
        A[p][q] = A[q][p] = gr[kGram + m];
      }
  }
#pragma unroll
  for (int k = 0; k < 2 * kGram; ++k) gr[k] = 0.0;
  if (!first) {
    // preconditioned residual of the first column in the K norm (w = T r, r = G x - mu K x):
    // w^T K w <= tol^2 mu^2 x^T K x; the eigenvalue error is about tol^2
    const double mu0 = E.mu[s * kCols];
    E.eta2[s] = L[2][2] / (mu0 * mu0 * L[0][0]);
    if (L[2][2] <= tol2 * mu0 * mu0 * L[0][0]) {   // converged: keep X
      E.active[s] = 0;
      return;
    }
    if (E.iters[s] >= max_iter) {   // cap: keep X, flag through iters
      E.iters[s] = max_iter + 1;
      E.active[s] = 0;
      return;
    }
    E.iters[s] += 1;
  }
#pragma unroll
  for (int k = 0; k < kSub; ++k) {
    dsc[k] = L[k][k] > 0.0 ? 1.0 / sqrt(L[k][k]) : 0.0;
    keep[k] = dsc[k] > 0.0;
  }
#pragma unroll
  for (int p = 0; p < kSub; ++p)
#pragma unroll
    for (int q = 0; q < kSub; ++q) {
      L[p][q] *= dsc[p] * dsc[q];
      A[p][q] *= dsc[p] * dsc[q];
    }
  // Cholesky of the scaled K in place (lower triangle), dropping dependent directions
#pragma unroll
  for (int k = 0; k < kSub; ++k) {
#pragma unroll
    for (int p = 0; p < k; ++p) {
      double v = L[k][p];
#pragma unroll
      for (int q = 0; q < p; ++q) v -= L[k][q] * L[p][q];
      L[k][p] = keep[p] ? v / L[p][p] : 0.0;
    }
    double d = L[k][k];
#pragma unroll
    for (int q = 0; q < k; ++q) d -= L[k][q] * L[k][q];
    if (keep[k] && d > 1e-6) {
      L[k][k] = sqrt(d);
    } else {
      keep[k] = false;
#pragma unroll
      for (int q = 0; q < k; ++q) L[k][q] = 0.0;
      L[k][k] = 1.0;
    }
  }
  int nk = 0;
#pragma unroll
  for (int k = 0; k < kSub; ++k) nk += keep[k] ? 1 : 0;
  if (nk == 0) {   // no usable direction (the iterate vanished): stop as not converged
    E.iters[s] = max_iter + 1;
    E.active[s] = 0;
    return;
  }
  // A <- L^-1 A (forward substitution per column) on the kept directions
#pragma unroll
  for (int p = 0; p < kSub; ++p)
#pragma unroll
    for (int q = 0; q < kSub; ++q)
      if (!keep[p] || !keep[q]) A[p][q] = 0.0;
#pragma unroll
  for (int c = 0; c < kSub; ++c)
#pragma unroll
    for (int r = 0; r < kSub; ++r) {
      double v = A[r][c];
#pragma unroll
      for (int q = 0; q < r; ++q) v -= L[r][q] * A[q][c];
      A[r][c] = v / L[r][r];
    }
  // T = L^-1 A^T = L^-1 G L^-T, symmetrised
  double T[kSub][kSub];
#pragma unroll
  for (int c = 0; c < kSub; ++c)
#pragma unroll
    for (int r = 0; r < kSub; ++r) {
      double v = A[c][r];
#pragma unroll
      for (int q = 0; q < r; ++q) v -= L[r][q] * T[q][c];
      T[r][c] = v / L[r][r];
    }
  // Jacobi in single precision on T scaled to a unit largest kept diagonal (dropped
  // directions get eigenvalue -1); the double-precision work stays in the Gram scaling,
  // the Cholesky factor and the back substitution. Eigenvalues come out within about
  // 1e-6 of the largest, far inside the stopping tolerance.
  double sc = 0.0;
#pragma unroll
  for (int r = 0; r < kSub; ++r)
    if (keep[r]) sc = fmax(sc, fabs(T[r][r]));
  if (!(sc > 0.0)) sc = 1.0;
  const double isc = 1.0 / sc;
  float Tf[kSub][kSub], Vf[kSub][kSub];
#pragma unroll
  for (int r = 0; r < kSub; ++r)
#pragma unroll
    for (int c = 0; c < kSub; ++c) {
      Tf[r][c] = (keep[r] && keep[c]) ? (float)(0.5 * (T[r][c] + T[c][r]) * isc) : 0.f;
      Vf[r][c] = r == c ? 1.f : 0.f;
    }
#pragma unroll
  for (int r = 0; r < kSub; ++r)
    if (!keep[r]) Tf[r][r] = -1.f;
  for (int sweep = 0; sweep < 10; ++sweep) {
    float off = 0.f, diag = 0.f;
#pragma unroll
    for (int p = 0; p < kSub; ++p) {
      diag += Tf[p][p] * Tf[p][p];
#pragma unroll
      for (int q = p + 1; q < kSub; ++q) off += Tf[p][q] * Tf[p][q];
    }
    if (off <= 1e-13f * diag) break;
#pragma unroll
    for (int p = 0; p < kSub; ++p)
#pragma unroll
      for (int q = p + 1; q < kSub; ++q) jacobi_rotate(Tf, Vf, p, q);
  }
  // the two largest eigenvalues (runtime indices only compared, never used to index)
  double best0 = -1e300, best1 = -1e300;
  int o0 = 0, o1 = 0;
#pragma unroll
  for (int k = 0; k < kSub; ++k)
    if (Tf[k][k] > best0) {
      best0 = Tf[k][k];
      o0 = k;
    }
#pragma unroll
  for (int k = 0; k < kSub; ++k)
    if (k != o0 && Tf[k][k] > best1) {
      best1 = Tf[k][k];
      o1 = k;
    }
  best0 *= sc;
  best1 *= sc;
  double* cf = E.coef + (size_t)s * kSub * kCols;
#pragma unroll
  for (int c = 0; c < kCols; ++c) {
    const int o = c == 0 ? o0 : o1;
    double y[kSub];
#pragma unroll
    for (int r = kSub - 1; r >= 0; --r) {   // back substitution L^T y = v
      double v = 0.0;
#pragma unroll
      for (int j = 0; j < kSub; ++j) v = j == o ? (double)Vf[r][j] : v;
#pragma unroll
      for (int q = r + 1; q < kSub; ++q) v -= L[q][r] * y[q];
      y[r] = v / L[r][r];
    }
#pragma unroll
    for (int r = 0; r < kSub; ++r) cf[r * kCols + c] = keep[r] ? y[r] * dsc[r] : 0.0;
  }
  E.mu[s * kCols] = best0;
  E.mu[s * kCols + 1] = best1;
  atomicAdd(E.count, 1);
}

// X = S C and P = [W P] C (their K and G images are recomputed by the caller). With
// two_part (thin plates): the combination in double and the new X's w kept in two
// floats (high in x, low in w), so that its rounding error, whose transverse shear
// energy dominates on coarse meshes of a thin plate, stays below the tolerance.
__global__ void __launch_bounds__(kThreads) k_update(PGrid g, Eig E, const __grid_constant__ Vecs V, int two_part) {
  float4* const* vp = V.v;
  const int s = blockIdx.y;
  if (!E.active[s]) return;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int nn = g.nodes();
  if (t >= nn) return;
  const double* c = E.coef + (size_t)s * kSub * kCols;
  {
    const int set = 0;   // X and P; K X, K P, G X, G P are recomputed from them
    float4 v[kSub];
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int k = 0; k < kCols; ++k) v[b * kCols + k] = vp[3 * set + b][((size_t)s * kCols + k) * nn + t];
#pragma unroll
    for (int k = 0; k < kCols; ++k) {
      const size_t o = ((size_t)s * kCols + k) * nn + t;
      if (two_part) {
        double x0 = 0.0, x1 = 0.0, x2 = 0.0, p0 = 0.0, p1 = 0.0, p2 = 0.0;
#pragma unroll
        for (int q = 0; q < kSub; ++q) {
          const double w = c[q * kCols + k];
          const double vw = (double)v[q].x + (q < kCols ? (double)v[q].w : 0.0);
          x0 += w * vw;
          x1 += w * (double)v[q].y;
          x2 += w * (double)v[q].z;
          if (q >= kCols) {
            p0 += w * vw;
            p1 += w * (double)v[q].y;
            p2 += w * (double)v[q].z;
          }
        }
        const float hi = (float)x0;
        vp[3 * set][o] = make_float4(hi, (float)x1, (float)x2, (float)(x0 - (double)hi));
        vp[3 * set + 2][o] = make_float4((float)p0, (float)p1, (float)p2, 0.f);
      } else {
        float x0 = 0.f, x1 = 0.f, x2 = 0.f, p0 = 0.f, p1 = 0.f, p2 = 0.f;
#pragma unroll
        for (int q = 0; q < kSub; ++q) {
          const float w = (float)c[q * kCols + k];
          x0 += w * v[q].x;
          x1 += w * v[q].y;
          x2 += w * v[q].z;
          if (q >= kCols) {
            p0 += w * v[q].x;
            p1 += w * v[q].y;
            p2 += w * v[q].z;
          }
        }
        vp[3 * set][o] = make_float4(x0, x1, x2, 0.f);
        vp[3 * set + 2][o] = make_float4(p0, p1, p2, 0.f);
      }
    }
  }
}

// x^T K x and x^T G x of column 0 in double, element by element
__global__ void __launch_bounds__(kThreads) k_energy(PGrid g, const double* __restrict__ ke64,
                                                     const float4* __restrict__ x, Eig E) {
  const int s = blockIdx.y;
  const int ne = g.nx * g.ny, nn = g.nodes();
  const double* K = ke64 + (size_t)s * 144;
  const float4* xs = x + (size_t)s * kCols * nn;   // column 0
  const double gsc = (double)g.hy / (4.0 * (double)g.hx);
  double ek = 0.0, eg = 0.0;
  for (int el = blockIdx.x * blockDim.x + threadIdx.x; el < ne; el += gridDim.x * blockDim.x) {
    const int ei = el % g.nx, ej = el / g.nx;
    double u[12];
    for (int a = 0; a < 4; ++a) {
      const float4 v = xs[(ej + corner_y(a)) * (g.nx + 1) + ei + corner_x(a)];
      u[3 * a] = (double)v.x + (double)v.w;   // w in two parts (low part zero unless kept)
      u[3 * a + 1] = v.y;
      u[3 * a + 2] = v.z;
    }
    for (int p = 0; p < 12; ++p) {
      double r = 0.0;
      for (int q = 0; q < 12; ++q) r += K[p * 12 + q] * u[q];
      ek += u[p] * r;
    }
    const double gs = -u[0] + u[3] + u[6] - u[9];
    eg += gsc * gs * gs;
  }
  ek = warp_sum_d(ek);
  eg = warp_sum_d(eg);
  if ((threadIdx.x & 31) == 0) {
    atomicAdd(&E.energy[2 * s], ek);
    atomicAdd(&E.energy[2 * s + 1], eg);
  }
}

__global__ void k_panel_qoi(Eig E, int n, double ly, double p_star, int max_iter, double* __restrict__ q,
                            int* __restrict__ status) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const double ek = E.energy[2 * s], eg = E.energy[2 * s + 1];
  const double lam = ek / eg;
  const bool ok = eg > 0.0 && isfinite(lam) && lam > 0.0 && E.iters[s] <= max_iter;
  const double P = lam * ly * 1e-3;
  q[2 * s] = P;
  q[2 * s + 1] = P < p_star ? 1.0 : 0.0;
  status[s] = ok ? 0 : (int)MLMC_ERR_NOT_CONVERGED;
}

inline dim3 grid_nodes(const PGrid& g, int rows) {
  return dim3((unsigned)((g.nodes() + kThreads - 1) / kThreads), (unsigned)rows);
}

}  // namespace

cudaError_t launch_laminate(const Laminate& lam, const double* xi, int n, double* dstar, double* kgt,
                            cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_laminate<<<(n + 127) / 128, 128, 0, st>>>(lam, xi, n, dstar, kgt);
  return cudaGetLastError();
}

cudaError_t launch_element_matrices(const double* dstar, const double* kgt, int n, double hx, double hy, float* k32,
                                    double* k64, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  const int64_t total = (int64_t)n * 144;
  k_element<<<(unsigned)((total + 255) / 256), 256, 0, st>>>(dstar, kgt, n, hx, hy, k32, k64);
  return cudaGetLastError();
}

cudaError_t launch_apply(const PGrid& g, const float* ke, const float4* x, const float4* b, float4* out,
                         float4* gout, const int* active, bool bc, cudaStream_t st) {
  if (g.nb <= 0) return cudaSuccess;
  k_apply<<<grid_nodes(g, g.nb), kThreads, 0, st>>>(g, ke, x, b, out, gout, active, bc ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_apply64(const PGrid& g, const double* ke64, const float4* x, float4* out, float4* gout,
                           float4* rout, const double* mu, const int* active, cudaStream_t st) {
  k_apply64<<<dim3((g.nodes() + kThreads - 1) / kThreads, g.nb), kThreads, 0, st>>>(g, ke64, x, out, gout, rout, mu,
                                                                                    active);
  return cudaGetLastError();
}

cudaError_t launch_smooth(const PGrid& g, const float* ke, const float4* b, const float4* x, float4* out,
                          const int* active, cudaStream_t st) {
  if (g.nb <= 0) return cudaSuccess;
  k_smooth<<<grid_nodes(g, g.nb), kThreads, 0, st>>>(g, ke, b, x, out, active);
  return cudaGetLastError();
}

cudaError_t launch_restrict(const PGrid& fine, const PGrid& coarse, const float4* rf, float4* bc, const int* active,
                            cudaStream_t st) {
  if (coarse.nb <= 0) return cudaSuccess;
  k_restrict<<<grid_nodes(coarse, coarse.nb), kThreads, 0, st>>>(fine, coarse, rf, bc, active);
  return cudaGetLastError();
}

cudaError_t launch_prolong(const PGrid& fine, const PGrid& coarse, const float4* xc, float4* xf, const int* active,
                           cudaStream_t st) {
  if (fine.nb <= 0) return cudaSuccess;
  k_prolong<<<grid_nodes(fine, fine.nb), kThreads, 0, st>>>(fine, coarse, xc, xf, active);
  return cudaGetLastError();
}

cudaError_t launch_coarse_setup(const PGrid& g, const float* ke, int n_samples, const int* freedofs, int nf,
                                float* ainv, cudaStream_t st) {
  if (n_samples <= 0) return cudaSuccess;
  if (nf <= 0 || nf > kMaxCoarseFree) return cudaErrorInvalidValue;
  const size_t smem = sizeof(float) * ((size_t)nf * nf + nf) + sizeof(int) * 4 * (size_t)g.nodes();
  cudaError_t e = cudaFuncSetAttribute(k_coarse_setup, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  k_coarse_setup<<<n_samples, 256, smem, st>>>(g, ke, freedofs, nf, ainv);
  return cudaGetLastError();
}

cudaError_t launch_coarse_solve(const PGrid& g, const float* ainv, const int* freedofs, int nf, const float4* b,
                                float4* x, const int* active, bool shared, cudaStream_t st) {
  if (g.nb <= 0) return cudaSuccess;
  if (nf <= 0 || nf > kMaxCoarseFree) return cudaErrorInvalidValue;
  k_coarse_solve<<<g.nb, kThreads, 0, st>>>(g, ainv, freedofs, nf, b, x, active, shared ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_patch_setup(const PGrid& g, const float* ke, int n_samples, float* pinv, cudaStream_t st) {
  if (n_samples <= 0) return cudaSuccess;
  if (g.nx < 4 || g.ny < 4) return cudaErrorInvalidValue;
  k_patch_setup<<<dim3(kPatchTypes, n_samples), kThreads, 0, st>>>(g, ke, pinv);
  return cudaGetLastError();
}

cudaError_t launch_patch_color(const PGrid& g, const float* ke, const float* pinv, bool pinv_per_sample,
                               const float4* b, const float4* in, float4* out, int sx, int sy, const int* active,
                               cudaStream_t st) {
  const int fx = sx == 2 ? -1 : sx, fy = sy == 2 ? -1 : sy;
  const int patches = ((g.nx + 1 - fx) / 3 + 1) * ((g.ny + 1 - fy) / 3 + 1);
  const int per_block = kThreads / 32 * kPatchesPerWarp;
  k_patch_color<<<dim3((patches + per_block - 1) / per_block, g.nb), kThreads, 0, st>>>(
      g, ke, pinv, b, in, out, sx, sy, pinv_per_sample ? 1 : 0, active);
  return cudaGetLastError();
}

cudaError_t launch_init_start(const PGrid& g, float4* z, cudaStream_t st) {
  if (g.nb <= 0) return cudaSuccess;
  k_init_start<<<grid_nodes(g, g.nb), kThreads, 0, st>>>(g, z);
  return cudaGetLastError();
}

cudaError_t launch_residual(const PGrid& g, const Eig& E, const float4* kx, const float4* gx, float4* r,
                            cudaStream_t st) {
  if (g.nb <= 0) return cudaSuccess;
  k_residual<<<grid_nodes(g, g.nb), kThreads, 0, st>>>(g, E, kx, gx, r);
  return cudaGetLastError();
}

cudaError_t launch_gram(const PGrid& g, const Eig& E, const Vecs& v, cudaStream_t st) {
  const int n = g.nb >> g.cshift;
  if (n <= 0) return cudaSuccess;
  const unsigned bx = (unsigned)std::min((g.nodes() + kThreads * 4 - 1) / (kThreads * 4), 64);
  k_gram<<<dim3(bx, (unsigned)n), kThreads, 0, st>>>(g, E, v);
  return cudaGetLastError();
}

cudaError_t launch_rayleigh_ritz(const Eig& E, int n, double tol, int max_iter, bool first, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_rayleigh_ritz<<<(n + 31) / 32, 32, 0, st>>>(E, n, tol * tol, max_iter, first ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_update(const PGrid& g, const Eig& E, const Vecs& v, bool two_part, cudaStream_t st) {
  const int n = g.nb >> g.cshift;
  if (n <= 0) return cudaSuccess;
  k_update<<<grid_nodes(g, n), kThreads, 0, st>>>(g, E, v, two_part ? 1 : 0);
  return cudaGetLastError();
}

cudaError_t launch_energy(const PGrid& g, const double* ke64, const float4* x, const Eig& E, cudaStream_t st) {
  const int n = g.nb >> g.cshift;
  if (n <= 0) return cudaSuccess;
  const unsigned bx = (unsigned)std::min((g.nx * g.ny + kThreads - 1) / kThreads, 32);
  k_energy<<<dim3(bx, (unsigned)n), kThreads, 0, st>>>(g, ke64, x, E);
  return cudaGetLastError();
}

cudaError_t launch_panel_qoi(const Eig& E, int n, double ly, double p_star, int max_iter, double* q, int* status,
                             cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_panel_qoi<<<(n + 127) / 128, 128, 0, st>>>(E, n, ly, p_star, max_iter, q, status);
  return cudaGetLastError();
}

}  // namespace mlmcp
