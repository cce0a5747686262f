// Shared device-side definitions of the level-pair engine.
//
// Element operator. Each element of the structured grid is a rectangle hx x hy with
// one rotated plane-strain stiffness C_bar (6 coefficients). For a rectangle the
// bilinear strain field splits exactly into its centroid value and two
// "hourglass" gradients:
//   e_xx = rx (a_u + eta g_u),  e_yy = ry (b_v + xi g_v),
//   g_xy = ry (b_u + xi g_u) + rx (a_v + eta g_v),      rx = 1/(2 hx), ry = 1/(2 hy)
// with a = -n1 + n2 + n3 - n4, b = -n1 - n2 + n3 + n4, g = n1 - n2 + n3 - n4 over the
// corner values (n1 = (-,-), n2 = (+,-), n3 = (+,+), n4 = (-,+)). The 2x2 Gauss rule
// of Eq. matrixinplane's element matrices sums xi, eta, xi*eta to zero and xi^2,
// eta^2 to 4/3, so K_e p = hx hy [D0^T C E0 + (1/3)(Dxi^T C Gxi + Deta^T C Geta)]
// exactly, at about 60 flops per element instead of an 8x8 matrix.
//
// Rotation (Sec. 3.1, C* = T^-1 C T). With the Tsai-Pagano invariants U1..U5 of the
// fibre-frame plane-strain stiffness, C_bar(theta) is affine in
// (cos 2t, sin 2t, cos 4t, sin 4t):
//   C11 = U1 + U2 c2 + U3 c4     C22 = U1 - U2 c2 + U3 c4
//   C12 = U4 - U3 c4             C66 = U5 - U3 c4
//   C16 = U2/2 s2 + U3 s4        C26 = U2/2 s2 - U3 s4
// so the average of C_bar over child elements is C_bar of the averaged trigonometric
// 4-vector, which is how coarse multigrid levels are rediscretised.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace mlmc {

constexpr int kWarp = 32;
constexpr int kStripCols = 30;     // output node columns per warp strip (32 lanes, 1 halo each side)
constexpr int kSmoothCols = 28;    // strips of the smoothing kernels (2 halo lanes each side, so that
                                   // every node pair {2m, 2m+1} of the smoother lies in one warp)
constexpr int kRowChunk = 32;      // output node rows per warp tile
constexpr int kPrefetch32 = 1;     // node rows in flight per warp (FP32 kernels)
constexpr int kPrefetch64 = 2;     // node rows in flight per warp (FP64 kernels)
constexpr int kWarpsPerBlock = 4;
// Smoother damping. The smoother is block Jacobi whose blocks are the u-DOFs of the
// node pairs {(2m, j), (2m+1, j)} (the strong fibre-direction coupling) and single
// v-DOFs; the block graph of the 9-point stencil is 4-colourable, so
// lambda_max(B^-1 K) <= 4 and w = 1/2 keeps the smoother convergent for any angle field.
constexpr double kOmega = 0.5;
constexpr int kMaxCoarsestDofs = 64;

struct Invariants {
  double U1, U2, U3, U4, U5;
  float F1, F2, F3, F4, F5;   // the same values rounded once to single precision
  double Q1, Q2, Q3, Q4, Q5;  // the values divided by 4 (square-element operator)
  float G1, G2, G3, G4, G5;   // and rounded to single precision
  void round_single() {
    F1 = (float)U1;
    F2 = (float)U2;
    F3 = (float)U3;
    F4 = (float)U4;
    F5 = (float)U5;
    Q1 = U1 / 4;
    Q2 = U2 / 4;
    Q3 = U3 / 4;
    Q4 = U4 / 4;
    Q5 = U5 / 4;
    G1 = (float)Q1;
    G2 = (float)Q2;
    G3 = (float)Q3;
    G4 = (float)Q4;
    G5 = (float)Q5;
  }
};

template <typename T>
struct Coef {
  T c11, c12, c16, c22, c26, c66;
};

template <typename T>
struct V2 {
  T u, v;
};

template <typename T>
__device__ __forceinline__ V2<T> v2(T u, T v) {
  V2<T> r;
  r.u = u;
  r.v = v;
  return r;
}

// Single-precision callers read the pre-rounded invariants: a double-to-float
// conversion per element would run at the (low) FP64 rate.
template <typename T, bool QUARTER = false>
__device__ __forceinline__ Coef<T> coef_from_trig(const Invariants& U, T c2, T s2, T c4, T s4) {
  Coef<T> c;
  T u1, u2, u3, u4, u5;
  if constexpr (QUARTER && sizeof(T) == sizeof(float)) {
    u1 = U.G1; u2 = U.G2; u3 = U.G3; u4 = U.G4; u5 = U.G5;
  } else if constexpr (QUARTER) {
    u1 = U.Q1; u2 = U.Q2; u3 = U.Q3; u4 = U.Q4; u5 = U.Q5;
  } else if constexpr (sizeof(T) == sizeof(float)) {
    u1 = U.F1; u2 = U.F2; u3 = U.F3; u4 = U.F4; u5 = U.F5;
  } else {
    u1 = U.U1; u2 = U.U2; u3 = U.U3; u4 = U.U4; u5 = U.U5;
  }
  c.c11 = u1 + u2 * c2 + u3 * c4;
  c.c22 = u1 - u2 * c2 + u3 * c4;
  c.c12 = u4 - u3 * c4;
  c.c66 = u5 - u3 * c4;
  c.c16 = (T)0.5 * u2 * s2 + u3 * s4;
  c.c26 = (T)0.5 * u2 * s2 - u3 * s4;
  return c;
}

__device__ __forceinline__ void sincos_t(float x, float* s, float* c) { sincosf(x, s, c); }
__device__ __forceinline__ void sincos_t(double x, double* s, double* c) { sincos(x, s, c); }

// (c2, s2, c4, s4) of an angle.
template <typename T>
__device__ __forceinline__ void trig4(T theta, T* c2, T* s2, T* c4, T* s4) {
  T s, c;
  sincos_t((T)2 * theta, &s, &c);
  *c2 = c;
  *s2 = s;
  *c4 = (T)2 * c * c - (T)1;
  *s4 = (T)2 * s * c;
}

// From the pair (cos 2t, sin 2t) stored per element of the finest mesh.
template <typename T, bool QUARTER = false>
__device__ __forceinline__ Coef<T> coef_from_trig2(const Invariants& U, T c2, T s2) {
  return coef_from_trig<T, QUARTER>(U, c2, s2, (T)2 * c2 * c2 - (T)1, (T)2 * s2 * c2);
}

template <typename T>
__device__ __forceinline__ Coef<T> coef_from_theta(const Invariants& U, T theta) {
  T c2, s2, c4, s4;
  trig4(theta, &c2, &s2, &c4, &s4);
  return coef_from_trig(U, c2, s2, c4, s4);
}

// Element operator: K_e applied to corner values n1..n4 (u, v each).
// Outputs the contributions to n1..n4.
template <typename T>
__device__ __forceinline__ void element_apply(const Coef<T>& C, T rx, T ry, T w,
                                              V2<T> n1, V2<T> n2, V2<T> n3, V2<T> n4,
                                              V2<T>& o1, V2<T>& o2, V2<T>& o3, V2<T>& o4) {
  const T du21 = n2.u - n1.u, du34 = n3.u - n4.u, du41 = n4.u - n1.u, du32 = n3.u - n2.u;
  const T dv21 = n2.v - n1.v, dv34 = n3.v - n4.v, dv41 = n4.v - n1.v, dv32 = n3.v - n2.v;
  const T au = du21 + du34, bu = du41 + du32, gu = du34 - du21;
  const T av = dv21 + dv34, bv = dv41 + dv32, gv = dv34 - dv21;
  // centroid strain and stress
  const T ex = rx * au, ey = ry * bv, exy = ry * bu + rx * av;
  const T sx = C.c11 * ex + C.c12 * ey + C.c16 * exy;
  const T sy = C.c12 * ex + C.c22 * ey + C.c26 * exy;
  const T sxy = C.c16 * ex + C.c26 * ey + C.c66 * exy;
  // hourglass parts: G_xi = (0, ry gv, ry gu), G_eta = (rx gu, 0, rx gv)
  const T gxi_y = ry * gv, gxi_g = ry * gu, get_x = rx * gu, get_g = rx * gv;
  const T sxi_y = C.c22 * gxi_y + C.c26 * gxi_g;      // (C G_xi)_y
  const T sxi_g = C.c26 * gxi_y + C.c66 * gxi_g;      // (C G_xi)_xy
  const T set_x = C.c11 * get_x + C.c16 * get_g;      // (C G_eta)_x
  const T set_g = C.c16 * get_x + C.c66 * get_g;      // (C G_eta)_xy
  const T third = (T)(1.0 / 3.0);
  const T A = w * rx * sx, B = w * ry * sy, Cx = w * ry * sxy, Cy = w * rx * sxy;
  const T Hu = w * third * (ry * sxi_g + rx * set_x);
  const T Hv = w * third * (ry * sxi_y + rx * set_g);
  // q_u = xi A + eta Cx + (xi eta) Hu ; q_v = eta B + xi Cy + (xi eta) Hv
  o1.u = -A - Cx + Hu;  o1.v = -B - Cy + Hv;
  o2.u = A - Cx - Hu;   o2.v = -B + Cy - Hv;
  o3.u = A + Cx + Hu;   o3.v = B + Cy + Hv;
  o4.u = -A + Cx - Hu;  o4.v = B - Cy - Hv;
}

// Square elements (hx = hy): every geometric factor of element_apply reduces to 1/4 on
// the centroid part and 1/12 on the hourglass part, and the two shear terms coincide.
// C4 holds C_bar / 4; the result equals element_apply's exactly in real arithmetic.
template <typename T>
__device__ __forceinline__ void element_apply_square(const Coef<T>& C4, V2<T> n1, V2<T> n2, V2<T> n3, V2<T> n4,
                                                     V2<T>& o1, V2<T>& o2, V2<T>& o3, V2<T>& o4) {
  const T du21 = n2.u - n1.u, du34 = n3.u - n4.u, du41 = n4.u - n1.u, du32 = n3.u - n2.u;
  const T dv21 = n2.v - n1.v, dv34 = n3.v - n4.v, dv41 = n4.v - n1.v, dv32 = n3.v - n2.v;
  const T au = du21 + du34, bu = du41 + du32, gu = du34 - du21;
  const T av = dv21 + dv34, bv = dv41 + dv32, gv = dv34 - dv21;
  const T e = bu + av;
  const T A = C4.c11 * au + C4.c12 * bv + C4.c16 * e;
  const T B = C4.c12 * au + C4.c22 * bv + C4.c26 * e;
  const T Cs = C4.c16 * au + C4.c26 * bv + C4.c66 * e;
  const T third = (T)(1.0 / 3.0);
  const T p1 = third * (C4.c11 + C4.c66), p2 = third * (C4.c16 + C4.c26), p3 = third * (C4.c22 + C4.c66);
  const T Hu = p1 * gu + p2 * gv;
  const T Hv = p2 * gu + p3 * gv;
  o1.u = -A - Cs + Hu;  o1.v = -B - Cs + Hv;
  o2.u = A - Cs - Hu;   o2.v = -B + Cs - Hv;
  o3.u = A + Cs + Hu;   o3.v = B + Cs + Hv;
  o4.u = -A + Cs - Hu;  o4.v = B - Cs - Hv;
}

// Diagonal of K_e at local node with xi*eta = sgn (+1 for n1, n3; -1 for n2, n4).
template <typename T>
__device__ __forceinline__ V2<T> element_diag(const Coef<T>& C, T rx, T ry, T w, T sgn) {
  const T f = (T)(4.0 / 3.0);
  V2<T> d;
  d.u = w * (f * (C.c11 * rx * rx + C.c66 * ry * ry) + (T)2 * C.c16 * rx * ry * sgn);
  d.v = w * (f * (C.c22 * ry * ry + C.c66 * rx * rx) + (T)2 * C.c26 * rx * ry * sgn);
  return d;
}

// Geometry of one multigrid level of one solve group.
struct Geo {
  int nx, ny;         // elements
  double rx, ry, w;   // 1/(2hx), 1/(2hy), hx*hy
  int square;         // hx == hy: the square-element operator applies
  int c0, c1;         // element columns whose centroid x lies in the stress region (c1 < c0: none)
  __host__ __device__ int nodes() const { return (nx + 1) * (ny + 1); }
};

__host__ __device__ __forceinline__ int strips_of(int nx, int cols = kStripCols) { return (nx + 1 + cols - 1) / cols; }
__host__ __device__ __forceinline__ int chunks_of(int ny, int rows = kRowChunk) { return (ny + 1 + rows - 1) / rows; }

// Kuu coupling of the two nodes of one horizontal element edge (exact, = 2x2 Gauss):
// w (-4/3 C11 rx^2 + 2/3 C66 ry^2); the C16 terms cancel on such an edge.
template <typename T>
__device__ __forceinline__ T element_edge_uu(const Coef<T>& C, T rx, T ry, T w) {
  return w * ((T)(-4.0 / 3.0) * C.c11 * rx * rx + (T)(2.0 / 3.0) * C.c66 * ry * ry);
}

// Dirichlet DOFs: u = v = 0 on column 0, u prescribed on column nx.
__device__ __forceinline__ bool dir_u(int i, int nx) { return i == 0 || i == nx; }
__device__ __forceinline__ bool dir_v(int i) { return i == 0; }

}  // namespace mlmc
