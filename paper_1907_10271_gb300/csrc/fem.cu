// Matrix-free Q1 plane-strain operator (Eq. matrixinplane) and the multigrid-PCG
// kernels built on it.
//
// Warp-strip scheme. A warp owns 32 consecutive node columns of one sample (halo
// columns on each side: one for the operator alone, two for the smoothing kernels,
// whose pair-block smoother couples columns 2m and 2m + 1) and walks up a chunk of
// node rows. Lane L computes the element to the upper right of its node from its own
// column values and its right neighbour's (warp shuffle down); the element's
// contributions to the right-hand nodes go back by a shuffle up, and the
// contributions to the upper nodes stay in registers for the next row. Every vector
// is read once per row with 256-byte coalesced accesses (FP32: staged through a
// per-warp ring of shared-memory slots filled by cp.async), and each element is
// evaluated once per warp.
//
// The kernels fuse each V-cycle / PCG step with the operator it needs:
//   Apply    q = K p (all rows; testing)
//   PreTop   PCG update  x += alpha p, r' = r - alpha q   (r' written to a second buffer),
//            Jacobi pre-smoothing from zero  x1 = w D^-1 r', residual r1 = r' - K x1,
//            ||r'||^2 reduced per sample
//   Pre      the same smoothing step on a coarse level: x1 = w D^-1 b, r1 = b - K x1
//   Post     prolongation + post-smoothing: x2 = w D^-1 b + P x_c, z = x2 + w D^-1 (b - K x2)
//   PostTop  Post on the finest level, also reducing b . z
//   PcgP     search direction p' = z + beta p (second buffer), q = K p', p' . q reduced
// Homogeneous Dirichlet rows (u, v on x = 0; u on x = lx) are zero in every vector;
// w D^-1 is stored with zeros there.
#include <cfloat>
#include <type_traits>

#include "../../include/mlmc.h"
#include "dfloat.cuh"
#include "fem.cuh"
#include "strip.cuh"

namespace mlmc {

namespace {

template <typename T>
struct Vec2;
template <>
struct Vec2<float> {
  using type = float2;
};
template <>
struct Vec2<double> {
  using type = double2;
};

template <typename T>
__device__ __forceinline__ V2<T> ld2(const T* p) {
  const typename Vec2<T>::type t = *reinterpret_cast<const typename Vec2<T>::type*>(p);
  return v2<T>(t.x, t.y);
}

template <typename T>
__device__ __forceinline__ void st2(T* p, V2<T> v) {
  typename Vec2<T>::type t;
  t.x = v.u;
  t.y = v.v;
  *reinterpret_cast<typename Vec2<T>::type*>(p) = t;
}

template <typename T>
__device__ __forceinline__ V2<T> zero2() {
  return v2<T>(T{}, T{});
}

__device__ __forceinline__ float shfl_dn(float a) { return __shfl_down_sync(0xffffffffu, a, 1); }
__device__ __forceinline__ double shfl_dn(double a) { return __shfl_down_sync(0xffffffffu, a, 1); }
__device__ __forceinline__ DF shfl_dn(DF a) { return shfl_down_df(a, 1); }
__device__ __forceinline__ float shfl_upv(float a) { return __shfl_up_sync(0xffffffffu, a, 1); }
__device__ __forceinline__ double shfl_upv(double a) { return __shfl_up_sync(0xffffffffu, a, 1); }
__device__ __forceinline__ DF shfl_upv(DF a) { return shfl_up_df(a, 1); }

template <typename T>
__device__ __forceinline__ V2<T> shfl_down2(V2<T> a) {
  return v2<T>(shfl_dn(a.u), shfl_dn(a.v));
}

template <typename T>
__device__ __forceinline__ V2<T> shfl_up2(V2<T> a) {
  return v2<T>(shfl_upv(a.u), shfl_upv(a.v));
}

// K_e applied in float-float to float-float corner values, float stiffness: the same
// steps as element_apply, with every intermediate kept to about 48 bits. The corner
// differences are the one place where large values (the displacements, up to the end
// shortening) cancel to small ones (a strain times h), so they take the full
// float-float sum; every later sum has operands at the scale of the differences or of
// the element forces, where the shorter sum's error (relative to its operands) is as
// small as the differences' own rounding, and takes df_add_short.
__device__ __forceinline__ void element_apply_df(const Coef<float>& C, float rx, float ry, float w, V2<DF> n1,
                                                 V2<DF> n2, V2<DF> n3, V2<DF> n4, V2<DF>& o1, V2<DF>& o2,
                                                 V2<DF>& o3, V2<DF>& o4) {
  const DF du21 = n2.u - n1.u, du34 = n3.u - n4.u, du41 = n4.u - n1.u, du32 = n3.u - n2.u;
  const DF dv21 = n2.v - n1.v, dv34 = n3.v - n4.v, dv41 = n4.v - n1.v, dv32 = n3.v - n2.v;
  auto ad = [](DF a, DF b) { return df_add_short(a, b); };
  auto sb = [](DF a, DF b) { return df_sub_short(a, b); };
  const DF au = ad(du21, du34), bu = ad(du41, du32), gu = sb(du34, du21);
  const DF av = ad(dv21, dv34), bv = ad(dv41, dv32), gv = sb(dv34, dv21);
  const DF ex = au * rx, ey = bv * ry, exy = ad(bu * ry, av * rx);
  const DF sx = ad(ad(ex * C.c11, ey * C.c12), exy * C.c16);
  const DF sy = ad(ad(ex * C.c12, ey * C.c22), exy * C.c26);
  const DF sxy = ad(ad(ex * C.c16, ey * C.c26), exy * C.c66);
  const DF gxi_y = gv * ry, gxi_g = gu * ry, get_x = gu * rx, get_g = gv * rx;
  const DF sxi_y = ad(gxi_y * C.c22, gxi_g * C.c26);
  const DF sxi_g = ad(gxi_y * C.c26, gxi_g * C.c66);
  const DF set_x = ad(get_x * C.c11, get_g * C.c16);
  const DF set_g = ad(get_x * C.c16, get_g * C.c66);
  const float third = (float)(1.0 / 3.0);
  const DF A = sx * (w * rx), B = sy * (w * ry), Cx = sxy * (w * ry), Cy = sxy * (w * rx);
  const DF Hu = ad(sxi_g * ry, set_x * rx) * (w * third);
  const DF Hv = ad(sxi_y * ry, set_g * rx) * (w * third);
  o1.u = sb(sb(Hu, A), Cx);  o1.v = sb(sb(Hv, B), Cy);
  o2.u = sb(sb(A, Cx), Hu);  o2.v = sb(sb(Cy, B), Hv);
  o3.u = ad(ad(A, Cx), Hu);  o3.v = ad(ad(B, Cy), Hv);
  o4.u = sb(sb(Cx, A), Hu);  o4.v = sb(sb(B, Cy), Hv);
}

// The refinement iterate d. The double path stores it as double; the mixed path as
// float-float (hi, lo interleaved per DOF, 8 bytes like a double) so that forming,
// updating and differencing it needs no double-precision arithmetic. TI is the inner
// precision.
template <typename TI>
struct DStore;
template <>
struct DStore<double> {
  using Val = double;
  __device__ static double get(const double* d, int64_t k) { return d[k]; }
  __device__ static void put(double* d, int64_t k, double v) { d[k] = v; }
  __device__ static void add(double* d, int64_t k, double x) { d[k] += x; }
  // (d_a - d_b) accurate to the double rounding of the difference
  __device__ static double diff(const double* d, int64_t a, int64_t b) { return d[a] - d[b]; }
  __device__ static double as_double(const double* d, int64_t k) { return d[k]; }
};
template <>
struct DStore<float> {
  using Val = DF;
  __device__ static DF get(const double* d, int64_t k) {
    const float2 t = reinterpret_cast<const float2*>(d)[k];
    return DF{t.x, t.y};
  }
  __device__ static void put(double* d, int64_t k, DF v) { reinterpret_cast<float2*>(d)[k] = make_float2(v.hi, v.lo); }
  __device__ static void add(double* d, int64_t k, float x) {
    const DF a = get(d, k);
    DF s = two_sum(a.hi, x);
    s.lo = __fadd_rn(s.lo, a.lo);
    put(d, k, fast_two_sum(s.hi, s.lo));
  }
  // neighbouring values: each part's float difference is exact or rounded relative to
  // that difference, so the sum carries single-precision relative error of d_a - d_b
  __device__ static float diff(const double* d, int64_t a, int64_t b) {
    const float2 x = reinterpret_cast<const float2*>(d)[a], y = reinterpret_cast<const float2*>(d)[b];
    return __fsub_rn(x.x, y.x) + __fsub_rn(x.y, y.y);
  }
  __device__ static double as_double(const double* d, int64_t k) { return df_to_double(get(d, k)); }
};

// ---------------------------------------------------------------- async row staging
// The FP32 strip kernels stage node rows (and element rows) in a per-warp ring of
// shared-memory slots filled by cp.async, several rows ahead of the row being
// processed, so that each warp keeps several rows of loads in flight without holding
// them in registers. Slots are field-major over the 32 lanes (lane l reads entry l of
// each field, entries it copied itself), so a lane waits only for its own copies.

// One element row of a strip: (cos 2t, sin 2t) on the finest mesh, the averaged trig
// 4-vector on coarse meshes.
struct ESlot {
  union {
    float2 t2[32];
    float4 t4[32];
  };
};

// This lane's node column of a strip kernel: column i of sample s (s clamped into the
// view, so that loads stay in bounds), whether it is a real node of a real sample
// (valid), whether that sample is still iterating (live) and whether the lane writes
// an output there (out: valid, live and one of the strip's output lanes).
struct LaneCol {
  int s, i;
  bool valid, live, out;
};

// Sums v over the output lanes of each sample whose columns this warp writes (one, or
// two on a packed view: lanes hold ascending virtual columns, so the first and last
// output lanes name them) and calls f(sample, total) on lane 0 for each.
template <typename F>
__device__ __forceinline__ void per_sample(const LaneCol& lc, double v, F&& f) {
  const unsigned m = __ballot_sync(0xffffffffu, lc.out);
  if (m == 0u) return;
  const int sa = __shfl_sync(0xffffffffu, lc.s, __ffs(m) - 1);
  const int sb = __shfl_sync(0xffffffffu, lc.s, 31 - __clz(m));
  const double ta = warp_sum(lc.out && lc.s == sa ? v : 0.0);
  const double tb = sb != sa ? warp_sum(lc.out && lc.s == sb ? v : 0.0) : 0.0;
  if ((threadIdx.x & 31) == 0) {
    f(sa, ta);
    if (sb != sa) f(sb, tb);
  }
}

template <typename T>
struct Vec4T {
  T x, y, z, w;
};

__device__ __forceinline__ Vec4T<float> ld4(const float* p) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  return Vec4T<float>{t.x, t.y, t.z, t.w};
}
__device__ __forceinline__ Vec4T<double> ld4(const double* p) {
  const double2 a = reinterpret_cast<const double2*>(p)[0], b = reinterpret_cast<const double2*>(p)[1];
  return Vec4T<double>{a.x, a.y, b.x, b.y};
}

// Raw element data of one element: the angle (top level) or the averaged trig 4-vector.
template <typename T>
struct RawE {
  T a, b, c, d;
};

// Per-row element pass shared by the strip loops. Element row er (between node rows
// er and er + 1) of lane l has corners n1 = (l, er), n2 = (l + 1, er), n3 = (l + 1,
// er + 1), n4 = (l, er + 1); its contributions o1..o4 go to those nodes. Node (l, er)
// therefore sums o1 of row er, o4 of row er - 1, and the left lane's o2 of row er and
// o3 of row er - 1: those two are added before the one shuffle up that brings them.
// The right neighbour's bottom values are its top values of the previous row, so one
// shuffle down per row suffices as well.
template <typename Val>
struct RowCarry {
  V2<Val> pb, pbr;   // bottom node values of the next element row: own and right lane's
  V2<Val> o3p, o4p;  // previous element row's contributions to its top nodes
  __device__ __forceinline__ explicit RowCarry(V2<Val> p0)
      : pb(p0), pbr(shfl_down2(p0)), o3p(zero2<Val>()), o4p(zero2<Val>()) {}
  // pt: top node values of element row er; returns K x at node (lane, er)
  template <typename Op, typename RE, typename Sc>
  __device__ __forceinline__ V2<Val> step(const Op& op, const Invariants& U, const RE& ce, Sc rx, Sc ry, Sc w,
                                          bool elem, V2<Val> pt) {
    const int lane = threadIdx.x & (kWarp - 1);
    const V2<Val> ptr = shfl_down2(pt);
    V2<Val> o1 = zero2<Val>(), o2 = zero2<Val>(), o3 = zero2<Val>(), o4 = zero2<Val>();
    if (elem) op.element(U, ce, rx, ry, w, pb, pbr, ptr, pt, o1, o2, o3, o4);
    V2<Val> f = shfl_up2(v2<Val>(o2.u + o3p.u, o2.v + o3p.v));
    if (lane == 0) f = zero2<Val>();
    const V2<Val> kx = v2<Val>((o1.u + o4p.u) + f.u, (o1.v + o4p.v) + f.v);
    o3p = o3;
    o4p = o4;
    pb = pt;
    pbr = ptr;
    return kx;
  }
  // K x at the top node row of the last element row
  __device__ __forceinline__ V2<Val> top() const {
    const int lane = threadIdx.x & (kWarp - 1);
    V2<Val> f = shfl_up2(o3p);
    if (lane == 0) f = zero2<Val>();
    return v2<Val>(o4p.u + f.u, o4p.v + f.v);
  }
};

// Walks the warp's strip up its chunk of node rows. Node-row data is prefetched P
// rows ahead into a register ring (static indices after unrolling), element data P
// element rows ahead, so each warp keeps P rows of loads in flight. Lane l holds
// virtual column strip * kCols - kHalo + l (lc: its sample and node column); lanes
// kHalo .. kHalo + kCols - 1 are the outputs. Neighbouring samples of a packed view
// never couple: the element flag is false on a sample's last column and on its
// padding column, so no element spans two samples and the shuffles across the seam
// carry zero contributions.
// in()/pair() and out() run on every lane (pair() and out() of the smoothing handlers
// exchange values with lane l ^ 1); out() stores only where is_out. in() and load() may
// shuffle too: every lane calls them (lanes outside the mesh on clamped columns, their
// values discarded).
template <typename T, int P, typename Op>
__device__ __forceinline__ void strip_loop(const Invariants& U, const View<T>& V, const LaneCol& lc, int chunk,
                                           Op& op) {
  using Val = typename Op::Val;
  using Sc = typename Op::Sc;
  const int lane = threadIdx.x & (kWarp - 1);
  const int nx = V.g.nx, ny = V.g.ny;
  const int i = lc.i;
  const bool col_in = lc.valid;
  const bool elem = lc.valid && (i < nx) && (lane < kWarp - 1);
  const bool out_col = lc.out;
  const int ic = min(max(i, 0), nx);       // in-bounds column for (discarded) loads of outside lanes
  const int ie = min(max(i, 0), nx - 1);
  const int rows = V.rows > 0 ? V.rows : kRowChunk;
  const int j0 = chunk * rows;
  const int j1 = min(j0 + rows - 1, ny);
  const int er0 = max(j0 - 1, 0);
  const int er1 = min(j1, ny - 1);
  const Sc rx = (Sc)V.g.rx, ry = (Sc)V.g.ry, w = (Sc)V.g.w;
  typename Op::Raw ring[P];
  RawE<typename Op::E> ering[P];
  V2<Val> pb;
  {
    const typename Op::Raw r0 = op.load(ic, er0);
    const V2<Val> v0 = op.in(r0, i, er0);
    pb = op.pair(col_in ? v0 : zero2<Val>(), col_in);
    op.shift();
  }
#pragma unroll
  for (int u = 0; u < P; ++u) {
    if (er0 + 1 + u <= er1 + 1) ring[u] = op.load(ic, er0 + 1 + u);
    if (er0 + u <= er1) ering[u] = op.loadE(ie, er0 + u);
  }
  RowCarry<Val> rc(pb);
  for (int base = er0; base <= er1; base += P) {
#pragma unroll
    for (int u = 0; u < P; ++u) {
      const int er = base + u;
      if (er <= er1) {
        const typename Op::Raw cur = ring[u];
        const RawE<typename Op::E> ce = ering[u];
        if (er + 1 + P <= er1 + 1) ring[u] = op.load(ic, er + 1 + P);
        if (er + P <= er1) ering[u] = op.loadE(ie, er + P);
        const V2<Val> vt = op.in(cur, i, er + 1);
        const V2<Val> pt = op.pair(col_in ? vt : zero2<Val>(), col_in);
        const V2<Val> kx = rc.step(op, U, ce, rx, ry, w, elem, pt);
        if (er >= j0) op.out(i, er, kx, out_col);
        op.shift();
      }
    }
  }
  // the top boundary row (only element row ny - 1 contributes) belongs to the chunk that owns it
  if (er1 + 1 == ny && ny >= j0 && ny <= j1) op.out(i, ny, rc.top(), out_col);
}

// strip_loop with node and element rows staged through a ring of D shared-memory
// slots (cp.async); step k holds node row er0 + k and element row er0 + k - 1.
template <typename T, int D, typename Op>
__device__ __forceinline__ void strip_loop_async(const Invariants& U, const View<T>& V, const LaneCol& lc, int chunk,
                                                 Op& op, typename Op::Slot* ring) {
  using Val = typename Op::Val;
  using Sc = typename Op::Sc;
  const int lane = threadIdx.x & (kWarp - 1);
  const int nx = V.g.nx, ny = V.g.ny;
  const int i = lc.i;
  const bool col_in = lc.valid;
  const bool elem = lc.valid && (i < nx) && (lane < kWarp - 1);
  const bool out_col = lc.out;
  const int ic = min(max(i, 0), nx);
  const int ie = min(max(i, 0), nx - 1);
  const int rows = V.rows > 0 ? V.rows : kRowChunk;
  const int j0 = chunk * rows;
  const int j1 = min(j0 + rows - 1, ny);
  const int er0 = max(j0 - 1, 0);
  const int er1 = min(j1, ny - 1);
  const int nsteps = er1 - er0 + 2;   // node rows er0 .. er1 + 1
  const Sc rx = (Sc)V.g.rx, ry = (Sc)V.g.ry, w = (Sc)V.g.w;
  // step k into slot k % D (passed in: the loop keeps the slot indices as counters)
  auto issue = [&](int k, int slot) {
    if (k < nsteps) {
      typename Op::Slot& sl = ring[slot];
      op.fetch(sl, lane, ic, er0 + k);
      if (k >= 1) op.fetchE(sl, lane, ie, er0 + k - 1);
    }
    cp_async_commit();   // one group per step, empty past the end
  };
#pragma unroll
  for (int k = 0; k < D; ++k) issue(k, k);
  cp_async_wait<D - 1>();
  V2<Val> pb;
  {
    const typename Op::Raw r0 = op.read(ring[0], lane, ic, er0);
    const V2<Val> v0 = op.in(r0, i, er0);
    pb = op.pair(col_in ? v0 : zero2<Val>(), col_in);
    op.shift();
  }
  RowCarry<Val> rc(pb);
  int refill = 0, slot = 1 % D;   // slots of steps k - 1 and k
  for (int k = 1; k < nsteps; ++k) {
    issue(k + D - 1, refill);   // refills the slot of step k - 1, already read
    cp_async_wait<D - 1>();
    const int er = er0 + k - 1;
    const typename Op::Slot& sl = ring[slot];
    const typename Op::Raw cur = op.read(sl, lane, ic, er + 1);
    const RawE<typename Op::E> ce = op.readE(sl, lane);
    const V2<Val> vt = op.in(cur, i, er + 1);
    const V2<Val> pt = op.pair(col_in ? vt : zero2<Val>(), col_in);
    const V2<Val> kx = rc.step(op, U, ce, rx, ry, w, elem, pt);
    if (er >= j0) op.out(i, er, kx, out_col);
    op.shift();
    refill = slot;
    slot = slot + 1 == D ? 0 : slot + 1;
  }
  cp_async_wait<0>();
  if (er1 + 1 == ny && ny >= j0 && ny <= j1) op.out(i, ny, rc.top(), out_col);
}

// ---------------------------------------------------------------- operand handlers
// Each handler provides: Raw load(i, j) (node data of row j, prefetched), in(raw, i, j)
// (value K is applied to; keeps what out() needs), out(i, j, K x), shift() (row
// advance), loadE / coef (element data), live() and finish() (reductions).

template <typename T>
struct OpBase {
  using E = T;     // element data type
  using Val = T;   // register type of node values
  using Sc = T;    // scalar type of stiffness and geometry
  static constexpr int kP32 = kPrefetch32;   // rows in flight of the FP32 variant
  static constexpr int kCols = kStripCols;    // output columns per strip
  static constexpr int kHalo = 1;             // halo lanes on each side
  static constexpr bool kAsync = false;       // rows staged by strip_loop_async (FP32 only)
  static constexpr int kDepth = 4;            // slots of the staging ring
  static constexpr int kMinBlocks = 7;        // FP32: resident 128-thread blocks per SM (<= 72 registers)
  const View<T>& V;
  int64_t nbase;   // first value of the sample's vectors
  int64_t ebase;   // first element of the sample
  int64_t lane;    // value offset of this lane's node column in row 0
  int64_t elane;   // element offset of this lane's element column in row 0
  int rs;          // values per node row
  __device__ OpBase(const View<T>& v, int s, int ic, int ie)
      : V(v),
        nbase((int64_t)s * 2 * (v.g.nx + 1) * (v.g.ny + 1)),
        ebase((int64_t)s * v.g.nx * v.g.ny),
        lane((int64_t)s * 2 * (v.g.nx + 1) * (v.g.ny + 1) + 2 * ic),
        elane((int64_t)s * v.g.nx * v.g.ny + ie),
        rs(2 * (v.g.nx + 1)) {}
  // value offset of (own column, row j): every load and store of a lane is in its column
  __device__ __forceinline__ int64_t at(int, int j) const { return lane + (int64_t)(j * rs); }
  __device__ __forceinline__ RawE<T> loadE(int, int j) const {
    const int64_t e = elane + (int64_t)(j * V.g.nx);
    RawE<T> r;
    if (V.trig2) {
      const V2<T> t = ld2(V.trig2 + 2 * e);
      r.a = t.u;
      r.b = t.v;
      r.c = r.d = (T)0;
    } else {
      const Vec4T<T> t = ld4(V.trig + 4 * e);
      r.a = t.x;
      r.b = t.y;
      r.c = t.z;
      r.d = t.w;
    }
    return r;
  }
  template <typename Slot>
  __device__ __forceinline__ void fetchE(Slot& S, int lane, int, int j) const {
    const int64_t e = elane + (int64_t)(j * V.g.nx);
    if (V.trig2) cp_async<8>(&S.e.t2[lane], V.trig2 + 2 * e);
    else cp_async<16>(&S.e.t4[lane], V.trig + 4 * e);
  }
  template <typename Slot>
  __device__ __forceinline__ RawE<T> readE(const Slot& S, int lane) const {
    RawE<T> r;
    if (V.trig2) {
      const float2 t = S.e.t2[lane];
      r.a = t.x;
      r.b = t.y;
      r.c = r.d = (T)0;
    } else {
      const float4 t = S.e.t4[lane];
      r.a = t.x;
      r.b = t.y;
      r.c = t.z;
      r.d = t.w;
    }
    return r;
  }
  __device__ __forceinline__ Coef<T> coef(const Invariants& U, const RawE<T>& r) const {
    return V.trig2 ? coef_from_trig2<T>(U, r.a, r.b) : coef_from_trig<T>(U, r.a, r.b, r.c, r.d);
  }
  // value K is applied to, after the smoother's pair exchange (none by default)
  __device__ __forceinline__ V2<T> pair(V2<T> x, bool) { return x; }
  __device__ __forceinline__ V2<T> mask(int i, V2<T> x) const {
    if (dir_u(i, V.g.nx)) x.u = (T)0;
    if (dir_v(i)) x.v = (T)0;
    return x;
  }
  __device__ __forceinline__ void element(const Invariants& U, const RawE<T>& ce, T rx, T ry, T w, V2<T> n1,
                                          V2<T> n2, V2<T> n3, V2<T> n4, V2<T>& o1, V2<T>& o2, V2<T>& o3,
                                          V2<T>& o4) const {
    if (V.g.square) {   // uniform over the launch's view
      const Coef<T> C4 = V.trig2 ? coef_from_trig2<T, true>(U, ce.a, ce.b)
                                 : coef_from_trig<T, true>(U, ce.a, ce.b, ce.c, ce.d);
      element_apply_square<T>(C4, n1, n2, n3, n4, o1, o2, o3, o4);
    } else {
      element_apply<T>(coef(U, ce), rx, ry, w, n1, n2, n3, n4, o1, o2, o3, o4);
    }
  }
};

template <typename T>
struct OpApply : OpBase<T> {
  using Raw = V2<T>;
  __device__ OpApply(const View<T>& v, int s, int ic, int ie, const SampleState&) : OpBase<T>(v, s, ic, ie) {}
  __device__ bool live() const { return true; }
  __device__ Raw load(int i, int j) const { return ld2(this->V.a + this->at(i, j)); }
  __device__ V2<T> in(const Raw& r, int, int) { return r; }
  __device__ void out(int i, int j, V2<T> kp, bool is_out) {
    if (is_out) st2(this->V.o0 + this->at(i, j), kp);
  }
  __device__ void shift() {}
  __device__ void finish(const SampleState&, const LaneCol&) {}
};

// Smoother of the pre-smoothing from zero, x1 = W b, for the handlers below: u gets
// its own and its pair partner's term (lane ^ 1, see kOmega), v its own.
template <typename T>
struct PairSmooth {
  T own_u, cross;   // the row being prepared: b.u and this node's partner coefficient
  __device__ __forceinline__ void set(T bu, T c) {
    own_u = bu;
    cross = c;
  }
  // every lane calls this (shuffle); lanes outside the mesh send and get nothing
  __device__ __forceinline__ T partner_term(bool col_in) const {
    const T other = __shfl_xor_sync(0xffffffffu, col_in ? own_u : (T)0, 1);
    return col_in ? cross * other : (T)0;
  }
};

// a = r (old), b = q, c = p, winvd + wc, o0 = x (read and updated); o1 = r (new), o2 = r1.
template <typename T>
struct OpPreTop : OpBase<T> {
  static constexpr int kCols = kSmoothCols, kHalo = 2;
  static constexpr bool kAsync = sizeof(T) == 4;
  static constexpr int kDepth = 2;   // 7 streams per row: a deeper ring costs occupancy
  struct Raw {
    V2<T> r, q, w, x, p;
    T c;
  };
  struct Slot {
    V2<T> r[32], q[32], w[32], x[32], p[32];
    T c[32];
    ESlot e;
  };
  struct Aux {
    V2<T> r, x, p;
  };
  T alpha;
  bool act;
  Aux at_, ab_;
  PairSmooth<T> ps;
  LaneSum<T> rr;
  __device__ OpPreTop(const View<T>& v, int s, int ic, int ie, const SampleState& S) : OpBase<T>(v, s, ic, ie) {
    act = S.active[v.sbase + s] != 0;
    alpha = (T)S.alpha[v.sbase + s];
  }
  __device__ bool live() const { return act; }
  __device__ Raw load(int i, int j) const {
    const int64_t k = this->at(i, j);
    return Raw{ld2(this->V.a + k), ld2(this->V.b + k), ld2(this->V.winvd + k), ld2(this->V.o0 + k),
               ld2(this->V.c + k), this->V.wc[k >> 1]};
  }
  __device__ void fetch(Slot& S, int lane, int i, int j) const {
    const int64_t k = this->at(i, j);
    cp_async<8>(&S.r[lane], this->V.a + k);
    cp_async<8>(&S.q[lane], this->V.b + k);
    cp_async<8>(&S.w[lane], this->V.winvd + k);
    cp_async<8>(&S.x[lane], this->V.o0 + k);
    cp_async<8>(&S.p[lane], this->V.c + k);
    cp_async<4>(&S.c[lane], this->V.wc + (k >> 1));
  }
  __device__ Raw read(const Slot& S, int lane, int, int) const {
    return Raw{S.r[lane], S.q[lane], S.w[lane], S.x[lane], S.p[lane], S.c[lane]};
  }
  __device__ V2<T> in(const Raw& R, int, int) {
    at_.r = v2<T>(R.r.u - alpha * R.q.u, R.r.v - alpha * R.q.v);
    at_.x = R.x;
    at_.p = R.p;
    ps.set(at_.r.u, R.c);
    return v2<T>(R.w.u * at_.r.u, R.w.v * at_.r.v);
  }
  __device__ V2<T> pair(V2<T> x1, bool col_in) {
    x1.u += ps.partner_term(col_in);
    return x1;
  }
  __device__ void out(int i, int j, V2<T> kx, bool is_out) {
    if (!is_out) return;
    const int64_t k = this->at(i, j);
    st2(this->V.o2 + k, this->mask(i, v2<T>(ab_.r.u - kx.u, ab_.r.v - kx.v)));
    st2(this->V.o1 + k, ab_.r);
    st2(this->V.o0 + k, v2<T>(ab_.x.u + alpha * ab_.p.u, ab_.x.v + alpha * ab_.p.v));
    rr.add(ab_.r.u * ab_.r.u + ab_.r.v * ab_.r.v);
  }
  __device__ void shift() { ab_ = at_; }
  __device__ void finish(const SampleState& S, const LaneCol& lc) {
    per_sample(lc, rr.value(), [&](int s, double t) { atomicAdd(&S.red_rr[this->V.sbase + s], t); });
  }
};

// Coarse-level smoothing with the restriction fused in: b = P^T r1_f (full weighting)
// is gathered from the finer level's residual (xc), kept for the post-smoothing (o1),
// then x1 = W b, r1 = b - K x1 (o2). winvd and wc of this level.
// Gather: a lane (coarse column i) loads fine columns 2i and 2i+1 of a fine row and
// takes 2i-1 from the lane to its left; the row sums of fine rows 2j-1, 2j, 2j+1 make
// coarse row j, and row 2j+1 is kept for coarse row j+1 (load() runs on ascending
// rows, on every lane).
template <typename T>
struct OpPreR : OpBase<T> {
  static constexpr int kCols = kSmoothCols, kHalo = 2;
  static constexpr bool kAsync = sizeof(T) == 4;
  static constexpr int kDepth = 3;
  static constexpr int kMinBlocks = 6;   // capped at 7 blocks it spills in the loop
  struct Raw {
    V2<T> b, w;
    T c;
  };
  // node row j of this level and fine rows 2j, 2j + 1 (columns 2i, 2i + 1; lane 0
  // also 2i - 1, which the other lanes take from their left neighbour)
  struct Slot {
    V2<T> w[32], fa[2][32], fb[2][32];
    T c[32];
    V2<T> fc[2];
    ESlot e;
  };
  bool act, have_prev = false;
  int nxf, nyf;
  int64_t fbase;
  V2<T> bt, bb, rs_prev;
  PairSmooth<T> ps;
  __device__ OpPreR(const View<T>& v, int s, int ic, int ie, const SampleState& S) : OpBase<T>(v, s, ic, ie) {
    act = S.active[v.sbase + s] != 0;
    nxf = 2 * v.g.nx;
    nyf = 2 * v.g.ny;
    fbase = (int64_t)s * 2 * (nxf + 1) * (nyf + 1);
  }
  __device__ bool live() const { return act; }
  // sum over fine columns 2i-1, 2i, 2i+1 of fine row jf, weights 1/2, 1, 1/2
  __device__ V2<T> row_sum(int ic, int jf) const {
    V2<T> a = zero2<T>(), b = zero2<T>(), c = zero2<T>();
    const bool row_in = jf >= 0 && jf <= nyf;
    const T* row = this->V.xc + fbase + 2 * (int64_t)jf * (nxf + 1);
    if (row_in) {
      a = ld2(row + 4 * ic);
      if (2 * ic + 1 <= nxf) b = ld2(row + 4 * ic + 2);
    }
    c.u = __shfl_up_sync(0xffffffffu, b.u, 1);
    c.v = __shfl_up_sync(0xffffffffu, b.v, 1);
    if ((threadIdx.x & 31) == 0 && row_in && ic >= 1) c = ld2(row + 4 * ic - 2);
    if (ic == 0) c = zero2<T>();   // fine column -1 (also lanes left of the mesh, discarded)
    return v2<T>(a.u + (T)0.5 * (b.u + c.u), a.v + (T)0.5 * (b.v + c.v));
  }
  __device__ void fetch(Slot& S, int lane, int i, int j) const {
    const int64_t k = this->at(i, j);
    cp_async<8>(&S.w[lane], this->V.winvd + k);
    cp_async<4>(&S.c[lane], this->V.wc + (k >> 1));
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int jf = 2 * j + q;
      const bool row_in = jf <= nyf;
      const T* row = this->V.xc + fbase + 2 * (int64_t)min(jf, nyf) * (nxf + 1);
      cp_async<8>(&S.fa[q][lane], row + 4 * i, row_in);
      cp_async<8>(&S.fb[q][lane], row + 4 * min(i, nxf / 2 - 1) + 2, row_in && 2 * i + 1 <= nxf);
      if (lane == 0) cp_async<8>(&S.fc[q], row + 4 * max(i, 1) - 2, row_in && i >= 1);
    }
  }
  // fine row sum over columns 2i-1, 2i, 2i+1 from staged values (every lane: shuffle)
  __device__ V2<T> slot_row_sum(const Slot& S, int lane, int q, int ic) const {
    const V2<T> a = S.fa[q][lane], b = S.fb[q][lane];
    V2<T> c;
    c.u = __shfl_up_sync(0xffffffffu, b.u, 1);
    c.v = __shfl_up_sync(0xffffffffu, b.v, 1);
    if (lane == 0) c = S.fc[q];
    if (ic == 0) c = zero2<T>();
    return v2<T>(a.u + (T)0.5 * (b.u + c.u), a.v + (T)0.5 * (b.v + c.v));
  }
  __device__ Raw read(const Slot& S, int lane, int i, int j) {
    Raw R;
    R.w = S.w[lane];
    R.c = S.c[lane];
    const V2<T> rm = have_prev ? rs_prev : row_sum(i, 2 * j - 1);
    const V2<T> r0 = slot_row_sum(S, lane, 0, i);
    const V2<T> rp = slot_row_sum(S, lane, 1, i);
    rs_prev = rp;
    have_prev = true;
    R.b = this->mask(i, v2<T>(r0.u + (T)0.5 * (rm.u + rp.u), r0.v + (T)0.5 * (rm.v + rp.v)));
    return R;
  }
  __device__ Raw load(int i, int j) {
    const int64_t k = this->at(i, j);
    Raw R;
    R.w = ld2(this->V.winvd + k);
    R.c = this->V.wc[k >> 1];
    const V2<T> rm = have_prev ? rs_prev : row_sum(i, 2 * j - 1);
    const V2<T> r0 = row_sum(i, 2 * j);
    const V2<T> rp = row_sum(i, 2 * j + 1);
    rs_prev = rp;
    have_prev = true;
    R.b = this->mask(i, v2<T>(r0.u + (T)0.5 * (rm.u + rp.u), r0.v + (T)0.5 * (rm.v + rp.v)));
    return R;
  }
  __device__ V2<T> in(const Raw& R, int, int) {
    bt = R.b;
    ps.set(R.b.u, R.c);
    return v2<T>(R.w.u * R.b.u, R.w.v * R.b.v);
  }
  __device__ V2<T> pair(V2<T> x1, bool col_in) {
    x1.u += ps.partner_term(col_in);
    return x1;
  }
  __device__ void out(int i, int j, V2<T> kx, bool is_out) {
    if (!is_out) return;
    const int64_t k = this->at(i, j);
    st2(this->V.o1 + k, bb);
    st2(this->V.o2 + k, this->mask(i, v2<T>(bb.u - kx.u, bb.v - kx.v)));
  }
  __device__ void shift() { bb = bt; }
  __device__ void finish(const SampleState&, const LaneCol&) {}
};

// a = b, xc (level below), winvd + wc; o0 = z = x2 + W (b - K x2) with x2 = W b + P xc.
// TOP also reduces b . z.
template <typename T, bool TOP>
struct OpPost : OpBase<T> {
  static constexpr int kP32 = 1;   // row record plus in-line coarse loads: keep registers low
  static constexpr int kCols = kSmoothCols, kHalo = 2;
  static constexpr bool kAsync = sizeof(T) == 4;
  static constexpr int kDepth = 3;
  struct Raw {
    V2<T> b, w;
    T c;
    V2<T> c0, c1;   // coarse correction at (I, J) and (I, J + 1) (staged path only)
  };
  struct Slot {
    V2<T> b[32], w[32], c0[32], c1[32];
    T c[32];
    ESlot e;
  };
  bool act;
  int nxc;
  int64_t cbase;
  V2<T> bt, bb, xt, xb, wt, wb;
  T ct, cb;
  PairSmooth<T> ps;
  LaneSum<T> rz;
  __device__ OpPost(const View<T>& v, int s, int ic, int ie, const SampleState& S) : OpBase<T>(v, s, ic, ie) {
    act = S.active[v.sbase + s] != 0;
    nxc = v.g.nx / 2;
    cbase = (int64_t)s * 2 * (nxc + 1) * (v.g.ny / 2 + 1);
  }
  __device__ bool live() const { return act; }
  __device__ V2<T> coarse(int I, int J) const { return ld2(this->V.xc + cbase + 2 * ((int64_t)J * (nxc + 1) + I)); }
  __device__ Raw load(int i, int j) const {
    const int64_t k = this->at(i, j);
    const int I = i >> 1, J = j >> 1;
    return Raw{ld2(this->V.a + k), ld2(this->V.winvd + k), this->V.wc[k >> 1], coarse(I, J),
               (j & 1) ? coarse(I, J + 1) : zero2<T>()};
  }
  // i is the lane's clamped column, so the coarse column I = i / 2 is in range
  __device__ void fetch(Slot& S, int lane, int i, int j) const {
    const int64_t k = this->at(i, j);
    const int I = i >> 1, J = j >> 1;
    cp_async<8>(&S.b[lane], this->V.a + k);
    cp_async<8>(&S.w[lane], this->V.winvd + k);
    cp_async<4>(&S.c[lane], this->V.wc + (k >> 1));
    cp_async<8>(&S.c0[lane], this->V.xc + cbase + 2 * ((int64_t)J * (nxc + 1) + I));
    const int J1 = (j & 1) ? J + 1 : J;   // even rows need no second coarse row (zero-filled)
    cp_async<8>(&S.c1[lane], this->V.xc + cbase + 2 * ((int64_t)J1 * (nxc + 1) + I), (j & 1) != 0);
  }
  __device__ Raw read(const Slot& S, int lane, int, int) const {
    return Raw{S.b[lane], S.w[lane], S.c[lane], S.c0[lane], S.c1[lane]};
  }
  // bilinear prolongation of the coarse correction: a lane loads coarse column
  // I = i / 2 (rows J and, on odd rows, J + 1; the row parity is the warp's), and an
  // odd column adds column I + 1, which is the next lane's own I. Every lane runs this
  // (shuffle); columns of lanes outside the mesh are clamped and their values unused.
  __device__ V2<T> in(const Raw& R, int i, int j) {
    const bool fi = i & 1, fj = j & 1;
    V2<T> c = R.c0;
    if (fj) c = v2<T>(c.u + R.c1.u, c.v + R.c1.v);
    const V2<T> r = shfl_down2(c);
    if (fi) c = v2<T>(c.u + r.u, c.v + r.v);
    const T f = (fi && fj) ? (T)0.25 : ((fi || fj) ? (T)0.5 : (T)1);
    bt = R.b;
    wt = R.w;
    ct = R.c;
    ps.set(R.b.u, R.c);
    xt = v2<T>(R.w.u * R.b.u + f * c.u, R.w.v * R.b.v + f * c.v);
    return xt;
  }
  __device__ V2<T> pair(V2<T> x, bool col_in) {
    const T t = ps.partner_term(col_in);
    if (!col_in) return x;
    xt.u += t;
    return xt;
  }
  // every lane forms its residual; output lanes pair with output lanes (kHalo even)
  __device__ void out(int i, int j, V2<T> kx, bool is_out) {
    const V2<T> res = v2<T>(bb.u - kx.u, bb.v - kx.v);
    const T other = __shfl_xor_sync(0xffffffffu, res.u, 1);
    if (!is_out) return;
    const V2<T> z = this->mask(i, v2<T>(xb.u + wb.u * res.u + cb * other, xb.v + wb.v * res.v));
    st2(this->V.o0 + this->at(i, j), z);
    if (TOP) rz.add(bb.u * z.u + bb.v * z.v);
  }
  __device__ void shift() {
    bb = bt;
    xb = xt;
    wb = wt;
    cb = ct;
  }
  __device__ void finish(const SampleState& S, const LaneCol& lc) {
    if (TOP) {
      per_sample(lc, rz.value(), [&](int s, double t) {
        const int g = this->V.sbase + s;
        atomicAdd(&S.red_rz[g], t);
        if (last_tile(S.arrive, g, tiles_of_sample(this->V, s, kCols))) after_post(S, g);
      });
    }
  }
};

// a = z, b = p (old); o0 = p (new), o1 = q.
template <typename T>
struct OpPcgP : OpBase<T> {
  static constexpr bool kAsync = sizeof(T) == 4;
  struct Raw {
    V2<T> z, p;
  };
  struct Slot {
    V2<T> z[32], p[32];
    ESlot e;
  };
  bool act;
  T beta;
  V2<T> pt, pb;
  LaneSum<T> pq;
  __device__ OpPcgP(const View<T>& v, int s, int ic, int ie, const SampleState& S) : OpBase<T>(v, s, ic, ie) {
    act = S.active[v.sbase + s] != 0;
    beta = (T)S.beta[v.sbase + s];
  }
  __device__ bool live() const { return act; }
  __device__ Raw load(int i, int j) const {
    const int64_t k = this->at(i, j);
    return Raw{ld2(this->V.a + k), ld2(this->V.b + k)};
  }
  __device__ void fetch(Slot& S, int lane, int i, int j) const {
    const int64_t k = this->at(i, j);
    cp_async<8>(&S.z[lane], this->V.a + k);
    cp_async<8>(&S.p[lane], this->V.b + k);
  }
  __device__ Raw read(const Slot& S, int lane, int, int) const { return Raw{S.z[lane], S.p[lane]}; }
  __device__ V2<T> in(const Raw& R, int, int) {
    pt = v2<T>(R.z.u + beta * R.p.u, R.z.v + beta * R.p.v);
    return pt;
  }
  __device__ void out(int i, int j, V2<T> kp, bool is_out) {
    if (!is_out) return;
    const int64_t k = this->at(i, j);
    const V2<T> q = this->mask(i, kp);
    st2(this->V.o0 + k, pb);
    st2(this->V.o1 + k, q);
    pq.add(pb.u * q.u + pb.v * q.v);
  }
  __device__ void shift() { pb = pt; }
  __device__ void finish(const SampleState& S, const LaneCol& lc) {
    per_sample(lc, pq.value(), [&](int s, double t) {
      const int g = this->V.sbase + s;
      atomicAdd(&S.red_pq[g], t);
      if (last_tile(S.arrive, g, tiles_of_sample(this->V, s, OpBase<T>::kCols))) after_p(S, g);
    });
  }
};

// Refinement residual r = -(K d) on free DOFs from the double-precision d:
// a = d; ext0 = trig2 (TI); ext1 = r output (TI); ||r||^2 into rr64 and the reaction
// sum of (K d)_u on x = lx into react. The rotated stiffness is formed in TI from the
// TI trig2 pair, exactly as in the inner solve, so both use one operator. With a
// single-precision inner solve (TI = float) the arithmetic is float-float (about 48
// bits, FP32 pipes only); with TI = double it is double.
template <typename TI>
struct OpResid : OpBase<double> {
  using E = TI;
  using Val = typename std::conditional<sizeof(TI) == 4, DF, double>::type;
  using Sc = TI;
  using Raw = V2<Val>;
  bool act;
  const TI* th;
  TI* r;
  LaneSum<TI> rr;
  Val react{};
  __device__ OpResid(const View<double>& v, int s, int ic, int ie, const SampleState& S)
      : OpBase<double>(v, s, ic, ie) {
    act = S.outer_active[v.sbase + s] != 0;
    th = static_cast<const TI*>(v.ext0);
    r = static_cast<TI*>(v.ext1);
  }
  __device__ bool live() const { return act; }
  __device__ RawE<TI> loadE(int, int j) const {
    RawE<TI> e;
    const V2<TI> t = ld2(th + 2 * (elane + (int64_t)(j * V.g.nx)));
    e.a = t.u;
    e.b = t.v;
    e.c = e.d = (TI)0;
    return e;
  }
  __device__ static Val to_val(double x) {
    if constexpr (sizeof(TI) == 4) return df_from_double(x);
    else return x;
  }
  __device__ static TI head(Val x) {
    if constexpr (sizeof(TI) == 4) return x.hi;
    else return x;
  }
  __device__ Raw load(int i, int j) const {
    if constexpr (sizeof(TI) == 4) {   // float-float iterate: one 16-byte load per node
      const float4 t = *reinterpret_cast<const float4*>(V.a + at(i, j));
      return v2<Val>(DF{t.x, t.y}, DF{t.z, t.w});
    } else {
      const V2<double> d = ld2(V.a + at(i, j));
      return v2<Val>(to_val(d.u), to_val(d.v));
    }
  }
  __device__ V2<Val> in(const Raw& d, int, int) { return d; }
  __device__ V2<Val> pair(V2<Val> x, bool) { return x; }
  __device__ void element(const Invariants& U, const RawE<TI>& ce, TI rx, TI ry, TI w, V2<Val> n1, V2<Val> n2,
                          V2<Val> n3, V2<Val> n4, V2<Val>& o1, V2<Val>& o2, V2<Val>& o3, V2<Val>& o4) const {
    const Coef<TI> C = coef_from_trig2<TI>(U, ce.a, ce.b);
    if constexpr (sizeof(TI) == 4) element_apply_df(C, rx, ry, w, n1, n2, n3, n4, o1, o2, o3, o4);
    else element_apply<double>(C, rx, ry, w, n1, n2, n3, n4, o1, o2, o3, o4);
  }
  __device__ void out(int i, int j, V2<Val> kd, bool is_out) {
    if (!is_out) return;
    const int64_t k = at(i, j);
    const TI ru = dir_u(i, V.g.nx) ? (TI)0 : -head(kd.u);
    const TI rv = dir_v(i) ? (TI)0 : -head(kd.v);
    r[k] = ru;
    r[k + 1] = rv;
    rr.add(ru * ru + rv * rv);
    if (i == V.g.nx) react = react + kd.u;
  }
  __device__ void shift() {}
  __device__ void finish(const SampleState& S, const LaneCol& lc) {
    double rv;
    if constexpr (sizeof(TI) == 4) rv = df_to_double(react);
    else rv = react;
    per_sample(lc, rr.value(), [&](int s, double t) { atomicAdd(&S.rr64[V.sbase + s], t); });
    per_sample(lc, rv, [&](int s, double t) { atomicAdd(&S.react[V.sbase + s], t); });
  }
};

template <typename T, int P, typename Op>
__global__ void __launch_bounds__(kWarpsPerBlock * kWarp, sizeof(T) == 4 ? Op::kMinBlocks : 0)
    k_strip(const __grid_constant__ ViewList<T> L, SampleState S) {
  const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  int vi, s, strip, chunk;
  if (!find_tile(L, gw, vi, s, strip, chunk)) return;
  const View<T>& V = L.v[vi];
  const int lane = (int)(threadIdx.x & 31);
  const int vcol = strip * Op::kCols - Op::kHalo + lane;
  LaneCol lc;
  if (V.packed) {   // virtual column -> (sample, column); the padding column nx + 1 is not valid
    const int q = vcol >= 0 ? vcol / V.vw : 0;
    lc.i = vcol >= 0 ? vcol - q * V.vw : vcol;
    lc.valid = vcol >= 0 && q < V.nsamp && lc.i <= V.g.nx;
    lc.s = min(q, V.nsamp - 1);
  } else {
    lc.s = s;
    lc.i = vcol;
    lc.valid = vcol >= 0 && vcol <= V.g.nx;
  }
  Op op(V, lc.s, min(max(lc.i, 0), V.g.nx), min(max(lc.i, 0), V.g.nx - 1), S);
  lc.live = op.live();
  if (!__any_sync(0xffffffffu, lc.valid && lc.live)) return;
  lc.out = lc.valid && lc.live && lane >= Op::kHalo && lane < Op::kHalo + Op::kCols;
  if (S.units) {
    const unsigned m = __ballot_sync(0xffffffffu, lc.out);
    if (lane == 0 && m) {
      const int rows = V.rows > 0 ? V.rows : kRowChunk;
      const int r0 = chunk * rows, r1 = min(r0 + rows - 1, V.g.ny);
      atomicAdd(&S.units[L.prof_op], (unsigned long long)(__popc(m) * (r1 - r0 + 1)));
    }
  }
  if constexpr (Op::kAsync) {
    extern __shared__ __align__(16) unsigned char strip_smem[];
    typename Op::Slot* ring = reinterpret_cast<typename Op::Slot*>(strip_smem) + (threadIdx.x >> 5) * Op::kDepth;
    strip_loop_async<T, Op::kDepth>(L.U, V, lc, chunk, op, ring);
  } else {
    strip_loop<T, P>(L.U, V, lc, chunk, op);
  }
  op.finish(S, lc);
}

// ---------------------------------------------------------------- pointwise kernels

template <typename T>
__device__ __forceinline__ bool find_point(const ViewList<T>& L, int64_t gt, int& vi, int64_t& local) {
  vi = 0;
  while (vi < L.n && gt >= (int64_t)L.v[vi].work_begin + L.v[vi].nwork) ++vi;
  if (vi >= L.n) return false;
  local = gt - L.v[vi].work_begin;
  return true;
}

// Coarse element data: o0 = trig (coarse, 4 per element) from the fine level's
// trig2 or trig (view geometry = fine level). One thread per coarse element.
template <typename T>
__global__ void k_trig_average(const __grid_constant__ ViewList<T> L) {
  int vi;
  int64_t loc;
  if (!find_point(L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, vi, loc)) return;
  const View<T>& V = L.v[vi];
  const int nx = V.g.nx, ny = V.g.ny, nxc = nx / 2, nyc = ny / 2;
  const int per = nxc * nyc;
  const int s = (int)loc / per;   // launch totals are int: loc < 2^31
  if (s >= V.nsamp) return;
  const int e = (int)(loc - (int64_t)s * per);
  const int J = e / nxc, I = e - J * nxc;
  T acc[4] = {0, 0, 0, 0};
  for (int b = 0; b < 2; ++b)
    for (int a = 0; a < 2; ++a) {
      const int64_t fe = (int64_t)s * nx * ny + (int64_t)(2 * J + b) * nx + (2 * I + a);
      T t4[4];
      if (V.trig2) {
        t4[0] = V.trig2[2 * fe];
        t4[1] = V.trig2[2 * fe + 1];
        t4[2] = (T)2 * t4[0] * t4[0] - (T)1;
        t4[3] = (T)2 * t4[1] * t4[0];
      } else {
        for (int c = 0; c < 4; ++c) t4[c] = V.trig[4 * fe + c];
      }
      for (int c = 0; c < 4; ++c) acc[c] += t4[c];
    }
  T* o = V.o0 + 4 * ((int64_t)s * per + e);
  for (int c = 0; c < 4; ++c) o[c] = (T)0.25 * acc[c];
}

template <typename T>
__device__ __forceinline__ Coef<T> element_coef(const ViewList<T>& L, const View<T>& V, int64_t e) {
  if (V.trig2) return coef_from_trig2<T>(L.U, V.trig2[2 * e], V.trig2[2 * e + 1]);
  return coef_from_trig<T>(L.U, V.trig[4 * e], V.trig[4 * e + 1], V.trig[4 * e + 2], V.trig[4 * e + 3]);
}

// Smoother coefficients of every node (see kOmega): the u-DOFs of the pair
// {(2m, j), (2m+1, j)} form a 2x2 block [[Kuu_a, k], [k, Kuu_b]] (k from the two
// elements sharing the pair's edge), v-DOFs are single. o0 = (w Kuu_b / det, w / Kvv)
// for node a (and symmetrically for b), o1 = -w k / det, det = Kuu_a Kuu_b - k^2. A
// Dirichlet u-DOF leaves the block: its coefficients are zero and its partner's
// block is 1x1. One thread per node pair (the last column pairs with nothing); the
// six elements around the pair are evaluated once.
template <typename T>
__global__ void k_invdiag(const __grid_constant__ ViewList<T> L) {
  int vi;
  int64_t loc;
  if (!find_point(L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, vi, loc)) return;
  const View<T>& V = L.v[vi];
  const int nx = V.g.nx, ny = V.g.ny, nxp = nx + 1;
  const int pairs = nx / 2 + 1;   // nx is even on every multigrid level
  const int per = pairs * (ny + 1);
  const int s = (int)loc / per;   // launch totals are int: loc < 2^31
  if (s >= V.nsamp) return;
  const int r = (int)(loc - (int64_t)s * per);
  const int j = r / pairs, m = r - j * pairs;
  const int ia = 2 * m, ib = ia + 1;
  const T rx = (T)V.g.rx, ry = (T)V.g.ry, w = (T)V.g.w;
  const int64_t eb = (int64_t)s * nx * ny;
  // element corner blocks around the pair: columns ia-1, ia, ia+1; rows j-1, j
  V2<T> da = zero2<T>(), db = zero2<T>();
  T k = 0;
#pragma unroll
  for (int c = 0; c < 3; ++c) {
    const int ei = ia - 1 + c;
    if (ei < 0 || ei >= nx) continue;
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int ej = j - 1 + q;
      if (ej < 0 || ej >= ny) continue;
      const Coef<T> C = element_coef(L, V, eb + (int64_t)ej * nx + ei);
      const T eta = q == 0 ? (T)1 : (T)-1;   // the pair's row is the top (q = 0) or bottom edge
      if (c <= 1) {   // node a is the element's right (c = 0) or left (c = 1) corner
        const V2<T> d = element_diag<T>(C, rx, ry, w, (c == 0 ? (T)1 : (T)-1) * eta);
        da.u += d.u;
        da.v += d.v;
      }
      if (c >= 1) {   // node b is the element's right (c = 1) or left (c = 2) corner
        const V2<T> d = element_diag<T>(C, rx, ry, w, (c == 1 ? (T)1 : (T)-1) * eta);
        db.u += d.u;
        db.v += d.v;
      }
      if (c == 1) k += element_edge_uu<T>(C, rx, ry, w);
    }
  }
  const T om = V.param > 0 ? (T)V.param : (T)kOmega;
  const bool has_b = ib <= nx;
  const bool pair = has_b && !dir_u(ia, nx) && !dir_u(ib, nx);
  const T det = da.u * db.u - k * k;
  const int64_t nb = (int64_t)s * nxp * (ny + 1) + (int64_t)j * nxp;
  {
    V2<T> o = v2<T>(pair ? om * db.u / det : om / da.u, om / da.v);
    if (dir_u(ia, nx)) o.u = 0;
    if (dir_v(ia)) o.v = 0;
    st2(V.o0 + 2 * (nb + ia), o);
    V.o1[nb + ia] = pair ? -om * k / det : (T)0;
  }
  if (has_b) {
    V2<T> o = v2<T>(pair ? om * da.u / det : om / db.u, om / db.v);
    if (dir_u(ib, nx)) o.u = 0;
    if (dir_v(ib)) o.v = 0;
    st2(V.o0 + 2 * (nb + ib), o);
    V.o1[nb + ib] = pair ? -om * k / det : (T)0;
  }
}

// Dense inverse of the coarsest operator per sample (Dirichlet rows/columns set to
// the identity): element columns assembled in parallel (one thread per element
// column, shared-memory atomics), then in-place Gauss-Jordan in the inner precision
// (the coarsest solve is part of the preconditioner). o0 = inverse [nsamp][n][n].
// One 64-thread block per sample.
template <typename T>
__global__ void __launch_bounds__(64) k_coarsest_setup(const __grid_constant__ ViewList<T> L) {
  __shared__ T A[kMaxCoarsestDofs][kMaxCoarsestDofs];
  __shared__ T pivrow[kMaxCoarsestDofs];
  __shared__ T pivcol[kMaxCoarsestDofs];
  int vi = 0;
  const int gb = blockIdx.x;
  while (vi < L.n && gb >= L.v[vi].work_begin + L.v[vi].nwork) ++vi;
  if (vi >= L.n) return;
  const View<T>& V = L.v[vi];
  const int s = gb - V.work_begin;
  if (s >= V.nsamp) return;
  const int nx = V.g.nx, ny = V.g.ny, nxp = nx + 1;
  const int n = 2 * (nx + 1) * (ny + 1);
  for (int k = threadIdx.x; k < n * n; k += blockDim.x) A[k / n][k % n] = (T)0;
  __syncthreads();
  const T rx = (T)V.g.rx, ry = (T)V.g.ry, w = (T)V.g.w;
  for (int job = threadIdx.x; job < nx * ny * 8; job += blockDim.x) {
    const int el = job >> 3, col = job & 7;
    const int ej = el / nx, ei = el - ej * nx;
    const int64_t e = (int64_t)s * nx * ny + el;
    const Coef<T> C = V.trig2 ? coef_from_trig2<T>(L.U, V.trig2[2 * e], V.trig2[2 * e + 1])
                              : coef_from_trig<T>(L.U, V.trig[4 * e], V.trig[4 * e + 1], V.trig[4 * e + 2],
                                                  V.trig[4 * e + 3]);
    const int nodes[4] = {ej * nxp + ei, ej * nxp + ei + 1, (ej + 1) * nxp + ei + 1, (ej + 1) * nxp + ei};
    V2<T> in[4];
    for (int a = 0; a < 4; ++a) in[a] = v2<T>((T)0, (T)0);
    if (col & 1) in[col >> 1].v = (T)1; else in[col >> 1].u = (T)1;
    V2<T> o[4];
    element_apply<T>(C, rx, ry, w, in[0], in[1], in[2], in[3], o[0], o[1], o[2], o[3]);
    const int gc = 2 * nodes[col >> 1] + (col & 1);
    for (int a = 0; a < 4; ++a) {
      atomicAdd(&A[2 * nodes[a]][gc], o[a].u);
      atomicAdd(&A[2 * nodes[a] + 1][gc], o[a].v);
    }
  }
  __syncthreads();
  // Dirichlet DOFs: identity rows and columns
  for (int j = threadIdx.x; j <= ny; j += blockDim.x) {
    const int dofs[3] = {2 * (j * nxp), 2 * (j * nxp) + 1, 2 * (j * nxp + nx)};
    for (int q = 0; q < 3; ++q) {
      const int d = dofs[q];
      for (int m = 0; m < n; ++m) {
        A[d][m] = (T)0;
        A[m][d] = (T)0;
      }
    }
  }
  __syncthreads();
  for (int j = threadIdx.x; j <= ny; j += blockDim.x) {
    A[2 * (j * nxp)][2 * (j * nxp)] = (T)1;
    A[2 * (j * nxp) + 1][2 * (j * nxp) + 1] = (T)1;
    A[2 * (j * nxp + nx)][2 * (j * nxp + nx)] = (T)1;
  }
  __syncthreads();
  // in-place Gauss-Jordan: row k and column k are snapshotted before any update
  for (int k = 0; k < n; ++k) {
    const T piv = A[k][k];
    for (int m = threadIdx.x; m < n; m += blockDim.x) {
      pivrow[m] = (m == k ? (T)1 : A[k][m]) / piv;
      pivcol[m] = A[m][k];
    }
    __syncthreads();
    for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) {
      const int r = idx / n, c = idx % n;
      if (r == k) {
        A[r][c] = pivrow[c];
      } else {
        A[r][c] = (c == k ? (T)0 : A[r][c]) - pivcol[r] * pivrow[c];
      }
    }
    __syncthreads();
  }
  T* out = V.o0 + (int64_t)s * n * n;
  for (int idx = threadIdx.x; idx < n * n; idx += blockDim.x) out[idx] = A[idx / n][idx % n];
}

// x = A^-1 b at the coarsest level: ext0 = inverse (T), o0 = x; b = a, or, when xc is
// set, b = P^T r1 gathered from the finer level's residual xc. One warp per sample.
template <typename T>
__global__ void k_coarsest_solve(const __grid_constant__ ViewList<T> L, SampleState S) {
  __shared__ T bsh[kWarpsPerBlock][kMaxCoarsestDofs];
  const int wib = threadIdx.x >> 5;
  const int gw = blockIdx.x * kWarpsPerBlock + wib;
  int vi = 0;
  while (vi < L.n && gw >= L.v[vi].work_begin + L.v[vi].nwork) ++vi;
  if (vi >= L.n) return;
  const View<T>& V = L.v[vi];
  const int s = gw - V.work_begin;
  if (s >= V.nsamp || !S.active[V.sbase + s]) return;
  const int nx = V.g.nx, ny = V.g.ny, nxp = nx + 1;
  const int n = 2 * (nx + 1) * (ny + 1);
  const int lane = threadIdx.x & 31;
  T* b = bsh[wib];
  if (V.xc) {
    const int nxf = 2 * nx, nyf = 2 * ny;
    const T* rf = V.xc + (int64_t)s * 2 * (nxf + 1) * (nyf + 1);
    for (int node = lane; node < n / 2; node += 32) {
      const int j = node / nxp, i = node - j * nxp;
      T su = (T)0, sv = (T)0;
      for (int dj = -1; dj <= 1; ++dj) {
        const int jf = 2 * j + dj;
        if (jf < 0 || jf > nyf) continue;
        const T wj = dj == 0 ? (T)1 : (T)0.5;
        for (int di = -1; di <= 1; ++di) {
          const int iff = 2 * i + di;
          if (iff < 0 || iff > nxf) continue;
          const T ww = wj * (di == 0 ? (T)1 : (T)0.5);
          su += ww * rf[2 * (jf * (nxf + 1) + iff)];
          sv += ww * rf[2 * (jf * (nxf + 1) + iff) + 1];
        }
      }
      b[2 * node] = dir_u(i, nx) ? (T)0 : su;
      b[2 * node + 1] = dir_v(i) ? (T)0 : sv;
    }
  } else {
    for (int r = lane; r < n; r += 32) b[r] = V.a[(int64_t)s * n + r];
  }
  __syncwarp();
  const T* Ai = static_cast<const T*>(V.ext0) + (int64_t)s * n * n;
  for (int r = lane; r < n; r += 32) {
    T acc = 0;
    for (int c = 0; c < n; ++c) acc += Ai[(int64_t)r * n + c] * b[c];
    V.o0[(int64_t)s * n + r] = acc;
  }
}

// ---------------------------------------------------------------- multigrid bottom (FP32)
// Small-mesh pieces of k_bottom (one warp per sample) and k_bottom_deep (one thread
// block per sample); vectors in shared memory as [node][2] with node = j (nx + 1) + i.
// The threads of group G share the work of each piece, which ends with G's barrier.
struct WarpGroup {
  int t;
  static constexpr int n = 32;
  __device__ __forceinline__ void sync() const { __syncwarp(); }
};
struct BlockGroup {
  int t, n;
  __device__ __forceinline__ void sync() const { __syncthreads(); }
};

// b = mask(R f): full weighting of the fine vector f (nodes of the 2nx x 2ny mesh)
template <typename Grp>
__device__ __forceinline__ void bot_restrict(const Geo& g, const float* f, float* b, const Grp& G) {
  const int nxp = g.nx + 1, nxf = 2 * g.nx, nyf = 2 * g.ny;
  for (int node = G.t; node < nxp * (g.ny + 1); node += G.n) {
    const int j = node / nxp, i = node - j * nxp;
    float su = 0.f, sv = 0.f;
    for (int dj = -1; dj <= 1; ++dj) {
      const int jf = 2 * j + dj;
      if (jf < 0 || jf > nyf) continue;
      const float wj = dj == 0 ? 1.f : 0.5f;
      for (int di = -1; di <= 1; ++di) {
        const int iff = 2 * i + di;
        if (iff < 0 || iff > nxf) continue;
        const float ww = wj * (di == 0 ? 1.f : 0.5f);
        su += ww * f[2 * (jf * (nxf + 1) + iff)];
        sv += ww * f[2 * (jf * (nxf + 1) + iff) + 1];
      }
    }
    b[2 * node] = dir_u(i, g.nx) ? 0.f : su;
    b[2 * node + 1] = dir_v(i) ? 0.f : sv;
  }
  G.sync();
}

// y = W v (pair-block smoother: u takes its pair partner's term, column i ^ 1), plus add
template <typename Grp>
__device__ __forceinline__ void bot_smooth(const Geo& g, const float* winv, const float* wc, const float* v,
                                           const float* add, float* y, const Grp& G) {
  const int nxp = g.nx + 1;
  for (int node = G.t; node < nxp * (g.ny + 1); node += G.n) {
    const int j = node / nxp, i = node - j * nxp;
    const int ip = i ^ 1;
    const float other = ip <= g.nx ? v[2 * (j * nxp + ip)] : 0.f;
    const float2 w = reinterpret_cast<const float2*>(winv)[node];
    float u = w.x * v[2 * node] + wc[node] * other, vv = w.y * v[2 * node + 1];
    if (add) {
      u += add[2 * node];
      vv += add[2 * node + 1];
    }
    y[2 * node] = u;
    y[2 * node + 1] = vv;
  }
  G.sync();
}

// t = K x (t zeroed here); element (i, j) has corners (i, j) (i+1, j) (i+1, j+1) (i, j+1)
template <typename Grp>
__device__ __forceinline__ void bot_apply(const Invariants& U, const Geo& g, const float* trig, const float* x,
                                          float* t, const Grp& G) {
  const int nxp = g.nx + 1;
  for (int r = G.t; r < 2 * nxp * (g.ny + 1); r += G.n) t[r] = 0.f;
  G.sync();
  const float rx = (float)g.rx, ry = (float)g.ry, w = (float)g.w;
  for (int e = G.t; e < g.nx * g.ny; e += G.n) {
    const int j = e / g.nx, i = e - j * g.nx;
    const float4 tr = reinterpret_cast<const float4*>(trig)[e];
    const int k1 = j * nxp + i, k2 = k1 + 1, k3 = k1 + nxp + 1, k4 = k1 + nxp;
    const V2<float> n1 = v2<float>(x[2 * k1], x[2 * k1 + 1]), n2 = v2<float>(x[2 * k2], x[2 * k2 + 1]);
    const V2<float> n3 = v2<float>(x[2 * k3], x[2 * k3 + 1]), n4 = v2<float>(x[2 * k4], x[2 * k4 + 1]);
    V2<float> o1, o2, o3, o4;
    if (g.square) {
      const Coef<float> C4 = coef_from_trig<float, true>(U, tr.x, tr.y, tr.z, tr.w);
      element_apply_square<float>(C4, n1, n2, n3, n4, o1, o2, o3, o4);
    } else {
      element_apply<float>(coef_from_trig<float>(U, tr.x, tr.y, tr.z, tr.w), rx, ry, w, n1, n2, n3, n4, o1, o2, o3,
                           o4);
    }
    atomicAdd(&t[2 * k1], o1.u);
    atomicAdd(&t[2 * k1 + 1], o1.v);
    atomicAdd(&t[2 * k2], o2.u);
    atomicAdd(&t[2 * k2 + 1], o2.v);
    atomicAdd(&t[2 * k3], o3.u);
    atomicAdd(&t[2 * k3 + 1], o3.v);
    atomicAdd(&t[2 * k4], o4.u);
    atomicAdd(&t[2 * k4 + 1], o4.v);
  }
  G.sync();
}

// r = mask(b - t)
template <typename Grp>
__device__ __forceinline__ void bot_resid(const Geo& g, const float* b, const float* t, float* r, const Grp& G) {
  const int nxp = g.nx + 1;
  for (int node = G.t; node < nxp * (g.ny + 1); node += G.n) {
    const int i = node % nxp;
    r[2 * node] = dir_u(i, g.nx) ? 0.f : b[2 * node] - t[2 * node];
    r[2 * node + 1] = dir_v(i) ? 0.f : b[2 * node + 1] - t[2 * node + 1];
  }
  G.sync();
}

// p = P xc (bilinear prolongation of the coarse vector)
template <typename Grp>
__device__ __forceinline__ void bot_prolong(const Geo& g, const float* xc, float* p, const Grp& G) {
  const int nxp = g.nx + 1, nxc = g.nx / 2;
  for (int node = G.t; node < nxp * (g.ny + 1); node += G.n) {
    const int j = node / nxp, i = node - j * nxp;
    const int I = i >> 1, J = j >> 1;
    float cu = xc[2 * (J * (nxc + 1) + I)], cv = xc[2 * (J * (nxc + 1) + I) + 1];
    if (j & 1) {
      cu += xc[2 * ((J + 1) * (nxc + 1) + I)];
      cv += xc[2 * ((J + 1) * (nxc + 1) + I) + 1];
    }
    if (i & 1) {
      cu += xc[2 * (J * (nxc + 1) + I + 1)];
      cv += xc[2 * (J * (nxc + 1) + I + 1) + 1];
      if (j & 1) {
        cu += xc[2 * ((J + 1) * (nxc + 1) + I + 1)];
        cv += xc[2 * ((J + 1) * (nxc + 1) + I + 1) + 1];
      }
    }
    const float f = ((i & 1) && (j & 1)) ? 0.25f : (((i & 1) || (j & 1)) ? 0.5f : 1.f);
    p[2 * node] = f * cu;
    p[2 * node + 1] = f * cv;
  }
  G.sync();
}

// post-smoothing of level g: x2 = W b + P xc, z = mask(x2 + W (b - K x2)) into out
template <typename Grp>
__device__ __forceinline__ void bot_post(const Invariants& U, const Geo& g, const float* winv, const float* wc,
                                         const float* trig, const float* b, const float* xc, float* x2, float* t,
                                         float* out, const Grp& G) {
  bot_prolong(g, xc, t, G);                 // t = P xc
  bot_smooth(g, winv, wc, b, t, x2, G);     // x2 = W b + P xc
  bot_apply(U, g, trig, x2, t, G);          // t = K x2
  const int nxp = g.nx + 1;
  for (int node = G.t; node < nxp * (g.ny + 1); node += G.n) {   // t = b - K x2 (unmasked: W is zero there)
    t[2 * node] = b[2 * node] - t[2 * node];
    t[2 * node + 1] = b[2 * node + 1] - t[2 * node + 1];
  }
  G.sync();
  for (int node = G.t; node < nxp * (g.ny + 1); node += G.n) {
    const int j = node / nxp, i = node - j * nxp;
    const int ip = i ^ 1;
    const float other = ip <= g.nx ? t[2 * (j * nxp + ip)] : 0.f;
    const float2 w = reinterpret_cast<const float2*>(winv)[node];
    float zu = x2[2 * node] + w.x * t[2 * node] + wc[node] * other;
    float zv = x2[2 * node + 1] + w.y * t[2 * node + 1];
    if (dir_u(i, g.nx)) zu = 0.f;
    if (dir_v(i)) zv = 0.f;
    out[2 * node] = zu;
    out[2 * node + 1] = zv;
  }
  G.sync();
}

constexpr int kBotFloats = 2 * kBotNodes * 3 + 2 * kBotNodesB * 3 + 2 * kMaxCoarsestDofs;

__global__ void __launch_bounds__(kWarpsPerBlock * kWarp) k_bottom(const __grid_constant__ BottomList L, SampleState S) {
  __shared__ __align__(16) float sm[kWarpsPerBlock][kBotFloats];
  const int wib = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const WarpGroup G{lane};
  const int gw = blockIdx.x * kWarpsPerBlock + wib;
  int vi = 0;
  while (vi < L.n && gw >= L.v[vi].work_begin + L.v[vi].nsamp) ++vi;
  if (vi >= L.n) return;
  const BottomView& V = L.v[vi];
  const int s = gw - V.work_begin;
  if (s < 0 || !S.active[V.sbase + s]) return;   // the whole warp
  const Geo& ga = V.ga;
  const Geo& gb = V.gb;
  const Geo& gc = V.gc;
  const int na = (ga.nx + 1) * (ga.ny + 1), nb = (gb.nx + 1) * (gb.ny + 1), nc = 2 * (gc.nx + 1) * (gc.ny + 1);
  const int nf = (2 * ga.nx + 1) * (2 * ga.ny + 1);
  float* bA = sm[wib];
  float* xA = bA + 2 * kBotNodes;
  float* tA = xA + 2 * kBotNodes;
  float* bB = tA + 2 * kBotNodes;
  float* xB = bB + 2 * kBotNodesB;
  float* tB = xB + 2 * kBotNodesB;
  float* bC = tB + 2 * kBotNodesB;
  const float* winvA = V.winv_a + (int64_t)s * 2 * na;
  const float* wcA = V.wc_a + (int64_t)s * na;
  const float* trA = V.trig_a + (int64_t)s * 4 * ga.nx * ga.ny;
  const float* winvB = V.winv_b + (int64_t)s * 2 * nb;
  const float* wcB = V.wc_b + (int64_t)s * nb;
  const float* trB = V.trig_b + (int64_t)s * 4 * gb.nx * gb.ny;
  // down: level A from the residual of the level above, then level B
  bot_restrict(ga, V.rin + (int64_t)s * 2 * nf, bA, G);
  bot_smooth(ga, winvA, wcA, bA, nullptr, xA, G);
  bot_apply(L.U, ga, trA, xA, tA, G);
  bot_resid(ga, bA, tA, tA, G);             // tA = r_A
  bot_restrict(gb, tA, bB, G);
  bot_smooth(gb, winvB, wcB, bB, nullptr, xB, G);
  bot_apply(L.U, gb, trB, xB, tB, G);
  bot_resid(gb, bB, tB, tB, G);             // tB = r_B
  // coarsest: x_C = A^-1 R r_B (into tA's space, free now: level C has <= 64 values)
  bot_restrict(gc, tB, bC, G);
  float* xC = tA;
  const float* Ai = V.ainv + (int64_t)s * nc * nc;
  for (int r = lane; r < nc; r += 32) {
    float acc = 0.f;
    for (int c = 0; c < nc; ++c) acc += Ai[(int64_t)r * nc + c] * bC[c];
    xC[r] = acc;
  }
  __syncwarp();
  // up: level B (its post-smoothed x into xB), then level A straight to the output
  bot_post(L.U, gb, winvB, wcB, trB, bB, xC, xB, tB, xB, G);   // scratch x2 = out = xB, t = tB
  float* outA = V.xout + (int64_t)s * 2 * na;
  bot_post(L.U, ga, winvA, wcA, trA, bA, xB, xA, tA, outA, G);   // scratch x2 = xA, t = tA
}


// The deepest levels of every group in one launch, one thread block per sample: the
// smoothed levels A_0 .. A_{nb-1} (finest first) and the coarsest C, with each
// smoothed level's smoother and element data copied into shared memory once at the
// start (cp.async), so that the V-cycle's many dependent steps on these small meshes
// wait on shared memory only. Same operations and order as PreR on A_0 .. A_{nb-1},
// the coarsest solve and Post back up: b_0 = R r_in, x_k = W b_k, r_k = b_k - K x_k,
// b_{k+1} = R r_k, ..., x_C = A^-1 R r_{nb-1}; then for k = nb-1 .. 0:
// x2 = W b_k + P x_{k+1}, x_k = x2 + W (b_k - K x2); writes x_0 (what Post or PostTop
// on the level above prolongates).
__global__ void __launch_bounds__(kDeepThreads) k_bottom_deep(const __grid_constant__ DeepList L, SampleState S) {
  extern __shared__ __align__(16) float dsm[];
  int vi = 0;
  const int gb = blockIdx.x;
  while (vi < L.n && gb >= L.v[vi].work_begin + L.v[vi].nsamp) ++vi;
  if (vi >= L.n) return;
  const DeepView& V = L.v[vi];
  const int s = gb - V.work_begin;
  if (s < 0 || !S.active[V.sbase + s]) return;   // the whole block
  const BlockGroup G{(int)threadIdx.x, (int)blockDim.x};
  const int nb = V.nb;
  float *b[kDeepMax], *x[kDeepMax], *t[kDeepMax], *w[kDeepMax], *c[kDeepMax], *tr[kDeepMax];
  float* p = dsm;
  auto take = [&](int count) {   // 16-byte aligned carving (float4 element data, float2 smoother)
    float* q = p;
    p += (count + 3) & ~3;
    return q;
  };
  for (int k = 0; k < nb; ++k) {
    const int n = V.g[k].nodes(), ne = V.g[k].nx * V.g[k].ny;
    b[k] = take(2 * n);
    x[k] = take(2 * n);
    t[k] = take(2 * n);
    w[k] = take(2 * n);
    c[k] = take(n);
    tr[k] = take(4 * ne);
    const float* ws = V.winv[k] + (int64_t)s * 2 * n;
    const float* cs = V.wc[k] + (int64_t)s * n;
    const float* ts = V.trig[k] + (int64_t)s * 4 * ne;
    for (int q = G.t; q < 2 * n; q += G.n) cp_async<4>(w[k] + q, ws + q);
    for (int q = G.t; q < n; q += G.n) cp_async<4>(c[k] + q, cs + q);
    for (int q = G.t; q < 4 * ne; q += G.n) cp_async<4>(tr[k] + q, ts + q);
  }
  const int nc = 2 * V.gc.nodes();
  float* bC = take(nc);
  float* xC = take(nc);
  cp_async_commit();
  // down; the first restriction reads the residual of the level above from global memory
  {
    const Geo& g0 = V.g[0];
    const int nf = (2 * g0.nx + 1) * (2 * g0.ny + 1);
    bot_restrict(g0, V.rin + (int64_t)s * 2 * nf, b[0], G);
  }
  cp_async_wait<0>();
  G.sync();
  for (int k = 0; k < nb; ++k) {
    if (k > 0) bot_restrict(V.g[k], t[k - 1], b[k], G);
    bot_smooth(V.g[k], w[k], c[k], b[k], nullptr, x[k], G);
    bot_apply(L.U, V.g[k], tr[k], x[k], t[k], G);
    bot_resid(V.g[k], b[k], t[k], t[k], G);      // t_k = r_k
  }
  bot_restrict(V.gc, t[nb - 1], bC, G);
  const float* Ai = V.ainv + (int64_t)s * nc * nc;
  for (int r = G.t; r < nc; r += G.n) {
    float acc = 0.f;
    for (int q = 0; q < nc; ++q) acc += Ai[(int64_t)r * nc + q] * bC[q];
    xC[r] = acc;
  }
  G.sync();
  // up: each level's post-smoothed x in place, level 0 straight to the output
  for (int k = nb - 1; k >= 0; --k) {
    const float* xc = k == nb - 1 ? xC : x[k + 1];
    float* out = k == 0 ? V.xout + (int64_t)s * 2 * V.g[0].nodes() : x[k];
    bot_post(L.U, V.g[k], w[k], c[k], tr[k], b[k], xc, x[k], t[k], out, G);
  }
}

// d += x on refinement-active samples: ext1 = d (DStore<T>), a = x (T). With o0 set,
// also moves the inner solve's final residual into o0 from b where it ended there
// (rpar), making it the next refinement residual.
template <typename T>
__global__ void k_update_d(const __grid_constant__ ViewList<T> L, SampleState S) {
  int vi;
  int64_t loc;
  if (!find_point(L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, vi, loc)) return;
  const View<T>& V = L.v[vi];
  const int64_t per = 2 * (int64_t)(V.g.nx + 1) * (V.g.ny + 1);
  const int s = per > INT32_MAX ? 0 : (int)loc / (int)per;   // launch totals are int: loc < 2^31
  const int t = V.sbase + s;
  if (s >= V.nsamp || !S.outer_active[t]) return;
  DStore<T>::add(static_cast<double*>(V.ext1), loc, V.a[loc]);
  if (V.o0 && S.rpar[t]) V.o0[loc] = V.b[loc];
}

// Lifting d0 (u = -shortening on x = lx, zero elsewhere) and its residual
// r = -(K d0) on free DOFs, in the inner precision T (the first refinement residual,
// after the first correction, supersedes it). K d0 is nonzero only on node columns
// nx - 1 and nx, the nodes of the elements that touch the prescribed column, so the
// caller clears d and r and this kernel writes d on column nx and r on columns
// nx - 1 and nx, ||r||^2 into rr64 and the reaction sum of (K d0)_u over x = lx into
// react. o0 = r (T), ext1 = d (DStore<T>). One thread per (sample, node row, column).
template <typename T>
__global__ void k_lift_resid(const __grid_constant__ ViewList<T> L, SampleState S, float sh_hi, float sh_lo,
                             double shortening) {
  int vi;
  int64_t loc;
  if (!find_point(L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, vi, loc)) return;
  const View<T>& V = L.v[vi];
  const int nx = V.g.nx, ny = V.g.ny, nxp = nx + 1;
  const int per = 2 * (ny + 1);
  const int s = (int)loc / per;   // launch totals are int: loc < 2^31
  if (s >= V.nsamp) return;
  const int k = (int)(loc - (int64_t)s * per);
  const int j = k >> 1, c = k & 1, i = nx - 1 + c;
  const int t = V.sbase + s;
  const T dl = (T)(-shortening);
  const T rx = (T)V.g.rx, ry = (T)V.g.ry, w = (T)V.g.w;
  V2<T> kd = zero2<T>();
#pragma unroll
  for (int q = 0; q < 2; ++q) {   // element rows j - 1 (node on its top edge) and j (bottom edge)
    const int ej = j - 1 + q;
    if (ej < 0 || ej >= ny) continue;
    const int64_t e = (int64_t)s * nx * ny + (int64_t)ej * nx + (nx - 1);
    const Coef<T> C = coef_from_trig2<T>(L.U, V.trig2[2 * e], V.trig2[2 * e + 1]);
    V2<T> o1, o2, o3, o4;
    element_apply<T>(C, rx, ry, w, zero2<T>(), v2<T>(dl, (T)0), v2<T>(dl, (T)0), zero2<T>(), o1, o2, o3, o4);
    const V2<T> o = c == 0 ? (q == 0 ? o4 : o1) : (q == 0 ? o3 : o2);
    kd.u += o.u;
    kd.v += o.v;
  }
  V2<T> r = v2<T>(-kd.u, -kd.v);
  if (dir_u(i, nx)) r.u = 0;
  if (dir_v(i)) r.v = 0;
  const int64_t node = (int64_t)s * nxp * (ny + 1) + (int64_t)j * nxp + i;
  st2(V.o0 + 2 * node, r);
  atomicAdd(&S.rr64[t], (double)r.u * r.u + (double)r.v * r.v);
  if (c == 1) {
    atomicAdd(&S.react[t], (double)kd.u);
    double* d = static_cast<double*>(V.ext1);
    if constexpr (sizeof(T) == 4) DStore<float>::put(d, 2 * node, DF{-sh_hi, -sh_lo});
    else d[2 * node] = -shortening;
  }
}

// Initial iterate from the same sample's solution on the next coarser mesh (nested
// iteration): bilinear prolongation of the coarse iterate, Dirichlet values included
// (both meshes prescribe the same end values, which the prolongation reproduces).
// ext0 = coarse d, ext1 = fine d (both DStore<TI>); view geometry = the fine mesh.
// One thread per fine node.
template <typename TI>
__global__ void k_prolong_d(const __grid_constant__ ViewList<TI> L) {
  int vi;
  int64_t loc;
  if (!find_point(L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, vi, loc)) return;
  const View<TI>& V = L.v[vi];
  const int nx = V.g.nx, ny = V.g.ny, nxp = nx + 1;
  const int per = nxp * (ny + 1);
  const int s = (int)loc / per;   // launch totals are int: loc < 2^31
  if (s >= V.nsamp) return;
  const int node = (int)(loc - (int64_t)s * per);
  const int j = node / nxp, i = node - j * nxp;
  const int nxc = nx / 2, nyc = ny / 2, I = i >> 1, J = j >> 1;
  const bool fi = i & 1, fj = j & 1;
  const double* dc = static_cast<const double*>(V.ext0);
  double* df = static_cast<double*>(V.ext1);
  const int64_t cb = (int64_t)s * 2 * (nxc + 1) * (nyc + 1);
  auto at = [&](int II, int JJ, int comp) { return cb + 2 * ((int64_t)JJ * (nxc + 1) + II) + comp; };
  const int64_t fo = (int64_t)s * 2 * per + 2 * (int64_t)node;
  using D = DStore<TI>;
#pragma unroll
  for (int comp = 0; comp < 2; ++comp) {
    typename D::Val v = D::get(dc, at(I, J, comp));
    if (fi) v = v + D::get(dc, at(I + 1, J, comp));
    if (fj) {
      typename D::Val t = D::get(dc, at(I, J + 1, comp));
      if (fi) t = t + D::get(dc, at(I + 1, J + 1, comp));
      v = v + t;
    }
    const TI f = (fi && fj) ? (TI)0.25 : ((fi || fj) ? (TI)0.5 : (TI)1);   // powers of two: exact
    if constexpr (sizeof(TI) == 4) D::put(df, fo + comp, DF{v.hi * f, v.lo * f});
    else D::put(df, fo + comp, v * f);
  }
}

// Fibre-direction compressive stress at centroids in [x0, x1]: a = d (DStore<TI>),
// ext0 = trig2 (TI). The displacement differences that form the centroid strain are
// taken from the stored iterate at its own accuracy (they cancel); strain, stress and
// the fibre-frame projection follow in TI (relative error ~1e-7 on the mixed path).
// One warp per element row: lanes stride over the row's central columns (Geo c0..c1,
// found on the host with the definition's double-precision centroid test), and the
// row maximum goes to qoi[2 s + 1] with one atomicMax on the ordered bit pattern of
// the non-negative double.
template <typename TI>
__global__ void k_stress(const __grid_constant__ ViewList<double> L, SampleState S) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  int vi;
  int64_t loc;
  if (!find_point(L, gw, vi, loc)) return;
  const View<double>& V = L.v[vi];
  const int nx = V.g.nx, ny = V.g.ny, nxp = nx + 1;
  const int s = (int)loc / ny;   // launch totals are int: loc < 2^31
  if (s >= V.nsamp) return;
  const int j = (int)(loc - (int64_t)s * ny);
  const int t = V.sbase + s;
  const int ia = V.g.c0, ib = V.g.c1;
  using R = TI;   // single precision on the mixed path, double on the double path
  using D = DStore<TI>;
  const double* d = V.a + (int64_t)s * 2 * nxp * (ny + 1);
  const TI* t2 = static_cast<const TI*>(V.ext0) + 2 * ((int64_t)s * nx * ny + (int64_t)j * nx);
  const R rx = (R)V.g.rx, ry = (R)V.g.ry;
  R vmax = (R)0;
  for (int i = ia + lane; i <= ib; i += 32) {
    const int n1 = j * nxp + i, n2 = n1 + 1, n3 = n1 + nxp + 1, n4 = n1 + nxp;
    const R au = D::diff(d, 2 * n2, 2 * n1) + D::diff(d, 2 * n3, 2 * n4);
    const R bu = D::diff(d, 2 * n4, 2 * n1) + D::diff(d, 2 * n3, 2 * n2);
    const R av = D::diff(d, 2 * n2 + 1, 2 * n1 + 1) + D::diff(d, 2 * n3 + 1, 2 * n4 + 1);
    const R bv = D::diff(d, 2 * n4 + 1, 2 * n1 + 1) + D::diff(d, 2 * n3 + 1, 2 * n2 + 1);
    const R ex = rx * au, ey = ry * bv, exy = ry * bu + rx * av;
    const R c2 = t2[2 * i], s2 = t2[2 * i + 1];
    const Coef<R> C = coef_from_trig2<R>(L.U, c2, s2);
    const R sx = C.c11 * ex + C.c12 * ey + C.c16 * exy;
    const R sy = C.c12 * ex + C.c22 * ey + C.c26 * exy;
    const R sxy = C.c16 * ex + C.c26 * ey + C.c66 * exy;
    // fibre-frame normal stress: cos^2 t sx + sin^2 t sy + 2 sin t cos t sxy
    const R s11 = (R)0.5 * ((R)1 + c2) * sx + (R)0.5 * ((R)1 - c2) * sy + s2 * sxy;
    vmax = max(vmax, -s11);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) vmax = max(vmax, __shfl_xor_sync(0xffffffffu, vmax, o));
  const double m = (double)vmax;
  if (lane == 0 && m > 0.0)
    atomicMax(reinterpret_cast<unsigned long long*>(&S.qoi[2 * t + 1]),
              (unsigned long long)__double_as_longlong(m));
}

template <typename T>
__global__ void k_react_delta(const __grid_constant__ ViewList<T> L, SampleState S) {
  int vi;
  int64_t loc;
  if (!find_point(L, (int64_t)blockIdx.x * blockDim.x + threadIdx.x, vi, loc)) return;
  const View<T>& V = L.v[vi];
  const int nx = V.g.nx, ny = V.g.ny, nxp = nx + 1;
  const int s = (int)loc / ny;   // launch totals are int: loc < 2^31
  if (s >= V.nsamp) return;
  const int t = V.sbase + s;
  if (!S.outer_active[t]) return;
  const int j = (int)(loc - (int64_t)s * ny), i = nx - 1;
  const T* x = V.a + (int64_t)s * 2 * nxp * (ny + 1);
  auto node = [&](int ii, int jj) { return v2<T>(x[2 * (jj * nxp + ii)], x[2 * (jj * nxp + ii) + 1]); };
  const int64_t e = (int64_t)s * nx * ny + (int64_t)j * nx + i;
  const Coef<T> C = V.trig2 ? coef_from_trig2<T>(L.U, V.trig2[2 * e], V.trig2[2 * e + 1])
                            : coef_from_trig<T>(L.U, V.trig[4 * e], V.trig[4 * e + 1], V.trig[4 * e + 2],
                                                V.trig[4 * e + 3]);
  V2<T> o1, o2, o3, o4;
  element_apply<T>(C, (T)V.g.rx, (T)V.g.ry, (T)V.g.w, node(i, j), node(i + 1, j), node(i + 1, j + 1), node(i, j + 1),
                   o1, o2, o3, o4);
  atomicAdd(&S.react[t], (double)o2.u + (double)o3.u);
}

// Energy-consistent reaction. With the load entering only through the prescribed end
// shortening, d^T K d = -d_F . (K d)_F + shortening * R, R = -sum of (K d)_u over x = lx,
// so at the exact discrete solution R = d^T K d / shortening; for an approximate d
// that form differs from the nodal sum by -(d_F . r_F) / shortening (r_F = -(K d)_F,
// the final refinement residual) and its error is quadratic in the solve error
// (||e||_K^2 / shortening) instead of linear. qoi[2 s] += -(d . r) / shortening for
// every converged sample: a = r (inner precision, zero on Dirichlet DOFs), ext0 = d.
// One warp per node row.
template <typename T>
__global__ void k_react_energy(const __grid_constant__ ViewList<T> L, SampleState S, double inv_shortening) {
  const int64_t gw = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  int vi;
  int64_t loc;
  if (!find_point(L, gw, vi, loc)) return;
  const View<T>& V = L.v[vi];
  const int rows = V.g.ny + 1;
  const int s = (int)loc / rows;   // launch totals are int: loc < 2^31
  if (s >= V.nsamp) return;
  const int t = V.sbase + s;
  if (S.status[t] != 0) return;
  const int j = (int)(loc - (int64_t)s * rows);
  const int nv = 2 * (V.g.nx + 1);
  const int64_t off = ((int64_t)s * rows + j) * nv;
  const double* d = static_cast<const double*>(V.ext0);
  const T* r = V.a + off;
  LaneSum<T> acc;   // the correction is needed to a few digits only
  for (int k = lane; k < nv; k += 32) {
    if constexpr (sizeof(T) == 4) {
      const DF x = DStore<float>::get(d, off + k);
      acc.add(x.hi * r[k] + x.lo * r[k]);
    } else {
      acc.add(d[off + k] * r[k]);
    }
  }
  const double sum = warp_sum((double)acc.value());
  if (lane == 0) atomicAdd(&S.qoi[2 * t], -sum * inv_shortening);
}

__global__ void k_inner_end(SampleState S, int total) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total || !S.outer_active[t]) return;
  if (S.active[t]) {   // iteration cap reached
    S.active[t] = 0;
    S.status[t] = MLMC_ERR_NOT_CONVERGED;
    S.outer_active[t] = 0;
    return;
  }
  if (!S.exact[t]) S.rr64[t] = S.red_rr[t];
}

__global__ void k_outer_init(SampleState S, int total) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total) return;
  S.rrf[t] = S.rr64[t];
}

// After a refinement residual: record the reaction, stop converged samples, and
// set up the next inner solve for the rest.
__global__ void k_outer_check(SampleState S, int total, double rtol, double floor_tol, int* outer_count) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= total || !S.outer_active[t]) return;
  const double rr = S.rr64[t];
  S.qoi[2 * t] = -S.react[t];
  S.rr64[t] = 0.0;
  const double target = rtol * rtol * S.rrf[t];
  if (rr <= target || S.status[t] != 0) {
    S.outer_active[t] = 0;
    S.active[t] = 0;
    return;
  }
  // solve the correction to what the outer target needs (with margin), no tighter
  // than the inner arithmetic supports
  double tol2 = 0.25 * target / rr;
  if (tol2 < floor_tol * floor_tol) tol2 = floor_tol * floor_tol;
  S.tol2[t] = tol2;
  S.rr_ref[t] = rr;
  S.active[t] = 1;
  S.alpha[t] = 0.0;
  S.beta[t] = 0.0;
  S.rz_old[t] = 0.0;
  S.red_rr[t] = 0.0;
  S.red_rz[t] = 0.0;
  S.red_pq[t] = 0.0;
  atomicAdd(outer_count, 1);
}

template <typename T, typename Op>
cudaError_t launch_strip_op(const ViewList<T>& L, SampleState S, int total_warps, cudaStream_t st) {
  if (total_warps <= 0) return cudaSuccess;
  const int blocks = (total_warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
  constexpr int P = sizeof(T) == 4 ? Op::kP32 : kPrefetch64;
  size_t smem = 0;
  if constexpr (Op::kAsync) smem = sizeof(typename Op::Slot) * Op::kDepth * kWarpsPerBlock;
  k_strip<T, P, Op><<<blocks, kWarpsPerBlock * kWarp, smem, st>>>(L, S);
  return cudaGetLastError();
}

inline int blocks_for(int64_t threads, int bs) { return (int)((threads + bs - 1) / bs); }

}  // namespace

int strip_cols(StripOp op) {
  switch (op) {
    case StripOp::PreTop:
    case StripOp::PreR:
    case StripOp::Post:
    case StripOp::PostTop: return kSmoothCols;
    default: return kStripCols;
  }
}

template <typename T>
cudaError_t launch_strip(StripOp op, const ViewList<T>& L, SampleState S, int total_warps, cudaStream_t st) {
  switch (op) {
    case StripOp::Apply: return launch_strip_op<T, OpApply<T>>(L, S, total_warps, st);
    case StripOp::PreTop: return launch_strip_op<T, OpPreTop<T>>(L, S, total_warps, st);
    case StripOp::PreR: return launch_strip_op<T, OpPreR<T>>(L, S, total_warps, st);
    case StripOp::Post: return launch_strip_op<T, OpPost<T, false>>(L, S, total_warps, st);
    case StripOp::PostTop: return launch_strip_op<T, OpPost<T, true>>(L, S, total_warps, st);
    case StripOp::PcgP: return launch_strip_op<T, OpPcgP<T>>(L, S, total_warps, st);
  }
  return cudaErrorInvalidValue;
}

template <typename TI>
cudaError_t launch_resid64(const ViewList<double>& L, SampleState S, int total_warps, cudaStream_t st) {
  return launch_strip_op<double, OpResid<TI>>(L, S, total_warps, st);
}

template <typename T>
cudaError_t launch_trig_average(const ViewList<T>& L, int total_threads, cudaStream_t st) {
  if (total_threads <= 0) return cudaSuccess;
  k_trig_average<T><<<blocks_for(total_threads, 256), 256, 0, st>>>(L);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_invdiag(const ViewList<T>& L, int total_threads, cudaStream_t st) {
  if (total_threads <= 0) return cudaSuccess;
  k_invdiag<T><<<blocks_for(total_threads, 256), 256, 0, st>>>(L);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarsest_setup(const ViewList<T>& L, int total_blocks, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  k_coarsest_setup<T><<<total_blocks, 64, 0, st>>>(L);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_coarsest_solve(const ViewList<T>& L, SampleState S, int total_warps, cudaStream_t st) {
  if (total_warps <= 0) return cudaSuccess;
  k_coarsest_solve<T><<<blocks_for(total_warps, kWarpsPerBlock), kWarpsPerBlock * kWarp, 0, st>>>(L, S);
  return cudaGetLastError();
}

bool bottom_fits(const Geo& ga, const Geo& gb, const Geo& gc) {
  return (ga.nx + 1) * (ga.ny + 1) <= kBotNodes && (gb.nx + 1) * (gb.ny + 1) <= kBotNodesB &&
         2 * (gc.nx + 1) * (gc.ny + 1) <= kMaxCoarsestDofs && ga.nx == 2 * gb.nx && ga.ny == 2 * gb.ny &&
         gb.nx == 2 * gc.nx && gb.ny == 2 * gc.ny;
}

cudaError_t launch_bottom(const BottomList& L, SampleState S, int total_warps, cudaStream_t st) {
  if (total_warps <= 0) return cudaSuccess;
  k_bottom<<<blocks_for(total_warps, kWarpsPerBlock), kWarpsPerBlock * kWarp, 0, st>>>(L, S);
  return cudaGetLastError();
}

int deep_floats(const Geo* g, int nb, const Geo& gc) {
  auto up4 = [](int c) { return (c + 3) & ~3; };
  int f = 0;
  for (int k = 0; k < nb; ++k) {
    const int n = g[k].nodes(), ne = g[k].nx * g[k].ny;
    f += 4 * up4(2 * n) + up4(n) + up4(4 * ne);
  }
  return f + 2 * up4(2 * gc.nodes());
}

bool deep_fits(const Geo* g, int nb, const Geo& gc) {
  if (nb < 1 || nb > kDeepMax || 2 * gc.nodes() > kMaxCoarsestDofs) return false;
  for (int k = 0; k < nb; ++k) {
    const Geo& nxt = k + 1 < nb ? g[k + 1] : gc;
    if (g[k].nx != 2 * nxt.nx || g[k].ny != 2 * nxt.ny) return false;
  }
  return deep_floats(g, nb, gc) <= kDeepFloats;
}

cudaError_t launch_bottom_deep(const DeepList& L, SampleState S, int total_blocks, int floats, cudaStream_t st) {
  if (total_blocks <= 0) return cudaSuccess;
  k_bottom_deep<<<total_blocks, kDeepThreads, sizeof(float) * (size_t)floats, st>>>(L, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_update_d(const ViewList<T>& L, SampleState S, int total_threads, cudaStream_t st) {
  if (total_threads <= 0) return cudaSuccess;
  k_update_d<T><<<blocks_for(total_threads, 256), 256, 0, st>>>(L, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_lift_resid(const ViewList<T>& L, SampleState S, double shortening, int total_threads,
                              cudaStream_t st) {
  if (total_threads <= 0) return cudaSuccess;
  const float hi = (float)shortening, lo = (float)(shortening - (double)hi);
  k_lift_resid<T><<<blocks_for(total_threads, 128), 128, 0, st>>>(L, S, hi, lo, shortening);
  return cudaGetLastError();
}

template <typename TI>
cudaError_t launch_prolong_d(const ViewList<TI>& L, int total_threads, cudaStream_t st) {
  if (total_threads <= 0) return cudaSuccess;
  k_prolong_d<TI><<<blocks_for(total_threads, 256), 256, 0, st>>>(L);
  return cudaGetLastError();
}

template <typename TI>
cudaError_t launch_stress(const ViewList<double>& L, SampleState S, int total_warps, cudaStream_t st) {
  if (total_warps <= 0) return cudaSuccess;
  k_stress<TI><<<blocks_for((int64_t)total_warps * 32, 256), 256, 0, st>>>(L, S);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_react_energy(const ViewList<T>& L, SampleState S, double shortening, int total_warps,
                                cudaStream_t st) {
  if (total_warps <= 0) return cudaSuccess;
  k_react_energy<T><<<blocks_for((int64_t)total_warps * 32, 128), 128, 0, st>>>(L, S, 1.0 / shortening);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_react_delta(const ViewList<T>& L, SampleState S, int total_threads, cudaStream_t st) {
  if (total_threads <= 0) return cudaSuccess;
  k_react_delta<T><<<blocks_for(total_threads, 128), 128, 0, st>>>(L, S);
  return cudaGetLastError();
}

cudaError_t launch_inner_end(SampleState S, int total, cudaStream_t st) {
  k_inner_end<<<blocks_for(total, 256), 256, 0, st>>>(S, total);
  return cudaGetLastError();
}

cudaError_t launch_outer_init(SampleState S, int total, cudaStream_t st) {
  k_outer_init<<<blocks_for(total, 256), 256, 0, st>>>(S, total);
  return cudaGetLastError();
}

cudaError_t launch_outer_check(SampleState S, int total, double rtol, double floor_tol, int* outer_count,
                               cudaStream_t st) {
  k_outer_check<<<blocks_for(total, 256), 256, 0, st>>>(S, total, rtol, floor_tol, outer_count);
  return cudaGetLastError();
}

#define MLMC_INST(T)                                                                                        \
  template cudaError_t launch_strip<T>(StripOp, const ViewList<T>&, SampleState, int, cudaStream_t);       \
  template cudaError_t launch_trig_average<T>(const ViewList<T>&, int, cudaStream_t);                      \
  template cudaError_t launch_invdiag<T>(const ViewList<T>&, int, cudaStream_t);                           \
  template cudaError_t launch_coarsest_setup<T>(const ViewList<T>&, int, cudaStream_t);                    \
  template cudaError_t launch_coarsest_solve<T>(const ViewList<T>&, SampleState, int, cudaStream_t);       \
  template cudaError_t launch_update_d<T>(const ViewList<T>&, SampleState, int, cudaStream_t);             \
  template cudaError_t launch_react_delta<T>(const ViewList<T>&, SampleState, int, cudaStream_t);          \
  template cudaError_t launch_react_energy<T>(const ViewList<T>&, SampleState, double, int, cudaStream_t);  \
  template cudaError_t launch_resid64<T>(const ViewList<double>&, SampleState, int, cudaStream_t);         \
  template cudaError_t launch_lift_resid<T>(const ViewList<T>&, SampleState, double, int, cudaStream_t);  \
  template cudaError_t launch_prolong_d<T>(const ViewList<T>&, int, cudaStream_t);                        \
  template cudaError_t launch_stress<T>(const ViewList<double>&, SampleState, int,                         \
                                        cudaStream_t);
MLMC_INST(float)
MLMC_INST(double)
#undef MLMC_INST

}  // namespace mlmc
