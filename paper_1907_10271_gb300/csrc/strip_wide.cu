// FP32 smoothing and PCG strip kernels with a node pair per lane: the operations of
// fem.cu's PreTop, PreR, Post, PostTop and PcgP (same arithmetic per node, Eq.
// matrixinplane's operator and the pair-block Jacobi smoother of the V-cycle), laid
// out so that lane l of a warp owns the two node columns 2l and 2l + 1 of its strip.
//
// Why a pair per lane. The one-column kernels are issue-bound on the finest mesh: per
// node and row a lane spends its instructions on staging copies and their addresses,
// the smoother's partner exchange (a shuffle), the two shuffles of the element pass
// and the loop, of which only the element arithmetic grows with the nodes it serves.
// With a pair per lane the smoother's pair {2m, 2m + 1} is in one thread, one shuffle
// each way per row serves two nodes, a strip has 60 output columns of 64 (one halo
// lane each side) instead of 28 of 32, and shared-memory reads are 16 bytes.
//
// Strip t of a view covers virtual columns vb .. vb + 63 with vb = 60 t - 2; lane l
// computes columns vb + 2l (node A) and vb + 2l + 1 (node B), lanes 1 .. 30 write
// them. A virtual column is a node column of one sample (packed views: samples side
// by side with one padding column, width vw = nx + 2, so a pair never spans two
// samples because nx is even on every level these kernels run on). Rows are staged
// per warp through a ring of shared-memory slots by cp.async, but the copies are
// contiguous over the lanes (lane l copies columns vb + l and vb + 32 + l), so a lane
// reads values other lanes copied: each step waits for its own copies and then meets
// the warp at __syncwarp() before reading, and meets it again before refilling a slot.
// Element column i is the element to the right of node column i: lane l evaluates
// elements A (between its nodes) and B (between its node B and the next lane's A).
#include <type_traits>

#include "../../include/mlmc.h"
#include "fem.cuh"
#include "strip.cuh"

namespace mlmc {

namespace {

constexpr int kWideHalo = 2;   // halo node columns on each side (one lane)

using F2 = V2<float>;

__device__ __forceinline__ F2 f2(float u, float v) { return v2<float>(u, v); }
__device__ __forceinline__ F2 zf2() { return v2<float>(0.f, 0.f); }
__device__ __forceinline__ F2 add2(F2 a, F2 b) { return f2(a.u + b.u, a.v + b.v); }
__device__ __forceinline__ F2 shdn(F2 a) {
  return f2(__shfl_down_sync(0xffffffffu, a.u, 1), __shfl_down_sync(0xffffffffu, a.v, 1));
}
__device__ __forceinline__ F2 shup(F2 a) {
  return f2(__shfl_up_sync(0xffffffffu, a.u, 1), __shfl_up_sync(0xffffffffu, a.v, 1));
}
__device__ __forceinline__ F2 get2(const float* p) {
  const float2 t = *reinterpret_cast<const float2*>(p);
  return f2(t.x, t.y);
}
__device__ __forceinline__ F2 lo2(float4 t) { return f2(t.x, t.y); }
__device__ __forceinline__ F2 hi2(float4 t) { return f2(t.z, t.w); }

// Homogeneous Dirichlet DOFs of node column i (u on x = 0 and x = lx, v on x = 0).
__device__ __forceinline__ F2 dmask(int i, int nx, F2 x) {
  if (dir_u(i, nx)) x.u = 0.f;
  if (dir_v(i)) x.v = 0.f;
  return x;
}

// The node pair of a lane: A at column i of sample s (s clamped into the view), B at
// i + 1; va / vb: real nodes of a real sample; oa / ob: written by this lane.
struct WCol {
  int s, i;
  bool va, vb, live, oa, ob;
};

// (sample, column) of virtual column v; valid when it is a node column of a sample.
__device__ __forceinline__ void vcol_of(const View<float>& V, int s, int v, int& q, int& i, bool& valid) {
  if (V.packed) {
    const int qq = v >= 0 ? v / V.vw : 0;
    i = v >= 0 ? v - qq * V.vw : v;
    valid = v >= 0 && qq < V.nsamp && i <= V.g.nx;
    q = min(qq, V.nsamp - 1);
  } else {
    q = s;
    i = v;
    valid = v >= 0 && v <= V.g.nx;
  }
}

__device__ __forceinline__ WCol wide_col(const View<float>& V, int s, int v) {
  WCol c;
  vcol_of(V, s, v, c.s, c.i, c.va);
  c.vb = c.va && c.i + 1 <= V.g.nx;
  c.live = c.oa = c.ob = false;
  return c;
}

// Sums v over the output lanes of every sample whose columns this warp writes (lanes
// hold ascending columns, so each pass takes one sample's run of lanes) and calls
// f(sample, total) on lane 0 for each.
template <typename F>
__device__ __forceinline__ void per_sample_wide(const WCol& lc, double v, F&& f) {
  const bool out = lc.oa || lc.ob;
  unsigned m = __ballot_sync(0xffffffffu, out);
  while (m != 0u) {
    const int sa = __shfl_sync(0xffffffffu, lc.s, __ffs(m) - 1);
    const bool mine = out && lc.s == sa;
    const double t = warp_sum(mine ? v : 0.0);
    if ((threadIdx.x & 31) == 0) f(sa, t);
    m &= ~__ballot_sync(0xffffffffu, mine);
  }
}

// Load side of a lane: node columns vb + lane and vb + 32 + lane (index of the node in
// row 0, clamped into the sample, and whether it is a node) and the element columns of
// the same numbers.
struct LoadCols {
  int64_t n0, n1, e0, e1;
  bool nv0, nv1, ev0, ev1;
  __device__ void init(const View<float>& V, int s, int vb, int lane) {
    const int nx = V.g.nx, ny = V.g.ny;
    const int64_t N = (int64_t)(nx + 1) * (ny + 1), NE = (int64_t)nx * ny;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      int q, i;
      bool valid;
      vcol_of(V, s, vb + lane + 32 * h, q, i, valid);
      const int64_t n = q * N + min(max(i, 0), nx);
      const int64_t e = q * NE + min(max(i, 0), nx - 1);
      const bool ev = valid && i < nx;
      if (h == 0) {
        n0 = n;
        e0 = e;
        nv0 = valid;
        ev0 = ev;
      } else {
        n1 = n;
        e1 = e;
        nv1 = valid;
        ev1 = ev;
      }
    }
  }
  // node row j of a vector of float2 per node into dst[64] (lane's entries l, l + 32)
  __device__ __forceinline__ void node2(float2* dst, const float* src, int64_t jr, int lane) const {
    cp_async<8>(&dst[lane], src + 2 * (n0 + jr), nv0);
    cp_async<8>(&dst[lane + 32], src + 2 * (n1 + jr), nv1);
  }
  // node row j of a vector of one float per node into dst[64]
  __device__ __forceinline__ void node1(float* dst, const float* src, int64_t jr, int lane) const {
    cp_async<4>(&dst[lane], src + (n0 + jr), nv0);
    cp_async<4>(&dst[lane + 32], src + (n1 + jr), nv1);
  }
  // element row (offset er = j nx) of the finest mesh's (cos 2t, sin 2t)
  __device__ __forceinline__ void elem2(float2* dst, const float* src, int64_t er, int lane) const {
    cp_async<8>(&dst[lane], src + 2 * (e0 + er), ev0);
    cp_async<8>(&dst[lane + 32], src + 2 * (e1 + er), ev1);
  }
  // element row of a coarse mesh's averaged trig 4-vectors
  __device__ __forceinline__ void elem4(float4* dst, const float* src, int64_t er, int lane) const {
    cp_async<16>(&dst[lane], src + 4 * (e0 + er), ev0);
    cp_async<16>(&dst[lane + 32], src + 4 * (e1 + er), ev1);
  }
};

// Element stiffness of the lane's elements A and B, from the staged element row:
// C_bar / 4 (square elements) or C_bar.
struct ElemCoef {
  Coef<float> a, b;
};
__device__ __forceinline__ ElemCoef coefs_top(const Invariants& U, const float2* e, int lane, bool square) {
  const float4 t = reinterpret_cast<const float4*>(e)[lane];
  ElemCoef c;
  if (square) {
    c.a = coef_from_trig2<float, true>(U, t.x, t.y);
    c.b = coef_from_trig2<float, true>(U, t.z, t.w);
  } else {
    c.a = coef_from_trig2<float>(U, t.x, t.y);
    c.b = coef_from_trig2<float>(U, t.z, t.w);
  }
  return c;
}
__device__ __forceinline__ ElemCoef coefs_coarse(const Invariants& U, const float4* e, int lane, bool square) {
  const float4 ta = e[2 * lane], tb = e[2 * lane + 1];
  ElemCoef c;
  if (square) {
    c.a = coef_from_trig<float, true>(U, ta.x, ta.y, ta.z, ta.w);
    c.b = coef_from_trig<float, true>(U, tb.x, tb.y, tb.z, tb.w);
  } else {
    c.a = coef_from_trig<float>(U, ta.x, ta.y, ta.z, ta.w);
    c.b = coef_from_trig<float>(U, tb.x, tb.y, tb.z, tb.w);
  }
  return c;
}

__device__ __forceinline__ void elem_apply(const Coef<float>& C, const Geo& g, F2 n1, F2 n2, F2 n3, F2 n4, F2& o1,
                                           F2& o2, F2& o3, F2& o4) {
  if (g.square) element_apply_square<float>(C, n1, n2, n3, n4, o1, o2, o3, o4);
  else element_apply<float>(C, (float)g.rx, (float)g.ry, (float)g.w, n1, n2, n3, n4, o1, o2, o3, o4);
}

// Values of the lane's pair.
struct P2 {
  F2 a, b;
};

// Element pass of one row for a node pair (the pair form of fem.cu's RowCarry): node A
// sums element A's o1 of row er and o4 of row er - 1 and the left lane's element B o2
// (row er) and o3 (row er - 1), those two added before the one shuffle up; node B sums
// element B's o1 and o4 and element A's o2 and o3, all in the thread. The right lane's
// bottom node A is its top node A of the previous row, so one shuffle down per row.
struct PairCarry {
  F2 pa, pb, pr;       // bottom values of the next element row: own A, B, right lane's A
  F2 a3, a4, b3, b4;   // previous element row's contributions to its top nodes
  __device__ __forceinline__ explicit PairCarry(P2 p0) : pa(p0.a), pb(p0.b), pr(shdn(p0.a)) {
    a3 = a4 = b3 = b4 = zf2();
  }
  // pt: top node values of element row er; returns K x at nodes (A, er), (B, er)
  __device__ __forceinline__ P2 step(const ElemCoef& C, const Geo& g, bool elA, bool elB, P2 pt) {
    const int lane = threadIdx.x & 31;
    const F2 ptr = shdn(pt.a);
    F2 oa1 = zf2(), oa2 = zf2(), oa3 = zf2(), oa4 = zf2();
    F2 ob1 = zf2(), ob2 = zf2(), ob3 = zf2(), ob4 = zf2();
    if (elA) elem_apply(C.a, g, pa, pb, pt.b, pt.a, oa1, oa2, oa3, oa4);
    if (elB) elem_apply(C.b, g, pb, pr, ptr, pt.b, ob1, ob2, ob3, ob4);
    F2 f = shup(add2(ob2, b3));
    if (lane == 0) f = zf2();
    P2 kx;
    kx.a = add2(add2(oa1, a4), f);
    kx.b = add2(add2(ob1, b4), add2(oa2, a3));
    a3 = oa3;
    a4 = oa4;
    b3 = ob3;
    b4 = ob4;
    pa = pt.a;
    pb = pt.b;
    pr = ptr;
    return kx;
  }
  // K x at the top node row of the last element row
  __device__ __forceinline__ P2 top() const {
    const int lane = threadIdx.x & 31;
    F2 f = shup(b3);
    if (lane == 0) f = zf2();
    P2 kx;
    kx.a = add2(a4, f);
    kx.b = add2(b4, a3);
    return kx;
  }
};

// Walks the warp's strip up its chunk of node rows with the rows staged through D
// slots (step k holds node row er0 + k and element row er0 + k - 1). Op provides
// fetch(slot, j) / fetchE(slot, er) (the copies of one row), in(slot, j) (the values K
// is applied to at row j, zero off the mesh, keeping what out() needs), coefs(slot),
// out(j, kx) and shift() (row advance).
template <int D, typename Op>
__device__ __forceinline__ void wide_loop(const Invariants& U, const View<float>& V, const WCol& lc, int chunk,
                                          Op& op, typename Op::Slot* ring) {
  const int lane = threadIdx.x & 31;
  const int ny = V.g.ny;
  const int rows = V.rows > 0 ? V.rows : kRowChunk;
  const int j0 = chunk * rows;
  const int j1 = min(j0 + rows - 1, ny);
  const int er0 = max(j0 - 1, 0);
  const int er1 = min(j1, ny - 1);
  const int nsteps = er1 - er0 + 2;   // node rows er0 .. er1 + 1
  const bool elA = lc.vb;
  const bool elB = lc.vb && lc.i + 1 < V.g.nx && lane < 31;
  auto issue = [&](int k, int slot) {
    __syncwarp();   // every lane has read the slot being refilled
    if (k < nsteps) {
      op.fetch(ring[slot], er0 + k);
      if (k >= 1) op.fetchE(ring[slot], er0 + k - 1);
    }
    cp_async_commit();   // one group per step, empty past the end
  };
#pragma unroll
  for (int k = 0; k < D; ++k) issue(k, k);
  cp_async_wait<D - 1>();
  __syncwarp();
  PairCarry rc(op.in(ring[0], er0));
  op.shift();
  int refill = 0, slot = 1 % D;
  for (int k = 1; k < nsteps; ++k) {
    issue(k + D - 1, refill);
    cp_async_wait<D - 1>();
    __syncwarp();
    const int er = er0 + k - 1;
    const typename Op::Slot& sl = ring[slot];
    const P2 pt = op.in(sl, er + 1);
    const ElemCoef C = op.coefs(U, sl);
    const P2 kx = rc.step(C, V.g, elA, elB, pt);
    if (er >= j0) op.out(er, kx);
    op.shift();
    refill = slot;
    slot = slot + 1 == D ? 0 : slot + 1;
  }
  cp_async_wait<0>();
  if (er1 + 1 == ny && ny >= j0 && ny <= j1) op.out(ny, rc.top());
}

// ---------------------------------------------------------------- operand handlers
// Vectors as in fem.cu (float2 per node, [sample][row][column]); the handlers differ
// from fem.cu's only in holding two nodes per lane.

__device__ __forceinline__ float4 lane4(const float2* a) { return reinterpret_cast<const float4*>(a)[threadIdx.x & 31]; }
__device__ __forceinline__ float2 lane2(const float* a) { return reinterpret_cast<const float2*>(a)[threadIdx.x & 31]; }

// Outputs go out through a per-warp stage in shared memory: lane l puts its pair at
// entry l (16 bytes), and after __syncwarp() stores the columns it copies in (vb + l
// and vb + 32 + l), so every store instruction writes 256 contiguous bytes of a sample
// row instead of every other 8 bytes of 512.
struct WideBase {
  const View<float>& V;
  const WCol& c;
  LoadCols ld;
  float4* stage;   // [outputs][32] of this warp
  bool so0, so1;   // columns vb + lane, vb + 32 + lane are outputs of this strip
  int rs;          // nodes per row
  int lane;
  __device__ WideBase(const View<float>& v, int s, int vb, const WCol& lc) : V(v), c(lc) {
    lane = threadIdx.x & 31;
    ld.init(v, s, vb, lane);
    rs = v.g.nx + 1;
    stage = nullptr;
    so0 = so1 = false;
  }
  // after the lanes' output flags are set (every lane)
  __device__ void set_outputs(float4* st) {
    stage = st;
    const unsigned ma = __ballot_sync(0xffffffffu, c.oa), mb = __ballot_sync(0xffffffffu, c.ob);
    so0 = (((lane & 1) ? mb : ma) >> (lane >> 1)) & 1u;
    so1 = (((lane & 1) ? mb : ma) >> (16 + (lane >> 1))) & 1u;
  }
  __device__ __forceinline__ int64_t jr(int j) const { return (int64_t)j * rs; }
  __device__ __forceinline__ int64_t er(int e) const { return (int64_t)e * V.g.nx; }
  __device__ __forceinline__ void put(int k, P2 v) const { stage[32 * k + lane] = make_float4(v.a.u, v.a.v, v.b.u, v.b.v); }
  // stores staged output k of node row j into dst (after flush_begin)
  __device__ __forceinline__ void store(int k, float* dst, int j) const {
    const float2* s2 = reinterpret_cast<const float2*>(stage + 32 * k);
    const int64_t r = jr(j);
    if (so0) *reinterpret_cast<float2*>(dst + 2 * (ld.n0 + r)) = s2[lane];
    if (so1) *reinterpret_cast<float2*>(dst + 2 * (ld.n1 + r)) = s2[lane + 32];
  }
};

// PreTop: a = r (old), b = q, c = p, winvd + wc, o0 = x (read and updated); o1 = r'
// = r - alpha q, o2 = r1 = r' - K x1 with x1 = W r' (pair-block Jacobi from zero);
// ||r'||^2 reduced per sample.
struct WPreTop : WideBase {
  static constexpr int kDepth = 2;
  static constexpr int kMinBlocks = 4;
  struct Slot {
    float2 r[64], q[64], w[64], x[64], p[64];
    float c[64];
    float2 e[64];
  };
  float alpha;
  bool act;
  P2 rt, xt, rb, xb;   // r' and the updated x of the row being prepared (t) and written (b)
  LaneSum<float> rr;
  __device__ WPreTop(const View<float>& v, int s, int vb, const WCol& lc, const SampleState& S)
      : WideBase(v, s, vb, lc) {
    act = S.active[v.sbase + lc.s] != 0;
    alpha = (float)S.alpha[v.sbase + lc.s];
  }
  __device__ bool live() const { return act; }
  __device__ void fetch(Slot& S, int j) const {
    const int64_t r = jr(j);
    ld.node2(S.r, V.a, r, lane);
    ld.node2(S.q, V.b, r, lane);
    ld.node2(S.w, V.winvd, r, lane);
    ld.node2(S.x, V.o0, r, lane);
    ld.node2(S.p, V.c, r, lane);
    ld.node1(S.c, V.wc, r, lane);
  }
  __device__ void fetchE(Slot& S, int e) const { ld.elem2(S.e, V.trig2, er(e), lane); }
  __device__ ElemCoef coefs(const Invariants& U, const Slot& S) const { return coefs_top(U, S.e, lane, V.g.square); }
  __device__ P2 in(const Slot& S, int) {
    const float4 r = lane4(S.r), q = lane4(S.q), w = lane4(S.w), x = lane4(S.x), p = lane4(S.p);
    const float2 cc = lane2(S.c);
    rt.a = f2(r.x - alpha * q.x, r.y - alpha * q.y);
    rt.b = f2(r.z - alpha * q.z, r.w - alpha * q.w);
    xt.a = f2(x.x + alpha * p.x, x.y + alpha * p.y);
    xt.b = f2(x.z + alpha * p.z, x.w + alpha * p.w);
    const float ua = c.va ? rt.a.u : 0.f, ub = c.vb ? rt.b.u : 0.f;
    P2 v;
    v.a = c.va ? f2(w.x * rt.a.u + cc.x * ub, w.y * rt.a.v) : zf2();
    v.b = c.vb ? f2(w.z * rt.b.u + cc.y * ua, w.w * rt.b.v) : zf2();
    return v;
  }
  __device__ void shift() {
    rb = rt;
    xb = xt;
  }
  static constexpr int kOut = 3;
  __device__ void out(int j, P2 kx) {
    const int nx = V.g.nx;
    P2 r1;
    r1.a = dmask(c.i, nx, f2(rb.a.u - kx.a.u, rb.a.v - kx.a.v));
    r1.b = dmask(c.i + 1, nx, f2(rb.b.u - kx.b.u, rb.b.v - kx.b.v));
    if (c.oa) rr.add(rb.a.u * rb.a.u + rb.a.v * rb.a.v);
    if (c.ob) rr.add(rb.b.u * rb.b.u + rb.b.v * rb.b.v);
    __syncwarp();
    put(0, r1);
    put(1, rb);
    put(2, xb);
    __syncwarp();
    store(0, V.o2, j);
    store(1, V.o1, j);
    store(2, V.o0, j);
  }
  __device__ void finish(const SampleState& S) {
    per_sample_wide(c, rr.value(), [&](int s, double t) { atomicAdd(&S.red_rr[V.sbase + s], t); });
  }
};

// PcgP: a = z, b = p (old); o0 = p' = z + beta p, o1 = q = K p', p' . q reduced per
// sample (the last warp of a sample takes alpha).
struct WPcgP : WideBase {
  static constexpr int kDepth = 4;
  static constexpr int kMinBlocks = 4;
  struct Slot {
    float2 z[64], p[64], e[64];
  };
  float beta;
  bool act;
  P2 pt, pb;
  LaneSum<float> pq;
  __device__ WPcgP(const View<float>& v, int s, int vb, const WCol& lc, const SampleState& S)
      : WideBase(v, s, vb, lc) {
    act = S.active[v.sbase + lc.s] != 0;
    beta = (float)S.beta[v.sbase + lc.s];
  }
  __device__ bool live() const { return act; }
  __device__ void fetch(Slot& S, int j) const {
    const int64_t r = jr(j);
    ld.node2(S.z, V.a, r, lane);
    ld.node2(S.p, V.b, r, lane);
  }
  __device__ void fetchE(Slot& S, int e) const { ld.elem2(S.e, V.trig2, er(e), lane); }
  __device__ ElemCoef coefs(const Invariants& U, const Slot& S) const { return coefs_top(U, S.e, lane, V.g.square); }
  __device__ P2 in(const Slot& S, int) {
    const float4 z = lane4(S.z), p = lane4(S.p);
    pt.a = f2(z.x + beta * p.x, z.y + beta * p.y);
    pt.b = f2(z.z + beta * p.z, z.w + beta * p.w);
    P2 v;
    v.a = c.va ? pt.a : zf2();
    v.b = c.vb ? pt.b : zf2();
    return v;
  }
  __device__ void shift() { pb = pt; }
  static constexpr int kOut = 2;
  __device__ void out(int j, P2 kx) {
    const int nx = V.g.nx;
    P2 q;
    q.a = dmask(c.i, nx, kx.a);
    q.b = dmask(c.i + 1, nx, kx.b);
    if (c.oa) pq.add(pb.a.u * q.a.u + pb.a.v * q.a.v);
    if (c.ob) pq.add(pb.b.u * q.b.u + pb.b.v * q.b.v);
    __syncwarp();
    put(0, pb);
    put(1, q);
    __syncwarp();
    store(0, V.o0, j);
    store(1, V.o1, j);
  }
  __device__ void finish(const SampleState& S) {
    per_sample_wide(c, pq.value(), [&](int s, double t) {
      const int g = V.sbase + s;
      atomicAdd(&S.red_pq[g], t);
      if (last_tile(S.arrive, g, tiles_of_sample(V, s, kWideCols))) after_p(S, g);
    });
  }
};

// Post / PostTop: a = b, xc (the level below), winvd + wc; o0 = z = x2 + W (b - K x2)
// with x2 = W b + P xc (bilinear prolongation). TOP also reduces b . z (the last warp
// of a sample takes the CG's beta and convergence test).
template <bool TOP>
struct WPost : WideBase {
  static constexpr int kDepth = 3;
  static constexpr int kMinBlocks = 4;
  using E = typename std::conditional<TOP, float2, float4>::type;
  struct Slot {
    float2 b[64], w[64];
    float c[64];
    float2 c0[32], c1[32];   // coarse rows J and (odd rows) J + 1 at the lane's coarse column
    E e[64];
  };
  bool act;
  int nxc;
  int64_t cI;   // coarse node index (row 0) of the lane's coarse column I = i / 2
  P2 bt, bb, xt, xb;
  float4 wt, wb;
  float2 ct, cb;
  LaneSum<float> rz;
  __device__ WPost(const View<float>& v, int s, int vb, const WCol& lc, const SampleState& S)
      : WideBase(v, s, vb, lc) {
    act = S.active[v.sbase + lc.s] != 0;
    nxc = v.g.nx / 2;
    cI = (int64_t)lc.s * (nxc + 1) * (v.g.ny / 2 + 1) + min(max(lc.i, 0), v.g.nx) / 2;
  }
  __device__ bool live() const { return act; }
  __device__ void fetch(Slot& S, int j) const {
    const int64_t r = jr(j);
    ld.node2(S.b, V.a, r, lane);
    ld.node2(S.w, V.winvd, r, lane);
    ld.node1(S.c, V.wc, r, lane);
    const int J = j >> 1, J1 = (j & 1) ? J + 1 : J;   // even rows need no second coarse row
    cp_async<8>(&S.c0[lane], V.xc + 2 * (cI + (int64_t)J * (nxc + 1)));
    cp_async<8>(&S.c1[lane], V.xc + 2 * (cI + (int64_t)J1 * (nxc + 1)), (j & 1) != 0);
  }
  __device__ void fetchE(Slot& S, int e) const {
    if constexpr (TOP) ld.elem2(S.e, V.trig2, er(e), lane);
    else ld.elem4(S.e, V.trig, er(e), lane);
  }
  __device__ ElemCoef coefs(const Invariants& U, const Slot& S) const {
    if constexpr (TOP) return coefs_top(U, S.e, lane, V.g.square);
    else return coefs_coarse(U, S.e, lane, V.g.square);
  }
  // node A (even column) takes coarse column I, node B (odd) columns I and I + 1, which
  // is the next lane's I (the same sample while B is a node)
  __device__ P2 in(const Slot& S, int j) {
    const bool fj = j & 1;
    const float4 b = lane4(S.b), w = lane4(S.w);
    const float2 cc = lane2(S.c);
    const int ln = min(lane + 1, 31);
    F2 ca = f2(S.c0[lane].x, S.c0[lane].y), cn = f2(S.c0[ln].x, S.c0[ln].y);
    if (fj) {
      ca = add2(ca, f2(S.c1[lane].x, S.c1[lane].y));
      cn = add2(cn, f2(S.c1[ln].x, S.c1[ln].y));
    }
    const F2 cB = add2(ca, cn);
    const float fa = fj ? 0.5f : 1.f, fb = fj ? 0.25f : 0.5f;
    bt.a = lo2(b);
    bt.b = hi2(b);
    wt = w;
    ct = cc;
    xt.a = f2(w.x * b.x + fa * ca.u, w.y * b.y + fa * ca.v);
    xt.b = f2(w.z * b.z + fb * cB.u, w.w * b.w + fb * cB.v);
    const float ua = c.va ? b.x : 0.f, ub = c.vb ? b.z : 0.f;
    if (c.va) xt.a.u += cc.x * ub;
    if (c.vb) xt.b.u += cc.y * ua;
    P2 v;
    v.a = c.va ? xt.a : zf2();
    v.b = c.vb ? xt.b : zf2();
    return v;
  }
  __device__ void shift() {
    bb = bt;
    xb = xt;
    wb = wt;
    cb = ct;
  }
  static constexpr int kOut = 1;
  __device__ void out(int j, P2 kx) {
    const F2 ra = f2(bb.a.u - kx.a.u, bb.a.v - kx.a.v), rb = f2(bb.b.u - kx.b.u, bb.b.v - kx.b.v);
    const int nx = V.g.nx;
    P2 z;
    z.a = dmask(c.i, nx, f2(xb.a.u + wb.x * ra.u + cb.x * (c.vb ? rb.u : 0.f), xb.a.v + wb.y * ra.v));
    z.b = dmask(c.i + 1, nx, f2(xb.b.u + wb.z * rb.u + cb.y * ra.u, xb.b.v + wb.w * rb.v));
    if (TOP) {
      if (c.oa) rz.add(bb.a.u * z.a.u + bb.a.v * z.a.v);
      if (c.ob) rz.add(bb.b.u * z.b.u + bb.b.v * z.b.v);
    }
    __syncwarp();
    put(0, z);
    __syncwarp();
    store(0, V.o0, j);
  }
  __device__ void finish(const SampleState& S) {
    if (TOP) {
      per_sample_wide(c, rz.value(), [&](int s, double t) {
        const int g = V.sbase + s;
        atomicAdd(&S.red_rz[g], t);
        if (last_tile(S.arrive, g, tiles_of_sample(V, s, kWideCols))) after_post(S, g);
      });
    }
  }
};

// PreR (coarse levels): b = P^T r1_f gathered from the finer level's residual (xc) by
// full weighting, kept for the post-smoothing (o1); x1 = W b, r1 = b - K x1 (o2).
// Coarse columns i, i + 1 of a lane take fine columns 2i - 1 .. 2i + 3 of fine rows
// 2j - 1, 2j, 2j + 1; each step stages fine rows 2j and 2j + 1 (fine virtual columns
// 2 vb - 1 .. 2 vb + 127, a fine virtual row having width 2 vw) and keeps row 2j + 1's
// sums for coarse row j + 1.
struct WPreR : WideBase {
  static constexpr int kDepth = 3;
  static constexpr int kMinBlocks = 4;
  struct Slot {
    float2 w[64];
    float c[64];
    float2 f[2][136];   // entry 4 + m: fine virtual column 2 vb + m; entry 3: 2 vb - 1
    float4 e[64];
  };
  bool act, have_prev = false;
  int nxf, nyf;
  int64_t fo[4], fl;   // load side: fine node index (row 0) of columns 2 vb + lane + 32 h, 2 vb - 1
  bool fv[4], flv;
  int64_t fA;          // compute side: fine node index (row 0) of column 2 i (clamped)
  P2 bt, bb, rp;
  __device__ WPreR(const View<float>& v, int s, int vb, const WCol& lc, const SampleState& S)
      : WideBase(v, s, vb, lc) {
    act = S.active[v.sbase + lc.s] != 0;
    nxf = 2 * v.g.nx;
    nyf = 2 * v.g.ny;
    const int64_t Nf = (int64_t)(nxf + 1) * (nyf + 1);
    auto fine = [&](int F, int64_t& idx, bool& valid) {
      int q, col;
      if (v.packed) {
        const int w2 = 2 * v.vw;
        const int qq = F >= 0 ? F / w2 : 0;
        col = F >= 0 ? F - qq * w2 : F;
        valid = F >= 0 && qq < v.nsamp && col <= nxf;
        q = min(qq, v.nsamp - 1);
      } else {
        q = s;
        col = F;
        valid = F >= 0 && F <= nxf;
      }
      idx = q * Nf + min(max(col, 0), nxf);
    };
#pragma unroll
    for (int h = 0; h < 4; ++h) fine(2 * vb + lane + 32 * h, fo[h], fv[h]);
    fine(2 * vb - 1, fl, flv);
    fA = lc.s * Nf + min(max(2 * lc.i, 0), nxf);
  }
  __device__ bool live() const { return act; }
  __device__ void fetch(Slot& S, int j) const {
    const int64_t r = jr(j);
    ld.node2(S.w, V.winvd, r, lane);
    ld.node1(S.c, V.wc, r, lane);
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const int jf = 2 * j + q;
      const bool row_in = jf <= nyf;
      const int64_t fr = (int64_t)min(jf, nyf) * (nxf + 1);
#pragma unroll
      for (int h = 0; h < 4; ++h) cp_async<8>(&S.f[q][4 + lane + 32 * h], V.xc + 2 * (fo[h] + fr), fv[h] && row_in);
      if (lane == 0) cp_async<8>(&S.f[q][3], V.xc + 2 * (fl + fr), flv && row_in);
    }
  }
  __device__ void fetchE(Slot& S, int e) const { ld.elem4(S.e, V.trig, er(e), lane); }
  __device__ ElemCoef coefs(const Invariants& U, const Slot& S) const { return coefs_coarse(U, S.e, lane, V.g.square); }
  // fine row sums (weights 1/2, 1, 1/2 over columns 2i - 1, 2i, 2i + 1) at the lane's
  // coarse columns, from staged fine row q
  __device__ P2 slot_sums(const Slot& S, int q) const {
    const float4 f01 = reinterpret_cast<const float4*>(S.f[q])[2 + 2 * lane];
    const float4 f23 = reinterpret_cast<const float4*>(S.f[q])[3 + 2 * lane];
    const float2 fm = S.f[q][3 + 4 * lane];
    P2 r;
    r.a = f2(f01.x + 0.5f * (f01.z + fm.x), f01.y + 0.5f * (f01.w + fm.y));
    r.b = f2(f23.x + 0.5f * (f23.z + f01.z), f23.y + 0.5f * (f23.w + f01.w));
    return r;
  }
  // the same sums of fine row jf read directly (the chunk's first coarse row)
  __device__ P2 direct_sums(int jf) const {
    F2 f[5];
    const bool row_in = jf >= 0 && jf <= nyf;
    const int i2 = 2 * min(max(c.i, 0), V.g.nx);
#pragma unroll
    for (int t = 0; t < 5; ++t) {
      const int col = i2 - 1 + t;
      f[t] = zf2();
      if (row_in && col >= 0 && col <= nxf) f[t] = get2(V.xc + 2 * (fA - i2 + col + (int64_t)jf * (nxf + 1)));
    }
    P2 r;
    r.a = f2(f[1].u + 0.5f * (f[2].u + f[0].u), f[1].v + 0.5f * (f[2].v + f[0].v));
    r.b = f2(f[3].u + 0.5f * (f[4].u + f[2].u), f[3].v + 0.5f * (f[4].v + f[2].v));
    return r;
  }
  __device__ P2 in(const Slot& S, int j) {
    const P2 rm = have_prev ? rp : direct_sums(2 * j - 1);
    const P2 r0 = slot_sums(S, 0), r1 = slot_sums(S, 1);
    rp = r1;
    have_prev = true;
    const int nx = V.g.nx;
    bt.a = dmask(c.i, nx, f2(r0.a.u + 0.5f * (rm.a.u + r1.a.u), r0.a.v + 0.5f * (rm.a.v + r1.a.v)));
    bt.b = dmask(c.i + 1, nx, f2(r0.b.u + 0.5f * (rm.b.u + r1.b.u), r0.b.v + 0.5f * (rm.b.v + r1.b.v)));
    const float4 w = lane4(S.w);
    const float2 cc = lane2(S.c);
    const float ua = c.va ? bt.a.u : 0.f, ub = c.vb ? bt.b.u : 0.f;
    P2 v;
    v.a = c.va ? f2(w.x * bt.a.u + cc.x * ub, w.y * bt.a.v) : zf2();
    v.b = c.vb ? f2(w.z * bt.b.u + cc.y * ua, w.w * bt.b.v) : zf2();
    return v;
  }
  __device__ void shift() { bb = bt; }
  static constexpr int kOut = 2;
  __device__ void out(int j, P2 kx) {
    const int nx = V.g.nx;
    P2 r1;
    r1.a = dmask(c.i, nx, f2(bb.a.u - kx.a.u, bb.a.v - kx.a.v));
    r1.b = dmask(c.i + 1, nx, f2(bb.b.u - kx.b.u, bb.b.v - kx.b.v));
    __syncwarp();
    put(0, bb);
    put(1, r1);
    __syncwarp();
    store(0, V.o1, j);
    store(1, V.o2, j);
  }
  __device__ void finish(const SampleState&) {}
};

template <typename Op>
__global__ void __launch_bounds__(kWarpsPerBlock * kWarp, Op::kMinBlocks)
    k_strip_wide(const __grid_constant__ ViewList<float> L, SampleState S) {
  const int gw = blockIdx.x * kWarpsPerBlock + (threadIdx.x >> 5);
  int vi, s, strip, chunk;
  if (!find_tile(L, gw, vi, s, strip, chunk)) return;
  const View<float>& V = L.v[vi];
  const int lane = (int)(threadIdx.x & 31);
  const int vb = strip * kWideCols - kWideHalo;
  WCol lc = wide_col(V, s, vb + 2 * lane);
  Op op(V, s, vb, lc, S);
  lc.live = op.live();
  if (!__any_sync(0xffffffffu, lc.va && lc.live)) return;
  const bool out_lane = lane >= 1 && lane <= 30;
  lc.oa = lc.va && lc.live && out_lane;
  lc.ob = lc.vb && lc.live && out_lane;
  if (S.units) {
    const int n = __popc(__ballot_sync(0xffffffffu, lc.oa)) + __popc(__ballot_sync(0xffffffffu, lc.ob));
    if (lane == 0 && n) {
      const int rows = V.rows > 0 ? V.rows : kRowChunk;
      const int r0 = chunk * rows, r1 = min(r0 + rows - 1, V.g.ny);
      atomicAdd(&S.units[L.prof_op], (unsigned long long)(n * (r1 - r0 + 1)));
    }
  }
  extern __shared__ __align__(16) unsigned char wide_smem[];
  typename Op::Slot* ring = reinterpret_cast<typename Op::Slot*>(wide_smem) + (threadIdx.x >> 5) * Op::kDepth;
  float4* stage = reinterpret_cast<float4*>(wide_smem + sizeof(typename Op::Slot) * Op::kDepth * kWarpsPerBlock) +
                  (threadIdx.x >> 5) * Op::kOut * 32;
  op.set_outputs(stage);
  wide_loop<Op::kDepth>(L.U, V, lc, chunk, op, ring);
  op.finish(S);
}

template <typename Op>
cudaError_t launch_wide_op(const ViewList<float>& L, SampleState S, int total_warps, cudaStream_t st) {
  if (total_warps <= 0) return cudaSuccess;
  const int blocks = (total_warps + kWarpsPerBlock - 1) / kWarpsPerBlock;
  const size_t smem = (sizeof(typename Op::Slot) * Op::kDepth + sizeof(float4) * 32 * Op::kOut) * kWarpsPerBlock;
  static_assert(sizeof(typename Op::Slot) % 16 == 0, "slots must keep 16-byte alignment");
  if (smem > 48 * 1024) {
    const cudaError_t e = cudaFuncSetAttribute(k_strip_wide<Op>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
  }
  k_strip_wide<Op><<<blocks, kWarpsPerBlock * kWarp, smem, st>>>(L, S);
  return cudaGetLastError();
}

}  // namespace

int wide_strip_bit(StripOp op) {
  switch (op) {
    case StripOp::PreTop: return 0;
    case StripOp::PreR: return 1;
    case StripOp::Post: return 2;
    case StripOp::PostTop: return 3;
    case StripOp::PcgP: return 4;
    default: return -1;
  }
}

cudaError_t launch_strip_wide(StripOp op, const ViewList<float>& L, SampleState S, int total_warps, cudaStream_t st) {
  switch (op) {
    case StripOp::PreTop: return launch_wide_op<WPreTop>(L, S, total_warps, st);
    case StripOp::PreR: return launch_wide_op<WPreR>(L, S, total_warps, st);
    case StripOp::Post: return launch_wide_op<WPost<false>>(L, S, total_warps, st);
    case StripOp::PostTop: return launch_wide_op<WPost<true>>(L, S, total_warps, st);
    case StripOp::PcgP: return launch_wide_op<WPcgP>(L, S, total_warps, st);
    default: break;
  }
  return cudaErrorInvalidValue;
}

}  // namespace mlmc
