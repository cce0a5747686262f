// Batched geometric-multigrid-preconditioned CG with double-precision iterative
// refinement, for many independent samples on several meshes at once.
//
// Outer loop (double): d starts as the lifting of the Dirichlet data; r = f - K d
// is evaluated in double (f = 0 in the interior, the load comes from the lifting);
// when ||r|| <= rtol ||f|| the sample is done, otherwise the correction system
// K e = r is solved in the inner precision T and d += e.
// Inner loop (T): preconditioned CG, preconditioner one symmetric V(1,1)-cycle:
// damped Jacobi smoothing (w = 1/2), full weighting restriction = P^T, bilinear
// prolongation P, coarse operators rediscretised from the child-averaged rotated
// stiffness, and an exact dense solve on the coarsest mesh.
//
// All groups (one mesh size each, any number of samples) advance in lock step:
// multigrid levels are aligned by their depth below each group's finest mesh, so one
// launch per depth serves every group that has that level. Every sample keeps its
// own CG scalars; converged samples drop out of all kernels.
#include <algorithm>
#include <type_traits>
#include <cstdio>
#include <cstdlib>
#include <cmath>
#include <cstring>

#include "context.h"

namespace mlmc {

// Launches EXPR (a cudaError_t expression) as timer operation OP, returning on error.
#define MLMC_LAUNCH(OP, NAME, EXPR)                      \
  do {                                                   \
    ctx.timer.begin((OP), st, (NAME));                   \
    const cudaError_t launch_err_ = (EXPR);              \
    ctx.timer.end(st);                                   \
    if (launch_err_ != cudaSuccess) return ctx.cuda_fail(launch_err_, (NAME)); \
  } while (0)

namespace {

template <typename T>
struct GroupBuf {
  const SolveGroup<T>* grp;
  int sbase;
  int nl;                     // multigrid levels, 0 = top
  std::vector<Geo> geo;
  // top level
  T *x, *r[2], *p[2], *z, *q;
  double* d;
  // every level k: winvd[k], wc[k] (smoother), r1[k]; coarse levels k >= 1: b[k], xl[k], trig[k]
  std::vector<T*> winvd, wc, r1, b, xl, trig;
  T* ainv;
};

template <typename T>
View<T> base_view(const GroupBuf<T>& g, int k) {
  View<T> v;
  std::memset(&v, 0, sizeof(v));
  v.g = g.geo[k];
  v.nsamp = (int)g.grp->nsamp;
  v.sbase = g.sbase;
  v.tiles_x = strips_of(v.g.nx);
  v.tiles_y = chunks_of(v.g.ny);
  if (k == 0) {
    v.trig2 = g.grp->trig2;
  } else {
    v.trig = g.trig[k];
  }
  return v;
}

// Assigns the strips of operation op, the row chunks and the work offsets of a strip
// kernel (warps); returns the total. A mesh's node rows are cut into chunks of equal
// height, at most ctx.max_rows (each chunk costs one extra element row and a pipeline
// fill). A warp walks its rows one after another, so a launch of fewer warps than
// ctx.target_waves waves (152 SMs x 28 resident warps each, 16 for the node-pair
// kernels) is bound by that walk: its views are cut into 2, 4 or 8 times as many chunks
// (at least ctx.min_rows rows each), which shortens every warp's walk. mlmc_autotune
// picks the three parameters.
// Where ctx.wide_strips has op's bit the FP32 kernel holds a node pair per lane
// (launch_strip_wide: 60 output columns per strip, views packed at any sample width);
// that needs an even nx on every view, which every level above a hierarchy's coarsest has.
template <typename T>
int finalize_warps(const Context& ctx, ViewList<T>& L, StripOp op) {
  const int bit = wide_strip_bit(op);
  bool wide = std::is_same<T, float>::value && bit >= 0 && ((ctx.wide_strips >> bit) & 1);
  for (int i = 0; i < L.n && wide; ++i) wide = L.v[i].g.nx % 2 == 0;
  L.wide = wide ? 1 : 0;
  // resident warps per SM: 28 of the one-column kernels, 16 of the node-pair kernels
  const int target_warps = (int)(152 * (wide ? 16 : 28) * ctx.target_waves);
  const int min_rows = std::max(1, ctx.min_rows);
  const int max_rows = std::min(64, std::max(min_rows, ctx.max_rows));
  auto layout = [&](int split) {
    int acc = 0;
    for (int i = 0; i < L.n; ++i) {
      View<T>& v = L.v[i];
      const int nodes_y = v.g.ny + 1;
      const int base = chunks_of(v.g.ny, max_rows);
      const int nch = std::max(base, std::min(base * split, nodes_y / min_rows));
      v.rows = (nodes_y + nch - 1) / nch;
      v.tiles_y = chunks_of(v.g.ny, v.rows);
      // samples side by side when a sample's width fills at least one strip (then a
      // warp's outputs span at most two samples)
      const int cols = wide ? kWideCols : strip_cols(op);
      v.vw = v.g.nx + 2;
      v.packed = ctx.pack_samples && (wide || v.vw >= cols) ? 1 : 0;
      if (v.packed) {
        v.tiles_x = (int)(((int64_t)v.nsamp * v.vw + cols - 1) / cols);
        v.nwork = v.tiles_x * v.tiles_y;
      } else {
        v.tiles_x = strips_of(v.g.nx, cols);
        v.nwork = v.nsamp * v.tiles_x * v.tiles_y;
      }
      v.work_begin = acc;
      acc += v.nwork;
    }
    return acc;
  };
  int split = 1, acc = layout(1);
  while (acc < target_warps && split < 8) acc = layout(split *= 2);
  return acc;
}

// A strip launch laid out by finalize_warps: the node-pair kernels when it chose them.
template <typename T>
cudaError_t strip_dispatch(StripOp op, const ViewList<T>& L, SampleState S, int total_warps, cudaStream_t st) {
  if constexpr (std::is_same<T, float>::value) {
    if (L.wide) return launch_strip_wide(op, L, S, total_warps, st);
  }
  return launch_strip<T>(op, L, S, total_warps, st);
}

template <typename T>
int finalize_points(ViewList<T>& L, const std::vector<int64_t>& per_sample) {
  int64_t acc = 0;
  for (int i = 0; i < L.n; ++i) {
    L.v[i].work_begin = (int)acc;
    L.v[i].nwork = (int)(L.v[i].nsamp * per_sample[i]);
    acc += L.v[i].nwork;
  }
  return (int)acc;
}

struct SizeAlloc {
  Sizer s;
  template <typename U>
  void vec(U*&, size_t n) { s.add<U>(n); }
};

struct CarveAlloc {
  Arena* a;
  template <typename U>
  void vec(U*& p, size_t n) { p = a->carve<U>(n); }
};

template <typename T>
ViewList<T> empty_list(const Context& ctx) {
  ViewList<T> L;
  std::memset(&L, 0, sizeof(L));
  L.n = 0;
  L.U = ctx.U;
  return L;
}

}  // namespace

namespace {

// Condition of the device-side batch loop: one more replay while samples are active and
// fewer than max_reps replays have run.
__global__ void k_loop_condition(cudaGraphConditionalHandle h, const int* __restrict__ count, int* reps,
                                 int max_reps) {
  const int r = ++(*reps);
  cudaGraphSetConditional(h, (*count > 0 && r < max_reps) ? 1u : 0u);
}

cudaError_t launch_loop_condition(cudaGraphConditionalHandle h, const int* count, int* reps, int max_reps,
                                  cudaStream_t st) {
  k_loop_condition<<<1, 1, 0, st>>>(h, count, reps, max_reps);
  return cudaGetLastError();
}

}  // namespace

// One solve of every group at the context's smoother damping; *failed (nullable) is
// set when some sample ends without converging.
template <typename T>
mlmc_status solve_groups_once(Context& ctx, std::vector<SolveGroup<T>>& groups, bool* failed) {
  cudaStream_t st = ctx.stream;
  const bool inner_double = sizeof(T) == sizeof(double);
  if (groups.empty()) return MLMC_OK;
  if ((int)groups.size() > kMaxViews) return ctx.fail(MLMC_ERR_INVALID_ARG, "too many mesh groups in one solve");

  // ---- hierarchy and workspace
  std::vector<GroupBuf<T>> G(groups.size());
  int total = 0;
  int dmax = 0;   // deepest coarsest-level index over the groups
  for (size_t gi = 0; gi < groups.size(); ++gi) {
    GroupBuf<T>& g = G[gi];
    g.grp = &groups[gi];
    g.sbase = total;
    total += (int)groups[gi].nsamp;
    const LevelLayout m = ctx.mesh(groups[gi].mesh_level);
    int nx = m.nx, ny = m.ny;
    g.geo.push_back(ctx.geo(nx, ny));
    // halve as far as the grid allows; the coarsest mesh is solved densely
    while (nx % 2 == 0 && ny % 2 == 0 && ny >= 2) {
      nx /= 2;
      ny /= 2;
      g.geo.push_back(ctx.geo(nx, ny));
    }
    g.nl = (int)g.geo.size();
    if (g.nl < 2) return ctx.fail(MLMC_ERR_INVALID_ARG, "mesh too small for the multigrid hierarchy");
    const Geo& c = g.geo.back();
    if (2 * (c.nx + 1) * (c.ny + 1) > kMaxCoarsestDofs)
      return ctx.fail(MLMC_ERR_INVALID_ARG, "coarsest mesh too large (mesh must halve down to <= 64 DOFs)");
    dmax = std::max(dmax, g.nl - 1);
  }
  if (total == 0) return MLMC_OK;
  // the multigrid bottom of every group in one launch (FP32, hierarchies of 4 levels or
  // more whose three smallest meshes fit a warp's shared memory): the sweeps then stop
  // three levels above each group's coarsest
  // or, one block per sample, the three smoothed levels above each group's coarsest and
  // the coarsest solve (hierarchies of 5 levels or more, small enough bottoms)
  const int bottom_mode = std::is_same<T, float>::value ? ctx.fused_bottom : 0;
  bool deep = bottom_mode == 2;
  for (auto& g : G)
    deep = deep && g.nl >= 5 && deep_fits(&g.geo[g.nl - 4], 3, g.geo[g.nl - 1]);
  bool fused = !deep && bottom_mode >= 1;
  for (auto& g : G)
    fused = fused && g.nl >= 4 && bottom_fits(g.geo[g.nl - 3], g.geo[g.nl - 2], g.geo[g.nl - 1]);
  const int bottom_depth = deep ? 4 : fused ? 3 : 1;
  const int max_iter = ctx.cfg.max_iter > 0 ? ctx.cfg.max_iter : 200;
  const int max_outer = ctx.cfg.max_outer > 0 ? ctx.cfg.max_outer : 8;

  auto plan = [&](auto& alloc) {
    for (auto& g : G) {
      const int64_t ns = g.grp->nsamp;
      auto nv = [&](int k) { return (size_t)(ns * 2 * (int64_t)(g.geo[k].nx + 1) * (g.geo[k].ny + 1)); };
      alloc.template vec<T>(g.x, nv(0));
      alloc.template vec<T>(g.r[0], nv(0));
      alloc.template vec<T>(g.r[1], nv(0));
      alloc.template vec<T>(g.p[0], nv(0));
      alloc.template vec<T>(g.p[1], nv(0));
      alloc.template vec<T>(g.z, nv(0));
      alloc.template vec<T>(g.q, nv(0));
      alloc.template vec<double>(g.d, nv(0));
      g.winvd.assign(g.nl, nullptr);
      g.wc.assign(g.nl, nullptr);
      g.r1.assign(g.nl, nullptr);
      g.b.assign(g.nl, nullptr);
      g.xl.assign(g.nl, nullptr);
      g.trig.assign(g.nl, nullptr);
      for (int k = 0; k < g.nl; ++k) {
        alloc.template vec<T>(g.winvd[k], nv(k));
        alloc.template vec<T>(g.wc[k], nv(k) / 2);
        alloc.template vec<T>(g.r1[k], nv(k));
        if (k >= 1) {
          alloc.template vec<T>(g.b[k], nv(k));
          alloc.template vec<T>(g.xl[k], nv(k));
          alloc.template vec<T>(g.trig[k], (size_t)(ns * 4 * (int64_t)g.geo[k].nx * g.geo[k].ny));
        }
      }
      const int nc = 2 * (g.geo.back().nx + 1) * (g.geo.back().ny + 1);
      alloc.template vec<T>(g.ainv, (size_t)(ns * nc * nc));
    }
  };
  SampleState S;
  int* outer_count = nullptr;
  auto plan_state = [&](auto& alloc) {
    alloc.template vec<double>(S.alpha, total);
    alloc.template vec<double>(S.beta, total);
    alloc.template vec<double>(S.rz_old, total);
    alloc.template vec<double>(S.rr_ref, total);
    alloc.template vec<double>(S.tol2, total);
    alloc.template vec<double>(S.red_rr, total);
    alloc.template vec<double>(S.red_rz, total);
    alloc.template vec<double>(S.red_pq, total);
    alloc.template vec<double>(S.rrf, total);
    alloc.template vec<double>(S.rr64, total);
    alloc.template vec<double>(S.react, total);
    alloc.template vec<double>(S.qoi, 2 * (size_t)total);
    alloc.template vec<int>(S.active, total);
    alloc.template vec<int>(S.outer_active, total);
    alloc.template vec<int>(S.iters, total);
    alloc.template vec<int>(S.status, total);
    alloc.template vec<int>(S.count, (size_t)std::max(ctx.check_every, 1));
    alloc.template vec<int>(S.rpar, total);
    alloc.template vec<int>(S.exact, total);
    alloc.template vec<unsigned>(S.arrive, total);
    alloc.template vec<int>(outer_count, 2);   // [0] refinement count, [1] device-loop replays
  };
  SizeAlloc sz;
  plan(sz);
  plan_state(sz);
  cudaError_t e = ctx.solve_arena.reserve(sz.s.used + 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return ctx.fail(MLMC_ERR_OOM, "solver workspace allocation failed");
  }
  ctx.solve_arena.reset();
  CarveAlloc ca{&ctx.solve_arena};
  plan(ca);
  plan_state(ca);
  S.units = ctx.timer.on ? ctx.timer.units_dev : nullptr;
  S.slot = 0;
  {
    char* state_begin = reinterpret_cast<char*>(S.alpha);
    char* state_end = reinterpret_cast<char*>(outer_count + 2);
    if ((e = cudaMemsetAsync(state_begin, 0, (size_t)(state_end - state_begin), st)) != cudaSuccess)
      return ctx.cuda_fail(e, "memset");
  }

  // ---- per-level element data, diagonal and coarsest inverse
  for (int k = 0; k + 1 < 64; ++k) {
    ViewList<T> L = empty_list<T>(ctx);
    std::vector<int64_t> per;
    for (auto& g : G) {
      if (k + 1 >= g.nl) continue;
      View<T> v = base_view(g, k);
      v.o0 = g.trig[k + 1];
      L.v[L.n++] = v;
      per.push_back((int64_t)(g.geo[k].nx / 2) * (g.geo[k].ny / 2));
    }
    if (L.n == 0) break;
    const int tt = finalize_points(L, per);
    MLMC_LAUNCH(kProfOther, "trig_average", launch_trig_average<T>(L, tt, st));
  }
  // smoothers of every level of every group: independent, so up to kMaxViews
  // (group, level) views share a launch
  {
    ViewList<T> L = empty_list<T>(ctx);
    std::vector<int64_t> per;
    auto flush = [&]() -> mlmc_status {
      if (L.n == 0) return MLMC_OK;
      const int tt = finalize_points(L, per);
      MLMC_LAUNCH(kProfOther, "invdiag", launch_invdiag<T>(L, tt, st));
      L = empty_list<T>(ctx);
      per.clear();
      return MLMC_OK;
    };
    for (auto& g : G)
      for (int k = 0; k < g.nl; ++k) {
        if (L.n == kMaxViews) {
          const mlmc_status fs = flush();
          if (fs != MLMC_OK) return fs;
        }
        View<T> v = base_view(g, k);
        v.o0 = g.winvd[k];
        v.o1 = g.wc[k];
        v.param = ctx.omega;
        L.v[L.n++] = v;
        per.push_back((int64_t)(g.geo[k].nx / 2 + 1) * (g.geo[k].ny + 1));   // node pairs
      }
    const mlmc_status fs = flush();
    if (fs != MLMC_OK) return fs;
  }
  {
    ViewList<T> L = empty_list<T>(ctx);
    int acc = 0;
    for (auto& g : G) {
      View<T> v = base_view(g, g.nl - 1);
      v.o0 = g.ainv;
      v.work_begin = acc;
      v.nwork = v.nsamp;
      acc += v.nwork;
      L.v[L.n++] = v;
    }
    MLMC_LAUNCH(kProfOther, "coarsest_setup", launch_coarsest_setup<T>(L, acc, st));
  }

  // ---- view lists reused every iteration
  // top-level views (PreTop / PostTop / PcgP and the refinement residual)
  auto top_list = [&](StripOp op, int parity) {
    ViewList<T> L = empty_list<T>(ctx);
    for (auto& g : G) {
      View<T> v = base_view(g, 0);
      switch (op) {
        case StripOp::PreTop:
          v.a = g.r[parity];
          v.b = g.q;
          v.c = g.p[parity];
          v.winvd = g.winvd[0];
          v.wc = g.wc[0];
          v.o0 = g.x;
          v.o1 = g.r[parity ^ 1];
          v.o2 = g.r1[0];
          break;
        case StripOp::PostTop:
          v.a = g.r[parity ^ 1];
          v.xc = g.xl[1];
          v.winvd = g.winvd[0];
          v.wc = g.wc[0];
          v.o0 = g.z;
          break;
        case StripOp::PcgP:
          v.a = g.z;
          v.b = g.p[parity];
          v.o0 = g.p[parity ^ 1];
          v.o1 = g.q;
          break;
        default:
          break;
      }
      L.v[L.n++] = v;
    }
    return L;
  };

  // One PCG iteration for every group. Multigrid levels are aligned by depth below
  // each group's finest mesh, so the finest-level kernels (the largest) are single
  // launches over all groups; a group's coarse levels join the launches of their depth,
  // and all coarsest solves share one launch between the down and up sweeps.
  auto run_vcycle_and_pcg = [&](int parity, int slot) -> mlmc_status {
    // down sweep: depth d gathers its right-hand side from depth d - 1 (full weighting),
    // smooths and forms its residual; depth 0 updates the PCG iterate first
    for (int d = 0; d < dmax; ++d) {
      ViewList<T> Lsm = empty_list<T>(ctx);
      for (auto& g : G) {
        if (d >= g.nl - bottom_depth) continue;
        View<T> v = base_view(g, d);
        if (d == 0) {
          v.a = g.r[parity];
          v.b = g.q;
          v.c = g.p[parity];
          v.winvd = g.winvd[0];
          v.wc = g.wc[0];
          v.o0 = g.x;
          v.o1 = g.r[parity ^ 1];
          v.o2 = g.r1[0];
        } else {
          v.xc = g.r1[d - 1];
          v.o1 = g.b[d];
          v.winvd = g.winvd[d];
          v.wc = g.wc[d];
          v.o2 = g.r1[d];
        }
        Lsm.v[Lsm.n++] = v;
      }
      if (!Lsm.n) continue;
      const int tw = finalize_warps(ctx, Lsm, d == 0 ? StripOp::PreTop : StripOp::PreR);
      if (d == 0) {
        Lsm.prof_op = kProfPreTop;
        MLMC_LAUNCH(kProfPreTop, "pre_top", strip_dispatch<T>(StripOp::PreTop, Lsm, S, tw, st));
      } else {
        Lsm.prof_op = kProfPre;
        MLMC_LAUNCH(kProfPre, "pre", strip_dispatch<T>(StripOp::PreR, Lsm, S, tw, st));
      }
    }
    // every group's bottom: levels nl-4 .. nl-2 and the coarsest in one launch (a block
    // per sample), levels nl-3, nl-2 and the coarsest in one launch (a warp per
    // sample), or the coarsest mesh alone (its right-hand side gathered from the level
    // above)
    if (deep) {
      DeepList L;
      std::memset(&L, 0, sizeof(L));
      L.U = ctx.U;
      int acc = 0, floats = 0;
      for (auto& g : G) {
        const int a = g.nl - 4;
        DeepView v;
        std::memset(&v, 0, sizeof(v));
        v.nb = 3;
        for (int k = 0; k < 3; ++k) {
          v.g[k] = g.geo[a + k];
          v.winv[k] = reinterpret_cast<const float*>(g.winvd[a + k]);
          v.wc[k] = reinterpret_cast<const float*>(g.wc[a + k]);
          v.trig[k] = reinterpret_cast<const float*>(g.trig[a + k]);
        }
        v.gc = g.geo[g.nl - 1];
        v.nsamp = (int)g.grp->nsamp;
        v.sbase = g.sbase;
        v.work_begin = acc;
        v.rin = reinterpret_cast<const float*>(g.r1[a - 1]);
        v.ainv = reinterpret_cast<const float*>(g.ainv);
        v.xout = reinterpret_cast<float*>(g.xl[a]);
        acc += v.nsamp;
        floats = std::max(floats, deep_floats(v.g, v.nb, v.gc));
        L.v[L.n++] = v;
      }
      MLMC_LAUNCH(kProfCoarsest, "bottom_deep", launch_bottom_deep(L, S, acc, floats, st));
    } else if (fused) {
      BottomList L;
      std::memset(&L, 0, sizeof(L));
      L.U = ctx.U;
      int acc = 0;
      for (auto& g : G) {
        const int a = g.nl - 3;
        BottomView v;
        std::memset(&v, 0, sizeof(v));
        v.ga = g.geo[a];
        v.gb = g.geo[a + 1];
        v.gc = g.geo[a + 2];
        v.nsamp = (int)g.grp->nsamp;
        v.sbase = g.sbase;
        v.work_begin = acc;
        v.rin = reinterpret_cast<const float*>(g.r1[a - 1]);
        v.winv_a = reinterpret_cast<const float*>(g.winvd[a]);
        v.wc_a = reinterpret_cast<const float*>(g.wc[a]);
        v.trig_a = reinterpret_cast<const float*>(g.trig[a]);
        v.winv_b = reinterpret_cast<const float*>(g.winvd[a + 1]);
        v.wc_b = reinterpret_cast<const float*>(g.wc[a + 1]);
        v.trig_b = reinterpret_cast<const float*>(g.trig[a + 1]);
        v.ainv = reinterpret_cast<const float*>(g.ainv);
        v.xout = reinterpret_cast<float*>(g.xl[a]);
        acc += v.nsamp;
        L.v[L.n++] = v;
      }
      MLMC_LAUNCH(kProfCoarsest, "bottom", launch_bottom(L, S, acc, st));
    } else {
      ViewList<T> L = empty_list<T>(ctx);
      int acc = 0;
      for (auto& g : G) {
        const int k = g.nl - 1;
        View<T> v = base_view(g, k);
        v.xc = g.r1[k - 1];
        v.o0 = g.xl[k];
        v.ext0 = g.ainv;
        v.work_begin = acc;
        v.nwork = v.nsamp;
        acc += v.nwork;
        L.v[L.n++] = v;
      }
      MLMC_LAUNCH(kProfCoarsest, "coarsest", launch_coarsest_solve<T>(L, S, acc, st));
    }
    // up sweep: prolongation and post-smoothing from the deepest level back to the top
    for (int d = dmax - 1; d >= 0; --d) {
      ViewList<T> L = empty_list<T>(ctx);
      for (auto& g : G) {
        if (d >= g.nl - bottom_depth) continue;
        View<T> v = base_view(g, d);
        v.xc = g.xl[d + 1];
        v.winvd = g.winvd[d];
        v.wc = g.wc[d];
        if (d == 0) {
          v.a = g.r[parity ^ 1];
          v.o0 = g.z;
        } else {
          v.a = g.b[d];
          v.o0 = g.xl[d];
        }
        L.v[L.n++] = v;
      }
      if (!L.n) continue;
      const int tw = finalize_warps(ctx, L, d == 0 ? StripOp::PostTop : StripOp::Post);
      if (d == 0) {   // its last warp per sample also takes the convergence test and beta
        L.prof_op = kProfPostTop;
        SampleState Ss = S;
        Ss.slot = slot;
        MLMC_LAUNCH(kProfPostTop, "post_top", strip_dispatch<T>(StripOp::PostTop, L, Ss, tw, st));
      } else {
        L.prof_op = kProfPost;
        MLMC_LAUNCH(kProfPost, "post", strip_dispatch<T>(StripOp::Post, L, S, tw, st));
      }
    }
    {   // its last warp per sample also forms alpha
      ViewList<T> L = top_list(StripOp::PcgP, parity);
      const int tw = finalize_warps(ctx, L, StripOp::PcgP);
      L.prof_op = kProfPcgP;
      MLMC_LAUNCH(kProfPcgP, "pcg_p", strip_dispatch<T>(StripOp::PcgP, L, S, tw, st));
    }
    return MLMC_OK;
  };

  // double-precision views for lifting, residual and stress
  // groups whose next refinement residual is formed exactly from d: those that start
  // from the lifting, after their first correction; those with initial iterates (nested
  // iteration) at the start. Each group keeps its own sequence, so a sample's solve does
  // not depend on the other groups of its batch.
  std::vector<char> exact(G.size());
  for (size_t gi = 0; gi < G.size(); ++gi) exact[gi] = G[gi].grp->d_guess == nullptr;
  auto d_list = [&](int want_exact = -1) {
    ViewList<double> L;
    std::memset(&L, 0, sizeof(L));
    L.U = ctx.U;
    for (size_t gi = 0; gi < G.size(); ++gi) {
      if (want_exact >= 0 && exact[gi] != want_exact) continue;
      auto& g = G[gi];
      View<double> v;
      std::memset(&v, 0, sizeof(v));
      v.g = g.geo[0];
      v.nsamp = (int)g.grp->nsamp;
      v.sbase = g.sbase;
      v.tiles_x = strips_of(v.g.nx);
      v.tiles_y = chunks_of(v.g.ny);
      v.a = g.d;
      v.o0 = g.d;
      v.ext0 = g.grp->trig2;
      v.ext1 = g.r[0];
      L.v[L.n++] = v;
    }
    return L;
  };
  auto resid = [&]() -> mlmc_status {   // the groups marked exact
    ViewList<double> L = d_list(1);
    if (L.n == 0) return MLMC_OK;
    int acc = 0;
    for (int i = 0; i < L.n; ++i) {
      L.v[i].work_begin = acc;
      L.v[i].nwork = L.v[i].nsamp * L.v[i].tiles_x * L.v[i].tiles_y;
      acc += L.v[i].nwork;
    }
    L.prof_op = kProfResid;
    MLMC_LAUNCH(kProfResid, "resid64", launch_resid64<T>(L, S, acc, st));
    return MLMC_OK;
  };

  {
    std::vector<int> ones(total, 1);
    if ((e = cudaMemcpyAsync(S.outer_active, ones.data(), sizeof(int) * total, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return ctx.cuda_fail(e, "init");
    if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return ctx.cuda_fail(e, "init");
  }
  // lifting d0 and its residual ||f||, in the inner precision (the first refinement
  // residual, after the first correction, supersedes it): both vectors are zero except
  // near x = lx
  {
    ViewList<T> L = empty_list<T>(ctx);
    std::vector<int64_t> per;
    for (auto& g : G) {
      const size_t nv = (size_t)g.grp->nsamp * 2 * (g.geo[0].nx + 1) * (g.geo[0].ny + 1);
      if ((e = cudaMemsetAsync(g.d, 0, sizeof(double) * nv, st)) != cudaSuccess ||
          (e = cudaMemsetAsync(g.r[0], 0, sizeof(T) * nv, st)) != cudaSuccess)
        return ctx.cuda_fail(e, "memset");
      View<T> v = base_view(g, 0);
      v.o0 = g.r[0];
      v.ext1 = g.d;
      L.v[L.n++] = v;
      per.push_back(2 * (int64_t)(g.geo[0].ny + 1));
    }
    const int tt = finalize_points(L, per);
    MLMC_LAUNCH(kProfOther, "lift_resid", launch_lift_resid<T>(L, S, ctx.cfg.shortening, tt, st));
  }
  mlmc_status rs = MLMC_OK;
  MLMC_LAUNCH(kProfOther, "outer_init", launch_outer_init(S, total, st));

  // nested iteration: start from the same samples' solutions on the next coarser mesh
  // (the lifting above still defines ||f||); their residual is formed exactly, and the
  // corrections that follow are small, so every later residual is the inner CG's
  // recursive one
  // nested iteration: groups with initial iterates start from the same samples'
  // solutions on the next coarser mesh (the lifting above still defines ||f||); their
  // residual is formed exactly, and the corrections that follow are small, so every
  // later residual is the inner CG's recursive one
  {
    ViewList<T> L = empty_list<T>(ctx);
    std::vector<int64_t> per;
    for (size_t gi = 0; gi < G.size(); ++gi) {
      auto& g = G[gi];
      if (!g.grp->d_guess) continue;
      View<T> v = base_view(g, 0);
      v.ext0 = g.grp->d_guess;
      v.ext1 = g.d;
      L.v[L.n++] = v;
      per.push_back((int64_t)(g.geo[0].nx + 1) * (g.geo[0].ny + 1));
      if ((e = cudaMemsetAsync(S.rr64 + g.sbase, 0, sizeof(double) * g.grp->nsamp, st)) != cudaSuccess ||
          (e = cudaMemsetAsync(S.react + g.sbase, 0, sizeof(double) * g.grp->nsamp, st)) != cudaSuccess)
        return ctx.cuda_fail(e, "memset");
    }
    if (L.n > 0) {
      const int tt = finalize_points(L, per);
      MLMC_LAUNCH(kProfOther, "prolong_d", launch_prolong_d<T>(L, tt, st));
      for (size_t gi = 0; gi < G.size(); ++gi) exact[gi] = G[gi].grp->d_guess != nullptr;
      rs = resid();
      if (rs != MLMC_OK) return rs;
    }
    // from here on: exact marks the groups whose residual after the next correction is
    // formed from d (those that started from the lifting)
    std::vector<int> ex(total, 0);
    for (size_t gi = 0; gi < G.size(); ++gi) {
      exact[gi] = G[gi].grp->d_guess == nullptr;
      for (int64_t k = 0; k < G[gi].grp->nsamp; ++k) ex[G[gi].sbase + k] = exact[gi];
    }
    // (from pageable memory: the call returns once ex has been staged)
    if ((e = cudaMemcpyAsync(S.exact, ex.data(), sizeof(int) * total, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return ctx.cuda_fail(e, "init");
  }

  // PCG iterations run in batches of check_every (even) between host convergence
  // checks. A full batch is captured once per solve into a CUDA graph and replayed: its
  // launches depend on the iteration only through the parity of the residual buffers
  // and the slot of the active-sample counter, both fixed within a batch that starts
  // at an even iteration. The kernel timer, which records events around each launch,
  // runs the same launches directly, and so does the legacy default stream, which
  // cannot be captured.
  cudaGraphExec_t batch_graph = nullptr;
  struct GraphGuard {
    cudaGraphExec_t* g;
    ~GraphGuard() {
      if (*g) cudaGraphExecDestroy(*g);
    }
  } graph_guard{&batch_graph};
  int64_t graph_launches = 0;
  const bool capturable = st != nullptr && st != cudaStreamLegacy && st != cudaStreamPerThread;
  const bool graphs = ctx.graphs && capturable && !ctx.timer.on && ctx.check_every % 2 == 0;
  auto capture_batch = [&]() -> mlmc_status {
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (ce != cudaSuccess) return ctx.cuda_fail(ce, "graph capture");
    const int64_t l0 = ctx.timer.launches;
    mlmc_status cs = MLMC_OK;
    ce = cudaMemsetAsync(S.count, 0, sizeof(int) * ctx.check_every, st);
    for (int b = 0; b < ctx.check_every && cs == MLMC_OK && ce == cudaSuccess; ++b) cs = run_vcycle_and_pcg(b & 1, b);
    const cudaError_t ee = cudaStreamEndCapture(st, &g);
    if (cs != MLMC_OK || ce != cudaSuccess || ee != cudaSuccess) {
      if (g) cudaGraphDestroy(g);
      cudaGetLastError();
      return cs != MLMC_OK ? cs : ctx.cuda_fail(ce != cudaSuccess ? ce : ee, "graph capture");
    }
    graph_launches = ctx.timer.launches - l0;
    ctx.timer.launches = l0;   // counted again at every replay
    ce = cudaGraphInstantiate(&batch_graph, g, 0);
    cudaGraphDestroy(g);
    if (ce != cudaSuccess) {
      batch_graph = nullptr;
      return ctx.cuda_fail(ce, "graph instantiate");
    }
    return MLMC_OK;
  };

  // The replays of the batch and the convergence test run on the device: a conditional
  // WHILE node repeats the batch while samples are active, at most max_iter / check_every
  // times (its condition kernel counts the replays), so an inner solve is one graph
  // launch and one host read instead of a host round trip per batch. A remainder of
  // fewer than check_every iterations, or a capped solve, continues in the loop below.
  cudaGraphExec_t loop_graph = nullptr;
  GraphGuard loop_guard{&loop_graph};
  int64_t loop_launches = 0;
  const int loop_reps = ctx.check_every > 0 ? max_iter / ctx.check_every : 0;
  auto build_loop = [&]() -> mlmc_status {
    cudaGraph_t g = nullptr;
    cudaError_t ce = cudaGraphCreate(&g, 0);
    if (ce != cudaSuccess) return ctx.cuda_fail(ce, "loop graph");
    struct Destroy {
      cudaGraph_t* g;
      ~Destroy() {
        if (*g) cudaGraphDestroy(*g);
      }
    } destroy{&g};
    cudaGraphConditionalHandle h;
    if ((ce = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault)) != cudaSuccess)
      return ctx.cuda_fail(ce, "loop graph");
    cudaGraphNodeParams cp = {};
    cp.type = cudaGraphNodeTypeConditional;
    cp.conditional.handle = h;
    cp.conditional.type = cudaGraphCondTypeWhile;
    cp.conditional.size = 1;
    cudaGraphNode_t cn;
    if ((ce = cudaGraphAddNode(&cn, g, nullptr, nullptr, 0, &cp)) != cudaSuccess) return ctx.cuda_fail(ce, "loop graph");
    cudaGraph_t body = cp.conditional.phGraph_out[0];
    if ((ce = cudaStreamBeginCaptureToGraph(st, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal)) !=
        cudaSuccess)
      return ctx.cuda_fail(ce, "loop capture");
    const int64_t l0 = ctx.timer.launches;
    mlmc_status cs = MLMC_OK;
    ce = cudaMemsetAsync(S.count, 0, sizeof(int) * ctx.check_every, st);
    for (int b = 0; b < ctx.check_every && cs == MLMC_OK && ce == cudaSuccess; ++b) cs = run_vcycle_and_pcg(b & 1, b);
    if (cs == MLMC_OK && ce == cudaSuccess)
      ce = launch_loop_condition(h, S.count + (ctx.check_every - 1), outer_count + 1, loop_reps, st);
    const cudaError_t ee = cudaStreamEndCapture(st, &body);
    loop_launches = ctx.timer.launches - l0 + 1;   // the batch and the condition kernel
    ctx.timer.launches = l0;
    if (cs != MLMC_OK || ce != cudaSuccess || ee != cudaSuccess) {
      cudaGetLastError();
      return cs != MLMC_OK ? cs : ctx.cuda_fail(ce != cudaSuccess ? ce : ee, "loop capture");
    }
    if ((ce = cudaGraphInstantiate(&loop_graph, g, 0)) != cudaSuccess) {
      loop_graph = nullptr;
      return ctx.cuda_fail(ce, "loop instantiate");
    }
    return MLMC_OK;
  };

  const double floor_tol = inner_double ? 1e-14 : ctx.floor_tol32;
  int outer = 0, max_it_seen = 0;
  for (;; ++outer) {
    if ((e = cudaMemsetAsync(outer_count, 0, sizeof(int), st)) != cudaSuccess) return ctx.cuda_fail(e, "memset");
    MLMC_LAUNCH(kProfOther, "outer_check", launch_outer_check(S, total, ctx.cfg.rtol, floor_tol, outer_count, st));
    int h_outer = 0;
    if ((e = cudaMemcpyAsync(&h_outer, outer_count, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return ctx.cuda_fail(e, "outer_count");
    if (std::getenv("MLMC_TRACE")) {   // diagnostic: refinement progress of the first samples
      const int m = std::min(total, 4);
      std::vector<double> rrf(m), tol2(m), rref(m);
      std::vector<int> its(m), stt(m), oa(m);
      cudaMemcpy(rrf.data(), S.rrf, sizeof(double) * m, cudaMemcpyDeviceToHost);
      cudaMemcpy(tol2.data(), S.tol2, sizeof(double) * m, cudaMemcpyDeviceToHost);
      cudaMemcpy(rref.data(), S.rr_ref, sizeof(double) * m, cudaMemcpyDeviceToHost);
      cudaMemcpy(its.data(), S.iters, sizeof(int) * m, cudaMemcpyDeviceToHost);
      cudaMemcpy(stt.data(), S.status, sizeof(int) * m, cudaMemcpyDeviceToHost);
      cudaMemcpy(oa.data(), S.outer_active, sizeof(int) * m, cudaMemcpyDeviceToHost);
      for (int t = 0; t < m; ++t)
        std::fprintf(stderr, "[mlmc] outer %d sample %d active %d status %d iters %d |r|/|f| %.3e inner_tol %.3e\n",
                     outer, t, oa[t], stt[t], its[t], std::sqrt(rref[t] / std::max(rrf[t], 1e-300)), std::sqrt(tol2[t]));
    }
    if (h_outer == 0 || outer >= max_outer) break;
    // fresh inner solve: x = 0, p = 0, q = 0
    for (auto& g : G) {
      const size_t bytes = sizeof(T) * (size_t)g.grp->nsamp * 2 * (g.geo[0].nx + 1) * (g.geo[0].ny + 1);
      if ((e = cudaMemsetAsync(g.x, 0, bytes, st)) != cudaSuccess ||
          (e = cudaMemsetAsync(g.p[0], 0, bytes, st)) != cudaSuccess ||
          (e = cudaMemsetAsync(g.q, 0, bytes, st)) != cudaSuccess)
        return ctx.cuda_fail(e, "memset");
    }
    int it = 0;
    bool done_on_device = false;
    if (graphs && ctx.device_loop && loop_reps > 0) {
      if (!loop_graph) {
        const mlmc_status cs = build_loop();
        if (cs != MLMC_OK) return cs;
      }
      int h_loop[2] = {0, 0};
      if ((e = cudaMemsetAsync(outer_count + 1, 0, sizeof(int), st)) != cudaSuccess ||
          (e = cudaGraphLaunch(loop_graph, st)) != cudaSuccess ||
          (e = cudaMemcpyAsync(&h_loop[0], S.count + (ctx.check_every - 1), sizeof(int), cudaMemcpyDeviceToHost,
                               st)) != cudaSuccess ||
          (e = cudaMemcpyAsync(&h_loop[1], outer_count + 1, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return ctx.cuda_fail(e, "device loop");
      it = h_loop[1] * ctx.check_every;   // even: the host loop's buffer parity continues
      ctx.timer.launches += loop_launches * h_loop[1];
      done_on_device = h_loop[0] == 0;
    }
    while (!done_on_device && it < max_iter) {
      const int batch = std::min(ctx.check_every, max_iter - it);
      if (graphs && batch == ctx.check_every) {
        if (!batch_graph) {
          const mlmc_status cs = capture_batch();
          if (cs != MLMC_OK) return cs;
        }
        if ((e = cudaGraphLaunch(batch_graph, st)) != cudaSuccess) return ctx.cuda_fail(e, "graph launch");
        ctx.timer.launches += graph_launches;
        it += batch;
      } else {
        if ((e = cudaMemsetAsync(S.count, 0, sizeof(int) * batch, st)) != cudaSuccess)
          return ctx.cuda_fail(e, "memset");
        for (int b = 0; b < batch; ++b, ++it) {
          mlmc_status s2 = run_vcycle_and_pcg(it & 1, b);
          if (s2 != MLMC_OK) return s2;
        }
      }
      int h_count = 0;
      if ((e = cudaMemcpyAsync(&h_count, S.count + (batch - 1), sizeof(int), cudaMemcpyDeviceToHost, st)) !=
              cudaSuccess ||
          (e = cudaStreamSynchronize(st)) != cudaSuccess)
        return ctx.cuda_fail(e, "pcg_count");
      if (h_count == 0) break;
    }
    max_it_seen = std::max(max_it_seen, it);
    MLMC_LAUNCH(kProfOther, "inner_end", launch_inner_end(S, total, st));
    // d += x; after the first correction the inner CG's recursive residual (accurate
    // to unit roundoff times the correction's size) is the new refinement residual,
    // moved into r0 where it ended in r1
    {
      ViewList<T> L = empty_list<T>(ctx);
      std::vector<int64_t> per;
      for (size_t gi = 0; gi < G.size(); ++gi) {
        auto& g = G[gi];
        View<T> v = base_view(g, 0);
        v.a = g.x;
        v.ext1 = g.d;
        if (!exact[gi]) {   // this correction's recursive residual becomes the refinement residual
          v.b = g.r[1];
          v.o0 = g.r[0];
        }
        L.v[L.n++] = v;
        per.push_back(2 * (int64_t)(g.geo[0].nx + 1) * (g.geo[0].ny + 1));
      }
      const int tt = finalize_points(L, per);
      MLMC_LAUNCH(kProfOther, "update_d", launch_update_d<T>(L, S, tt, st));
    }
    // the groups marked exact: the one double-precision residual f - K d after their
    // first correction; the others: the reaction increment of the correction
    bool any_exact = false, any_rec = false;
    for (size_t gi = 0; gi < G.size(); ++gi) {
      if (exact[gi]) {
        any_exact = true;
        if ((e = cudaMemsetAsync(S.react + G[gi].sbase, 0, sizeof(double) * G[gi].grp->nsamp, st)) != cudaSuccess)
          return ctx.cuda_fail(e, "memset");
      } else {
        any_rec = true;
      }
    }
    if (any_exact) {
      rs = resid();
      if (rs != MLMC_OK) return rs;
    }
    if (any_rec) {
      ViewList<T> R = empty_list<T>(ctx);
      std::vector<int64_t> rows;
      for (size_t gi = 0; gi < G.size(); ++gi) {
        if (exact[gi]) continue;
        View<T> w = base_view(G[gi], 0);
        w.a = G[gi].x;
        R.v[R.n++] = w;
        rows.push_back(G[gi].geo[0].ny);
      }
      const int tr = finalize_points(R, rows);
      MLMC_LAUNCH(kProfOther, "react_delta", launch_react_delta<T>(R, S, tr, st));
    }
    if (any_exact) {
      std::fill(exact.begin(), exact.end(), 0);
      if ((e = cudaMemsetAsync(S.exact, 0, sizeof(int) * total, st)) != cudaSuccess) return ctx.cuda_fail(e, "memset");
    }
  }
  ctx.last_outer = outer;
  ctx.last_iters = max_it_seen;

  // not converged: still refinement-active
  {
    std::vector<int> oa(total), stv(total);
    if ((e = cudaMemcpyAsync(oa.data(), S.outer_active, sizeof(int) * total, cudaMemcpyDeviceToHost, st)) !=
            cudaSuccess ||
        (e = cudaMemcpyAsync(stv.data(), S.status, sizeof(int) * total, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return ctx.cuda_fail(e, "status");
    bool changed = false;
    for (int t = 0; t < total; ++t)
      if (oa[t] && stv[t] == 0) {
        stv[t] = MLMC_ERR_NOT_CONVERGED;
        changed = true;
      }
    if (failed)
      for (int t = 0; t < total; ++t) *failed = *failed || stv[t] != 0;
    if (changed &&
        (e = cudaMemcpyAsync(S.status, stv.data(), sizeof(int) * total, cudaMemcpyHostToDevice, st)) != cudaSuccess)
      return ctx.cuda_fail(e, "status");
    if (changed && (e = cudaStreamSynchronize(st)) != cudaSuccess) return ctx.cuda_fail(e, "status");
  }
  // reaction in its energy-consistent form (quadratic in the solve error)
  {
    ViewList<T> L = empty_list<T>(ctx);
    std::vector<int64_t> rows;
    for (auto& g : G) {
      View<T> v = base_view(g, 0);
      v.a = g.r[0];
      v.ext0 = g.d;
      L.v[L.n++] = v;
      rows.push_back(g.geo[0].ny + 1);
    }
    const int tw = finalize_points(L, rows);
    MLMC_LAUNCH(kProfOther, "react_energy", launch_react_energy<T>(L, S, ctx.cfg.shortening, tw, st));
  }
  // stress quantity from the final d
  {
    ViewList<double> L = d_list();
    int64_t acc = 0;
    for (int i = 0; i < L.n; ++i) {
      L.v[i].work_begin = (int)acc;
      L.v[i].nwork = (int)(L.v[i].nsamp * (int64_t)L.v[i].g.ny);   // one warp per element row
      acc += L.v[i].nwork;
    }
    MLMC_LAUNCH(kProfOther, "stress", launch_stress<T>(L, S, (int)acc, st));
  }
  for (auto& g : G) {
    const SolveGroup<T>& sg = *g.grp;
    if (sg.d_out &&
        (e = cudaMemcpyAsync(sg.d_out, g.d, sizeof(double) * sg.nsamp * 2 * (g.geo[0].nx + 1) * (g.geo[0].ny + 1),
                             cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return ctx.cuda_fail(e, "copy d");
    if ((e = cudaMemcpyAsync(sg.q, S.qoi + 2 * (size_t)g.sbase, sizeof(double) * 2 * sg.nsamp,
                             cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
      return ctx.cuda_fail(e, "copy q");
    if (sg.status &&
        (e = cudaMemcpyAsync(sg.status, S.status + g.sbase, sizeof(int) * sg.nsamp, cudaMemcpyDeviceToDevice, st)) !=
            cudaSuccess)
      return ctx.cuda_fail(e, "copy status");
    if (sg.iters &&
        (e = cudaMemcpyAsync(sg.iters, S.iters + g.sbase, sizeof(int) * sg.nsamp, cudaMemcpyDeviceToDevice, st)) !=
            cudaSuccess)
      return ctx.cuda_fail(e, "copy iters");
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return ctx.cuda_fail(e, "solve");
  return MLMC_OK;
}

// The V-cycle preconditioner is symmetric positive definite while the smoother's damping
// stays below 2 / lambda_max(B^-1 K) (B the pair-block diagonal). kOmega = 1/2 keeps that
// for every angle field (lambda_max <= 4 by the colouring bound); a larger ctx.omega
// smooths better where lambda_max is smaller, which it is for fields near the fibre axis
// (about 2.75 at 0 degrees). If a solve at such a damping leaves any sample
// unconverged (an indefinite preconditioner shows as a breakdown or a stall), the whole
// call is solved again at kOmega: its inputs (fields, nested-iteration starts) are
// unchanged, and every output is overwritten.
template <typename T>
mlmc_status solve_groups(Context& ctx, std::vector<SolveGroup<T>>& groups) {
  bool failed = false;
  mlmc_status s = solve_groups_once(ctx, groups, ctx.omega > kOmega ? &failed : nullptr);
  if (s == MLMC_OK && failed) {
    const double om = ctx.omega;
    ctx.omega = kOmega;
    s = solve_groups_once<T>(ctx, groups, nullptr);
    ctx.omega = om;
    ++ctx.omega_retries;
  }
  return s;
}

template <typename T>
mlmc_status apply_operator(Context& ctx, int mesh_level, int64_t n, const T* trig2, const T* p, T* q) {
  ViewList<T> L = empty_list<T>(ctx);
  const LevelLayout m = ctx.mesh(mesh_level);
  View<T> v;
  std::memset(&v, 0, sizeof(v));
  v.g = ctx.geo(m.nx, m.ny);
  v.nsamp = (int)n;
  v.tiles_x = strips_of(m.nx);
  v.tiles_y = chunks_of(m.ny);
  v.trig2 = trig2;
  v.a = p;
  v.o0 = q;
  L.v[L.n++] = v;
  const int tw = finalize_warps(ctx, L, StripOp::Apply);
  SampleState S;
  std::memset(&S, 0, sizeof(S));
  cudaError_t e = launch_strip<T>(StripOp::Apply, L, S, tw, ctx.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx.stream);
  return e == cudaSuccess ? MLMC_OK : ctx.cuda_fail(e, "apply");
}

template mlmc_status solve_groups<float>(Context&, std::vector<SolveGroup<float>>&);
template mlmc_status solve_groups<double>(Context&, std::vector<SolveGroup<double>>&);
template mlmc_status apply_operator<float>(Context&, int, int64_t, const float*, const float*, float*);
template mlmc_status apply_operator<double>(Context&, int, int64_t, const double*, const double*, double*);

}  // namespace mlmc
