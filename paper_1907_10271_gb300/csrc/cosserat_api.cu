// C ABI of the Cosserat engine (mlmc_cosserat.h): context, batching of the meshes of a
// call into one lock-stepped solve, the refinement / correction-CG loop on the host
// side, CUDA-graph replay of the correction iterations and the level moments.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mlmc_cosserat.h"
#include "cosserat.cuh"
#include "cosserat_host.h"
#include "engine.h"
#include "moments.cuh"

namespace {

thread_local std::string g_create_error_c;

bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// kernel kinds of the profile (mlmcc_profile_get)
enum Op {
  kOpXi, kOpSynth, kOpBuild, kOpRap, kOpInverse, kOpPre, kOpRestrict, kOpCoarse, kOpProlong, kOpPost,
  kOpCgApply, kOpCgUpdate, kOpScalar, kOpResid64, kOpAccumulate, kOpQoi, kOpMoments, kOpLayout, kOpCount
};
const char* const kOpNames[kOpCount] = {
    "kl_coefficients", "kl_synthesis", "build_fine", "rap", "coarsest_inverse", "pre", "restrict",
    "bottom", "prolong", "post", "cg_apply", "cg_update", "scalars", "resid64", "accumulate", "qoi",
    "moments", "layout"};

constexpr int kGraphIters = 4;        // correction iterations per graph replay (even)
constexpr int kMaxRefine = 30;        // FP64 residual evaluations per solve
constexpr size_t kArenaBudget = size_t(24) << 30;

// One batch: the samples (level stream, id) of one call solved on one mesh.
struct Group {
  int mesh;
  std::vector<int> levels;
  std::vector<uint64_t> ids;
};

// Device buffers of one batch, carved from the context's arena.
struct GroupBufs {
  int mesh, n, N, S, nkl, K;   // K multigrid levels (n, n/2, .., 2)
  int* levels;
  uint64_t* ids;
  double* xi;
  float* trig;   // [S][n_el][8] (or phi [S][n_el] doubles in field mode)
  mlmcc::FineSys F;
  std::vector<mlmcc::Lev> lev;
  float* Ainv;
};

}  // namespace

struct mlmcc_ctx {
  mlmcc_config cfg;
  cudaStream_t st = nullptr;
  std::string err;
  mlmcc::Consts consts;
  mlmcc::Consts* consts_dev = nullptr;
  std::vector<float*> basis;    // per mesh [2][n_el][n_kl]: hi, lo floats of the double basis, made on first use
  std::vector<int> klo, khi;
  mlmc::LevelAcc* acc_dev = nullptr;
  std::vector<mlmc::LevelAcc> acc_host;
  char* arena = nullptr;
  size_t cap = 0;
  int* pinned = nullptr;   // host-pinned count / iteration words
  int64_t launches = 0;
  int last_iters = 0, last_refine = 0;
  std::vector<int64_t> next_id;   // ids mlmcc_estimate has drawn per level since the last reset
  struct GraphEntry {
    std::vector<int64_t> key;
    cudaGraphExec_t exec;
    int64_t kernels;
  };
  std::vector<GraphEntry> graphs;
  // profile: CUDA events around every launch (graphs bypassed) while enabled
  bool prof_on = false;
  struct Pending {
    int op;
    int64_t items;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> ev_free;
  double prof_ms[kOpCount] = {};
  int64_t prof_launches[kOpCount] = {}, prof_items[kOpCount] = {};
  cudaEvent_t ev_get() {
    if (!ev_free.empty()) {
      cudaEvent_t e = ev_free.back();
      ev_free.pop_back();
      return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
  }
  // after a synchronize: fold the recorded launches into the totals
  void prof_collect() {
    for (const Pending& q : pending) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) prof_ms[q.op] += ms;
      prof_launches[q.op] += 1;
      prof_items[q.op] += q.items;
      ev_free.push_back(q.a);
      ev_free.push_back(q.b);
    }
    pending.clear();
    cudaGetLastError();
  }

  mlmc_status fail(mlmc_status s, const std::string& m) {
    err = m;
    return s;
  }
  mlmc_status cuda_fail(cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return MLMC_ERR_CUDA;
  }
  int mesh_n(int m) const { return cfg.n0 << m; }
  void drop_graphs() {
    for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
    graphs.clear();
  }
  ~mlmcc_ctx() {
    drop_graphs();
    for (const Pending& q : pending) {
      cudaEventDestroy(q.a);
      cudaEventDestroy(q.b);
    }
    for (cudaEvent_t e : ev_free) cudaEventDestroy(e);
    for (float* b : basis)
      if (b) cudaFree(b);
    if (acc_dev) cudaFree(acc_dev);
    if (consts_dev) cudaFree(consts_dev);
    if (arena) cudaFree(arena);
    if (pinned) cudaFreeHost(pinned);
  }
};

namespace {

#define CK(EXPR, WHAT)                                        \
  do {                                                        \
    const cudaError_t ck_ = (EXPR);                           \
    if (ck_ != cudaSuccess) return c.cuda_fail(ck_, (WHAT));  \
  } while (0)

using mlmcc::Lev;
using mlmcc::View;
using mlmcc::Views;

inline size_t align_up(size_t x) { return (x + 255) & ~size_t(255); }

// Lays out the buffers of all batches from base (sizes only when base is null).
size_t layout(const mlmcc_ctx& c, const std::vector<Group>& groups, char* base, std::vector<GroupBufs>& out,
              int** count_dev) {
  size_t off = 0;
  auto take = [&](size_t bytes) -> char* {
    char* p = base ? base + off : nullptr;
    off += align_up(std::max<size_t>(bytes, 1));
    return p;
  };
  out.clear();
  *count_dev = (int*)take(4 * sizeof(int));
  for (const Group& g : groups) {
    GroupBufs b{};
    b.mesh = g.mesh;
    b.n = c.mesh_n(g.mesh);
    b.N = (b.n + 1) * (b.n + 1);
    b.S = (int)g.ids.size();
    b.nkl = mlmcc::n_kl(c.cfg, g.mesh);
    b.K = 0;
    for (int m = b.n; m >= mlmcc::kCoarsest; m /= 2) {
      ++b.K;
      if (m == mlmcc::kCoarsest) break;
    }
    const size_t S = b.S, N = b.N, nel = (size_t)b.n * b.n;
    b.levels = (int*)take(S * sizeof(int));
    b.ids = (uint64_t*)take(S * sizeof(uint64_t));
    b.xi = (double*)take(S * b.nkl * sizeof(double));
    b.trig = (float*)take(S * nel * 8 * sizeof(float));
    b.F.Alo = (float4*)take(S * mlmcc::kGroups * N * sizeof(float4));
    b.F.bh = (float4*)take(S * N * sizeof(float4));
    b.F.bl = (float4*)take(S * N * sizeof(float4));
    b.F.dh = (float4*)take(S * N * sizeof(float4));
    b.F.dl = (float4*)take(S * N * sizeof(float4));
    b.F.trig = b.trig;
    b.F.c = (float4*)take(S * N * sizeof(float4));
    b.F.p0 = (float4*)take(S * N * sizeof(float4));
    b.F.p1 = (float4*)take(S * N * sizeof(float4));
    b.F.q = (float4*)take(S * N * sizeof(float4));
    b.F.st = (mlmcc::SampleState*)take(S * sizeof(mlmcc::SampleState));
    b.F.acc = (double*)take(S * 4 * sizeof(double));
    b.F.q_out = (double*)take(S * 2 * sizeof(double));
    b.F.stat_out = (int*)take(S * sizeof(int));
    b.F.iters = *count_dev + 2;
    b.F.mesh = g.mesh;
    b.F.klo = c.klo[g.mesh];
    b.F.khi = c.khi[g.mesh];
    int n = b.n;
    for (int k = 0; k < b.K; ++k, n /= 2) {
      Lev l{};
      l.n = n;
      l.N = (n + 1) * (n + 1);
      l.S = b.S;
      l.A = (float4*)take(S * mlmcc::kGroups * l.N * sizeof(float4));
      l.Dinv = (float4*)take(S * mlmcc::kDinvGroups * l.N * sizeof(float4));
      l.r = (float4*)take(S * l.N * sizeof(float4));
      l.x = (float4*)take(S * l.N * sizeof(float4));
      l.t = (float4*)take(S * l.N * sizeof(float4));
      b.lev.push_back(l);
    }
    b.Ainv = (float*)take(S * mlmcc::kCoarseDofs * mlmcc::kCoarseDofs * sizeof(float));
    out.push_back(b);
  }
  return off;
}

enum class Kind { Nodes, CoarseNodes, Bottom, Inverse, Qoi, Samples, Build };

// multigrid level at which a batch enters the fused bottom: its first mesh of at most
// kBottomN elements per side
int bottom_level(const GroupBufs& b) {
  int k = 0;
  while ((b.n >> k) > mlmcc::kBottomN) ++k;
  return k;
}

// View table of one launch: batches with multigrid level k (f) and k + 1 (c);
// `need` filters the batches (e.g. those whose coarsest level lies below k).
template <class Need>
Views make_views(const std::vector<GroupBufs>& G, int k, Kind kind, Need need, const mlmcc::Consts* cc) {
  Views V{};
  V.cc = cc;
  int blk = 0;
  for (const GroupBufs& b : G) {
    if (!need(b) || V.nv >= mlmcc::kMaxViews) continue;
    View& v = V.v[V.nv];
    const int kf = kind == Kind::Inverse ? b.K - 1 : (kind == Kind::Bottom ? bottom_level(b) : k);
    v.f = b.lev[kf];
    if (kf + 1 < b.K) v.c = b.lev[kf + 1];
    v.F = b.F;
    v.Ainv = b.Ainv;
    int threads = mlmcc::kThreads;
    switch (kind) {
      case Kind::Nodes: v.items = b.S * v.f.N; break;
      case Kind::CoarseNodes: v.items = b.S * v.c.N; break;
      case Kind::Bottom:
        v.items = b.S;
        threads = 1;   // one block per sample
        break;
      case Kind::Inverse:
        v.items = b.S;
        threads = mlmcc::kInverseWarps;   // samples per block of the inverse kernel
        break;
      case Kind::Qoi: {
        const int ncen = b.F.khi - b.F.klo + 1;
        v.items = b.S * (ncen * ncen + b.n);
        break;
      }
      case Kind::Samples: v.items = b.S; break;
      case Kind::Build: v.items = b.S * 5 * v.f.N; break;
    }
    v.blk0 = blk;
    blk += (v.items + threads - 1) / threads;
    ++V.nv;
  }
  V.nblk = blk;
  return V;
}

// All view tables of one solve.
struct Sched {
  int maxK = 0;
  Views fine, build, samples, qoi, bottom, inverse;
  int top_mask = 0;   // views of `bottom` whose entry mesh is their solve mesh
  std::vector<Views> pre, restr, prol, post, rap;
  int64_t vcycle_kernels = 0;
};

Sched schedule(const std::vector<GroupBufs>& G, const mlmcc::Consts* cc) {
  Sched s;
  auto all = [](const GroupBufs&) { return true; };
  for (const GroupBufs& b : G) s.maxK = std::max(s.maxK, b.K);
  s.fine = make_views(G, 0, Kind::Nodes, all, cc);
  s.build = make_views(G, 0, Kind::Build, all, cc);
  s.samples = make_views(G, 0, Kind::Samples, all, cc);
  s.qoi = make_views(G, 0, Kind::Qoi, all, cc);
  s.bottom = make_views(G, 0, Kind::Bottom, all, cc);
  s.inverse = make_views(G, 0, Kind::Inverse, all, cc);
  int nb = 0;
  for (const GroupBufs& b : G) {
    if (bottom_level(b) == 0) s.top_mask |= 1 << nb;
    ++nb;
  }
  int depth = 0;
  for (const GroupBufs& b : G) depth = std::max(depth, bottom_level(b));
  for (int k = 0; k < depth; ++k) {
    auto above = [k](const GroupBufs& b) { return k < bottom_level(b); };
    s.pre.push_back(make_views(G, k, Kind::Nodes, above, cc));
    s.restr.push_back(make_views(G, k, Kind::CoarseNodes, above, cc));
    s.prol.push_back(make_views(G, k, Kind::Nodes, above, cc));
    s.post.push_back(make_views(G, k, Kind::Nodes, above, cc));
  }
  for (int k = 0; k + 1 < s.maxK; ++k) {
    auto below = [k](const GroupBufs& b) { return k + 1 < b.K; };
    s.rap.push_back(make_views(G, k, Kind::CoarseNodes, below, cc));
  }
  s.vcycle_kernels = 4 * (int64_t)s.pre.size() + 1;
  return s;
}


mlmc_status ensure_basis(mlmcc_ctx& c, int m) {
  if (c.basis[m]) return MLMC_OK;
  const int n = c.mesh_n(m), nk = mlmcc::n_kl(c.cfg, m);
  std::vector<double> B;
  mlmcc::kl_basis(c.cfg, n, nk, B);
  // float-float split: hi = fl(b), lo = fl(b - hi)
  std::vector<float> hl(2 * B.size());
  for (size_t k = 0; k < B.size(); ++k) {
    hl[k] = (float)B[k];
    hl[B.size() + k] = (float)(B[k] - (double)hl[k]);
  }
  float* d = nullptr;
  CK(cudaMalloc(&d, sizeof(float) * hl.size()), "basis alloc");
  c.basis[m] = d;
  CK(cudaMemcpyAsync(d, hl.data(), sizeof(float) * hl.size(), cudaMemcpyHostToDevice, c.st), "basis upload");
  CK(cudaStreamSynchronize(c.st), "basis upload");
  return MLMC_OK;
}

mlmc_status ensure_arena(mlmcc_ctx& c, size_t bytes) {
  if (bytes <= c.cap) return MLMC_OK;
  CK(cudaStreamSynchronize(c.st), "arena");
  c.drop_graphs();
  if (c.arena) cudaFree(c.arena);
  c.arena = nullptr;
  c.cap = 0;
  const size_t want = bytes + bytes / 4;
  const cudaError_t e = cudaMalloc(&c.arena, want);
  if (e != cudaSuccess) {
    cudaGetLastError();
    c.arena = nullptr;
    return c.fail(MLMC_ERR_OOM, "device memory for the solve workspace");
  }
  c.cap = want;
  return MLMC_OK;
}

int64_t items_of(const Views& V) {
  int64_t n = 0;
  for (int k = 0; k < V.nv; ++k) n += V.v[k].items;
  return n;
}

// Counts every launch (and times it while profiling); after a failure it launches
// nothing more and keeps the first error.
struct Launcher {
  mlmcc_ctx& c;
  mlmc_status status = MLMC_OK;
  template <class F>
  bool operator()(int op, int64_t items, F launch) {
    if (status != MLMC_OK) return false;
    cudaEvent_t a = nullptr;
    if (c.prof_on) {
      a = c.ev_get();
      cudaEventRecord(a, c.st);
    }
    const cudaError_t e = launch();
    if (c.prof_on) {
      cudaEvent_t b = c.ev_get();
      cudaEventRecord(b, c.st);
      c.pending.push_back({op, items, a, b});
    }
    ++c.launches;
    if (e != cudaSuccess) {
      status = c.cuda_fail(e, kOpNames[op]);
      return false;
    }
    return true;
  }
  bool operator()(int op, const Views& V, cudaError_t (*fn)(const Views&, cudaStream_t)) {
    return (*this)(op, items_of(V), [&] { return fn(V, c.st); });
  }
};

// One V(1,1) cycle of every batch on its level-0 residual: z = level-0 t.
void vcycle(Launcher& L, const Sched& s, cudaStream_t st) {
  const int nd = (int)s.pre.size();
  for (int k = 0; k < nd; ++k) {
    L(kOpPre, s.pre[k], mlmcc::launch_pre);
    L(kOpRestrict, s.restr[k], mlmcc::launch_restrict);
  }
  L(kOpCoarse, items_of(s.bottom), [&] { return mlmcc::launch_bottom(s.bottom, s.top_mask, st); });
  for (int k = nd - 1; k >= 0; --k) {
    L(kOpProlong, s.prol[k], mlmcc::launch_prolong);
    const Views& V = s.post[k];
    L(kOpPost, items_of(V), [&] { return mlmcc::launch_post(V, k == 0, st); });
  }
}

// One correction-CG iteration of every active sample.
void cg_iteration(Launcher& L, const Sched& s, bool odd, int max_iter, cudaStream_t st) {
  L(kOpCgApply, items_of(s.fine), [&] { return mlmcc::launch_cg_apply(s.fine, odd, st); });
  L(kOpScalar, s.samples, mlmcc::launch_scal_a);
  L(kOpCgUpdate, items_of(s.fine), [&] { return mlmcc::launch_cg_update(s.fine, odd, st); });
  vcycle(L, s, st);
  L(kOpScalar, items_of(s.samples), [&] { return mlmcc::launch_scal_b(s.samples, max_iter, st); });
}

// kGraphIters iterations and the active count (into count_dev[0]), from a cached graph
// when the stream can be captured, else launched directly.
mlmc_status iterations(mlmcc_ctx& c, const Sched& s, const std::vector<GroupBufs>& G, int* count_dev,
                       int max_iter) {
  Launcher L{c};
  auto enqueue = [&]() {
    for (int k = 0; k < kGraphIters; ++k) cg_iteration(L, s, (k & 1) != 0, max_iter, c.st);
    if (L.status == MLMC_OK) {
      const cudaError_t e = cudaMemsetAsync(count_dev, 0, sizeof(int), c.st);
      if (e != cudaSuccess) L.status = c.cuda_fail(e, "memset");
    }
    L(kOpScalar, items_of(s.samples), [&] { return mlmcc::launch_count_active(s.samples, count_dev, c.st); });
  };
  if (!c.st || c.prof_on) {
    enqueue();
    return L.status;
  }
  std::vector<int64_t> key{(int64_t)(uintptr_t)c.arena, (int64_t)c.cap, max_iter};
  for (const GroupBufs& b : G) {
    key.push_back(b.mesh);
    key.push_back(b.S);
  }
  for (auto& g : c.graphs)
    if (g.key == key) {
      CK(cudaGraphLaunch(g.exec, c.st), "graph launch");
      c.launches += g.kernels;
      return MLMC_OK;
    }
  CK(cudaStreamBeginCapture(c.st, cudaStreamCaptureModeThreadLocal), "capture");
  const int64_t before = c.launches;
  enqueue();
  cudaGraph_t graph = nullptr;
  const cudaError_t ec = cudaStreamEndCapture(c.st, &graph);
  if (L.status != MLMC_OK) {
    if (graph) cudaGraphDestroy(graph);
    return L.status;
  }
  CK(ec, "capture");
  const int64_t kernels = c.launches - before;
  c.launches = before;
  cudaGraphExec_t exec = nullptr;
  const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  CK(ei, "graph instantiate");
  if (c.graphs.size() >= 8) {
    cudaGraphExecDestroy(c.graphs.front().exec);
    c.graphs.erase(c.graphs.begin());
  }
  c.graphs.push_back({key, exec, kernels});
  CK(cudaGraphLaunch(exec, c.st), "graph launch");
  c.launches += kernels;
  return MLMC_OK;
}

mlmc_status read_count(mlmcc_ctx& c, const int* count_dev, int* out) {
  CK(cudaMemcpyAsync(c.pinned, count_dev, sizeof(int), cudaMemcpyDeviceToHost, c.st), "count");
  CK(cudaStreamSynchronize(c.st), "count");
  *out = c.pinned[0];
  return MLMC_OK;
}


struct GroupOut {
  std::vector<double> q;     // [S][2]
  std::vector<int> status;   // [S]
  std::vector<double> phi;   // field mode: [S][n_el]
  std::vector<double> d;     // displacement mode: [S][N][3]
};
enum class Mode { Solve, Field, Apply, Displacement };

template <typename U>
mlmc_status copy_from(mlmcc_ctx& c, const U* src, size_t count, std::vector<U>& out) {
  out.resize(count);
  if (!count) return MLMC_OK;
  CK(cudaMemcpyAsync(out.data(), src, sizeof(U) * count, cudaMemcpyDeviceToHost, c.st), "copy");
  return MLMC_OK;
}

mlmc_status run_once(mlmcc_ctx& c, const std::vector<Group>& groups, Mode mode, std::vector<GroupOut>& out,
                     const double* x_in, double* y_out) {
  std::vector<GroupBufs> G;
  int* count_dev = nullptr;
  const size_t bytes = layout(c, groups, nullptr, G, &count_dev);
  mlmc_status s = ensure_arena(c, bytes);
  if (s != MLMC_OK) return s;
  layout(c, groups, c.arena, G, &count_dev);
  for (const GroupBufs& b : G)
    if ((s = ensure_basis(c, b.mesh)) != MLMC_OK) return s;
  Launcher L{c};
  CK(cudaMemsetAsync(count_dev, 0, 4 * sizeof(int), c.st), "memset");
  for (size_t g = 0; g < G.size(); ++g) {
    const GroupBufs& b = G[g];
    CK(cudaMemcpyAsync(b.levels, groups[g].levels.data(), sizeof(int) * b.S, cudaMemcpyHostToDevice, c.st), "ids");
    CK(cudaMemcpyAsync(b.ids, groups[g].ids.data(), sizeof(uint64_t) * b.S, cudaMemcpyHostToDevice, c.st), "ids");
    L(kOpXi, b.S, [&] {
      return mlmc::launch_kl_coefficients(c.cfg.seed, 0, 0, b.levels, b.ids, b.S, b.nkl, b.xi, nullptr,
                                          count_dev + 1, c.st);
    });
    L(kOpSynth, (int64_t)b.S * b.n * b.n, [&] {
      const size_t nb = (size_t)b.n * b.n * b.nkl;
      return mlmcc::launch_synth_ff(b.xi, c.basis[b.mesh], c.basis[b.mesh] + nb, b.S, b.n * b.n, b.nkl, b.trig,
                                    mode != Mode::Field, c.st);
    });
  }
  if (L.status != MLMC_OK) return L.status;
  out.assign(G.size(), GroupOut{});
  if (mode == Mode::Field) {
    for (size_t g = 0; g < G.size(); ++g)
      if ((s = copy_from(c, (const double*)G[g].trig, (size_t)G[g].S * G[g].n * G[g].n, out[g].phi)) != MLMC_OK)
        return s;
    CK(cudaStreamSynchronize(c.st), "field");
    return MLMC_OK;
  }
  const Sched sc = schedule(G, c.consts_dev);
  for (const GroupBufs& b : G) {
    CK(cudaMemsetAsync(b.F.st, 0, sizeof(mlmcc::SampleState) * b.S, c.st), "memset");
    CK(cudaMemsetAsync(b.F.acc, 0, sizeof(double) * 4 * b.S, c.st), "memset");
    CK(cudaMemsetAsync(b.F.c, 0, sizeof(float4) * b.S * b.N, c.st), "memset");
  }
  L(kOpBuild, sc.build, mlmcc::launch_build_fine);
  if (mode == Mode::Apply) {
    const GroupBufs& b = G[0];
    const size_t cnt = (size_t)b.S * 3 * b.N;
    double* xs = nullptr;
    CK(cudaMallocAsync(&xs, sizeof(double) * cnt * 2, c.st), "apply alloc");
    double* ys = xs + cnt;
    CK(cudaMemcpyAsync(xs, x_in, sizeof(double) * cnt, cudaMemcpyDefault, c.st), "apply input");
    L(kOpResid64, items_of(sc.fine), [&] { return mlmcc::launch_apply64(sc.fine, xs, ys, c.st); });
    if (L.status == MLMC_OK) CK(cudaMemcpyAsync(y_out, ys, sizeof(double) * cnt, cudaMemcpyDefault, c.st), "copy");
    cudaFreeAsync(xs, c.st);
    CK(cudaStreamSynchronize(c.st), "apply");
    return L.status;
  }
  for (size_t k = 0; k < sc.rap.size(); ++k) L(kOpRap, sc.rap[k], mlmcc::launch_rap);
  L(kOpInverse, sc.inverse, mlmcc::launch_coarsest_inverse);
  if (L.status != MLMC_OK) return L.status;
  const double rtol = c.cfg.rtol > 0 ? c.cfg.rtol : 1e-8;
  const int max_iter = c.cfg.max_iter > 0 ? c.cfg.max_iter : 400;
  for (int refine = 0; refine < kMaxRefine; ++refine) {
    L(kOpResid64, items_of(sc.fine), [&] { return mlmcc::launch_resid64(sc.fine, refine == 0, c.st); });
    L(kOpScalar, items_of(sc.samples), [&] { return mlmcc::launch_outer_check(sc.samples, rtol, max_iter, c.st); });
    CK(cudaMemsetAsync(count_dev, 0, sizeof(int), c.st), "memset");
    L(kOpScalar, items_of(sc.samples), [&] { return mlmcc::launch_count_active(sc.samples, count_dev, c.st); });
    if (L.status != MLMC_OK) return L.status;
    int act = 0;
    if ((s = read_count(c, count_dev, &act)) != MLMC_OK) return s;
    if (act == 0) break;
    vcycle(L, sc, c.st);
    L(kOpScalar, items_of(sc.samples), [&] { return mlmcc::launch_scal_b(sc.samples, max_iter, c.st); });
    if (L.status != MLMC_OK) return L.status;
    for (int rep = 0; rep < max_iter / kGraphIters + 2; ++rep) {
      if ((s = iterations(c, sc, G, count_dev, max_iter)) != MLMC_OK) return s;
      if ((s = read_count(c, count_dev, &act)) != MLMC_OK) return s;
      if (act == 0) break;
    }
    L(kOpAccumulate, sc.fine, mlmcc::launch_accumulate);
  }
  L(kOpQoi, sc.qoi, mlmcc::launch_qoi);
  L(kOpScalar, sc.samples, mlmcc::launch_qoi_final);
  if (L.status != MLMC_OK) return L.status;
  for (size_t g = 0; g < G.size(); ++g) {
    if ((s = copy_from(c, G[g].F.q_out, 2 * (size_t)G[g].S, out[g].q)) != MLMC_OK) return s;
    if ((s = copy_from(c, G[g].F.stat_out, (size_t)G[g].S, out[g].status)) != MLMC_OK) return s;
  }
  if (mode == Mode::Displacement) {
    const GroupBufs& b = G[0];
    const size_t cnt = (size_t)b.S * 3 * b.N;
    double* tmp = nullptr;
    CK(cudaMallocAsync(&tmp, sizeof(double) * cnt, c.st), "alloc");
    L(kOpLayout, cnt, [&] { return mlmcc::launch_ff_to_aos(b.F.dh, b.F.dl, tmp, b.S, b.n, c.cfg.shortening, c.st); });
    if (L.status == MLMC_OK) {
      out[0].d.resize(cnt);
      CK(cudaMemcpyAsync(out[0].d.data(), tmp, sizeof(double) * cnt, cudaMemcpyDeviceToHost, c.st), "copy");
    }
    cudaFreeAsync(tmp, c.st);
    if (L.status != MLMC_OK) return L.status;
  }
  CK(cudaMemcpyAsync(c.pinned, count_dev, 4 * sizeof(int), cudaMemcpyDeviceToHost, c.st), "copy");
  CK(cudaStreamSynchronize(c.st), "solve");
  if (c.prof_on) c.prof_collect();
  if (c.pinned[1]) return c.fail(MLMC_ERR_CUDA, "normal generator exceeded its draw cap");
  c.last_iters = std::max(c.last_iters, c.pinned[2]);
  c.last_refine = std::max(c.last_refine, c.pinned[3]);
  return MLMC_OK;
}

// Splits the batches into rounds whose workspace fits the arena budget.
mlmc_status run_groups(mlmcc_ctx& c, const std::vector<Group>& groups, Mode mode, std::vector<GroupOut>& out,
                       const double* x_in = nullptr, double* y_out = nullptr) {
  c.last_iters = c.last_refine = 0;
  std::vector<GroupBufs> G;
  int* cd = nullptr;
  const size_t bytes = layout(c, groups, nullptr, G, &cd);
  const size_t rounds = (bytes + kArenaBudget - 1) / kArenaBudget;
  if (rounds <= 1 || mode == Mode::Apply || mode == Mode::Displacement)
    return run_once(c, groups, mode, out, x_in, y_out);
  out.assign(groups.size(), GroupOut{});
  for (size_t r = 0; r < rounds; ++r) {
    std::vector<Group> part;
    std::vector<size_t> which;
    for (size_t g = 0; g < groups.size(); ++g) {
      const size_t S = groups[g].ids.size(), per = (S + rounds - 1) / rounds;
      const size_t lo = std::min(S, r * per), hi = std::min(S, lo + per);
      if (hi <= lo) continue;
      Group p{groups[g].mesh, {}, {}};
      p.levels.assign(groups[g].levels.begin() + lo, groups[g].levels.begin() + hi);
      p.ids.assign(groups[g].ids.begin() + lo, groups[g].ids.begin() + hi);
      part.push_back(std::move(p));
      which.push_back(g);
    }
    std::vector<GroupOut> po;
    const int it = c.last_iters, rf = c.last_refine;
    mlmc_status s = run_once(c, part, mode, po, x_in, y_out);
    if (s != MLMC_OK) return s;
    c.last_iters = std::max(it, c.last_iters);
    c.last_refine = std::max(rf, c.last_refine);
    for (size_t k = 0; k < part.size(); ++k) {
      GroupOut& o = out[which[k]];
      o.q.insert(o.q.end(), po[k].q.begin(), po[k].q.end());
      o.status.insert(o.status.end(), po[k].status.begin(), po[k].status.end());
      o.phi.insert(o.phi.end(), po[k].phi.begin(), po[k].phi.end());
    }
  }
  return MLMC_OK;
}

template <typename U>
mlmc_status copy_out(mlmcc_ctx& c, U* dst, const U* src, size_t count) {
  if (!dst || !count) return MLMC_OK;
  CK(cudaMemcpyAsync(dst, src, sizeof(U) * count, dev_ptr(dst) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost,
                     c.st),
     "copy");
  CK(cudaStreamSynchronize(c.st), "copy");
  return MLMC_OK;
}


mlmc_status check_ids(mlmcc_ctx& c, int level, int mesh, int64_t n) {
  if (level < 0 || level >= c.cfg.levels) return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  if (mesh < 0 || mesh >= c.cfg.levels) return c.fail(MLMC_ERR_INVALID_ARG, "mesh level out of range");
  if (n < 0 || n > (int64_t(1) << 24)) return c.fail(MLMC_ERR_INVALID_ARG, "bad sample count");
  return MLMC_OK;
}

Group one_group(int level, int mesh, uint64_t first_id, int64_t n) {
  Group g{mesh, std::vector<int>((size_t)n, level), std::vector<uint64_t>((size_t)n)};
  for (int64_t k = 0; k < n; ++k) g.ids[k] = first_id + (uint64_t)k;
  return g;
}

}  // namespace

extern "C" {

mlmc_status mlmcc_create(const mlmcc_config* cfg, void* cuda_stream, mlmcc_ctx** out) {
  if (!out) return MLMC_ERR_INVALID_ARG;
  *out = nullptr;
  if (!cfg) {
    g_create_error_c = "null config";
    return MLMC_ERR_INVALID_ARG;
  }
  std::string msg;
  if (!mlmcc::validate(*cfg, msg)) {
    g_create_error_c = msg;
    return MLMC_ERR_INVALID_ARG;
  }
  mlmcc_ctx* h = new mlmcc_ctx();
  mlmcc_ctx& c = *h;
  c.cfg = *cfg;
  c.st = (cudaStream_t)cuda_stream;
  const int L = cfg->levels;
  double C[16], D[4], Cm[5][16], Dm[5][4];
  mlmcc::fibre_constants(*cfg, C, D);
  mlmcc::trig_basis(C, D, Cm, Dm);
  std::memset(&c.consts, 0, sizeof(c.consts));
  for (int m = 0; m < mlmcc::kTerms; ++m)
    for (int k = 0; k < 16; ++k) c.consts.Cm[m][k] = Cm[m][k];
  c.klo.assign(L, 0);
  c.khi.assign(L, -1);
  for (int lv = 0; lv < L; ++lv) {
    const double hh = cfg->L / c.mesh_n(lv);
    c.consts.h[lv] = hh;
    // the element matrix is linear in (C*, D*): the trig-basis matrices of K follow
    for (int m = 0; m < mlmcc::kTerms; ++m) {
      mlmcc::element_matrix(Cm[m], Dm[m], hh, c.consts.Km[lv][m]);
      for (int k = 0; k < 144; ++k) {
        const double v = c.consts.Km[lv][m][k];
        c.consts.Kmh[lv][m][k] = (float)v;
        c.consts.Kml[lv][m][k] = (float)(v - (double)c.consts.Kmh[lv][m][k]);
      }
    }
    mlmcc::centre_range(*cfg, c.mesh_n(lv), &c.klo[lv], &c.khi[lv]);
  }
  c.consts.shortening = cfg->shortening;
  c.consts.msh_hi = (float)(-cfg->shortening);
  c.consts.msh_lo = (float)(-cfg->shortening - (double)c.consts.msh_hi);
  c.consts.tau_y = cfg->tau_y;
  c.consts.R = cfg->R_ratio;
  c.basis.assign(L, nullptr);
  c.acc_host.assign(L, mlmc::LevelAcc{});
  c.next_id.assign(L, 0);
  cudaError_t e = cudaMalloc(&c.consts_dev, sizeof(mlmcc::Consts));
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(c.consts_dev, &c.consts, sizeof(mlmcc::Consts), cudaMemcpyHostToDevice, c.st);
  if (e == cudaSuccess) e = cudaMalloc(&c.acc_dev, sizeof(mlmc::LevelAcc) * L);
  if (e == cudaSuccess) e = cudaMemsetAsync(c.acc_dev, 0, sizeof(mlmc::LevelAcc) * L, c.st);
  if (e == cudaSuccess) e = cudaMallocHost(&c.pinned, 16 * sizeof(int));
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.st);
  if (e != cudaSuccess) {
    g_create_error_c = std::string("CUDA: ") + cudaGetErrorString(e);
    cudaGetLastError();
    delete h;
    return MLMC_ERR_CUDA;
  }
  *out = h;
  return MLMC_OK;
}

void mlmcc_destroy(mlmcc_ctx* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  delete h;
}

const char* mlmcc_last_error(const mlmcc_ctx* h) { return h ? h->err.c_str() : g_create_error_c.c_str(); }

mlmc_status mlmcc_sample_levels(mlmcc_ctx* h, int32_t n_req, const int32_t* levels, const uint64_t* first_ids,
                                const int64_t* counts, double* q_fine, double* q_coarse, int32_t* status) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmcc_ctx& c = *h;
  if (n_req < 0 || (n_req > 0 && (!levels || !first_ids || !counts)))
    return c.fail(MLMC_ERR_INVALID_ARG, "bad request arrays");
  int64_t total = 0;
  std::vector<int> seen(c.cfg.levels, 0);
  for (int r = 0; r < n_req; ++r) {
    mlmc_status s = check_ids(c, levels[r], levels[r], counts[r]);
    if (s != MLMC_OK) return s;
    if (seen[levels[r]]++) return c.fail(MLMC_ERR_INVALID_ARG, "a level appears twice");
    total += counts[r];
  }
  if (total > (int64_t(1) << 24)) return c.fail(MLMC_ERR_INVALID_ARG, "too many samples");
  if (total == 0) return MLMC_OK;
  // one batch per mesh: level m's fine solves and level m + 1's coarse solves
  std::vector<Group> groups;
  std::vector<int> gidx(c.cfg.levels, -1);
  auto group_of = [&](int mesh) -> Group& {
    if (gidx[mesh] < 0) {
      gidx[mesh] = (int)groups.size();
      groups.push_back(Group{mesh, {}, {}});
    }
    return groups[gidx[mesh]];
  };
  std::vector<size_t> off_f(n_req), off_c(n_req);
  for (int r = 0; r < n_req; ++r) {
    const int lv = levels[r];
    if (!counts[r]) continue;
    Group& gf = group_of(lv);
    off_f[r] = gf.ids.size();
    for (int64_t k = 0; k < counts[r]; ++k) {
      gf.levels.push_back(lv);
      gf.ids.push_back(first_ids[r] + (uint64_t)k);
    }
    if (lv > 0) {
      Group& gc = group_of(lv - 1);
      off_c[r] = gc.ids.size();
      for (int64_t k = 0; k < counts[r]; ++k) {
        gc.levels.push_back(lv);
        gc.ids.push_back(first_ids[r] + (uint64_t)k);
      }
    }
  }
  std::vector<GroupOut> out;
  mlmc_status s = run_groups(c, groups, Mode::Solve, out);
  if (s != MLMC_OK) return s;
  std::vector<double> qf(2 * (size_t)total), qc(2 * (size_t)total, 0.0);
  std::vector<int> sts((size_t)total, 0);
  size_t base = 0;
  double* tmp = nullptr;
  CK(cudaMallocAsync(&tmp, sizeof(double) * 4 * (size_t)total + sizeof(int) * (size_t)total, c.st), "alloc");
  for (int r = 0; r < n_req; ++r) {
    const int lv = levels[r];
    const size_t n = (size_t)counts[r];
    if (!n) continue;
    const GroupOut& of = out[gidx[lv]];
    for (size_t k = 0; k < n; ++k) {
      qf[2 * (base + k)] = of.q[2 * (off_f[r] + k)];
      qf[2 * (base + k) + 1] = of.q[2 * (off_f[r] + k) + 1];
      sts[base + k] = of.status[off_f[r] + k];
    }
    if (lv > 0) {
      const GroupOut& oc = out[gidx[lv - 1]];
      for (size_t k = 0; k < n; ++k) {
        qc[2 * (base + k)] = oc.q[2 * (off_c[r] + k)];
        qc[2 * (base + k) + 1] = oc.q[2 * (off_c[r] + k) + 1];
        if (oc.status[off_c[r] + k]) sts[base + k] = oc.status[off_c[r] + k];
      }
    }
    double* dqf = tmp + 4 * base;
    double* dqc = dqf + 2 * n;
    int* dst = (int*)(tmp + 4 * (size_t)total) + base;
    CK(cudaMemcpyAsync(dqf, &qf[2 * base], sizeof(double) * 2 * n, cudaMemcpyHostToDevice, c.st), "copy");
    CK(cudaMemcpyAsync(dqc, &qc[2 * base], sizeof(double) * 2 * n, cudaMemcpyHostToDevice, c.st), "copy");
    CK(cudaMemcpyAsync(dst, &sts[base], sizeof(int) * n, cudaMemcpyHostToDevice, c.st), "copy");
    Launcher L{c};
    if (!L(kOpMoments, (int64_t)n,
           [&] { return mlmc::launch_moments(dqf, lv > 0 ? dqc : nullptr, dst, (int64_t)n, c.acc_dev + lv, c.st); }))
      return L.status;
    base += n;
  }
  cudaFreeAsync(tmp, c.st);
  CK(cudaStreamSynchronize(c.st), "moments");
  if (c.prof_on) c.prof_collect();
  if ((s = copy_out(c, q_fine, qf.data(), qf.size())) != MLMC_OK) return s;
  if ((s = copy_out(c, q_coarse, qc.data(), qc.size())) != MLMC_OK) return s;
  return copy_out(c, status, sts.data(), sts.size());
}

mlmc_status mlmcc_sample_level(mlmcc_ctx* h, int32_t level, uint64_t first_id, int64_t n, double* q_fine,
                               double* q_coarse, int32_t* status) {
  return mlmcc_sample_levels(h, 1, &level, &first_id, &n, q_fine, q_coarse, status);
}

mlmc_status mlmcc_solve_batch(mlmcc_ctx* h, const mlmc_item* items, int64_t n, double* q, int32_t* status) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmcc_ctx& c = *h;
  if (n < 0 || n > (int64_t(1) << 24) || (n > 0 && (!items || !q))) return c.fail(MLMC_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return MLMC_OK;
  std::vector<mlmc_item> it((size_t)n);
  if (dev_ptr(items)) {
    CK(cudaMemcpy(it.data(), items, sizeof(mlmc_item) * n, cudaMemcpyDeviceToHost), "items");
  } else {
    std::memcpy(it.data(), items, sizeof(mlmc_item) * n);
  }
  std::vector<Group> groups;
  std::vector<int> gidx(c.cfg.levels, -1);
  std::vector<std::pair<int, size_t>> where((size_t)n);
  for (int64_t k = 0; k < n; ++k) {
    mlmc_status s = check_ids(c, it[k].level, it[k].mesh_level, 1);
    if (s != MLMC_OK) return s;
    const int m = it[k].mesh_level;
    if (gidx[m] < 0) {
      gidx[m] = (int)groups.size();
      groups.push_back(Group{m, {}, {}});
    }
    Group& g = groups[gidx[m]];
    where[k] = {gidx[m], g.ids.size()};
    g.levels.push_back(it[k].level);
    g.ids.push_back(it[k].sample_id);
  }
  std::vector<GroupOut> out;
  mlmc_status s = run_groups(c, groups, Mode::Solve, out);
  if (s != MLMC_OK) return s;
  std::vector<double> qo(2 * (size_t)n);
  std::vector<int> so((size_t)n);
  for (int64_t k = 0; k < n; ++k) {
    const GroupOut& o = out[where[k].first];
    qo[2 * k] = o.q[2 * where[k].second];
    qo[2 * k + 1] = o.q[2 * where[k].second + 1];
    so[k] = o.status[where[k].second];
  }
  if ((s = copy_out(c, q, qo.data(), qo.size())) != MLMC_OK) return s;
  return copy_out(c, status, so.data(), so.size());
}

mlmc_status mlmcc_level_stats_get(mlmcc_ctx* h, int32_t level, mlmc_level_stats* out) {
  if (!h || !out) return MLMC_ERR_INVALID_ARG;
  mlmcc_ctx& c = *h;
  if (level < 0 || level >= c.cfg.levels) return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  CK(cudaMemcpyAsync(c.acc_host.data(), c.acc_dev, sizeof(mlmc::LevelAcc) * c.cfg.levels, cudaMemcpyDeviceToHost,
                     c.st),
     "stats");
  CK(cudaStreamSynchronize(c.st), "stats");
  const mlmc::LevelAcc& a = c.acc_host[level];
  std::memset(out, 0, sizeof(*out));
  out->n = a.n;
  for (int k = 0; k < 2; ++k) {
    out->mean[k] = a.mean[k];
    out->m2[k] = a.m2[k];
    out->var[k] = a.n > 0 ? a.m2[k] / (double)a.n : 0.0;
    out->sum_qf[k] = a.sum_qf[k] - a.comp_qf[k];
    out->sum_qc[k] = a.sum_qc[k] - a.comp_qc[k];
  }
  auto dofs = [&](int m) { return 3.0 * (c.mesh_n(m) + 1.0) * (c.mesh_n(m) + 1.0); };
  out->cost = dofs(level) + (level > 0 ? dofs(level - 1) : 0.0);
  return MLMC_OK;
}

mlmc_status mlmcc_reset_stats(mlmcc_ctx* h) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmcc_ctx& c = *h;
  CK(cudaMemsetAsync(c.acc_dev, 0, sizeof(mlmc::LevelAcc) * c.cfg.levels, c.st), "reset");
  CK(cudaStreamSynchronize(c.st), "reset");
  std::fill(c.next_id.begin(), c.next_id.end(), 0);
  return MLMC_OK;
}

mlmc_status mlmcc_estimate(mlmcc_ctx* h, double e, double theta, int64_t n_star, int32_t max_level, int32_t qoi,
                           double m, double alpha, double gamma, double* estimate, mlmc_level_stats* stats,
                           int32_t* L_out) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmcc_ctx& c = *h;
  if (!(e > 0) || !(theta > 0 && theta < 1) || n_star < 1 || max_level < 0 || qoi < 0 || qoi > 1 || !(m > 1) ||
      !(alpha > 0) || !(gamma > 0))
    return c.fail(MLMC_ERR_INVALID_ARG, "bad Algorithm 1 parameters");
  max_level = std::min<int32_t>(max_level, c.cfg.levels - 1);
  const double es2 = theta * e * e, eb = std::sqrt(1.0 - theta) * e;
  auto dofs = [&](int l) { return 3.0 * (c.mesh_n(l) + 1.0) * (c.mesh_n(l) + 1.0); };
  auto cost = [&](int l) { return std::pow(dofs(l), gamma) + (l > 0 ? std::pow(dofs(l - 1), gamma) : 0.0); };
  auto refresh = [&]() -> mlmc_status {
    CK(cudaMemcpyAsync(c.acc_host.data(), c.acc_dev, sizeof(mlmc::LevelAcc) * c.cfg.levels, cudaMemcpyDeviceToHost,
                       c.st),
       "stats");
    CK(cudaStreamSynchronize(c.st), "stats");
    return MLMC_OK;
  };
  auto take = [&](int l, int64_t upto) -> mlmc_status {
    if (c.next_id[l] >= upto) return MLMC_OK;
    const int64_t cnt = upto - c.next_id[l];
    const mlmc_status s = mlmcc_sample_level(h, l, (uint64_t)c.next_id[l], cnt, nullptr, nullptr, nullptr);
    if (s != MLMC_OK) return s;
    c.next_id[l] = upto;
    return MLMC_OK;
  };
  int L = -1;
  bool converged = false;
  mlmc_status s = MLMC_OK;
  while (!converged) {
    if (L + 1 > max_level) break;
    ++L;
    if ((s = take(L, n_star)) != MLMC_OK || (s = refresh()) != MLMC_OK) return s;
    std::vector<double> V(L + 1);
    double tot = 0.0;
    for (int l = 0; l <= L; ++l) {
      const mlmc::LevelAcc& a = c.acc_host[l];
      V[l] = a.n > 0 ? a.m2[qoi] / (double)a.n : 0.0;
      tot += std::sqrt(V[l] * cost(l));
    }
    for (int l = 0; l <= L; ++l) {
      const int64_t nhat = (int64_t)std::ceil(tot * std::sqrt(V[l] / cost(l)) / es2);
      if ((s = take(l, nhat)) != MLMC_OK) return s;
    }
    if ((s = refresh()) != MLMC_OK) return s;
    if (std::fabs(c.acc_host[L].mean[qoi]) / (std::pow(m, alpha) - 1.0) < eb) converged = true;
  }
  double est = 0.0;
  for (int l = 0; l <= L; ++l) est += c.acc_host[l].mean[qoi];
  if (estimate) *estimate = est;
  if (L_out) *L_out = L;
  if (stats)
    for (int l = 0; l <= L; ++l)
      if ((s = mlmcc_level_stats_get(h, l, &stats[l])) != MLMC_OK) return s;
  return converged ? MLMC_OK : c.fail(MLMC_ERR_NOT_CONVERGED, "max_level reached before the bias test passed");
}

mlmc_status mlmcc_field(mlmcc_ctx* h, int32_t level, int32_t mesh_level, uint64_t first_id, int64_t n,
                        double* phi) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmcc_ctx& c = *h;
  mlmc_status s = check_ids(c, level, mesh_level, n);
  if (s != MLMC_OK) return s;
  if (n == 0) return MLMC_OK;
  if (!phi) return c.fail(MLMC_ERR_INVALID_ARG, "phi is required");
  std::vector<GroupOut> out;
  if ((s = run_groups(c, {one_group(level, mesh_level, first_id, n)}, Mode::Field, out)) != MLMC_OK) return s;
  return copy_out(c, phi, out[0].phi.data(), out[0].phi.size());
}

mlmc_status mlmcc_apply(mlmcc_ctx* h, int32_t level, int32_t mesh_level, uint64_t first_id, int64_t n,
                        const double* x, double* y) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmcc_ctx& c = *h;
  mlmc_status s = check_ids(c, level, mesh_level, n);
  if (s != MLMC_OK) return s;
  if (n == 0) return MLMC_OK;
  if (!x || !y) return c.fail(MLMC_ERR_INVALID_ARG, "x and y are required");
  std::vector<GroupOut> out;
  return run_groups(c, {one_group(level, mesh_level, first_id, n)}, Mode::Apply, out, x, y);
}

mlmc_status mlmcc_displacement(mlmcc_ctx* h, int32_t level, int32_t mesh_level, uint64_t first_id, int64_t n,
                               double* d, int32_t* status) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmcc_ctx& c = *h;
  mlmc_status s = check_ids(c, level, mesh_level, n);
  if (s != MLMC_OK) return s;
  if (n == 0) return MLMC_OK;
  if (!d) return c.fail(MLMC_ERR_INVALID_ARG, "d is required");
  std::vector<GroupOut> out;
  if ((s = run_groups(c, {one_group(level, mesh_level, first_id, n)}, Mode::Displacement, out)) != MLMC_OK)
    return s;
  if ((s = copy_out(c, d, out[0].d.data(), out[0].d.size())) != MLMC_OK) return s;
  return copy_out(c, status, out[0].status.data(), out[0].status.size());
}

mlmc_status mlmcc_last_iters(mlmcc_ctx* h, int32_t* iterations, int32_t* refinements) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  if (iterations) *iterations = h->last_iters;
  if (refinements) *refinements = h->last_refine;
  return MLMC_OK;
}

mlmc_status mlmcc_profile_enable(mlmcc_ctx* h, int32_t on) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  cudaStreamSynchronize(h->st);
  h->prof_collect();
  h->prof_on = on != 0;
  for (int k = 0; k < kOpCount; ++k) {
    h->prof_ms[k] = 0.0;
    h->prof_launches[k] = h->prof_items[k] = 0;
  }
  return MLMC_OK;
}

mlmc_status mlmcc_profile_get(mlmcc_ctx* h, int32_t op, double* ms, int64_t* launches, int64_t* items) {
  if (!h || op < 0 || op >= kOpCount) return MLMC_ERR_INVALID_ARG;
  if (ms) *ms = h->prof_ms[op];
  if (launches) *launches = h->prof_launches[op];
  if (items) *items = h->prof_items[op];
  return MLMC_OK;
}

const char* mlmcc_profile_name(int32_t op) { return (op >= 0 && op < kOpCount) ? kOpNames[op] : nullptr; }

mlmc_status mlmcc_launch_count(mlmcc_ctx* h, int64_t* launches) {
  if (!h || !launches) return MLMC_ERR_INVALID_ARG;
  *launches = h->launches;
  return MLMC_OK;
}

}  // extern "C"
