// C ABI of the panel-buckling engine (include/mlmc_panel.h): context, the batched
// LOBPCG solve driver and the level-pair / moments entry points.
//
// Solve of one group (n samples on one mesh): the ply perturbations xi give each
// sample's laminate (D*, k G t) and its element matrices on every multigrid mesh; the
// coarsest mesh's K is inverted per sample. Block LOBPCG with two vectors runs on all
// samples in lock step (per-sample Rayleigh-Ritz and convergence flags), its
// preconditioner one V(2,2) cycle on K for both residual columns at once (a column is a
// batch entry of the multigrid kernels). The converged first Ritz vector's Rayleigh
// quotient is evaluated in double.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mlmc_panel.h"
#include "engine.h"
#include "hex3d.cuh"
#include "moments.cuh"
#include "panel.cuh"

using mlmcp::PGrid;

namespace {

std::string g_create_error_p;

bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

struct Mesh {
  int nx, ny;
};

// multigrid meshes of a solve mesh: halve while both counts are even and ny stays >= 4
std::vector<Mesh> hierarchy(int nx, int ny) {
  std::vector<Mesh> h{{nx, ny}};
  while (nx % 2 == 0 && ny % 2 == 0 && ny / 2 >= 4) {
    nx /= 2;
    ny /= 2;
    h.push_back({nx, ny});
  }
  return h;
}

// free DOFs (4 node + component) of a mesh under the support conditions
std::vector<int> free_dofs(const Mesh& m, bool hard) {
  std::vector<int> f;
  for (int j = 0; j <= m.ny; ++j)
    for (int i = 0; i <= m.nx; ++i) {
      const bool bx = i == 0 || i == m.nx, by = j == 0 || j == m.ny;
      const int n = j * (m.nx + 1) + i;
      if (!(bx || by)) f.push_back(4 * n);
      if (!(hard && by)) f.push_back(4 * n + 1);
      if (!(hard && bx)) f.push_back(4 * n + 2);
    }
  return f;
}

}  // namespace

struct mlmcp_ctx {
  mlmcp_config cfg;
  cudaStream_t st = nullptr;
  std::string err;
  mlmcp::Laminate lam;
  std::vector<std::vector<Mesh>> hier;   // per MLMC mesh level
  std::vector<int*> free_dev;            // coarsest free DOFs per MLMC mesh level
  std::vector<int> nfree;
  mlmc::LevelAcc* acc_dev = nullptr;
  std::vector<mlmc::LevelAcc> acc_host;
  int last_iters = 0;
  double tol = 1e-4;
  int max_iter = 120;
  // patch smoother: the pristine laminate's patch inverses per mesh size (nx, ny), made
  // on first use and shared by every sample and solve
  std::vector<std::pair<std::pair<int, int>, float*>> patch_cache;
  // per MLMC mesh level: the coarsest mesh's inverse for the pristine laminate, shared by
  // every sample's multigrid cycle
  std::vector<float*> coarse_cache;
  // per MLMC mesh level: the executable graph of four LOBPCG iterations, updated with
  // each call's pointers and sizes (cudaGraphExecUpdate) rather than re-instantiated
  std::vector<cudaGraphExec_t> lobpcg_exec;

  mlmc_status fail(mlmc_status s, const std::string& m) {
    err = m;
    return s;
  }
  mlmc_status cuda_fail(cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return MLMC_ERR_CUDA;
  }
  PGrid grid(const Mesh& m, int nb, int cshift) const {
    PGrid g;
    g.nx = m.nx;
    g.ny = m.ny;
    g.nb = nb;
    g.cshift = cshift;
    g.hard = cfg.hard_support ? 1 : 0;
    g.hx = (float)(cfg.lx / m.nx);
    g.hy = (float)(cfg.ly / m.ny);
    return g;
  }
  ~mlmcp_ctx() {
    for (float* p : coarse_cache)
      if (p) cudaFree(p);
    for (cudaGraphExec_t g : lobpcg_exec)
      if (g) cudaGraphExecDestroy(g);
    for (auto& kv : patch_cache) cudaFree(kv.second);
    for (int* p : free_dev) cudaFree(p);
    if (acc_dev) cudaFree(acc_dev);
  }
};

namespace {

#define CK(EXPR, WHAT)                                        \
  do {                                                        \
    const cudaError_t ck_ = (EXPR);                           \
    if (ck_ != cudaSuccess) return c.cuda_fail(ck_, (WHAT));  \
  } while (0)

// stream-ordered scratch allocations released together
struct Scratch {
  cudaStream_t st;
  std::vector<void*> ptrs;
  cudaError_t err = cudaSuccess;
  template <typename U>
  U* take(size_t count) {
    void* p = nullptr;
    if (err == cudaSuccess) err = cudaMallocAsync(&p, sizeof(U) * std::max<size_t>(count, 1), st);
    if (err != cudaSuccess) return nullptr;
    ptrs.push_back(p);
    return static_cast<U*>(p);
  }
  ~Scratch() {
    for (void* p : ptrs) cudaFreeAsync(p, st);
  }
};

// Draws the ply perturbations (standard normals) of n samples: per-sample (level, id)
// from levels/ids (device) or (level, first_id + k).
mlmc_status draw_xi(mlmcp_ctx& c, int level, uint64_t first_id, const int* levels, const uint64_t* ids, int n,
                    double* xi) {
  Scratch sc{c.st};
  int* fail = sc.take<int>(2);
  CK(sc.err, "alloc");
  CK(cudaMemsetAsync(fail, 0, sizeof(int) * 2, c.st), "memset");
  CK(mlmc::launch_kl_coefficients(c.cfg.seed, level, first_id, levels, ids, n, c.cfg.n_plies, xi, nullptr, fail,
                                  c.st),
     "ply perturbations");
  int h_fail = 0;
  CK(cudaMemcpyAsync(&h_fail, fail, sizeof(int), cudaMemcpyDeviceToHost, c.st), "copy");
  CK(cudaStreamSynchronize(c.st), "ply perturbations");
  if (h_fail) return c.fail(MLMC_ERR_CUDA, "normal generator exceeded its draw cap");
  return MLMC_OK;
}

// The patch smoother's inverses on mesh m, built once from the pristine laminate (no
// perturbation) and kept in the context.
mlmc_status patch_inverses(mlmcp_ctx& c, const Mesh& m, float** out) {
  for (auto& kv : c.patch_cache)
    if (kv.first.first == m.nx && kv.first.second == m.ny) {
      *out = kv.second;
      return MLMC_OK;
    }
  Scratch sc{c.st};
  double* xi0 = sc.take<double>(c.cfg.n_plies);
  double* dstar = sc.take<double>(6);
  double* kgt = sc.take<double>(1);
  float* ke = sc.take<float>(144);
  CK(sc.err, "alloc");
  float* pinv = nullptr;
  CK(cudaMalloc(&pinv, sizeof(float) * mlmcp::kPatchTypes * mlmcp::kPatchDofs * mlmcp::kPatchDofs), "alloc");
  c.patch_cache.push_back({{m.nx, m.ny}, pinv});
  CK(cudaMemsetAsync(xi0, 0, sizeof(double) * c.cfg.n_plies, c.st), "memset");
  CK(mlmcp::launch_laminate(c.lam, xi0, 1, dstar, kgt, c.st), "laminate");
  CK(mlmcp::launch_element_matrices(dstar, kgt, 1, c.cfg.lx / m.nx, c.cfg.ly / m.ny, ke, nullptr, c.st), "element");
  CK(mlmcp::launch_patch_setup(c.grid(m, 1, 0), ke, 1, pinv, c.st), "patch setup");
  CK(cudaStreamSynchronize(c.st), "patch setup");
  *out = pinv;
  return MLMC_OK;
}

// n samples (perturbations xi, device [n][plies]) on MLMC mesh m; q [n][2], status [n]
// (device)
// The coarsest-mesh inverse of MLMC mesh level m's hierarchy for the pristine laminate
// (no perturbation), made on first use and shared by every sample: the coarsest level
// only preconditions, and the ply perturbations change its matrix by a few per cent.
mlmc_status coarse_inverse(mlmcp_ctx& c, int m, float** out) {
  if (c.coarse_cache.size() < (size_t)c.cfg.levels) c.coarse_cache.assign(c.cfg.levels, nullptr);
  if (c.coarse_cache[m]) {
    *out = c.coarse_cache[m];
    return MLMC_OK;
  }
  const Mesh& M = c.hier[m].back();
  const int nf = c.nfree[m];
  Scratch sc{c.st};
  double* xi0 = sc.take<double>(c.cfg.n_plies);
  double* dstar = sc.take<double>(6);
  double* kgt = sc.take<double>(1);
  float* ke = sc.take<float>(144);
  CK(sc.err, "alloc");
  float* ainv = nullptr;
  CK(cudaMalloc(&ainv, sizeof(float) * nf * nf), "alloc");
  c.coarse_cache[m] = ainv;
  CK(cudaMemsetAsync(xi0, 0, sizeof(double) * c.cfg.n_plies, c.st), "memset");
  CK(mlmcp::launch_laminate(c.lam, xi0, 1, dstar, kgt, c.st), "laminate");
  CK(mlmcp::launch_element_matrices(dstar, kgt, 1, c.cfg.lx / M.nx, c.cfg.ly / M.ny, ke, nullptr, c.st), "element");
  CK(mlmcp::launch_coarse_setup(c.grid(M, 1, 0), ke, 1, c.free_dev[m], nf, ainv, c.st), "coarse setup");
  CK(cudaStreamSynchronize(c.st), "coarse setup");
  *out = ainv;
  return MLMC_OK;
}

mlmc_status solve_p(mlmcp_ctx& c, int m, int n, const double* xi, double* q, int* status) {
  if (n <= 0) return MLMC_OK;
  {
    // a solve holds about 15 vectors of 2 n (nodes) float4: chunk it so that one vector
    // stays within 1 GB and the 2 n batch entries within a grid's y extent
    const int64_t nodes = (int64_t)((c.cfg.nx0 << m) + 1) * ((c.cfg.ny0 << m) + 1);
    const int per = (int)std::max<int64_t>(
        1, std::min<int64_t>(16384, ((int64_t)1 << 30) / (2 * nodes * (int64_t)sizeof(float4))));
    if (n > per) {
      int its = 0;
      for (int off = 0; off < n; off += per) {
        const int k = std::min(per, n - off);
        const mlmc_status s = solve_p(c, m, k, xi + (size_t)off * c.cfg.n_plies, q + 2 * (size_t)off, status + off);
        if (s != MLMC_OK) return s;
        its = std::max(its, c.last_iters);
      }
      c.last_iters = its;
      return MLMC_OK;
    }
  }
  cudaStream_t st = c.st;
  const std::vector<Mesh>& H = c.hier[m];
  const int L = (int)H.size();
  const int nb = n * mlmcp::kCols, cs = 1;
  const int nf = c.nfree[m];
  Scratch sc{st};
  double* dstar = sc.take<double>((size_t)n * 6);
  double* kgt = sc.take<double>(n);
  double* ke64 = sc.take<double>((size_t)n * 144);
  std::vector<float*> ke(L);
  for (int l = 0; l < L; ++l) ke[l] = sc.take<float>((size_t)n * 144);
  CK(sc.err, "alloc");
  float* ainv = nullptr;
  {
    const mlmc_status cs = coarse_inverse(c, m, &ainv);
    if (cs != MLMC_OK) return cs;
  }
  CK(mlmcp::launch_laminate(c.lam, xi, n, dstar, kgt, st), "laminate");
  for (int l = 0; l < L; ++l)
    CK(mlmcp::launch_element_matrices(dstar, kgt, n, c.cfg.lx / H[l].nx, c.cfg.ly / H[l].ny, ke[l],
                                      l == 0 ? ke64 : nullptr, st),
       "element matrices");
  const bool patch = c.cfg.smoother == 1;
  std::vector<float*> pinv(L, nullptr);   // patch smoother: shared inverses per smoothed mesh
  if (patch) {
    for (int l = 0; l + 1 < L; ++l) {
      const mlmc_status ps = patch_inverses(c, H[l], &pinv[l]);
      if (ps != MLMC_OK) return ps;
    }
  }

  // multigrid buffers (batch of nb entries) and the LOBPCG sets
  std::vector<PGrid> G(L);
  std::vector<float4*> bb(L, nullptr), xx(L), tt(L), rr(L);
  for (int l = 0; l < L; ++l) {
    G[l] = c.grid(H[l], nb, cs);
    const size_t v = (size_t)nb * G[l].nodes();
    if (l > 0) bb[l] = sc.take<float4>(v);
    xx[l] = sc.take<float4>(v);
    tt[l] = sc.take<float4>(v);
    rr[l] = sc.take<float4>(v);
  }
  const size_t v0 = (size_t)nb * G[0].nodes();
  mlmcp::Vecs V;
  for (int k = 0; k < 9; ++k) V.v[k] = sc.take<float4>(v0);
  float4* R = sc.take<float4>(v0);
  mlmcp::Eig E;
  E.gram = sc.take<double>((size_t)n * 2 * mlmcp::kGram);
  E.coef = sc.take<double>((size_t)n * mlmcp::kSub * mlmcp::kCols);
  E.mu = sc.take<double>((size_t)n * mlmcp::kCols);
  E.energy = sc.take<double>((size_t)n * 2);
  E.eta2 = sc.take<double>(n);
  E.active = sc.take<int>(n);
  E.iters = sc.take<int>(n);
  E.count = sc.take<int>(1);
  CK(sc.err, "alloc");
  CK(cudaMemsetAsync(E.gram, 0, sizeof(double) * n * 2 * mlmcp::kGram, st), "memset");
  CK(cudaMemsetAsync(E.mu, 0, sizeof(double) * n * mlmcp::kCols, st), "memset");
  CK(cudaMemsetAsync(E.energy, 0, sizeof(double) * n * 2, st), "memset");
  CK(cudaMemsetAsync(E.iters, 0, sizeof(int) * n, st), "memset");
  for (int k = 0; k < 9; ++k) CK(cudaMemsetAsync(V.v[k], 0, sizeof(float4) * v0, st), "memset");
  {
    std::vector<int> ones(n, 1);
    CK(cudaMemcpyAsync(E.active, ones.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st), "copy");
    CK(cudaStreamSynchronize(st), "copy");
  }
  const int* act = E.active;
  float4 *X = V.v[0], *W = V.v[1], *P = V.v[2], *KX = V.v[3], *KW = V.v[4], *KP = V.v[5], *GX = V.v[6],
         *GW = V.v[7], *GP = V.v[8];

  // patch smoother: one sweep over the nine colours (reversed: 8 .. 0) from x0 (null:
  // zero); steps 0 .. 7 alternate between the scratch buffers s1 and s2, step 8 writes
  // `last` (every step reads one buffer and writes another; x0 and last are neither s1
  // nor s2)
  auto patch_sweep = [&](int l, const float4* b, const float4* x0, float4* s1, float4* s2, bool reversed,
                         float4* last) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    const float4* in = x0;
    for (int k = 0; k < 9 && e == cudaSuccess; ++k) {
      const int col = reversed ? 8 - k : k;
      float4* o = k == 8 ? last : ((k & 1) ? s2 : s1);
      e = mlmcp::launch_patch_color(G[l], ke[l], pinv[l], false, b, in, o, col % 3, col / 3, act, st);
      in = o;
    }
    return e;
  };
  // one V(1,1) cycle with the patch smoother: out = T b0
  auto vcycle_patch = [&](const float4* b0, float4* out) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    for (int l = 0; l + 1 < L && e == cudaSuccess; ++l) {
      const float4* b = l == 0 ? b0 : bb[l];
      e = patch_sweep(l, b, nullptr, tt[l], rr[l], false, xx[l]);
      if (e == cudaSuccess) e = mlmcp::launch_apply(G[l], ke[l], xx[l], b, rr[l], nullptr, act, true, st);
      if (e == cudaSuccess) e = mlmcp::launch_restrict(G[l], G[l + 1], rr[l], bb[l + 1], act, st);
    }
    if (e != cudaSuccess) return e;
    float4* coarse_out = L == 1 ? out : xx[L - 1];
    e = mlmcp::launch_coarse_solve(G[L - 1], ainv, c.free_dev[m], nf, L == 1 ? b0 : bb[L - 1], coarse_out, act, true,
                                    st);
    for (int l = L - 2; l >= 0 && e == cudaSuccess; --l) {
      const float4* b = l == 0 ? b0 : bb[l];
      const float4* below = xx[l + 1];   // every level's post-smoothed x ends in xx
      e = mlmcp::launch_prolong(G[l], G[l + 1], below, xx[l], act, st);
      // from xx through tt and rr (free now), ending in out (level 0) or xx
      if (e == cudaSuccess) e = patch_sweep(l, b, xx[l], tt[l], rr[l], true, l == 0 ? out : xx[l]);
    }
    return e;
  };
  // one V(2,2) cycle: out = T b0 (level-0 batch entries)
  auto vcycle = [&](const float4* b0, float4* out) -> cudaError_t {
    if (patch) return vcycle_patch(b0, out);
    cudaError_t e = cudaSuccess;
    for (int l = 0; l + 1 < L && e == cudaSuccess; ++l) {
      const float4* b = l == 0 ? b0 : bb[l];
      e = mlmcp::launch_smooth(G[l], ke[l], b, nullptr, xx[l], act, st);
      if (e == cudaSuccess) e = mlmcp::launch_smooth(G[l], ke[l], b, xx[l], tt[l], act, st);
      if (e == cudaSuccess) e = mlmcp::launch_apply(G[l], ke[l], tt[l], b, rr[l], nullptr, act, true, st);
      if (e == cudaSuccess) e = mlmcp::launch_restrict(G[l], G[l + 1], rr[l], bb[l + 1], act, st);
    }
    if (e != cudaSuccess) return e;
    float4* coarse_out = L == 1 ? out : xx[L - 1];
    e = mlmcp::launch_coarse_solve(G[L - 1], ainv, c.free_dev[m], nf, L == 1 ? b0 : bb[L - 1], coarse_out, act, true,
                                    st);
    for (int l = L - 2; l >= 0 && e == cudaSuccess; --l) {
      const float4* b = l == 0 ? b0 : bb[l];
      const float4* below = (l + 1 == L - 1) ? xx[L - 1] : tt[l + 1];
      e = mlmcp::launch_prolong(G[l], G[l + 1], below, tt[l], act, st);
      if (e == cudaSuccess) e = mlmcp::launch_smooth(G[l], ke[l], b, tt[l], xx[l], act, st);
      if (e == cudaSuccess) e = mlmcp::launch_smooth(G[l], ke[l], b, xx[l], l == 0 ? out : tt[l], act, st);
    }
    return e;
  };

  // K and G images of a set of LOBPCG vectors: in double sums for thin plates (patch
  // smoother mode), where single-precision sums lose the small transverse shear strain
  auto images = [&](const float4* x, float4* kx, float4* gx) -> cudaError_t {
    return patch ? mlmcp::launch_apply64(G[0], ke64, x, kx, gx, nullptr, nullptr, act, st)
                 : mlmcp::launch_apply(G[0], ke[0], x, nullptr, kx, gx, act, true, st);
  };
  // start: X = T G Z for a fixed pseudo-random w field Z, then Rayleigh-Ritz on X
  CK(mlmcp::launch_init_start(G[0], W, st), "start");
  CK(mlmcp::launch_apply(G[0], ke[0], W, nullptr, KW, R, act, true, st), "start");
  CK(vcycle(R, X), "start");
  CK(cudaMemsetAsync(W, 0, sizeof(float4) * v0, st), "memset");
  CK(cudaMemsetAsync(KW, 0, sizeof(float4) * v0, st), "memset");
  CK(images(X, KX, GX), "apply");
  CK(mlmcp::launch_gram(G[0], E, V, st), "gram");
  CK(mlmcp::launch_rayleigh_ritz(E, n, c.tol, c.max_iter, true, st), "rayleigh-ritz");
  CK(mlmcp::launch_update(G[0], E, V, patch, st), "update");

  int it = 0;
  const int check_every = 4;
  // diagnostic: MLMC_TRACE=<k> prints sample k's Ritz values and convergence measure
  // after every iteration of this solve (synchronising each time)
  const char* trace_env = std::getenv("MLMC_TRACE");
  const int trace = trace_env ? std::atoi(trace_env) : -1;
  // one LOBPCG iteration of every active sample (launches only)
  auto iteration = [&]() -> cudaError_t {
    cudaError_t e = cudaMemsetAsync(E.count, 0, sizeof(int), st);
    // K and G images of the new X and P, recomputed (not updated by the Ritz
    // coefficients, whose single-precision drift raises the residual floor); in patch
    // mode X's images and its residual G X - mu K X come from one double-precision pass
    if (e == cudaSuccess)
      e = patch ? mlmcp::launch_apply64(G[0], ke64, X, KX, GX, R, E.mu, act, st) : images(X, KX, GX);
    if (e == cudaSuccess) e = images(P, KP, GP);
    if (e == cudaSuccess && !patch) e = mlmcp::launch_residual(G[0], E, KX, GX, R, st);
    if (e == cudaSuccess) e = vcycle(R, W);
    if (e == cudaSuccess) e = images(W, KW, GW);
    if (e == cudaSuccess) e = mlmcp::launch_gram(G[0], E, V, st);
    if (e == cudaSuccess) e = mlmcp::launch_rayleigh_ritz(E, n, c.tol, c.max_iter, false, st);
    if (e == cudaSuccess) e = mlmcp::launch_update(G[0], E, V, patch, st);
    return e;
  };
  // check_every iterations per CUDA-graph replay on a capturable stream (the samples
  // past max_iter are inactive, so a replay's last iterations cost only launches);
  // the direct loop with the trace or on the legacy default stream
  const bool graphs = st != nullptr && trace < 0;
  if (graphs) {
    if (c.lobpcg_exec.size() < (size_t)c.cfg.levels) c.lobpcg_exec.assign(c.cfg.levels, nullptr);
    cudaGraphExec_t& ex = c.lobpcg_exec[m];
    CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal), "capture");
    cudaError_t e = cudaSuccess;
    for (int k = 0; k < check_every && e == cudaSuccess; ++k) e = iteration();
    cudaGraph_t gr = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(st, &gr);
    if (e != cudaSuccess || ec != cudaSuccess) {
      if (gr) cudaGraphDestroy(gr);
      CK(e != cudaSuccess ? e : ec, "lobpcg capture");
    }
    if (ex) {
      cudaGraphExecUpdateResultInfo info;
      if (cudaGraphExecUpdate(ex, gr, &info) != cudaSuccess) {
        cudaGetLastError();
        cudaGraphExecDestroy(ex);
        ex = nullptr;
      }
    }
    if (!ex) {
      const cudaError_t ei = cudaGraphInstantiate(&ex, gr, 0);
      if (ei != cudaSuccess) ex = nullptr;
      cudaGraphDestroy(gr);
      CK(ei, "lobpcg graph");
    } else {
      cudaGraphDestroy(gr);
    }
    for (; it <= c.max_iter; it += check_every) {
      CK(cudaGraphLaunch(ex, st), "lobpcg graph");
      int h_count = 0;
      CK(cudaMemcpyAsync(&h_count, E.count, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
      CK(cudaStreamSynchronize(st), "lobpcg");
      if (h_count == 0) break;
    }
  }
  for (; !graphs && it <= c.max_iter; ++it) {
    CK(iteration(), "lobpcg");
    if (trace >= 0 && trace < n) {
      double h_mu[2], h_eta2;
      int h_act, h_it;
      CK(cudaMemcpyAsync(h_mu, E.mu + 2 * trace, sizeof(double) * 2, cudaMemcpyDeviceToHost, st), "trace");
      CK(cudaMemcpyAsync(&h_eta2, E.eta2 + trace, sizeof(double), cudaMemcpyDeviceToHost, st), "trace");
      CK(cudaMemcpyAsync(&h_act, E.active + trace, sizeof(int), cudaMemcpyDeviceToHost, st), "trace");
      CK(cudaMemcpyAsync(&h_it, E.iters + trace, sizeof(int), cudaMemcpyDeviceToHost, st), "trace");
      CK(cudaStreamSynchronize(st), "trace");
      std::fprintf(stderr, "panel trace mesh %d sample %d it %d active %d mu %.12e %.12e eta2 %.3e\n", m, trace,
                   h_it, h_act, h_mu[0], h_mu[1], h_eta2);
    }
    if ((it + 1) % check_every == 0 || it == c.max_iter) {
      int h_count = 0;
      CK(cudaMemcpyAsync(&h_count, E.count, sizeof(int), cudaMemcpyDeviceToHost, st), "copy");
      CK(cudaStreamSynchronize(st), "lobpcg");
      if (h_count == 0) break;
    }
  }
  CK(mlmcp::launch_energy(G[0], ke64, X, E, st), "energy");
  CK(mlmcp::launch_panel_qoi(E, n, c.cfg.ly, c.cfg.p_star, c.max_iter, q, status, st), "qoi");
  std::vector<int> its(n);
  CK(cudaMemcpyAsync(its.data(), E.iters, sizeof(int) * n, cudaMemcpyDeviceToHost, st), "copy");
  CK(cudaStreamSynchronize(st), "solve");
  c.last_iters = 0;
  for (int k = 0; k < n; ++k) c.last_iters = std::max(c.last_iters, std::min(its[k], c.max_iter + 1));
  return MLMC_OK;
}

template <typename U>
mlmc_status copy_out(mlmcp_ctx& c, U* dst, const U* src, size_t count) {
  if (!dst || !count) return MLMC_OK;
  CK(cudaMemcpyAsync(dst, src, sizeof(U) * count, dev_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c.st),
     "copy");
  CK(cudaStreamSynchronize(c.st), "copy");
  return MLMC_OK;
}

}  // namespace

extern "C" {

mlmc_status mlmcp_create(const mlmcp_config* cfg, void* cuda_stream, mlmcp_ctx** out) {
  if (!out) return MLMC_ERR_INVALID_ARG;
  *out = nullptr;
  auto bad = [](const char* m) {
    g_create_error_p = m;
    return MLMC_ERR_INVALID_ARG;
  };
  if (!cfg) return bad("null config");
  const mlmcp_config& k = *cfg;
  if (!(k.lx > 0) || !(k.ly > 0)) return bad("panel dimensions must be positive");
  if (k.nx0 < 1 || k.ny0 < 1 || k.nx0 > 4096 || k.ny0 > 4096) return bad("bad level-0 mesh");
  if (k.levels < 1 || k.levels > 8) return bad("levels must be 1..8");
  if ((int64_t)(k.nx0 << (k.levels - 1)) * (k.ny0 << (k.levels - 1)) > (int64_t)1 << 22)
    return bad("finest mesh too large");
  if (!(k.E11 > 0) || !(k.E22 > 0) || !(k.G12 > 0) || !(k.G13 > 0)) return bad("moduli must be positive");
  if (!(k.nu12 > -1.0) || !(k.nu12 * k.nu12 * k.E22 / k.E11 < 1.0)) return bad("bad Poisson ratio");
  if (!(k.k_shear > 0)) return bad("shear correction must be positive");
  if (k.n_plies < 1 || k.n_plies > MLMCP_MAX_PLIES) return bad("n_plies must be 1..32");
  if (!(k.t_ply > 0)) return bad("ply thickness must be positive");
  if (!(k.ply_std_deg >= 0) || !std::isfinite(k.ply_std_deg)) return bad("bad ply angle deviation");
  if (k.hard_support != 0 && k.hard_support != 1) return bad("hard_support must be 0 or 1");
  if (!(k.tol >= 0) || k.max_iter < 0) return bad("bad solver tolerances");
  for (int p = 0; p < k.n_plies; ++p)
    if (!std::isfinite(k.plies_deg[p])) return bad("bad ply angle");
  auto c = new mlmcp_ctx;
  c->cfg = k;
  c->st = static_cast<cudaStream_t>(cuda_stream);
  c->tol = k.tol > 0 ? k.tol : 1e-4;
  c->max_iter = k.max_iter > 0 ? k.max_iter : 120;
  c->lam.E11 = k.E11;
  c->lam.E22 = k.E22;
  c->lam.G12 = k.G12;
  c->lam.nu12 = k.nu12;
  c->lam.G13 = k.G13;
  c->lam.k_shear = k.k_shear;
  c->lam.t_ply = k.t_ply;
  c->lam.std_rad = k.ply_std_deg * M_PI / 180.0;
  c->lam.n_plies = k.n_plies;
  for (int p = 0; p < mlmcp::kMaxPlies; ++p) c->lam.psi[p] = p < k.n_plies ? k.plies_deg[p] * M_PI / 180.0 : 0.0;
  std::vector<std::vector<int>> frees;
  for (int m = 0; m < k.levels; ++m) {   // host checks first: nothing below runs on a bad config
    c->hier.push_back(hierarchy(k.nx0 << m, k.ny0 << m));
    frees.push_back(free_dofs(c->hier[m].back(), k.hard_support != 0));
    if (frees[m].empty() || (int)frees[m].size() > mlmcp::kMaxCoarseFree) {
      delete c;
      return bad("coarsest multigrid mesh has more than 192 free DOFs (or none)");
    }
  }
  for (int m = 0; m < k.levels; ++m) {
    const std::vector<int>& f = frees[m];
    int* d = nullptr;
    cudaError_t e = cudaMalloc(&d, sizeof(int) * f.size());
    if (e == cudaSuccess) e = cudaMemcpy(d, f.data(), sizeof(int) * f.size(), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) {
      if (d) cudaFree(d);
      g_create_error_p = std::string("create: ") + cudaGetErrorString(e);
      cudaGetLastError();
      delete c;
      return MLMC_ERR_CUDA;
    }
    c->free_dev.push_back(d);
    c->nfree.push_back((int)f.size());
  }
  c->acc_host.resize(k.levels);
  cudaError_t e = cudaMalloc(&c->acc_dev, sizeof(mlmc::LevelAcc) * k.levels);
  if (e == cudaSuccess) e = cudaMemset(c->acc_dev, 0, sizeof(mlmc::LevelAcc) * k.levels);
  if (e != cudaSuccess) {
    g_create_error_p = std::string("create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    delete c;
    return MLMC_ERR_CUDA;
  }
  *out = c;
  return MLMC_OK;
}

void mlmcp_destroy(mlmcp_ctx* h) {
  if (!h) return;
  cudaStreamSynchronize(h->st);
  delete h;
}

const char* mlmcp_last_error(const mlmcp_ctx* h) { return h ? h->err.c_str() : g_create_error_p.c_str(); }

mlmc_status mlmcp_sample_level(mlmcp_ctx* h, int32_t level, uint64_t first_id, int64_t n, double* q_fine,
                               double* q_coarse, int32_t* status) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmcp_ctx& c = *h;
  if (level < 0 || level >= c.cfg.levels) return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  if (n < 0 || n > (1 << 20)) return c.fail(MLMC_ERR_INVALID_ARG, "bad sample count");
  if (n == 0) return MLMC_OK;
  const int ni = (int)n;
  Scratch sc{c.st};
  double* xi = sc.take<double>((size_t)n * c.cfg.n_plies);
  double* qf = sc.take<double>(2 * (size_t)n);
  double* qc = sc.take<double>(2 * (size_t)n);
  int* sf = sc.take<int>(n);
  int* sco = sc.take<int>(n);
  CK(sc.err, "alloc");
  CK(cudaMemsetAsync(qc, 0, sizeof(double) * 2 * n, c.st), "memset");
  CK(cudaMemsetAsync(sco, 0, sizeof(int) * n, c.st), "memset");
  mlmc_status s = draw_xi(c, level, first_id, nullptr, nullptr, ni, xi);
  if (s == MLMC_OK) s = solve_p(c, level, ni, xi, qf, sf);
  const int it_f = c.last_iters;
  if (s == MLMC_OK && level > 0) {
    s = solve_p(c, level - 1, ni, xi, qc, sco);
    c.last_iters = std::max(it_f, c.last_iters);
  }
  if (s == MLMC_OK) {
    CK(mlmc3::launch_combine_status(sf, sco, ni, c.st), "status");
    CK(mlmc::launch_moments(qf, level > 0 ? qc : nullptr, sf, n, c.acc_dev + level, c.st), "moments");
    s = copy_out(c, q_fine, qf, 2 * (size_t)n);
    if (s == MLMC_OK) s = copy_out(c, q_coarse, qc, 2 * (size_t)n);
    if (s == MLMC_OK) s = copy_out(c, status, sf, (size_t)n);
  }
  cudaStreamSynchronize(c.st);
  return s;
}

mlmc_status mlmcp_solve_batch(mlmcp_ctx* h, const mlmc_item* items, int64_t n, double* q, int32_t* status) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmcp_ctx& c = *h;
  if (n < 0 || (n > 0 && !items)) return c.fail(MLMC_ERR_INVALID_ARG, "bad item array");
  if (n > (1 << 20)) return c.fail(MLMC_ERR_INVALID_ARG, "bad item count");
  if (n == 0) return MLMC_OK;
  std::vector<mlmc_item> it(n);
  if (dev_ptr(items)) {
    CK(cudaMemcpy(it.data(), items, sizeof(mlmc_item) * n, cudaMemcpyDeviceToHost), "items");
  } else {
    std::memcpy(it.data(), items, sizeof(mlmc_item) * n);
  }
  for (const auto& x : it)
    if (x.level < 0 || x.level >= c.cfg.levels || x.mesh_level < 0 || x.mesh_level >= c.cfg.levels)
      return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  std::vector<double> qo(2 * n, 0.0);
  std::vector<int> so(n, 0);
  int its = 0;
  for (int m = 0; m < c.cfg.levels; ++m) {
    std::vector<int> idx, lv;
    std::vector<uint64_t> ids;
    for (int64_t k = 0; k < n; ++k)
      if (it[k].mesh_level == m) {
        idx.push_back((int)k);
        lv.push_back(it[k].level);
        ids.push_back(it[k].sample_id);
      }
    if (idx.empty()) continue;
    const int ng = (int)idx.size();
    std::vector<double> qh(2 * ng);
    std::vector<int> sh(ng);
    {
      Scratch sc{c.st};
      int* lv_d = sc.take<int>(ng);
      uint64_t* ids_d = sc.take<uint64_t>(ng);
      double* xi = sc.take<double>((size_t)ng * c.cfg.n_plies);
      double* qd = sc.take<double>(2 * (size_t)ng);
      int* sd = sc.take<int>(ng);
      CK(sc.err, "alloc");
      CK(cudaMemcpyAsync(lv_d, lv.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, c.st), "copy");
      CK(cudaMemcpyAsync(ids_d, ids.data(), sizeof(uint64_t) * ng, cudaMemcpyHostToDevice, c.st), "copy");
      mlmc_status s = draw_xi(c, 0, 0, lv_d, ids_d, ng, xi);
      if (s == MLMC_OK) s = solve_p(c, m, ng, xi, qd, sd);
      if (s != MLMC_OK) return s;
      its = std::max(its, c.last_iters);
      CK(cudaMemcpyAsync(qh.data(), qd, sizeof(double) * 2 * ng, cudaMemcpyDeviceToHost, c.st), "copy");
      CK(cudaMemcpyAsync(sh.data(), sd, sizeof(int) * ng, cudaMemcpyDeviceToHost, c.st), "copy");
      CK(cudaStreamSynchronize(c.st), "solve_batch");
    }
    for (int k = 0; k < ng; ++k) {
      qo[2 * idx[k]] = qh[2 * k];
      qo[2 * idx[k] + 1] = qh[2 * k + 1];
      so[idx[k]] = sh[k];
    }
  }
  c.last_iters = its;
  if (q) {
    if (dev_ptr(q)) CK(cudaMemcpy(q, qo.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice), "copy");
    else std::memcpy(q, qo.data(), sizeof(double) * 2 * n);
  }
  if (status) {
    if (dev_ptr(status)) CK(cudaMemcpy(status, so.data(), sizeof(int) * n, cudaMemcpyHostToDevice), "copy");
    else std::memcpy(status, so.data(), sizeof(int) * n);
  }
  return MLMC_OK;
}

mlmc_status mlmcp_level_stats_get(mlmcp_ctx* h, int32_t level, mlmc_level_stats* out) {
  if (!h || !out) return MLMC_ERR_INVALID_ARG;
  mlmcp_ctx& c = *h;
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
  auto dofs = [&](int m) { return 3.0 * ((c.cfg.nx0 << m) + 1.0) * ((c.cfg.ny0 << m) + 1.0); };
  out->cost = dofs(level) + (level > 0 ? dofs(level - 1) : 0.0);
  return MLMC_OK;
}

mlmc_status mlmcp_reset_stats(mlmcp_ctx* h) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmcp_ctx& c = *h;
  CK(cudaMemsetAsync(c.acc_dev, 0, sizeof(mlmc::LevelAcc) * c.cfg.levels, c.st), "reset");
  CK(cudaStreamSynchronize(c.st), "reset");
  return MLMC_OK;
}

mlmc_status mlmcp_laminate(mlmcp_ctx* h, int32_t level, uint64_t first_id, int64_t n, double* dstar, double* kgt) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmcp_ctx& c = *h;
  if (level < 0 || level >= c.cfg.levels) return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  if (n < 0 || n > (1 << 20) || (n > 0 && !dstar)) return c.fail(MLMC_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return MLMC_OK;
  Scratch sc{c.st};
  double* xi = sc.take<double>((size_t)n * c.cfg.n_plies);
  double* ds = sc.take<double>((size_t)n * 6);
  double* kg = sc.take<double>(n);
  CK(sc.err, "alloc");
  mlmc_status s = draw_xi(c, level, first_id, nullptr, nullptr, (int)n, xi);
  if (s != MLMC_OK) return s;
  CK(mlmcp::launch_laminate(c.lam, xi, (int)n, ds, kg, c.st), "laminate");
  s = copy_out(c, dstar, ds, 6 * (size_t)n);
  if (s == MLMC_OK) s = copy_out(c, kgt, kg, (size_t)n);
  return s;
}

mlmc_status mlmcp_apply(mlmcp_ctx* h, int32_t mesh_level, int32_t level, uint64_t first_id, int64_t n, const float* x,
                        float* y, float* g) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmcp_ctx& c = *h;
  if (mesh_level < 0 || mesh_level >= c.cfg.levels || level < 0 || level >= c.cfg.levels)
    return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  if (n < 0 || n > 65535 || (n > 0 && (!x || !y))) return c.fail(MLMC_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return MLMC_OK;
  const Mesh M{c.cfg.nx0 << mesh_level, c.cfg.ny0 << mesh_level};
  const PGrid pg = c.grid(M, (int)n, 0);
  const size_t nv = (size_t)n * pg.nodes();
  Scratch sc{c.st};
  double* xi = sc.take<double>((size_t)n * c.cfg.n_plies);
  double* ds = sc.take<double>((size_t)n * 6);
  double* kg = sc.take<double>(n);
  float* ke = sc.take<float>((size_t)n * 144);
  float4* xd = sc.take<float4>(nv);
  float4* yd = sc.take<float4>(nv);
  float4* gd = sc.take<float4>(nv);
  CK(sc.err, "alloc");
  mlmc_status s = draw_xi(c, level, first_id, nullptr, nullptr, (int)n, xi);
  if (s != MLMC_OK) return s;
  CK(mlmcp::launch_laminate(c.lam, xi, (int)n, ds, kg, c.st), "laminate");
  CK(mlmcp::launch_element_matrices(ds, kg, (int)n, c.cfg.lx / M.nx, c.cfg.ly / M.ny, ke, nullptr, c.st), "element");
  CK(cudaMemcpyAsync(xd, x, sizeof(float4) * nv, dev_ptr(x) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     c.st),
     "copy");
  CK(mlmcp::launch_apply(pg, ke, xd, nullptr, yd, g ? gd : nullptr, nullptr, false, c.st), "apply");
  s = copy_out(c, reinterpret_cast<float4*>(y), yd, nv);
  if (s == MLMC_OK && g) s = copy_out(c, reinterpret_cast<float4*>(g), gd, nv);
  return s;
}

mlmc_status mlmcp_apply_bench(mlmcp_ctx* h, int32_t mesh_level, int64_t n, int32_t reps, double* ms, double* bytes) {
  if (!h || !ms || n <= 0 || n > 65535 || reps <= 0) return MLMC_ERR_INVALID_ARG;
  mlmcp_ctx& c = *h;
  if (mesh_level < 0 || mesh_level >= c.cfg.levels) return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  const Mesh M{c.cfg.nx0 << mesh_level, c.cfg.ny0 << mesh_level};
  const PGrid pg = c.grid(M, (int)n, 0);
  const size_t nv = (size_t)n * pg.nodes();
  Scratch sc{c.st};
  double* xi = sc.take<double>((size_t)n * c.cfg.n_plies);
  double* ds = sc.take<double>((size_t)n * 6);
  double* kg = sc.take<double>(n);
  float* ke = sc.take<float>((size_t)n * 144);
  float4* xd = sc.take<float4>(nv);
  float4* yd = sc.take<float4>(nv);
  float4* gd = sc.take<float4>(nv);
  CK(sc.err, "alloc");
  mlmc_status s = draw_xi(c, mesh_level, 0, nullptr, nullptr, (int)n, xi);
  if (s != MLMC_OK) return s;
  CK(mlmcp::launch_laminate(c.lam, xi, (int)n, ds, kg, c.st), "laminate");
  CK(mlmcp::launch_element_matrices(ds, kg, (int)n, c.cfg.lx / M.nx, c.cfg.ly / M.ny, ke, nullptr, c.st), "element");
  CK(cudaMemsetAsync(xd, 0, sizeof(float4) * nv, c.st), "memset");
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  CK(mlmcp::launch_apply(pg, ke, xd, nullptr, yd, gd, nullptr, false, c.st), "apply");
  CK(cudaEventRecord(e0, c.st), "event");
  for (int r = 0; r < reps; ++r) CK(mlmcp::launch_apply(pg, ke, xd, nullptr, yd, gd, nullptr, false, c.st), "apply");
  CK(cudaEventRecord(e1, c.st), "event");
  CK(cudaEventSynchronize(e1), "event");
  float t_ms = 0.f;
  CK(cudaEventElapsedTime(&t_ms, e0, e1), "event");
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  *ms = t_ms / reps;
  // per node: x read, K x and G x written (float4 each); per sample its element matrix
  if (bytes) *bytes = 48.0 * (double)nv + 576.0 * (double)n;
  CK(cudaStreamSynchronize(c.st), "apply_bench");
  return MLMC_OK;
}

mlmc_status mlmcp_last_iters(mlmcp_ctx* h, int32_t* iters) {
  if (!h || !iters) return MLMC_ERR_INVALID_ARG;
  *iters = h->last_iters;
  return MLMC_OK;
}

}  // extern "C"
