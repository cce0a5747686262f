// C ABI of the 3D fibre-waviness block (include/mlmc3d.h): context, the batched
// mixed-precision solve driver and the level-pair / moments entry points.
//
// Solve of one group (n samples on one mesh): the column angles are synthesised from
// each sample's xi (Eq. inftyKL) and expanded to (cos 2t, sin 2t, cos 4t, sin 4t);
// every coarser multigrid mesh averages its children's 4-vectors (rediscretisation
// with the averaged rotated stiffness). The FP32 PCG, preconditioned by one V(1,1)
// cycle, runs on all samples in lock step with per-sample scalars and convergence
// flags. Refinement: the iterate d is float-float; the lifting residual (FP32) starts
// the first inner solve; after its correction the residual f - K d is formed with
// float-float element arithmetic summed in double; later corrections take the inner
// CG's recursive residual. The final pass forms K d on the x = lx nodes only (the last
// element column) for the energy-consistent reaction R - (d_F . r_F) / shortening, and
// the centroid stresses.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/mlmc3d.h"
#include "engine.h"
#include "hex3d.cuh"
#include "moments.cuh"

using mlmc3::Grid3;
using mlmc3::State3;

namespace {

std::string g_create_error3;

bool dev_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Bond stress-transformation matrix of a rotation R (Voigt 11, 22, 33, 23, 13, 12):
// sigma' = M sigma, and the stiffness of a frame rotated by R is M C M^T.
void bond(const double R[3][3], double M[6][6]) {
  static const int I[6][2] = {{0, 0}, {1, 1}, {2, 2}, {1, 2}, {0, 2}, {0, 1}};
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      const int i = I[a][0], j = I[a][1], k = I[b][0], l = I[b][1];
      M[a][b] = b < 3 ? R[i][k] * R[j][l] : R[i][k] * R[j][l] + R[i][l] * R[j][k];
    }
}

bool invert6(const double A[6][6], double X[6][6]) {
  double M[6][12];
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 12; ++j) M[i][j] = j < 6 ? A[i][j] : (j - 6 == i ? 1.0 : 0.0);
  for (int p = 0; p < 6; ++p) {
    int best = p;
    for (int r = p + 1; r < 6; ++r)
      if (std::fabs(M[r][p]) > std::fabs(M[best][p])) best = r;
    if (!(std::fabs(M[best][p]) > 0.0)) return false;
    for (int j = 0; j < 12; ++j) std::swap(M[p][j], M[best][j]);
    const double d = M[p][p];
    for (int j = 0; j < 12; ++j) M[p][j] /= d;
    for (int r = 0; r < 6; ++r)
      if (r != p) {
        const double f = M[r][p];
        for (int j = 0; j < 12; ++j) M[r][j] -= f * M[p][j];
      }
  }
  for (int i = 0; i < 6; ++i)
    for (int j = 0; j < 6; ++j) X[i][j] = M[i][j + 6];
  return true;
}

// The rotated stiffness about y is a trigonometric polynomial of degree 4 in the angle
// with only even harmonics; its coefficients are the discrete Fourier sums over 8
// equally spaced angles of [0, pi). Also checks that the entries outside the 13
// monoclinic ones vanish.
bool harmonics(const mlmc3d_config& c, mlmc3::Harmonics& H, std::string& msg) {
  double S[6][6] = {};
  S[0][0] = 1 / c.E11;
  S[1][1] = 1 / c.E22;
  S[2][2] = 1 / c.E33;
  S[0][1] = S[1][0] = -c.nu12 / c.E11;
  S[0][2] = S[2][0] = -c.nu13 / c.E11;
  S[1][2] = S[2][1] = -c.nu23 / c.E22;
  S[3][3] = 1 / c.G23;
  S[4][4] = 1 / c.G13;
  S[5][5] = 1 / c.G12;
  double C[6][6];
  if (!invert6(S, C)) {
    msg = "singular ply compliance";
    return false;
  }
  static const int E[mlmc3::kEntries][2] = {{0, 0}, {0, 1}, {0, 2}, {0, 4}, {1, 1}, {1, 2}, {1, 4},
                                            {2, 2}, {2, 4}, {3, 3}, {3, 5}, {4, 4}, {5, 5}};
  double acc[6][6][5] = {};
  const int N = 8;
  double cmax = 0.0;
  for (int m = 0; m < N; ++m) {
    const double t = M_PI * m / N, ct = std::cos(t), st = std::sin(t);
    const double R[3][3] = {{ct, 0, st}, {0, 1, 0}, {-st, 0, ct}};
    double M[6][6], Cr[6][6];
    bond(R, M);
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b) {
        double v = 0;
        for (int p = 0; p < 6; ++p)
          for (int q = 0; q < 6; ++q) v += M[a][p] * C[p][q] * M[b][q];
        Cr[a][b] = v;
        cmax = std::max(cmax, std::fabs(v));
      }
    const double w[5] = {1.0 / N, 2.0 * std::cos(2 * t) / N, 2.0 * std::sin(2 * t) / N, 2.0 * std::cos(4 * t) / N,
                         2.0 * std::sin(4 * t) / N};
    for (int a = 0; a < 6; ++a)
      for (int b = 0; b < 6; ++b)
        for (int h = 0; h < 5; ++h) acc[a][b][h] += w[h] * Cr[a][b];
  }
  for (int a = 0; a < 6; ++a)
    for (int b = 0; b < 6; ++b) {
      bool mono = false;
      for (int e = 0; e < mlmc3::kEntries; ++e)
        if ((E[e][0] == a && E[e][1] == b) || (E[e][0] == b && E[e][1] == a)) mono = true;
      if (!mono)
        for (int h = 0; h < 5; ++h)
          if (std::fabs(acc[a][b][h]) > 1e-9 * cmax) {
            msg = "rotated stiffness is not monoclinic about y";
            return false;
          }
    }
  for (int e = 0; e < mlmc3::kEntries; ++e)
    for (int h = 0; h < 5; ++h) {
      H.d[e][h] = acc[E[e][0]][E[e][1]][h];
      H.f[e][h] = (float)H.d[e][h];
    }
  return true;
}

// Grow-only device arena carved with 256-byte alignment.
struct Arena {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  ~Arena() {
    if (base) cudaFree(base);
  }
  cudaError_t reserve(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (base) cudaFree(base);
    base = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&base, bytes);
    if (e == cudaSuccess) cap = bytes;
    return e;
  }
  template <typename U>
  U* take(size_t count) {
    used = (used + 255) & ~(size_t)255;
    U* p = reinterpret_cast<U*>(base + used);
    used += sizeof(U) * std::max<size_t>(count, 1);
    return p;
  }
};
struct Sizer3 {
  size_t used = 0;
  template <typename U>
  U* take(size_t count) {
    used = ((used + 255) & ~(size_t)255) + sizeof(U) * std::max<size_t>(count, 1);
    return nullptr;
  }
};

}  // namespace

struct mlmc3d_ctx {
  mlmc3d_config cfg;
  cudaStream_t st = nullptr;
  std::string err;
  mlmc3::Harmonics H;
  std::vector<float*> basis32;   // per mesh [cols][n_kl]
  mlmc::LevelAcc* acc_dev = nullptr;
  std::vector<mlmc::LevelAcc> acc_host;
  Arena ws, io, kl;   // solver workspace, per-call buffers, KL coefficients (all grow-only)
  int last_iters = 0;
  int max_iter = 200, max_outer = 8;

  mlmc_status fail(mlmc_status s, const std::string& m) {
    err = m;
    return s;
  }
  mlmc_status cuda_fail(cudaError_t e, const char* what) {
    err = std::string(what) + ": " + cudaGetErrorString(e);
    cudaGetLastError();
    return MLMC_ERR_CUDA;
  }
  Grid3 mesh(int m, int n) const {
    Grid3 g;
    g.nx = cfg.nx0 << m;
    g.ny = cfg.ny0 << m;
    g.nz = cfg.nz0 << m;
    g.nsamp = n;
    g.h = (float)(cfg.lx / g.nx);
    return g;
  }
  ~mlmc3d_ctx() {
    for (float* p : basis32) cudaFree(p);
    if (acc_dev) cudaFree(acc_dev);
  }
};

namespace {

// Multigrid meshes below mesh m: halve while every dimension is even and the mesh has
// more than kMaxCoarse3 DOFs; the last one is solved densely.
std::vector<Grid3> hierarchy(const mlmc3d_ctx& c, int m, int n) {
  std::vector<Grid3> G{c.mesh(m, n)};
  while (3 * G.back().nodes() > mlmc3::kMaxCoarse3) {
    Grid3 g = G.back();
    if (g.nx % 2 || g.ny % 2 || g.nz % 2) break;
    g.nx /= 2;
    g.ny /= 2;
    g.nz /= 2;
    g.h *= 2.f;
    G.push_back(g);
  }
  return G;
}

struct Bufs {
  std::vector<float*> trig;              // per MG level [n][cols][4]
  std::vector<float4*> dinv, b, x, t;    // per MG level (b unused at 0: r)
  float4 *r, *p, *q, *xs, *xl;           // top: residual, search direction, K p, PCG iterate, lifting
  float* d;                              // refinement iterate, float-float, 8 floats per node
  double* kd;                            // K d, 4 doubles per node
  float* ainv;
  State3 S;
  int* outer_count;
};

template <typename A>
void plan(A& a, const std::vector<Grid3>& G, int n, Bufs& B) {
  const int L = (int)G.size();
  B.trig.resize(L);
  B.dinv.resize(L);
  B.b.resize(L);
  B.x.resize(L);
  B.t.resize(L);
  for (int k = 0; k < L; ++k) {
    const size_t nv = (size_t)n * G[k].nodes();
    B.trig[k] = a.template take<float>((size_t)n * G[k].cols() * 4);
    B.dinv[k] = a.template take<float4>(nv);
    B.b[k] = k ? a.template take<float4>(nv) : nullptr;
    B.x[k] = a.template take<float4>(nv);
    B.t[k] = a.template take<float4>(nv);
  }
  const size_t nv = (size_t)n * G[0].nodes();
  B.r = a.template take<float4>(nv);
  B.p = a.template take<float4>(nv);
  B.q = a.template take<float4>(nv);
  B.xs = a.template take<float4>(nv);
  B.xl = a.template take<float4>(nv);
  B.d = a.template take<float>(8 * nv);
  B.kd = a.template take<double>(4 * nv);
  const size_t nc = 3 * (size_t)G.back().nodes();
  B.ainv = a.template take<float>((size_t)n * nc * nc);
  for (double** p : {&B.S.rz, &B.S.rz_old, &B.S.pq, &B.S.rr, &B.S.rr0, &B.S.rrf, &B.S.tol2, &B.S.alpha, &B.S.beta,
                     &B.S.react, &B.S.dr, &B.S.stress})
    *p = a.template take<double>(n);
  for (int** p : {&B.S.active, &B.S.outer_active, &B.S.iters, &B.S.status}) *p = a.template take<int>(n);
  B.S.count = a.template take<int>(8);
  B.outer_count = a.template take<int>(1);
}

#define CK(EXPR, WHAT)                           \
  do {                                           \
    const cudaError_t ck_ = (EXPR);              \
    if (ck_ != cudaSuccess) return c.cuda_fail(ck_, (WHAT)); \
  } while (0)

// n samples on mesh m with column data trig2 ([n][cols][2], device); q [n][2], status [n] (device)
mlmc_status solve3(mlmc3d_ctx& c, int m, int n, const float* trig2, double* q, int* status) {
  cudaStream_t st = c.st;
  const std::vector<Grid3> G = hierarchy(c, m, n);
  const int L = (int)G.size();
  if (3 * G.back().nodes() > mlmc3::kMaxCoarse3) return c.fail(MLMC_ERR_INVALID_ARG, "coarsest mesh too large");
  Bufs B;
  Sizer3 sz;
  plan(sz, G, n, B);
  CK(c.ws.reserve(sz.used + 256), "workspace");
  c.ws.used = 0;
  plan(c.ws, G, n, B);
  CK(cudaMemsetAsync(c.ws.base, 0, c.ws.used, st), "memset");
  const State3& S = B.S;
  // field and smoother setup
  CK(mlmc3::launch_expand_trig(trig2, (int64_t)n * G[0].cols(), B.trig[0], st), "expand_trig");
  for (int k = 0; k + 1 < L; ++k) CK(mlmc3::launch_average_trig(G[k], B.trig[k], B.trig[k + 1], st), "average_trig");
  for (int k = 0; k < L; ++k) CK(mlmc3::launch_dinv(G[k], B.trig[k], B.dinv[k], st), "dinv");
  CK(mlmc3::launch_coarsest_setup(G[L - 1], B.trig[L - 1], B.ainv, st), "coarsest_setup");
  // lifting and its residual (FP32: superseded by the first double residual)
  CK(mlmc3::launch_lift(G[0], c.cfg.shortening, B.d, B.xl, st), "lift");
  CK(mlmc3::launch_apply(G[0], B.trig[0], B.xl, B.t[0], nullptr, st), "apply");
  CK(mlmc3::launch_lift_resid(G[0], S, B.t[0], B.r, st), "lift_resid");
  {
    std::vector<int> ones(n, 1);
    CK(cudaMemcpyAsync(S.outer_active, ones.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st), "init");
    CK(cudaStreamSynchronize(st), "init");
  }
  const int64_t nv0 = (int64_t)n * G[0].nodes();
  auto vcycle = [&]() -> mlmc_status {
    CK(mlmc3::launch_smooth_first(G[0], B.dinv[0], B.r, B.x[0], B.t[0], S.active, st), "smooth");
    for (int k = 0; k + 1 < L; ++k) {
      CK(mlmc3::launch_apply(G[k], B.trig[k], B.x[k], B.t[k], S.active, st), "apply");
      const float4* bk = k ? B.b[k] : B.r;
      CK(mlmc3::launch_restrict(G[k], bk, B.t[k], G[k + 1], B.dinv[k + 1], B.b[k + 1], B.x[k + 1], B.t[k + 1],
                                S.active, st),
         "restrict");
    }
    CK(mlmc3::launch_coarsest_solve(G[L - 1], B.ainv, B.b[L - 1], B.x[L - 1], S.active, st), "coarsest");
    for (int k = L - 2; k >= 0; --k) {
      CK(mlmc3::launch_prolong(G[k], B.x[k + 1], B.x[k], B.t[k], S.active, st), "prolong");
      CK(mlmc3::launch_apply(G[k], B.trig[k], B.x[k], B.t[k], S.active, st), "apply");
      const float4* bk = k ? B.b[k] : B.r;
      CK(mlmc3::launch_post(G[k], B.dinv[k], bk, B.t[k], B.x[k], k ? nullptr : S.rz, S.active, st), "post");
    }
    return MLMC_OK;
  };
  const double floor_tol = 3e-6;
  int max_it_seen = 0;
  for (int outer = 0;; ++outer) {
    int h_outer = 0;
    CK(cudaMemsetAsync(B.outer_count, 0, sizeof(int), st), "memset");
    CK(mlmc3::launch_outer_check(S, n, c.cfg.rtol, B.outer_count, st), "outer_check");
    CK(cudaMemcpyAsync(&h_outer, B.outer_count, sizeof(int), cudaMemcpyDeviceToHost, st), "outer_count");
    CK(cudaStreamSynchronize(st), "outer_count");
    if (h_outer == 0 || outer >= c.max_outer) break;
    CK(mlmc3::launch_inner_begin(S, n, c.cfg.rtol, floor_tol, outer, st), "inner_begin");
    CK(mlmc3::launch_zero4(B.xs, nv0, st), "zero");
    CK(mlmc3::launch_zero4(B.p, nv0, st), "zero");
    int it = 0;
    while (it < c.max_iter) {
      const int batch = std::min(2, c.max_iter - it);
      CK(cudaMemsetAsync(S.count, 0, sizeof(int) * batch, st), "memset");
      for (int b = 0; b < batch; ++b, ++it) {
        const mlmc_status vs = vcycle();
        if (vs != MLMC_OK) return vs;
        CK(mlmc3::launch_beta(S, n, it == 0 ? 1 : 0, st), "beta");
        CK(mlmc3::launch_update_p(G[0], S, B.x[0], B.p, B.q, st), "update_p");
        CK(mlmc3::launch_apply(G[0], B.trig[0], B.p, B.q, S.active, st, S.pq), "apply");   // q = K p, p . q
        CK(mlmc3::launch_alpha(S, n, st), "alpha");
        CK(mlmc3::launch_update_xr(G[0], S, B.p, B.q, B.xs, B.r, st), "update_xr");
        CK(mlmc3::launch_check(S, n, it, c.max_iter, b, st), "check");
      }
      int h_count = 0;
      CK(cudaMemcpyAsync(&h_count, S.count + batch - 1, sizeof(int), cudaMemcpyDeviceToHost, st), "count");
      CK(cudaStreamSynchronize(st), "count");
      if (h_count == 0) break;
    }
    max_it_seen = std::max(max_it_seen, it);
    CK(mlmc3::launch_update_d(G[0], S, B.xs, B.d, st), "update_d");
    if (outer == 0) {   // the exact (float-float) residual after the first correction
      CK(cudaMemsetAsync(B.kd, 0, sizeof(double) * 4 * nv0, st), "memset");
      CK(cudaMemsetAsync(S.rr, 0, sizeof(double) * n, st), "memset");
      CK(mlmc3::launch_apply_df(G[0], B.trig[0], B.d, B.kd, S.outer_active, false, st), "apply_df");
      CK(mlmc3::launch_resid_exact(G[0], S, B.kd, B.r, st), "resid_exact");
    }
  }
  c.last_iters = max_it_seen;
  // final pass: K d on the x = lx nodes (last element column) for the reaction, d . r
  // with the latest residual, stresses
  CK(cudaMemsetAsync(B.kd, 0, sizeof(double) * 4 * nv0, st), "memset");
  CK(mlmc3::launch_apply_df(G[0], B.trig[0], B.d, B.kd, nullptr, true, st), "apply_df");
  CK(mlmc3::launch_final(G[0], S, B.kd, B.d, B.r, st), "final");
  CK(mlmc3::launch_stress(G[0], S, B.trig[0], B.d, c.cfg.omega_x0, c.cfg.omega_x1, st), "stress");
  CK(mlmc3::launch_qoi(S, n, c.cfg.shortening, q, status, st), "qoi");
  CK(cudaStreamSynchronize(st), "solve");
  return MLMC_OK;
}

// (cos 2t, sin 2t) per column of n samples (ids / levels per sample) on mesh m into the io arena
mlmc_status synthesize(mlmc3d_ctx& c, int m, int level, uint64_t first_id, const int* levels_dev,
                       const uint64_t* ids_dev, int n, float* out, bool trig2) {
  const int nkl = c.cfg.kl_terms;
  const Grid3 g = c.mesh(m, n);
  double* xi = nullptr;
  float* xi32 = nullptr;
  int* fail = nullptr;
  auto carve = [&](auto& a) {
    xi = a.template take<double>((size_t)n * nkl);
    xi32 = a.template take<float>((size_t)n * nkl);
    fail = a.template take<int>(2);
  };
  Sizer3 sz;
  carve(sz);
  CK(c.kl.reserve(sz.used + 256), "KL buffers");
  c.kl.used = 0;
  carve(c.kl);
  CK(cudaMemsetAsync(fail, 0, sizeof(int) * 2, c.st), "memset");
  CK(mlmc::launch_kl_coefficients(c.cfg.seed, level, first_id, levels_dev, ids_dev, n, nkl, xi, xi32, fail, c.st),
     "kl_coefficients");
  CK(mlmc::launch_kl_synthesis<float>(xi32, c.basis32[m], n, (int)g.cols(), nkl, out, trig2, c.st), "kl_synthesis");
  int h_fail = 0;
  CK(cudaMemcpyAsync(&h_fail, fail, sizeof(int), cudaMemcpyDeviceToHost, c.st), "kl");
  CK(cudaStreamSynchronize(c.st), "kl");
  if (h_fail) return c.fail(MLMC_ERR_CUDA, "normal generator exceeded its draw cap");
  return MLMC_OK;
}

template <typename U>
mlmc_status copy_out(mlmc3d_ctx& c, U* dst, const U* src, size_t count) {
  if (!dst || !count) return MLMC_OK;
  CK(cudaMemcpyAsync(dst, src, sizeof(U) * count, dev_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost,
                     c.st),
     "copy");
  CK(cudaStreamSynchronize(c.st), "copy");
  return MLMC_OK;
}

}  // namespace

extern "C" {

mlmc_status mlmc3d_create(const mlmc3d_config* cfg, void* cuda_stream, mlmc3d_ctx** out) {
  if (!cfg || !out) return MLMC_ERR_INVALID_ARG;
  *out = nullptr;
  const mlmc3d_config& c = *cfg;
  auto bad = [](const char* m) {
    g_create_error3 = m;
    return MLMC_ERR_INVALID_ARG;
  };
  if (c.levels < 1 || c.levels > 8) return bad("levels must be in [1, 8]");
  if (c.nx0 < 2 || c.ny0 < 2 || c.nz0 < 1) return bad("mesh too small");
  if (!(c.lx > 0 && c.ly > 0 && c.lz > 0)) return bad("block dimensions must be positive");
  const double h = c.lx / c.nx0;
  if (std::fabs(c.ly / c.ny0 - h) > 1e-12 * h || std::fabs(c.lz / c.nz0 - h) > 1e-12 * h)
    return bad("elements must be cubes (lx / nx0 = ly / ny0 = lz / nz0)");
  if (c.kl_terms < 1 || c.kl_terms > 512) return bad("kl_terms must be in [1, 512]");
  if (!(c.rtol > 0 && c.rtol < 1)) return bad("rtol must be in (0, 1)");
  mlmc3d_ctx* h3 = new mlmc3d_ctx();
  h3->cfg = c;
  h3->st = static_cast<cudaStream_t>(cuda_stream);
  h3->max_iter = c.max_iter > 0 ? c.max_iter : 200;
  h3->max_outer = c.max_outer > 0 ? c.max_outer : 8;
  std::string msg;
  if (!harmonics(c, h3->H, msg)) {
    delete h3;
    g_create_error3 = msg;
    return MLMC_ERR_INVALID_ARG;
  }
  for (int m = 0; m < c.levels; ++m) {
    const std::vector<Grid3> G = hierarchy(*h3, m, 1);
    if (G.size() < 2) {
      delete h3;
      return bad("mesh 0 must have more than 192 DOFs (one multigrid level below it at least)");
    }
    if (3 * G.back().nodes() > mlmc3::kMaxCoarse3) {
      delete h3;
      return bad("the mesh does not coarsen to a dense coarsest mesh of <= 192 DOFs");
    }
  }
  // the waviness field lives on the (x, z) plane: the 2D KL basis of [0, lx] x [0, lz]
  mlmc_config k2;
  std::memset(&k2, 0, sizeof(k2));
  k2.lx = c.lx;
  k2.ly = c.lz;
  k2.nx0 = c.nx0;
  k2.ny0 = c.nz0;
  k2.levels = c.levels;
  k2.kl_terms = c.kl_terms;
  k2.kl_std = c.kl_std;
  k2.kl_corr = c.kl_corr;
  k2.kl_quad = c.kl_quad;
  std::vector<mlmc::KLBasis> bases;
  if (!mlmc::build_kl_bases(k2, bases, msg)) {
    delete h3;
    g_create_error3 = msg;
    return MLMC_ERR_INVALID_ARG;
  }
  cudaError_t e = mlmc3::set_harmonics(h3->H);
  for (int m = 0; m < c.levels && e == cudaSuccess; ++m) {
    std::vector<float> b32(bases[m].B.begin(), bases[m].B.end());
    float* d = nullptr;
    e = cudaMalloc(&d, sizeof(float) * b32.size());
    if (e == cudaSuccess) e = cudaMemcpy(d, b32.data(), sizeof(float) * b32.size(), cudaMemcpyHostToDevice);
    h3->basis32.push_back(d);
  }
  if (e == cudaSuccess) e = cudaMalloc(&h3->acc_dev, sizeof(mlmc::LevelAcc) * c.levels);
  if (e == cudaSuccess) e = cudaMemset(h3->acc_dev, 0, sizeof(mlmc::LevelAcc) * c.levels);
  if (e != cudaSuccess) {
    g_create_error3 = std::string("create: ") + cudaGetErrorString(e);
    cudaGetLastError();
    delete h3;
    return MLMC_ERR_CUDA;
  }
  h3->acc_host.assign(c.levels, mlmc::LevelAcc{});
  *out = h3;
  return MLMC_OK;
}

void mlmc3d_destroy(mlmc3d_ctx* h) {
  if (h) {
    cudaStreamSynchronize(h->st);
    delete h;
  }
}

const char* mlmc3d_last_error(const mlmc3d_ctx* h) { return h ? h->err.c_str() : g_create_error3.c_str(); }

mlmc_status mlmc3d_sample_level(mlmc3d_ctx* h, int32_t level, uint64_t first_id, int64_t n, double* q_fine,
                                double* q_coarse, int32_t* status) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmc3d_ctx& c = *h;
  if (level < 0 || level >= c.cfg.levels) return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  if (n < 0 || n > (1 << 24)) return c.fail(MLMC_ERR_INVALID_ARG, "bad sample count");
  if (n == 0) return MLMC_OK;
  const int ni = (int)n;
  float* t2f = nullptr;
  float* t2c = nullptr;
  double *qf = nullptr, *qc = nullptr;
  int *sf = nullptr, *sc = nullptr;
  const Grid3 gf = c.mesh(level, ni);
  auto carve = [&](auto& a) {
    t2f = a.template take<float>(2 * gf.cols() * n);
    if (level > 0) t2c = a.template take<float>(2 * c.mesh(level - 1, ni).cols() * n);
    qf = a.template take<double>(2 * n);
    qc = a.template take<double>(2 * n);
    sf = a.template take<int>(n);
    sc = a.template take<int>(n);
  };
  Sizer3 sz;
  carve(sz);
  CK(c.io.reserve(sz.used + 256), "call buffers");
  c.io.used = 0;
  carve(c.io);
  CK(cudaMemsetAsync(qc, 0, sizeof(double) * 2 * n, c.st), "memset");
  CK(cudaMemsetAsync(sc, 0, sizeof(int) * n, c.st), "memset");
  mlmc_status s = synthesize(c, level, level, first_id, nullptr, nullptr, ni, t2f, true);
  if (s == MLMC_OK) s = solve3(c, level, ni, t2f, qf, sf);
  int it_f = c.last_iters;
  if (s == MLMC_OK && level > 0) {
    s = synthesize(c, level - 1, level, first_id, nullptr, nullptr, ni, t2c, true);
    if (s == MLMC_OK) s = solve3(c, level - 1, ni, t2c, qc, sc);
    c.last_iters = std::max(it_f, c.last_iters);
  }
  if (s == MLMC_OK) {
    CK(mlmc3::launch_combine_status(sf, sc, ni, c.st), "status");
    CK(mlmc::launch_moments(qf, level > 0 ? qc : nullptr, sf, n, c.acc_dev + level, c.st), "moments");
    s = copy_out(c, q_fine, qf, 2 * (size_t)n);
    if (s == MLMC_OK) s = copy_out(c, q_coarse, qc, 2 * (size_t)n);
    if (s == MLMC_OK) s = copy_out(c, status, sf, (size_t)n);
  }
  cudaStreamSynchronize(c.st);
  return s;
}

mlmc_status mlmc3d_solve_batch(mlmc3d_ctx* h, const mlmc_item* items, int64_t n, double* q, int32_t* status) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmc3d_ctx& c = *h;
  if (n < 0 || (n > 0 && !items)) return c.fail(MLMC_ERR_INVALID_ARG, "bad item array");
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
    const Grid3 g = c.mesh(m, ng);
    int* lv_d = nullptr;
    uint64_t* ids_d = nullptr;
    float* t2 = nullptr;
    double* qd = nullptr;
    int* sd = nullptr;
    auto carve = [&](auto& a) {
      lv_d = a.template take<int>(ng);
      ids_d = a.template take<uint64_t>(ng);
      t2 = a.template take<float>(2 * g.cols() * ng);
      qd = a.template take<double>(2 * ng);
      sd = a.template take<int>(ng);
    };
    Sizer3 sz;
    carve(sz);
    CK(c.io.reserve(sz.used + 256), "call buffers");
    c.io.used = 0;
    carve(c.io);
    CK(cudaMemcpyAsync(lv_d, lv.data(), sizeof(int) * ng, cudaMemcpyHostToDevice, c.st), "copy");
    CK(cudaMemcpyAsync(ids_d, ids.data(), sizeof(uint64_t) * ng, cudaMemcpyHostToDevice, c.st), "copy");
    mlmc_status s = synthesize(c, m, 0, 0, lv_d, ids_d, ng, t2, true);
    if (s == MLMC_OK) s = solve3(c, m, ng, t2, qd, sd);
    std::vector<double> qh(2 * ng);
    std::vector<int> sh(ng);
    if (s == MLMC_OK) {
      CK(cudaMemcpyAsync(qh.data(), qd, sizeof(double) * 2 * ng, cudaMemcpyDeviceToHost, c.st), "copy");
      CK(cudaMemcpyAsync(sh.data(), sd, sizeof(int) * ng, cudaMemcpyDeviceToHost, c.st), "copy");
    }
    CK(cudaStreamSynchronize(c.st), "solve_batch");
    if (s != MLMC_OK) return s;
    for (int k = 0; k < ng; ++k) {
      qo[2 * idx[k]] = qh[2 * k];
      qo[2 * idx[k] + 1] = qh[2 * k + 1];
      so[idx[k]] = sh[k];
    }
  }
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

mlmc_status mlmc3d_level_stats_get(mlmc3d_ctx* h, int32_t level, mlmc_level_stats* out) {
  if (!h || !out) return MLMC_ERR_INVALID_ARG;
  mlmc3d_ctx& c = *h;
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
  auto dofs = [&](int m) { return 3.0 * ((c.cfg.nx0 << m) + 1.0) * ((c.cfg.ny0 << m) + 1.0) * ((c.cfg.nz0 << m) + 1.0); };
  out->cost = dofs(level) + (level > 0 ? dofs(level - 1) : 0.0);
  return MLMC_OK;
}

mlmc_status mlmc3d_reset_stats(mlmc3d_ctx* h) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  mlmc3d_ctx& c = *h;
  CK(cudaMemsetAsync(c.acc_dev, 0, sizeof(mlmc::LevelAcc) * c.cfg.levels, c.st), "reset");
  CK(cudaStreamSynchronize(c.st), "reset");
  return MLMC_OK;
}

mlmc_status mlmc3d_theta(mlmc3d_ctx* h, int32_t mesh_level, int32_t level, uint64_t first_id, int64_t n,
                         double* theta) {
  if (!h || (n > 0 && !theta)) return MLMC_ERR_INVALID_ARG;
  mlmc3d_ctx& c = *h;
  if (level < 0 || level >= c.cfg.levels || mesh_level < 0 || mesh_level >= c.cfg.levels)
    return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  if (n <= 0) return MLMC_OK;
  const Grid3 g = c.mesh(mesh_level, (int)n);
  CK(c.io.reserve(sizeof(float) * g.cols() * n + 256), "call buffers");
  c.io.used = 0;
  float* t = c.io.take<float>(g.cols() * n);
  mlmc_status s = synthesize(c, mesh_level, level, first_id, nullptr, nullptr, (int)n, t, false);
  std::vector<float> th(g.cols() * n);
  if (s == MLMC_OK) {
    CK(cudaMemcpyAsync(th.data(), t, sizeof(float) * th.size(), cudaMemcpyDeviceToHost, c.st), "copy");
  }
  CK(cudaStreamSynchronize(c.st), "theta");
  if (s != MLMC_OK) return s;
  std::vector<double> out(th.begin(), th.end());
  if (dev_ptr(theta)) CK(cudaMemcpy(theta, out.data(), sizeof(double) * out.size(), cudaMemcpyHostToDevice), "copy");
  else std::memcpy(theta, out.data(), sizeof(double) * out.size());
  return MLMC_OK;
}

mlmc_status mlmc3d_apply(mlmc3d_ctx* h, int32_t mesh_level, int64_t n, const double* theta, const float* x,
                         float* y) {
  if (!h || (n > 0 && (!theta || !x || !y))) return MLMC_ERR_INVALID_ARG;
  mlmc3d_ctx& c = *h;
  if (mesh_level < 0 || mesh_level >= c.cfg.levels) return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  if (n <= 0) return MLMC_OK;
  const Grid3 g = c.mesh(mesh_level, (int)n);
  const size_t nc = g.cols() * n, nv = g.nodes() * n;
  double* th;
  float *t2, *t4;
  float4 *xd, *yd;
  CK(cudaMallocAsync(&th, sizeof(double) * nc, c.st), "alloc");
  CK(cudaMallocAsync(&t2, sizeof(float) * 2 * nc, c.st), "alloc");
  CK(cudaMallocAsync(&t4, sizeof(float) * 4 * nc, c.st), "alloc");
  CK(cudaMallocAsync(&xd, sizeof(float4) * nv, c.st), "alloc");
  CK(cudaMallocAsync(&yd, sizeof(float4) * nv, c.st), "alloc");
  CK(cudaMemcpyAsync(th, theta, sizeof(double) * nc, dev_ptr(theta) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice,
                     c.st),
     "copy");
  CK(cudaMemcpyAsync(xd, x, sizeof(float4) * nv, dev_ptr(x) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, c.st),
     "copy");
  CK(cudaMemsetAsync(yd, 0, sizeof(float4) * nv, c.st), "memset");
  CK(mlmc::launch_theta_to_trig2<float>(th, (int64_t)nc, t2, c.st), "trig2");
  CK(mlmc3::launch_expand_trig(t2, (int64_t)nc, t4, c.st), "expand");
  CK(mlmc3::launch_apply(g, t4, xd, yd, nullptr, c.st), "apply");
  CK(cudaMemcpyAsync(y, yd, sizeof(float4) * nv, dev_ptr(y) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, c.st),
     "copy");
  cudaFreeAsync(th, c.st);
  cudaFreeAsync(t2, c.st);
  cudaFreeAsync(t4, c.st);
  cudaFreeAsync(xd, c.st);
  cudaFreeAsync(yd, c.st);
  CK(cudaStreamSynchronize(c.st), "apply");
  return MLMC_OK;
}

mlmc_status mlmc3d_apply_bench(mlmc3d_ctx* h, int32_t mesh_level, int64_t n, int32_t reps, double* ms, double* bytes,
                               double* flops) {
  if (!h || !ms || n <= 0 || reps <= 0) return MLMC_ERR_INVALID_ARG;
  mlmc3d_ctx& c = *h;
  if (mesh_level < 0 || mesh_level >= c.cfg.levels) return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  const Grid3 g = c.mesh(mesh_level, (int)n);
  const size_t nc = g.cols() * n, nv = g.nodes() * n;
  float* t4;
  float4 *xd, *yd;
  cudaEvent_t e0, e1;
  CK(cudaMallocAsync(&t4, sizeof(float) * 4 * nc, c.st), "alloc");
  CK(cudaMallocAsync(&xd, sizeof(float4) * nv, c.st), "alloc");
  CK(cudaMallocAsync(&yd, sizeof(float4) * nv, c.st), "alloc");
  {
    std::vector<float> t(4 * nc);
    for (size_t k = 0; k < nc; ++k) {
      t[4 * k] = 1.f;   // theta = 0: (cos 2t, sin 2t, cos 4t, sin 4t) = (1, 0, 1, 0)
      t[4 * k + 1] = 0.f;
      t[4 * k + 2] = 1.f;
      t[4 * k + 3] = 0.f;
    }
    CK(cudaMemcpyAsync(t4, t.data(), sizeof(float) * t.size(), cudaMemcpyHostToDevice, c.st), "copy");
    CK(cudaStreamSynchronize(c.st), "copy");
  }
  CK(cudaMemsetAsync(xd, 0, sizeof(float4) * nv, c.st), "memset");
  CK(cudaMemsetAsync(yd, 0, sizeof(float4) * nv, c.st), "memset");
  CK(cudaEventCreate(&e0), "event");
  CK(cudaEventCreate(&e1), "event");
  CK(mlmc3::launch_apply(g, t4, xd, yd, nullptr, c.st), "apply");
  CK(cudaEventRecord(e0, c.st), "event");
  for (int r = 0; r < reps; ++r) CK(mlmc3::launch_apply(g, t4, xd, yd, nullptr, c.st), "apply");
  CK(cudaEventRecord(e1, c.st), "event");
  CK(cudaEventSynchronize(e1), "event");
  float t_ms = 0.f;
  CK(cudaEventElapsedTime(&t_ms, e0, e1), "event");
  *ms = t_ms / reps;
  if (bytes) *bytes = 32.0 * (double)nv + 16.0 * (double)nc;
  if (flops) *flops = mlmc3::kElementFlops * (double)g.elems() * (double)n;
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFreeAsync(t4, c.st);
  cudaFreeAsync(xd, c.st);
  cudaFreeAsync(yd, c.st);
  CK(cudaStreamSynchronize(c.st), "apply_bench");
  return MLMC_OK;
}

mlmc_status mlmc3d_last_iters(mlmc3d_ctx* h, int32_t* iters) {
  if (!h || !iters) return MLMC_ERR_INVALID_ARG;
  *iters = h->last_iters;
  return MLMC_OK;
}

}  // extern "C"
