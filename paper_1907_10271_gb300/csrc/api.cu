// C ABI of the level-pair engine (see include/mlmc.h for the contract).
#include <algorithm>
#include <cmath>
#include <cstring>
#include <map>
#include <numeric>
#include <string>
#include <type_traits>
#include <vector>

#include "context.h"
#include "moments.cuh"

struct mlmc_ctx {
  mlmc::Context c;
  std::vector<mlmc::LevelAcc> acc_host;
  mlmc::LevelAcc* acc_dev = nullptr;   // [levels]
  std::vector<int64_t> next_id;        // ids consumed per level by mlmc_estimate
};

namespace {

std::string g_create_error;

using mlmc::Context;

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// Copy count values of U from src (host or device) into device dst.
template <typename U>
cudaError_t to_device(U* dst, const U* src, size_t count, cudaStream_t st) {
  if (count == 0) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, sizeof(U) * count, is_device_ptr(src) ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice, st);
}

template <typename U>
cudaError_t from_device(U* dst, const U* src, size_t count, cudaStream_t st) {
  if (count == 0 || !dst) return cudaSuccess;
  return cudaMemcpyAsync(dst, src, sizeof(U) * count, is_device_ptr(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st);
}

__global__ void k_convert_d2f(const double* __restrict__ a, float* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (float)a[i];
}
__global__ void k_convert_f2d(const float* __restrict__ a, double* __restrict__ b, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) b[i] = (double)a[i];
}

cudaError_t convert(const double* a, float* b, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_convert_d2f<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}
cudaError_t convert(const float* a, double* b, int64_t n, cudaStream_t st) {
  if (n <= 0) return cudaSuccess;
  k_convert_f2d<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(a, b, n);
  return cudaGetLastError();
}

// dst[i][0 .. per) = src[i][0 .. per) for the items of a pointer table (null: skipped);
// one thread per value, item-major.
__global__ void k_copy_iterates(const double* const* src, int64_t src_stride, double* const* dst,
                                int64_t dst_stride, const double* src_base, double* dst_base, int64_t per, int n) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= per * n) return;
  const int i = (int)(t / per);
  const int64_t j = t - (int64_t)i * per;
  const double* s = src ? src[i] : src_base + (int64_t)i * src_stride;
  double* d = dst ? dst[i] : dst_base + (int64_t)i * dst_stride;
  if (s && d) d[j] = s[j];
}

__global__ void k_combine_status(const int* a, const int* b, int* out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) out[i] = a[i] != 0 ? a[i] : (b ? b[i] : 0);
}

struct LevelReq {
  int level;
  uint64_t first_id;
  int64_t n;
  int64_t out_off;   // first sample of this request in the caller's output arrays
};

struct ReqBuffers {
  double* xi;
  float* xi32;
  float* xi_tc;   // TF32 split of xi: hi [n][kp] then lo [n][kp] (tensor-core synthesis)
  void* theta_f;   // the field on the finest mesh (nested: of the phase being solved)
  void* theta_c;   // the field on the coarse mesh (single lock-stepped solve only)
  double* qf;
  double* qc;
  int* st_f;
  int* st_c;
  int* it_f;
  int* it_c;
  int* status;
};

// Device bytes the solver needs per sample of `level` (both meshes), with margin.
double bytes_per_sample(const Context& c, int level) {
  const double tb = c.mixed() ? 4.0 : 8.0;
  auto dofs = [&](int l) { return l < 0 ? 0.0 : 2.0 * ((c.cfg.nx0 << l) + 1.0) * ((c.cfg.ny0 << l) + 1.0); };
  return (dofs(level) + dofs(level - 1)) * (14.0 * tb + 16.0) * 1.4 + 64.0 * c.cfg.kl_terms + 256.0;
}

// Every level pair in `reqs`. Large calls are solved by nested iteration along each
// sample's mesh chain: phase j solves, in one lock-stepped multigrid-PCG, every sample
// whose level is at least j on mesh j (its field synthesised on mesh j from its own
// xi), starting from its phase j-1 solution prolongated to mesh j (phase 0 from the
// lifting). The sample's level-l pair takes Q_l from phase l and Q_{l-1} from phase
// l-1; the phases below l-1 only provide starting iterates, at a small fraction of
// the cost. Small calls solve the fine and coarse meshes of every pair together in
// one lock-stepped solve from the lifting (below Context::nested_min_nodes finest-mesh
// nodes the launches of a phase are too small to fill the GPU, and the sequence of
// phases costs more latency than their fewer iterations save). Either way each solve reaches
// ||f - K d|| <= rtol ||f|| on its own mesh. Then the per-level moments and outputs.
template <typename T>
mlmc_status run_level_requests(mlmc_ctx* h, const std::vector<LevelReq>& reqs, double* q_fine, double* q_coarse,
                               int32_t* status) {
  Context& c = h->c;
  cudaStream_t st = c.stream;
  const int nkl = c.cfg.kl_terms;
  const bool tc = c.kl_on_tensor_cores();
  mlmc::Sizer sz;
  int top = 0;
  int64_t fine_nodes = 0;
  for (const auto& r : reqs) {
    top = std::max(top, r.level);
    fine_nodes += r.n * c.mesh(r.level).n_nodes();
  }
  const bool nested = fine_nodes >= c.nested_min_nodes;
  std::vector<ReqBuffers> B(reqs.size());
  std::vector<double*> dA(reqs.size()), dB(reqs.size());   // iterates of alternate phases
  std::vector<double*> qs(reqs.size());                    // QoI of phases below l - 1 (unused)
  std::vector<int*> ss(reqs.size()), is(reqs.size());
  auto plan = [&](auto& alloc) {
    for (size_t k = 0; k < reqs.size(); ++k) {
      const LevelReq& r = reqs[k];
      const int64_t nel = c.mesh(r.level).n_el(), dofs = 2 * c.mesh(r.level).n_nodes();
      alloc(B[k].xi, r.n * nkl);
      alloc(B[k].xi32, c.mixed() && !tc ? r.n * nkl : 1);
      alloc(B[k].xi_tc, tc ? 2 * r.n * c.kl_kpad() : 1);
      alloc(reinterpret_cast<T*&>(B[k].theta_f), 2 * r.n * nel);
      alloc(reinterpret_cast<T*&>(B[k].theta_c), !nested && r.level > 0 ? 2 * r.n * c.mesh(r.level - 1).n_el() : 1);
      alloc(dA[k], nested && r.level > 0 ? r.n * dofs : 1);
      alloc(dB[k], nested && r.level > 1 ? r.n * dofs : 1);
      alloc(B[k].qf, 2 * r.n);
      alloc(B[k].qc, 2 * r.n);
      alloc(qs[k], 2 * r.n);
      alloc(B[k].st_f, r.n);
      alloc(B[k].st_c, r.n);
      alloc(ss[k], r.n);
      alloc(B[k].it_f, r.n);
      alloc(B[k].it_c, r.n);
      alloc(is[k], r.n);
      alloc(B[k].status, r.n);
    }
  };
  int* fail = nullptr;
  {
    auto count = [&](auto*& p, int64_t n) { sz.add<std::remove_reference_t<decltype(*p)>>((size_t)n); };
    plan(count);
    sz.add<int>(2);
  }
  cudaError_t e = c.batch_arena.reserve(sz.used + 512);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return c.fail(MLMC_ERR_OOM, "batch buffers");
  }
  c.batch_arena.reset();
  {
    auto carve = [&](auto*& p, int64_t n) { p = c.batch_arena.carve<std::remove_reference_t<decltype(*p)>>((size_t)n); };
    plan(carve);
    fail = c.batch_arena.carve<int>(2);   // [0] normal generator cap, [1] tensor-core synthesis wait
  }
  if ((e = cudaMemsetAsync(fail, 0, 2 * sizeof(int), st)) != cudaSuccess) return c.cuda_fail(e, "memset");
  // KL coefficients once per request, shared by all of its meshes
  std::vector<mlmc::KlTcOperand> xop(reqs.size());
  for (size_t k = 0; k < reqs.size(); ++k) {
    const LevelReq& r = reqs[k];
    c.timer.begin(mlmc::kProfOther, st, "kl_coefficients");
    e = mlmc::launch_kl_coefficients(c.cfg.seed, r.level, r.first_id, nullptr, nullptr, r.n, nkl, B[k].xi,
                                     c.mixed() && !tc ? B[k].xi32 : nullptr, fail, st);
    c.timer.end(st);
    if (e != cudaSuccess) return c.cuda_fail(e, "kl_coefficients");
    if (tc) {
      const int kp = c.kl_kpad();
      c.timer.begin(mlmc::kProfOther, st, "kl_split");
      e = mlmc::launch_tf32_split(B[k].xi, r.n, nkl, kp, B[k].xi_tc, B[k].xi_tc + r.n * kp, st);
      c.timer.end(st);
      if (e == cudaSuccess)
        e = mlmc::make_kl_tc_operand(B[k].xi_tc, B[k].xi_tc + r.n * kp, r.n, kp, mlmc::kKlTcSamples, &xop[k]);
      if (e != cudaSuccess) return c.cuda_fail(e, "kl_split");
    }
  }
  auto synthesize = [&](size_t k, int m, T* th) -> cudaError_t {
    const LevelReq& r = reqs[k];
    c.timer.begin(mlmc::kProfOther, st, "kl_synthesis");
    cudaError_t err;
    if (tc) {
      err = mlmc::launch_kl_synthesis_tc(c.basis_tc_op[m], xop[k], (int)c.mesh(m).n_el(), r.n, (float*)(void*)th, true,
                                         fail + 1, st);
    } else {
      const T* xiT = c.mixed() ? (const T*)(const void*)B[k].xi32 : (const T*)(const void*)B[k].xi;
      const T* basis = c.mixed() ? (const T*)(const void*)c.basis32[m] : (const T*)(const void*)c.basis64[m];
      err = mlmc::launch_kl_synthesis<T>(xiT, basis, r.n, (int)c.mesh(m).n_el(), nkl, th, true, st);
    }
    c.timer.end(st);
    return err;
  };
  auto check_fail = [&]() -> mlmc_status {
    int h_fail[2] = {0, 0};
    cudaError_t err;
    if ((err = cudaMemcpyAsync(h_fail, fail, 2 * sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (err = cudaStreamSynchronize(st)) != cudaSuccess)
      return c.cuda_fail(err, "kl_coefficients");
    if (h_fail[0]) return c.fail(MLMC_ERR_CUDA, "normal generator exceeded its draw cap");
    if (h_fail[1]) return c.fail(MLMC_ERR_TIMEOUT, "tensor-core KL synthesis: a wait expired");
    return MLMC_OK;
  };
  if (!nested) {
    std::vector<mlmc::SolveGroup<T>> groups;
    for (size_t k = 0; k < reqs.size(); ++k) {
      const LevelReq& r = reqs[k];
      if ((e = synthesize(k, r.level, (T*)B[k].theta_f)) != cudaSuccess) return c.cuda_fail(e, "kl_synthesis");
      groups.push_back({r.level, r.n, (T*)B[k].theta_f, B[k].qf, B[k].st_f, B[k].it_f});
      if (r.level > 0) {
        if ((e = synthesize(k, r.level - 1, (T*)B[k].theta_c)) != cudaSuccess) return c.cuda_fail(e, "kl_synthesis");
        groups.push_back({r.level - 1, r.n, (T*)B[k].theta_c, B[k].qc, B[k].st_c, B[k].it_c});
      }
    }
    mlmc_status s = check_fail();
    if (s == MLMC_OK) s = mlmc::solve_groups<T>(c, groups);
    if (s != MLMC_OK) return s;
  }
  for (int j = 0; nested && j <= top; ++j) {
    std::vector<mlmc::SolveGroup<T>> groups;
    for (size_t k = 0; k < reqs.size(); ++k) {
      const LevelReq& r = reqs[k];
      if (r.level < j) continue;
      T* th = (T*)B[k].theta_f;
      if ((e = synthesize(k, j, th)) != cudaSuccess) return c.cuda_fail(e, "kl_synthesis");
      mlmc::SolveGroup<T> g{j, r.n, th, qs[k], ss[k], is[k]};
      if (j == r.level) g = mlmc::SolveGroup<T>{j, r.n, th, B[k].qf, B[k].st_f, B[k].it_f};
      if (j + 1 == r.level) g = mlmc::SolveGroup<T>{j, r.n, th, B[k].qc, B[k].st_c, B[k].it_c};
      double* prev = (j & 1) ? dA[k] : dB[k];   // written by phase j - 1
      double* cur = (j & 1) ? dB[k] : dA[k];
      g.d_guess = j > 0 ? prev : nullptr;
      g.d_out = j < r.level ? cur : nullptr;
      groups.push_back(g);
    }
    mlmc_status s = check_fail();
    if (s == MLMC_OK) s = mlmc::solve_groups<T>(c, groups);
    if (s != MLMC_OK) return s;
  }
  for (size_t k = 0; k < reqs.size(); ++k) {
    const LevelReq& r = reqs[k];
    const int64_t nb = r.n;
    c.timer.begin(mlmc::kProfOther, st, "combine_status");
    k_combine_status<<<(unsigned)((nb + 255) / 256), 256, 0, st>>>(B[k].st_f, r.level > 0 ? B[k].st_c : nullptr,
                                                                  B[k].status, nb);
    c.timer.end(st);
    if ((e = cudaGetLastError()) != cudaSuccess) return c.cuda_fail(e, "status");
    if (r.level == 0 && (e = cudaMemsetAsync(B[k].qc, 0, sizeof(double) * 2 * nb, st)) != cudaSuccess)
      return c.cuda_fail(e, "memset");
    c.timer.begin(mlmc::kProfOther, st, "moments");
    e = mlmc::launch_moments(B[k].qf, r.level > 0 ? B[k].qc : nullptr, B[k].status, nb, h->acc_dev + r.level, st);
    c.timer.end(st);
    if (e != cudaSuccess) return c.cuda_fail(e, "moments");
    if ((e = from_device(q_fine ? q_fine + 2 * r.out_off : nullptr, B[k].qf, 2 * nb, st)) != cudaSuccess ||
        (e = from_device(q_coarse ? q_coarse + 2 * r.out_off : nullptr, B[k].qc, 2 * nb, st)) != cudaSuccess ||
        (e = from_device(status ? status + r.out_off : nullptr, B[k].status, nb, st)) != cudaSuccess)
      return c.cuda_fail(e, "copy out");
  }
  if ((e = cudaStreamSynchronize(st)) != cudaSuccess) return c.cuda_fail(e, "sample_levels");
  return MLMC_OK;
}

// Splits the requests into solves that fit the memory budget and mesh-group limit.
mlmc_status sample_levels_impl(mlmc_ctx* h, std::vector<LevelReq> reqs, double* q_fine, double* q_coarse,
                               int32_t* status) {
  Context& c = h->c;
  // one lock-stepped solve for as much of the request as half the free device memory
  // holds (at most 64 GB), unless the caller fixed the batch size
  double budget = 8.0e9;
  {
    size_t free_b = 0, total_b = 0;
    if (cudaMemGetInfo(&free_b, &total_b) == cudaSuccess)
      budget = std::min(64.0e9, std::max(budget, 0.5 * (double)(free_b + c.solve_arena.cap + c.batch_arena.cap)));
    else
      cudaGetLastError();
  }
  if (c.cfg.max_batch > 0) budget = 1e300;
  // cut requests larger than the budget (or than max_batch) into pieces
  std::vector<LevelReq> pieces;
  for (const auto& r : reqs) {
    int64_t cap = c.cfg.max_batch > 0 ? c.cfg.max_batch
                                      : std::max<int64_t>(1, (int64_t)(budget / bytes_per_sample(c, r.level)));
    for (int64_t off = 0; off < r.n; off += cap)
      pieces.push_back(LevelReq{r.level, r.first_id + (uint64_t)off, std::min(cap, r.n - off), r.out_off + off});
  }
  size_t i = 0;
  while (i < pieces.size()) {
    std::vector<LevelReq> solve;
    double bytes = 0;
    int groups = 0;
    while (i < pieces.size()) {
      const LevelReq& r = pieces[i];
      const double b = bytes_per_sample(c, r.level) * r.n;
      const int g = r.level > 0 ? 2 : 1;
      if (!solve.empty() && (bytes + b > budget || groups + g > mlmc::kMaxViews)) break;
      bool dup = false;   // one request per level per solve keeps the moment order simple
      for (const auto& x : solve) dup = dup || x.level == r.level;
      if (dup) break;
      solve.push_back(r);
      bytes += b;
      groups += g;
      ++i;
    }
    mlmc_status s = c.mixed() ? run_level_requests<float>(h, solve, q_fine, q_coarse, status)
                              : run_level_requests<double>(h, solve, q_fine, q_coarse, status);
    if (s != MLMC_OK) return s;
  }
  return MLMC_OK;
}

mlmc_status sync_stats(mlmc_ctx* h) {
  Context& c = h->c;
  cudaError_t e = cudaMemcpyAsync(h->acc_host.data(), h->acc_dev, sizeof(mlmc::LevelAcc) * h->acc_host.size(),
                                  cudaMemcpyDeviceToHost, c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(c.stream);
  return e == cudaSuccess ? MLMC_OK : c.cuda_fail(e, "stats");
}

double level_cost(const Context& c, int l) {
  auto dofs = [&](int m) { return 2.0 * ((c.cfg.nx0 << m) + 1.0) * ((c.cfg.ny0 << m) + 1.0); };
  const double g = c.cfg.mlmc_gamma > 0 ? c.cfg.mlmc_gamma : 1.0;
  double cost = std::pow(dofs(l), g);
  if (l > 0) cost += std::pow(dofs(l - 1), g);
  return cost;
}

void fill_stats(const mlmc_ctx* h, int l, mlmc_level_stats* out) {
  const mlmc::LevelAcc& a = h->acc_host[l];
  std::memset(out, 0, sizeof(*out));
  out->n = a.n;
  for (int k = 0; k < 2; ++k) {
    out->mean[k] = a.mean[k];
    out->m2[k] = a.m2[k];
    out->var[k] = a.n > 0 ? a.m2[k] / (double)a.n : 0.0;
    out->sum_qf[k] = a.sum_qf[k] - a.comp_qf[k];
    out->sum_qc[k] = a.sum_qc[k] - a.comp_qc[k];
  }
  out->cost = level_cost(h->c, l);
}

}  // namespace

namespace mlmc {

Invariants invariants(const mlmc_config& c, bool& ok) {
  // plane-strain fibre-frame stiffness: (1,2) block of the inverse 3D normal compliance
  double S[3][3] = {{1.0 / c.E11, -c.nu12 / c.E11, -c.nu13 / c.E11},
                    {-c.nu12 / c.E11, 1.0 / c.E22, -c.nu23 / c.E22},
                    {-c.nu13 / c.E11, -c.nu23 / c.E22, 1.0 / c.E33}};
  // inverse by cofactors
  const double det = S[0][0] * (S[1][1] * S[2][2] - S[1][2] * S[2][1]) -
                     S[0][1] * (S[1][0] * S[2][2] - S[1][2] * S[2][0]) +
                     S[0][2] * (S[1][0] * S[2][1] - S[1][1] * S[2][0]);
  ok = std::isfinite(det) && det > 0.0;
  const double Q11 = (S[1][1] * S[2][2] - S[1][2] * S[2][1]) / det;
  const double Q12 = -(S[0][1] * S[2][2] - S[0][2] * S[2][1]) / det;
  const double Q22 = (S[0][0] * S[2][2] - S[0][2] * S[2][0]) / det;
  const double Q66 = c.G12;
  ok = ok && Q11 > 0 && Q22 > 0 && Q66 > 0 && Q11 * Q22 > Q12 * Q12;
  Invariants U;
  U.U1 = (3.0 * Q11 + 3.0 * Q22 + 2.0 * Q12 + 4.0 * Q66) / 8.0;
  U.U2 = (Q11 - Q22) / 2.0;
  U.U3 = (Q11 + Q22 - 2.0 * Q12 - 4.0 * Q66) / 8.0;
  U.U4 = (Q11 + Q22 + 6.0 * Q12 - 4.0 * Q66) / 8.0;
  U.U5 = (Q11 + Q22 - 2.0 * Q12 + 4.0 * Q66) / 8.0;
  U.round_single();
  return U;
}

std::string validate(const mlmc_config& c) {
  if (!(c.lx > 0 && c.ly > 0)) return "lx, ly must be positive";
  if (c.nx0 < 2 || c.ny0 < 2) return "nx0, ny0 must be >= 2";
  if (c.levels < 1 || c.levels > 12) return "levels must be in [1, 12]";
  if ((int64_t)(c.nx0 << (c.levels - 1)) > (1 << 16) || (int64_t)(c.ny0 << (c.levels - 1)) > (1 << 16))
    return "finest mesh too large";
  if (c.kl_terms < 1 || c.kl_terms > 512) return "kl_terms must be in [1, 512]";
  if (!(c.kl_std >= 0) || !(c.kl_corr > 0)) return "kl_std >= 0 and kl_corr > 0 required";
  if (!(c.rtol > 0 && c.rtol < 1)) return "rtol must be in (0, 1)";
  if (c.precision != MLMC_PREC_FP64 && c.precision != MLMC_PREC_MIXED) return "unknown precision";
  if (!(c.E11 > 0 && c.E22 > 0 && c.E33 > 0 && c.G12 > 0)) return "moduli must be positive";
  // the multigrid hierarchy halves the level-0 mesh down to <= 64 DOFs
  int nx = c.nx0, ny = c.ny0;
  while (nx % 2 == 0 && ny % 2 == 0 && ny >= 2) {
    nx /= 2;
    ny /= 2;
  }
  if (nx == c.nx0) return "level-0 mesh must halve at least once (nx0, ny0 even)";
  if (2 * (nx + 1) * (ny + 1) > kMaxCoarsestDofs) return "level-0 mesh does not halve down to <= 64 DOFs";
  return "";
}

mlmc_status reserve_workspace(mlmc_ctx* h, size_t solve_bytes, size_t batch_bytes) {
  Context& c = h->c;
  cudaError_t e = c.solve_arena.reserve(solve_bytes);
  if (e == cudaSuccess) e = c.batch_arena.reserve(batch_bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return c.fail(MLMC_ERR_OOM, "workspace reservation failed");
  }
  return MLMC_OK;
}

void set_graph_replay(mlmc_ctx* h, bool on) { h->c.graphs = on; }

int64_t iterate_values(const mlmc_config& cfg, int m) {
  return 2 * (((int64_t)cfg.nx0 << m) + 1) * (((int64_t)cfg.ny0 << m) + 1);
}

mlmc_status solve_batch_carry(mlmc_ctx* h, const mlmc_item* items, int64_t n, double* q, int32_t* status,
                              const double* const* guess, double* const* out, int32_t* iters) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  if (n < 0 || (n > 0 && !items)) return c.fail(MLMC_ERR_INVALID_ARG, "bad item array");
  if (n == 0) return MLMC_OK;
  std::vector<mlmc_item> it(n);
  if (is_device_ptr(items)) {
    cudaMemcpy(it.data(), items, sizeof(mlmc_item) * n, cudaMemcpyDeviceToHost);
  } else {
    std::memcpy(it.data(), items, sizeof(mlmc_item) * n);
  }
  for (int64_t k = 0; k < n; ++k) {
    const auto& x = it[k];
    if (x.level < 0 || x.level >= c.cfg.levels || x.mesh_level < 0 || x.mesh_level >= c.cfg.levels)
      return c.fail(MLMC_ERR_INVALID_ARG, "item level out of range");
    if (guess && guess[k] && x.mesh_level == 0)
      return c.fail(MLMC_ERR_INVALID_ARG, "an initial iterate for a mesh-0 item (no coarser mesh)");
  }
  auto has_guess = [&](int64_t k) { return guess && guess[k] ? 1 : 0; };
  // groups: items of one mesh, those with initial iterates apart, stable order
  std::vector<int64_t> order(n);
  std::iota(order.begin(), order.end(), 0);
  std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
    if (it[a].mesh_level != it[b].mesh_level) return it[a].mesh_level < it[b].mesh_level;
    return has_guess(a) < has_guess(b);
  });
  struct Run {
    int64_t k0, k1;
    int mesh;
    bool guessed, outs;
  };
  std::vector<Run> runs;
  for (int64_t k = 0; k < n;) {
    const int m = it[order[k]].mesh_level, gflag = has_guess(order[k]);
    int64_t k1 = k;
    bool outs = false;
    while (k1 < n && it[order[k1]].mesh_level == m && has_guess(order[k1]) == gflag) {
      outs = outs || (out && out[order[k1]]);
      ++k1;
    }
    runs.push_back(Run{k, k1, m, gflag != 0, outs});
    k = k1;
  }
  std::vector<int> lv(n);
  std::vector<uint64_t> ids(n);
  for (int64_t k = 0; k < n; ++k) {
    lv[k] = it[order[k]].level;
    ids[k] = it[order[k]].sample_id;
  }
  const bool mixed = c.mixed();
  const size_t tb = mixed ? 4 : 8;
  int64_t nel_total = 0, carry_values = 0;
  for (int64_t k = 0; k < n; ++k) nel_total += c.mesh(it[order[k]].mesh_level).n_el();
  for (const Run& r : runs) {
    if (r.guessed) carry_values += (r.k1 - r.k0) * iterate_values(c.cfg, r.mesh - 1);
    if (r.outs) carry_values += (r.k1 - r.k0) * iterate_values(c.cfg, r.mesh);
  }
  const bool tc = c.kl_on_tensor_cores();
  const int kp = c.kl_kpad();
  mlmc::Sizer sz;
  sz.add<double>(n * c.cfg.kl_terms);
  sz.add<float>(n * c.cfg.kl_terms);
  sz.add<float>(tc ? 2 * n * kp : 1);
  sz.add<int>(2);
  sz.add<int>(n);
  sz.add<uint64_t>(n);
  sz.add<char>(2 * nel_total * tb);
  sz.add<double>(2 * n);
  sz.add<int>(n);
  sz.add<int>(n);
  sz.add<double>(carry_values);
  sz.add<const double*>(2 * n);
  cudaError_t e = c.batch_arena.reserve(sz.used + 256);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return c.fail(MLMC_ERR_OOM, "batch buffers");
  }
  c.batch_arena.reset();
  double* xi = c.batch_arena.carve<double>(n * c.cfg.kl_terms);
  float* xi32 = c.batch_arena.carve<float>(n * c.cfg.kl_terms);
  float* xi_tc = c.batch_arena.carve<float>(tc ? 2 * n * kp : 1);
  int* fail = c.batch_arena.carve<int>(2);
  int* lv_dev = c.batch_arena.carve<int>(n);
  uint64_t* id_dev = c.batch_arena.carve<uint64_t>(n);
  char* theta = c.batch_arena.carve<char>(2 * nel_total * tb);
  double* qd = c.batch_arena.carve<double>(2 * n);
  int* sd = c.batch_arena.carve<int>(n);
  int* itd = c.batch_arena.carve<int>(n);
  double* carry = c.batch_arena.carve<double>(carry_values);
  const double** ptr_dev = c.batch_arena.carve<const double*>(2 * n);   // [guess (sorted) | out (sorted)]
  cudaStream_t st = c.stream;
  if ((e = cudaMemcpyAsync(lv_dev, lv.data(), sizeof(int) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(id_dev, ids.data(), sizeof(uint64_t) * n, cudaMemcpyHostToDevice, st)) != cudaSuccess ||
      (e = cudaMemsetAsync(fail, 0, 2 * sizeof(int), st)) != cudaSuccess)
    return c.cuda_fail(e, "items");
  // initial iterates into one buffer per guessed group (a copy kernel over a pointer table)
  std::vector<double*> run_guess(runs.size(), nullptr), run_out(runs.size(), nullptr);
  if (carry_values > 0) {
    std::vector<const double*> ptrs(2 * n, nullptr);
    for (int64_t k = 0; k < n; ++k) {
      ptrs[k] = guess ? guess[order[k]] : nullptr;
      ptrs[n + k] = out ? out[order[k]] : nullptr;
    }
    if ((e = cudaMemcpyAsync(ptr_dev, ptrs.data(), sizeof(const double*) * 2 * n, cudaMemcpyHostToDevice, st)) !=
        cudaSuccess)
      return c.cuda_fail(e, "iterate table");
    double* p = carry;
    for (size_t r = 0; r < runs.size(); ++r) {
      const Run& R = runs[r];
      const int nb = (int)(R.k1 - R.k0);
      if (R.guessed) {
        const int64_t per = iterate_values(c.cfg, R.mesh - 1);
        run_guess[r] = p;
        c.timer.begin(mlmc::kProfOther, st, "carry_in");
        k_copy_iterates<<<(unsigned)((per * nb + 255) / 256), 256, 0, st>>>(ptr_dev + R.k0, 0, nullptr, per, nullptr,
                                                                          p, per, nb);
        c.timer.end(st);
        if ((e = cudaGetLastError()) != cudaSuccess) return c.cuda_fail(e, "carry_in");
        p += per * nb;
      }
      if (R.outs) {
        run_out[r] = p;
        p += iterate_values(c.cfg, R.mesh) * nb;
      }
    }
  }
  if ((e = mlmc::launch_kl_coefficients(c.cfg.seed, 0, 0, lv_dev, id_dev, n, c.cfg.kl_terms, xi,
                                        mixed && !tc ? xi32 : nullptr, fail, st)) != cudaSuccess)
    return c.cuda_fail(e, "kl_coefficients");
  if (tc && (e = mlmc::launch_tf32_split(xi, n, c.cfg.kl_terms, kp, xi_tc, xi_tc + n * kp, st)) != cudaSuccess)
    return c.cuda_fail(e, "kl_split");
  auto run = [&](auto tag) -> mlmc_status {
    using T = decltype(tag);
    std::vector<mlmc::SolveGroup<T>> groups;
    const T* xiT = mixed ? (const T*)(const void*)xi32 : (const T*)(const void*)xi;
    int64_t eoff = 0;
    for (size_t r = 0; r < runs.size(); ++r) {
      const Run& R = runs[r];
      const int m = R.mesh;
      const int64_t k = R.k0, nb = R.k1 - R.k0;
      const int64_t nel = c.mesh(m).n_el();
      T* th = reinterpret_cast<T*>(theta) + eoff;
      const T* B = mixed ? (const T*)(const void*)c.basis32[m] : (const T*)(const void*)c.basis64[m];
      cudaError_t err;
      if (tc) {
        mlmc::KlTcOperand xop;
        err = mlmc::make_kl_tc_operand(xi_tc + k * kp, xi_tc + (n + k) * kp, nb, kp, mlmc::kKlTcSamples, &xop);
        if (err == cudaSuccess)
          err = mlmc::launch_kl_synthesis_tc(c.basis_tc_op[m], xop, (int)nel, nb, (float*)(void*)th, true, fail + 1,
                                             st);
      } else {
        err = mlmc::launch_kl_synthesis<T>(xiT + k * c.cfg.kl_terms, B, nb, (int)nel, c.cfg.kl_terms, th, true, st);
      }
      if (err != cudaSuccess) return c.cuda_fail(err, "kl_synthesis");
      mlmc::SolveGroup<T> g{m, nb, th, qd + 2 * k, sd + k, itd + k};
      g.d_guess = run_guess[r];
      g.d_out = run_out[r];
      groups.push_back(g);
      eoff += 2 * nb * nel;
    }
    int h_err = 0;
    cudaError_t err;
    if ((err = cudaMemcpyAsync(&h_err, fail + 1, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (err = cudaStreamSynchronize(st)) != cudaSuccess)
      return c.cuda_fail(err, "kl_synthesis");
    if (h_err) return c.fail(MLMC_ERR_TIMEOUT, "tensor-core KL synthesis: a wait expired");
    // at most kMaxViews groups per lock-stepped solve
    for (size_t g0 = 0; g0 < groups.size(); g0 += kMaxViews) {
      std::vector<mlmc::SolveGroup<T>> part(groups.begin() + g0,
                                            groups.begin() + std::min(groups.size(), g0 + (size_t)kMaxViews));
      const mlmc_status ps = mlmc::solve_groups<T>(c, part);
      if (ps != MLMC_OK) return ps;
    }
    return MLMC_OK;
  };
  mlmc_status s = mixed ? run(float()) : run(double());
  if (s != MLMC_OK) return s;
  // final iterates to the items' own storage
  for (size_t r = 0; r < runs.size(); ++r) {
    const Run& R = runs[r];
    if (!R.outs) continue;
    const int64_t per = iterate_values(c.cfg, R.mesh);
    const int nb = (int)(R.k1 - R.k0);
    c.timer.begin(mlmc::kProfOther, st, "carry_out");
    k_copy_iterates<<<(unsigned)((per * nb + 255) / 256), 256, 0, st>>>(nullptr, per, const_cast<double* const*>(
                                                                             ptr_dev + n + R.k0), 0, run_out[r],
                                                                       nullptr, per, nb);
    c.timer.end(st);
    if ((e = cudaGetLastError()) != cudaSuccess) return c.cuda_fail(e, "carry_out");
  }
  // scatter back to item order
  std::vector<double> qh(2 * n), qo(2 * n);
  std::vector<int> sh(n), so(n), ih(n);
  if ((e = cudaMemcpyAsync(qh.data(), qd, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(sh.data(), sd, sizeof(int) * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaMemcpyAsync(ih.data(), itd, sizeof(int) * n, cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
      (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return c.cuda_fail(e, "copy out");
  for (int64_t k = 0; k < n; ++k) {
    qo[2 * order[k]] = qh[2 * k];
    qo[2 * order[k] + 1] = qh[2 * k + 1];
    so[order[k]] = sh[k];
    if (iters) iters[order[k]] = ih[k];
  }
  if (q) {
    if (is_device_ptr(q)) e = cudaMemcpy(q, qo.data(), sizeof(double) * 2 * n, cudaMemcpyHostToDevice);
    else std::memcpy(q, qo.data(), sizeof(double) * 2 * n);
  }
  if (status) {
    if (is_device_ptr(status)) e = cudaMemcpy(status, so.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
    else std::memcpy(status, so.data(), sizeof(int) * n);
  }
  return e == cudaSuccess ? MLMC_OK : c.cuda_fail(e, "copy out");
}

double solve_bytes_per_sample(const mlmc_config& cfg, int mesh) {
  const double tb = cfg.precision == MLMC_PREC_MIXED ? 4.0 : 8.0;
  const double nx = (double)((int64_t)cfg.nx0 << mesh), ny = (double)((int64_t)cfg.ny0 << mesh);
  const double dofs = 2.0 * (nx + 1.0) * (ny + 1.0);
  // plus the carried iterates of a served escalation (its previous mesh's and its own)
  return dofs * (14.0 * tb + 16.0) * 1.4 + 2.0 * nx * ny * tb + 96.0 * cfg.kl_terms + 512.0 + 1.25 * 8.0 * dofs + 16.0;
}

}  // namespace mlmc

extern "C" {

mlmc_status mlmc_create(const mlmc_config* cfg, void* cuda_stream, mlmc_ctx** out) {
  if (!cfg || !out) {
    g_create_error = "null argument";
    return MLMC_ERR_INVALID_ARG;
  }
  *out = nullptr;
  std::string v = mlmc::validate(*cfg);
  if (!v.empty()) {
    g_create_error = v;
    return MLMC_ERR_INVALID_ARG;
  }
  bool ok = true;
  mlmc::Invariants U = mlmc::invariants(*cfg, ok);
  if (!ok) {
    g_create_error = "material constants do not give a positive definite plane-strain stiffness";
    return MLMC_ERR_INVALID_ARG;
  }
  int dev_count = 0;
  if (cudaGetDeviceCount(&dev_count) != cudaSuccess || dev_count == 0) {
    cudaGetLastError();
    g_create_error = "no CUDA device";
    return MLMC_ERR_CUDA;
  }
  mlmc_ctx* h = new mlmc_ctx();
  Context& c = h->c;
  c.cfg = *cfg;
  c.U = U;
  c.stream = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&c.device);
  std::string msg;
  if (!mlmc::build_kl_bases(c.cfg, c.bases_host, msg)) {
    g_create_error = msg;
    delete h;
    return MLMC_ERR_INVALID_ARG;
  }
  for (int l = 0; l < c.cfg.levels; ++l) {
    const std::vector<double>& B = c.bases_host[l].B;
    double* d64 = nullptr;
    float* d32 = nullptr;
    if (cudaMalloc(&d64, sizeof(double) * B.size()) != cudaSuccess ||
        cudaMalloc(&d32, sizeof(float) * B.size()) != cudaSuccess) {
      cudaGetLastError();
      g_create_error = "basis allocation failed";
      if (d64) cudaFree(d64);
      for (auto p : c.basis64) cudaFree(p);
      for (auto p : c.basis32) cudaFree(p);
      delete h;
      return MLMC_ERR_OOM;
    }
    std::vector<float> B32(B.begin(), B.end());
    cudaMemcpy(d64, B.data(), sizeof(double) * B.size(), cudaMemcpyHostToDevice);
    cudaMemcpy(d32, B32.data(), sizeof(float) * B.size(), cudaMemcpyHostToDevice);
    c.basis64.push_back(d64);
    c.basis32.push_back(d32);
    if (c.kl_on_tensor_cores()) {
      const int kp = c.kl_kpad();
      const int64_t rows = (int64_t)c.bases_host[l].nx * c.bases_host[l].ny;
      std::vector<float> split(2 * (size_t)rows * kp);
      mlmc::tf32_split_host(B.data(), rows, c.cfg.kl_terms, kp, split.data(), split.data() + rows * kp);
      float* dtc = nullptr;
      mlmc::KlTcOperand op;
      cudaError_t e = cudaMalloc(&dtc, sizeof(float) * split.size());
      if (e == cudaSuccess) {
        c.basis_tc.push_back(dtc);
        e = cudaMemcpy(dtc, split.data(), sizeof(float) * split.size(), cudaMemcpyHostToDevice);
      }
      if (e == cudaSuccess) e = mlmc::make_kl_tc_operand(dtc, dtc + rows * kp, rows, kp, mlmc::kKlTcElements, &op);
      if (e != cudaSuccess) {
        cudaGetLastError();
        g_create_error = std::string("tensor-core KL basis: ") + cudaGetErrorString(e);
        mlmc_destroy(h);
        return e == cudaErrorMemoryAllocation ? MLMC_ERR_OOM : MLMC_ERR_CUDA;
      }
      c.basis_tc_op.push_back(op);
    }
  }
  h->acc_host.assign(c.cfg.levels, mlmc::LevelAcc{});
  std::memset(h->acc_host.data(), 0, sizeof(mlmc::LevelAcc) * c.cfg.levels);
  h->next_id.assign(c.cfg.levels, 0);
  if (cudaMalloc(&h->acc_dev, sizeof(mlmc::LevelAcc) * c.cfg.levels) != cudaSuccess ||
      cudaMemset(h->acc_dev, 0, sizeof(mlmc::LevelAcc) * c.cfg.levels) != cudaSuccess) {
    cudaGetLastError();
    g_create_error = "stats allocation failed";
    mlmc_destroy(h);
    return MLMC_ERR_OOM;
  }
  cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    g_create_error = cudaGetErrorString(e);
    mlmc_destroy(h);
    return MLMC_ERR_CUDA;
  }
  *out = h;
  return MLMC_OK;
}

void mlmc_destroy(mlmc_ctx* h) {
  if (!h) return;
  cudaStreamSynchronize(h->c.stream);
  for (auto p : h->c.basis64) cudaFree(p);
  for (auto p : h->c.basis32) cudaFree(p);
  for (auto p : h->c.basis_tc) cudaFree(p);
  h->c.solve_arena.release();
  h->c.batch_arena.release();
  h->c.timer.release();
  if (h->acc_dev) cudaFree(h->acc_dev);
  delete h;
}

const char* mlmc_last_error(const mlmc_ctx* h) { return h ? h->c.err.c_str() : g_create_error.c_str(); }

mlmc_status mlmc_sample_level(mlmc_ctx* h, int32_t level, uint64_t first_id, int64_t n, double* q_fine,
                              double* q_coarse, int32_t* status) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  if (level < 0 || level >= c.cfg.levels) return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  if (n < 0) return c.fail(MLMC_ERR_INVALID_ARG, "negative sample count");
  if (n == 0) return MLMC_OK;
  mlmc_status s = sample_levels_impl(h, {LevelReq{level, first_id, n, 0}}, q_fine, q_coarse, status);
  if (s != MLMC_OK) return s;
  return sync_stats(h);
}

mlmc_status mlmc_sample_levels(mlmc_ctx* h, int32_t n_req, const int32_t* levels, const uint64_t* first_ids,
                               const int64_t* counts, double* q_fine, double* q_coarse, int32_t* status) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  if (n_req < 0 || (n_req > 0 && (!levels || !first_ids || !counts)))
    return c.fail(MLMC_ERR_INVALID_ARG, "bad request arrays");
  std::vector<LevelReq> reqs;
  int64_t off = 0;
  for (int k = 0; k < n_req; ++k) {
    if (levels[k] < 0 || levels[k] >= c.cfg.levels) return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
    if (counts[k] < 0) return c.fail(MLMC_ERR_INVALID_ARG, "negative sample count");
    if (counts[k] > 0) reqs.push_back(LevelReq{levels[k], first_ids[k], counts[k], off});
    off += counts[k];
  }
  if (reqs.empty()) return MLMC_OK;
  mlmc_status s = sample_levels_impl(h, reqs, q_fine, q_coarse, status);
  if (s != MLMC_OK) return s;
  return sync_stats(h);
}

mlmc_status mlmc_set_nested_threshold(mlmc_ctx* h, int64_t min_nodes) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  if (min_nodes < 0) return h->c.fail(MLMC_ERR_INVALID_ARG, "nested threshold must be >= 0");
  h->c.nested_min_nodes = min_nodes;
  return MLMC_OK;
}

mlmc_status mlmc_get_tuning(mlmc_ctx* h, mlmc_tuning* out) {
  if (!h || !out) return MLMC_ERR_INVALID_ARG;
  const Context& c = h->c;
  out->max_rows = c.max_rows;
  out->min_rows = c.min_rows;
  out->target_waves = c.target_waves;
  out->nested_min_nodes = c.nested_min_nodes;
  out->fused_bottom = c.fused_bottom;
  out->pack_samples = c.pack_samples ? 1 : 0;
  out->device_loop = c.device_loop ? 1 : 0;
  out->wide_strips = c.wide_strips;
  out->omega = c.omega;
  out->omega_retries = c.omega_retries;
  out->step_ms = 0.0;
  return MLMC_OK;
}

mlmc_status mlmc_set_tuning(mlmc_ctx* h, const mlmc_tuning* t) {
  if (!h || !t) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  if (t->max_rows < 1 || t->max_rows > 64 || t->min_rows < 1 || t->min_rows > t->max_rows ||
      !(t->target_waves >= 0.0 && t->target_waves <= 64.0) || t->nested_min_nodes < 0 ||
      t->fused_bottom < 0 || t->fused_bottom > 2 || (t->pack_samples != 0 && t->pack_samples != 1) ||
      (t->device_loop != 0 && t->device_loop != 1) || t->wide_strips < 0 || t->wide_strips > MLMC_WIDE_ALL ||
      !(t->omega > 0.0 && t->omega < 1.0))
    return c.fail(MLMC_ERR_INVALID_ARG, "tuning value out of range");
  c.fused_bottom = t->fused_bottom;
  c.pack_samples = t->pack_samples != 0;
  c.device_loop = t->device_loop != 0;
  c.wide_strips = t->wide_strips;
  c.omega = t->omega;
  c.max_rows = t->max_rows;
  c.min_rows = t->min_rows;
  c.target_waves = t->target_waves;
  c.nested_min_nodes = t->nested_min_nodes;
  return MLMC_OK;
}

mlmc_status mlmc_autotune(mlmc_ctx* h, int32_t n_req, const int32_t* levels, const int64_t* counts, int32_t reps,
                          mlmc_tuning* out) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  if (n_req <= 0 || !levels || !counts || reps < 1 || reps > 64) return c.fail(MLMC_ERR_INVALID_ARG, "bad tuning request");
  std::vector<LevelReq> reqs;
  int64_t total = 0;
  for (int k = 0; k < n_req; ++k) {
    if (levels[k] < 0 || levels[k] >= c.cfg.levels) return c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
    if (counts[k] < 0) return c.fail(MLMC_ERR_INVALID_ARG, "negative sample count");
    // sample ids from 2^62 up: the tuning solves draw fields no caller's ids reach
    if (counts[k] > 0) reqs.push_back(LevelReq{levels[k], (uint64_t)1 << 62, counts[k], total});
    total += counts[k];
  }
  if (reqs.empty()) return c.fail(MLMC_ERR_INVALID_ARG, "empty tuning request");
  // the tuning solves fold into the moments: keep the caller's and put them back
  std::vector<mlmc::LevelAcc> saved(c.cfg.levels);
  cudaError_t e;
  if ((e = cudaMemcpyAsync(saved.data(), h->acc_dev, sizeof(mlmc::LevelAcc) * c.cfg.levels, cudaMemcpyDeviceToHost,
                           c.stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c.stream)) != cudaSuccess)
    return c.cuda_fail(e, "autotune");
  std::vector<double> qf(2 * total), qc(2 * total);
  std::vector<int32_t> st(total);
  cudaEvent_t e0, e1;
  if ((e = cudaEventCreate(&e0)) != cudaSuccess || (e = cudaEventCreate(&e1)) != cudaSuccess)
    return c.cuda_fail(e, "autotune");
  struct Cand {
    int64_t nested;
    double waves;
    int max_rows, min_rows;
    int fused;
    int wide;
    double omega;
  };
  Cand best{c.nested_min_nodes, c.target_waves, c.max_rows, c.min_rows, c.fused_bottom, c.wide_strips, c.omega};
  double best_ms = 1e300;
  mlmc_status s = MLMC_OK;
  auto measure = [&](const Cand& k, double& ms) -> mlmc_status {
    c.nested_min_nodes = k.nested;
    c.target_waves = k.waves;
    c.max_rows = k.max_rows;
    c.min_rows = k.min_rows;
    c.fused_bottom = k.fused;
    c.wide_strips = k.wide;
    c.omega = k.omega;
    std::vector<double> t;
    for (int r = 0; r <= reps; ++r) {
      cudaEventRecord(e0, c.stream);
      mlmc_status ss = sample_levels_impl(h, reqs, qf.data(), qc.data(), st.data());
      if (ss != MLMC_OK) return ss;
      cudaEventRecord(e1, c.stream);
      cudaEventSynchronize(e1);
      float v = 0.f;
      cudaEventElapsedTime(&v, e0, e1);
      if (r > 0) t.push_back(v);   // the first call warms up
    }
    std::sort(t.begin(), t.end());
    ms = t[t.size() / 2];
    return MLMC_OK;
  };
  // a candidate replaces the best only when it is faster by more than 1 %: ties (such
  // as thresholds on either side of the workload's size) keep the current value
  auto consider = [&](Cand k) -> mlmc_status {
    double ms = 0;
    mlmc_status ss = measure(k, ms);
    if (ss == MLMC_OK && ms < 0.99 * best_ms) {
      best_ms = ms;
      best = k;
    }
    return ss;
  };
  // coordinate descent from the current values, timed first
  const int64_t nested_vals[2] = {0, (int64_t)1 << 62};
  const double wave_vals[3] = {0.75, 1.5, 3.0};
  const int max_vals[2] = {32, 64}, min_vals[3] = {4, 6, 8};
  s = consider(best);
  auto with = [&](auto&& edit) {   // best with one coordinate changed
    Cand k = best;
    edit(k);
    if (s == MLMC_OK) s = consider(k);
  };
  for (int64_t v : nested_vals) with([&](Cand& k) { k.nested = v; });
  for (int v : {1, 2, 0}) with([&](Cand& k) { k.fused = v; });
  for (double v : {0.5, 0.6, 0.65}) with([&](Cand& k) { k.omega = v; });   // smoother damping (solve_groups)
  for (int b = 0; b < 5; ++b) with([&](Cand& k) { k.wide ^= 1 << b; });    // each node-pair kernel on / off
  for (double v : wave_vals) with([&](Cand& k) { k.waves = v; });
  for (int v : max_vals)
    with([&](Cand& k) {
      k.max_rows = v;
      k.min_rows = std::min(k.min_rows, v);
    });
  for (int v : min_vals) with([&](Cand& k) { k.min_rows = std::min(v, k.max_rows); });
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c.nested_min_nodes = best.nested;
  c.target_waves = best.waves;
  c.max_rows = best.max_rows;
  c.min_rows = best.min_rows;
  c.fused_bottom = best.fused;
  c.wide_strips = best.wide;
  c.omega = best.omega;
  if ((e = cudaMemcpyAsync(h->acc_dev, saved.data(), sizeof(mlmc::LevelAcc) * c.cfg.levels, cudaMemcpyHostToDevice,
                           c.stream)) != cudaSuccess ||
      (e = cudaStreamSynchronize(c.stream)) != cudaSuccess)
    return c.cuda_fail(e, "autotune");
  if (s != MLMC_OK) return s;
  if (out) {
    mlmc_get_tuning(h, out);
    out->step_ms = best_ms;
  }
  return MLMC_OK;
}

mlmc_status mlmc_profile_enable(mlmc_ctx* h, int32_t on) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return c.cuda_fail(e, "profile");
  if (!c.timer.units_dev) {
    if ((e = cudaMalloc(&c.timer.units_dev, sizeof(unsigned long long) * mlmc::kProfOps)) != cudaSuccess)
      return c.cuda_fail(e, "profile");
  }
  if ((e = cudaMemset(c.timer.units_dev, 0, sizeof(unsigned long long) * mlmc::kProfOps)) != cudaSuccess)
    return c.cuda_fail(e, "profile");
  c.timer.reset();
  c.timer.on = on != 0;
  return MLMC_OK;
}

static_assert((int)mlmc::kProfOps == (int)MLMC_OP_COUNT, "kernel timer operations and MLMC_OP_* ids differ");

mlmc_status mlmc_profile_get(mlmc_ctx* h, int32_t op, double* ms_total, int64_t* launches, uint64_t* nodes) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  if (op < 0 || op >= mlmc::kProfOps) return c.fail(MLMC_ERR_INVALID_ARG, "unknown operation id");
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return c.cuda_fail(e, "profile");
  double ms = 0.0;
  int64_t cnt = 0;
  for (const auto& r : c.timer.recs) {
    if (r.op != op) continue;
    float t = 0.f;
    if ((e = cudaEventElapsedTime(&t, c.timer.pool[r.ev], c.timer.pool[r.ev + 1])) != cudaSuccess)
      return c.cuda_fail(e, "profile");
    ms += t;
    ++cnt;
  }
  if (ms_total) *ms_total = ms;
  if (launches) *launches = cnt;
  if (nodes) {
    unsigned long long u[mlmc::kProfOps] = {0};
    if (c.timer.units_dev &&
        (e = cudaMemcpy(u, c.timer.units_dev, sizeof(u), cudaMemcpyDeviceToHost)) != cudaSuccess)
      return c.cuda_fail(e, "profile");
    *nodes = u[op];
  }
  return MLMC_OK;
}

mlmc_status mlmc_profile_report(mlmc_ctx* h, char* buf, int64_t cap) {
  if (!h || !buf || cap <= 0) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  cudaError_t e = cudaStreamSynchronize(c.stream);
  if (e != cudaSuccess) return c.cuda_fail(e, "profile");
  std::map<std::string, std::pair<int64_t, double>> agg;
  for (const auto& r : c.timer.recs) {
    float t = 0.f;
    if ((e = cudaEventElapsedTime(&t, c.timer.pool[r.ev], c.timer.pool[r.ev + 1])) != cudaSuccess)
      return c.cuda_fail(e, "profile");
    auto& a = agg[r.name];
    a.first += 1;
    a.second += t;
  }
  std::string out;
  for (const auto& kv : agg)
    out += kv.first + " " + std::to_string(kv.second.first) + " " + std::to_string(kv.second.second) + "\n";
  const size_t n = std::min<size_t>(out.size(), (size_t)cap - 1);
  std::memcpy(buf, out.data(), n);
  buf[n] = 0;
  return MLMC_OK;
}

mlmc_status mlmc_launch_count(mlmc_ctx* h, int64_t* launches) {
  if (!h || !launches) return MLMC_ERR_INVALID_ARG;
  *launches = h->c.timer.launches;
  return MLMC_OK;
}

mlmc_status mlmc_level_stats_get(mlmc_ctx* h, int32_t level, mlmc_level_stats* out) {
  if (!h || !out) return MLMC_ERR_INVALID_ARG;
  if (level < 0 || level >= h->c.cfg.levels) return h->c.fail(MLMC_ERR_INVALID_ARG, "level out of range");
  mlmc_status s = sync_stats(h);
  if (s != MLMC_OK) return s;
  fill_stats(h, level, out);
  return MLMC_OK;
}

mlmc_status mlmc_reset_stats(mlmc_ctx* h) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  cudaError_t e = cudaMemsetAsync(h->acc_dev, 0, sizeof(mlmc::LevelAcc) * h->c.cfg.levels, h->c.stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->c.stream);
  if (e != cudaSuccess) return h->c.cuda_fail(e, "reset");
  std::memset(h->acc_host.data(), 0, sizeof(mlmc::LevelAcc) * h->acc_host.size());
  std::fill(h->next_id.begin(), h->next_id.end(), 0);
  return MLMC_OK;
}

mlmc_status mlmc_solve_batch(mlmc_ctx* h, const mlmc_item* items, int64_t n, double* q, int32_t* status) {
  return mlmc::solve_batch_carry(h, items, n, q, status, nullptr, nullptr, nullptr);
}

mlmc_status mlmc_estimate(mlmc_ctx* h, double e, double theta, int64_t n_star, int32_t max_level, int32_t qoi,
                          double* estimate, mlmc_level_stats* stats, int32_t* L_out) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  if (!(e > 0) || !(theta > 0 && theta < 1) || n_star < 1 || max_level < 0 || qoi < 0 || qoi > 1)
    return c.fail(MLMC_ERR_INVALID_ARG, "bad Algorithm 1 parameters");
  max_level = std::min<int32_t>(max_level, c.cfg.levels - 1);
  const double es2 = theta * e * e, eb = std::sqrt(1.0 - theta) * e;
  const double m = c.cfg.mlmc_m > 0 ? c.cfg.mlmc_m : 4.0;
  const double alpha = c.cfg.mlmc_alpha > 0 ? c.cfg.mlmc_alpha : 1.0;
  auto take = [&](int l, int64_t upto) -> mlmc_status {
    if (h->next_id[l] >= upto) return MLMC_OK;
    const int64_t cnt = upto - h->next_id[l];
    mlmc_status s = mlmc_sample_level(h, l, (uint64_t)h->next_id[l], cnt, nullptr, nullptr, nullptr);
    if (s != MLMC_OK) return s;
    h->next_id[l] = upto;
    return MLMC_OK;
  };
  int L = -1;
  bool converged = false;
  while (!converged) {
    if (L + 1 > max_level) break;
    ++L;
    mlmc_status s = take(L, n_star);
    if (s != MLMC_OK) return s;
    std::vector<double> V(L + 1), C(L + 1);
    for (int l = 0; l <= L; ++l) {
      const mlmc::LevelAcc& a = h->acc_host[l];
      V[l] = a.n > 0 ? a.m2[qoi] / (double)a.n : 0.0;
      C[l] = level_cost(c, l);
    }
    double tot = 0.0;
    for (int l = 0; l <= L; ++l) tot += std::sqrt(V[l] * C[l]);
    for (int l = 0; l <= L; ++l) {
      const int64_t nhat = (int64_t)std::ceil(tot * std::sqrt(V[l] / C[l]) / es2);
      if (h->next_id[l] < nhat) {
        s = take(l, nhat);
        if (s != MLMC_OK) return s;
      }
    }
    const double bias = std::fabs(h->acc_host[L].mean[qoi]) / (std::pow(m, alpha) - 1.0);
    if (bias < eb) converged = true;
  }
  double est = 0.0;
  for (int l = 0; l <= L; ++l) est += h->acc_host[l].mean[qoi];
  if (estimate) *estimate = est;
  if (L_out) *L_out = L;
  if (stats)
    for (int l = 0; l <= L; ++l) fill_stats(h, l, &stats[l]);
  return converged ? MLMC_OK : c.fail(MLMC_ERR_NOT_CONVERGED, "max_level reached before the bias test passed");
}

mlmc_status mlmc_merge_stats(const mlmc_level_stats* a, const mlmc_level_stats* b, mlmc_level_stats* out) {
  if (!a || !b || !out) return MLMC_ERR_INVALID_ARG;
  mlmc_level_stats r;
  std::memset(&r, 0, sizeof(r));
  r.n = a->n + b->n;
  r.cost = a->n > 0 ? a->cost : b->cost;
  const double na = (double)a->n, nb = (double)b->n, n = (double)r.n;
  for (int k = 0; k < 2; ++k) {
    if (r.n == 0) break;
    const double d = b->mean[k] - a->mean[k];
    r.mean[k] = a->mean[k] + d * (nb / n);
    r.m2[k] = a->m2[k] + b->m2[k] + d * d * (na * nb / n);
    r.var[k] = r.m2[k] / n;
    r.sum_qf[k] = a->sum_qf[k] + b->sum_qf[k];
    r.sum_qc[k] = a->sum_qc[k] + b->sum_qc[k];
  }
  *out = r;
  return MLMC_OK;
}

mlmc_status mlmc_kl_coefficients(mlmc_ctx* h, int32_t level, uint64_t first_id, int64_t n, double* xi) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  if (level < 0 || n < 0 || (n > 0 && !xi)) return c.fail(MLMC_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return MLMC_OK;
  const size_t cnt = (size_t)n * c.cfg.kl_terms;
  cudaError_t e = c.batch_arena.reserve(sizeof(double) * cnt + 1024);
  if (e != cudaSuccess) return c.fail(MLMC_ERR_OOM, "xi buffer");
  c.batch_arena.reset();
  double* d = c.batch_arena.carve<double>(cnt);
  int* fail = c.batch_arena.carve<int>(1);
  if ((e = cudaMemsetAsync(fail, 0, sizeof(int), c.stream)) != cudaSuccess ||
      (e = mlmc::launch_kl_coefficients(c.cfg.seed, level, first_id, nullptr, nullptr, n, c.cfg.kl_terms, d,
                                        nullptr, fail, c.stream)) != cudaSuccess ||
      (e = from_device(xi, d, cnt, c.stream)) != cudaSuccess || (e = cudaStreamSynchronize(c.stream)) != cudaSuccess)
    return c.cuda_fail(e, "kl_coefficients");
  return MLMC_OK;
}

mlmc_status mlmc_theta(mlmc_ctx* h, int32_t level, int32_t mesh_level, uint64_t first_id, int64_t n,
                       double* theta) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  if (level < 0 || mesh_level < 0 || mesh_level >= c.cfg.levels || n < 0 || (n > 0 && !theta))
    return c.fail(MLMC_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return MLMC_OK;
  const int nkl = c.cfg.kl_terms;
  const int64_t nel = c.mesh(mesh_level).n_el();
  mlmc::Sizer sz;
  const bool tc = c.kl_on_tensor_cores();
  const int kp = c.kl_kpad();
  sz.add<double>(n * nkl);
  sz.add<float>(n * nkl);
  sz.add<float>(tc ? 2 * n * kp : 1);
  sz.add<int>(2);
  sz.add<double>(n * nel);
  sz.add<float>(n * nel);
  cudaError_t e = c.batch_arena.reserve(sz.used + 256);
  if (e != cudaSuccess) return c.fail(MLMC_ERR_OOM, "theta buffers");
  c.batch_arena.reset();
  double* xi = c.batch_arena.carve<double>(n * nkl);
  float* xi32 = c.batch_arena.carve<float>(n * nkl);
  float* xi_tc = c.batch_arena.carve<float>(tc ? 2 * n * kp : 1);
  int* fail = c.batch_arena.carve<int>(2);
  double* th = c.batch_arena.carve<double>(n * nel);
  float* th32 = c.batch_arena.carve<float>(n * nel);
  cudaStream_t st = c.stream;
  if ((e = cudaMemsetAsync(fail, 0, 2 * sizeof(int), st)) != cudaSuccess ||
      (e = mlmc::launch_kl_coefficients(c.cfg.seed, level, first_id, nullptr, nullptr, n, nkl, xi, xi32, fail, st)) !=
          cudaSuccess)
    return c.cuda_fail(e, "kl_coefficients");
  if (tc) {
    mlmc::KlTcOperand xop;
    if ((e = mlmc::launch_tf32_split(xi, n, nkl, kp, xi_tc, xi_tc + n * kp, st)) != cudaSuccess ||
        (e = mlmc::make_kl_tc_operand(xi_tc, xi_tc + n * kp, n, kp, mlmc::kKlTcSamples, &xop)) != cudaSuccess ||
        (e = mlmc::launch_kl_synthesis_tc(c.basis_tc_op[mesh_level], xop, (int)nel, n, th32, false, fail + 1, st)) !=
            cudaSuccess ||
        (e = convert(th32, th, n * nel, st)) != cudaSuccess)
      return c.cuda_fail(e, "kl_synthesis");
    int h_err = 0;
    if ((e = cudaMemcpyAsync(&h_err, fail + 1, sizeof(int), cudaMemcpyDeviceToHost, st)) != cudaSuccess ||
        (e = cudaStreamSynchronize(st)) != cudaSuccess)
      return c.cuda_fail(e, "kl_synthesis");
    if (h_err) return c.fail(MLMC_ERR_TIMEOUT, "tensor-core KL synthesis: a wait expired");
  } else if (c.mixed()) {
    if ((e = mlmc::launch_kl_synthesis<float>(xi32, c.basis32[mesh_level], n, (int)nel, nkl, th32, false, st)) !=
            cudaSuccess ||
        (e = convert(th32, th, n * nel, st)) != cudaSuccess)
      return c.cuda_fail(e, "kl_synthesis");
  } else if ((e = mlmc::launch_kl_synthesis<double>(xi, c.basis64[mesh_level], n, (int)nel, nkl, th, false, st)) !=
             cudaSuccess) {
    return c.cuda_fail(e, "kl_synthesis");
  }
  if ((e = from_device(theta, th, n * nel, st)) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return c.cuda_fail(e, "copy out");
  return MLMC_OK;
}

mlmc_status mlmc_apply(mlmc_ctx* h, int32_t mesh_level, int64_t n, const double* theta, const double* p, double* q) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  if (mesh_level < 0 || mesh_level >= c.cfg.levels || n < 0 || (n > 0 && (!theta || !p || !q)))
    return c.fail(MLMC_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return MLMC_OK;
  const mlmc::LevelLayout m = c.mesh(mesh_level);
  const int64_t ne = n * m.n_el(), nd = n * 2 * m.n_nodes();
  mlmc::Sizer sz;
  sz.add<double>(ne);
  sz.add<double>(nd);
  sz.add<double>(nd);
  sz.add<double>(2 * ne);
  sz.add<float>(2 * ne);
  sz.add<float>(nd);
  sz.add<float>(nd);
  cudaError_t e = c.batch_arena.reserve(sz.used + 256);
  if (e != cudaSuccess) return c.fail(MLMC_ERR_OOM, "apply buffers");
  c.batch_arena.reset();
  double* th = c.batch_arena.carve<double>(ne);
  double* pd = c.batch_arena.carve<double>(nd);
  double* qd = c.batch_arena.carve<double>(nd);
  double* t2 = c.batch_arena.carve<double>(2 * ne);
  float* t232 = c.batch_arena.carve<float>(2 * ne);
  float* p32 = c.batch_arena.carve<float>(nd);
  float* q32 = c.batch_arena.carve<float>(nd);
  cudaStream_t st = c.stream;
  if ((e = to_device(th, theta, ne, st)) != cudaSuccess || (e = to_device(pd, p, nd, st)) != cudaSuccess)
    return c.cuda_fail(e, "copy in");
  mlmc_status s;
  if (c.mixed()) {
    if ((e = mlmc::launch_theta_to_trig2<float>(th, ne, t232, st)) != cudaSuccess ||
        (e = convert(pd, p32, nd, st)) != cudaSuccess)
      return c.cuda_fail(e, "convert");
    s = mlmc::apply_operator<float>(c, mesh_level, n, t232, p32, q32);
    if (s != MLMC_OK) return s;
    if ((e = convert(q32, qd, nd, st)) != cudaSuccess) return c.cuda_fail(e, "convert");
  } else {
    if ((e = mlmc::launch_theta_to_trig2<double>(th, ne, t2, st)) != cudaSuccess) return c.cuda_fail(e, "convert");
    s = mlmc::apply_operator<double>(c, mesh_level, n, t2, pd, qd);
    if (s != MLMC_OK) return s;
  }
  if ((e = from_device(q, qd, nd, st)) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return c.cuda_fail(e, "copy out");
  return MLMC_OK;
}

mlmc_status mlmc_solve_theta(mlmc_ctx* h, int32_t mesh_level, int64_t n, const double* theta, double* q,
                             int32_t* status, int32_t* iterations) {
  if (!h) return MLMC_ERR_INVALID_ARG;
  Context& c = h->c;
  if (mesh_level < 0 || mesh_level >= c.cfg.levels || n < 0 || (n > 0 && (!theta || !q)))
    return c.fail(MLMC_ERR_INVALID_ARG, "bad arguments");
  if (n == 0) return MLMC_OK;
  const int64_t ne = n * c.mesh(mesh_level).n_el();
  mlmc::Sizer sz;
  sz.add<double>(ne);
  sz.add<double>(2 * ne);
  sz.add<float>(2 * ne);
  sz.add<double>(2 * n);
  sz.add<int>(n);
  sz.add<int>(n);
  cudaError_t e = c.batch_arena.reserve(sz.used + 256);
  if (e != cudaSuccess) return c.fail(MLMC_ERR_OOM, "solve buffers");
  c.batch_arena.reset();
  double* th = c.batch_arena.carve<double>(ne);
  double* t2 = c.batch_arena.carve<double>(2 * ne);
  float* t232 = c.batch_arena.carve<float>(2 * ne);
  double* qd = c.batch_arena.carve<double>(2 * n);
  int* sd = c.batch_arena.carve<int>(n);
  int* itd = c.batch_arena.carve<int>(n);
  cudaStream_t st = c.stream;
  if ((e = to_device(th, theta, ne, st)) != cudaSuccess) return c.cuda_fail(e, "copy in");
  mlmc_status s;
  if (c.mixed()) {
    if ((e = mlmc::launch_theta_to_trig2<float>(th, ne, t232, st)) != cudaSuccess) return c.cuda_fail(e, "convert");
    std::vector<mlmc::SolveGroup<float>> g{{mesh_level, n, t232, qd, sd, itd}};
    s = mlmc::solve_groups<float>(c, g);
  } else {
    if ((e = mlmc::launch_theta_to_trig2<double>(th, ne, t2, st)) != cudaSuccess) return c.cuda_fail(e, "convert");
    std::vector<mlmc::SolveGroup<double>> g{{mesh_level, n, t2, qd, sd, itd}};
    s = mlmc::solve_groups<double>(c, g);
  }
  if (s != MLMC_OK) return s;
  if ((e = from_device(q, qd, 2 * n, st)) != cudaSuccess ||
      (e = from_device(status, sd, n, st)) != cudaSuccess ||
      (e = from_device(iterations, itd, n, st)) != cudaSuccess || (e = cudaStreamSynchronize(st)) != cudaSuccess)
    return c.cuda_fail(e, "copy out");
  return MLMC_OK;
}

}  // extern "C"
