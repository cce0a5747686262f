// Library context (host side).
#pragma once
#include <algorithm>
#include <string>
#include <vector>

#include "engine.h"
#include "fem.cuh"
#include "kl_tc.h"

namespace mlmc {

// Grow-only device arena: carve() hands out 256-byte aligned ranges of one allocation.
struct Arena {
  char* base = nullptr;
  size_t cap = 0, used = 0;
  bool borrowed = false;   // memory owned by someone else: never reallocated or freed here
  cudaError_t reserve(size_t bytes) {
    if (bytes <= cap) return cudaSuccess;
    if (borrowed) return cudaErrorMemoryAllocation;
    if (base) cudaFree(base);
    base = nullptr;
    cap = 0;
    cudaError_t e = cudaMalloc(&base, bytes);
    if (e != cudaSuccess) return e;
    cap = bytes;
    return cudaSuccess;
  }
  void reset() { used = 0; }
  template <typename T>
  T* carve(size_t count) {
    const size_t off = (used + 255) & ~(size_t)255;
    used = off + count * sizeof(T);
    return reinterpret_cast<T*>(base + off);
  }
  void release() {
    if (base && !borrowed) cudaFree(base);
    base = nullptr;
    cap = used = 0;
  }
};

// Size accounting twin of Arena (same alignment rule).
struct Sizer {
  size_t used = 0;
  template <typename T>
  void add(size_t count) {
    used = ((used + 255) & ~(size_t)255) + count * sizeof(T);
  }
};

// Optional per-operation kernel timing (CUDA events on the library stream) and a
// count of every kernel the library launches.
struct KernelTimer {
  bool on = false;
  int64_t launches = 0;
  std::vector<cudaEvent_t> pool;
  size_t used = 0;
  struct Rec {
    int op;
    size_t ev;
    const char* name;
  };
  std::vector<Rec> recs;
  unsigned long long* units_dev = nullptr;   // [kProfOps]
  int pending_op = -1;
  size_t pending_ev = 0;
  const char* pending_name = "";

  cudaEvent_t next() {
    if (used == pool.size()) {
      cudaEvent_t e;
      cudaEventCreate(&e);
      pool.push_back(e);
    }
    return pool[used++];
  }
  void begin(int op, cudaStream_t st, const char* name = "") {
    ++launches;
    if (!on) return;
    pending_op = op;
    pending_ev = used;
    pending_name = name;
    cudaEventRecord(next(), st);
  }
  void end(cudaStream_t st) {
    if (pending_op < 0) return;
    cudaEventRecord(next(), st);
    recs.push_back(Rec{pending_op, pending_ev, pending_name});
    pending_op = -1;
  }
  void reset() {
    used = 0;
    recs.clear();
    launches = 0;
    pending_op = -1;
  }
  void release() {
    for (auto e : pool) cudaEventDestroy(e);
    pool.clear();
    if (units_dev) cudaFree(units_dev);
    units_dev = nullptr;
  }
};

struct LevelLayout {
  int nx, ny;
  int64_t n_el() const { return (int64_t)nx * ny; }
  int64_t n_nodes() const { return (int64_t)(nx + 1) * (ny + 1); }
};

struct Context {
  mlmc_config cfg;
  cudaStream_t stream = nullptr;
  int device = 0;
  Invariants U;
  std::vector<KLBasis> bases_host;
  std::vector<double*> basis64;   // device, per mesh level
  std::vector<float*> basis32;
  std::vector<float*> basis_tc;          // device, per mesh level: TF32 hi [n_el][kp] then lo
  std::vector<KlTcOperand> basis_tc_op;  // their TMA descriptors
  Arena solve_arena;              // solver workspace
  Arena batch_arena;              // per-call inputs (xi, theta, outputs)
  std::vector<mlmc_level_stats> stats;
  std::vector<double> comp;       // Kahan compensation of sum_qf / sum_qc per level [l][4]
  std::string err;
  KernelTimer timer;
  double floor_tol32 = 3e-6;      // tightest inner relative tolerance of the FP32 solve
  int check_every = 4;            // PCG iterations between host convergence checks
  bool graphs = true;             // replay PCG batches from a CUDA graph captured per solve
  bool device_loop = false;       // with graphs: repeat the batches on the device (conditional node)
  int64_t nested_min_nodes = int64_t(1) << 22;   // finest-mesh nodes per call for nested iteration
  // launch shapes of the strip kernels (mlmc_autotune): row chunks of at most max_rows
  // rows; launches of fewer warps than target_waves resident waves split their chunks
  // (up to 8 ways, at least min_rows rows each)
  int max_rows = 64;
  int min_rows = 6;
  double target_waves = 1.5;
  // multigrid bottom (FP32 path, small enough bottoms): 2 = the three smallest
  // non-coarsest meshes and the coarsest solve of each hierarchy in one launch, one
  // thread block per sample; 1 = the two smallest and the coarsest, one warp per
  // sample; 0 = a launch per level
  int fused_bottom = 1;
  // strip kernels tile the samples of a view side by side (see View::packed)
  bool pack_samples = true;
  // FP32 strip kernels with a node pair per lane (strip_wide.cu), bit mask over
  // wide_strip_bit(op) (mlmc_tuning.wide_strips)
  int wide_strips = MLMC_WIDE_POST | MLMC_WIDE_POST_TOP;
  // damping of the pair-block Jacobi smoother (see solve_groups: calls that leave a
  // sample unconverged at omega > kOmega are solved again at kOmega)
  double omega = 0.6;
  int64_t omega_retries = 0;
  int last_outer = 0;             // refinement steps of the last solve (diagnostic)
  int last_iters = 0;             // max PCG iterations of the last solve (diagnostic)

  bool mixed() const { return cfg.precision == MLMC_PREC_MIXED; }
  // KL synthesis of the mixed path on the tensor cores (3xTF32); FP32 CUDA cores past 128 terms
  bool kl_on_tensor_cores() const { return mixed() && kl_tc_supported(cfg.kl_terms); }
  int kl_kpad() const { return kl_tc_kpad(cfg.kl_terms); }
  LevelLayout mesh(int l) const { return LevelLayout{cfg.nx0 << l, cfg.ny0 << l}; }
  Geo geo(int nx, int ny) const {
    Geo g;
    g.nx = nx;
    g.ny = ny;
    const double hx = cfg.lx / nx, hy = cfg.ly / ny;
    g.rx = 0.5 / hx;
    g.ry = 0.5 / hy;
    g.w = hx * hy;
    g.square = hx == hy ? 1 : 0;
    // centroid x = (i + 1/2) (lx / nx), tested in double exactly as the definition reads
    g.c0 = nx;
    g.c1 = -1;
    for (int i = 0; i < nx; ++i) {
      const double cx = ((double)i + 0.5) * (cfg.lx / nx);
      if (cx >= cfg.omega_x0 && cx <= cfg.omega_x1) {
        g.c0 = std::min(g.c0, i);
        g.c1 = std::max(g.c1, i);
      }
    }
    return g;
  }
  mlmc_status fail(mlmc_status s, const std::string& m) {
    err = m;
    return s;
  }
  mlmc_status cuda_fail(cudaError_t e, const char* where) {
    cudaGetLastError();  // clear a non-sticky error so later launch checks do not see it
    err = std::string(where) + ": " + cudaGetErrorString(e);
    return MLMC_ERR_CUDA;
  }
};

}  // namespace mlmc
