// Internal interfaces of the level-pair engine (host side).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mlmc.h"
#include "common.cuh"

namespace mlmc {

// ---------------------------------------------------------------- kernels (launchers)
cudaError_t launch_kl_coefficients(uint64_t seed, int level, uint64_t first_id, const int* levels,
                                   const uint64_t* ids, int64_t n, int n_kl, double* xi, float* xi32, int* fail,
                                   cudaStream_t st);

// theta = Xi B^T; with trig2 set, writes (cos 2 theta, sin 2 theta) per element
// ([nsamp][n_el][2]) instead of theta ([nsamp][n_el]).
template <typename T>
cudaError_t launch_kl_synthesis(const T* xi, const T* basis, int64_t nsamp, int n_el, int n_kl,
                                T* out, bool trig2, cudaStream_t st);

// (cos 2 theta, sin 2 theta) of given angles (double input).
template <typename T>
cudaError_t launch_theta_to_trig2(const double* theta, int64_t n, T* trig2, cudaStream_t st);

// ---------------------------------------------------------------- KL basis (host)
struct KLBasis {
  int nx, ny, n_kl;
  std::vector<double> B;   // [n_el][n_kl], B[e][n] = sqrt(mu_n) phi_n(centroid_e)
};

// Builds the basis of every mesh level 0..levels-1. Returns false with msg on failure.
bool build_kl_bases(const mlmc_config& cfg, std::vector<KLBasis>& out, std::string& msg);

// ---------------------------------------------------------------- solver
struct Context;  // defined in api.cu

// One set of n samples on one mesh, each with its own field theta (device, T).
template <typename T>
struct SolveGroup {
  int mesh_level;      // MLMC mesh index
  int64_t nsamp;
  const T* trig2;      // [nsamp][n_el][2] device: cos 2 theta, sin 2 theta per element
  double* q;           // [nsamp][2] device output
  int* status;         // [nsamp] device output
  int* iters;          // [nsamp] device output (total PCG iterations)
  // nested iteration (optional): the same samples' final iterates on mesh
  // mesh_level - 1, prolongated as the initial iterate, and where to copy this
  // solve's final iterates (both in the refinement iterate's storage layout)
  const double* d_guess = nullptr;
  double* d_out = nullptr;
};

// Solves every group to cfg.rtol (fp64 path: T = double throughout; mixed path:
// T = float inner solve with double refinement) and writes q, status, iters.
template <typename T>
mlmc_status solve_groups(Context& ctx, std::vector<SolveGroup<T>>& groups);

template <typename T>
mlmc_status apply_operator(Context& ctx, int mesh_level, int64_t n, const T* trig2, const T* p, T* q);

// Grows a context's solver and batch workspaces to at least the given sizes now, so
// that later calls within them allocate nothing (cudaFree synchronises the device).
mlmc_status reserve_workspace(mlmc_ctx* h, size_t solve_bytes, size_t batch_bytes);

// Whether solves of this context replay their PCG batches from captured CUDA graphs
// (on by default). A capture and instantiation per solve pays off over a few replays
// of a fixed batch; a request loop whose every batch differs turns it off.
void set_graph_replay(mlmc_ctx* h, bool on);

// mlmc_solve_batch with per-item starting iterates: guess[k] (device: item k's final
// iterate on mesh mesh_level - 1, in the refinement iterate's storage layout, 2 values
// per node; null: the item starts from the lifting) and out[k] (device: where item k's
// final iterate on its mesh is stored, or null). guess and out may be null as a whole.
// iters (host, nullable): each item's PCG iterations.
mlmc_status solve_batch_carry(mlmc_ctx* h, const mlmc_item* items, int64_t n, double* q, int32_t* status,
                              const double* const* guess, double* const* out, int32_t* iters);

// Values of a refinement iterate on mesh m (2 per node; 8 bytes each).
int64_t iterate_values(const mlmc_config& cfg, int m);

// Checks a strip configuration: the reason it is rejected, or "" when it is valid.
std::string validate(const mlmc_config& cfg);

// Tsai-Pagano invariants of the plane-strain fibre-frame stiffness of cfg's ply; ok is
// false when the constants do not give a positive definite stiffness.
Invariants invariants(const mlmc_config& cfg, bool& ok);

// Device bytes one solve on `mesh` needs in a batch (solver workspace, field and
// outputs), with margin.
double solve_bytes_per_sample(const mlmc_config& cfg, int mesh);

}  // namespace mlmc
