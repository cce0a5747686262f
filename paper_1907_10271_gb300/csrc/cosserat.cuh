// Cosserat engine (Sec. 3, the first test problem): device data layout and kernels.
//
// Layout. A batch of S samples on an n x n mesh has N = (n + 1)^2 nodes, node
// p = j (n + 1) + i. A vector is one float4 (u, v, theta_3, 0) per node, v[s * N + p],
// so that a thread loads a neighbour's three components in one instruction. The operator
// is the assembled 9-point stencil of 3 x 3 blocks, stored as half of it per node (the
// rest follows from symmetry), 42 coefficients k padded to 44 and grouped in float4s:
// group g = k / 4 of node p at A[(s * kGroups + g) * N + p], component k % 4, so that a
// warp's 32 consecutive nodes load one 512-byte line set per group. The coefficients:
//   k 0 .. 5    the diagonal block, upper triangle (00, 01, 02, 11, 12, 22),
//   k 6 .. 14   block to the east neighbour (+1, 0), row-major [row of p][column of q],
//   k 15 .. 23  north (0, +1), k 24 .. 32 north-east (+1, +1), k 33 .. 41 north-west (-1, +1);
// the blocks to the W, S, SW and SE neighbours are the transposes of those neighbours'
// E, N, NE and NW blocks. Dirichlet DOFs (u on x = 0 and x = L, v on y = 0 and y = L)
// have identity rows and columns. Dinv holds omega times the inverse of the diagonal
// block (upper triangle, 6 values padded to 8 in two float4 groups per node) for the
// block-Jacobi smoother.
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mlmcc {

constexpr int kMaxViews = 8;      // meshes of one call (one per MLMC mesh level)
constexpr int kMaxMeshes = 8;
constexpr int kStencil = 42;
constexpr int kGroups = 11;      // float4 groups of the stencil per node (44 floats)
constexpr int kDinv = 6;
constexpr int kDinvGroups = 2;
constexpr int kTerms = 5;         // trig terms of the element matrix: 1, c2, s2, c4, s4
constexpr int kCoarsest = 2;      // elements per side of the coarsest multigrid mesh
constexpr int kCoarseDofs = 27;   // 3 (kCoarsest + 1)^2
constexpr int kThreads = 256;
constexpr int kInverseWarps = 8;   // samples (one warp each) per block of the coarsest inverse
// block-Jacobi damping: the V-cycle is SPD for omega < 2 / lambda_max(B^-1 A) (B the
// nodal 3 x 3 blocks); lambda_max is 2.27 - 2.78 over the workload's fields, fields ten
// times rougher and uniform angles, so 0.65 keeps an 11 % margin
constexpr float kOmega = 0.65f;
constexpr int kBottomN = 8;       // the fused bottom covers the meshes of at most 8 x 8 elements
constexpr int kBottomThreads = 96;

// One multigrid level of one batch.
struct Lev {
  int n, N, S;
  float4* A;      // [S][kGroups][N]
  float4* Dinv;   // [S][kDinvGroups][N]
  float4* r;      // [S][N] right-hand side of the level's correction equation
  float4* x;      // [S][N] iterate
  float4* t;      // [S][N] residual for restriction, then the smoothed result
};

// Per-sample solver state (FP64 scalars of the correction CG and the refinement).
struct SampleState {
  double rz, rz_new, pq, rr, rr0, tol2, bnorm2, r64n2;
  double alpha, beta;
  int act;       // correction CG running
  int done;      // refinement finished (converged or out of iterations)
  int it;        // correction iterations of the current refinement step
  int it_total;  // all correction iterations
  int refine;    // FP64 residual evaluations
  int first;     // next direction update is the first of a refinement step
  int conv;      // converged to rtol
  int pad;
};

// The solve mesh of one batch: FP64 system, CG vectors and per-element trig values.
struct FineSys {
  float4* Alo;     // [S][kGroups][N] low part of the float-float stencil (high part: level 0's A)
  float4 *bh, *bl;   // [S][N] right-hand side, float-float
  float4 *dh, *dl;   // [S][N] solution without the prescribed values, float-float
  const float* trig;   // [S][n * n][8]: cos 2 phi, sin 2 phi, cos 4 phi, sin 4 phi as (hi, lo) pairs
  float4 *c, *p0, *p1, *q;   // [S][N]
  SampleState* st;          // [S]
  double* acc;              // [S][4]: f*, int sigma_x, reaction, spare
  double* q_out;            // [S][2]
  int* stat_out;            // [S]: 0 or 4 (not converged)
  int* iters;               // [2]: max correction iterations, max FP64 residuals (atomicMax)
  int mesh;                 // element-matrix basis index
  int klo, khi;             // element rows / columns inside Omega'
};

// A launch's work: up to kMaxViews batches, each with a finer level f, the next coarser
// level c (when the kernel moves data between levels) and its solve-mesh system.
struct View {
  Lev f, c;
  FineSys F;
  float* Ainv;   // [S][27][27] coarsest inverse (coarse-solve kernels)
  int blk0;      // first block of this view
  int items;     // work items (threads) of this view
};
struct Consts;
struct Views {
  int nv;
  int nblk;
  const Consts* cc;   // the context's constants (device memory)
  View v[kMaxViews];
};

// Constants of a context, computed on the host and kept in device memory: per mesh the
// element matrix of a square element as sum_m t_m Km[m] (t = 1, cos 2 phi, sin 2 phi,
// cos 4 phi, sin 4 phi), and C*(phi) as sum_m t_m Cm[m] for the stresses.
struct Consts {
  double Km[kMaxMeshes][kTerms][144];
  float Kmh[kMaxMeshes][kTerms][144], Kml[kMaxMeshes][kTerms][144];   // Km split hi + lo
  double Cm[kTerms][16];
  double h[kMaxMeshes];
  double shortening, tau_y, R;
  float msh_hi, msh_lo;   // -shortening, float-float
};

// setup
cudaError_t launch_build_fine(const Views& v, cudaStream_t st);       // A + Alo, b64, Dinv, |b|^2
cudaError_t launch_rap(const Views& v, cudaStream_t st);              // c-level A, Dinv from f-level A
cudaError_t launch_coarsest_inverse(const Views& v, cudaStream_t st);  // Ainv from the f level (n = 2)
// V-cycle
cudaError_t launch_pre(const Views& v, cudaStream_t st);               // x = Dinv r, t = r - A x
cudaError_t launch_restrict(const Views& v, cudaStream_t st);          // c.r = P^T f.t (masked)
// the cycle below and including f (n <= kBottomN) of each view in one block per sample;
// bit v of top_mask: view v's f is its solve mesh (r . z into rz_new)
cudaError_t launch_bottom(const Views& v, int top_mask, cudaStream_t st);
cudaError_t launch_prolong(const Views& v, cudaStream_t st);           // f.x += P c.t
cudaError_t launch_post(const Views& v, bool top, cudaStream_t st);    // f.t = x + Dinv (r - A x)
// correction CG on the solve mesh (f = level 0)
cudaError_t launch_cg_apply(const Views& v, bool odd, cudaStream_t st);
cudaError_t launch_scal_a(const Views& v, cudaStream_t st);
cudaError_t launch_cg_update(const Views& v, bool odd, cudaStream_t st);
cudaError_t launch_scal_b(const Views& v, int max_iter, cudaStream_t st);
cudaError_t launch_count_active(const Views& v, int* count, cudaStream_t st);
// FP64 refinement
cudaError_t launch_resid64(const Views& v, bool first, cudaStream_t st);   // first: d = 0
cudaError_t launch_outer_check(const Views& v, double rtol, int max_iter, cudaStream_t st);
cudaError_t launch_accumulate(const Views& v, cudaStream_t st);
// quantities of interest
cudaError_t launch_qoi(const Views& v, cudaStream_t st);
cudaError_t launch_qoi_final(const Views& v, cudaStream_t st);
// y = A x on the solve mesh with the float-float stencil (x, y [S][N][3] doubles)
cudaError_t launch_apply64(const Views& v, const double* x, double* y, cudaStream_t st);
// KL synthesis in float-float: basis (hi, lo) [n_el][K] floats, xi [S][K] doubles ->
// with trig, out = float [S][n_el][8] (cos 2 phi, sin 2 phi, cos 4 phi, sin 4 phi as
// hi, lo pairs); else out = double phi [S][n_el]
cudaError_t launch_synth_ff(const double* xi, const float* Bh, const float* Bl, int S, int n_el, int K, void* out,
                            bool trig, cudaStream_t st);
// float-float [S][N] (hi, lo) float4s -> double [S][N][3], adding u = shortening on x = L
cudaError_t launch_ff_to_aos(const float4* hi, const float4* lo, double* out, int S, int n, double shortening,
                             cudaStream_t st);

}  // namespace mlmcc
