// Internal interfaces of the panel-buckling engine (Reissner-Mindlin Q4 plates).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mlmcp {

constexpr int kMaxPlies = 32;
constexpr int kMaxCoarseFree = 192;   // free DOFs of the coarsest mesh (dense inverse in shared memory)
constexpr int kCols = 2;              // LOBPCG block size
constexpr int kSub = 3 * kCols;       // Rayleigh-Ritz subspace [X, W, P]
constexpr int kGram = kSub * (kSub + 1) / 2;
constexpr float kOmegaP = 0.5f;       // block-Jacobi damping of the smoother

// Laminate constants, identical for every sample: ply stiffness, stacking, thickness.
struct Laminate {
  double E11, E22, G12, nu12, G13, k_shear, t_ply, std_rad;
  int n_plies;
  double psi[kMaxPlies];   // pristine angles, radians, bottom ply first
};

// One mesh of one solve: nb vectors ("batch entries") on nx x ny square elements; a
// vector entry b belongs to sample b >> cshift. Vectors are [entry][node][4] floats
// (w, theta_x, theta_y, 0), node = j (nx + 1) + i.
struct PGrid {
  int nx, ny, nb, cshift, hard;
  float hx, hy;
  __host__ __device__ int nodes() const { return (nx + 1) * (ny + 1); }
};

// Per-sample laminate of a solve: dstar [n][6] (11, 12, 16, 22, 26, 66), kgt [n].
cudaError_t launch_laminate(const Laminate& lam, const double* xi, int n, double* dstar, double* kgt,
                            cudaStream_t st);
// Element matrices [n][144] (row-major, local DOF 3 a + c, corners (i, j), (i+1, j),
// (i+1, j+1), (i, j+1)) of every sample on elements hx x hy; k32 and k64 nullable.
cudaError_t launch_element_matrices(const double* dstar, const double* kgt, int n, double hx, double hy, float* k32,
                                    double* k64, cudaStream_t st);

// out = K x (or b - K x with b set) and optionally gout = G x, for entries whose
// sample is active (null: all). bc: zero the constrained DOFs of inputs and outputs.
cudaError_t launch_apply(const PGrid& g, const float* ke, const float4* x, const float4* b, float4* out,
                         float4* gout, const int* active, bool bc, cudaStream_t st);
// out = K x with the double element matrices ke64 and double sums, gout = G x, and
// (rout set) rout = G x - mu K x with mu[sample][column] of each entry, also in double;
// the input's w in two parts (x.x + x.w); the constrained DOFs of inputs and outputs
// zeroed (the images and residuals of the LOBPCG vectors of thin plates)
cudaError_t launch_apply64(const PGrid& g, const double* ke64, const float4* x, float4* out, float4* gout,
                           float4* rout, const double* mu, const int* active, cudaStream_t st);
// out = x + w D^-1 (b - K x) (x null: out = w D^-1 b), D the nodal 3x3 diagonal blocks
cudaError_t launch_smooth(const PGrid& g, const float* ke, const float4* b, const float4* x, float4* out,
                          const int* active, cudaStream_t st);
// bc = P^T rf (full weighting), xf += P xc (bilinear)
cudaError_t launch_restrict(const PGrid& fine, const PGrid& coarse, const float4* rf, float4* bc, const int* active,
                            cudaStream_t st);
cudaError_t launch_prolong(const PGrid& fine, const PGrid& coarse, const float4* xc, float4* xf, const int* active,
                           cudaStream_t st);
// Patch smoother (thin plates): multiplicative Schwarz over 3 x 3-node patches in nine
// colours. Colour (sx, sy) tiles the mesh with the patches centred on the nodes
// (sx + 3 k, sy + 3 l), k, l integers (centres from -1 to n + 1, patches cut at the
// boundary), so one colour step is block Jacobi on that tiling:
//   out = in + sum_p R_p^T A_p^-1 R_p (b - K in),   A_p = R_p K R_p^T,
// with R_p the free DOFs of patch p. K is uniform inside the mesh, so A_p depends only
// on how the mesh boundary cuts the patch: 7 cases per axis (centre -1, 0, 1, interior,
// n - 1, n, n + 1), 49 inverses per sample and mesh, each [27][27] with identity rows
// for the slots outside the mesh or held. kPatchTypes * kPatchDofs^2 floats per sample.
constexpr int kPatchTypes = 49;
constexpr int kPatchDofs = 27;
cudaError_t launch_patch_setup(const PGrid& g, const float* ke, int n_samples, float* pinv, cudaStream_t st);
// one colour step (in null: zero); in and out are different buffers. The residual uses
// each sample's own element matrix ke; the patch inverses are each sample's
// (pinv_per_sample) or one set shared by all samples (those of the pristine laminate:
// the perturbed samples' patches differ from it by a few per cent, which a smoother
// tolerates, and the setup is once per mesh instead of per sample)
cudaError_t launch_patch_color(const PGrid& g, const float* ke, const float* pinv, bool pinv_per_sample,
                               const float4* b, const float4* in, float4* out, int sx, int sy, const int* active,
                               cudaStream_t st);

// Coarsest mesh: dense inverse of K on the free DOFs (free[k] = 4 node + c), one per
// sample of ke; the solve applies inverse s to entry s, or one inverse to every entry
// with shared
cudaError_t launch_coarse_setup(const PGrid& g, const float* ke, int n_samples, const int* free, int nf, float* ainv,
                                cudaStream_t st);
cudaError_t launch_coarse_solve(const PGrid& g, const float* ainv, const int* free, int nf, const float4* b,
                                float4* x, const int* active, bool shared, cudaStream_t st);

// LOBPCG state of a solve (per sample unless noted).
struct Eig {
  double* gram;     // [n][2][kGram]: K and G Gram matrices of [X0 X1 W0 W1 P0 P1]
  double* coef;     // [n][kSub][kCols]: Ritz coefficients
  double* mu;       // [n][kCols]
  double* energy;   // [n][2]: x^T K x, x^T G x of the final vector (double)
  double* eta2;     // [n]: (w^T K w) / (mu^2 x^T K x) of the first column at the latest test
  int* active;      // [n]
  int* iters;       // [n]
  int* count;       // [1] samples still active after the latest Rayleigh-Ritz
};

// X (both columns) from a fixed pseudo-random w field: X = G Z (to be preconditioned)
cudaError_t launch_init_start(const PGrid& g, float4* z, cudaStream_t st);
// R = G X - mu K X per column
cudaError_t launch_residual(const PGrid& g, const Eig& E, const float4* kx, const float4* gx, float4* r,
                            cudaStream_t st);
// The Rayleigh-Ritz vector sets: v[0..2] = X, W, P; v[3..5] = K X, K W, K P;
// v[6..8] = G X, G W, G P, each [n][kCols][nodes].
struct Vecs {
  float4* v[9];
};
cudaError_t launch_gram(const PGrid& g, const Eig& E, const Vecs& v, cudaStream_t st);
// Rayleigh-Ritz per sample; convergence test on the preconditioned residual W of the
// current iterate (its K norm against mu times X's); bumps count
cudaError_t launch_rayleigh_ritz(const Eig& E, int n, double tol, int max_iter, bool first, cudaStream_t st);
// X and P from the Ritz coefficients (their K and G images are recomputed by the caller:
// carried along as combinations they drift in single precision). two_part: combined in
// double, X's w kept as high (x) plus low (w) float (thin plates)
cudaError_t launch_update(const PGrid& g, const Eig& E, const Vecs& v, bool two_part, cudaStream_t st);
// energies of column 0 in double with the double element matrices
cudaError_t launch_energy(const PGrid& g, const double* ke64, const float4* x, const Eig& E, cudaStream_t st);
// q[n][2] = (P [kN], P < p_star); status from the iteration cap and the energies
cudaError_t launch_panel_qoi(const Eig& E, int n, double ly, double p_star, int max_iter, double* q, int* status,
                             cudaStream_t st);

}  // namespace mlmcp
