/*
 * mlmc3d.h - C ABI of the 3D fibre-waviness block (the strip problem of mlmc.h
 * generalised to trilinear Hex8 elements), same library as mlmc.h.
 *
 * What the library computes. For sample j of level l it draws the KL coefficients
 * xi^(j) from the counter stream keyed by (seed, l) exactly as mlmc.h does (Eq.
 * inftyKL), synthesises the out-of-plane waviness angle theta(x, z) at the centroids
 * of the element columns of mesh l and mesh l-1 from the SAME xi (Sec. 2.2, Eq.
 * MLMC_defn; theta is constant through y), rotates the orthotropic ply stiffness of
 * every element about the y axis by its angle (Sec. 3.1, C* = T^-1 C T, here the
 * rotation of the fourth-order tensor by R_y(theta), whose first column (cos t, 0,
 * -sin t) is the fibre direction), solves K d = f on both meshes (Eq. matrixinplane in
 * 3D: 3 DOF per node, 2x2x2 Gauss), extracts the quantities of interest and folds
 * Y_l = Q_l - Q_{l-1} into per-level moments (Eq. varianceestim).
 *
 * Problem: the block [0, lx] x [0, ly] x [0, lz] meshed by cube elements of side
 * lx / nx, level l having (nx0, ny0, nz0) * 2^l elements (h halved per level, Sec.
 * 2.3, m = 8). u = v = w = 0 on x = 0; u = -shortening on x = lx with v, w free; the
 * other faces traction free.
 *
 * Quantities of interest (n_qoi = 2, in this order):
 *   0  reaction: compressive end force, -sum over the u-DOFs on x = lx of (K d)_i [N],
 *      evaluated in its energy-consistent form (equal at the discrete solution);
 *   1  stress: max over elements whose centroid x lies in [omega_x0, omega_x1] of
 *      max(0, -sigma_fibre) at the centroid, sigma_fibre = a1 . sigma a1 [Pa].
 *
 * Solver: FP32 matrix-free operator inside a batched geometric-multigrid (V(1,1),
 * damped Jacobi, full weighting, trilinear prolongation, rediscretised coarse
 * operators, dense coarsest solve) preconditioned CG, with the refinement residual in
 * double, until ||f - K d|| <= rtol ||f|| per sample.
 *
 * Memory, streams and errors as in mlmc.h: array arguments may be host or device
 * memory of the context's GPU; work is issued on the context's stream and the calls
 * return after it finished; every call returns an mlmc_status and none aborts.
 */
#ifndef MLMC3D_H
#define MLMC3D_H

#include <stdint.h>

#include "mlmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlmc3d_ctx mlmc3d_ctx;

typedef struct {
  double lx, ly, lz;          /* block dimensions; lx / nx0 = ly / ny0 = lz / nz0 (cube elements) */
  int32_t nx0, ny0, nz0;      /* level-0 mesh (even, halving down to a coarsest mesh of <= 192 DOFs) */
  int32_t levels;             /* MLMC levels (meshes 0 .. levels-1) */
  double E11, E22, E33, G12, G13, G23, nu12, nu13, nu23;   /* orthotropic ply constants, Pa */
  int32_t kl_terms;           /* N_KL of theta(x, z), 1 .. 512 */
  double kl_std;              /* standard deviation of theta, radians */
  double kl_corr;             /* correlation length of the squared-exponential kernel */
  int32_t kl_quad;            /* Gauss-Legendre points per axis, 8 .. 512 */
  double shortening;
  double omega_x0, omega_x1;  /* central region of the stress quantity */
  uint64_t seed;
  double rtol;                /* relative residual ||f - K d|| / ||f|| to reach */
  int32_t max_iter;           /* PCG iterations per refinement step (0: 200) */
  int32_t max_outer;          /* refinement steps (0: 8) */
} mlmc3d_config;

/* Validates cfg, builds the KL bases of all meshes and the rotated-stiffness
   expansion. cuda_stream: a cudaStream_t (NULL = legacy default stream).
   Errors: MLMC_ERR_INVALID_ARG, MLMC_ERR_CUDA. */
mlmc_status mlmc3d_create(const mlmc3d_config* cfg, void* cuda_stream, mlmc3d_ctx** out);
void mlmc3d_destroy(mlmc3d_ctx* ctx);
/* Message of the last failure on ctx (or of the last failed create when ctx is NULL). */
const char* mlmc3d_last_error(const mlmc3d_ctx* ctx);

/* Level pair (Sec. 2.2, Eq. MLMC_defn): samples first_id .. first_id + n - 1 of level
   `level`. Writes q_fine[n * 2] (Q_l), q_coarse[n * 2] (Q_{l-1}, zeros on level 0),
   status[n] (nullable: 0 or MLMC_ERR_NOT_CONVERGED) and folds Y of the converged
   samples into the level's moments. n = 0 is a no-op. */
mlmc_status mlmc3d_sample_level(mlmc3d_ctx* ctx, int32_t level, uint64_t first_id, int64_t n, double* q_fine,
                                double* q_coarse, int32_t* status);

/* n independent solves of (level, mesh_level, sample_id) items; q[n * 2], status[n]
   (nullable). Does not touch the moments. */
mlmc_status mlmc3d_solve_batch(mlmc3d_ctx* ctx, const mlmc_item* items, int64_t n, double* q, int32_t* status);

mlmc_status mlmc3d_level_stats_get(mlmc3d_ctx* ctx, int32_t level, mlmc_level_stats* out);
mlmc_status mlmc3d_reset_stats(mlmc3d_ctx* ctx);

/* theta[n][nx * nz] (column (i, k) at k * nx + i) of samples first_id.. of `level`
   on mesh `mesh_level`, as synthesised for the solves (FP32 synthesis). */
mlmc_status mlmc3d_theta(mlmc3d_ctx* ctx, int32_t mesh_level, int32_t level, uint64_t first_id, int64_t n,
                         double* theta);

/* y = K x on mesh `mesh_level` for n samples with given column angles theta[n][nx*nz]
   (FP32 operator, every DOF, no boundary conditions). x, y: [n][nodes][4] floats
   (u, v, w, unused), node = (k (ny+1) + j) (nx+1) + i. */
mlmc_status mlmc3d_apply(mlmc3d_ctx* ctx, int32_t mesh_level, int64_t n, const double* theta, const float* x,
                         float* y);

/* Timing of the FP32 operator alone: mean device time (ms) of one application to n
   samples of mesh mesh_level (theta = 0, device-resident data), over `reps` launches
   timed with CUDA events on the context's stream after one warm-up launch. *bytes
   receives the launch's algorithmic DRAM bytes (x read once and y written once per
   node, 16 bytes each; 16 bytes of column data per element column) and *flops its
   floating-point operations (the element operator's count times the elements).
   Outputs nullable except ms. */
mlmc_status mlmc3d_apply_bench(mlmc3d_ctx* ctx, int32_t mesh_level, int64_t n, int32_t reps, double* ms,
                               double* bytes, double* flops);

/* PCG iterations of the last solve (maximum over samples, all refinement steps). */
mlmc_status mlmc3d_last_iters(mlmc3d_ctx* ctx, int32_t* iters);

#ifdef __cplusplus
}
#endif

#endif /* MLMC3D_H */
