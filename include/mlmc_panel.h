/*
 * mlmc_panel.h - C ABI of the panel-buckling engine (Sec. 4, the second test problem),
 * same library as mlmc.h.
 *
 * What the library computes. For sample j of level l it draws n_plies standard normals
 * xi^(j) from the counter stream keyed by (seed, l), exactly as mlmc.h draws its KL
 * coefficients, and perturbs ply k of the pristine stacking sequence by
 * phi_k = ply_std * xi_k (Sec. 4.1; the same phi on both meshes of a level pair, Sec.
 * 2.2). Classical laminate theory gives A, B, D of the perturbed laminate and the
 * knocked-down bending stiffness D* = D - B^T A^-1 B (Eq. CLTABD). The Reissner-Mindlin
 * plate (Eq. momentequil, weak form Eq. MomentWeakForm) is discretised by bilinear Q4
 * elements for (w, theta_x, theta_y): bending by 2x2 Gauss with D*, transverse shear by
 * the 1-point rule with stiffness k G13 t, the geometric form int w_x w^_x of a unit
 * compressive line load N_x = 1 N/mm by the 1-point rule. The critical load is the
 * smallest lambda of K d = lambda G d (Eq. matrixeig), found as 1 / mu for the largest mu
 * of G d = mu K d.
 *
 * Panel: [0, lx] x [0, ly] mm, level l meshed by (nx0, ny0) * 2^l elements (h halved
 * per level, Sec. 2.3). Simply supported: w = 0 on the boundary; with
 * hard_support also the tangential rotation (theta_y = 0 on x = 0, lx; theta_x = 0 on
 * y = 0, ly), which is what reproduces the paper's pristine load (Sec. 4.2).
 *
 * Quantities of interest (n_qoi = 2, in this order):
 *   0  critical load P = lambda * ly [kN] (lambda in N/mm);
 *   1  failure indicator 1 if P < p_star, else 0 (Sec. 4.2's Q(lambda)).
 *
 * Solver: per sample, block LOBPCG (two vectors) on (G, K) in FP32 with FP64 Gram
 * matrices and Rayleigh-Ritz, preconditioned by one geometric-multigrid V(2,2) cycle on
 * K (nodal 3x3 block Jacobi, bilinear transfers, rediscretised coarse operators, and the
 * dense coarsest inverse of the pristine laminate shared by every sample), four
 * iterations per CUDA-graph replay. The reported lambda is the Rayleigh quotient of the
 * converged FP32 eigenvector evaluated in double, so its error is quadratic in the
 * vector's.
 *
 * Memory, streams and errors as in mlmc.h: array arguments may be host or device
 * memory of the context's GPU; work is issued on the context's stream and the calls
 * return after it finished; every call returns an mlmc_status and none aborts.
 */
#ifndef MLMC_PANEL_H
#define MLMC_PANEL_H

#include <stdint.h>

#include "mlmc.h"

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlmcp_ctx mlmcp_ctx;

#define MLMCP_MAX_PLIES 32

typedef struct {
  double lx, ly;               /* panel dimensions, mm (elements lx / nx by ly / ny) */
  int32_t nx0, ny0;            /* level-0 mesh (elements) */
  int32_t levels;              /* MLMC levels (meshes 0 .. levels-1) */
  double E11, E22, G12, nu12;  /* ply constants, MPa */
  double G13;                  /* transverse shear modulus, MPa */
  double k_shear;              /* shear correction factor (5/6) */
  int32_t n_plies;             /* 1 .. MLMCP_MAX_PLIES */
  double plies_deg[MLMCP_MAX_PLIES];   /* pristine ply angles, bottom ply first, degrees */
  double t_ply;                /* ply thickness, mm */
  double ply_std_deg;          /* standard deviation of each ply's perturbation, degrees */
  int32_t hard_support;        /* 1: tangential rotation held on the boundary; 0: free */
  double p_star;               /* failure threshold of quantity 1, kN */
  uint64_t seed;
  double tol;                  /* LOBPCG stop: (w^T K w)^1/2 <= tol mu (x^T K x)^1/2 with w the
                                  preconditioned residual of the first vector (0: 1e-4;
                                  the load error is about tol^2) */
  int32_t max_iter;            /* LOBPCG iterations (0: 120) */
  int32_t smoother;            /* multigrid smoother: 0 = damped nodal 3x3 block Jacobi, V(2,2);
                                  1 = multiplicative Schwarz on 3x3-node patches in nine
                                  colours, V(1,1), for thin plates (b / t in the hundreds),
                                  where the nodal smoother does not resolve the nearly held
                                  transverse shear; meshes of the hierarchy must then have at
                                  least 4 elements per side */
} mlmcp_config;

/* Validates cfg and builds the mesh hierarchies. The multigrid coarsens each mesh by
   halving while both element counts stay even and ny stays >= 4; the coarsest mesh must
   have at most 192 free DOFs. cuda_stream: a cudaStream_t (NULL = legacy default).
   Errors: MLMC_ERR_INVALID_ARG, MLMC_ERR_CUDA. */
mlmc_status mlmcp_create(const mlmcp_config* cfg, void* cuda_stream, mlmcp_ctx** out);
void mlmcp_destroy(mlmcp_ctx* ctx);
/* Message of the last failure on ctx (or of the last failed create when ctx is NULL). */
const char* mlmcp_last_error(const mlmcp_ctx* ctx);

/* Level pair (Sec. 2.2, Eq. MLMC_defn): samples first_id .. first_id + n - 1 of level
   `level`. Writes q_fine[n * 2] (Q_l), q_coarse[n * 2] (Q_{l-1}, zeros on level 0),
   status[n] (nullable: 0 or MLMC_ERR_NOT_CONVERGED) and folds Y of the converged
   samples into the level's moments. n = 0 is a no-op. */
mlmc_status mlmcp_sample_level(mlmcp_ctx* ctx, int32_t level, uint64_t first_id, int64_t n, double* q_fine,
                               double* q_coarse, int32_t* status);

/* n independent solves of (level, mesh_level, sample_id) items (the perturbations of
   `level`'s stream, solved on mesh `mesh_level`); q[n * 2], status[n] (nullable). Does
   not touch the moments. */
mlmc_status mlmcp_solve_batch(mlmcp_ctx* ctx, const mlmc_item* items, int64_t n, double* q, int32_t* status);

mlmc_status mlmcp_level_stats_get(mlmcp_ctx* ctx, int32_t level, mlmc_level_stats* out);
mlmc_status mlmcp_reset_stats(mlmcp_ctx* ctx);

/* Laminate of samples first_id.. of `level`: dstar[n][6] = (D*11, D*12, D*16, D*22,
   D*26, D*66) in N mm and kgt[n] = k G13 t in N/mm (nullable), as used by the solves. */
mlmc_status mlmcp_laminate(mlmcp_ctx* ctx, int32_t level, uint64_t first_id, int64_t n, double* dstar, double* kgt);

/* y = K x and g = G x on mesh `mesh_level` (FP32, every DOF, no boundary conditions)
   for n samples with the laminates of samples first_id.. of `level`. x, y, g:
   [n][nodes][4] floats (w, theta_x, theta_y, unused), node = j (nx + 1) + i; g nullable. */
mlmc_status mlmcp_apply(mlmcp_ctx* ctx, int32_t mesh_level, int32_t level, uint64_t first_id, int64_t n,
                        const float* x, float* y, float* g);

/* Times `reps` launches of the FP32 operator kernel that LOBPCG uses (K x and G x of n
   samples of level mesh_level's stream on mesh mesh_level, every DOF) between CUDA events
   on the context's stream: *ms = mean time per launch, *bytes (nullable) = its algorithmic
   bytes (x read, K x and G x written: 48 B per node; 576 B per sample's element matrix).
   n <= 65535. */
mlmc_status mlmcp_apply_bench(mlmcp_ctx* ctx, int32_t mesh_level, int64_t n, int32_t reps, double* ms, double* bytes);
/* LOBPCG iterations of the last solve (maximum over samples). */
mlmc_status mlmcp_last_iters(mlmcp_ctx* ctx, int32_t* iters);

/* ---- serving (the request loop of mlmc.h's serving section, for panel samples) ----
   Starts a request loop whose workers solve panel samples (each worker one mlmcp
   context on its own stream); mlmc_server_submit / poll / drain / counters / destroy /
   last_error then work as for the strip. SOLVE requests return (P, indicator) on their
   mesh; a SELECTIVE request runs Algorithm 2 (Sec. 2.4) on the critical load P
   (quantity 0): from mesh j >= 1 it stops at the first j with
   |P_j - p*| >= sr_factor max(eps_rel |P_j|, |P_j - P_{j-1}| / (m^alpha - 1)), and its
   failure indicators are 1(P < p*) (Sec. 4.2's Q(lambda)), p* = scfg->threshold (kN).
   mlmc_m, mlmc_alpha: the convergence constants of the bias estimate (e.g. 4 and 1).
   Every solve starts from scratch (carry_iterates is ignored); a result's
   pcg_iterations hold the LOBPCG iterations of the slowest sample of its batch. The
   workers' solver workspace is stream-ordered device allocation per batch. */
mlmc_status mlmcp_server_create(const mlmcp_config* cfg, const mlmc_server_config* scfg, double mlmc_m,
                                double mlmc_alpha, mlmc_server** out);

#ifdef __cplusplus
}
#endif

#endif /* MLMC_PANEL_H */
