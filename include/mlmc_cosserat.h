/*
 * mlmc_cosserat.h - C ABI of the Cosserat engine: the paper's first test problem as
 * published (Sec. 3, compressive strength of a composite with random fibre
 * waviness), same library as mlmc.h.
 *
 * What the library computes. For sample j of level l it draws N_KL^l = kl_terms0 +
 * kl_terms_step * l standard normals xi^(j) from the counter stream keyed by (seed, l),
 * exactly as mlmc.h draws its KL coefficients, and synthesises the misalignment angle
 * of every element, phi(e) = sum_k s_Phi sqrt(mu_k) phi_k(centroid of e) xi_k
 * (Eq. inftyKL truncated), from the exponential covariance
 * k(x, y) = s_Phi^2 exp(-|x1 - y1| / omega1 - |x2 - y2| / omega2) on [0, L]^2
 * (Eq. covarianceFunction). Its eigenpairs are separable and known in closed form:
 * per axis, with c = 1 / omega and A = L / 2, mode i (i = 0, 1, ..) has the frequency
 * w_i in (i pi / L, (i + 1) pi / L) that solves c cos(w A) = w sin(w A) (i even,
 * phi_i ~ cos(w (x - A))) or w cos(w A) = -c sin(w A) (i odd, phi_i ~ sin(w (x - A))),
 * eigenvalue 2 c / (w^2 + c^2), unit L2 norm on [0, L] and the sign that makes
 * phi_i(0) > 0; the 2D modes are the products ordered by decreasing eigenvalue (ties by
 * i + j, then i). The coarse solve of a level pair uses the first N_KL^{l-1} of the
 * same xi (Sec. 2.2).
 *
 * Model (Sec. 3.1). Plane-strain Cosserat continuum with displacements u, v and the
 * Cosserat rotation theta_3 at every node (M = 3 nnode; 8 x 8 elements give M_0 = 243):
 * strains (u,x, v,y, u,y + theta_3, v,x - theta_3) with stresses sigma = C*(phi) eps,
 * curvatures (theta_3,x, theta_3,y) with couple stresses m = D*(phi) kappa, C* and D*
 * the fibre-frame C and D rotated by the element's phi (Eq. VarCosserat). Fibre-frame
 * constants from the constituents (v_f, E_f, E_m, G_f, G_m, d, nu_12, nu_23) by the
 * rules of mixtures: E_11 = v_f E_f + (1 - v_f) E_m, E_22 = (v_f / E_f + (1 - v_f) /
 * E_m)^-1, G_par (sigma_12) = (v_f / G_f + (1 - v_f) / G_m)^-1, G_perp (sigma_21) =
 * v_f G_f + (1 - v_f) G_m, the normal block the plane-strain part of the inverse
 * orthotropic compliance, D_1 = v_f E_f d^2 / 16, D_2 = (1 - v_f) E_m d^2 / 16.
 * Bilinear Q1 elements on the uniform n x n grid of [0, L]^2, n = n0 2^l, 2 x 2 Gauss
 * (Eq. matrixinplane). Boundary: u = 0 on x = 0, u = shortening (< 0) on x = L, v = 0
 * on y = 0 and y = L.
 *
 * Quantities of interest (n_qoi = 2, in this order):
 *   0  compressive strength sigma = -(1 / |Omega'|) int_Omega' sigma_x / f*, f* the
 *      largest tau_e / tau_y, tau_e = sqrt(sigma_12^2 + (sigma_22 / R)^2) in the fibre
 *      frame, over the 2 x 2 Gauss points of the elements inside the central square
 *      Omega' of side omega_side (Eq. failureCriterion) [MPa];
 *   1  end reaction: minus the sum of (K d)_u over the nodes on x = L [N per mm depth].
 *
 * Solver: the Dirichlet values are lifted to the right-hand side and their rows and
 * columns replaced by the identity. Each solve is FP64 iterative refinement (residual
 * b - K d with the stencil assembled in double) around an FP32 conjugate-gradient
 * correction solve, preconditioned by one geometric-multigrid V(1,1) cycle: damped
 * (0.6) nodal 3 x 3 block Jacobi, bilinear transfers, Galerkin coarse operators down
 * to the 2 x 2 mesh, whose 27 x 27 operator is inverted; the meshes of at most 8 x 8
 * elements run in one fused launch, a block per sample. All meshes of one call advance
 * together. A solve stops when ||b - K d||_2 <= rtol ||b||_2; samples that do not
 * reach it within max_iter correction iterations get status MLMC_ERR_NOT_CONVERGED.
 *
 * Memory, streams and errors as in mlmc.h: array arguments may be host or device
 * memory of the context's GPU; work is issued on the context's stream and the calls
 * return after it finished; every call returns an mlmc_status and none aborts.
 */
#ifndef MLMC_COSSERAT_H
#define MLMC_COSSERAT_H
#include <stdint.h>
#include "mlmc.h"
#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlmcc_ctx mlmcc_ctx;

#define MLMCC_MAX_LEVELS 8

typedef struct {
  double L;                    /* side of the square domain, mm */
  double omega_side;           /* side of the central square Omega', mm (0 < omega_side <= L) */
  double omega1, omega2;       /* correlation lengths along x and y, mm */
  double kl_std;               /* s_Phi, rad */
  double d_fibre;              /* fibre diameter d, mm */
  double vf, Ef, Em, Gf, Gm;   /* fibre volume fraction and constituent moduli, MPa */
  double nu12, nu23;
  double R_ratio;              /* R: transverse over shear yield strength */
  double tau_y;                /* shear strength, MPa */
  double shortening;           /* end shortening Delta on x = L, mm (negative) */
  int32_t n0;                  /* level-0 mesh: n0 x n0 elements (a power of two >= 4) */
  int32_t levels;              /* MLMC levels, meshes 0 .. levels-1 (1 .. MLMCC_MAX_LEVELS) */
  int32_t kl_terms0;           /* N_KL of level 0 */
  int32_t kl_terms_step;       /* N_KL^l = kl_terms0 + kl_terms_step l */
  uint64_t seed;
  double rtol;                 /* relative residual target (0: 1e-8) */
  int32_t max_iter;            /* correction-solve iterations per sample, all refinements (0: 400) */
} mlmcc_config;

/* Validates cfg (positive lengths and moduli, 0 < vf < 1, n0 a power of two >= 4, levels and
   KL terms >= 1, the finest mesh at most 1024 x 1024 elements, Omega' holding at least
   one element of mesh 0), computes the KL modes, the fibre-frame C and D and the
   per-mesh element matrices on the host in double. cuda_stream: a cudaStream_t (NULL =
   legacy default). Errors: MLMC_ERR_INVALID_ARG, MLMC_ERR_CUDA. */
mlmc_status mlmcc_create(const mlmcc_config* cfg, void* cuda_stream, mlmcc_ctx** out);
void mlmcc_destroy(mlmcc_ctx* ctx);
/* Message of the last failure on ctx (or of the last failed create when ctx is NULL). */
const char* mlmcc_last_error(const mlmcc_ctx* ctx);

/* Level pair (Sec. 2.2, Eq. MLMC_defn): samples first_id .. first_id + n - 1 of level
   `level`. Writes q_fine[n * 2] (Q_l), q_coarse[n * 2] (Q_{l-1}, zeros on level 0),
   status[n] (nullable: 0 or MLMC_ERR_NOT_CONVERGED) and folds Y of the converged samples
   into the level's moments. n = 0 is a no-op. */
mlmc_status mlmcc_sample_level(mlmcc_ctx* ctx, int32_t level, uint64_t first_id, int64_t n, double* q_fine,
                               double* q_coarse, int32_t* status);
/* Several level pairs in one call, all meshes solved together: request k asks for
   counts[k] samples of level levels[k] with ids first_ids[k] .. (HOST arrays of n_req
   entries, each level at most once). Outputs concatenated in request order, each
   request folded into its level's moments, as n_req calls of mlmcc_sample_level. */
mlmc_status mlmcc_sample_levels(mlmcc_ctx* ctx, int32_t n_req, const int32_t* levels, const uint64_t* first_ids,
                                const int64_t* counts, double* q_fine, double* q_coarse, int32_t* status);
/* n independent solves of (level, mesh_level, sample_id) items (the field of `level`'s
   stream solved on mesh `mesh_level`, any mesh of the context); q[n * 2], status[n]
   (nullable). Does not touch the moments. */
mlmc_status mlmcc_solve_batch(mlmcc_ctx* ctx, const mlmc_item* items, int64_t n, double* q, int32_t* status);
/* Algorithm 1 (Sec. 2.3) on quantity `qoi` (0 strength, 1 reaction): adds levels from 0
   until the bias estimate |Y_hat_L| / (m^alpha - 1) (Eq. bias_estimate) falls below
   sqrt(1 - theta) e, topping each level up to N_hat_l of Eq. optimal_Nl with
   e_s^2 = theta e^2 (Eq. tausplit) and the cost of a level pair C_l = M_l^gamma +
   M_{l-1}^gamma (M the DOFs of a mesh; the paper fits gamma = 1.3 for this problem).
   Level l's samples are ids 0, 1, 2, .. in order, continuing from the samples the
   context's moments already hold (mlmcc_reset_stats starts afresh). Writes the estimate
   sum_l mean(Y_l), stats[0..L] (nullable, max_level + 1 entries) and *L_out (nullable).
   Returns MLMC_ERR_NOT_CONVERGED if max_level was reached without passing the bias test
   (outputs still written). Errors: MLMC_ERR_INVALID_ARG for e <= 0, theta outside (0, 1),
   n_star < 1, max_level < 0, qoi not 0 or 1, m <= 1, alpha <= 0, gamma <= 0. */
mlmc_status mlmcc_estimate(mlmcc_ctx* ctx, double e, double theta, int64_t n_star, int32_t max_level, int32_t qoi,
                           double m, double alpha, double gamma, double* estimate, mlmc_level_stats* stats,
                           int32_t* L_out);
mlmc_status mlmcc_level_stats_get(mlmcc_ctx* ctx, int32_t level, mlmc_level_stats* out);
mlmc_status mlmcc_reset_stats(mlmcc_ctx* ctx);

/* Misalignment angles of samples first_id .. of `level` on mesh `mesh_level`:
   phi[n][n_el] (double, element e = j n + i). */
mlmc_status mlmcc_field(mlmcc_ctx* ctx, int32_t level, int32_t mesh_level, uint64_t first_id, int64_t n,
                        double* phi);
/* y = K x for the same samples: K the stiffness with the boundary conditions applied
   (Dirichlet rows and columns replaced by the identity), assembled in double as the
   solves use it. x, y: [n][nodes][3] doubles (u, v, theta_3), node = j (n + 1) + i. */
mlmc_status mlmcc_apply(mlmcc_ctx* ctx, int32_t level, int32_t mesh_level, uint64_t first_id, int64_t n,
                        const double* x, double* y);
/* Solutions d (with the prescribed values) of the same samples: [n][nodes][3] doubles;
   status[n] nullable. */
mlmc_status mlmcc_displacement(mlmcc_ctx* ctx, int32_t level, int32_t mesh_level, uint64_t first_id, int64_t n,
                               double* d, int32_t* status);
/* Correction-solve iterations of the last solve call (maximum over samples) and the
   number of FP64 residual evaluations it took. */
mlmc_status mlmcc_last_iters(mlmcc_ctx* ctx, int32_t* iterations, int32_t* refinements);
/* Kernels this context has launched so far (graph replays count every kernel node). */
mlmc_status mlmcc_launch_count(mlmcc_ctx* ctx, int64_t* launches);
/* Per-kernel profile. While enabled (on != 0; enabling clears the totals) every launch is
   issued directly, without graphs, between two CUDA events on the context's stream, and
   calls accumulate per kernel kind `op` (0 .. mlmcc_profile_name(op) == NULL) the event
   time, the launches and the work items (threads' nodes, samples or elements). Kinds:
   kl_coefficients, kl_synthesis, build_fine, rap, coarsest_inverse, pre, restrict,
   bottom, prolong, post, cg_apply, cg_update, scalars, resid64, accumulate, qoi,
   moments, layout. */
mlmc_status mlmcc_profile_enable(mlmcc_ctx* ctx, int32_t on);
mlmc_status mlmcc_profile_get(mlmcc_ctx* ctx, int32_t op, double* ms, int64_t* launches, int64_t* items);
const char* mlmcc_profile_name(int32_t op);

#ifdef __cplusplus
}
#endif
#endif /* MLMC_COSSERAT_H */
