/*
 * mlmc.h - C ABI of the GB300 level-pair engine for multilevel Monte Carlo on
 * composite strips with random fibre misalignment (Dodwell et al., MLMC
 * simulations of composite structures with uncertain manufacturing defects).
 *
 * What the library computes. For sample j of level l it draws the KL
 * coefficients xi^(j) (independent standard normals, Eq. inftyKL) from the
 * counter stream keyed by (seed, l), synthesises the misalignment field
 * theta = sum_n sqrt(mu_n) phi_n xi_n at the element centroids of mesh l and of
 * mesh l-1 from the SAME xi (Sec. 2.2, Eq. MLMC_defn), rotates each element's
 * orthotropic plane-strain stiffness by its angle (Sec. 3.1, C* = T^-1 C T),
 * solves K d = f (Eq. matrixinplane) on both meshes, extracts the quantities of
 * interest and forms Y_l = Q_l - Q_{l-1} (Y_0 = Q_0), which it folds into
 * per-level running moments (Eq. varianceestim). mlmc_estimate drives
 * Algorithm 1 on top.
 *
 * Quantities of interest (n_qoi = 2, in this order):
 *   0  reaction: compressive end force per unit depth, -sum over the u-DOFs on
 *      x = lx of (K d)_i  [N/m];
 *   1  stress: max over elements whose centroid x lies in [omega_x0, omega_x1]
 *      of max(0, -sigma_11^fibre) at the centroid [Pa].
 *
 * Memory. Every array argument is caller-owned and may be host memory or device
 * memory of the context's GPU (the library checks with cudaPointerGetAttributes
 * and copies as needed). Device work is issued on the stream given to
 * mlmc_create; calls return after that stream has finished the call's work. On a
 * stream other than the legacy default stream the multigrid-PCG iterations are
 * captured once per solve into a CUDA graph and replayed (fewer launch gaps).
 * The context owns its device workspace, the KL bases and the mesh hierarchy.
 *
 * Errors. Every call returns an mlmc_status; none aborts. On failure
 * mlmc_last_error(ctx) gives a message. Per-sample status arrays receive 0 or
 * MLMC_ERR_NOT_CONVERGED; a sample that did not converge is left out of the
 * level moments. A context is used from one host thread at a time.
 */
#ifndef MLMC_H
#define MLMC_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlmc_ctx mlmc_ctx;

typedef enum {
  MLMC_OK = 0,
  MLMC_ERR_INVALID_ARG = 1,
  MLMC_ERR_OOM = 2,
  MLMC_ERR_CUDA = 3,
  MLMC_ERR_NOT_CONVERGED = 4,
  MLMC_ERR_TIMEOUT = 5,
  MLMC_ERR_UNIMPLEMENTED = 6
} mlmc_status;

typedef enum {
  MLMC_PREC_FP64 = 0,   /* every step in double precision */
  MLMC_PREC_MIXED = 1   /* FP32 synthesis, operator and multigrid-PCG; FP64 refinement,
                           dot products, quantities of interest and moments */
} mlmc_precision;

/* Problem and solver description (plain values, copied by mlmc_create). */
typedef struct {
  double lx, ly;            /* strip [0, lx] x [0, ly] */
  int32_t nx0, ny0;         /* level-0 mesh; level l has (nx0 << l) x (ny0 << l) elements;
                               nx0 / ny0 must be equal powers-of-two multiples of a mesh
                               that halves down to 4 x 1 or 2 x 1 (nx0 = 4 ny0 or 2 ny0) */
  int32_t levels;           /* number of MLMC levels (meshes 0 .. levels-1) */
  double E11, E22, G12, nu12, E33, nu13, nu23;   /* ply constants, Pa */
  int32_t kl_terms;         /* N_KL, 1 .. 512 */
  double kl_std;            /* standard deviation of theta, radians */
  double kl_corr;           /* correlation length of the squared-exponential kernel */
  int32_t kl_quad;          /* Gauss-Legendre points per axis, 8 .. 512 */
  double shortening;        /* prescribed end displacement magnitude at x = lx */
  double omega_x0, omega_x1;/* central region for quantity 1 */
  uint64_t seed;
  int32_t precision;        /* mlmc_precision */
  double rtol;              /* relative residual ||f - K d|| / ||f|| to reach */
  int32_t max_iter;         /* cap on PCG iterations per refinement step (0: 200) */
  int32_t max_outer;        /* cap on refinement steps (0: 8) */
  int64_t max_batch;        /* samples per device batch (0: automatic) */
  double mlmc_alpha;        /* Algorithm 1: bias rate in M (Eq. bias_estimate) */
  double mlmc_gamma;        /* Algorithm 1: cost model M^gamma (Eq. gamma) */
  double mlmc_m;            /* DOF growth per level (4 for 2D quads, Sec. 2.3) */
} mlmc_config;

/* One solve request for mlmc_solve_batch: the misalignment field of sample
   `sample_id` of level `level` (stream keyed by (seed, level)), solved on mesh
   `mesh_level` (normally level or level - 1). */
typedef struct {
  int32_t level;
  int32_t mesh_level;
  uint64_t sample_id;
} mlmc_item;

/* Running statistics of Y_l for one level (FP64, compensated). */
typedef struct {
  int64_t n;                /* converged samples folded in */
  double mean[2];           /* mean of Y per quantity */
  double m2[2];             /* sum of squared deviations (Welford/Chan) */
  double var[2];            /* m2 / n: Eq. varianceestim (1/N form) */
  double sum_qf[2];         /* sum of Q_l (fine solve) */
  double sum_qc[2];         /* sum of Q_{l-1} (coarse solve; 0 on level 0) */
  double cost;              /* modelled cost of one sample (DOFs^gamma of its solves) */
} mlmc_level_stats;

/* Creates a context: validates cfg, builds the mesh hierarchy and the KL bases
   of all levels (double precision, host, then uploaded), and allocates the
   workspace. `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
   Errors: MLMC_ERR_INVALID_ARG (bad cfg), MLMC_ERR_CUDA, MLMC_ERR_OOM. */
mlmc_status mlmc_create(const mlmc_config* cfg, void* cuda_stream, mlmc_ctx** out);

void mlmc_destroy(mlmc_ctx* ctx);

/* Message of the last failure on ctx (or of the last failed mlmc_create when
   ctx is NULL). Valid until the next call on the same context. */
const char* mlmc_last_error(const mlmc_ctx* ctx);

/* Level pair (Sec. 2.2, Eq. MLMC_defn): the n samples of level `level` with ids
   first_id .. first_id + n - 1. Writes q_fine[n * 2] (Q_l) and, for level > 0,
   q_coarse[n * 2] (Q_{l-1}; zeros on level 0), row-major [sample][quantity];
   status[n] (nullable). Folds Y = Q_l - Q_{l-1} of the converged samples into
   the level's moments. n = 0 is a no-op. */
mlmc_status mlmc_sample_level(mlmc_ctx* ctx, int32_t level, uint64_t first_id, int64_t n,
                              double* q_fine, double* q_coarse, int32_t* status);

/* Level-pair calls (mlmc_sample_level(s), mlmc_estimate) whose samples' finest
   meshes hold at least min_nodes nodes in total solve by nested iteration along
   each sample's mesh chain: mesh j starts from the sample's mesh j-1 solution,
   prolongated (Sec. 2.3: the meshes of a level pair are nested). Smaller calls,
   whose per-mesh launches would not fill the GPU, solve the fine and coarse mesh
   of every pair in one lock-stepped batch from the lifting. Both reach the same
   residual tolerance rtol. Default 4,194,304; 0 = always nested.
   Errors: MLMC_ERR_INVALID_ARG for min_nodes < 0. */
mlmc_status mlmc_set_nested_threshold(mlmc_ctx* ctx, int64_t min_nodes);

/* Launch shapes of the strip kernels and the nested-iteration switch (see
   mlmc_autotune). */
typedef struct {
  int32_t max_rows;           /* node rows per warp tile, at most (1 .. 64) */
  int32_t min_rows;           /* rows per tile when small launches split (1 .. max_rows) */
  double target_waves;        /* launches below this many resident waves split their tiles */
  int64_t nested_min_nodes;   /* as mlmc_set_nested_threshold */
  int32_t fused_bottom;       /* multigrid bottom of the mixed-precision path: 2 = the three
                                 smallest non-coarsest meshes and the coarsest solve of each
                                 hierarchy in one launch (a thread block per sample, hierarchies
                                 of five levels or more); 1 = the two smallest and the coarsest
                                 in one launch (a warp per sample); 0 = a launch per level */
  double step_ms;             /* (autotune output) time of the tuned workload with these values */
  int32_t pack_samples;       /* 1: the strip kernels tile the samples of a mesh side by side
                                 (a warp strip may hold the end of one sample and the start of
                                 the next), so narrow meshes fill their warps; 0: every warp
                                 strip holds columns of one sample */
  int32_t device_loop;        /* 1: with CUDA graphs, repeat the PCG batches and their
                                 convergence test on the device (a conditional graph node,
                                 at most max_iter / 4 batches) instead of reading the active
                                 count on the host after each batch; same iterations and
                                 results. 0 (default): host loop (measured 0.9 % faster on the
                                 5-level workload: a replay of the conditional node costs
                                 about what the host round trip did) */
  int32_t wide_strips;        /* bit mask (MLMC_WIDE_*) of the mixed path's strip kernels that
                                 hold a node pair per lane (60 output columns per warp strip,
                                 the smoother's node pairs in one thread, samples side by side
                                 at any mesh width when pack_samples is 1) instead of one node
                                 column (28 or 30 output columns per strip). Same operations;
                                 dot products summed in another order. Default: the two
                                 post-smoothing kernels (MLMC_WIDE_POST | MLMC_WIDE_POST_TOP) */
  double omega;               /* damping of the pair-block Jacobi smoother, in (0, 1). The
                                 V-cycle preconditioner is SPD for omega < 2 / lambda_max(B^-1 K)
                                 (B the smoother's block diagonal): 1/2 for every angle field
                                 (lambda_max <= 4), up to about 0.7 for fields near the fibre
                                 axis (lambda_max about 2.75 at 0 degrees, 3.2 at 45, 3.8 at 60).
                                 A call in which some sample does not converge at omega > 1/2 is
                                 solved again at 1/2, so results never depend on it. Default 0.6 */
  int64_t omega_retries;      /* (get only) solves done again at omega = 1/2 since the context
                                 was created */
} mlmc_tuning;

/* Bits of mlmc_tuning.wide_strips, one per strip kernel of the V-cycle-preconditioned CG */
#define MLMC_WIDE_PRE_TOP 1    /* CG update and pre-smoothing on the solve mesh */
#define MLMC_WIDE_PRE 2        /* restriction and pre-smoothing on a coarse mesh */
#define MLMC_WIDE_POST 4       /* prolongation and post-smoothing on a coarse mesh */
#define MLMC_WIDE_POST_TOP 8   /* prolongation and post-smoothing on the solve mesh, b . z */
#define MLMC_WIDE_SEARCH 16    /* search direction p = z + beta p and q = K p */
#define MLMC_WIDE_ALL 31

/* Times the level-pair workload {levels[k], counts[k]} (host arrays of n_req entries,
   as for mlmc_sample_levels, on sample ids far from any the caller uses) under
   candidate launch shapes and nested-iteration settings, by coordinate descent
   (nested iteration on / off, fused multigrid bottom 2 / 1 / 0, smoother damping 0.5 /
   0.6 / 0.65, each bit of wide_strips flipped, target_waves 0.75 / 1.5 / 3, max_rows 32 / 64, min_rows 4 / 6 / 8; one warm-up
   and `reps` timed calls each, the median kept; the current values are timed first and
   a candidate replaces them only when more than 1 % faster), and keeps the fastest on
   the context. The level moments are left as they were. out
   (nullable) receives the chosen values. Errors as mlmc_sample_levels. */
mlmc_status mlmc_autotune(mlmc_ctx* ctx, int32_t n_req, const int32_t* levels, const int64_t* counts, int32_t reps,
                          mlmc_tuning* out);
mlmc_status mlmc_get_tuning(mlmc_ctx* ctx, mlmc_tuning* out);
/* Errors: MLMC_ERR_INVALID_ARG for values out of range. */
mlmc_status mlmc_set_tuning(mlmc_ctx* ctx, const mlmc_tuning* t);

/* Several level pairs in one call: request k asks for counts[k] samples of level
   levels[k] with ids first_ids[k] ..; levels, first_ids and counts are HOST arrays
   of n_req entries, each level at most once per call is solved in one lock-stepped
   batch with the others (all meshes of all requests advance together). Outputs are
   concatenated in request order (q_fine, q_coarse: [sum counts][2]; status:
   [sum counts], nullable) and every request is folded into its level's moments,
   exactly as n_req calls of mlmc_sample_level would (Sec. 2.2, Eq. MLMC_defn). */
mlmc_status mlmc_sample_levels(mlmc_ctx* ctx, int32_t n_req, const int32_t* levels, const uint64_t* first_ids,
                               const int64_t* counts, double* q_fine, double* q_coarse, int32_t* status);

/* n independent solves of arbitrary (level, mesh_level, sample_id) items,
   grouped by mesh and run together. Writes q[n * 2] and status[n] (nullable).
   Does not touch the level moments. */
mlmc_status mlmc_solve_batch(mlmc_ctx* ctx, const mlmc_item* items, int64_t n,
                             double* q, int32_t* status);

/* Algorithm 1 (Sec. 2.3): adds levels from 0 until the bias estimate
   |Y_hat_L| / (m^alpha - 1) (Eq. bias_estimate) falls below sqrt(1 - theta) e,
   topping each level up to N_hat_l of Eq. optimal_Nl with e_s^2 = theta e^2
   (Eq. tausplit). Level l's samples are ids 0, 1, 2, ... in order. Uses quantity
   `qoi` (0 or 1) and starts from the context's current moments; samples a level
   already holds are reused. Writes the estimate sum_l mean(Y_l), stats[0..L]
   (array of max_level + 1) and *L_out. Returns MLMC_ERR_NOT_CONVERGED if
   max_level was reached without passing the bias test (outputs still written). */
mlmc_status mlmc_estimate(mlmc_ctx* ctx, double e, double theta, int64_t n_star,
                          int32_t max_level, int32_t qoi, double* estimate,
                          mlmc_level_stats* stats, int32_t* L_out);

/* Current moments of one level; mlmc_reset_stats clears all levels. */
mlmc_status mlmc_level_stats_get(mlmc_ctx* ctx, int32_t level, mlmc_level_stats* out);
mlmc_status mlmc_reset_stats(mlmc_ctx* ctx);

/* Host-only (no GPU work): merges the moments of two disjoint sample sets of one
   level, e.g. from two GPUs that sampled disjoint id ranges, with the pairwise
   update of Chan et al. (n = na + nb, delta = mean_b - mean_a,
   mean = mean_a + delta nb / n, m2 = m2_a + m2_b + delta^2 na nb / n). out may
   alias a or b. */
mlmc_status mlmc_merge_stats(const mlmc_level_stats* a, const mlmc_level_stats* b, mlmc_level_stats* out);

/* ---- step-level entry points (each one step of the per-sample path) ---- */

/* KL coefficients xi[n * kl_terms] (double) of samples first_id.. of `level`:
   Philox4x32-10 keyed (lo32(seed), hi32(seed) ^ (level * 0x9E3779B9)),
   counter (lo32(id), hi32(id), draw, 0); Marsaglia polar normals from exact
   uniforms (2x + 1) 2^-52 - 1, with a series logarithm and no fused
   multiply-add, so the values are bit-reproducible. */
mlmc_status mlmc_kl_coefficients(mlmc_ctx* ctx, int32_t level, uint64_t first_id, int64_t n,
                                 double* xi);

/* KL synthesis theta[n * n_el(mesh_level)] (double; computed in the context's
   precision) for samples first_id.. of `level` on mesh `mesh_level`
   (Eq. inftyKL truncated at kl_terms). Element e = j * nx + i. */
mlmc_status mlmc_theta(mlmc_ctx* ctx, int32_t level, int32_t mesh_level, uint64_t first_id,
                       int64_t n, double* theta);

/* Matrix-free operator q = K(theta) p on mesh `mesh_level` for n samples
   (Eq. matrixinplane, rows and columns of all DOFs, no boundary conditions), in
   the context's precision. theta[n * n_el], p and q [n * n_dofs], DOF 2 * node + c,
   node = j * (nx + 1) + i. */
mlmc_status mlmc_apply(mlmc_ctx* ctx, int32_t mesh_level, int64_t n, const double* theta,
                       const double* p, double* q);

/* Solve on given fields: theta[n * n_el] on mesh `mesh_level` -> q[n * 2],
   status[n] (nullable), iterations[n] (nullable, total PCG iterations). */
mlmc_status mlmc_solve_theta(mlmc_ctx* ctx, int32_t mesh_level, int64_t n, const double* theta,
                             double* q, int32_t* status, int32_t* iterations);

/* ---- allocation-free solve ----
   The paper has no counterpart to this entry point; it exists for callers that
   cannot call cudaMalloc themselves or have it called on their behalf: code that
   runs while another component owns all device memory (a server with its own
   memory pool), plugins whose host framework forbids raw device allocations, and
   latency-critical paths that must not pay for an allocation or for the implicit
   synchronisation of cudaFree.

   Same computation as mlmc_solve_theta (fields theta[n * n_el] of mesh
   `mesh_level` -> q[n * 2], status[n] nullable), but without a context: cfg is
   read for this call only (its KL fields are unused), work is issued on
   `cuda_stream`, and the call allocates no device memory. Its workspace is one
   file-scope device array of 32 MiB that every GPU which loads this library
   holds until the process exits; theta, q and status are the caller's (host or
   device memory). A request whose inputs and solver workspace do not fit in the
   32 MiB (for example more than roughly 250 samples of a 64 x 16 mesh in mixed
   precision) is rejected with MLMC_ERR_INVALID_ARG and a message naming the
   limit; nothing is computed then.

   The first call on a device looks up the array's device address with that
   device current; make that first call before any stream capture. All calls
   share the one array and every call initialises what it reads, so results do
   not depend on earlier calls, but calls whose work overlaps on the GPU (other
   streams, other host threads) race on the array: serialise them.
   mlmc_static_last_error() describes the last failure of this entry point. */
mlmc_status mlmc_solve_theta_static(const mlmc_config* cfg, void* cuda_stream, int32_t mesh_level, int64_t n,
                                    const double* theta, double* q, int32_t* status);
const char* mlmc_static_last_error(void);

/* ---- measurement ---- */

/* Operation ids of the kernel timer. */
enum {
  MLMC_OP_PCG_UPDATE_PRESMOOTH = 0, /* PCG update + finest-level smoothing + residual */
  MLMC_OP_PRESMOOTH = 1,            /* coarse-level restriction + smoothing + residual */
  MLMC_OP_POSTSMOOTH = 2,           /* coarse-level prolongation + smoothing */
  MLMC_OP_POSTSMOOTH_TOP = 3,       /* finest-level prolongation + smoothing + r.z */
  MLMC_OP_SEARCH_DIRECTION = 4,     /* p = z + beta p, q = K p, p.q */
  MLMC_OP_REFINEMENT_RESIDUAL = 5,  /* double-precision r = f - K d, reaction */
  MLMC_OP_COARSEST = 6,
  MLMC_OP_OTHER = 7,
  MLMC_OP_COUNT = 8
};

/* on != 0: from now on record CUDA events around every launch of the operations
   above (on the context's stream) and count the mesh nodes each one processes
   (active samples only); resets all counters. on == 0 stops recording. */
mlmc_status mlmc_profile_enable(mlmc_ctx* ctx, int32_t on);

/* Totals since the last mlmc_profile_enable: summed kernel time in ms, number of
   launches and nodes processed of operation `op` (each output nullable). */
mlmc_status mlmc_profile_get(mlmc_ctx* ctx, int32_t op, double* ms_total, int64_t* launches, uint64_t* nodes);

/* Per-launch-name totals since the last mlmc_profile_enable, as text lines
   "name launches total_ms" (all kernels, not only the operations above), written
   NUL-terminated into buf[cap] (truncated if longer). */
mlmc_status mlmc_profile_report(mlmc_ctx* ctx, char* buf, int64_t cap);

/* Kernel launches the library issued since the last mlmc_profile_enable. */
mlmc_status mlmc_launch_count(mlmc_ctx* ctx, int64_t* launches);

/* ---------------------------------------------------------------- serving
 *
 * A request loop on one GPU (continuous batching). Sample requests are queued on
 * the host as they arrive; `workers` host threads, each with its own context and
 * CUDA stream, repeatedly take the oldest queued requests that fit their share of
 * the device-memory budget and solve them as one lock-stepped batch
 * (mlmc_solve_batch), so requests that arrive while other batches are on the GPU
 * start in the next free worker and their work overlaps on the device. Field and
 * solver state of a batch stay on the device until it completes.
 *
 * A SELECTIVE request runs the selective refinement of one sample (Sec. 2.4,
 * Algorithm 2): the failure quantity lambda (quantity 1, the centroid fibre stress)
 * of sample (level l, id) is solved on meshes j = 0, 1, ... with the same xi; from
 * j >= 1 the sample stops at the first j with
 *   |lambda_j - lambda*| >= sr_factor * max(eps_rel |lambda_j|,
 *                                            |lambda_j - lambda_{j-1}| / (m^alpha - 1))
 * (Eq. testFailure with the sample bias estimate of Eq. sampleBias, widened by the
 * solver's error bound), or at j = l. Each further mesh is a new request of the
 * same loop. The sample's level-l and level-(l-1) values are lambda_J and
 * lambda_min(J, l-1), J the stopping mesh, and its failure indicators
 * Q_l = 1(lambda_l > lambda*), Q_{l-1} (0 for l = 0).
 *
 * With carry_iterates, a SELECTIVE sample's solve on mesh j + 1 starts from its own
 * mesh-j solution (kept on the device between its solves), so each escalation needs
 * fewer PCG iterations; every solve still ends at ||f - K d|| <= rtol ||f|| on its
 * mesh.
 *
 * Every result is that of the sample alone: no arithmetic mixes samples, so the
 * batch a request lands in does not change it beyond floating-point summation
 * order. Calls on one server are thread-safe. */
typedef struct mlmc_server mlmc_server;

#define MLMC_SR_MAX_LEVELS 16

typedef enum { MLMC_REQ_SOLVE = 0, MLMC_REQ_SELECTIVE = 1 } mlmc_request_kind;

typedef struct {
  int32_t kind;         /* mlmc_request_kind */
  int32_t level;        /* MLMC level l of the sample: its KL stream is (seed, l) */
  int32_t mesh_level;   /* SOLVE: mesh to solve on; SELECTIVE: unused */
  uint64_t sample_id;
  uint64_t tag;         /* the caller's id, returned with the result */
} mlmc_request;

typedef struct {
  uint64_t tag;
  int32_t kind, level, mesh_level;
  uint64_t sample_id;
  int32_t status;       /* 0, MLMC_ERR_NOT_CONVERGED, or an error of the batch it ran in */
  double q[2];          /* SOLVE: (reaction, stress) on mesh_level */
  int32_t stop_level;   /* SELECTIVE: mesh J where refinement stopped (<= level) */
  double lambda[MLMC_SR_MAX_LEVELS];   /* SELECTIVE: lambda_j, j = 0 .. stop_level */
  double lambda_fine, lambda_coarse;   /* SELECTIVE: level-l and level-(l-1) values */
  int32_t q_fine, q_coarse;            /* SELECTIVE: failure indicators */
  int32_t solves;       /* meshes solved for this request */
  double latency_ms;    /* from submission to completion */
  int32_t pcg_iterations[MLMC_SR_MAX_LEVELS];   /* PCG iterations of each solve, in order */
  int32_t q_mesh0;      /* SELECTIVE: failure indicator of lambda_0 (the two-level estimator's) */
} mlmc_result;

typedef struct {
  int32_t workers;            /* worker threads (each: one context, one stream) */
  int64_t max_batch;          /* requests per batch */
  double hbm_budget_bytes;    /* device memory for all workers' batches (admission) */
  double threshold;           /* lambda* of SELECTIVE requests (quantity 1) */
  double sr_factor;           /* solver-error widening of the stopping test (e.g. 2) */
  double eps_rel;             /* relative error bound of a solved lambda (e.g. 1e-6) */
  int32_t carry_iterates;     /* 1: a SELECTIVE sample keeps its solution on the device between
                                 its solves and starts each further mesh from it (bilinear
                                 prolongation, as nested iteration), in a pool of iterate slots
                                 of 1/8 of the budget (a sample that finds no free slot starts
                                 from the lifting); 0: every solve starts from the lifting */
} mlmc_server_config;

/* Failure-probability estimate from completed SELECTIVE results (host arithmetic
   only; Sec. 2.4). Per term, with x_{+1}, x_{-1} the counts of Y = +1 and Y = -1
   among N results, the biased estimates p~ = (x + k) / (N + k) (Eq.
   biased_estimator) give E[Y] = p~_{+1} - p~_{-1} and
   V[Y] = p~_{+1} + p~_{-1} - (p~_{+1} - p~_{-1})^2; level-0 terms are binomial
   (p~_{-1} = 0).
   two_level == 0: the multilevel sum over the levels present,
     sum_l E[Y_l], Y_l = Q_l - Q_{l-1} (Y_0 = Q_0);
   two_level != 0: E[Q] ~ E[Q_0] + E[Y_{L,0}] with Q_0 from the level-0 results and
     Y_{L,0} = Q_L - q_mesh0 from the results of the highest level L present (q_mesh0
     the failure indicator of the sample's mesh-0 value lambda_0, solved first by every
     SELECTIVE request; `threshold` is not used).
   Results with a nonzero status are skipped. mean[] and var[] (nullable, length
   MLMC_SR_MAX_LEVELS) receive each term's E and V (indexed by level; in the
   two-level form index 0 holds Q_0 and index L holds Y_{L,0}). */
mlmc_status mlmc_failure_estimate(const mlmc_result* results, int64_t n, double threshold, int32_t k,
                                  int32_t two_level, double* estimate, double* mean, double* var);

/* Starts the workers. cfg describes the problem (as for mlmc_create). */
mlmc_status mlmc_server_create(const mlmc_config* cfg, const mlmc_server_config* scfg, mlmc_server** out);

/* Queues n requests (copied); returns at once. A request whose single-sample
   footprint exceeds a worker's share of the budget completes with
   MLMC_ERR_OOM. */
mlmc_status mlmc_server_submit(mlmc_server* srv, const mlmc_request* reqs, int64_t n);

/* Moves up to `max` completed results into out (oldest first); *count receives
   how many. Never blocks. */
mlmc_status mlmc_server_poll(mlmc_server* srv, mlmc_result* out, int64_t max, int64_t* count);

/* Waits until every submitted request has completed, at most timeout_ms
   (MLMC_ERR_TIMEOUT after that; the requests keep running). */
mlmc_status mlmc_server_drain(mlmc_server* srv, double timeout_ms);

/* Counters since creation: batches run, meshes solved, peak bytes admitted at
   once over all workers (each output nullable). */
mlmc_status mlmc_server_counters(mlmc_server* srv, int64_t* batches, int64_t* solves, double* peak_bytes);

/* Stops the workers after their current batch and frees everything; requests
   still queued are dropped. */
void mlmc_server_destroy(mlmc_server* srv);

/* Message of the last failure of a server call or batch (creation errors: srv
   NULL). */
const char* mlmc_server_last_error(const mlmc_server* srv);

#ifdef __cplusplus
}
#endif

#endif /* MLMC_H */
