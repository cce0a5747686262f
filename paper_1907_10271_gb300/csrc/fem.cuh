// Device views and launchers of the matrix-free Q1 operator family.
#pragma once
#include "common.cuh"

namespace mlmc {

constexpr int kMaxViews = 12;

// One multigrid level of one solve group, as seen by a kernel. Pointer meaning
// depends on the kernel (documented at each launcher). Vectors are
// [nsamp][ny+1][nx+1][2]; element data [nsamp][ny][nx][2] on the finest mesh
// (trig2 = cos 2t, sin 2t of the element's angle) or [nsamp][ny][nx][4] on coarse
// meshes (trig = child averages of cos 2t, sin 2t, cos 4t, sin 4t).
template <typename T>
struct View {
  Geo g;
  int nsamp;
  int sbase;        // first sample of the group in the per-sample arrays
  int work_begin;   // first warp (strip kernels) or thread (pointwise kernels) of this view
  int nwork;
  int tiles_x, tiles_y;
  int rows;         // node rows per warp tile of a strip kernel (0: kRowChunk)
  // strip kernels, packed views: the samples lie side by side along one virtual row of
  // nsamp * vw node columns (vw = nx + 2: the nx + 1 real columns and one padding
  // column, so that every sample starts on an even column), and warp strips tile that
  // row, so a narrow mesh does not leave most of a sample's last strip idle;
  // tiles_x then counts the strips of the whole virtual row
  int packed;
  int vw;
  const T* trig2;
  const T* trig;
  const T* a;
  const T* b;
  const T* c;
  const T* winvd;   // smoother, per node: (u self coefficient, v coefficient), damping included
  const T* wc;      // smoother, per node: u coefficient of the pair partner (column i ^ 1)
  const T* xc;      // prolongation source (level below)
  T* o0;
  T* o1;
  T* o2;
  const void* ext0; // kernel-specific (e.g. angle array of another precision, dense inverse)
  void* ext1;
  double param;     // kernel-specific scalar (e.g. the prescribed end shortening)
};

// Operation ids of the kernel timer (mlmc_profile_get).
enum ProfOp { kProfPreTop = 0, kProfPre, kProfPost, kProfPostTop, kProfPcgP, kProfResid, kProfCoarsest,
              kProfOther, kProfOps };

template <typename T>
struct ViewList {
  int n;
  int prof_op;      // ProfOp of the launch (node counting when SampleState::units is set)
  int wide;         // laid out for the node-pair strip kernels (launch_strip_wide)
  Invariants U;
  View<T> v[kMaxViews];
};

// Per-sample solver state (structure of arrays, indexed by sbase + s).
struct SampleState {
  double* alpha;
  double* beta;
  double* rz_old;
  double* rr_ref;     // ||b||^2 of the current inner system
  double* tol2;       // inner relative tolerance squared
  double* red_rr;
  double* red_rz;
  double* red_pq;
  double* rrf;        // ||f||^2 (residual of the lifting)
  double* rr64;       // ||f - K d||^2 of the latest refinement residual
  double* react;      // sum of (K d)_u on x = lx from the latest residual
  double* qoi;        // [2] per sample
  int* active;        // inner PCG running
  int* outer_active;  // refinement running
  int* iters;         // PCG iterations (all refinement steps)
  int* status;        // 0 ok, MLMC_ERR_NOT_CONVERGED
  int* count;         // [batch] active samples after each iteration of the current batch
  int* rpar;          // buffer (0/1) holding the latest inner residual
  int* exact;         // 1: the next refinement residual is formed from d (not the inner CG's)
  unsigned* arrive;   // warps of the running launch that added their share of a sample's
                      // reduction; zero between launches (see last_tile in fem.cu)
  unsigned long long* units;   // [kProfOps] nodes processed per operation (null: not counted)
  int slot;           // the PCG iteration's position in its batch (post-smoothing launch)
};

// Strip kernels (q = K p family); see fem.cu for the operand conventions.
enum class StripOp { Apply, PreTop, PreR, Post, PostTop, PcgP };

// Output node columns per warp strip of a strip kernel (sets the views' tiles_x).
int strip_cols(StripOp op);

// The FP32 smoothing and PCG strip kernels with a node pair per lane (strip_wide.cu):
// kWideCols output node columns per warp strip, views packed at any sample width, every
// view's nx even. Same operand conventions as launch_strip.
constexpr int kWideCols = 60;
// bit of op in the node-pair mask (mlmc_tuning.wide_strips); -1: no node-pair kernel
int wide_strip_bit(StripOp op);
cudaError_t launch_strip_wide(StripOp op, const ViewList<float>& L, SampleState S, int total_warps, cudaStream_t st);

template <typename T>
cudaError_t launch_strip(StripOp op, const ViewList<T>& L, SampleState S, int total_warps, cudaStream_t st);

// Refinement residual r = -(K d) on free DOFs (double d, T output), ||r||^2 and reaction.
template <typename TI>
cudaError_t launch_resid64(const ViewList<double>& L, SampleState S, int total_warps, cudaStream_t st);

// Energy-consistent reaction correction of converged samples (see fem.cu): a = final
// refinement residual, ext0 = d (double); one warp per node row.
template <typename T>
cudaError_t launch_react_energy(const ViewList<T>& L, SampleState S, double shortening, int total_warps,
                                cudaStream_t st);

template <typename T>
cudaError_t launch_trig_average(const ViewList<T>& L, int total_threads, cudaStream_t st);

template <typename T>
cudaError_t launch_invdiag(const ViewList<T>& L, int total_threads, cudaStream_t st);

template <typename T>
cudaError_t launch_coarsest_setup(const ViewList<T>& L, int total_blocks, cudaStream_t st);

template <typename T>
cudaError_t launch_coarsest_solve(const ViewList<T>& L, SampleState S, int total_warps, cudaStream_t st);

// The bottom of a group's multigrid hierarchy in one launch (FP32): levels A = nl-3
// and B = nl-2 and the coarsest C = nl-1 of every sample, one warp per sample in
// shared memory. Does what PreR (A, B), the coarsest solve and Post (B, A) do, in
// the same order and arithmetic: b_A = R r_in, x_A = W b_A, r_A = b_A - K x_A,
// b_B = R r_A, ..., x_C = A^-1 R r_B, x_B = W b_B + P x_C, x_B += W (b_B - K x_B),
// x_A likewise; writes x_A (what Post at level nl-4 prolongates).
constexpr int kBotNodes = 96;   // nodes of level A at most
constexpr int kBotNodesB = 32;  // of level B
struct BottomView {
  Geo ga, gb, gc;
  int nsamp, sbase, work_begin;
  const float *rin;                        // level nl-4 residual [s][nodes][2]
  const float *winv_a, *wc_a, *trig_a;     // level A smoother and coarse element data
  const float *winv_b, *wc_b, *trig_b;
  const float* ainv;                       // coarsest inverses [s][n][n]
  float* xout;                             // x_A [s][nodes][2]
};
struct BottomList {
  int n;
  Invariants U;
  BottomView v[kMaxViews];
};
bool bottom_fits(const Geo& ga, const Geo& gb, const Geo& gc);
cudaError_t launch_bottom(const BottomList& L, SampleState S, int total_warps, cudaStream_t st);

// The deepest levels of a group's hierarchy with one thread block per sample (FP32):
// nb smoothed levels (finest first, each twice the next) and the coarsest, with every
// smoothed level's smoother and element data staged in shared memory; same operations
// as PreR on those levels, the coarsest solve and Post back up; writes the finest
// bottom level's correction (what Post or PostTop on the level above prolongates).
constexpr int kDeepMax = 4;          // smoothed levels at most
constexpr int kDeepThreads = 128;
constexpr int kDeepFloats = 12288;   // shared memory per block at most (48 KB)
struct DeepView {
  Geo g[kDeepMax];
  Geo gc;
  int nb, nsamp, sbase, work_begin;
  const float* rin;                  // residual of the level above g[0] [s][nodes][2]
  const float* winv[kDeepMax];
  const float* wc[kDeepMax];
  const float* trig[kDeepMax];
  const float* ainv;                 // coarsest inverses [s][n][n]
  float* xout;                       // correction on g[0] [s][nodes][2]
};
struct DeepList {
  int n;
  Invariants U;
  DeepView v[kMaxViews];
};
int deep_floats(const Geo* g, int nb, const Geo& gc);   // shared floats one block needs
bool deep_fits(const Geo* g, int nb, const Geo& gc);
cudaError_t launch_bottom_deep(const DeepList& L, SampleState S, int total_blocks, int floats, cudaStream_t st);

// d += x (a = x, ext1 = d); with o0 set also r0 = r1 where the inner residual ended
// in r1 (b = r1, o0 = r0). One thread per value.
template <typename T>
cudaError_t launch_update_d(const ViewList<T>& L, SampleState S, int total_threads, cudaStream_t st);

// Lifting d0 and its inner-precision residual on the last two node columns (d and r
// cleared by the caller): o0 = r, ext1 = d. One thread per (sample, node row, column).
template <typename T>
cudaError_t launch_lift_resid(const ViewList<T>& L, SampleState S, double shortening, int total_threads,
                              cudaStream_t st);

// Nested iteration: fine d (ext1) from the coarser mesh's d (ext0) by bilinear
// prolongation; views at the fine mesh. One thread per fine node.
template <typename TI>
cudaError_t launch_prolong_d(const ViewList<TI>& L, int total_threads, cudaStream_t st);

template <typename TI>
cudaError_t launch_stress(const ViewList<double>& L, SampleState S, int total_warps, cudaStream_t st);

// Reaction increment of the correction: react += sum_j (K x)_u at nodes (nx, j), from
// the last element column only. Views at the top level, a = x. One thread per element row.
template <typename T>
cudaError_t launch_react_delta(const ViewList<T>& L, SampleState S, int total_threads, cudaStream_t st);

// After an inner solve: samples still running hit the iteration cap (not converged);
// for the others whose next refinement residual is not formed exactly (S.exact),
// ||r||^2 of the new refinement residual is the PCG's last reduced ||r||^2.
cudaError_t launch_inner_end(SampleState S, int total, cudaStream_t st);

cudaError_t launch_outer_init(SampleState S, int total, cudaStream_t st);
cudaError_t launch_outer_check(SampleState S, int total, double rtol, double floor_tol, int* outer_count,
                               cudaStream_t st);

}  // namespace mlmc
