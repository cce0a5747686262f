// Internal interfaces of the 3D Hex8 block engine (fibre waviness, cube elements).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mlmc3 {

// Rotated stiffness about y: the 13 entries a monoclinic (x-z symmetry plane) 6x6
// stiffness can hold, Voigt (11, 22, 33, 23, 13, 12), in this order:
// C11 C12 C13 C15 C22 C23 C25 C33 C35 C44 C46 C55 C66. Each entry is a trigonometric
// polynomial of the angle: e = h0 + h1 cos 2t + h2 sin 2t + h3 cos 4t + h4 sin 4t.
constexpr int kEntries = 13;
struct Harmonics {
  float f[kEntries][5];
  double d[kEntries][5];
};

// Floating-point operations of one element application (an FMA counts 2): stiffness
// entries 104, edge differences 72, three gradient interpolations 144, stresses and
// fluxes at the 8 Gauss points 368, three transposed interpolations 144, nodal
// accumulation 144.
constexpr double kElementFlops = 976.0;

// Jacobi damping: the V-cycle is SPD for omega < 2 / lambda_max(D^-1 K), and lambda_max <= 5.4
// over all angle fields (4.3 - 4.6 on 3-degree waviness), so 0.35 holds for every field
constexpr float kOmega3 = 0.35f;
constexpr int kMaxCoarse3 = 192;         // DOFs of the coarsest mesh (dense inverse in shared memory)

// One mesh of one solve group: nsamp samples on nx x ny x nz cube elements of side h.
// Vectors are [sample][node][4] (u, v, w, unused), node = (k (ny+1) + j) (nx+1) + i;
// element-column data [sample][k][i][4] = (cos 2t, sin 2t, cos 4t, sin 4t).
struct Grid3 {
  int nx, ny, nz, nsamp;
  float h;
  __host__ __device__ int64_t nodes() const { return (int64_t)(nx + 1) * (ny + 1) * (nz + 1); }
  __host__ __device__ int64_t elems() const { return (int64_t)nx * ny * nz; }
  __host__ __device__ int64_t cols() const { return (int64_t)nx * nz; }
};

// Per-sample solver state.
struct State3 {
  double *rz, *rz_old, *pq, *rr, *rr0, *rrf, *tol2, *alpha, *beta;
  double *react, *dr, *stress;
  int *active, *outer_active, *iters, *status, *count;
};

cudaError_t set_harmonics(const Harmonics& H);

// (c2, s2) per column -> (c2, s2, c4, s4); coarse columns average their four children
cudaError_t launch_expand_trig(const float* trig2, int64_t n_cols_total, float* trig4, cudaStream_t st);
cudaError_t launch_average_trig(const Grid3& fine, const float* tf, float* tc, cudaStream_t st);
// Dinv = omega / diag(K) per DOF, zero on prescribed DOFs
cudaError_t launch_dinv(const Grid3& g, const float* trig4, float4* dinv, cudaStream_t st);
// y += K x (FP32, every DOF, unmasked); only samples with active[s] (null: all); with
// energy set also energy[s] += x . K x (summed over elements)
cudaError_t launch_apply(const Grid3& g, const float* trig4, const float4* x, float4* y, const int* active,
                         cudaStream_t st, double* energy = nullptr);
// y += K d for the float-float iterate d ([sample][node][8] floats: u, v, w as (hi, lo)),
// float-float element arithmetic summed into y in double ([sample][node][4] doubles);
// with boundary only the last element column (the x = lx nodes' complete sums)
cudaError_t launch_apply_df(const Grid3& g, const float* trig4, const float* d, double* y, const int* active,
                            bool boundary, cudaStream_t st);
cudaError_t launch_coarsest_setup(const Grid3& g, const float* trig4, float* ainv, cudaStream_t st);
cudaError_t launch_coarsest_solve(const Grid3& g, const float* ainv, const float4* b, float4* x, const int* active,
                                  cudaStream_t st);
// V-cycle pieces (masked on prescribed DOFs)
cudaError_t launch_smooth_first(const Grid3& g, const float4* dinv, const float4* b, float4* x, float4* t,
                                const int* active, cudaStream_t st);
cudaError_t launch_restrict(const Grid3& fine, const float4* bf, const float4* tf, const Grid3& coarse,
                            const float4* dinv_c, float4* bc, float4* xc, float4* tc, const int* active,
                            cudaStream_t st);
cudaError_t launch_prolong(const Grid3& fine, const float4* xc, float4* xf, float4* tf, const int* active,
                           cudaStream_t st);
// x += Dinv (b - t); with rz set, rz[s] += b . x (the PCG's r . z)
cudaError_t launch_post(const Grid3& g, const float4* dinv, const float4* b, const float4* t, float4* x,
                        double* rz, const int* active, cudaStream_t st);
// PCG
cudaError_t launch_beta(const State3& S, int n, int first, cudaStream_t st);
cudaError_t launch_update_p(const Grid3& g, const State3& S, const float4* z, float4* p, float4* q, cudaStream_t st);
cudaError_t launch_dot_pq(const Grid3& g, const State3& S, const float4* p, const float4* q, cudaStream_t st);
cudaError_t launch_alpha(const State3& S, int n, cudaStream_t st);
cudaError_t launch_update_xr(const Grid3& g, const State3& S, const float4* p, const float4* q, float4* x, float4* r,
                             cudaStream_t st);
cudaError_t launch_check(const State3& S, int n, int it, int max_iter, int slot, cudaStream_t st);
// refinement
cudaError_t launch_lift(const Grid3& g, double shortening, float* d, float4* xl, cudaStream_t st);
cudaError_t launch_lift_resid(const Grid3& g, const State3& S, const float4* t, float4* r, cudaStream_t st);
cudaError_t launch_update_d(const Grid3& g, const State3& S, const float4* x, float* d, cudaStream_t st);
// r = -(K d) on free DOFs from kd, ||r||^2
cudaError_t launch_resid_exact(const Grid3& g, const State3& S, const double* kd, float4* r, cudaStream_t st);
// reaction from the boundary column's kd, d_F . r_F from the latest residual
cudaError_t launch_final(const Grid3& g, const State3& S, const double* kd, const float* d, const float4* r,
                         cudaStream_t st);
cudaError_t launch_inner_begin(const State3& S, int n, double rtol, double floor_tol, int outer, cudaStream_t st);
cudaError_t launch_outer_check(const State3& S, int n, double rtol, int* outer_count, cudaStream_t st);
cudaError_t launch_stress(const Grid3& g, const State3& S, const float* trig4, const float* d, double x0, double x1,
                          cudaStream_t st);
cudaError_t launch_qoi(const State3& S, int n, double shortening, double* q, int* status, cudaStream_t st);
cudaError_t launch_zero4(float4* v, int64_t n, cudaStream_t st);
cudaError_t launch_combine_status(int* a, const int* b, int n, cudaStream_t st);

}  // namespace mlmc3
