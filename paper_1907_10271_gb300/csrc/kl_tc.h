// KL synthesis on the tensor cores (mixed-precision path): theta = Xi B^T
// (Eq. inftyKL truncated at N_KL terms) as tcgen05 TF32 MMAs with FP32 accumulation
// in tensor memory, operands split hi + lo ("3xTF32") so that the product keeps
// about 21 bits: theta = Xh Bh^T + Xh Bl^T + Xl Bh^T.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <cstdint>

namespace mlmc {

constexpr int kKlTcMaxTerms = 128;   // K blocks of 32 terms held in shared memory (<= 4)

// One operand matrix [rows][kp] (K innermost) split into TF32 hi and lo parts, with
// its two TMA descriptors (128-byte swizzle, boxes of 32 terms x box_rows rows).
struct KlTcOperand {
  CUtensorMap hi, lo;
  int kp;   // padded row length (multiple of 8; terms n_kl..kp-1 are zero)
};

inline bool kl_tc_supported(int n_kl) { return n_kl >= 1 && n_kl <= kKlTcMaxTerms; }
inline int kl_tc_kpad(int n_kl) { return (n_kl + 7) / 8 * 8; }

// Rows of the per-sample operand (Xi) per tile: the MMA's N.
constexpr int kKlTcSamples = 64;
// Rows of the basis operand per tile: the MMA's M.
constexpr int kKlTcElements = 128;

// x (double, [rows][n_kl]) -> hi = tf32(x), lo = tf32(x - hi), [rows][kp] with zero
// padding; round to nearest even at 10 stored mantissa bits.
void tf32_split_host(const double* x, int64_t rows, int n_kl, int kp, float* hi, float* lo);
cudaError_t launch_tf32_split(const double* x, int64_t rows, int n_kl, int kp, float* hi, float* lo,
                              cudaStream_t st);

// TMA descriptors of device arrays hi, lo [rows][kp] (16-byte aligned); box_rows is
// kKlTcElements for the basis and kKlTcSamples for Xi.
cudaError_t make_kl_tc_operand(const float* hi, const float* lo, int64_t rows, int kp, int box_rows,
                               KlTcOperand* out);

// theta for nsamp samples on a mesh of n_el elements: out = (cos 2 theta, sin 2 theta)
// per element ([nsamp][n_el][2]) with trig2 set, else theta ([nsamp][n_el]). err is
// set to 1 if a wait inside the kernel gave up (the output is then incomplete).
cudaError_t launch_kl_synthesis_tc(const KlTcOperand& basis, const KlTcOperand& xi, int n_el, int64_t nsamp,
                                   float* out, bool trig2, int* err, cudaStream_t st);

}  // namespace mlmc
