// Per-level running moments of Y_l (device resident).
#pragma once
#include <cuda_runtime.h>

#include <cstdint>

namespace mlmc {

struct LevelAcc {
  long long n;
  double mean[2];
  double m2[2];
  double sum_qf[2], comp_qf[2];
  double sum_qc[2], comp_qc[2];
};

// Folds Y = qf - qc (qc may be null: Y = qf) of samples with status 0 into *acc.
cudaError_t launch_moments(const double* qf, const double* qc, const int* status, int64_t n, LevelAcc* acc,
                           cudaStream_t st);

}  // namespace mlmc
