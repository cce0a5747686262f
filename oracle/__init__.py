"""Plain, slow, double-precision CPU oracle for the MLMC level-pair hot path.

TEST INFRASTRUCTURE ONLY. Nothing in the product library uses this package: only
the tests, the smoke check and the benchmark's CPU-baseline leg may import it.
It shares no code, constants generator or table with the CUDA path.

Modules
  rng       Philox4x32-10 counter generator, own natural logarithm, Marsaglia polar
            normals: the KL coefficients xi of one (seed, level, sample id).
  kl        Nystrom discretisation of the squared-exponential covariance and the
            truncated KL expansion theta = sum_n sqrt(mu_n) phi_n xi_n (Eq. inftyKL).
  material  Plane-strain orthotropic stiffness and its rotation by the local
            misalignment angle (Sec. 3.1, C* = T^-1 C T).
  fem       Bilinear Q1 assembly K d = f (Eq. matrixinplane), Dirichlet lifting,
            sparse direct solve, quantities of interest.
  mlmc      Level differences Y_l = Q_l - Q_{l-1} on identical xi (Eq. MLMC_defn),
            sample moments (Eq. varianceestim), optimal N_l (Eq. optimal_Nl), bias
            estimate (Eq. bias_estimate) and Algorithm 1.
"""
