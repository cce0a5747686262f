// KL basis of the misalignment field at element centroids (host, double precision).
//
// The covariance of the strip workloads is the separable squared-exponential kernel
// k(x, y) = s^2 exp(-(x1 - y1)^2 / (2 l^2)) exp(-(x2 - y2)^2 / (2 l^2)) (the paper's
// Eq. covarianceFunction is the exponential kernel, also separable). Its
// eigenpairs are products of the eigenpairs of the two 1D integral operators
// (Eq. inftyKL: mu_n, phi_n). Each 1D operator is discretised by the Nystrom
// method on Gauss-Legendre points: the symmetric matrix W^1/2 K W^1/2 is
// diagonalised by cyclic Jacobi rotations, phi(x_q) = v_q / sqrt(w_q), and values at
// other points come from the Nystrom interpolant phi(x) = (1/mu) sum_q w_q k(x, x_q) phi(x_q).
//
// Conventions fixed here: each 1D eigenfunction is positive at the quadrature node
// nearest its interval's origin; 2D modes are ranked by mu_x * mu_y descending, ties
// by (i + j, i) ascending; B[e][n] = s sqrt(mu_x mu_y) phi_x(cx_e) phi_y(cy_e).
#include <algorithm>
#include <cmath>
#include <tuple>

#include "engine.h"

namespace mlmc {

namespace {

// n-point Gauss-Legendre rule on [-1, 1]: roots of P_n by Newton's method from
// the asymptotic guess cos(pi (i + 3/4) / (n + 1/2)); weights 2 / ((1 - x^2) P_n'(x)^2).
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 0.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) p0 = 1.0;
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    // recompute derivative at the converged root
    double p0 = 1.0, p1 = z;
    for (int k = 2; k <= n; ++k) {
      const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
      p0 = p1;
      p1 = p2;
    }
    dp = n * (z * p1 - p0) / (z * z - 1.0);
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Cyclic Jacobi eigen-decomposition of a symmetric n x n matrix (row-major, in place).
// On return A's diagonal holds the eigenvalues and V's columns the eigenvectors.
void jacobi_eigen(int n, std::vector<double>& A, std::vector<double>& V) {
  V.assign((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;
  auto a = [&](int i, int j) -> double& { return A[(size_t)i * n + j]; };
  for (int sweep = 0; sweep < 40; ++sweep) {
    double off = 0.0, diag = 0.0;
    for (int i = 0; i < n; ++i) {
      diag += a(i, i) * a(i, i);
      for (int j = i + 1; j < n; ++j) off += a(i, j) * a(i, j);
    }
    if (off <= 1e-32 * diag) break;
    for (int p = 0; p < n - 1; ++p) {
      for (int q = p + 1; q < n; ++q) {
        const double apq = a(p, q);
        if (std::fabs(apq) < 1e-300) continue;
        const double app = a(p, p), aqq = a(q, q);
        const double tau = (aqq - app) / (2.0 * apq);
        const double t = (tau >= 0.0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t), s = t * c;
        for (int k = 0; k < n; ++k) {
          const double akp = a(k, p), akq = a(k, q);
          a(k, p) = c * akp - s * akq;
          a(k, q) = s * akp + c * akq;
        }
        for (int k = 0; k < n; ++k) {
          const double apk = a(p, k), aqk = a(q, k);
          a(p, k) = c * apk - s * aqk;
          a(q, k) = s * apk + c * aqk;
        }
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
    }
  }
}

struct Eig1D {
  std::vector<double> x, w, mu;
  std::vector<double> phi;   // [q][i] at nodes
  int n;
};

Eig1D eig_1d(double a, double corr, int nq) {
  Eig1D r;
  r.n = nq;
  std::vector<double> gx, gw;
  gauss_legendre(nq, gx, gw);
  r.x.resize(nq);
  r.w.resize(nq);
  for (int q = 0; q < nq; ++q) {
    r.x[q] = (gx[q] + 1.0) * 0.5 * a;
    r.w[q] = gw[q] * 0.5 * a;
  }
  std::vector<double> A((size_t)nq * nq);
  const double inv2l2 = 1.0 / (2.0 * corr * corr);
  for (int p = 0; p < nq; ++p)
    for (int q = 0; q < nq; ++q) {
      const double d = r.x[p] - r.x[q];
      A[(size_t)p * nq + q] = std::sqrt(r.w[p]) * std::exp(-d * d * inv2l2) * std::sqrt(r.w[q]);
    }
  std::vector<double> V;
  jacobi_eigen(nq, A, V);
  std::vector<int> order(nq);
  for (int i = 0; i < nq; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int i, int j) {
    return A[(size_t)i * nq + i] > A[(size_t)j * nq + j];
  });
  r.mu.resize(nq);
  r.phi.assign((size_t)nq * nq, 0.0);
  // node nearest the origin of the interval (the smallest x)
  int q0 = 0;
  for (int q = 1; q < nq; ++q)
    if (r.x[q] < r.x[q0]) q0 = q;
  for (int k = 0; k < nq; ++k) {
    const int i = order[k];
    r.mu[k] = A[(size_t)i * nq + i];
    const double sgn = V[(size_t)q0 * nq + i] < 0.0 ? -1.0 : 1.0;
    for (int q = 0; q < nq; ++q) r.phi[(size_t)q * nq + k] = sgn * V[(size_t)q * nq + i] / std::sqrt(r.w[q]);
  }
  return r;
}

// phi_mode at point px by Nystrom interpolation.
double eval_1d(const Eig1D& e, double corr, int mode, double px) {
  const double inv2l2 = 1.0 / (2.0 * corr * corr);
  double acc = 0.0;
  for (int q = 0; q < e.n; ++q) {
    const double d = px - e.x[q];
    acc += e.w[q] * std::exp(-d * d * inv2l2) * e.phi[(size_t)q * e.n + mode];
  }
  return acc / e.mu[mode];
}

}  // namespace

bool build_kl_bases(const mlmc_config& cfg, std::vector<KLBasis>& out, std::string& msg) {
  const int nq = cfg.kl_quad, nkl = cfg.kl_terms;
  if (nq < 8 || nq > 512) {
    msg = "kl_quad must be in [8, 512]";
    return false;
  }
  const Eig1D ex = eig_1d(cfg.lx, cfg.kl_corr, nq);
  const Eig1D ey = eig_1d(cfg.ly, cfg.kl_corr, nq);
  // rank products; only the first nkl + 1 1D modes of each axis can enter the top nkl
  const int mx = std::min(nq, nkl + 1), my = std::min(nq, nkl + 1);
  std::vector<std::tuple<double, int, int, int>> cand;
  cand.reserve((size_t)mx * my);
  for (int i = 0; i < mx; ++i)
    for (int j = 0; j < my; ++j) cand.emplace_back(-(ex.mu[i] * ey.mu[j]), i + j, i, j);
  std::sort(cand.begin(), cand.end());
  if ((int)cand.size() < nkl) {
    msg = "kl_terms exceeds the number of available modes";
    return false;
  }
  std::vector<int> mi(nkl), mj(nkl);
  std::vector<double> amp(nkl);
  for (int n = 0; n < nkl; ++n) {
    mi[n] = std::get<2>(cand[n]);
    mj[n] = std::get<3>(cand[n]);
    const double prod = ex.mu[mi[n]] * ey.mu[mj[n]];
    if (!(prod > 0.0)) {
      msg = "kl_terms reaches eigenvalues at rounding level";
      return false;
    }
    amp[n] = cfg.kl_std * std::sqrt(prod);
  }
  int maxi = 0, maxj = 0;
  for (int n = 0; n < nkl; ++n) {
    maxi = std::max(maxi, mi[n]);
    maxj = std::max(maxj, mj[n]);
  }
  out.clear();
  for (int l = 0; l < cfg.levels; ++l) {
    KLBasis b;
    b.nx = cfg.nx0 << l;
    b.ny = cfg.ny0 << l;
    b.n_kl = nkl;
    const double hx = cfg.lx / b.nx, hy = cfg.ly / b.ny;
    // separable evaluation: phi_x at the nx centroid abscissae, phi_y at the ny ordinates
    std::vector<double> fx((size_t)b.nx * (maxi + 1)), fy((size_t)b.ny * (maxj + 1));
    for (int i = 0; i < b.nx; ++i)
      for (int m = 0; m <= maxi; ++m) fx[(size_t)i * (maxi + 1) + m] = eval_1d(ex, cfg.kl_corr, m, (i + 0.5) * hx);
    for (int j = 0; j < b.ny; ++j)
      for (int m = 0; m <= maxj; ++m) fy[(size_t)j * (maxj + 1) + m] = eval_1d(ey, cfg.kl_corr, m, (j + 0.5) * hy);
    b.B.resize((size_t)b.nx * b.ny * nkl);
    for (int j = 0; j < b.ny; ++j)
      for (int i = 0; i < b.nx; ++i) {
        double* row = &b.B[((size_t)j * b.nx + i) * nkl];
        for (int n = 0; n < nkl; ++n)
          row[n] = amp[n] * fx[(size_t)i * (maxi + 1) + mi[n]] * fy[(size_t)j * (maxj + 1) + mj[n]];
      }
    out.push_back(std::move(b));
  }
  return true;
}

}  // namespace mlmc
