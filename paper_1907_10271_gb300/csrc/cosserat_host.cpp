// Host-side mathematics of the Cosserat engine (Sec. 3.1 - 3.2), double precision.
#include "cosserat_host.h"

#include <algorithm>
#include <cmath>
#include <tuple>

namespace mlmcc {

namespace {

void inv3(const double a[9], double out[9]) {
  const double c00 = a[4] * a[8] - a[5] * a[7], c01 = a[5] * a[6] - a[3] * a[8], c02 = a[3] * a[7] - a[4] * a[6];
  const double det = a[0] * c00 + a[1] * c01 + a[2] * c02;
  out[0] = c00 / det;
  out[1] = (a[2] * a[7] - a[1] * a[8]) / det;
  out[2] = (a[1] * a[5] - a[2] * a[4]) / det;
  out[3] = c01 / det;
  out[4] = (a[0] * a[8] - a[2] * a[6]) / det;
  out[5] = (a[2] * a[3] - a[0] * a[5]) / det;
  out[6] = c02 / det;
  out[7] = (a[1] * a[6] - a[0] * a[7]) / det;
  out[8] = (a[0] * a[4] - a[1] * a[3]) / det;
}

// tensor (2 x 2, row-major) <-> vector (11, 22, 12, 21)
inline void to_mat(const double v[4], double m[4]) {
  m[0] = v[0];
  m[1] = v[2];
  m[2] = v[3];
  m[3] = v[1];
}
inline void to_vec(const double m[4], double v[4]) {
  v[0] = m[0];
  v[1] = m[3];
  v[2] = m[1];
  v[3] = m[2];
}
// out = P^T M P (transpose = true) or P M P^T
void congruence(const double P[4], const double M[4], bool transpose, double out[4]) {
  double t[4];
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double s = 0.0;
      for (int k = 0; k < 2; ++k) s += (transpose ? P[k * 2 + i] : P[i * 2 + k]) * M[k * 2 + j];
      t[i * 2 + j] = s;
    }
  for (int i = 0; i < 2; ++i)
    for (int j = 0; j < 2; ++j) {
      double s = 0.0;
      for (int k = 0; k < 2; ++k) s += t[i * 2 + k] * (transpose ? P[k * 2 + j] : P[j * 2 + k]);
      out[i * 2 + j] = s;
    }
}

}  // namespace

int n_kl(const mlmcc_config& cfg, int level) { return cfg.kl_terms0 + cfg.kl_terms_step * level; }

void fibre_constants(const mlmcc_config& c, double C[16], double D[4]) {
  const double vf = c.vf, vm = 1.0 - c.vf;
  const double E11 = vf * c.Ef + vm * c.Em;
  const double E22 = 1.0 / (vf / c.Ef + vm / c.Em);
  const double Gpar = 1.0 / (vf / c.Gf + vm / c.Gm);
  const double Gperp = vf * c.Gf + vm * c.Gm;
  // orthotropic compliance with E33 = E22, nu13 = nu12; plane strain keeps the (1, 2)
  // block of its inverse
  const double S[9] = {1.0 / E11,        -c.nu12 / E11,   -c.nu12 / E11,   -c.nu12 / E11, 1.0 / E22,
                       -c.nu23 / E22,    -c.nu12 / E11,   -c.nu23 / E22,   1.0 / E22};
  double Q[9];
  inv3(S, Q);
  for (int k = 0; k < 16; ++k) C[k] = 0.0;
  C[0] = Q[0];
  C[1] = Q[1];
  C[4] = Q[3];
  C[5] = Q[4];
  C[10] = Gpar;
  C[15] = Gperp;
  const double d2 = c.d_fibre * c.d_fibre;
  D[0] = vf * c.Ef * d2 / 16.0;
  D[1] = D[2] = 0.0;
  D[3] = vm * c.Em * d2 / 16.0;
}

void rotate_constants(const double C[16], const double D[4], double phi, double Cg[16], double Dg[4]) {
  const double cs = std::cos(phi), sn = std::sin(phi);
  const double R[4] = {cs, -sn, sn, cs};
  // T[:, k] = vec(R^T mat(e_k) R)
  double T[16];
  for (int k = 0; k < 4; ++k) {
    double e[4] = {0, 0, 0, 0}, m[4], r[4], v[4];
    e[k] = 1.0;
    to_mat(e, m);
    congruence(R, m, true, r);
    to_vec(r, v);
    for (int i = 0; i < 4; ++i) T[i * 4 + k] = v[i];
  }
  // Cg = T^T C T
  double CT[16];
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += C[i * 4 + k] * T[k * 4 + j];
      CT[i * 4 + j] = s;
    }
  for (int i = 0; i < 4; ++i)
    for (int j = 0; j < 4; ++j) {
      double s = 0.0;
      for (int k = 0; k < 4; ++k) s += T[k * 4 + i] * CT[k * 4 + j];
      Cg[i * 4 + j] = s;
    }
  congruence(R, D, false, Dg);
}

void trig_basis(const double C[16], const double D[4], double Cm[5][16], double Dm[5][4]) {
  for (int m = 0; m < 5; ++m) {
    for (int k = 0; k < 16; ++k) Cm[m][k] = 0.0;
    for (int k = 0; k < 4; ++k) Dm[m][k] = 0.0;
  }
  for (int s = 0; s < 5; ++s) {
    const double psi = 2.0 * M_PI * s / 5.0;   // 2 phi
    double Cg[16], Dg[4];
    rotate_constants(C, D, 0.5 * psi, Cg, Dg);
    const double w[5] = {0.2, 0.4 * std::cos(psi), 0.4 * std::sin(psi), 0.4 * std::cos(2 * psi),
                         0.4 * std::sin(2 * psi)};
    for (int m = 0; m < 5; ++m) {
      for (int k = 0; k < 16; ++k) Cm[m][k] += w[m] * Cg[k];
      for (int k = 0; k < 4; ++k) Dm[m][k] += w[m] * Dg[k];
    }
  }
}

void element_matrix(const double Cg[16], const double Dg[4], double h, double K[144]) {
  static const double corner[4][2] = {{-1, -1}, {1, -1}, {1, 1}, {-1, 1}};
  const double g = 1.0 / std::sqrt(3.0);
  for (int k = 0; k < 144; ++k) K[k] = 0.0;
  for (int gx = 0; gx < 2; ++gx)
    for (int gy = 0; gy < 2; ++gy) {
      const double xi = gx ? g : -g, eta = gy ? g : -g;
      double Be[4][12] = {}, Bk[2][12] = {};
      for (int a = 0; a < 4; ++a) {
        const double N = 0.25 * (1 + corner[a][0] * xi) * (1 + corner[a][1] * eta);
        const double dx = 0.25 * corner[a][0] * (1 + corner[a][1] * eta) * 2.0 / h;
        const double dy = 0.25 * corner[a][1] * (1 + corner[a][0] * xi) * 2.0 / h;
        Be[0][3 * a] = dx;          // u,x
        Be[1][3 * a + 1] = dy;      // v,y
        Be[2][3 * a] = dy;          // u,y + theta
        Be[2][3 * a + 2] = N;
        Be[3][3 * a + 1] = dx;      // v,x - theta
        Be[3][3 * a + 2] = -N;
        Bk[0][3 * a + 2] = dx;      // theta,x
        Bk[1][3 * a + 2] = dy;      // theta,y
      }
      const double wdet = 0.25 * h * h;
      for (int i = 0; i < 12; ++i)
        for (int j = 0; j < 12; ++j) {
          double s = 0.0;
          for (int p = 0; p < 4; ++p)
            for (int q = 0; q < 4; ++q) s += Be[p][i] * Cg[p * 4 + q] * Be[q][j];
          for (int p = 0; p < 2; ++p)
            for (int q = 0; q < 2; ++q) s += Bk[p][i] * Dg[p * 2 + q] * Bk[q][j];
          K[i * 12 + j] += wdet * s;
        }
    }
}

void exp_modes_1d(double a, double omega, int n, std::vector<double>& mu, std::vector<double>& w) {
  const double c = 1.0 / omega, A = 0.5 * a;
  mu.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    // the root lies strictly inside (i pi / a, (i + 1) pi / a), where f changes sign
    auto f = [&](double x) {
      return (i % 2 == 0) ? c * std::cos(x * A) - x * std::sin(x * A) : x * std::cos(x * A) + c * std::sin(x * A);
    };
    double lo = i * M_PI / a, hi = (i + 1) * M_PI / a;
    double flo = f(lo);
    for (int it = 0; it < 200 && hi - lo > 0.0; ++it) {
      const double mid = 0.5 * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      const double fm = f(mid);
      if ((fm > 0) == (flo > 0)) {
        lo = mid;
        flo = fm;
      } else {
        hi = mid;
      }
    }
    w[i] = 0.5 * (lo + hi);
    mu[i] = 2.0 * c / (w[i] * w[i] + c * c);
  }
}

double exp_mode_1d(double a, double w, int i, double x) {
  const double A = 0.5 * a, xp = x - A;
  if (i % 2 == 0) {
    const double v = std::cos(w * xp) / std::sqrt(A + std::sin(2 * w * A) / (2 * w));
    return std::cos(w * A) >= 0 ? v : -v;
  }
  const double v = std::sin(w * xp) / std::sqrt(A - std::sin(2 * w * A) / (2 * w));
  return std::sin(w * A) <= 0 ? v : -v;
}

void kl_basis(const mlmcc_config& cfg, int n, int nk, std::vector<double>& B) {
  std::vector<double> mux, wx, muy, wy;
  exp_modes_1d(cfg.L, cfg.omega1, nk + 1, mux, wx);
  exp_modes_1d(cfg.L, cfg.omega2, nk + 1, muy, wy);
  std::vector<std::tuple<double, int, int, int>> cand;
  cand.reserve((size_t)(nk + 1) * (nk + 1));
  for (int i = 0; i <= nk; ++i)
    for (int j = 0; j <= nk; ++j) cand.emplace_back(-(mux[i] * muy[j]), i + j, i, j);
  std::partial_sort(cand.begin(), cand.begin() + nk, cand.end());
  const double h = cfg.L / n;
  std::vector<double> fx((size_t)nk * n), fy((size_t)nk * n), amp(nk);
  for (int k = 0; k < nk; ++k) {
    const int i = std::get<2>(cand[k]), j = std::get<3>(cand[k]);
    amp[k] = cfg.kl_std * std::sqrt(mux[i] * muy[j]);
    for (int c = 0; c < n; ++c) {
      const double x = (c + 0.5) * h;
      fx[(size_t)k * n + c] = exp_mode_1d(cfg.L, wx[i], i, x);
      fy[(size_t)k * n + c] = exp_mode_1d(cfg.L, wy[j], j, x);
    }
  }
  B.assign((size_t)n * n * nk, 0.0);
  for (int jy = 0; jy < n; ++jy)
    for (int ix = 0; ix < n; ++ix) {
      double* row = &B[((size_t)jy * n + ix) * nk];
      for (int k = 0; k < nk; ++k) row[k] = amp[k] * fx[(size_t)k * n + ix] * fy[(size_t)k * n + jy];
    }
}

void centre_range(const mlmcc_config& cfg, int n, int* klo, int* khi) {
  const double h = cfg.L / n, lo = 0.5 * (cfg.L - cfg.omega_side), hi = 0.5 * (cfg.L + cfg.omega_side);
  const double tol = 1e-9 * cfg.L;
  *klo = n;
  *khi = -1;
  for (int k = 0; k < n; ++k)
    if (k * h >= lo - tol && (k + 1) * h <= hi + tol) {
      *klo = std::min(*klo, k);
      *khi = std::max(*khi, k);
    }
}

bool validate(const mlmcc_config& c, std::string& msg) {
  auto bad = [&](const char* m) {
    msg = m;
    return false;
  };
  if (!(c.L > 0) || !(c.omega_side > 0) || !(c.omega_side <= c.L)) return bad("need 0 < omega_side <= L");
  if (!(c.omega1 > 0) || !(c.omega2 > 0) || !(c.kl_std >= 0)) return bad("need omega1, omega2 > 0, kl_std >= 0");
  if (!(c.d_fibre > 0) || !(c.vf > 0) || !(c.vf < 1)) return bad("need d_fibre > 0 and 0 < vf < 1");
  if (!(c.Ef > 0) || !(c.Em > 0) || !(c.Gf > 0) || !(c.Gm > 0)) return bad("moduli must be positive");
  if (!(c.nu12 > -1 && c.nu12 < 0.5) || !(c.nu23 > -1 && c.nu23 < 1)) return bad("Poisson ratio out of range");
  if (!(c.R_ratio > 0) || !(c.tau_y > 0)) return bad("need R_ratio > 0 and tau_y > 0");
  if (!(c.shortening < 0)) return bad("shortening must be negative (compression)");
  if (c.n0 < 4 || (c.n0 & (c.n0 - 1))) return bad("n0 must be a power of two >= 4");
  if (c.levels < 1 || c.levels > MLMCC_MAX_LEVELS) return bad("levels out of range");
  if ((int64_t)c.n0 << (c.levels - 1) > 1024) return bad("finest mesh above 1024 x 1024 elements");
  if (c.kl_terms0 < 1 || c.kl_terms_step < 0 || n_kl(c, c.levels - 1) > 4096) return bad("KL terms out of range");
  if (!(c.rtol >= 0 && c.rtol < 1) || c.max_iter < 0) return bad("rtol must be in [0, 1), max_iter >= 0");
  // the plane-strain normal block must be positive definite
  double C[16], D[4];
  fibre_constants(c, C, D);
  if (!(C[0] > 0) || !(C[0] * C[5] - C[1] * C[4] > 0)) return bad("constituents give an indefinite stiffness");
  int klo, khi;
  centre_range(c, c.n0, &klo, &khi);
  if (khi < klo) return bad("Omega' holds no element of mesh 0");
  return true;
}

}  // namespace mlmcc
