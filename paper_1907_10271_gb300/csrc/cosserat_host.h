// Host-side mathematics of the Cosserat engine (double precision): the fibre-frame
// constitutive matrices, their rotation, the trig-basis element matrices and the
// closed-form KL modes of the exponential covariance.
#pragma once
#include <cstdint>
#include <string>
#include <vector>

#include "../../include/mlmc_cosserat.h"

namespace mlmcc {

// Fibre-frame C (4 x 4 on (11, 22, 12, 21), row-major) and D (2 x 2) from the
// constituents (Sec. 3.1; rules of mixtures, plane strain).
void fibre_constants(const mlmcc_config& cfg, double C[16], double D[4]);
// C*(phi) = T^T C T with T the map eps_global -> eps_fibre = R^T eps R, and
// D*(phi) = R D R^T, R the rotation by phi.
void rotate_constants(const double C[16], const double D[4], double phi, double Cg[16], double Dg[4]);
// Cm, Dm with C*(phi) = sum_m t_m(phi) Cm[m], D*(phi) = sum_m t_m(phi) Dm[m],
// t = (1, cos 2 phi, sin 2 phi, cos 4 phi, sin 4 phi): C* is a quartic and D* a quadratic
// form in (cos phi, sin phi), even under phi -> phi + pi, so five samples of the angle
// 2 phi on the circle determine them (a five-point discrete Fourier transform).
void trig_basis(const double C[16], const double D[4], double Cm[5][16], double Dm[5][4]);
// 12 x 12 stiffness (row-major, DOF 3 a + c of local node a = (0,0), (1,0), (1,1), (0,1))
// of a square element of side h with constant C*, D*, 2 x 2 Gauss.
void element_matrix(const double Cg[16], const double Dg[4], double h, double K[144]);

// First n eigenpairs of exp(-|x - y| / omega) on [0, a]: mu[i], w[i] (frequencies).
void exp_modes_1d(double a, double omega, int n, std::vector<double>& mu, std::vector<double>& w);
// Eigenfunction i with frequency w at x (unit norm, positive at x = 0).
double exp_mode_1d(double a, double w, int i, double x);
// B[e * n_kl + k] = s sqrt(mu_k) phi_k(centroid e) of the n x n mesh, the 2D modes
// ordered by decreasing eigenvalue (ties by i + j, then i).
void kl_basis(const mlmcc_config& cfg, int n, int n_kl, std::vector<double>& B);
// Element rows / columns k with [k h, (k + 1) h] inside the central square.
void centre_range(const mlmcc_config& cfg, int n, int* klo, int* khi);

bool validate(const mlmcc_config& cfg, std::string& msg);
int n_kl(const mlmcc_config& cfg, int level);

}  // namespace mlmcc
