// Stable Neo-Hookean energy density and its first two derivatives, FP64.
//
// TEST INFRASTRUCTURE (oracle).  The paper names the Stable Neo-Hookean model
// for 3D solids (Sec. 5.1, "Boundary conditions and materials") without
// printing it.  Reading used here:
//   psi(F) = mu/2 (tr F^T F - 3) - mu (J - 1) + lam_s/2 (J - 1)^2,   J = det F
//   mu = E / (2 (1 + nu)),  lam_s = E nu / ((1 + nu)(1 - 2 nu)) + mu
// so that the tangent at F = I is the isotropic linear-elastic tensor with the
// Lame parameters of (E, nu).
//
// Index convention: F[3*i + j] = F_ij, vec index (i, j) -> 3 i + j.
#include <cmath>

#include "ppn_oracle.h"

namespace {

// Levi-Civita symbol
int eps3(int i, int j, int k) {
  if (i == j || j == k || i == k) return 0;
  // even permutations of (0,1,2)
  if ((i == 0 && j == 1 && k == 2) || (i == 1 && j == 2 && k == 0) || (i == 2 && j == 0 && k == 1))
    return 1;
  return -1;
}

double det3(const double* F) {
  double J = 0.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k) J += eps3(i, j, k) * F[0 * 3 + i] * F[1 * 3 + j] * F[2 * 3 + k];
  return J;
}

// cof(F)_ij = dJ/dF_ij = 1/2 eps_ikm eps_jln F_kl F_mn
void cofactor(const double* F, double* C) {
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double c = 0.0;
      for (int k = 0; k < 3; ++k)
        for (int m = 0; m < 3; ++m)
          for (int l = 0; l < 3; ++l)
            for (int n = 0; n < 3; ++n)
              c += 0.5 * eps3(i, k, m) * eps3(j, l, n) * F[3 * k + l] * F[3 * m + n];
      C[3 * i + j] = c;
    }
}

}  // namespace

extern "C" {

void ora_lame(double E, double nu, double* mu, double* lam_s) {
  const double m = E / (2.0 * (1.0 + nu));
  const double l = E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu));
  *mu = m;
  *lam_s = l + m;
}

double ora_snh_psi(const double* F, double mu, double lam_s) {
  double trc = 0.0;
  for (int a = 0; a < 9; ++a) trc += F[a] * F[a];
  const double J = det3(F);
  return 0.5 * mu * (trc - 3.0) - mu * (J - 1.0) + 0.5 * lam_s * (J - 1.0) * (J - 1.0);
}

// P = dpsi/dF = mu F - mu cof F + lam_s (J - 1) cof F
void ora_snh_pk1(const double* F, double mu, double lam_s, double* P) {
  double C[9];
  cofactor(F, C);
  const double J = det3(F);
  for (int a = 0; a < 9; ++a) P[a] = mu * F[a] - mu * C[a] + lam_s * (J - 1.0) * C[a];
}

// dP/dF = mu I_9 + lam_s vec(cof F) vec(cof F)^T + (lam_s (J - 1) - mu) d2J/dF2,
// d2J / dF_ij dF_kl = eps_ikm eps_jln F_mn.
void ora_snh_dpdf(const double* F, double mu, double lam_s, double* A) {
  double C[9];
  cofactor(F, C);
  const double J = det3(F);
  const double s = lam_s * (J - 1.0) - mu;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      for (int k = 0; k < 3; ++k)
        for (int l = 0; l < 3; ++l) {
          double d2J = 0.0;
          for (int m = 0; m < 3; ++m)
            for (int n = 0; n < 3; ++n) d2J += eps3(i, k, m) * eps3(j, l, n) * F[3 * m + n];
          const int r = 3 * i + j, c = 3 * k + l;
          A[9 * r + c] = (r == c ? mu : 0.0) + lam_s * C[r] * C[c] + s * d2J;
        }
}

}  // extern "C"
