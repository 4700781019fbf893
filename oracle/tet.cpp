// One linear tetrahedron: deformation gradient, element energy, gradient and
// 12x12 Hessian, FP64, written from the definitions.
//
// TEST INFRASTRUCTURE (oracle).  The element contributions g^e and H^e are the
// per-element terms whose sums give the global gradient and Hessian of Newton's
// method (Sec. 3, Eq. newton).  With D_m = [X1-X0, X2-X0, X3-X0] (columns),
// D_s likewise from the current corners, F = D_s D_m^{-1}, V = det(D_m) / 6:
//   psi_e = V psi(F),   g^e = V B^T vec(P(F)),   H^e = V B^T (dP/dF) B,
// with B = dvec(F)/dx_e the 9x12 matrix of the linear map x_e -> vec(F).
#include <cmath>
#include <cstring>

#include "ppn_oracle.h"

namespace ora {

double det3x3(const double* M) {
  return M[0] * (M[4] * M[8] - M[5] * M[7]) - M[1] * (M[3] * M[8] - M[5] * M[6]) +
         M[2] * (M[3] * M[7] - M[4] * M[6]);
}

// inverse via the adjugate; returns the determinant
double inv3x3(const double* M, double* Mi) {
  const double d = det3x3(M);
  Mi[0] = (M[4] * M[8] - M[5] * M[7]) / d;
  Mi[1] = (M[2] * M[7] - M[1] * M[8]) / d;
  Mi[2] = (M[1] * M[5] - M[2] * M[4]) / d;
  Mi[3] = (M[5] * M[6] - M[3] * M[8]) / d;
  Mi[4] = (M[0] * M[8] - M[2] * M[6]) / d;
  Mi[5] = (M[2] * M[3] - M[0] * M[5]) / d;
  Mi[6] = (M[3] * M[7] - M[4] * M[6]) / d;
  Mi[7] = (M[1] * M[6] - M[0] * M[7]) / d;
  Mi[8] = (M[0] * M[4] - M[1] * M[3]) / d;
  return d;
}

// D = [c1-c0, c2-c0, c3-c0] as columns, D[3*i + a] = c_{a+1,i} - c_{0,i}
void edge_matrix(const double* c, double* D) {
  for (int i = 0; i < 3; ++i)
    for (int a = 0; a < 3; ++a) D[3 * i + a] = c[3 * (a + 1) + i] - c[i];
}

// B[(3i+j)*12 + 3a+k] = dF_ij / dx_{a,k}
void shape_jacobian(const double* DmInv, double* B) {
  std::memset(B, 0, sizeof(double) * 9 * 12);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      // F_ij = sum_c (x_{c+1,i} - x_{0,i}) DmInv_{c j}
      double col_sum = 0.0;
      for (int c = 0; c < 3; ++c) {
        B[(3 * i + j) * 12 + 3 * (c + 1) + i] += DmInv[3 * c + j];
        col_sum += DmInv[3 * c + j];
      }
      B[(3 * i + j) * 12 + 0 + i] -= col_sum;
    }
}

}  // namespace ora

extern "C" int ora_tet_eval(const double* X, const double* x, double mu, double lam_s,
                            double* psi_e, double* g12, double* H144) {
  double Dm[9], Ds[9], DmInv[9], F[9];
  ora::edge_matrix(X, Dm);
  ora::edge_matrix(x, Ds);
  const double det = ora::inv3x3(Dm, DmInv);
  if (!(det > 0.0)) return ORA_ERR_DEGENERATE;
  const double V = det / 6.0;
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double f = 0.0;
      for (int c = 0; c < 3; ++c) f += Ds[3 * i + c] * DmInv[3 * c + j];
      F[3 * i + j] = f;
    }
  if (psi_e) *psi_e = V * ora_snh_psi(F, mu, lam_s);
  if (!g12 && !H144) return ORA_OK;

  double B[9 * 12];
  ora::shape_jacobian(DmInv, B);
  if (g12) {
    double P[9];
    ora_snh_pk1(F, mu, lam_s, P);
    for (int m = 0; m < 12; ++m) {
      double s = 0.0;
      for (int r = 0; r < 9; ++r) s += B[r * 12 + m] * P[r];
      g12[m] = V * s;
    }
  }
  if (H144) {
    double A[81], AB[9 * 12];
    ora_snh_dpdf(F, mu, lam_s, A);
    for (int r = 0; r < 9; ++r)
      for (int n = 0; n < 12; ++n) {
        double s = 0.0;
        for (int q = 0; q < 9; ++q) s += A[9 * r + q] * B[q * 12 + n];
        AB[r * 12 + n] = s;
      }
    for (int m = 0; m < 12; ++m)
      for (int n = 0; n < 12; ++n) {
        double s = 0.0;
        for (int r = 0; r < 9; ++r) s += B[r * 12 + m] * AB[r * 12 + n];
        H144[12 * m + n] = V * s;
      }
  }
  return ORA_OK;
}
