// Dense symmetric eigendecomposition by cyclic Jacobi, and eigenvalue clamping.
//
// TEST INFRASTRUCTURE (oracle).  Projection of an element Hessian follows the
// clamping definition of Sec. 3: H = Q D Q^T, Hhat = Q Dhat Q^T with
// Dhat_ii = max(D_ii, eps), eps = 1e-8 (Sec. 5.1).  The eigendecomposition is
// the textbook cyclic-by-row Jacobi method with the symmetric 2x2 Schur
// rotation (Golub & Van Loan, "Matrix Computations", Sec. 8.5), run in FP64
// until the off-diagonal Frobenius norm is below 1e-15 ||A||_F.
#include <cmath>
#include <cstring>
#include <vector>

#include "ppn_oracle.h"

extern "C" int ora_eigh(int n, const double* A_in, double* w, double* Q) {
  if (n <= 0) return ORA_ERR_INVALID;
  std::vector<double> A(A_in, A_in + (size_t)n * n);
  std::vector<double> V((size_t)n * n, 0.0);
  for (int i = 0; i < n; ++i) V[(size_t)i * n + i] = 1.0;

  double fro = 0.0;
  for (double a : A) fro += a * a;
  fro = std::sqrt(fro);
  const double tol = 1e-15 * fro;

  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < n; ++i)
      for (int j = 0; j < n; ++j)
        if (i != j) off += A[(size_t)i * n + j] * A[(size_t)i * n + j];
    if (std::sqrt(off) <= tol) break;
    for (int p = 0; p < n - 1; ++p)
      for (int q = p + 1; q < n; ++q) {
        const double apq = A[(size_t)p * n + q];
        if (apq == 0.0) continue;
        // symmetric Schur decomposition of the (p, q) 2x2 sub-block
        const double tau = (A[(size_t)q * n + q] - A[(size_t)p * n + p]) / (2.0 * apq);
        const double t = (tau >= 0.0) ? 1.0 / (tau + std::sqrt(1.0 + tau * tau))
                                      : -1.0 / (-tau + std::sqrt(1.0 + tau * tau));
        const double c = 1.0 / std::sqrt(1.0 + t * t);
        const double s = t * c;
        // A <- A J (columns p, q)
        for (int k = 0; k < n; ++k) {
          const double akp = A[(size_t)k * n + p], akq = A[(size_t)k * n + q];
          A[(size_t)k * n + p] = c * akp - s * akq;
          A[(size_t)k * n + q] = s * akp + c * akq;
        }
        // A <- J^T A (rows p, q)
        for (int k = 0; k < n; ++k) {
          const double apk = A[(size_t)p * n + k], aqk = A[(size_t)q * n + k];
          A[(size_t)p * n + k] = c * apk - s * aqk;
          A[(size_t)q * n + k] = s * apk + c * aqk;
        }
        // V <- V J
        for (int k = 0; k < n; ++k) {
          const double vkp = V[(size_t)k * n + p], vkq = V[(size_t)k * n + q];
          V[(size_t)k * n + p] = c * vkp - s * vkq;
          V[(size_t)k * n + q] = s * vkp + c * vkq;
        }
      }
  }
  for (int i = 0; i < n; ++i) w[i] = A[(size_t)i * n + i];
  std::memcpy(Q, V.data(), sizeof(double) * (size_t)n * n);
  return ORA_OK;
}

// Hhat = Q f(D) Q^T and dH = Hhat - H (the in-place update of Sec. 4.1), with
// f(lambda) = max(lambda, eps) (clamping, Sec. 3) or max(|lambda|, eps)
// (eigenvalue mirroring, which the paper compares against clamping, Sec. 5.2).
extern "C" int ora_project(int n, const double* H, double eps, int kind, double* Hhat, double* dH) {
  if (kind != ORA_PROJ_CLAMP && kind != ORA_PROJ_MIRROR) return ORA_ERR_INVALID;
  std::vector<double> w(n), Q((size_t)n * n), Hh((size_t)n * n);
  int rc = ora_eigh(n, H, w.data(), Q.data());
  if (rc) return rc;
  for (int k = 0; k < n; ++k) w[k] = std::fmax(kind == ORA_PROJ_MIRROR ? std::fabs(w[k]) : w[k], eps);
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      double s = 0.0;
      for (int k = 0; k < n; ++k) s += Q[(size_t)i * n + k] * w[k] * Q[(size_t)j * n + k];
      Hh[(size_t)i * n + j] = s;
    }
  if (Hhat) std::memcpy(Hhat, Hh.data(), sizeof(double) * (size_t)n * n);
  if (dH)
    for (size_t k = 0; k < (size_t)n * n; ++k) dH[k] = Hh[k] - H[k];
  return ORA_OK;
}

extern "C" int ora_clamp(int n, const double* H, double eps, double* Hhat, double* dH) {
  return ora_project(n, H, eps, ORA_PROJ_CLAMP, Hhat, dH);
}
