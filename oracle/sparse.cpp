// 3x3-block sparse (BSR) matrices and block-diagonal PCG with a curvature exit.
//
// TEST INFRASTRUCTURE (oracle).  The linear solver of Algorithm 1 must solve
// H dx = -g and report whether indefiniteness was met (Sec. 4, Algorithm 1;
// Sec. 4.1, "Linear Solvers").  PCG starts from the zero vector, monitors
// d^T H d for every search direction d and stops with ind = true when it is
// not positive.  The preconditioner is the 3x3 block diagonal (Sec. 5.1,
// "Hardware and software"), applied as the exact inverse of each diagonal block
// computed through its Cholesky factor; a block whose Cholesky fails cannot
// belong to an SPD matrix and also reports ind = true.  Convergence is
// ||r|| <= rel_tol ||r0|| with rel_tol = 1e-4 in the paper (Sec. 5.1).
#include <cmath>
#include <cstring>
#include <vector>

#include "ppn_oracle.h"

namespace ora {

// y = A x on a BSR matrix with 3x3 row-major blocks
void bsr_spmv(int64_t n_rows, const int64_t* row_ptr, const int32_t* col, const double* vals,
              const double* x, double* y) {
  // rows are independent: with OpenMP they are shared out over the host's cores (same results)
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n_rows; ++i) {
    double acc[3] = {0.0, 0.0, 0.0};
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k) {
      const double* blk = vals + 9 * k;
      const double* xj = x + 3 * (int64_t)col[k];
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) acc[r] += blk[3 * r + c] * xj[c];
    }
    for (int r = 0; r < 3; ++r) y[3 * i + r] = acc[r];
  }
}

// Inverse of a symmetric 3x3 block through its Cholesky factor (lower triangle
// of D is read).  Returns false when a pivot is not positive.
bool spd_inverse3(const double* D, double* Dinv) {
  double L[9] = {0};
  for (int j = 0; j < 3; ++j) {
    double d = D[3 * j + j];
    for (int k = 0; k < j; ++k) d -= L[3 * j + k] * L[3 * j + k];
    if (!(d > 0.0)) return false;
    L[3 * j + j] = std::sqrt(d);
    for (int i = j + 1; i < 3; ++i) {
      double s = D[3 * i + j];
      for (int k = 0; k < j; ++k) s -= L[3 * i + k] * L[3 * j + k];
      L[3 * i + j] = s / L[3 * j + j];
    }
  }
  // Linv by forward substitution, then Dinv = Linv^T Linv
  double Li[9] = {0};
  for (int c = 0; c < 3; ++c) {
    for (int i = 0; i < 3; ++i) {
      double s = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= L[3 * i + k] * Li[3 * k + c];
      Li[3 * i + c] = s / L[3 * i + i];
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      double s = 0.0;
      for (int k = 0; k < 3; ++k) s += Li[3 * k + i] * Li[3 * k + j];
      Dinv[3 * i + j] = s;
    }
  return true;
}

double dot(const std::vector<double>& a, const std::vector<double>& b) {
  double s = 0.0;
  for (size_t i = 0; i < a.size(); ++i) s += a[i] * b[i];
  return s;
}

// Block-Jacobi PCG from x = 0.  info: [iters, ind, precond_fail, hit_max]
void pcg(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* vals,
         const double* b, double rel_tol, int max_iter, double* x_out, int* info) {
  const size_t N = (size_t)(3 * n);
  std::vector<double> x(N, 0.0), r(b, b + N), z(N), d(N), q(N), Pinv(9 * (size_t)n);
  info[0] = info[1] = info[2] = info[3] = 0;
  const double rr0 = dot(r, r);
  if (rr0 == 0.0) {
    std::memset(x_out, 0, sizeof(double) * N);
    return;
  }
  for (int64_t i = 0; i < n; ++i) {
    const double* D = nullptr;
    for (int64_t k = row_ptr[i]; k < row_ptr[i + 1]; ++k)
      if (col[k] == i) D = vals + 9 * k;
    if (!D || !spd_inverse3(D, &Pinv[9 * i])) {
      info[1] = 1;
      info[2] = 1;
      std::memset(x_out, 0, sizeof(double) * N);
      return;
    }
  }
  auto apply_P = [&](const std::vector<double>& in, std::vector<double>& out) {
    for (int64_t i = 0; i < n; ++i)
      for (int a = 0; a < 3; ++a) {
        double s = 0.0;
        for (int c = 0; c < 3; ++c) s += Pinv[9 * i + 3 * a + c] * in[3 * i + c];
        out[3 * i + a] = s;
      }
  };
  apply_P(r, z);
  d = z;
  double rz = dot(r, z);
  int it = 0;
  for (; it < max_iter; ++it) {
    bsr_spmv(n, row_ptr, col, vals, d.data(), q.data());
    const double dq = dot(d, q);
    if (dq <= 0.0) {
      info[1] = 1;
      break;
    }
    const double alpha = rz / dq;
    for (size_t k = 0; k < N; ++k) {
      x[k] += alpha * d[k];
      r[k] -= alpha * q[k];
    }
    const double rr = dot(r, r);
    if (rr <= rel_tol * rel_tol * rr0) {
      ++it;
      break;
    }
    apply_P(r, z);
    const double rz_new = dot(r, z);
    const double beta = rz_new / rz;
    rz = rz_new;
    for (size_t k = 0; k < N; ++k) d[k] = z[k] + beta * d[k];
  }
  if (it >= max_iter && !info[1]) info[3] = 1;
  info[0] = it;
  std::memcpy(x_out, x.data(), sizeof(double) * N);
}

}  // namespace ora

extern "C" int ora_pcg_bsr(int64_t n_rows, const int64_t* row_ptr, const int32_t* col,
                           const double* vals, const double* b, double rel_tol, int max_iter,
                           double* x, int* info) {
  if (n_rows < 0 || !row_ptr || !b || !x || !info) return ORA_ERR_INVALID;
  ora::pcg(n_rows, row_ptr, col, vals, b, rel_tol, max_iter, x, info);
  return ORA_OK;
}
