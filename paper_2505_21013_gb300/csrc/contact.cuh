// Frictionless log-barrier contact against analytic surfaces (the IPC
// potentials of the paper's contact scenes with a backtracking line search and
// intersection-based filtering, Sec. 5.1), per vertex and in FP64.
//
//   kappa b(d),  b(d) = -(d - dhat)^2 ln(d / dhat) on (0, dhat), 0 beyond, +inf at d <= 0
//   plane          d = a . (x - p)
//   cylinder, in   d = r - |q_perp|,  q = x - p, q_perp = q - (a . q) a
//   sphere, out    d = |x - p| - r
// gradient kappa b' grad d, Hessian kappa (b'' grad d grad d^T + b' hess d).  A
// free vertex within dhat of some surface is one contact element of the
// projection heuristic, with the 3x3 Hessian of its summed potential.
#pragma once

#include <limits>

#include "common.cuh"
#include "tetmath.cuh"

namespace ppn {

PPN_HD void barrier(double d, double dhat, double& b, double& db, double& ddb) {
  if (d >= dhat) {
    b = db = ddb = 0.0;
    return;
  }
  const double t = d - dhat, L = log(d / dhat);
  b = -t * t * L;
  db = -2.0 * t * L - t * t / d;
  ddb = -2.0 * L - 4.0 * t / d + t * t / (d * d);
}

// distance, its gradient and Hessian; false where the direction is undefined
PPN_HD bool obst_eval(const ObstDev& o, const double* x, double& d, double* g, double* H) {
  const double q[3] = {x[0] - o.p[0], x[1] - o.p[1], x[2] - o.p[2]};
  for (int k = 0; k < 9; ++k) H[k] = 0.0;
  if (o.type == OBST_PLANE) {
    d = o.a[0] * q[0] + o.a[1] * q[1] + o.a[2] * q[2];
    for (int k = 0; k < 3; ++k) g[k] = o.a[k];
    return true;
  }
  double e[3], rho;
  if (o.type == OBST_CYLINDER_IN) {
    const double aq = o.a[0] * q[0] + o.a[1] * q[1] + o.a[2] * q[2];
    const double qp[3] = {q[0] - aq * o.a[0], q[1] - aq * o.a[1], q[2] - aq * o.a[2]};
    rho = sqrt(qp[0] * qp[0] + qp[1] * qp[1] + qp[2] * qp[2]);
    if (!(rho > 0.0)) return false;
    for (int k = 0; k < 3; ++k) e[k] = qp[k] / rho;
    d = o.r - rho;
    for (int k = 0; k < 3; ++k) g[k] = -e[k];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) H[3 * i + j] = -((i == j ? 1.0 : 0.0) - o.a[i] * o.a[j] - e[i] * e[j]) / rho;
    return true;
  }
  // sphere, outside
  rho = sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
  if (!(rho > 0.0)) return false;
  for (int k = 0; k < 3; ++k) e[k] = q[k] / rho;
  d = rho - o.r;
  for (int k = 0; k < 3; ++k) g[k] = e[k];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) H[3 * i + j] = ((i == j ? 1.0 : 0.0) - e[i] * e[j]) / rho;
  return true;
}

// first gamma > 0 at which x + gamma dx reaches the surface, or +infinity
PPN_HD double obst_ccd(const ObstDev& o, const double* x, const double* dx) {
  const double inf = std::numeric_limits<double>::infinity();
  double q[3] = {x[0] - o.p[0], x[1] - o.p[1], x[2] - o.p[2]};
  double u[3] = {dx[0], dx[1], dx[2]};
  if (o.type == OBST_PLANE) {
    const double d0 = o.a[0] * q[0] + o.a[1] * q[1] + o.a[2] * q[2];
    const double s = o.a[0] * u[0] + o.a[1] * u[1] + o.a[2] * u[2];
    return s < 0.0 ? -d0 / s : inf;
  }
  if (o.type == OBST_CYLINDER_IN) {
    const double aq = o.a[0] * q[0] + o.a[1] * q[1] + o.a[2] * q[2];
    const double au = o.a[0] * u[0] + o.a[1] * u[1] + o.a[2] * u[2];
    for (int k = 0; k < 3; ++k) {
      q[k] -= aq * o.a[k];
      u[k] -= au * o.a[k];
    }
  }
  const double A = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double B = 2.0 * (q[0] * u[0] + q[1] * u[1] + q[2] * u[2]);
  const double C = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] - o.r * o.r;
  if (!(A > 0.0)) return inf;
  const double disc = B * B - 4.0 * A * C;
  if (o.type == OBST_CYLINDER_IN) return (-B + sqrt(fmax(disc, 0.0))) / (2.0 * A);  // C < 0: one root ahead
  if (disc < 0.0 || B >= 0.0) return inf;                                              // sphere: nearer root
  return (-B - sqrt(disc)) / (2.0 * A);
}

// summed potential of a vertex at x: energy, gradient, Hessian (each optional);
// false when x is not strictly feasible; active: some distance below dhat
template <typename T>
PPN_HD bool vertex_contact(const SceneDev<T>& S, const double* x, double* E, double* g, double* H, bool* active) {
  if (E) *E = 0.0;
  if (g) g[0] = g[1] = g[2] = 0.0;
  if (H)
    for (int k = 0; k < 9; ++k) H[k] = 0.0;
  if (active) *active = false;
  const int n = S.obs->n;
  for (int k = 0; k < n; ++k) {
    double d, gd[3], Hd[9];
    if (!obst_eval(S.obs->o[k], x, d, gd, Hd) || !(d > 0.0)) return false;
    if (d >= S.dhat) continue;
    double b, db, ddb;
    barrier(d, S.dhat, b, db, ddb);
    if (active) *active = true;
    if (E) *E += S.kappa * b;
    if (g)
      for (int i = 0; i < 3; ++i) g[i] += S.kappa * db * gd[i];
    if (H)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[3 * i + j] += S.kappa * (ddb * gd[i] * gd[j] + db * Hd[3 * i + j]);
  }
  return true;
}

// dH = Q f(L) Q^T - A for a symmetric 3x3 A = Q L Q^T (cyclic Jacobi), with
// f(l) = max(l, eps) (clamp) or max(|l|, eps) (mirror) on eigenvalues below eps
template <typename T>
PPN_HD void clamp3(const T* A0, T eps, bool mirror, T* dH) {
  T a[3][3], v[3][3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      a[i][j] = (T)0.5 * (A0[3 * i + j] + A0[3 * j + i]);
      v[i][j] = i == j ? (T)1 : (T)0;
    }
  const int pp[3] = {0, 0, 1}, qq[3] = {1, 2, 2};
  for (int sweep = 0; sweep < 30; ++sweep) {
    const T off = a[0][1] * a[0][1] + a[0][2] * a[0][2] + a[1][2] * a[1][2];
    const T nrm = a[0][0] * a[0][0] + a[1][1] * a[1][1] + a[2][2] * a[2][2] + 2 * off;
    if (!(off > (T)1e-30 * nrm) || off == (T)0) break;
    for (int r = 0; r < 3; ++r) {
      const int p = pp[r], q = qq[r];
      if (a[p][q] == (T)0) continue;
      const T th = (a[q][q] - a[p][p]) / ((T)2 * a[p][q]);
      const T t = (th >= (T)0 ? (T)1 : (T)-1) / (fabs(th) + sqrt(th * th + (T)1));
      const T c = (T)1 / sqrt(t * t + (T)1), s = t * c;
      for (int k = 0; k < 3; ++k) {  // columns p, q
        const T akp = a[k][p], akq = a[k][q];
        a[k][p] = c * akp - s * akq;
        a[k][q] = s * akp + c * akq;
      }
      for (int k = 0; k < 3; ++k) {  // rows p, q
        const T apk = a[p][k], aqk = a[q][k];
        a[p][k] = c * apk - s * aqk;
        a[q][k] = s * apk + c * aqk;
      }
      for (int k = 0; k < 3; ++k) {
        const T vkp = v[k][p], vkq = v[k][q];
        v[k][p] = c * vkp - s * vkq;
        v[k][q] = s * vkp + c * vkq;
      }
    }
  }
  for (int k = 0; k < 9; ++k) dH[k] = (T)0;
  for (int m = 0; m < 3; ++m) {
    const T l = a[m][m];
    if (!(l < eps)) continue;
    const T w = (mirror ? (-l > eps ? -l : eps) : eps) - l;
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) dH[3 * i + j] += w * v[i][m] * v[j][m];
  }
}

}  // namespace ppn
