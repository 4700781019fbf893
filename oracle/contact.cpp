// Frictionless log-barrier contact against analytic surfaces, FP64.
//
// TEST INFRASTRUCTURE (oracle).  The paper's contact scenes use IPC barrier
// potentials with a backtracking line search and intersection-based filtering
// (Sec. 5.1).  Against analytic obstacles the potential of a vertex x is
//   kappa b(d(x)),  b(d) = -(d - dhat)^2 ln(d / dhat) for 0 < d < dhat, else 0,
// with d the distance to the surface:
//   plane          d = a . (x - p)                         (a: unit normal)
//   cylinder, in   d = r - |q_perp|,  q = x - p, q_perp = q - (a . q) a
//   sphere, out    d = |x - p| - r
// Gradient kappa b'(d) grad d; Hessian kappa (b''(d) grad d grad d^T + b'(d) hess d).
// The line search starts at gamma0 = min(1, safety * gamma_ccd), gamma_ccd the
// first gamma at which a vertex on x + gamma dx reaches a surface.
#include <cmath>
#include <limits>

#include "ppn_oracle.h"

extern "C" {

int ora_barrier(double d, double dhat, double* b, double* db, double* ddb) {
  if (!(d > 0.0)) {
    if (b) *b = std::numeric_limits<double>::infinity();
    if (db) *db = 0.0;
    if (ddb) *ddb = 0.0;
    return ORA_ERR_INVALID;
  }
  if (d >= dhat) {
    if (b) *b = 0.0;
    if (db) *db = 0.0;
    if (ddb) *ddb = 0.0;
    return ORA_OK;
  }
  const double t = d - dhat, L = std::log(d / dhat);
  if (b) *b = -t * t * L;
  if (db) *db = -2.0 * t * L - t * t / d;
  if (ddb) *ddb = -2.0 * L - 4.0 * t / d + t * t / (d * d);
  return ORA_OK;
}

int ora_obstacle_eval(const ora_obstacle* o, const double* x, double* d, double* grad, double* hess) {
  double q[3] = {x[0] - o->p[0], x[1] - o->p[1], x[2] - o->p[2]};
  double g[3] = {0, 0, 0}, H[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0}, dist;
  if (o->type == ORA_OBST_PLANE) {
    dist = o->a[0] * q[0] + o->a[1] * q[1] + o->a[2] * q[2];
    for (int k = 0; k < 3; ++k) g[k] = o->a[k];
  } else if (o->type == ORA_OBST_CYLINDER_IN) {
    const double aq = o->a[0] * q[0] + o->a[1] * q[1] + o->a[2] * q[2];
    double qp[3];
    for (int k = 0; k < 3; ++k) qp[k] = q[k] - aq * o->a[k];
    const double rho = std::sqrt(qp[0] * qp[0] + qp[1] * qp[1] + qp[2] * qp[2]);
    if (!(rho > 0.0)) return ORA_ERR_INVALID;  // on the axis: direction undefined
    dist = o->r - rho;
    double e[3];
    for (int k = 0; k < 3; ++k) {
      e[k] = qp[k] / rho;
      g[k] = -e[k];
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j)
        H[3 * i + j] = -((i == j ? 1.0 : 0.0) - o->a[i] * o->a[j] - e[i] * e[j]) / rho;
  } else if (o->type == ORA_OBST_SPHERE_OUT) {
    const double rho = std::sqrt(q[0] * q[0] + q[1] * q[1] + q[2] * q[2]);
    if (!(rho > 0.0)) return ORA_ERR_INVALID;
    dist = rho - o->r;
    double e[3];
    for (int k = 0; k < 3; ++k) {
      e[k] = q[k] / rho;
      g[k] = e[k];
    }
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) H[3 * i + j] = ((i == j ? 1.0 : 0.0) - e[i] * e[j]) / rho;
  } else {
    return ORA_ERR_INVALID;
  }
  if (d) *d = dist;
  if (grad)
    for (int k = 0; k < 3; ++k) grad[k] = g[k];
  if (hess)
    for (int k = 0; k < 9; ++k) hess[k] = H[k];
  return ORA_OK;
}

// smallest gamma > 0 with d(x + gamma dx) = 0, or +infinity
double ora_obstacle_ccd(const ora_obstacle* o, const double* x, const double* dx) {
  const double inf = std::numeric_limits<double>::infinity();
  double q[3] = {x[0] - o->p[0], x[1] - o->p[1], x[2] - o->p[2]};
  double u[3] = {dx[0], dx[1], dx[2]};
  if (o->type == ORA_OBST_PLANE) {
    const double d0 = o->a[0] * q[0] + o->a[1] * q[1] + o->a[2] * q[2];
    const double s = o->a[0] * u[0] + o->a[1] * u[1] + o->a[2] * u[2];
    return s < 0.0 ? -d0 / s : inf;
  }
  if (o->type == ORA_OBST_CYLINDER_IN) {  // project out the axis, then |q + gamma u| = r from inside
    const double aq = o->a[0] * q[0] + o->a[1] * q[1] + o->a[2] * q[2];
    const double au = o->a[0] * u[0] + o->a[1] * u[1] + o->a[2] * u[2];
    for (int k = 0; k < 3; ++k) {
      q[k] -= aq * o->a[k];
      u[k] -= au * o->a[k];
    }
  }
  const double A = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
  const double B = 2.0 * (q[0] * u[0] + q[1] * u[1] + q[2] * u[2]);
  const double C = q[0] * q[0] + q[1] * q[1] + q[2] * q[2] - o->r * o->r;
  if (!(A > 0.0)) return inf;
  const double disc = B * B - 4.0 * A * C;
  if (o->type == ORA_OBST_CYLINDER_IN) {  // C < 0 inside: exactly one positive root
    return (-B + std::sqrt(std::fmax(disc, 0.0))) / (2.0 * A);
  }
  if (o->type == ORA_OBST_SPHERE_OUT) {  // C > 0 outside: the nearer root, if ahead
    if (disc < 0.0 || B >= 0.0) return inf;
    return (-B - std::sqrt(disc)) / (2.0 * A);
  }
  return inf;
}

}  // extern "C"
