// Scene state, incremental potential and the Newton / PN / PPN time step, FP64.
//
// TEST INFRASTRUCTURE (oracle).  One call of ora_scene_step is one backward
// Euler step, solved as the minimisation of the incremental potential by
// Newton's method (Sec. 3) in one of four modes:
//   ORA_NEWTON  no element is projected (Sec. 1; Newton-CG fallback on ind)
//   ORA_PN      every element Hessian is clamped before assembly (Sec. 3)
//   ORA_PPN     Algorithm 1: start unprojected; while the solver reports
//               indefiniteness, project the elements with ||S^e g||_inf > delta
//               in place and solve again, tightening delta by alpha; relax it by
//               beta after a successful solve (Sec. 4).
//   ORA_PDN     project-on-demand (Sec. 2.2, Sec. 5.1): solve unprojected; when
//               the solver reports indefiniteness, project every element in
//               place and solve again, then assemble projected for the next
//               pdn_countdown iterations (countdown 4) before trying
//               unprojected again.  The countdown starts at 0 every time step.
// The step then takes a backtracking line search (Sec. 5.1) and updates x.
// Dirichlet vertices are eliminated (their targets set, zero gradient, identity
// rows) unless params.dirichlet_penalty = k > 0: then, as Sec. 5.1 enforces
// Dirichlet constraints with penalty potentials, they stay free and carry
// k m_v / (2 dt^2) |x_v - t_v|^2 (a stiffness k times the vertex's inertia term).
// Either way the initial iterate starts them at their targets.
#include <cmath>
#include <cstring>
#include <limits>
#include <string>
#include <vector>

#include "ppn_oracle.h"

#ifdef _OPENMP
#include <omp.h>
#endif

namespace ora {
double det3x3(const double* M);
void edge_matrix(const double* c, double* D);
void bsr_spmv(int64_t n_rows, const int64_t* row_ptr, const int32_t* col, const double* vals,
              const double* x, double* y);
bool spd_inverse3(const double* D, double* Dinv);
void pcg(int64_t n, const int64_t* row_ptr, const int32_t* col, const double* vals,
         const double* b, double rel_tol, int max_iter, double* x_out, int* info);
}  // namespace ora

static thread_local std::string g_err;

struct ora_scene {
  int64_t nv = 0, nt = 0;
  std::vector<double> X;
  std::vector<int32_t> tets;
  double mu = 0, lam = 0, rho = 0, dt = 0, grav[3] = {0, 0, 0};
  std::vector<double> mass;
  std::vector<uint8_t> fixed;          // eliminated Dirichlet vertices (none with a penalty)
  std::vector<int32_t> fixed_list;     // Dirichlet vertices, in the order of `targets`
  std::vector<double> targets;
  std::vector<int32_t> pen;            // penalty: the vertex's index in fixed_list, else -1
  std::vector<double> x, v;
  std::vector<int64_t> row_ptr;
  std::vector<int32_t> col;
  ora_params p;
  std::vector<ora_obstacle> obst;      // applied poses (those the barrier acts with)
  std::vector<ora_obstacle> obst_req;  // requested poses
  ora_solve_hook hook = nullptr;
  void* hook_user = nullptr;
  std::vector<ora_iter_stats> iters;
  std::vector<ora_attempt> attempts;
  std::vector<std::vector<int32_t>> attempt_sel;  // PPN selection before each attempt
  bool record = false;                            // keep each iteration's gradient
  std::vector<std::vector<double>> iter_g;
};

namespace {

const double kInf = std::numeric_limits<double>::infinity();

void corners(const ora_scene* s, int64_t e, const double* x, double* c) {
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) c[3 * a + k] = x[3 * (int64_t)s->tets[4 * e + a] + k];
}

void element(const ora_scene* s, int64_t e, const double* x, double* psi, double* g, double* H) {
  double Xc[12], xc[12];
  corners(s, e, s->X.data(), Xc);
  corners(s, e, x, xc);
  ora_tet_eval(Xc, xc, s->mu, s->lam, psi, g, H);
}

// Contact potential of one vertex at xv, summed over the obstacles: energy,
// gradient (3) and Hessian (9), each optional.  Returns false when xv is not
// strictly feasible (some distance <= 0); *active: some distance < dhat.
bool vertex_contact(const ora_scene* s, const double* xv, double* E, double* g, double* H, bool* active) {
  if (E) *E = 0.0;
  if (g)
    for (int k = 0; k < 3; ++k) g[k] = 0.0;
  if (H)
    for (int k = 0; k < 9; ++k) H[k] = 0.0;
  if (active) *active = false;
  const double kap = s->p.contact_kappa, dhat = s->p.contact_dhat;
  for (const ora_obstacle& o : s->obst) {
    double d, gd[3], Hd[9];
    if (ora_obstacle_eval(&o, xv, &d, gd, Hd) != ORA_OK || !(d > 0.0)) return false;
    if (d >= dhat) continue;
    double b, db, ddb;
    ora_barrier(d, dhat, &b, &db, &ddb);
    if (active) *active = true;
    if (E) *E += kap * b;
    if (g)
      for (int k = 0; k < 3; ++k) g[k] += kap * db * gd[k];
    if (H)
      for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) H[3 * i + j] += kap * (ddb * gd[i] * gd[j] + db * Hd[3 * i + j]);
  }
  return true;
}

// penalty weight k m_v / dt^2 of a Dirichlet vertex held by a penalty potential (0 otherwise)
double pen_weight(const ora_scene* s, int64_t v) {
  return s->pen.empty() || s->pen[v] < 0 ? 0.0 : s->p.dirichlet_penalty * s->mass[v] / (s->dt * s->dt);
}
const double* pen_target(const ora_scene* s, int64_t v) { return &s->targets[3 * (size_t)s->pen[v]]; }

double energy(const ora_scene* s, const double* x, const double* xhat) {
  double E = 0.0;
  const double w = 0.5 / (s->dt * s->dt);
  for (int64_t v = 0; v < s->nv; ++v) {
    if (s->fixed[v]) continue;
    double d2 = 0.0;
    for (int k = 0; k < 3; ++k) {
      const double d = x[3 * v + k] - xhat[3 * v + k];
      d2 += d * d;
    }
    E += w * s->mass[v] * d2;
    if (const double wp = pen_weight(s, v)) {  // Dirichlet penalty potential
      const double* t = pen_target(s, v);
      double p2 = 0.0;
      for (int k = 0; k < 3; ++k) p2 += (x[3 * v + k] - t[k]) * (x[3 * v + k] - t[k]);
      E += 0.5 * wp * p2;
    }
    if (!s->obst.empty()) {
      double Ec;
      if (!vertex_contact(s, x + 3 * v, &Ec, nullptr, nullptr, nullptr))
        return std::numeric_limits<double>::infinity();  // not feasible
      E += Ec;
    }
  }
  for (int64_t e = 0; e < s->nt; ++e) {
    double psi;
    element(s, e, x, &psi, nullptr, nullptr);
    E += psi;
  }
  return E;
}

// g = M (x - xhat) / dt^2 + sum_e S^eT g^e, zero on Dirichlet vertices
void gradient_from(const ora_scene* s, const double* x, const double* xhat,
                   const std::vector<double>& ge, double* g) {
  const double w = 1.0 / (s->dt * s->dt);
  for (int64_t v = 0; v < s->nv; ++v)
    for (int k = 0; k < 3; ++k) g[3 * v + k] = w * s->mass[v] * (x[3 * v + k] - xhat[3 * v + k]);
  for (int64_t e = 0; e < s->nt; ++e)
    for (int a = 0; a < 4; ++a)
      for (int k = 0; k < 3; ++k) g[3 * (int64_t)s->tets[4 * e + a] + k] += ge[12 * e + 3 * a + k];
  for (int64_t v = 0; v < s->nv; ++v)
    if (const double wp = pen_weight(s, v))
      for (int k = 0; k < 3; ++k) g[3 * v + k] += wp * (x[3 * v + k] - pen_target(s, v)[k]);
  if (!s->obst.empty())
    for (int64_t v = 0; v < s->nv; ++v) {
      if (s->fixed[v]) continue;
      double gc[3];
      vertex_contact(s, x + 3 * v, nullptr, gc, nullptr, nullptr);
      for (int k = 0; k < 3; ++k) g[3 * v + k] += gc[k];
    }
  for (int64_t v = 0; v < s->nv; ++v)
    if (s->fixed[v])
      for (int k = 0; k < 3; ++k) g[3 * v + k] = 0.0;
}

// ||s||_2 with s_v = m_v |x_v - xhat_v| / dt^2 + sum_e |g^e_v| (component-wise, free
// vertices): the size of the terms whose sum is the residual g.  Rounding in that
// sum is a few ulps of s, so the relative test ||g|| <= tol ||g0|| cannot be met
// once ||g0|| itself is at that level (a scene already at rest).
double residual_scale(const ora_scene* s, const double* x, const double* xhat, const std::vector<double>& ge) {
  const double w = 1.0 / (s->dt * s->dt);
  std::vector<double> a((size_t)3 * s->nv);
  for (int64_t v = 0; v < s->nv; ++v)
    for (int k = 0; k < 3; ++k) a[3 * v + k] = w * s->mass[v] * std::fabs(x[3 * v + k] - xhat[3 * v + k]);
  for (int64_t e = 0; e < s->nt; ++e)
    for (int i = 0; i < 4; ++i)
      for (int k = 0; k < 3; ++k) a[3 * (int64_t)s->tets[4 * e + i] + k] += std::fabs(ge[12 * e + 3 * i + k]);
  for (int64_t v = 0; v < s->nv; ++v)
    if (const double wp = pen_weight(s, v))
      for (int k = 0; k < 3; ++k) a[3 * v + k] += std::fabs(wp * (x[3 * v + k] - pen_target(s, v)[k]));
  double n2 = 0.0;
  for (int64_t v = 0; v < s->nv; ++v)
    if (!s->fixed[v]) {
      double gc[3] = {0, 0, 0};
      if (!s->obst.empty()) vertex_contact(s, x + 3 * v, nullptr, gc, nullptr, nullptr);
      for (int k = 0; k < 3; ++k) n2 += (a[3 * v + k] + std::fabs(gc[k])) * (a[3 * v + k] + std::fabs(gc[k]));
    }
  return std::sqrt(n2);
}

int64_t find_block(const ora_scene* s, int32_t i, int32_t j) {
  for (int64_t k = s->row_ptr[i]; k < s->row_ptr[i + 1]; ++k)
    if (s->col[k] == j) return k;
  return -1;
}

// vals += S^eT M12 S^e restricted to free rows and columns
void scatter_element(const ora_scene* s, int64_t e, const double* M12, double* vals) {
  for (int a = 0; a < 4; ++a) {
    const int32_t i = s->tets[4 * e + a];
    if (s->fixed[i]) continue;
    for (int b = 0; b < 4; ++b) {
      const int32_t j = s->tets[4 * e + b];
      if (s->fixed[j]) continue;
      double* blk = vals + 9 * find_block(s, i, j);
      for (int r = 0; r < 3; ++r)
        for (int c = 0; c < 3; ++c) blk[3 * r + c] += M12[12 * (3 * a + r) + 3 * b + c];
    }
  }
}

// H = M / dt^2 + sum_e S^eT H^e S^e (+ the contact Hessians of the free vertices at x,
// when x is given and the scene has obstacles); identity rows for eliminated Dirichlet
// vertices, k m_v / dt^2 I added on the diagonal of penalised ones
void assemble(const ora_scene* s, const double* x, const std::vector<double>& He, std::vector<double>& vals) {
  vals.assign(9 * s->col.size(), 0.0);
  for (int64_t e = 0; e < s->nt; ++e) scatter_element(s, e, &He[144 * e], vals.data());
  const double w = 1.0 / (s->dt * s->dt);
  for (int64_t v = 0; v < s->nv; ++v) {
    double* blk = vals.data() + 9 * find_block(s, (int32_t)v, (int32_t)v);
    for (int r = 0; r < 3; ++r) {
      if (s->fixed[v])
        blk[3 * r + r] = 1.0;
      else
        blk[3 * r + r] += w * s->mass[v] + pen_weight(s, v);
    }
    if (x && !s->fixed[v] && !s->obst.empty()) {
      double Hc[9];
      vertex_contact(s, x + 3 * v, nullptr, nullptr, Hc, nullptr);
      for (int k = 0; k < 9; ++k) blk[k] += Hc[k];
    }
  }
}

// r_e = ||S^e g||_inf : largest assembled gradient entry over the element's DOFs
double element_residual(const ora_scene* s, int64_t e, const double* g) {
  double r = 0.0;
  for (int a = 0; a < 4; ++a)
    for (int k = 0; k < 3; ++k) r = std::fmax(r, std::fabs(g[3 * (int64_t)s->tets[4 * e + a] + k]));
  return r;
}

int64_t select(const ora_scene* s, const double* g, double delta, const uint8_t* already,
               uint8_t* out_new) {
  int64_t n = 0;
  for (int64_t e = 0; e < s->nt; ++e) {
    out_new[e] = 0;
    if (already && already[e]) continue;
    if (element_residual(s, e, g) > delta || delta <= s->p.eps_delta) {
      out_new[e] = 1;
      ++n;
    }
  }
  return n;
}

int pcg_max(const ora_scene* s) {
  if (s->p.pcg_max_iter > 0) return s->p.pcg_max_iter;
  return (int)std::max<int64_t>(1000, 3 * s->nv);
}

// preconditioned (or mass-scaled) negative gradient, used when a solve gives no usable iterate
int fallback_direction(const ora_scene* s, const std::vector<double>& vals, const double* g,
                       double* dx) {
  std::vector<double> Pinv(9 * (size_t)s->nv);
  bool spd = true;
  for (int64_t v = 0; v < s->nv && spd; ++v)
    spd = ora::spd_inverse3(vals.data() + 9 * find_block(s, (int32_t)v, (int32_t)v), &Pinv[9 * v]);
  if (spd) {
    for (int64_t v = 0; v < s->nv; ++v)
      for (int a = 0; a < 3; ++a) {
        double t = 0.0;
        for (int c = 0; c < 3; ++c) t += Pinv[9 * v + 3 * a + c] * g[3 * v + c];
        dx[3 * v + a] = -t;
      }
    return 2;
  }
  for (int64_t v = 0; v < s->nv; ++v)
    for (int a = 0; a < 3; ++a)
      dx[3 * v + a] = s->fixed[v] ? 0.0 : -(s->dt * s->dt / s->mass[v]) * g[3 * v + a];
  return 3;
}

}  // namespace

extern "C" {

int ora_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void ora_set_num_threads(int n) {
#ifdef _OPENMP
  if (n > 0) omp_set_num_threads(n);
#else
  (void)n;
#endif
}

ora_params ora_default_params(void) {
  ora_params p;
  p.alpha = 0.5;
  p.beta = 2.0;
  p.eps_delta = 1e-12;
  p.eig_eps = 1e-8;
  p.pcg_rel_tol = 1e-4;
  p.armijo_c = 1e-4;
  p.pcg_max_iter = 0;
  p.newton_max_iter = 100;
  p.ls_max_halvings = 30;
  p.tol_kind = 0;
  p.init_guess = 0;
  p.pdn_countdown = 4;
  p.projection = ORA_PROJ_CLAMP;
  p.grad_floor = 1e-12;
  p.ls_slack = 1e-12;
  p.contact_kappa = 1e3;
  p.contact_dhat = 1e-3;
  p.ccd_safety = 0.9;
  p.dirichlet_penalty = 0.0;
  p.tie_band = 1e-12;
  return p;
}

const char* ora_last_error(void) { return g_err.c_str(); }

ora_scene* ora_scene_create(const double* rest, int64_t n_v, const int32_t* tets, int64_t n_t,
                            double E, double nu, double rho, double dt, const double* gravity,
                            const int32_t* fixed, int64_t n_fixed, const ora_params* params) {
  if (n_v <= 0 || n_t <= 0 || !rest || !tets || !(dt > 0) || !(rho > 0) || !(E > 0) ||
      !(nu > -1.0 && nu < 0.5)) {
    g_err = "invalid argument";
    return nullptr;
  }
  ora_scene* s = new ora_scene();
  s->nv = n_v;
  s->nt = n_t;
  s->X.assign(rest, rest + 3 * n_v);
  s->tets.assign(tets, tets + 4 * n_t);
  ora_lame(E, nu, &s->mu, &s->lam);
  s->rho = rho;
  s->dt = dt;
  for (int k = 0; k < 3; ++k) s->grav[k] = gravity ? gravity[k] : 0.0;
  s->p = params ? *params : ora_default_params();

  // orientation and degeneracy, lumped mass
  s->mass.assign(n_v, 0.0);
  for (int64_t e = 0; e < n_t; ++e) {
    for (int a = 0; a < 4; ++a)
      if (s->tets[4 * e + a] < 0 || s->tets[4 * e + a] >= n_v) {
        g_err = "tet index out of range";
        delete s;
        return nullptr;
      }
    double Xc[12], D[9];
    corners(s, e, s->X.data(), Xc);
    ora::edge_matrix(Xc, D);
    double det = ora::det3x3(D);
    double hmax = 0.0;
    for (int a = 0; a < 4; ++a)
      for (int b = a + 1; b < 4; ++b) {
        double l2 = 0.0;
        for (int k = 0; k < 3; ++k) l2 += (Xc[3 * a + k] - Xc[3 * b + k]) * (Xc[3 * a + k] - Xc[3 * b + k]);
        hmax = std::fmax(hmax, std::sqrt(l2));
      }
    if (std::fabs(det) <= 1e-14 * hmax * hmax * hmax) {
      g_err = "degenerate tet " + std::to_string(e);
      delete s;
      return nullptr;
    }
    if (det < 0) {
      std::swap(s->tets[4 * e + 2], s->tets[4 * e + 3]);
      det = -det;
    }
    for (int a = 0; a < 4; ++a) s->mass[s->tets[4 * e + a]] += rho * (det / 6.0) / 4.0;
  }
  s->fixed.assign(n_v, 0);
  if (!(s->p.dirichlet_penalty >= 0.0)) {
    g_err = "dirichlet_penalty must be >= 0";
    delete s;
    return nullptr;
  }
  const bool penalty = s->p.dirichlet_penalty > 0.0;
  if (penalty) s->pen.assign(n_v, -1);
  // The Dirichlet set is a set of vertices, each with one prescribed target (Sec. 5.1's
  // boundary conditions): an index listed twice would give a vertex two targets, which
  // the method does not define, so it is rejected like an index out of range.
  for (int64_t f = 0; f < n_fixed; ++f) {
    if (fixed[f] < 0 || fixed[f] >= n_v || (penalty ? s->pen[fixed[f]] >= 0 : s->fixed[fixed[f]] != 0)) {
      g_err = "fixed index out of range or repeated";
      delete s;
      return nullptr;
    }
    if (penalty)
      s->pen[fixed[f]] = (int32_t)s->fixed_list.size();
    else
      s->fixed[fixed[f]] = 1;
    s->fixed_list.push_back(fixed[f]);
  }
  for (int64_t v = 0; v < n_v; ++v)
    if (!s->fixed[v] && !(s->mass[v] > 0)) {
      g_err = "free vertex without incident tet";
      delete s;
      return nullptr;
    }
  s->targets.resize(3 * s->fixed_list.size());
  for (size_t f = 0; f < s->fixed_list.size(); ++f)
    for (int k = 0; k < 3; ++k) s->targets[3 * f + k] = s->X[3 * (int64_t)s->fixed_list[f] + k];
  s->x = s->X;
  s->v.assign(3 * n_v, 0.0);

  // full symmetric block pattern: row i holds every j sharing a tet with i (and i)
  std::vector<std::vector<int32_t>> nb(n_v);
  for (int64_t e = 0; e < n_t; ++e)
    for (int a = 0; a < 4; ++a)
      for (int b = 0; b < 4; ++b) nb[s->tets[4 * e + a]].push_back(s->tets[4 * e + b]);
  s->row_ptr.assign(n_v + 1, 0);
  for (int64_t v = 0; v < n_v; ++v) {
    nb[v].push_back((int32_t)v);
    std::vector<int32_t>& r = nb[v];
    // insertion sort + unique (plain)
    for (size_t i = 1; i < r.size(); ++i)
      for (size_t j = i; j > 0 && r[j - 1] > r[j]; --j) std::swap(r[j - 1], r[j]);
    std::vector<int32_t> u;
    for (int32_t c : r)
      if (u.empty() || u.back() != c) u.push_back(c);
    r.swap(u);
    s->row_ptr[v + 1] = s->row_ptr[v] + (int64_t)r.size();
    s->col.insert(s->col.end(), r.begin(), r.end());
  }
  return s;
}

void ora_scene_destroy(ora_scene* s) { delete s; }

int64_t ora_scene_nnzb(const ora_scene* s) { return (int64_t)s->col.size(); }

void ora_scene_pattern(const ora_scene* s, int64_t* row_ptr, int32_t* col) {
  std::memcpy(row_ptr, s->row_ptr.data(), sizeof(int64_t) * s->row_ptr.size());
  std::memcpy(col, s->col.data(), sizeof(int32_t) * s->col.size());
}

void ora_scene_tets(const ora_scene* s, int32_t* tets) {
  std::memcpy(tets, s->tets.data(), sizeof(int32_t) * s->tets.size());
}

void ora_scene_lumped_mass(const ora_scene* s, double* m) {
  std::memcpy(m, s->mass.data(), sizeof(double) * s->nv);
}

void ora_scene_set_params(ora_scene* s, const ora_params* p) {
  // the Dirichlet treatment (elimination or penalty) is fixed at creation; a
  // penalty scene may change its stiffness
  const double k = s->p.dirichlet_penalty;
  s->p = *p;
  if ((p->dirichlet_penalty > 0.0) != (k > 0.0) || !(p->dirichlet_penalty >= 0.0)) s->p.dirichlet_penalty = k;
}

int ora_scene_set_targets(ora_scene* s, const double* xyz) {
  std::memcpy(s->targets.data(), xyz, sizeof(double) * s->targets.size());
  return ORA_OK;
}

void ora_scene_get_state(const ora_scene* s, double* x, double* v) {
  if (x) std::memcpy(x, s->x.data(), sizeof(double) * 3 * s->nv);
  if (v) std::memcpy(v, s->v.data(), sizeof(double) * 3 * s->nv);
}

void ora_scene_set_state(ora_scene* s, const double* x, const double* v) {
  if (x) std::memcpy(s->x.data(), x, sizeof(double) * 3 * s->nv);
  if (v) std::memcpy(s->v.data(), v, sizeof(double) * 3 * s->nv);
}

void ora_scene_xhat(const ora_scene* s, double* xhat) {
  for (int64_t v = 0; v < s->nv; ++v)
    for (int k = 0; k < 3; ++k)
      xhat[3 * v + k] = s->x[3 * v + k] + s->dt * s->v[3 * v + k] + s->dt * s->dt * s->grav[k];
}

void ora_scene_set_solve_hook(ora_scene* s, ora_solve_hook hook, void* user) {
  s->hook = hook;
  s->hook_user = user;
}

double ora_scene_energy(const ora_scene* s, const double* x, const double* xhat) {
  return energy(s, x, xhat);
}

void ora_scene_gradient(const ora_scene* s, const double* x, const double* xhat, double* g) {
  std::vector<double> ge(12 * s->nt);
  for (int64_t e = 0; e < s->nt; ++e) element(s, e, x, nullptr, &ge[12 * e], nullptr);
  gradient_from(s, x, xhat, ge, g);
}

void ora_scene_element_eval(const ora_scene* s, const double* x, double* psi_e, double* ge,
                            double* He) {
  for (int64_t e = 0; e < s->nt; ++e)
    element(s, e, x, psi_e ? psi_e + e : nullptr, ge ? ge + 12 * e : nullptr,
            He ? He + 144 * e : nullptr);
}

void ora_scene_assemble(const ora_scene* s, const double* x, const uint8_t* proj, double* out) {
  std::vector<double> He(144 * s->nt), vals;
  for (int64_t e = 0; e < s->nt; ++e) element(s, e, x, nullptr, nullptr, &He[144 * e]);
  assemble(s, x, He, vals);
  if (proj) {
    std::vector<double> dH(144);
    for (int64_t e = 0; e < s->nt; ++e)
      if (proj[e]) {
        ora_project(12, &He[144 * e], s->p.eig_eps, s->p.projection, nullptr, dH.data());
        scatter_element(s, e, dH.data(), vals.data());
      }
  }
  std::memcpy(out, vals.data(), sizeof(double) * vals.size());
}

int64_t ora_scene_select(const ora_scene* s, const double* g, double delta, const uint8_t* already,
                         uint8_t* out_new) {
  return select(s, g, delta, already, out_new);
}

void ora_scene_project(const ora_scene* s, const double* x, const int32_t* sel, int64_t n_sel,
                       double* dH) {
  double H[144];
  for (int64_t i = 0; i < n_sel; ++i) {
    element(s, sel[i], x, nullptr, nullptr, H);
    ora_project(12, H, s->p.eig_eps, s->p.projection, nullptr, dH + 144 * i);
  }
}

int ora_scene_step(ora_scene* s, int mode, double tol, double* out_x, ora_step_stats* out) {
  if (mode < ORA_NEWTON || mode > ORA_PDN) return ORA_ERR_INVALID;
  const int64_t nv = s->nv, nt = s->nt, N = 3 * nv;
  const ora_params& p = s->p;
  std::vector<double> xn = s->x, vn = s->v, xhat(N), g(N), dx(N), xt(N);
  std::vector<double> He(144 * nt), ge(12 * nt), vals, dH(144);
  std::vector<uint8_t> proj(nt + nv), fresh(nt + nv);  // tets, then one contact element per vertex
  ora_scene_xhat(s, xhat.data());
  std::vector<double>& x = s->x;
  if (p.init_guess == 1)
    for (int64_t v = 0; v < nv; ++v)
      for (int k = 0; k < 3; ++k) x[3 * v + k] = xn[3 * v + k] + s->dt * vn[3 * v + k];
  for (size_t f = 0; f < s->fixed_list.size(); ++f)
    for (int k = 0; k < 3; ++k) x[3 * (int64_t)s->fixed_list[f] + k] = s->targets[3 * f + k];
  // Moving planes: a plane advances toward the bodies by at most ccd_safety times the
  // smallest distance of a free vertex to it; the rest of its motion waits for later
  // steps.  Every obstacle must leave the initial iterate strictly feasible.
  for (size_t k = 0; k < s->obst.size(); ++k) {
    ora_obstacle& o = s->obst[k];
    double m = kInf;
    for (int64_t v = 0; v < nv; ++v) {
      if (s->fixed[v]) continue;
      double d;
      if (ora_obstacle_eval(&o, x.data() + 3 * v, &d, nullptr, nullptr) != ORA_OK) d = -1.0;
      m = std::fmin(m, d);
    }
    if (!(m > 0.0)) {
      g_err = "the state is not feasible for obstacle " + std::to_string(k);
      return ORA_ERR_INVALID;
    }
    const ora_obstacle& q = s->obst_req[k];
    if (o.type == ORA_OBST_PLANE) {
      const double adv = o.a[0] * (q.p[0] - o.p[0]) + o.a[1] * (q.p[1] - o.p[1]) + o.a[2] * (q.p[2] - o.p[2]);
      const double f = adv > 0.0 ? std::fmin(1.0, p.ccd_safety * m / adv) : 1.0;
      for (int c = 0; c < 3; ++c) o.p[c] += f * (q.p[c] - o.p[c]);
    }
  }

  s->iters.clear();
  s->attempts.clear();
  s->attempt_sel.clear();
  s->iter_g.clear();
  double delta = kInf;  // Algorithm 1, before the Newton loop
  double g0 = -1.0;
  int status = ORA_ERR_NEWTON_MAXITER;
  int total_proj = 0, total_cg = 0, total_att = 0, total_ties = 0;
  int countdown = 0;  // PDN: iterations left that assemble projected

  for (int k = 0; k < p.newton_max_iter; ++k) {
    // elements are independent (each writes its own g^e, H^e): OpenMP shares them out
#pragma omp parallel for schedule(static)
    for (int64_t e = 0; e < nt; ++e) element(s, e, x.data(), nullptr, &ge[12 * e], &He[144 * e]);
    gradient_from(s, x.data(), xhat.data(), ge, g.data());
    if (s->record) s->iter_g.push_back(g);
    double gn2 = 0.0, gninf = 0.0;
    for (int64_t i = 0; i < N; ++i) {
      gn2 += g[i] * g[i];
      gninf = std::fmax(gninf, std::fabs(g[i]));
    }
    gn2 = std::sqrt(gn2);
    if (!std::isfinite(gn2)) {
      status = ORA_ERR_NONFINITE;
      break;
    }
    if (k == 0) g0 = gn2;
    const double floor = p.grad_floor * residual_scale(s, x.data(), xhat.data(), ge);
    if (p.tol_kind == 0 && (gn2 <= tol * g0 || gn2 <= floor)) {
      status = ORA_OK;
      break;
    }

    ora_iter_stats st;
    std::memset(&st, 0, sizeof(st));
    st.newton_iter = k;
    st.grad_norm2 = gn2;
    st.grad_norminf = gninf;

    // contact elements: one per free vertex within dhat of an obstacle, with its 3x3
    // barrier Hessian (the per-vertex potential of the contact model)
    std::vector<double> Hc;
    std::vector<uint8_t> cact(nv, 0);
    int n_elem = (int)nt;
    if (!s->obst.empty()) {
      Hc.assign(9 * (size_t)nv, 0.0);
      for (int64_t v = 0; v < nv; ++v) {
        if (s->fixed[v]) continue;
        bool act = false;
        vertex_contact(s, x.data() + 3 * v, nullptr, nullptr, &Hc[9 * v], &act);
        cact[v] = act;
        n_elem += act;
      }
    }
    // unprojected H (PN, and PDN within its countdown: every element clamped before assembly)
    assemble(s, x.data(), He, vals);
    std::fill(proj.begin(), proj.end(), 0);
    int n_proj = 0;
    auto project_one = [&](int64_t e) {  // in-place update with dH^e = Hhat^e - H^e
      if (e < nt) {
        ora_project(12, &He[144 * e], p.eig_eps, p.projection, nullptr, dH.data());
        scatter_element(s, e, dH.data(), vals.data());
      } else {
        const int64_t v = e - nt;
        double d3[9];
        ora_project(3, &Hc[9 * v], p.eig_eps, p.projection, nullptr, d3);
        double* blk = vals.data() + 9 * find_block(s, (int32_t)v, (int32_t)v);
        for (int q = 0; q < 9; ++q) blk[q] += d3[q];
      }
      proj[e] = 1;
    };
    auto project_all = [&]() {
      for (int64_t e = 0; e < nt + nv; ++e)
        if (!proj[e] && (e < nt || cact[e - nt])) project_one(e);
      n_proj = n_elem;
    };
    const bool pre = mode == ORA_PN || (mode == ORA_PDN && countdown > 0);
    if (pre) {
      project_all();
      if (mode == ORA_PDN) --countdown;
    }
    std::vector<double> b(N);
    for (int64_t i = 0; i < N; ++i) b[i] = -g[i];

    int info[4];
    int attempt = 0;
    int ties_pending = 0;               // ties of the selection rounds since the last solve
    std::vector<int32_t> sel_pending;   // elements they selected
    auto solve = [&](int n_new, double delta_used) {
      ora::pcg(nv, s->row_ptr.data(), s->col.data(), vals.data(), b.data(), p.pcg_rel_tol,
               pcg_max(s), dx.data(), info);
      if (s->hook) {
        const int o = s->hook(k, attempt, n_proj, s->hook_user);
        if (o >= 0) info[1] = o;
      }
      ora_attempt a;
      a.newton_iter = k;
      a.attempt = attempt;
      a.n_new_projected = n_new;
      a.ind = info[1];
      a.cg_iters = info[0];
      a.delta = delta_used;
      a.n_ties = ties_pending;
      s->attempts.push_back(a);
      s->attempt_sel.push_back(sel_pending);
      ties_pending = 0;
      sel_pending.clear();
      st.pcg_attempts += 1;
      st.cg_iters += info[0];
      st.precond_fail = info[2];
      ++attempt;
      return info[1] != 0;
    };

    bool ind = solve(pre ? n_elem : 0, kInf);
    bool fallback = ind && mode != ORA_PPN;
    if (mode == ORA_PDN && ind && !pre) {  // indefinite: project everything, solve again
      project_all();
      st.n_new_projected = n_elem;
      ind = solve(n_elem, -1.0);
      fallback = ind;
      countdown = p.pdn_countdown;
    }
    if (mode == ORA_PPN) {
      while (ind) {
        if (delta == kInf) delta = p.alpha * gninf;
        int64_t n_new = select(s, g.data(), delta, proj.data(), fresh.data());
        for (int64_t v = 0; v < nv; ++v) {  // contact elements: ||g_v||_inf > delta
          const int64_t e = nt + v;
          fresh[e] = 0;
          if (!cact[v] || proj[e]) continue;
          const double r = std::fmax(std::fabs(g[3 * v]), std::fmax(std::fabs(g[3 * v + 1]), std::fabs(g[3 * v + 2])));
          if (r > delta || delta <= p.eps_delta) {
            fresh[e] = 1;
            ++n_new;
          }
        }
        // ties: elements not yet projected whose key lies within tie_band delta of delta
        if (delta > p.eps_delta)
          for (int64_t e = 0; e < nt + nv; ++e) {
            if (proj[e] || (e >= nt && !cact[e - nt])) continue;
            double r;
            if (e < nt) {
              r = element_residual(s, e, g.data());
            } else {
              const int64_t v = e - nt;
              r = std::fmax(std::fabs(g[3 * v]), std::fmax(std::fabs(g[3 * v + 1]), std::fabs(g[3 * v + 2])));
            }
            if (std::fabs(r - delta) <= p.tie_band * delta) ++ties_pending, ++total_ties;
          }
        for (int64_t e = 0; e < nt + nv; ++e)
          if (fresh[e]) {
            project_one(e);
            sel_pending.push_back((int32_t)e);
          }
        n_proj += (int)n_new;
        st.n_new_projected += (int)n_new;
        if (n_new > 0) ind = solve((int)n_new, delta);  // unchanged matrix: same verdict
        if (ind) {
          if (n_proj == n_elem) {  // fully projected and still indefinite (rounding)
            fallback = true;
            break;
          }
          delta *= p.alpha;  // tighten
        }
      }
      delta *= p.beta;  // relax
    }
    st.n_projected_total = n_proj;
    st.delta = delta;
    total_proj += n_proj;
    total_cg += st.cg_iters;
    total_att += st.pcg_attempts;

    if (fallback) {
      bool zero = true;
      for (int64_t i = 0; i < N && zero; ++i) zero = (dx[i] == 0.0);
      st.fallback = zero ? fallback_direction(s, vals, g.data(), dx.data()) : 1;
    }
    double dd = 0.0;
    for (int64_t i = 0; i < N; ++i) dd += g[i] * dx[i];
    if (!(dd < 0.0)) {
      st.fallback = fallback_direction(s, vals, g.data(), dx.data());
      dd = 0.0;
      for (int64_t i = 0; i < N; ++i) dd += g[i] * dx[i];
    }
    st.dir_deriv = dd;

    // backtracking line search for sufficient decrease (Armijo)
    const double E0 = energy(s, x.data(), xhat.data());
    st.energy = E0;
    // intersection-based filtering: start at min(1, safety * first contact time)
    double gamma = 1.0, Et = 0.0;
    if (!s->obst.empty()) {
      double gmax = kInf;
      for (int64_t v = 0; v < nv; ++v) {
        if (s->fixed[v]) continue;
        for (const ora_obstacle& o : s->obst) gmax = std::fmin(gmax, ora_obstacle_ccd(&o, x.data() + 3 * v, dx.data() + 3 * v));
      }
      gamma = std::fmin(1.0, p.ccd_safety * gmax);
    }
    bool ok = false;
    for (int h = 0; h <= p.ls_max_halvings; ++h) {
      for (int64_t i = 0; i < N; ++i) xt[i] = x[i] + gamma * dx[i];
      Et = energy(s, xt.data(), xhat.data());
      // the FP64 sums resolve E only to a few ulps: a slack of ls_slack |E0| keeps a
      // step whose predicted decrease is below that resolution from being rejected
      if (Et <= E0 + p.armijo_c * gamma * dd + p.ls_slack * std::fabs(E0)) {
        ok = true;
        st.ls_halvings = h;
        break;
      }
      gamma *= 0.5;
    }
    if (!ok) {
      st.ls_halvings = p.ls_max_halvings;
      s->iters.push_back(st);
      status = ORA_ERR_LINESEARCH;
      break;
    }
    x = xt;
    st.gamma = gamma;
    st.energy_new = Et;
    s->iters.push_back(st);
    if (p.tol_kind == 1) {
      double m = 0.0;
      for (int64_t i = 0; i < N; ++i) m = std::fmax(m, std::fabs(gamma * dx[i]));
      if (m / s->dt < tol) {
        status = ORA_OK;
        break;
      }
    }
  }
  for (int64_t i = 0; i < N; ++i) s->v[i] = (x[i] - xn[i]) / s->dt;
  if (out_x) std::memcpy(out_x, x.data(), sizeof(double) * N);
  if (out) {
    out->newton_iters = (int)s->iters.size();
    out->total_projections = total_proj;
    out->total_cg_iters = total_cg;
    out->total_attempts = total_att;
    out->status = status;
    out->n_ties = total_ties;
  }
  return status;
}

int ora_scene_iter_stats(const ora_scene* s, ora_iter_stats* buf, int cap) {
  const int n = (int)s->iters.size();
  for (int i = 0; i < n && i < cap; ++i) buf[i] = s->iters[i];
  return n;
}

int ora_scene_attempts(const ora_scene* s, ora_attempt* buf, int cap) {
  const int n = (int)s->attempts.size();
  for (int i = 0; i < n && i < cap; ++i) buf[i] = s->attempts[i];
  return n;
}

void ora_scene_set_record(ora_scene* s, int on) {
  s->record = on != 0;
  s->iter_g.clear();
}

int ora_scene_iteration_gradient(const ora_scene* s, int k, double* g) {
  if (k < 0 || k >= (int)s->iter_g.size()) return -1;
  std::memcpy(g, s->iter_g[k].data(), sizeof(double) * s->iter_g[k].size());
  return 0;
}

int64_t ora_scene_attempt_selection(const ora_scene* s, int idx, int32_t* buf, int64_t cap) {
  if (idx < 0 || idx >= (int)s->attempt_sel.size()) return -1;
  const std::vector<int32_t>& l = s->attempt_sel[idx];
  for (int64_t i = 0; i < (int64_t)l.size() && i < cap; ++i) buf[i] = l[i];
  return (int64_t)l.size();
}

}  // extern "C"

// Requested poses; the applied ones follow them at the next step (planes as far as
// feasible).  A new set of a different size or kind is applied at once.
extern "C" void ora_scene_set_obstacles(ora_scene* s, const ora_obstacle* obs, int n) {
  s->obst_req.assign(obs, obs + (n > 0 ? n : 0));
  bool same = s->obst.size() == s->obst_req.size();
  for (size_t k = 0; same && k < s->obst.size(); ++k)
    same = s->obst[k].type == s->obst_req[k].type && s->obst[k].a[0] == s->obst_req[k].a[0] &&
           s->obst[k].a[1] == s->obst_req[k].a[1] && s->obst[k].a[2] == s->obst_req[k].a[2];
  if (!same) s->obst = s->obst_req;
  for (size_t k = 0; k < s->obst.size(); ++k)
    if (s->obst[k].type != ORA_OBST_PLANE) s->obst[k] = s->obst_req[k];  // only planes are held back
}
