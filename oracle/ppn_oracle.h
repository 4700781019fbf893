/*
 * FP64 CPU oracle for Progressively Projected Newton (arXiv 2505.21013).
 *
 * TEST INFRASTRUCTURE ONLY.  This library is the slow, plain reference that the
 * CUDA path is checked against.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load it; the product library never links,
 * loads or calls it, and it shares no code, header or table with the product.
 *
 * What it computes, and where each part comes from:
 *   - Newton's method on the incremental potential, H dx = -g with
 *     H = sum_e H^e and g = sum_e g^e                       (Sec. 3, Eq. newton)
 *   - descent identity dx^T g = -dx^T H dx                   (Sec. 3, Eq. spd)
 *   - per-element eigenvalue clamping H^e = Q D Q^T ->
 *     Q max(D, eps) Q^T, eps = 1e-8                          (Sec. 3; Sec. 5.1)
 *   - residual heuristic ||S^e g||_inf > delta, delta schedule
 *     alpha = 0.5, beta = 2, eps_delta = 1e-12               (Sec. 4, "Projection heuristic")
 *   - Algorithm 1 (PPN), with PN (project all) and plain Newton (project none)
 *   - in-place incremental update dH^e = Hhat^e - H^e        (Sec. 4.1, "Incremental Hessian updates")
 *   - PCG with negative-curvature exit, zero initial guess   (Sec. 4.1, "Linear Solvers")
 *   - 3x3 block-diagonal preconditioner, PCG tol 1e-4        (Sec. 5.1)
 *   - backward Euler incremental potential, Stable Neo-Hookean tets,
 *     backtracking line search                                (Sec. 2.1, Sec. 5.1)
 *
 * Readings where the paper is silent or leaves a choice open:
 *   - psi(F) = mu/2 (tr F^T F - 3) - mu (J - 1) + lam_s/2 (J - 1)^2 with
 *     mu = E / (2 (1 + nu)), lam_s = E nu / ((1 + nu)(1 - 2 nu)) + mu.
 *   - Psi(x) = sum_free m_v / (2 dt^2) |x_v - xhat_v|^2 + sum_e V_e psi(F_e),
 *     xhat = x_n + dt v_n + dt^2 a_grav, lumped mass m_v = sum_{e ∋ v} rho V_e / 4.
 *   - Dirichlet vertices are eliminated: set to their targets, zero gradient,
 *     identity diagonal block, zero coupling blocks.
 *   - negative curvature is d^T H d <= 0; a diagonal block that fails a 3x3
 *     Cholesky also reports indefiniteness before any CG iteration.
 *   - selection is strict (r_e > delta); a re-solve after a round that
 *     projected no new element is skipped (the matrix is unchanged).
 *   - Armijo c = 1e-4, gamma0 = 1, halving, at most 30 halvings.
 *
 * Layouts: positions are (n_v, 3) row-major doubles; tets are (n_t, 4) int32,
 * 0-based; element vectors are ordered (vertex a, component k) -> 3a + k;
 * BSR blocks are 3x3 row-major (block k occupies vals[9k .. 9k+8]), full
 * symmetric pattern, columns sorted, diagonal included.
 */
#ifndef PPN_ORACLE_H
#define PPN_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum { ORA_NEWTON = 0, ORA_PN = 1, ORA_PPN = 2, ORA_PDN = 3 };
enum { ORA_PROJ_CLAMP = 0, ORA_PROJ_MIRROR = 1 };

enum {
  ORA_OK = 0,
  ORA_ERR_INVALID = 1,
  ORA_ERR_DEGENERATE = 2,
  ORA_ERR_LINESEARCH = 3,
  ORA_ERR_NEWTON_MAXITER = 4,
  ORA_ERR_NONFINITE = 5
};

typedef struct {
  double alpha;        /* tightening factor, default 0.5 */
  double beta;         /* release factor, default 2 */
  double eps_delta;    /* fall back to PN below this delta, default 1e-12 */
  double eig_eps;      /* clamp value, default 1e-8 */
  double pcg_rel_tol;  /* ||r|| / ||r0||, default 1e-4 */
  double armijo_c;     /* default 1e-4 */
  int pcg_max_iter;    /* 0 -> max(1000, 3 n_v) */
  int newton_max_iter; /* default 100 */
  int ls_max_halvings; /* default 30 */
  int tol_kind;        /* 0: ||g||_2 <= tol ||g0||_2 ; 1: ||gamma dx||_inf / dt < tol */
  int init_guess;      /* 0: x_n ; 1: x_n + dt v_n (free vertices) */
  int pdn_countdown;   /* PDN: iterations that stay projected after an indefinite solve, default 4 */
  int projection;      /* ORA_PROJ_CLAMP: max(lambda, eps); ORA_PROJ_MIRROR: max(|lambda|, eps) */
  double grad_floor;   /* tol_kind 0 also stops at ||g||_2 <= grad_floor ||s||_2 (rounding floor), default 1e-12 */
  double ls_slack;     /* Armijo test allows ls_slack |E0| of energy rounding, default 1e-12 */
  double contact_kappa; /* barrier stiffness kappa [N/m], default 1e3 */
  double contact_dhat;  /* barrier activation distance dhat [m], default 1e-3 */
  double ccd_safety;    /* line search starts at min(1, ccd_safety * gamma_ccd), default 0.9 */
  double dirichlet_penalty; /* 0: Dirichlet vertices eliminated (default); k > 0: they stay free and
                               carry the penalty potential k m_v / (2 dt^2) |x_v - t_v|^2 */
  double tie_band;     /* a selection tie: an element not yet projected with |r_e - delta| <= tie_band
                          delta (counted, not a change of the strict test r_e > delta), default 1e-12 */
} ora_params;

/* analytic obstacles for frictionless log-barrier contact (contact.cpp) */
enum { ORA_OBST_PLANE = 0, ORA_OBST_CYLINDER_IN = 1, ORA_OBST_SPHERE_OUT = 2 };
typedef struct {
  int type;   /* ORA_OBST_* */
  double p[3]; /* plane point / axis point / centre */
  double a[3]; /* plane unit normal (bodies on the positive side) / cylinder unit axis */
  double r;    /* cylinder or sphere radius */
} ora_obstacle;

typedef struct {
  int newton_iter;
  int pcg_attempts;
  int cg_iters;
  int n_new_projected;
  int n_projected_total;
  int ls_halvings;
  int fallback;        /* 1: last CG iterate used, 2: preconditioned gradient, 3: mass-scaled gradient */
  int precond_fail;    /* last solve failed the block Cholesky */
  double grad_norm2;
  double grad_norminf;
  double delta;        /* delta after the relax step of this iteration */
  double gamma;
  double energy;       /* Psi at the start of the iteration */
  double energy_new;   /* Psi after the update */
  double dir_deriv;    /* g^T dx of the accepted direction */
} ora_iter_stats;

typedef struct {
  int newton_iter;
  int attempt;         /* 0 = first solve on the unprojected matrix */
  int n_new_projected; /* newly projected before this solve */
  int ind;
  int cg_iters;
  double delta;        /* delta used for the selection before this solve (inf for attempt 0) */
  int n_ties;          /* selection ties of the rounds since the previous solve */
} ora_attempt;

typedef struct {
  int newton_iters;
  int total_projections;
  int total_cg_iters;
  int total_attempts;
  int status;
  int n_ties;          /* selection ties of every round of the step */
} ora_step_stats;

typedef struct ora_scene ora_scene;

/* Optional hook replacing the indefiniteness verdict of a solve (tests of the
 * delta schedule).  Return -1 to keep the real verdict, 0 or 1 to override. */
typedef int (*ora_solve_hook)(int newton_iter, int attempt, int n_projected_total, void* user);

/* obstacles of the scene for the next step (copied).  A plane of the same normal as
 * before is moved toward the bodies only as far as keeps the step's initial iterate
 * feasible (ccd_safety x the smallest vertex distance); the rest follows in later
 * steps.  A set of another size, kind or normal replaces the old one at once. */
void ora_scene_set_obstacles(ora_scene* s, const ora_obstacle* obs, int n);
ora_params ora_default_params(void);
/* threads the oracle's parallel loops use (OMP_NUM_THREADS; 1 without OpenMP).  Only
 * loops over independent elements and SpMV rows run in parallel: the results do not
 * depend on the thread count. */
int ora_num_threads(void);
void ora_set_num_threads(int n); /* n > 0; no effect without OpenMP */
const char* ora_last_error(void);

/* ---- material (Stable Neo-Hookean reading) ---- */
void ora_lame(double E, double nu, double* mu, double* lam_s);
double ora_snh_psi(const double* F, double mu, double lam_s);
void ora_snh_pk1(const double* F, double mu, double lam_s, double* P);
void ora_snh_dpdf(const double* F, double mu, double lam_s, double* A81);

/* ---- one tet ---- */
/* rest corners X (12), current corners x (12); outputs may be NULL */
int ora_tet_eval(const double* X, const double* x, double mu, double lam_s,
                 double* psi_e, double* g12, double* H144);

/* ---- dense symmetric eigen (cyclic Jacobi) and clamping ---- */
int ora_eigh(int n, const double* A, double* w, double* Q);
int ora_clamp(int n, const double* H, double eps, double* Hhat, double* dH);
/* barrier b(d) and its first two derivatives; d <= 0 gives b = +inf and ORA_ERR_INVALID */
int ora_barrier(double d, double dhat, double* b, double* db, double* ddb);
/* distance to an obstacle with its gradient (3) and Hessian (9); any output may be NULL */
int ora_obstacle_eval(const ora_obstacle* o, const double* x, double* d, double* grad, double* hess);
/* first gamma > 0 at which x + gamma dx reaches the obstacle, or +infinity */
double ora_obstacle_ccd(const ora_obstacle* o, const double* x, const double* dx);
/* the same with a projection kind: ORA_PROJ_CLAMP or ORA_PROJ_MIRROR */
int ora_project(int n, const double* H, double eps, int kind, double* Hhat, double* dH);

/* ---- BSR PCG on a caller matrix ---- */
/* info[0] = iterations, info[1] = ind, info[2] = precond_fail, info[3] = hit max_iter */
int ora_pcg_bsr(int64_t n_rows, const int64_t* row_ptr, const int32_t* col, const double* vals,
                const double* b, double rel_tol, int max_iter, double* x, int* info);

/* ---- scenes ---- */
ora_scene* ora_scene_create(const double* rest, int64_t n_v, const int32_t* tets, int64_t n_t,
                            double E, double nu, double rho, double dt, const double* gravity,
                            const int32_t* fixed, int64_t n_fixed, const ora_params* params);
void ora_scene_destroy(ora_scene* s);
int64_t ora_scene_nnzb(const ora_scene* s);
void ora_scene_pattern(const ora_scene* s, int64_t* row_ptr, int32_t* col);
void ora_scene_tets(const ora_scene* s, int32_t* tets);           /* after orientation */
void ora_scene_lumped_mass(const ora_scene* s, double* m);
/* replaces the parameters; dirichlet_penalty keeps its creation value when it
   would switch between elimination (0) and penalty (> 0) */
void ora_scene_set_params(ora_scene* s, const ora_params* p);
int ora_scene_set_targets(ora_scene* s, const double* xyz_fixed);
void ora_scene_get_state(const ora_scene* s, double* x, double* v);
void ora_scene_set_state(ora_scene* s, const double* x, const double* v);
void ora_scene_xhat(const ora_scene* s, double* xhat);              /* of the next step */
void ora_scene_set_solve_hook(ora_scene* s, ora_solve_hook hook, void* user);

double ora_scene_energy(const ora_scene* s, const double* x, const double* xhat);
void ora_scene_gradient(const ora_scene* s, const double* x, const double* xhat, double* g);
void ora_scene_element_eval(const ora_scene* s, const double* x, double* psi_e, double* ge,
                            double* He);
/* proj: n_t flags (NULL = none); projected elements enter as Hhat^e */
void ora_scene_assemble(const ora_scene* s, const double* x, const uint8_t* proj, double* vals);
/* marks new[e] = 1 for elements not in `already` with r_e > delta or delta <= eps_delta */
int64_t ora_scene_select(const ora_scene* s, const double* g, double delta,
                         const uint8_t* already, uint8_t* out_new);
/* dH for a list of elements at positions x: n_sel * 144 */
void ora_scene_project(const ora_scene* s, const double* x, const int32_t* sel, int64_t n_sel,
                       double* dH);

int ora_scene_step(ora_scene* s, int mode, double tol, double* out_x, ora_step_stats* out);
int ora_scene_iter_stats(const ora_scene* s, ora_iter_stats* buf, int cap);
int ora_scene_attempts(const ora_scene* s, ora_attempt* buf, int cap);
/* elements newly selected by the PPN rounds before attempt `idx` of the last step, ascending
 * (tets e in [0, n_t), the contact element of vertex v as n_t + v); attempts without a
 * PPN selection (the first solve, PN, PDN) have none.  Returns the count (-1: no such
 * attempt); at most cap are written. */
int64_t ora_scene_attempt_selection(const ora_scene* s, int idx, int32_t* buf, int64_t cap);
/* with recording on, the assembled gradient of every Newton iteration of the next steps is
 * kept (3 n_v doubles each); ora_scene_iteration_gradient copies that of iteration k of the
 * last step and returns 0, or -1 when there is none */
void ora_scene_set_record(ora_scene* s, int on);
int ora_scene_iteration_gradient(const ora_scene* s, int k, double* g);

#ifdef __cplusplus
}
#endif

#endif
