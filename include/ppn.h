/*
 * ppn.h — C ABI of the GB300 (sm_103a) Progressively Projected Newton library.
 *
 * The library advances implicit-Euler tetrahedral FEM scenes by one time step
 * per call, minimising the incremental potential with Newton's method in one
 * of three modes (arXiv 2505.21013):
 *   PPN_MODE_NEWTON  no element Hessian is projected            (Sec. 1, Sec. 3)
 *   PPN_MODE_PN      every element Hessian is clamped           (Sec. 3, "Projected Newton")
 *   PPN_MODE_PPN     Algorithm 1: elements with ||S^e g||_inf > delta are
 *                    clamped in place only after the linear solver reports
 *                    indefiniteness; delta tightens by alpha, relaxes by beta (Sec. 4)
 * Every step of the per-iteration pipeline runs in this library's CUDA kernels.
 *
 * Conventions shared by every entry point:
 *   - Host pointers unless a name ends in _device.  Inputs are copied; the
 *     library keeps no caller pointer after a call returns.
 *   - Positions and velocities are (n_verts, 3) row-major doubles; tets are
 *     (n_tets, 4) int32, 0-based.  Tet orientation is normalised at creation
 *     (two corners swapped when det[x1-x0, x2-x0, x3-x0] < 0).
 *   - Every call returns a ppn_status; the library never aborts.  On failure
 *     ppn_last_error() (thread-local) holds a one-line reason.  Device waits
 *     inside kernels are bounded and report PPN_ERR_TIMEOUT.
 *   - A scene owns its device memory (cudaMalloc at creation, or the allocator
 *     installed with ppn_set_allocator; freed at destruction) and runs on its own
 *     stream unless ppn_set_stream is called.
 *   - Not thread-safe per scene: calls on one scene must not overlap.
 */
#ifndef PPN_H
#define PPN_H

#include <stdint.h>

#if defined(__GNUC__)
#define PPN_API __attribute__((visibility("default")))
#else
#define PPN_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef struct ppn_scene ppn_scene;

typedef enum {
  PPN_OK = 0,
  PPN_ERR_INVALID_ARG = 1,
  PPN_ERR_OOM = 2,
  PPN_ERR_CUDA = 3,
  PPN_ERR_DEGENERATE_TET = 4,
  PPN_ERR_LINESEARCH = 5,
  PPN_ERR_NEWTON_MAXITER = 6,
  PPN_ERR_PCG_MAXITER = 7,
  PPN_ERR_NONFINITE = 8,
  PPN_ERR_TIMEOUT = 9,
  PPN_ERR_ADMISSION = 10
} ppn_status;

/* NEWTON: project nothing; PN: clamp every element Hessian before assembly;
 * PPN: Algorithm 1; PDN: project-on-demand, the comparison method of Sec. 2.2 /
 * Sec. 5.1 (solve unprojected; on indefiniteness project every element and
 * solve again, then stay projected for pdn_countdown iterations). */
typedef enum { PPN_MODE_NEWTON = 0, PPN_MODE_PN = 1, PPN_MODE_PPN = 2, PPN_MODE_PDN = 3 } ppn_mode;

/* element projection: CLAMP max(lambda, eps) (Sec. 3, the paper's default);
 * MIRROR max(|lambda|, eps) (eigenvalue mirroring, compared in Sec. 5.2) */
typedef enum { PPN_PROJ_CLAMP = 0, PPN_PROJ_MIRROR = 1 } ppn_projection;

/* FP64: every step in double.  MIXED: element Hessians, eigensolves, the BSR
 * matrix and PCG in float; element energies, the assembled gradient and its
 * norms, dot products, line-search sums and the position update in double. */
typedef enum { PPN_PREC_FP64 = 0, PPN_PREC_MIXED = 1 } ppn_precision;

typedef struct {
  double E;   /* Young's modulus [Pa] */
  double nu;  /* Poisson ratio, (-1, 0.5) */
  double rho; /* density [kg/m^3] */
} ppn_material;

typedef struct {
  double alpha;        /* delta tightening factor, Sec. 4 (default 0.5) */
  double beta;         /* delta release factor, Sec. 4 (default 2) */
  double eps_delta;    /* project every element once delta <= eps_delta (1e-12) */
  double eig_eps;      /* eigenvalue clamp, Sec. 5.1 (1e-8) */
  double pcg_rel_tol;  /* PCG stop at ||r|| <= tol ||r0||, Sec. 5.1 (1e-4) */
  double armijo_c;     /* sufficient-decrease constant (1e-4) */
  double gravity[3];   /* (0, -9.81, 0) */
  int pcg_max_iter;    /* 0: max(1000, 3 n_verts) */
  int newton_max_iter; /* 100 */
  int ls_max_halvings; /* 30 */
  int precision;       /* ppn_precision (PPN_PREC_MIXED) */
  int tol_kind;        /* 0: ||g||_2 <= tol ||g0||_2 ; 1: ||gamma dx||_inf / dt < tol (Sec. 5.1) */
  int init_guess;      /* 0: x_n ; 1: x_n + dt v_n */
  int pdn_countdown;   /* PDN: iterations that stay projected after an indefinite solve (4, Sec. 5.1) */
  int projection;      /* ppn_projection (PPN_PROJ_CLAMP) */
  double grad_floor;   /* tol_kind 0 also stops at ||g||_2 <= grad_floor ||s||_2, s_v = m_v|x_v - xhat_v|/dt^2
                        * + sum_e |g^e_v| (the rounding floor of the residual; 1e-12) */
  double ls_slack;     /* the Armijo test allows ls_slack |E0| of energy rounding (1e-12) */
  double contact_kappa; /* barrier stiffness kappa [N/m] of the contact potential (1e3) */
  double contact_dhat;  /* barrier activation distance dhat [m] (1e-3) */
  double ccd_safety;    /* the line search starts at min(1, ccd_safety x first contact time) (0.9) */
  double dirichlet_penalty; /* 0: Dirichlet vertices eliminated (default).  k > 0: Dirichlet
                             * constraints by penalty potentials (Sec. 5.1): the constrained vertices
                             * stay free and carry k m_v / (2 dt^2) |x_v - t_v|^2, t_v the target; new
                             * targets take effect at once.  Fixed at scene creation; finite, >= 0. */
  double tie_band;     /* selection ties (Algorithm 1's strict test r_e > delta, Sec. 4): an element not
                        * yet projected with |r_e - delta| <= tie_band delta is counted as a tie in the
                        * attempt and step statistics (the strict test still decides).  0: by precision,
                        * 1e-12 in FP64, 1e-5 in the mixed mode (0).  Finite, >= 0. */
} ppn_params;

typedef struct {
  int newton_iter;
  int pcg_attempts;      /* solves in this iteration (1 + PPN retries) */
  int cg_iters;          /* CG iterations summed over those solves */
  int n_new_projected;   /* elements projected in this iteration */
  int n_projected_total; /* |H_p| at the end of the iteration */
  int ls_halvings;
  int fallback;          /* 0 none, 1 last CG iterate, 2 preconditioned gradient, 3 mass-scaled gradient */
  int precond_fail;      /* the last solve's block-Jacobi setup met a non-SPD diagonal block */
  double grad_norm2;
  double grad_norminf;
  double delta;          /* after the relax step */
  double gamma;
  double energy;         /* incremental potential at the start of the iteration */
  double energy_new;     /* after the update */
  double dir_deriv;      /* g^T dx */
} ppn_iter_stats;

typedef struct {
  int newton_iter;
  int attempt;           /* 0 = first solve on the unprojected matrix */
  int n_new_projected;
  int ind;               /* the solver reported indefiniteness */
  int cg_iters;
  double delta;          /* delta of the selection before this solve (inf for attempt 0) */
  int n_ties;            /* selection ties (params.tie_band) of the rounds since the previous solve */
} ppn_attempt;

typedef struct {
  int newton_iters;
  int total_projections;
  int total_cg_iters;
  int total_attempts;
  int status;            /* ppn_status of the step */
  double final_grad_norm2;
  double device_ms;      /* stream time between the step's first and last kernel */
  int n_ties;            /* selection ties of every PPN selection round of the step */
} ppn_step_stats;

typedef struct {
  int64_t n_verts, n_tets, n_fixed, nnzb, n_map;
  int64_t device_bytes;  /* device memory owned by the scene */
  int precision;
  /* layout of the scene's last linear solve: -1 none yet; FP32 single-reduction
   * kernel 0 resident, 1 blocks streamed, 2 global vectors, 3 resident with the
   * halo replicated; 4 the standard resident kernel; 5 the global-memory kernel */
  int pcg_layout;
} ppn_scene_info;

/* Per kernel family: launches and summed device time (CUDA events on the scene
 * stream) since the last reset; filled only while profiling is on. */
typedef struct {
  char name[32];
  int64_t launches;
  double total_ms;
  double bytes;          /* algorithmic bytes moved by those launches */
} ppn_kernel_time;

PPN_API ppn_params ppn_default_params(void);
PPN_API const char* ppn_status_string(ppn_status s);
PPN_API const char* ppn_last_error(void);

/* Scene creation (problem statement of Sec. 3 with the backward-Euler
 * incremental potential of Sec. 2.1/5.1).  rest_xyz: n_verts*3 rest positions
 * (also the initial state, zero velocity); tets: n_tets*4; fixed: n_fixed
 * Dirichlet vertex indices (targets default to their rest positions).
 * params NULL = defaults.  Errors: INVALID_ARG (sizes, indices, material),
 * DEGENERATE_TET (|det| <= 1e-14 h^3), OOM, CUDA. */
PPN_API ppn_status ppn_create_scene(const double* rest_xyz, int64_t n_verts, const int32_t* tets,
                            int64_t n_tets, const ppn_material* mat, double dt,
                            const int32_t* fixed, int64_t n_fixed, const ppn_params* params,
                            ppn_scene** out);
PPN_API void ppn_destroy_scene(ppn_scene* s);
PPN_API ppn_status ppn_scene_get_info(const ppn_scene* s, ppn_scene_info* out);

/* Use a caller stream (a cudaStream_t passed as void*); NULL = the scene's own. */
PPN_API ppn_status ppn_set_stream(ppn_scene* s, void* cuda_stream);

/* Device memory from a caller's allocator (e.g. a framework's caching allocator).
 * By default scenes, the scene groups that step them together and servers take their
 * device buffers from cudaMalloc.  ppn_set_allocator installs alloc_fn / free_fn for
 * the owners created after the call; each owner keeps the allocator it was created
 * with until it is destroyed, so the caller keeps both functions and ctx valid that
 * long.  alloc_fn(bytes, ctx) returns device memory of the current device, aligned to
 * at least 256 bytes, or NULL: the creation then fails with PPN_ERR_OOM (a pointer
 * that is not 256-byte aligned is handed back to free_fn and counts as a failure).
 * free_fn(ptr, ctx) releases a pointer alloc_fn returned; the library synchronises the
 * owner's stream first.  Both are called from the thread that creates, steps or
 * destroys the owner.  Both NULL restores cudaMalloc / cudaFree; exactly one NULL is
 * PPN_ERR_INVALID_ARG.  Pinned host staging buffers are not affected. */
typedef void* (*ppn_device_alloc_fn)(size_t bytes, void* ctx);
typedef void (*ppn_device_free_fn)(void* ptr, void* ctx);
PPN_API ppn_status ppn_set_allocator(ppn_device_alloc_fn alloc_fn, ppn_device_free_fn free_fn, void* ctx);

/* Dirichlet targets for the next step, n_fixed*3 doubles in the order of `fixed`. */
PPN_API ppn_status ppn_set_kinematic_targets(ppn_scene* s, const double* xyz_of_fixed);
PPN_API ppn_status ppn_set_kinematic_targets_device(ppn_scene* s, const double* xyz_of_fixed_device);

/* One backward-Euler step (Algorithm 1 for PPN).  tol: see params.tol_kind.
 * out_xyz: n_verts*3 host buffer for the new positions, or NULL.  out: may be NULL.
 * Returns the step status (also in out->status); the state advances even on
 * NEWTON_MAXITER (last iterate kept). */
PPN_API ppn_status ppn_step(ppn_scene* s, ppn_mode mode, double tol, double* out_xyz,
                    ppn_step_stats* out);

/* Same step for several scenes advanced together: every kernel of a phase is
 * one launch over all scenes that are still iterating.  All scenes must share
 * the precision.  out: n entries or NULL.  Returns the first non-OK status. */
PPN_API ppn_status ppn_step_batch(ppn_scene* const* scenes, int n, const ppn_mode* modes, double tol,
                          ppn_step_stats* out);

PPN_API ppn_status ppn_get_iter_stats(const ppn_scene* s, ppn_iter_stats* buf, int cap, int* n_written);
PPN_API ppn_status ppn_get_attempts(const ppn_scene* s, ppn_attempt* buf, int cap, int* n_written);
/* Selected sets of Algorithm 1 (Sec. 4: each round projects the elements with
 * ||S^e g||_inf > delta that are not yet projected).  With recording on, every
 * following step keeps, per attempt (the order of ppn_get_attempts), the elements
 * that the PPN selection rounds since the previous solve chose: tets as their index
 * e, contact elements as n_tets + v.  Attempts without a PPN selection (the first
 * solve of an iteration, PN, PDN) have none.  Recording copies each selection to
 * the host (diagnostics; it adds a device synchronisation per round). */
PPN_API ppn_status ppn_set_record_selection(ppn_scene* s, int on);
/* The elements of attempt idx of the last step, ascending; *n receives their count
 * and min(cap, count) are written to buf (buf may be NULL when cap is 0).
 * INVALID_ARG when idx is out of range or recording was off during the step. */
PPN_API ppn_status ppn_get_attempt_selection(const ppn_scene* s, int idx, int32_t* buf, int64_t cap, int64_t* n);
/* With recording on (ppn_set_record_selection), the assembled gradient g of Newton
 * iteration newton_iter of the last step, the vector the selection keys of Sec. 4
 * (||S^e g||_inf) are taken from: n_verts*3 doubles, zero on eliminated Dirichlet
 * vertices.  Every evaluated iterate is kept, also the last one (where the step
 * stopped).  INVALID_ARG when no such record exists. */
PPN_API ppn_status ppn_get_iteration_gradient(const ppn_scene* s, int newton_iter, double* g);
PPN_API ppn_status ppn_get_state(const ppn_scene* s, double* x, double* v);
PPN_API ppn_status ppn_set_state(ppn_scene* s, const double* x, const double* v);
/* Exact checkpoint of the internal state: displacement u = x - rest and
 * velocity, n_verts*3 doubles each (either may be NULL).  Restoring it and
 * stepping reproduces an uninterrupted run bit for bit. */
PPN_API ppn_status ppn_get_displacement(const ppn_scene* s, double* u, double* v);
PPN_API ppn_status ppn_set_displacement(ppn_scene* s, const double* u, const double* v);

/* The FP32 linear solver's autotuner (process-wide).  Where several launch configurations of
 * the single-reduction PCG give bitwise-identical results (the streamed layouts: vectors in
 * shared memory with the blocks streamed, or everything in global memory; and the L2
 * priority of the streamed blocks: evict-first, or normal, which lets a matrix smaller than
 * L2 stay resident), the first launches of each shape class try each configuration, timed
 * by CUDA events, and later launches keep the fastest per CG iteration.  One record per
 * shape class seen so far; n_written receives the count, at most cap are written. */
typedef struct {
  int tiles_per_cta;     /* shape class: 128-row tiles of the busiest CTA, */
  int blocks_per_row;    /* BSR blocks per row, */
  int log2_matrix_mb;    /* and floor(log2(the launch's matrix in MB)) */
  int choice;            /* kept configuration: layout (0 streamed blocks, 1 global vectors) + 2 x
                          * L2 priority (0 evict-first, 1 normal); -1 while still exploring */
  int launches[4];       /* timed launches of each configuration (0: untried or not allowed) */
  double us_per_iter[4]; /* their mean device time per CG iteration */
} ppn_pcg_tuning;
PPN_API ppn_status ppn_get_pcg_tuning(ppn_pcg_tuning* buf, int cap, int* n_written);

PPN_API ppn_status ppn_set_profiling(ppn_scene* s, int on);
PPN_API ppn_status ppn_get_kernel_times(const ppn_scene* s, ppn_kernel_time* buf, int cap, int* n_written);

/* ---- stage probes: run one stage of the pipeline on caller data (host
 * buffers) through the scene's kernels, leaving the scene's state unchanged.
 * Used by the parity tests; all outputs are widened to double. ---- */

/* psi_e: n_tets element energies (FP64 kernel); ge: n_tets*12 element
 * gradients; He: n_tets*144 element Hessians (12x12 row-major, vertex-major
 * DOF order 3a+k).  Any output may be NULL. */
PPN_API ppn_status ppn_probe_elements(ppn_scene* s, const double* x, double* psi_e, double* ge,
                              double* He);
/* assembled gradient (zero on Dirichlet vertices), norms[0] = ||g||_2, norms[1] = ||g||_inf,
 * energy = incremental potential at x (any output may be NULL) */
PPN_API ppn_status ppn_probe_gradient(ppn_scene* s, const double* x, const double* xhat, double* g,
                              double* norms, double* energy);
/* BSR pattern: row_ptr (n_verts+1), col (nnzb) */
PPN_API ppn_status ppn_probe_pattern(const ppn_scene* s, int64_t* row_ptr, int32_t* col);
/* assembled matrix at x: vals nnzb*9 (3x3 row-major blocks); proj: n_tets flags
 * (NULL = none) of elements that enter projected */
PPN_API ppn_status ppn_probe_assemble(ppn_scene* s, const double* x, const uint8_t* proj, double* vals);
/* K4 selection on a given assembled gradient g (n_verts*3): out_new (n_tets flags),
 * n_new, and n_ties, the elements not in `already` within the tie band of delta
 * (params.tie_band); any output may be NULL */
PPN_API ppn_status ppn_probe_select(ppn_scene* s, const double* g, double delta, const uint8_t* already,
                            uint8_t* out_new, int64_t* n_new, int64_t* n_ties);
/* tets after the orientation normalisation of ppn_create_scene (n_tets*4 int32),
 * as the kernels read them */
PPN_API ppn_status ppn_probe_tets(const ppn_scene* s, int32_t* tets);
/* K5 clamping updates dH^e = Hhat^e - H^e (n_sel*144) of the listed elements at x */
PPN_API ppn_status ppn_probe_project(ppn_scene* s, const double* x, const int32_t* sel, int64_t n_sel,
                             double* dH);
/* block-Jacobi PCG on the scene's pattern with values vals (nnzb*9) and right-hand
 * side b (n_verts*3); info: [iterations, ind, precond_fail, hit_max] */
/* Bounded-wait check (the grid-wide waits of the PCG kernels, Sec. 4.1 "Linear
 * Solvers" runs the solve as one resident kernel): one warp polls n_words stamped
 * 64-bit words in device memory with the PCG's wait routine, at most spin_limit
 * rounds.  preset != 0 sets the words first (the wait succeeds: PPN_OK); preset
 * == 0 leaves them at zero, nothing else writes them, and the wait runs out:
 * PPN_ERR_TIMEOUT.  The device stays usable either way.  1 <= n_words <= 4096,
 * 1 <= spin_limit <= 1<<20, else PPN_ERR_INVALID_ARG.  Allocates and frees its own
 * words on the current device. */
PPN_API ppn_status ppn_probe_bounded_wait(int n_words, int spin_limit, int preset);

/* Host-side tables of the linear solver's halo layout (Sec. 4.1's block-Jacobi
 * PCG, one CTA per SM; no GPU needed): for each CTA, the rows of other CTAs that
 * columns of its rows refer to, and each block's column in the CTA's local
 * numbering.  n_scenes (1..8) BSR patterns in launch order: row_ptr[k]
 * (n_verts[k] + 1 int64) and col[k] (row_ptr[k][n_verts[k]] int32, ascending
 * per row).  Rows are split into 128-row tiles, every tile of scene 0 first;
 * CTA b of `grid` owns tiles [b T / grid, (b + 1) T / grid) of the T tiles.
 * out (int32, caller-owned, out_cap words) receives, one after the other:
 *   2 (grid + 1) words: first block and first halo row of each CTA, then the totals;
 *   one word per block (the CTA's tiles, their rows, each row's blocks in order):
 *     the column's local index, (tile - first tile of the CTA) * 128 + row % 128
 *     for a row the CTA owns, else the CTA's row count + its index in the halo list;
 *   one word per halo row: scene << 26 | row, ascending within each CTA.
 * *out_len: the words written (or needed), *max_halo: the most halo rows of one
 * CTA.  INVALID_ARG for null pointers, n_scenes outside 1..8, a scene with no
 * rows or 2^26 rows or more, grid outside 1..T, or out_cap < *out_len (then
 * nothing is written but *out_len). */
PPN_API ppn_status ppn_probe_halo_tables(int n_scenes, const int64_t* const* row_ptr, const int32_t* const* col,
                                         const int64_t* n_verts, int grid, int32_t* out, int64_t out_cap,
                                         int64_t* out_len, int32_t* max_halo);

PPN_API ppn_status ppn_probe_pcg(ppn_scene* s, const double* vals, const double* b, double rel_tol,
                         int max_iter, double* x, int* info);

/* ---- Contact with analytic obstacles (the paper's frictionless IPC barrier potentials,
 * backtracking line search with intersection-based filtering, Sec. 5.1) ----
 *
 * Every free vertex x gets the potential kappa b(d(x)) for each obstacle, with
 * b(d) = -(d - dhat)^2 ln(d / dhat) for 0 < d < dhat and 0 beyond, d the distance:
 *   PLANE        d = a . (x - p), bodies on the side the unit normal a points to
 *   CYLINDER_IN  d = r - |(x - p) - (a . (x - p)) a|, bodies inside the cylinder of unit axis a
 *   SPHERE_OUT   d = |x - p| - r, bodies outside the sphere
 * A free vertex within dhat of an obstacle is one contact element of the projection
 * heuristic (key ||g_v||_inf, 3x3 Hessian clamped like the tets' in PN/PPN/PDN).
 * The line search starts at min(1, ccd_safety x the first time a vertex on
 * x + gamma dx reaches an obstacle).  The state must be feasible (d > 0) when a
 * step starts. */
typedef enum { PPN_OBST_PLANE = 0, PPN_OBST_CYLINDER_IN = 1, PPN_OBST_SPHERE_OUT = 2 } ppn_obstacle_kind;
typedef struct {
  int type;    /* ppn_obstacle_kind */
  double p[3]; /* plane point / axis point / centre [m] */
  double a[3]; /* plane unit normal / cylinder unit axis */
  double r;    /* cylinder or sphere radius [m] */
} ppn_obstacle;
#define PPN_MAX_OBSTACLES 8
/* obstacles for the next steps (copied; n = 0 removes contact); moving obstacles
 * are set before every step.  PPN_ERR_INVALID_ARG for n > PPN_MAX_OBSTACLES, an
 * unknown type, a non-unit direction or a non-positive radius. */
PPN_API ppn_status ppn_set_obstacles(ppn_scene* s, const ppn_obstacle* obs, int n);

/* ---- Serving: time-step requests over resident scenes (continuous batching) ----
 *
 * The paper has no serving layer; this is the request loop around the same
 * time step (Sec. 3 with Algorithm 1).  A server owns a CUDA stream, a worker
 * thread and its scenes, which stay resident on the device (mesh, BSR pattern,
 * state) between requests.
 *   - Admission by HBM footprint: ppn_server_add_scene admits a scene only when
 *     the device memory of all resident scenes stays within hbm_fraction of the
 *     device's memory; otherwise PPN_ERR_ADMISSION (nothing is kept).  Removing
 *     a scene frees its memory for later admissions.
 *   - A request is one time step of one scene (mode, tolerance, optional new
 *     kinematic targets).  Requests of one scene run in submission order.
 *   - Continuous batching: up to max_batch scenes step together, one launch per
 *     phase over all of them.  At every Newton-iteration boundary the finished
 *     scenes leave the batch (their results become available) and queued
 *     requests join in the free slots, so requests that arrive while others
 *     run are admitted as slots free up and their work overlaps on the device.
 *     A scene's result does not depend on the other scenes of the batch
 *     (every reduction is per scene and in a fixed order).
 * Every call returns a status; waits on the worker are bounded only by the
 * requests themselves (each time step has its own iteration caps). */
typedef struct ppn_server ppn_server;

typedef struct {
  double hbm_fraction; /* admission cap: resident scenes' device memory <= this x device memory (0.8) */
  int max_batch;       /* scenes that step together (64) */
  int precision;       /* ppn_precision of every scene of the server (PPN_PREC_MIXED) */
} ppn_server_config;

typedef struct {
  double t_submit_ms; /* times since the server was created */
  double t_start_ms;  /* the request joined the batch */
  double t_done_ms;   /* its result was available */
  int batch_max;      /* largest batch the request was part of */
} ppn_request_times;

typedef struct {
  int64_t submitted, completed, rejected_scenes;
  int resident_scenes;
  double resident_bytes, budget_bytes;
  double p50_ms, p99_ms; /* latency (done - submit) percentiles over completed requests */
  double steps_per_s;    /* completed requests / (last completion - first submission) */
} ppn_server_stats;

PPN_API ppn_server_config ppn_server_default_config(void);
PPN_API ppn_status ppn_server_create(const ppn_server_config* cfg, ppn_server** out);
/* Finishes the requests already submitted, then frees the server and its scenes. */
PPN_API void ppn_server_destroy(ppn_server* srv);
/* Same arguments as ppn_create_scene (params->precision must equal the server's);
 * scene_id receives the server's handle of the scene. */
PPN_API ppn_status ppn_server_add_scene(ppn_server* srv, const double* rest_xyz, int64_t n_verts,
                                        const int32_t* tets, int64_t n_tets, const ppn_material* mat, double dt,
                                        const int32_t* fixed, int64_t n_fixed, const ppn_params* params,
                                        int32_t* scene_id);
/* PPN_ERR_INVALID_ARG while the scene has unfinished requests. */
PPN_API ppn_status ppn_server_remove_scene(ppn_server* srv, int32_t scene_id);
/* targets: NULL (keep the scene's current kinematic targets) or n_fixed*3 positions,
 * copied before the call returns.  ticket receives the request's handle. */
PPN_API ppn_status ppn_server_submit(ppn_server* srv, int32_t scene_id, ppn_mode mode, double tol,
                                     const double* targets, int64_t* ticket);
/* wait != 0 blocks until the request is done.  *done = 1 when it is; then out_xyz
 * (n_verts*3, may be NULL), stats and times (may be NULL) are filled, the ticket
 * is released, and the request's own status is returned. */
PPN_API ppn_status ppn_server_poll(ppn_server* srv, int64_t ticket, int wait, int* done, double* out_xyz,
                                   ppn_step_stats* stats, ppn_request_times* times);
PPN_API ppn_status ppn_server_get_stats(ppn_server* srv, ppn_server_stats* out);

/* ---- PCG without per-call device allocation (the paper has no counterpart) ----
 *
 * Block-Jacobi PCG with the negative-curvature exit (the linear solve of Sec. 4.1,
 * "Linear Solvers", and Sec. 5.1) on a caller's device-resident FP32 BSR system,
 * using only a fixed scratch arena in device global memory (a file-scope
 * __device__ array sized for PPN_PCG_STATIC_MAX_ROWS block rows, about 8 MB).
 * It is for callers that must not allocate device memory per call, e.g. a
 * serving loop running under a fixed HBM budget, where cudaMalloc may fail and
 * cudaFree synchronises the device.
 *
 * All pointers except `info` are DEVICE pointers owned by the caller:
 *   row_ptr  n_rows+1 int32, non-decreasing, row_ptr[0] = 0, row_ptr[n_rows] = nnzb
 *   col      nnzb int32 block columns in [0, n_rows); every row holds its diagonal block
 *   val      9*nnzb float, component-major: entry c (row-major in the 3x3 block) of
 *            block k at val[c*nnzb + k]
 *   b        n_rows 16-byte records {b_x, b_y, b_z, ignored} (16-byte aligned)
 *   x        n_rows 16-byte records, written with the solution (16-byte aligned)
 * rel_tol: stop at ||r|| <= rel_tol ||b||; max_iter <= 0: max(1000, 3 n_rows).
 * info (host, may be NULL): [iterations, ind, precond_fail, hit_max].  A solve that
 * meets negative curvature (ind) or a diagonal block without a Cholesky factor
 * (precond_fail, then also ind) is a valid outcome and returns PPN_OK: x holds the
 * last iterate before the offending direction (zero when that is the first one, or
 * when the preconditioner failed).  Pass info to tell such a solve from a
 * converged one; with info NULL nothing distinguishes them.
 * stream: a cudaStream_t on the current device, or NULL; the call waits for it
 * before returning (a stream of another device: PPN_ERR_INVALID_ARG).
 *
 * Errors: PPN_ERR_INVALID_ARG for null pointers, n_rows > PPN_PCG_STATIC_MAX_ROWS,
 * or a malformed pattern (checked on the device before the solve: row pointers,
 * column range, exactly one diagonal block per row);
 * PPN_ERR_TIMEOUT when a grid-wide wait runs out; PPN_ERR_NONFINITE; PPN_ERR_CUDA.
 * The first call on a device (and the first after cudaDeviceReset, in the new
 * context) looks up the arena's address and the solver's occupancy; make it once at
 * start-up, before any stream capture.  The arena is shared per device: calls
 * on the same device must not overlap, and the library serialises its host
 * threads with a lock.  The barrier and status words that must start at zero
 * are cleared by every call. */
#define PPN_PCG_STATIC_MAX_ROWS 65536
PPN_API ppn_status ppn_pcg_solve_static(const int32_t* row_ptr, const int32_t* col, const float* val,
                                        int32_t n_rows, int32_t nnzb, const float* b, float* x,
                                        double rel_tol, int32_t max_iter, int32_t* info, void* stream);

#ifdef __cplusplus
}
#endif

#endif /* PPN_H */
