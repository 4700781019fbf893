// Device-side data layout shared by every kernel of the library.
//
// A launch covers one or more scenes.  Each scene is described by a SceneDev
// record in device memory; work is cut into fixed-size tiles of one scene
// (TILE tets or vertices, PCG_TILE matrix rows) and a launch gets a table of
// TileRef entries, one CTA (or one PCG work unit) per tile.  Reductions write
// one partial per tile and are summed per scene in tile order, so a scene's
// arithmetic is the same whether it runs alone or inside a batch.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "tetmath.cuh"

namespace ppn {

constexpr int TILE = 256;      // tets or vertices per element/vertex tile (= CTA size)
constexpr int PCG_TILE = 128;  // BSR rows per PCG reduction tile
constexpr int HE_STRIDE = 96;  // values per element Hessian record (10 blocks x 9, padded)
constexpr int GE_STRIDE = 12;  // values per element gradient record
constexpr int TETC_STRIDE = 12;  // Dm^-1 (9), V, mu, lam_s

template <typename T> struct Vec4;
template <> struct Vec4<float> { using type = float4; };
template <> struct Vec4<double> { using type = double4; };
template <typename T> using vec4_t = typename Vec4<T>::type;

// analytic obstacle of the contact model (contact.cuh)
constexpr int OBST_PLANE = 0, OBST_CYLINDER_IN = 1, OBST_SPHERE_OUT = 2;
constexpr int MAX_OBST = 8;
struct ObstDev {
  int type, pad;
  double p[3];  // plane point / axis point / centre
  double a[3];  // plane unit normal / cylinder unit axis
  double r;     // radius
};
struct ObstSet {  // a scene's obstacles, in device memory (updated between steps)
  int n, pad;
  ObstDev o[MAX_OBST];
};

// Per-scene control block: written by kernels, copied to the host at sync points.
struct Ctl {
  double grad[4];        // ||g||_2^2, ||s||_2^2 (residual scale), contact elements, ||g||_inf
  double ccd;            // 1 / (first contact time along dx), from the contact-time kernel
  double gap[4];         // 1 / (smallest free-vertex distance) to obstacles k0..k0+3 (inf: not feasible)
  double energy[3];      // incremental potential, g^T dx, max |dx| over free vertices
  double pcg_rr0, pcg_rr, pcg_rz, pcg_dq, pcg_alpha, pcg_beta;
  int n_new;             // elements selected by the last selection
  int n_new_c;           // contact elements selected by the last selection
  int n_ties;            // selection ties of the last selection (|r_e - delta| <= tie_band delta)
  int n_touched;         // BSR blocks touched by the elements of the last selection (incremental update)
  int pcg_iters;         // CG updates performed (x = sum of alpha d)
  int pcg_ind;           // negative curvature or a non-SPD diagonal block
  int pcg_precond_fail;
  int pcg_hit_max;
  int pcg_done;
  int error;             // bit flags, see kErr*
  int pad0;
  unsigned tiles_done[5];  // last-tile counters of the reductions (gradient, energy, ccd, gap, g^T dx)
};

constexpr int kErrTimeout = 1;
constexpr int kErrNonFinite = 2;

template <typename T>
struct SceneDev {
  // sizes
  int nv, nt, nnzb, nmap;
  int n_vtiles, n_ttiles, n_ptiles;  // vertex, tet and PCG-row tiles
  // constant geometry and topology
  const int4* tets;
  const T* tetc;           // nt x TETC_STRIDE
  const double* mass;      // nv
  const uint8_t* fixed;    // nv
  const double4* X;        // nv rest positions
  const int* vt_ptr;       // nv+1 vertex -> incident (tet << 2 | corner)
  const int* vt_src;
  const int* row_ptr;      // nv+1 BSR rows
  const int* col;          // nnzb
  const int* blk_row;      // nnzb
  const int* blk_ptr;      // nnzb+1 block -> contributions (tet << 4 | a << 2 | b)
  const int* blk_src;
  const unsigned char* blk_lane;  // nmap: the block of each contribution, modulo 32 (its lane in k_assemble)
  const int* diag_idx;     // nv
  const int* tet_blk;      // nt x 16: BSR block of each (a, b) corner pair of a tet
  // state
  double4* u;              // displacement x - X
  double4* u_n;
  double4* vel;
  double4* uhat;           // xhat - X
  double4* u_probe;        // scratch displacement for probes
  // per-iteration
  double* ge;              // nt x GE_STRIDE element gradients (FP64 in both precisions)
  T* He;                   // nt x HE_STRIDE
  T* dH;                   // nt x HE_STRIDE, clamping updates
  double4* g;              // assembled gradient
  double* gmax;            // per-vertex |g_v|_inf
  T* val;                  // BSR values, component-major: val[c * nnzb + k]
  int* proj_stamp;         // Newton-iteration id at which the element was projected
  int* round_stamp;        // selection-round id at which it was projected
  int* sel_list;           // compacted newly selected elements
  int* blk_mark;           // nnzb: selection round that last listed the block as touched
  int* touched;            // nnzb: blocks touched by the last selection (n_touched of them)
  // PCG vectors (nv each) and block-Jacobi inverse (nv x 9)
  vec4_t<T>* dx;
  vec4_t<T>* r;
  vec4_t<T>* z;
  vec4_t<T>* q;
  vec4_t<T>* d0;
  vec4_t<T>* d1;
  T* Pinv;
  // reduction scratch: partials[tile * 4 + k]
  double* vpart;           // vertex tiles
  double* tpart;           // tet tiles
  double* ppart;           // PCG tiles
  unsigned long long* pword;  // PCG tile partials as stamped words, [4][n_ptiles][<= 2]
  T* zrec;                    // FP32 path: [2][nv] 32-byte records {z, 0, d_prev, 0} of the resident PCG
  double* psi_out;         // optional per-element energies (probes)
  Ctl* ctl;
  // scalars of the current phase
  double dt, inv_dt2;
  double grav[3];
  double delta, eps_delta, eig_eps;
  double tie_band;         // relative half-width of the tie band around delta (counted, not selected)
  double gamma;
  double pcg_tol2;
  int pcg_max_iter;
  int it_id, round_id;
  int mode;
  int proj_kind;           // ppn_projection: 0 clamp, 1 mirror
  int init_guess;          // 0: x_n ; 1: x_n + dt v_n
  // contact against analytic obstacles
  const ObstSet* obs;       // device: the scene's obstacles (obs->n = 0: no contact)
  double kappa, dhat;
  int* cproj_stamp;        // nv: Newton-iteration id at which the contact element was projected
  int* cround_stamp;       // nv: selection round of that projection
  T* dHc;                  // nv x 9: clamping update of the contact element
  T* Hc;                   // nv x 9: Hessian of the vertex's contact potential at the iterate of the last gradient
  // Dirichlet by penalty (pen_k > 0): constrained vertices are free and carry pen_k m / (2 dt^2) |u - t|^2
  double pen_k;
  const uint8_t* con;      // nv: 1 for a constrained vertex
  double4* tgt;            // nv: its target displacement
  int active;              // the scene takes part in the current launch
};

struct TileRef {
  int scene;
  int tile;
};

// Spacing, in 64-bit words, of the stamped tile partials of the single-reduction PCG.
// Every CTA polls every tile's word once per CG iteration; packed 16 to a 128-byte L2
// line, the words of a few hundred tiles sit in a few dozen lines that all 152 SMs poll
// at once, and the requests queue at those lines' L2 slices.  One word per line spreads
// them over the slices (a 250-tile reduction fell from 4.2 to 1.4 us per iteration in
// a same-box A/B); past a few hundred tiles the extra lines cost more than the queueing,
// and two words per 16 bytes measured best (2000 tiles).  The partials' array holds
// 8 x n_ptiles x pword_stride(n_ptiles) words.
__host__ __device__ inline int pword_stride(int n_ptiles) { return n_ptiles <= 512 ? 16 : 2; }

// ---- small helpers ----
__device__ __forceinline__ double4 ld_d4(const double4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  double2 a = q[0], b = q[1];
  return make_double4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_d4(double4* p, double4 v) {
  double2* q = reinterpret_cast<double2*>(p);
  q[0] = make_double2(v.x, v.y);
  q[1] = make_double2(v.z, v.w);
}

// fixed-order block reduction of one double per thread (blockDim.x == TILE);
// result valid in thread 0
template <int NT>
__device__ __forceinline__ double block_sum(double v, double* sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < NT / 32) ? sm[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  }
  return s;
}
template <int NT>
__device__ __forceinline__ double block_max(double v, double* sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_down_sync(0xffffffffu, v, o));
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  __syncthreads();
  if (l == 0) sm[w] = v;
  __syncthreads();
  double s = 0.0;
  if (threadIdx.x < 32) {
    s = (threadIdx.x < NT / 32) ? sm[threadIdx.x] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s = fmax(s, __shfl_down_sync(0xffffffffu, s, o));
  }
  return s;
}

// Last-tile finish of a per-scene reduction: every tile has written K partials
// to part[tile * 4 + k]; the CTA that completes the count sums them in tile
// order (sum for k < n_sum, max for the rest) and writes out[0..K).
template <int NT, int K>
__device__ __forceinline__ void finish_reduction(double* part, unsigned* counter, int n_tiles,
                                                 int n_sum, double* out, double* sm) {
  __shared__ int is_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    const unsigned done = atomicAdd(counter, 1u);
    is_last = (done == (unsigned)(n_tiles - 1));
  }
  __syncthreads();
  if (!is_last) return;
  __threadfence();
#pragma unroll
  for (int k = 0; k < K; ++k) {
    // thread t sums tiles t, t + NT, ... in order; then a fixed tree
    double acc = 0.0;
    for (int t = threadIdx.x; t < n_tiles; t += NT) {
      const double v = __ldcg(part + 4 * t + k);
      acc = (k < n_sum) ? acc + v : fmax(acc, v);
    }
    const double tot = (k < n_sum) ? block_sum<NT>(acc, sm) : block_max<NT>(acc, sm);
    if (threadIdx.x == 0) out[k] = tot;
  }
  if (threadIdx.x == 0) *counter = 0u;
}

}  // namespace ppn
