// Element, assembly, selection, projection and vector kernels of one Newton
// iteration (everything except the PCG solve, which lives in pcg.cu).
//
//   k_element   per tet: displacement gradient, stress, g^e (12) and the ten
//               3x3 Hessian blocks H^e_ab, a <= b (Sec. 3, Eq. newton terms)
//   k_gradient  per vertex: g_v = m_v/dt^2 (u_v - uhat_v) + sum_e g^e (FP64),
//               |g_v|_inf for the selection, ||g||_2^2 and ||g||_inf reductions
//   k_assemble  per BSR block: H_ij = sum of H^e contributions (+ dH^e of the
//               elements projected before assembly, + m_i/dt^2 I on the diagonal),
//               Dirichlet rows/columns eliminated; atomic-free via a
//               precomputed block -> (tet, a, b) map (Sec. 4.1 assembly)
//   k_select    per tet: r_e = max over corners of |g_v|_inf, selected when
//               r_e > delta or delta <= eps_delta and not yet projected
//               (Sec. 4, Algorithm 1); warp-aggregated compaction
//   k_project   per selected tet: clamped update dH^e (Sec. 3 clamping)
//   k_update    per BSR block touched by newly projected tets: H_ij += dH^e_ab,
//               the in-place incremental update of Sec. 4.1
//   k_energy    per tet and per vertex: incremental potential at u + gamma dx
//               and g^T dx, FP64 sums (line search, Sec. 5.1)
//   small vector kernels: predictor, position update, velocity, fallback direction
#include <cstdlib>

#include "common.cuh"
#include "contact.cuh"
#include "eigclamp.cuh"
#include "kernels.h"

namespace ppn {

template <typename T>
__device__ __forceinline__ void load_tetc(const T* tetc, int e, T* W, T& V, T& mu, T& lam) {
  const T* p = tetc + (size_t)e * TETC_STRIDE;
#pragma unroll
  for (int k = 0; k < 9; ++k) W[k] = p[k];
  V = p[9];
  mu = p[10];
  lam = p[11];
}
template <>
__device__ __forceinline__ void load_tetc<float>(const float* tetc, int e, float* W, float& V,
                                                 float& mu, float& lam) {
  const float4* p = reinterpret_cast<const float4*>(tetc + (size_t)e * TETC_STRIDE);
  const float4 a = __ldg(p), b = __ldg(p + 1), c = __ldg(p + 2);
  W[0] = a.x; W[1] = a.y; W[2] = a.z; W[3] = a.w;
  W[4] = b.x; W[5] = b.y; W[6] = b.z; W[7] = b.w;
  W[8] = c.x; V = c.y; mu = c.z; lam = c.w;
}

__device__ __forceinline__ void load_u(const double4* U, int v, double* out) {
  const double4 a = ld_d4(U + v);
  out[0] = a.x;
  out[1] = a.y;
  out[2] = a.z;
}

// ---------------------------------------------------------------- K1 element
template <typename T>
__global__ void __launch_bounds__(TILE) k_element(const SceneDev<T>* scenes, const TileRef* tiles,
                                                  int use_probe) {
  // each 3x3 block goes through shared memory so that a warp writes its 32 tets'
  // blocks as 36-byte runs (one warp store covers ~4 tets, not 32 records)
  __shared__ T s_blk[TILE / 32][32][9];
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const int e0 = tr.tile * TILE + wid * 32;  // the warp's first tet
  if (e0 >= S.nt) return;                    // warp-uniform
  const int e = e0 + lane;
  const bool valid = e < S.nt;
  T dN[4][3], cN[4][3], V = (T)0, mu = (T)0, lam = (T)0;
  TetState<T> st;
  if (valid) {
    const int4 t = S.tets[e];
    const double4* U = use_probe ? S.u_probe : S.u;
    double u[4][3];
    load_u(U, t.x, u[0]);
    load_u(U, t.y, u[1]);
    load_u(U, t.z, u[2]);
    load_u(U, t.w, u[3]);
    T W[9];
    load_tetc(S.tetc, e, W, V, mu, lam);
    // g^e in FP64 in both precisions: the assembled residual drives convergence and
    // selection, and near equilibrium it is a small sum of large element forces
    double Wd[9], Hd[9];
#pragma unroll
    for (int k = 0; k < 9; ++k) Wd[k] = (double)W[k];
    disp_grad(u[0], u[1], u[2], u[3], Wd, Hd);
    TetState<double> sd;
    tet_state(Hd, (double)mu, (double)lam, sd);
    double Pd[9];
    snh_pk1_disp(sd, (double)mu, (double)lam, Pd);
    double dNd[4][3];
    shape_grads(Wd, dNd);
    double* ge = S.ge + (size_t)e * GE_STRIDE;
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      double pa[3];
      matvec3(Pd, dNd[a], pa);
#pragma unroll
      for (int k = 0; k < 3; ++k) ge[3 * a + k] = (double)V * pa[k];
    }
    // Hessian blocks in the storage type
    if constexpr (sizeof(T) == sizeof(double)) {
      st = sd;
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int k = 0; k < 3; ++k) dN[a][k] = dNd[a][k];
    } else {
      T H[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) H[k] = (T)Hd[k];
      tet_state(H, mu, lam, st);
      shape_grads(W, dN);
    }
#pragma unroll
    for (int a = 0; a < 4; ++a) matvec3(st.C, dN[a], cN[a]);
  }
  const int n_here = min(32, S.nt - e0);
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = a; b < 4; ++b) {
      if (valid) {
        T blk[9];
        hess_block(st, V, mu, lam, dN[a], dN[b], cN[a], cN[b], blk);
#pragma unroll
        for (int k = 0; k < 9; ++k) s_blk[wid][lane][k] = blk[k];
      }
      __syncwarp();
      const size_t off = (size_t)9 * tri4(a, b);
      for (int j = lane; j < 9 * n_here; j += 32) {
        const int t = j / 9, k = j - 9 * t;
        S.He[(size_t)(e0 + t) * HE_STRIDE + off + k] = s_blk[wid][t][k];
      }
      __syncwarp();
    }
}

// ------------------------------------------------------------- K2 gradient
template <typename T>
__global__ void __launch_bounds__(TILE) k_gradient(const SceneDev<T>* scenes, const TileRef* tiles,
                                                   int use_probe) {
  __shared__ double sm[32];
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int v = tr.tile * TILE + threadIdx.x;
  double n2 = 0.0, ninf = 0.0, s2 = 0.0, nc = 0.0;
  if (v < S.nv) {
    double g[3] = {0.0, 0.0, 0.0};
    if (!S.fixed[v]) {
      const double4* U = use_probe ? S.u_probe : S.u;
      const double4 uv = ld_d4(U + v), uh = ld_d4(S.uhat + v);
      const double w = S.mass[v] * S.inv_dt2;
      g[0] = w * (uv.x - uh.x);
      g[1] = w * (uv.y - uh.y);
      g[2] = w * (uv.z - uh.z);
      // s: the same terms in magnitude (the rounding scale of g)
      double a[3] = {fabs(g[0]), fabs(g[1]), fabs(g[2])};
      for (int c = S.vt_ptr[v]; c < S.vt_ptr[v + 1]; ++c) {
        const int src = S.vt_src[c];
        const double* ge = S.ge + (size_t)(src >> 2) * GE_STRIDE + 3 * (src & 3);
        g[0] += ge[0];
        g[1] += ge[1];
        g[2] += ge[2];
        a[0] += fabs(ge[0]);
        a[1] += fabs(ge[1]);
        a[2] += fabs(ge[2]);
      }
      if (S.pen_k > 0.0 && S.con[v]) {  // Dirichlet penalty potential: k m / dt^2 (u - t)
        const double4 t = ld_d4(S.tgt + v);
        const double wp = S.pen_k * w;
        const double p[3] = {wp * (uv.x - t.x), wp * (uv.y - t.y), wp * (uv.z - t.z)};
        for (int k = 0; k < 3; ++k) {
          g[k] += p[k];
          a[k] += fabs(p[k]);
        }
      }
      if (S.obs->n > 0) {  // barrier potentials of the analytic obstacles
        const double4 X = ld_d4(S.X + v);
        const double x[3] = {X.x + uv.x, X.y + uv.y, X.z + uv.z};
        double gc[3], hc[9];
        bool act = false;
        vertex_contact(S, x, nullptr, gc, hc, &act);
#pragma unroll
        for (int k = 0; k < 9; ++k) S.Hc[(size_t)9 * v + k] = (T)hc[k];  // for the assembly's diagonal
        for (int k = 0; k < 3; ++k) {
          g[k] += gc[k];
          a[k] += fabs(gc[k]);
        }
        nc = act ? 1.0 : 0.0;
      }
      s2 = a[0] * a[0] + a[1] * a[1] + a[2] * a[2];
    }
    st_d4(S.g + v, make_double4(g[0], g[1], g[2], 0.0));
    const double m = fmax(fabs(g[0]), fmax(fabs(g[1]), fabs(g[2])));
    S.gmax[v] = m;
    n2 = g[0] * g[0] + g[1] * g[1] + g[2] * g[2];
    ninf = m;
  }
  const double s = block_sum<TILE>(n2, sm);
  const double ss = block_sum<TILE>(s2, sm);
  const double cs = block_sum<TILE>(nc, sm);
  const double mx = block_max<TILE>(ninf, sm);
  if (threadIdx.x == 0) {
    S.vpart[4 * tr.tile + 0] = s;
    S.vpart[4 * tr.tile + 1] = ss;
    S.vpart[4 * tr.tile + 2] = cs;
    S.vpart[4 * tr.tile + 3] = mx;
  }
  finish_reduction<TILE, 4>(S.vpart, &S.ctl->tiles_done[0], S.n_vtiles, 3, S.ctl->grad, sm);
}

// ------------------------------------------------------------- K3 assembly
// FP32 records: block t (floats 9t..9t+8 of a 16-byte-aligned record) lies within the
// three 16-byte words that start at float 9t - (t mod 4), since 9t mod 4 = t mod 4 <= 3:
// three aligned vector loads instead of nine scalar ones, then the nine values by offset
__device__ __forceinline__ void elem_block_f(const float* rec, int t, float* blk) {
  const int o = t & 3;
  const float4* p = reinterpret_cast<const float4*>(rec + 9 * t - o);
  const float4 x = __ldg(p), y = __ldg(p + 1), z = __ldg(p + 2);
  const float w[12] = {x.x, x.y, x.z, x.w, y.x, y.y, y.z, y.w, z.x, z.y, z.z, z.w};
#pragma unroll
  for (int k = 0; k < 9; ++k) blk[k] = o == 0 ? w[k] : o == 1 ? w[k + 1] : o == 2 ? w[k + 2] : w[k + 3];
}
template <typename T>
__device__ __forceinline__ void add_elem_block(const T* rec, int a, int b, T* acc) {
  if constexpr (sizeof(T) == 4) {
    float p[9];
    elem_block_f(rec, a <= b ? tri4(a, b) : tri4(b, a), p);
    if (a <= b) {
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[k] += p[k];
    } else {
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[3 * i + k] += p[3 * k + i];
    }
    return;
  }
  if (a <= b) {
    const T* p = rec + 9 * tri4(a, b);
#pragma unroll
    for (int k = 0; k < 9; ++k) acc[k] += p[k];
  } else {
    const T* p = rec + 9 * tri4(b, a);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int k = 0; k < 3; ++k) acc[3 * i + k] += p[3 * k + i];
  }
}

// A warp assembles 32 consecutive blocks from their contribution list (the
// blocks' (tet, a, b) sources, contiguous in blk_src), 32 contributions at a time:
// lane l loads contribution c0 + l and its block's place among the warp's 32 (a
// byte per contribution, built at scene creation), a segmented scan across the warp sums the
// contributions of each block in the chunk, and the last lane of each block's
// run adds the run's sum to the block's total in shared memory (chunks in
// order).  Work per warp follows the number of contributions, not the longest
// block (a diagonal block has ~24, an off-diagonal one ~4-6).  Then lane l writes
// block k0 + l, with the inertia (and contact) terms on the diagonal.
template <typename T>
__global__ void __launch_bounds__(TILE, sizeof(T) == 4 ? 6 : 4) k_assemble(const SceneDev<T>* scenes, const TileRef* tiles, int use_probe) {
  constexpr int NWA = TILE / 32;
  __shared__ T s_acc[NWA][32][9];
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int k0 = tr.tile * TILE + warp * 32;
  if (k0 >= S.nnzb) return;  // warp-uniform
  const int nk = min(32, S.nnzb - k0);
  const int it = S.it_id;
#pragma unroll
  for (int c = 0; c < 9; ++c) s_acc[warp][lane][c] = (T)0;
  const int cb = S.blk_ptr[k0], ce = S.blk_ptr[k0 + nk];
  __syncwarp();
  // the next chunk's sources are loaded one chunk ahead, so that a chunk's element
  // blocks are one dependent load away from the loop's start
  int src_n = 0, bl_n = nk;
  if (cb + lane < ce) {
    src_n = S.blk_src[cb + lane];
    bl_n = S.blk_lane[cb + lane];
  }
  for (int cbase = cb; cbase < ce; cbase += 32) {
    const int c = cbase + lane;
    const int src = src_n;
    int bl = bl_n;  // local block of contribution c (the warp's blocks start at a multiple of 32); nk: none
    if (c + 32 < ce) {
      src_n = S.blk_src[c + 32];
      bl_n = S.blk_lane[c + 32];
    } else {
      bl_n = nk;
    }
    T v[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) v[q] = (T)0;
    if (c < ce) {
      const int e = src >> 4, a = (src >> 2) & 3, b = src & 3;
      add_elem_block(S.He + (size_t)e * HE_STRIDE, a, b, v);
      if (S.proj_stamp[e] == it) add_elem_block(S.dH + (size_t)e * HE_STRIDE, a, b, v);
    }
    // inclusive sums over each run of equal bl (bl non-decreasing across lanes); a run of
    // length L needs the offsets below L, so the rounds stop at the chunk's longest run
    // (the rounds left out would add nothing: the same sums)
    const int bp = __shfl_up_sync(0xffffffffu, bl, 1);
    const unsigned heads = __ballot_sync(0xffffffffu, lane == 0 || bp != bl);
    const unsigned later = heads & ~((2u << lane) - 1u);  // heads above this lane (none for lane 31)
    const int run = (later ? __ffs(later) - 1 : 32) - lane;  // a head's run length
    const int longest = (int)__reduce_max_sync(0xffffffffu, (heads >> lane) & 1u ? (unsigned)run : 0u);
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      if (o >= longest) break;  // warp-uniform
      const int bo = __shfl_up_sync(0xffffffffu, bl, o);
#pragma unroll
      for (int q = 0; q < 9; ++q) {
        const T x = __shfl_up_sync(0xffffffffu, v[q], o);
        if (lane >= o && bo == bl) v[q] += x;
      }
    }
    const int bn = __shfl_down_sync(0xffffffffu, bl, 1);
    if (c < ce && (lane == 31 || bn != bl)) {
#pragma unroll
      for (int q = 0; q < 9; ++q) s_acc[warp][bl][q] += v[q];
    }
    __syncwarp();
  }
  if (lane >= nk) return;
  const int k = k0 + lane;
  const int i = S.blk_row[k], j = S.col[k];
  T acc[9];
  if (S.fixed[i] || S.fixed[j]) {
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = (T)0;
    if (i == j) acc[0] = acc[4] = acc[8] = (T)1;
  } else {
#pragma unroll
    for (int q = 0; q < 9; ++q) acc[q] = s_acc[warp][lane][q];
    if (i == j) {  // inertia, and the Dirichlet penalty k m / dt^2 of a constrained vertex
      const T m = (T)(S.mass[i] * S.inv_dt2 * (S.pen_k > 0.0 && S.con[i] ? 1.0 + S.pen_k : 1.0));
      acc[0] += m;
      acc[4] += m;
      acc[8] += m;
      if (S.obs->n > 0) {  // the contact element of vertex i (Hessian from k_gradient at this iterate), and
#pragma unroll             // its clamping if projected before assembly
        for (int q = 0; q < 9; ++q) acc[q] += S.Hc[(size_t)9 * i + q];
        if (S.cproj_stamp[i] == it)
#pragma unroll
          for (int q = 0; q < 9; ++q) acc[q] += S.dHc[(size_t)9 * i + q];
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) S.val[(size_t)q * S.nnzb + k] = acc[q];
}

// Off-diagonal blocks: a thread per block sums its contributions (the block's (tet, a,
// b) sources, a != b, in element order) one after another, the next source loaded one
// step ahead; a contribution is formed (He, plus dH if projected) before it is added.
// The sums run in the order of the plain per-element scatter.
template <typename T>
__device__ __forceinline__ void assemble_offdiag(const SceneDev<T>& S, int tile) {
  const int k = tile * TILE + (int)threadIdx.x;
  if (k >= S.nnzb) return;
  const int i = S.blk_row[k], j = S.col[k];
  if (i == j) return;  // (the diagonal blocks: assemble_diag)
  const int it = S.it_id;
  T acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = (T)0;
  if (!S.fixed[i] && !S.fixed[j]) {
    const int c0 = S.blk_ptr[k], c1 = S.blk_ptr[k + 1];
    int src_n = c0 < c1 ? S.blk_src[c0] : 0;
    for (int c = c0; c < c1; ++c) {
      const int src = src_n;
      if (c + 1 < c1) src_n = S.blk_src[c + 1];
      const int e = src >> 4, a = (src >> 2) & 3, b = src & 3;
      T v[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) v[q] = (T)0;
      add_elem_block(S.He + (size_t)e * HE_STRIDE, a, b, v);
      if (S.proj_stamp[e] == it) add_elem_block(S.dH + (size_t)e * HE_STRIDE, a, b, v);
#pragma unroll
      for (int q = 0; q < 9; ++q) acc[q] += v[q];
    }
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) S.val[(size_t)q * S.nnzb + k] = acc[q];
}

// Diagonal blocks: a thread per vertex i sums the blocks (a, a) of the tets incident to
// i (the vertex -> tet incidence, in its order; the next incidence loaded one step
// ahead), then adds the inertia (and contact) terms.  Each contribution is formed as in
// the off-diagonal form (He, plus dH if projected) before it is added.
template <typename T>
__device__ __forceinline__ void assemble_diag(const SceneDev<T>& S, int tile) {
  const int i = tile * TILE + (int)threadIdx.x;
  if (i >= S.nv) return;
  const int it = S.it_id;
  const int k = S.diag_idx[i];
  T acc[9];
#pragma unroll
  for (int q = 0; q < 9; ++q) acc[q] = (T)0;
  if (S.fixed[i]) {
    acc[0] = acc[4] = acc[8] = (T)1;
  } else {
    const int c0 = S.vt_ptr[i], c1 = S.vt_ptr[i + 1];
    int src_n = c0 < c1 ? S.vt_src[c0] : 0;  // the next incidence, loaded one step ahead
    for (int c = c0; c < c1; ++c) {
      const int src = src_n;
      if (c + 1 < c1) src_n = S.vt_src[c + 1];
      const int e = src >> 2, a = src & 3;
      T v[9];
#pragma unroll
      for (int q = 0; q < 9; ++q) v[q] = (T)0;
      add_elem_block(S.He + (size_t)e * HE_STRIDE, a, a, v);
      if (S.proj_stamp[e] == it) add_elem_block(S.dH + (size_t)e * HE_STRIDE, a, a, v);
#pragma unroll
      for (int q = 0; q < 9; ++q) acc[q] += v[q];
    }
    // inertia, and the Dirichlet penalty k m / dt^2 of a constrained vertex
    const T m = (T)(S.mass[i] * S.inv_dt2 * (S.pen_k > 0.0 && S.con[i] ? 1.0 + S.pen_k : 1.0));
    acc[0] += m;
    acc[4] += m;
    acc[8] += m;
    if (S.obs->n > 0) {  // the contact element of vertex i (Hessian from k_gradient at this iterate), and
#pragma unroll           // its clamping if projected before assembly
      for (int q = 0; q < 9; ++q) acc[q] += S.Hc[(size_t)9 * i + q];
      if (S.cproj_stamp[i] == it)
#pragma unroll
        for (int q = 0; q < 9; ++q) acc[q] += S.dHc[(size_t)9 * i + q];
    }
  }
#pragma unroll
  for (int q = 0; q < 9; ++q) S.val[(size_t)q * S.nnzb + k] = acc[q];
}

// K3, element-order form (the FP64 path): blocks [0, n_btiles) of the grid take
// BSR-block tiles (a thread per off-diagonal block), the rest vertex tiles (a thread per
// diagonal block).  Every block sums its contributions one after another in element
// order, the order of a plain per-element scatter, so that the FP64 matrix follows that
// reference's rounding; the warp form above is the faster FP32 path.
template <typename T>
__global__ void __launch_bounds__(TILE)
    k_assemble_seq(const SceneDev<T>* scenes, const TileRef* btiles, int n_btiles, const TileRef* vtiles) {
  const bool off = (int)blockIdx.x < n_btiles;
  const TileRef tr = off ? btiles[blockIdx.x] : vtiles[blockIdx.x - n_btiles];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  if (off)
    assemble_offdiag(S, tr.tile);
  else
    assemble_diag(S, tr.tile);
}

// ----------------------------------------------------- K6 incremental update
// dH contributions of block k from the elements selected in round rd, summed in the
// block's contribution order; the map entries and the stamps are loaded eight at a
// time so that a block's list is not one dependent load after another.  Returns
// whether any contribution matched.
template <typename T>
__device__ __forceinline__ bool round_contributions(const SceneDev<T>& S, int k, int rd, T* acc) {
#pragma unroll
  for (int c = 0; c < 9; ++c) acc[c] = (T)0;
  bool any = false;
  const int cb = S.blk_ptr[k], ce = S.blk_ptr[k + 1];
  for (int c0 = cb; c0 < ce; c0 += 8) {
    int src[8], hit[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) src[u] = c0 + u < ce ? S.blk_src[c0 + u] : -1;
#pragma unroll
    for (int u = 0; u < 8; ++u) hit[u] = src[u] >= 0 && S.round_stamp[src[u] >> 4] == rd;
#pragma unroll
    for (int u = 0; u < 8; ++u)
      if (hit[u]) {
        any = true;
        add_elem_block(S.dH + (size_t)(src[u] >> 4) * HE_STRIDE, (src[u] >> 2) & 3, src[u] & 3, acc);
      }
  }
  return any;
}

template <typename T>
__global__ void __launch_bounds__(TILE) k_update(const SceneDev<T>* scenes, const TileRef* tiles) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int k = tr.tile * TILE + threadIdx.x;
  if (k >= S.nnzb) return;
  const int i = S.blk_row[k], j = S.col[k];
  if (S.fixed[i] || S.fixed[j]) return;
  T acc[9];
  if (!round_contributions(S, k, S.round_id, acc)) return;
#pragma unroll
  for (int c = 0; c < 9; ++c) S.val[(size_t)c * S.nnzb + k] += acc[c];
}

// Touched-block form of the same update (Sec. 4.1, "Incremental Hessian updates":
// only the blocks of the newly projected elements change).  k_touch lists, once
// each, the blocks that the 16 corner pairs of the last selection's tets map to
// (a per-block mark of the selection round deduplicates them; the mark's exchange
// and the list's counter are the only atomics).  k_update_touched then sums each
// listed block's contributions of that round exactly as k_update does, in the
// block's contribution order, so both forms give the same bits.
template <typename T>
__global__ void __launch_bounds__(TILE) k_touch(const SceneDev<T>* scenes, const TileRef* tiles) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int q = tr.tile * TILE + threadIdx.x;  // (selected element, corner pair)
  bool fresh = false;
  int k = 0;
  if (q < 16 * S.ctl->n_new) {
    const int e = S.sel_list[q >> 4];
    k = S.tet_blk[(size_t)16 * e + (q & 15)];
    const int i = S.blk_row[k], j = S.col[k];
    if (!S.fixed[i] && !S.fixed[j]) fresh = atomicExch(&S.blk_mark[k], S.round_id) != S.round_id;
  }
  const unsigned mask = __ballot_sync(0xffffffffu, fresh);
  if (mask == 0u) return;
  const int lane = threadIdx.x & 31;
  int base = 0;
  if (lane == __ffs(mask) - 1) base = atomicAdd(&S.ctl->n_touched, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
  if (fresh) S.touched[base + __popc(mask & ((1u << lane) - 1u))] = k;
}

template <typename T>
__global__ void __launch_bounds__(TILE) k_update_touched(const SceneDev<T>* scenes, const TileRef* tiles) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int q = tr.tile * TILE + threadIdx.x;
  if (q >= S.ctl->n_touched) return;
  const int k = S.touched[q];
  T acc[9];
  round_contributions(S, k, S.round_id, acc);
#pragma unroll
  for (int c = 0; c < 9; ++c) S.val[(size_t)c * S.nnzb + k] += acc[c];
}

// ------------------------------------------------------------ K4 selection
// delta < 0 selects every element (PN: project all before assembly)
template <typename T>
__global__ void __launch_bounds__(TILE) k_select(const SceneDev<T>* scenes, const TileRef* tiles) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int e = tr.tile * TILE + threadIdx.x;
  bool sel = false, tie = false;
  if (e < S.nt && S.proj_stamp[e] != S.it_id) {
    if (S.delta < 0.0 || S.delta <= S.eps_delta) {
      sel = true;
    } else {
      const int4 t = S.tets[e];
      const double r = fmax(fmax(S.gmax[t.x], S.gmax[t.y]), fmax(S.gmax[t.z], S.gmax[t.w]));
      sel = r > S.delta;
      tie = fabs(r - S.delta) <= S.tie_band * S.delta;  // reported: the strict test decides
    }
  }
  const int lane = threadIdx.x & 31;
  const unsigned tmask = __ballot_sync(0xffffffffu, tie);
  if (tmask != 0u && lane == 0) atomicAdd(&S.ctl->n_ties, __popc(tmask));
  const unsigned mask = __ballot_sync(0xffffffffu, sel);
  if (mask == 0u) return;
  int base = 0;
  if (lane == __ffs(mask) - 1) base = atomicAdd(&S.ctl->n_new, __popc(mask));
  base = __shfl_sync(0xffffffffu, base, __ffs(mask) - 1);
  if (sel) {
    const int idx = base + __popc(mask & ((1u << lane) - 1u));
    S.sel_list[idx] = e;
    S.proj_stamp[e] = S.it_id;
    S.round_stamp[e] = S.round_id;
  }
}

// ------------------------------------------------------- K5 eigen + clamp
template <typename T>
__global__ void __launch_bounds__(PROJ_CTA) k_project(const SceneDev<T>* scenes, const TileRef* tiles,
                                                      int use_probe) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int idx = tr.tile * PROJ_CTA + threadIdx.x;
  if (idx >= S.ctl->n_new) return;
  const int e = S.sel_list[idx];
  const int4 t = S.tets[e];
  const double4* U = use_probe ? S.u_probe : S.u;
  double u[4][3];
  load_u(U, t.x, u[0]);
  load_u(U, t.y, u[1]);
  load_u(U, t.z, u[2]);
  load_u(U, t.w, u[3]);
  T W[9], V, mu, lam;
  load_tetc(S.tetc, e, W, V, mu, lam);
  T H[9];
  disp_grad(u[0], u[1], u[2], u[3], W, H);
  TetState<T> st;
  tet_state(H, mu, lam, st);
  T out[90];
  clamp_tet(st, W, V, mu, lam, (T)S.eig_eps, S.proj_kind == 1, out);
  T* dst = S.dH + (size_t)e * HE_STRIDE;
#pragma unroll
  for (int k = 0; k < 90; ++k) dst[k] = out[k];
}

// K5, warp form, for the few hundred to few thousand tets of a PPN selection round,
// where one thread per tet leaves the launch as long as one thread's serial Jacobi.
// Three tets per warp, nine lanes per tet (lanes 27..31 idle): lane 9 g + i holds
// row i of tet g's reduced matrix M and row i of its eigenvector matrix.  The four
// rotations of a round-robin round (disjoint pairs) go at once: the lane of each
// pair's first index forms its rotation as the one-thread form does, every lane
// rotates the four column pairs of its rows of M and of the eigenvectors, each row of
// a pair then combines with its partner row (fetched by shuffle), and the pair's 2x2
// block is set as in the one-thread form (diagonal app - t apq and aqq + t apq,
// off-diagonal 0).  Sweeps stop per tet at the one-thread form's test.  The clamped
// update, the sum over clamped eigenpairs of w q q^T plus eps/4 I per block, is
// formed by lane i for block i of the upper block triangle and entry i of block 9.
constexpr unsigned kFull = 0xffffffffu;

template <typename T>
__device__ __forceinline__ T wsel(const T* a, int idx) {  // a[idx] for a lane-varying idx, in registers
  T x = a[0];
#pragma unroll
  for (int c = 1; c < 9; ++c) x = c == idx ? a[c] : x;
  return x;
}

template <typename T, int R>
__device__ __forceinline__ void wround(T* a, T* v, int i, int base, bool done) {
  constexpr int p0 = rr_p(R, 0), q0 = rr_q(R, 0), p1 = rr_p(R, 1), q1 = rr_q(R, 1);
  constexpr int p2 = rr_p(R, 2), q2 = rr_q(R, 2), p3 = rr_p(R, 3), q3 = rr_q(R, 3);
  const int mate = rr_mate(R, i);  // (index R meets itself: it sits the round out)
  const bool first = i < mate;
  const T dii = wsel(a, i), dim = wsel(a, mate);
  const T dmm = __shfl_sync(kFull, dii, base + mate);
  // the pair's rotation, formed by its first lane (jrot_params on (i, mate))
  const bool skip = done || !first || dim == (T)0;
  const T apq = skip ? (T)1 : dim;
  const T tau = (dmm - dii) / ((T)2 * apq);
  const T at = tau < (T)0 ? -tau : tau;
  T t = at > JacobiCfg<T>::big_tau ? (T)0.5 / at : (T)1 / (at + sqrt((T)1 + at * at));
  if (tau < (T)0) t = -t;
  if (skip) t = (T)0;
  const T cs = rsqrt_t<T>((T)1 + t * t);
  const T c = skip ? (T)1 : cs, s = skip ? (T)0 : t * cs;
  // the four rotations for the column pairs, from their first lanes
  const T c0 = __shfl_sync(kFull, c, base + p0), s0 = __shfl_sync(kFull, s, base + p0);
  const T c1 = __shfl_sync(kFull, c, base + p1), s1 = __shfl_sync(kFull, s, base + p1);
  const T c2 = __shfl_sync(kFull, c, base + p2), s2 = __shfl_sync(kFull, s, base + p2);
  const T c3 = __shfl_sync(kFull, c, base + p3), s3 = __shfl_sync(kFull, s, base + p3);
  // this lane's own pair, from its first lane
  const int src = base + (first ? i : mate);
  const T tm = __shfl_sync(kFull, t, src), cm = __shfl_sync(kFull, c, src), sm = __shfl_sync(kFull, s, src);
  const T apqm = __shfl_sync(kFull, dim, src);
  const int rot = __shfl_sync(kFull, (int)!skip, src);
  auto colrot = [&](T* m, int P, int Q, T cc, T ss) {
    const T mp = m[P], mq = m[Q];
    m[P] = cc * mp - ss * mq;
    m[Q] = ss * mp + cc * mq;
  };
  colrot(a, p0, q0, c0, s0);
  colrot(a, p1, q1, c1, s1);
  colrot(a, p2, q2, c2, s2);
  colrot(a, p3, q3, c3, s3);
  colrot(v, p0, q0, c0, s0);
  colrot(v, p1, q1, c1, s1);
  colrot(v, p2, q2, c2, s2);
  colrot(v, p3, q3, c3, s3);
  T b[9];
#pragma unroll
  for (int k = 0; k < 9; ++k) b[k] = __shfl_sync(kFull, a[k], base + mate);
  const T nd = first ? dii - tm * apqm : dii + tm * apqm;
  if (rot) {
#pragma unroll
    for (int k = 0; k < 9; ++k) {
      const T r = first ? cm * a[k] - sm * b[k] : sm * b[k] + cm * a[k];
      a[k] = k == i ? nd : k == mate ? (T)0 : r;
    }
  }
}

template <typename T, int R>
struct WRounds {
  __device__ __forceinline__ static void run(T* a, T* v, int i, int base, bool done) {
    wround<T, R>(a, v, i, base, done);
    if constexpr (R < 8) WRounds<T, R + 1>::run(a, v, i, base, done);
  }
};

template <typename T>
__global__ void __launch_bounds__(PROJW_CTA) k_project_w(const SceneDev<T>* scenes, const TileRef* tiles,
                                                         int use_probe) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int lane = threadIdx.x & 31;
  const int wt = 3 * (tr.tile * (PROJW_CTA / 32) + (int)(threadIdx.x >> 5));  // the warp's first tet
  const int n = S.ctl->n_new;
  if (wt >= n) return;  // warp-uniform
  const int grp = lane < 27 ? lane / 9 : 3;
  const int i = lane < 27 ? lane - 9 * grp : 0;
  const int base = lane < 27 ? 9 * grp : 0;  // (idle lanes read tet 0's lanes; their results are dropped)
  const bool live = grp < 3 && wt + grp < n;
  const int e = live ? S.sel_list[wt + grp] : 0;
  T A[45], Sl[4][3];
  {
    const int4 tt = S.tets[e];
    const double4* U = use_probe ? S.u_probe : S.u;
    double u[4][3];
    load_u(U, tt.x, u[0]);
    load_u(U, tt.y, u[1]);
    load_u(U, tt.z, u[2]);
    load_u(U, tt.w, u[3]);
    T W[9], V, mu, lam;
    load_tetc(S.tetc, e, W, V, mu, lam);
    T H[9];
    disp_grad(u[0], u[1], u[2], u[3], W, H);
    TetState<T> st;
    tet_state(H, mu, lam, st);
    reduce9(st, W, V, mu, lam, A, Sl);
  }
  T a[9], v[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) {
    T x = A[s9(0, c)];
#pragma unroll
    for (int r = 1; r < 9; ++r) x = r == i ? A[s9(r, c)] : x;
    a[c] = live ? x : (T)0;
    v[c] = c == i ? (T)1 : (T)0;
  }
  // sums over a tet's nine lanes, in lane order (the same value on each)
  auto gsum = [&](T x) {
    T s = (T)0;
#pragma unroll
    for (int r = 0; r < 9; ++r) s += __shfl_sync(kFull, x, base + r);
    return s;
  };
  T f = (T)0, o = (T)0;
#pragma unroll
  for (int c = 0; c < 9; ++c) f += a[c] * a[c];
  const T tol2 = JacobiCfg<T>::rel_tol * JacobiCfg<T>::rel_tol * gsum(f);
  bool done = !live;
  for (int sweep = 0; sweep < JacobiCfg<T>::max_sweeps; ++sweep) {
    o = (T)0;
#pragma unroll
    for (int c = 0; c < 9; ++c) o += c == i ? (T)0 : a[c] * a[c];
    const T off2 = gsum(o);  // (every lane takes part in the shuffles, done or not)
    done = done || !(off2 > tol2);
    if (__all_sync(kFull, done)) break;
    WRounds<T, 0>::run(a, v, i, base, done);
  }
  // clamping weights (lane i: eigenvalue i), and this lane's output entries
  const T li = wsel(a, i), eps = (T)S.eig_eps;
  const bool mirror = S.proj_kind == 1;
  const T wi = li < eps ? (mirror ? (-li > eps ? -li : eps) : eps) - li : (T)0;
  const T e4 = eps * (T)0.25;
  const int ba = (i >= 4) + (i >= 7), bb = i < 4 ? i : i < 7 ? i - 3 : i - 5;  // block i = (ba, bb)
  const int r9 = i / 3, c9 = i - 3 * r9;                                          // entry i of block 9 = (3, 3)
  T acc[9], acc9 = r9 == c9 ? e4 : (T)0;
#pragma unroll
  for (int k = 0; k < 9; ++k) acc[k] = (k == 0 || k == 4 || k == 8) ? e4 : (T)0;
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const T wp = __shfl_sync(kFull, wi, base + p);
    T col[9];  // eigenvector p: column p of the eigenvector matrix, one row per lane
#pragma unroll
    for (int r = 0; r < 9; ++r) col[r] = __shfl_sync(kFull, v[p], base + r);
    if (wp != (T)0) {
      T q[4][3];
#pragma unroll
      for (int aa = 0; aa < 4; ++aa)
#pragma unroll
        for (int ii = 0; ii < 3; ++ii)
          q[aa][ii] = Sl[aa][0] * col[ii] + Sl[aa][1] * col[3 + ii] + Sl[aa][2] * col[6 + ii];
      T qa[3], qb[3];
#pragma unroll
      for (int ii = 0; ii < 3; ++ii) {
        qa[ii] = ba == 0 ? q[0][ii] : ba == 1 ? q[1][ii] : q[2][ii];
        qb[ii] = bb == 0 ? q[0][ii] : bb == 1 ? q[1][ii] : bb == 2 ? q[2][ii] : q[3][ii];
      }
#pragma unroll
      for (int ii = 0; ii < 3; ++ii)
#pragma unroll
        for (int k = 0; k < 3; ++k) acc[3 * ii + k] += wp * qa[ii] * qb[k];
      const T q3r = r9 == 0 ? q[3][0] : r9 == 1 ? q[3][1] : q[3][2];
      const T q3c = c9 == 0 ? q[3][0] : c9 == 1 ? q[3][1] : q[3][2];
      acc9 += wp * q3r * q3c;
    }
  }
  if (!live) return;
  T* dst = S.dH + (size_t)e * HE_STRIDE;
#pragma unroll
  for (int k = 0; k < 9; ++k) dst[9 * i + k] = acc[k];
  dst[81 + i] = acc9;
}

// ------------------------------------------------------ contact elements
// Selection and clamping of contact elements (one per free vertex within dhat
// of an obstacle): key ||g_v||_inf > delta (or delta <= eps_delta; delta < 0:
// every contact element), not yet projected in this Newton iteration.  The
// clamping update dHc of the vertex's 3x3 barrier Hessian is computed here.
template <typename T>
__global__ void __launch_bounds__(TILE) k_select_contact(const SceneDev<T>* scenes, const TileRef* tiles) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active || S.obs->n == 0) return;
  const int v = tr.tile * TILE + threadIdx.x;
  if (v >= S.nv || S.fixed[v] || S.cproj_stamp[v] == S.it_id) return;
  const bool all = S.delta < 0.0 || S.delta <= S.eps_delta;
  const bool tie = !all && fabs(S.gmax[v] - S.delta) <= S.tie_band * S.delta;
  if (!all && !(S.gmax[v] > S.delta) && !tie) return;
  const double4 X = ld_d4(S.X + v), u = ld_d4(S.u + v);
  const double x[3] = {X.x + u.x, X.y + u.y, X.z + u.z};
  double Hc[9];
  bool act = false;
  vertex_contact(S, x, nullptr, nullptr, Hc, &act);
  if (!act) return;
  if (tie) atomicAdd(&S.ctl->n_ties, 1);  // a contact element within the tie band (rare)
  if (!all && !(S.gmax[v] > S.delta)) return;
  T H3[9], d3[9];
#pragma unroll
  for (int c = 0; c < 9; ++c) H3[c] = (T)Hc[c];
  clamp3(H3, (T)S.eig_eps, S.proj_kind == 1, d3);
#pragma unroll
  for (int c = 0; c < 9; ++c) S.dHc[(size_t)9 * v + c] = d3[c];
  S.cproj_stamp[v] = S.it_id;
  S.cround_stamp[v] = S.round_id;
  atomicAdd(&S.ctl->n_new_c, 1);
}

// in-place update of the diagonal blocks of the contact elements selected in this round
template <typename T>
__global__ void __launch_bounds__(TILE) k_update_contact(const SceneDev<T>* scenes, const TileRef* tiles) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active || S.obs->n == 0) return;
  const int v = tr.tile * TILE + threadIdx.x;
  if (v >= S.nv || S.fixed[v] || S.cround_stamp[v] != S.round_id || S.cproj_stamp[v] != S.it_id) return;
  const size_t k = (size_t)S.diag_idx[v];
#pragma unroll
  for (int c = 0; c < 9; ++c) S.val[(size_t)c * S.nnzb + k] += S.dHc[(size_t)9 * v + c];
}

// first contact time along dx over the free vertices and obstacles, reduced as
// ctl->ccd = max 1 / gamma >= 0 (the reductions' max starts at 0; intersection-based
// filtering of the line search: gamma_ccd = 1 / ctl->ccd)
template <typename T>
__global__ void __launch_bounds__(TILE) k_ccd(const SceneDev<T>* scenes, const TileRef* tiles) {
  __shared__ double sm[32];
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int v = tr.tile * TILE + threadIdx.x;
  double inv = 0.0;
  if (v < S.nv && !S.fixed[v]) {
    const double4 X = ld_d4(S.X + v), u = ld_d4(S.u + v);
    const vec4_t<T> d = S.dx[v];
    const double x[3] = {X.x + u.x, X.y + u.y, X.z + u.z};
    const double dx[3] = {(double)d.x, (double)d.y, (double)d.z};
    for (int k = 0; k < S.obs->n; ++k) inv = fmax(inv, 1.0 / obst_ccd(S.obs->o[k], x, dx));
  }
  const double mx = block_max<TILE>(inv, sm);
  if (threadIdx.x == 0) S.vpart[4 * tr.tile] = mx;
  finish_reduction<TILE, 1>(S.vpart, &S.ctl->tiles_done[2], S.n_vtiles, 0, &S.ctl->ccd, sm);
}

// smallest distance of a free vertex to obstacles k0..k0+3, reduced as
// ctl->gap[j] = max 1 / d (+inf when some vertex is not strictly feasible)
template <typename T>
__global__ void __launch_bounds__(TILE) k_obst_gap(const SceneDev<T>* scenes, const TileRef* tiles, int k0) {
  __shared__ double sm[32];
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int v = tr.tile * TILE + threadIdx.x;
  double inv[4] = {0.0, 0.0, 0.0, 0.0};
  if (v < S.nv && !S.fixed[v]) {
    const double4 X = ld_d4(S.X + v), u = ld_d4(S.u + v);
    const double x[3] = {X.x + u.x, X.y + u.y, X.z + u.z};
    for (int j = 0; j < 4 && k0 + j < S.obs->n; ++j) {
      double d, g[3], H[9];
      const bool ok = obst_eval(S.obs->o[k0 + j], x, d, g, H);
      inv[j] = ok && d > 0.0 ? 1.0 / d : std::numeric_limits<double>::infinity();
    }
  }
  double mx[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) mx[j] = block_max<TILE>(inv[j], sm);
  if (threadIdx.x == 0)
#pragma unroll
    for (int j = 0; j < 4; ++j) S.vpart[4 * tr.tile + j] = mx[j];
  finish_reduction<TILE, 4>(S.vpart, &S.ctl->tiles_done[3], S.n_vtiles, 0, S.ctl->gap, sm);
}

// ---------------------------------------------------------- K10 energy
// tile index < n_ttiles: tet tile; otherwise vertex tile (index - n_ttiles).
// Reductions: [0] incremental potential at u + gamma dx (FP64), [1] g^T dx,
// [2] max |dx| over free vertices.
template <typename T>
__global__ void __launch_bounds__(TILE) k_energy(const SceneDev<T>* scenes, const TileRef* tiles,
                                                 int use_probe) {
  __shared__ double sm[32];
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const double4* U = use_probe ? S.u_probe : S.u;
  const double gam = S.gamma;
  double en = 0.0, dd = 0.0, dmax = 0.0;
  if (tr.tile < S.n_ttiles) {
    const int e = tr.tile * TILE + threadIdx.x;
    if (e < S.nt) {
      const int4 t = S.tets[e];
      const int vs[4] = {t.x, t.y, t.z, t.w};
      double u[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a) {
        load_u(U, vs[a], u[a]);
        if (gam != 0.0) {
          const vec4_t<T> d = S.dx[vs[a]];
          u[a][0] += gam * (double)d.x;
          u[a][1] += gam * (double)d.y;
          u[a][2] += gam * (double)d.z;
        }
      }
      T Wt[9], Vt, mut, lamt;
      load_tetc(S.tetc, e, Wt, Vt, mut, lamt);
      double W[9];
#pragma unroll
      for (int k = 0; k < 9; ++k) W[k] = (double)Wt[k];
      double H[9];
      disp_grad(u[0], u[1], u[2], u[3], W, H);
      en = (double)Vt * snh_psi_disp(H, (double)mut, (double)lamt);
      if (S.psi_out) S.psi_out[e] = en;
    }
  } else {
    const int vt = tr.tile - S.n_ttiles;
    const int v = vt * TILE + threadIdx.x;
    if (v < S.nv && !S.fixed[v]) {
      // the trial displacement u + gamma dx first, formed as k_axpy_u forms the accepted
      // update, so that the energy of an accepted trial is that of the new iterate bit for bit
      double4 uv = ld_d4(U + v);
      const double4 uh = ld_d4(S.uhat + v);
      if (!use_probe) {
        const vec4_t<T> d = S.dx[v];
        if (gam != 0.0) {
          uv.x = uv.x + gam * (double)d.x;
          uv.y = uv.y + gam * (double)d.y;
          uv.z = uv.z + gam * (double)d.z;
        }
        const double4 g = ld_d4(S.g + v);
        dd = g.x * (double)d.x + g.y * (double)d.y + g.z * (double)d.z;
        dmax = fmax(fabs((double)d.x), fmax(fabs((double)d.y), fabs((double)d.z)));
      }
      const double d0 = uv.x - uh.x, d1 = uv.y - uh.y, d2 = uv.z - uh.z;
      en = 0.5 * S.mass[v] * S.inv_dt2 * (d0 * d0 + d1 * d1 + d2 * d2);
      if (S.pen_k > 0.0 && S.con[v]) {  // Dirichlet penalty potential at u + gamma dx
        const double4 t = ld_d4(S.tgt + v);
        const double p0 = uv.x - t.x, p1 = uv.y - t.y, p2 = uv.z - t.z;
        en += 0.5 * S.pen_k * S.mass[v] * S.inv_dt2 * (p0 * p0 + p1 * p1 + p2 * p2);
      }
      if (S.obs->n > 0) {  // barrier potentials; +inf where a surface is reached
        const double4 X = ld_d4(S.X + v);
        const double x[3] = {X.x + uv.x, X.y + uv.y, X.z + uv.z};
        double Ec;
        en += vertex_contact(S, x, &Ec, nullptr, nullptr, nullptr) ? Ec : std::numeric_limits<double>::infinity();
      }
    }
  }
  const double s0 = block_sum<TILE>(en, sm);
  const double s1 = block_sum<TILE>(dd, sm);
  const double s2 = block_max<TILE>(dmax, sm);
  if (threadIdx.x == 0) {
    S.tpart[4 * tr.tile + 0] = s0;
    S.tpart[4 * tr.tile + 1] = s1;
    S.tpart[4 * tr.tile + 2] = s2;
  }
  finish_reduction<TILE, 3>(S.tpart, &S.ctl->tiles_done[1], S.n_ttiles + S.n_vtiles, 2,
                            S.ctl->energy, sm);
}

// g^T dx and max |dx| over the free vertices into ctl->energy[1], [2] (the line search's
// directional derivative when the energy at gamma = 0 is already known: the previous
// iteration's accepted trial energy, computed at the same displacement bits)
template <typename T>
__global__ void __launch_bounds__(TILE) k_dirderiv(const SceneDev<T>* scenes, const TileRef* tiles) {
  __shared__ double sm[32];
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int v = tr.tile * TILE + threadIdx.x;
  double dd = 0.0, dmax = 0.0;
  if (v < S.nv && !S.fixed[v]) {
    const vec4_t<T> d = S.dx[v];
    const double4 g = ld_d4(S.g + v);
    dd = g.x * (double)d.x + g.y * (double)d.y + g.z * (double)d.z;
    dmax = fmax(fabs((double)d.x), fmax(fabs((double)d.y), fabs((double)d.z)));
  }
  const double s0 = block_sum<TILE>(dd, sm);
  const double s1 = block_max<TILE>(dmax, sm);
  if (threadIdx.x == 0) {
    S.vpart[4 * tr.tile + 0] = s0;
    S.vpart[4 * tr.tile + 1] = s1;
  }
  finish_reduction<TILE, 2>(S.vpart, &S.ctl->tiles_done[4], S.n_vtiles, 1, S.ctl->energy + 1, sm);
}

// per-vertex |g_v|_inf of a given assembled gradient (selection probe)
template <typename T>
__global__ void k_gmax(const SceneDev<T>* scenes, const TileRef* tiles) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int v = tr.tile * TILE + threadIdx.x;
  if (v >= S.nv) return;
  const double4 g = ld_d4(S.g + v);
  S.gmax[v] = fmax(fabs(g.x), fmax(fabs(g.y), fabs(g.z)));
}

// ------------------------------------------------------- small vector kernels
// start of a step: u_n = u, uhat = u + dt v + dt^2 a_grav, u = initial guess,
// Dirichlet vertices set to their targets (targets are positions, n_fixed x 3)
template <typename T>
__global__ void k_predict(const SceneDev<T>* scenes, const TileRef* tiles, const int* fixed_list,
                          const double* targets, int n_fixed) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int v = tr.tile * TILE + threadIdx.x;
  if (v >= S.nv) return;
  const double4 u = ld_d4(S.u + v), w = ld_d4(S.vel + v);
  const double dt = S.dt, dt2 = S.dt * S.dt;
  st_d4(S.u_n + v, u);
  st_d4(S.uhat + v, make_double4(u.x + dt * w.x + dt2 * S.grav[0], u.y + dt * w.y + dt2 * S.grav[1],
                                 u.z + dt * w.z + dt2 * S.grav[2], 0.0));
  if (S.init_guess == 1 && !S.fixed[v])
    st_d4(S.u + v, make_double4(u.x + dt * w.x, u.y + dt * w.y, u.z + dt * w.z, 0.0));
}

// Dirichlet targets (positions) into u (use_probe 0), u_probe (1) or neither (2);
// with a penalty also into the per-vertex targets of the penalty potential
template <typename T>
__global__ void k_apply_targets(const SceneDev<T>* scenes, int scene, const int* fixed_list,
                                const double* targets, int n_fixed, int use_probe) {
  const SceneDev<T>& S = scenes[scene];
  const int f = blockIdx.x * blockDim.x + threadIdx.x;
  if (f >= n_fixed) return;
  const int v = fixed_list[f];
  const double4 X = ld_d4(S.X + v);
  const double4 t = make_double4(targets[3 * f] - X.x, targets[3 * f + 1] - X.y, targets[3 * f + 2] - X.z, 0.0);
  if (use_probe < 2) st_d4((use_probe ? S.u_probe : S.u) + v, t);
  if (S.pen_k > 0.0) st_d4(S.tgt + v, t);  // the penalty's target
}

// u += gamma dx on free vertices
template <typename T>
__global__ void k_axpy_u(const SceneDev<T>* scenes, const TileRef* tiles) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int v = tr.tile * TILE + threadIdx.x;
  if (v >= S.nv || S.fixed[v]) return;
  const double gam = S.gamma;
  const vec4_t<T> d = S.dx[v];
  const double4 u = ld_d4(S.u + v);
  st_d4(S.u + v, make_double4(u.x + gam * (double)d.x, u.y + gam * (double)d.y, u.z + gam * (double)d.z, 0.0));
}

template <typename T>
__global__ void k_velocity(const SceneDev<T>* scenes, const TileRef* tiles) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int v = tr.tile * TILE + threadIdx.x;
  if (v >= S.nv) return;
  const double4 u = ld_d4(S.u + v), un = ld_d4(S.u_n + v);
  const double idt = 1.0 / S.dt;
  st_d4(S.vel + v, make_double4((u.x - un.x) * idt, (u.y - un.y) * idt, (u.z - un.z) * idt, 0.0));
}

// dx = -P^-1 g (kind 2, P = block-Jacobi inverse from the last PCG setup) or
// dx = -(dt^2 / m) g (kind 3)
template <typename T>
__global__ void k_fallback_dir(const SceneDev<T>* scenes, const TileRef* tiles, int kind) {
  const TileRef tr = tiles[blockIdx.x];
  const SceneDev<T>& S = scenes[tr.scene];
  if (!S.active) return;
  const int v = tr.tile * TILE + threadIdx.x;
  if (v >= S.nv) return;
  const double4 g = ld_d4(S.g + v);
  vec4_t<T> d;
  d.w = (T)0;
  if (S.fixed[v]) {
    d.x = d.y = d.z = (T)0;
  } else if (kind == 2) {
    const T* P = S.Pinv + (size_t)9 * v;
    const T g0 = (T)g.x, g1 = (T)g.y, g2 = (T)g.z;
    d.x = -(P[0] * g0 + P[1] * g1 + P[2] * g2);
    d.y = -(P[3] * g0 + P[4] * g1 + P[5] * g2);
    d.z = -(P[6] * g0 + P[7] * g1 + P[8] * g2);
  } else {
    const double s = -1.0 / (S.mass[v] * S.inv_dt2);
    d.x = (T)(s * g.x);
    d.y = (T)(s * g.y);
    d.z = (T)(s * g.z);
  }
  S.dx[v] = d;
}

// ---------------------------------------------------------------- launchers
template <typename T>
void launch_select_contact(const SceneDev<T>* s, const TileRef* t, int n, cudaStream_t st) {
  if (n) k_select_contact<T><<<n, TILE, 0, st>>>(s, t);
}
template <typename T>
void launch_update_contact(const SceneDev<T>* s, const TileRef* t, int n, cudaStream_t st) {
  if (n) k_update_contact<T><<<n, TILE, 0, st>>>(s, t);
}
template <typename T>
void launch_ccd(const SceneDev<T>* s, const TileRef* t, int n, cudaStream_t st) {
  if (n) k_ccd<T><<<n, TILE, 0, st>>>(s, t);
}
template <typename T>
void launch_obst_gap(const SceneDev<T>* s, const TileRef* t, int n, int k0, cudaStream_t st) {
  if (n) k_obst_gap<T><<<n, TILE, 0, st>>>(s, t, k0);
}
template <typename T>
void launch_element(const SceneDev<T>* s, const TileRef* t, int n, int probe, cudaStream_t st) {
  if (n) k_element<T><<<n, TILE, 0, st>>>(s, t, probe);
}
template <typename T>
void launch_gradient(const SceneDev<T>* s, const TileRef* t, int n, int probe, cudaStream_t st) {
  if (n) k_gradient<T><<<n, TILE, 0, st>>>(s, t, probe);
}
template <typename T>
void launch_assemble(const SceneDev<T>* s, const TileRef* bt, int nb, const TileRef* vt, int nv, cudaStream_t st,
                     int use_probe) {
  if constexpr (sizeof(T) == 8) {
    if (nb + nv) k_assemble_seq<T><<<nb + nv, TILE, 0, st>>>(s, bt, nb, vt);
  } else {
    if (nb) k_assemble<T><<<nb, TILE, 0, st>>>(s, bt, use_probe);
  }
}
template <typename T>
void launch_update(const SceneDev<T>* s, const TileRef* t, int n, cudaStream_t st) {
  if (n) k_update<T><<<n, TILE, 0, st>>>(s, t);
}
template <typename T>
void launch_update_touched(const SceneDev<T>* s, const TileRef* t, int n, cudaStream_t st) {
  if (n) {
    k_touch<T><<<n, TILE, 0, st>>>(s, t);
    k_update_touched<T><<<n, TILE, 0, st>>>(s, t);
  }
}
template <typename T>
void launch_select(const SceneDev<T>* s, const TileRef* t, int n, cudaStream_t st) {
  if (n) k_select<T><<<n, TILE, 0, st>>>(s, t);
}
bool project_warp_form(bool selection_round) {
  if (std::getenv("PPN_PROJECT_THREAD")) return false;
  if (std::getenv("PPN_PROJECT_WARP")) return true;
  return selection_round;
}
template <typename T>
void launch_project(const SceneDev<T>* s, const TileRef* t, int n, int probe, cudaStream_t st, int warp) {
  if (n && warp) k_project_w<T><<<n, PROJW_CTA, 0, st>>>(s, t, probe);
  else if (n) k_project<T><<<n, PROJ_CTA, 0, st>>>(s, t, probe);
}
template <typename T>
void launch_energy(const SceneDev<T>* s, const TileRef* t, int n, int probe, cudaStream_t st) {
  if (n) k_energy<T><<<n, TILE, 0, st>>>(s, t, probe);
}
template <typename T>
void launch_dirderiv(const SceneDev<T>* s, const TileRef* t, int n, cudaStream_t st) {
  if (n) k_dirderiv<T><<<n, TILE, 0, st>>>(s, t);
}
template <typename T>
void launch_predict(const SceneDev<T>* s, const TileRef* t, int n, cudaStream_t st) {
  if (n) k_predict<T><<<n, TILE, 0, st>>>(s, t, nullptr, nullptr, 0);
}
template <typename T>
void launch_apply_targets(const SceneDev<T>* s, int scene, const int* fl, const double* tg, int nf,
                          int probe, cudaStream_t st) {
  if (nf) k_apply_targets<T><<<(nf + 255) / 256, 256, 0, st>>>(s, scene, fl, tg, nf, probe);
}
template <typename T>
void launch_gmax(const SceneDev<T>* s, const TileRef* t, int n, cudaStream_t st) {
  if (n) k_gmax<T><<<n, TILE, 0, st>>>(s, t);
}
template <typename T>
void launch_axpy_u(const SceneDev<T>* s, const TileRef* t, int n, cudaStream_t st) {
  if (n) k_axpy_u<T><<<n, TILE, 0, st>>>(s, t);
}
template <typename T>
void launch_velocity(const SceneDev<T>* s, const TileRef* t, int n, cudaStream_t st) {
  if (n) k_velocity<T><<<n, TILE, 0, st>>>(s, t);
}
template <typename T>
void launch_fallback(const SceneDev<T>* s, const TileRef* t, int n, int kind, cudaStream_t st) {
  if (n) k_fallback_dir<T><<<n, TILE, 0, st>>>(s, t, kind);
}

#define PPN_INST(T)                                                                            \
  template void launch_element<T>(const SceneDev<T>*, const TileRef*, int, int, cudaStream_t); \
  template void launch_gradient<T>(const SceneDev<T>*, const TileRef*, int, int, cudaStream_t); \
  template void launch_assemble<T>(const SceneDev<T>*, const TileRef*, int, const TileRef*, int, cudaStream_t, int); \
  template void launch_update<T>(const SceneDev<T>*, const TileRef*, int, cudaStream_t);       \
  template void launch_update_touched<T>(const SceneDev<T>*, const TileRef*, int, cudaStream_t); \
  template void launch_select<T>(const SceneDev<T>*, const TileRef*, int, cudaStream_t);       \
  template void launch_project<T>(const SceneDev<T>*, const TileRef*, int, int, cudaStream_t, int); \
  template void launch_energy<T>(const SceneDev<T>*, const TileRef*, int, int, cudaStream_t);  \
  template void launch_predict<T>(const SceneDev<T>*, const TileRef*, int, cudaStream_t); \
  template void launch_dirderiv<T>(const SceneDev<T>*, const TileRef*, int, cudaStream_t); \
  template void launch_select_contact<T>(const SceneDev<T>*, const TileRef*, int, cudaStream_t); \
  template void launch_update_contact<T>(const SceneDev<T>*, const TileRef*, int, cudaStream_t); \
  template void launch_ccd<T>(const SceneDev<T>*, const TileRef*, int, cudaStream_t); \
  template void launch_obst_gap<T>(const SceneDev<T>*, const TileRef*, int, int, cudaStream_t); \
  template void launch_apply_targets<T>(const SceneDev<T>*, int, const int*, const double*, int, \
                                        int, cudaStream_t);                                    \
  template void launch_axpy_u<T>(const SceneDev<T>*, const TileRef*, int, cudaStream_t);       \
  template void launch_gmax<T>(const SceneDev<T>*, const TileRef*, int, cudaStream_t);         \
  template void launch_velocity<T>(const SceneDev<T>*, const TileRef*, int, cudaStream_t);     \
  template void launch_fallback<T>(const SceneDev<T>*, const TileRef*, int, int, cudaStream_t);

PPN_INST(float)
PPN_INST(double)

}  // namespace ppn
