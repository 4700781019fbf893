// Single-reduction block-Jacobi PCG (the linear solve of Algorithm 1; Sec. 4.1
// "Linear Solvers", Sec. 5.1) for the FP32 path: one grid-wide reduction per
// iteration, instead of the two of the textbook recurrences.
//
// Method.  The recurrences of Chronopoulos & Gear (1989) for preconditioned
// CG.  With u = M r, w = A u, s = A p, iteration i (i >= 1) computes
//   x += alpha p, r -= alpha s, u = M r, w = A u           (local, then SpMV)
//   gamma = r.u, delta = w.u, rho = r.r                     (one reduction)
//   beta = gamma / gamma_prev, d = delta - beta gamma / alpha_prev  (= p^T A p)
//   alpha = gamma / d, p = u + beta p, s = w + beta s.
// In exact arithmetic these are the iterates of the standard kernels, with
// the same stopping test on ||r|| / ||r0|| checked after each update, d equal
// to the curvature p^T A p of the new direction (d <= 0: stop with the iterate
// before it) and the same failed-diagonal-block exit.  Only s is carried by a
// recurrence (w is recomputed by the SpMV every iteration), which keeps the
// FP32 iteration counts and attained residuals those of the standard kernel.
//
// Data.  Four layouts.  SR_RES and SR_STREAM keep each CTA's rows'
// block-Jacobi inverse and vectors x, r, u, w, p, s in shared memory; SR_RES
// also keeps the rows' BSR blocks there, SR_STREAM streams them from global
// memory (L2 / HBM) every iteration through the read-only path.  SR_GLOBAL,
// for rows that do not fit, keeps the vectors in the scene's global PCG arrays
// as well (x in dx, r in z, w in q, p in d0, s in d1, the inverse in Pinv),
// each row touched only by its own CTA.  In these three layouts only u crosses
// CTAs, through a global array.  SR_HALO keeps what SR_RES keeps and
// replicates the CTA's halo (the rows of other CTAs that columns of its rows
// refer to; tables from build_halo_tables): for each halo row it holds r, s
// and the block-Jacobi inverse and repeats the owner's update of them, so u of
// the halo rows is formed in place and the SpMV reads shared memory only.
// What crosses CTAs is then w of the halo rows, which the update needs.
//
// Synchronisation.  The reduction's tile partials go out as stamped words
// after the SpMV, into one of two parity buffers, and every CTA sums them in
// tile order.  Each CTA raises a progress flag with the iteration's stamp as
// it starts an iteration.  Once a scene of the launch has finished, so that a
// CTA may have no live tile left to post, the reduction also waits for every
// CTA's flag.  Either way a buffer is overwritten two iterations later, after
// every CTA has finished reading it.
//   SR_RES, SR_STREAM, SR_GLOBAL: the progress flag also publishes the CTA's
// u (released by a fence); before its SpMV a CTA waits only for the flags of
// the CTAs that own the columns of its rows (a contiguous CTA range found at
// set-up).  One u array suffices: a CTA overwrites it only after it has seen
// every CTA's partials of the previous iteration, which each CTA posts after
// finishing the SpMV that read the old values.
//   SR_HALO: the SpMV stores w of each row as three stamped 64-bit words (the
// partials' format) in one of two parity buffers; while some warps wait for
// the reduction's words, the others read the halo rows' w words, each valid
// once it carries the iteration's stamp.  A buffer is overwritten two
// iterations later, after every CTA has raised the progress flag that follows
// its reads.  This leaves one synchronisation per iteration, the reduction.
//
// All waits are bounded.  Every layout evaluates the same expressions in the
// same order, through the explicit fused multiply-adds of the helpers below:
// all four give the same bits, and a replicated halo row the bits of its
// owner.
#include "pcg_common.cuh"

namespace ppn {

using namespace pcgdev;

namespace {

constexpr int NTP = 512;  // threads per CTA
constexpr int NQ = 4;     // reduction slots: gamma, delta, rho, failed diagonal blocks
constexpr int SP_GP = 2;  // lanes per BSR row in the SpMV
static_assert(SP_GP == 2, "the resident blocks' slots pair the two lanes of a row");

// SpMV lanes: a warp works on 32 / SP_GP consecutive rows; its lanes 0..15 take the
// first lane of each row, lanes 16..31 the second.  An 8-lane phase of a 16-byte
// gather then reads u of 8 consecutive rows at the same column offset (128 contiguous
// bytes, no bank conflict), where interleaving the two lanes of a row read two
// overlapping runs.  The per-row sum (lane 0 + lane 1) and the warp's fixed tree over
// its rows pair the same values in the same order either way.
__device__ __forceinline__ int spmv_row(int tid) { return (tid >> 5) * (32 / SP_GP) + (tid & (32 / SP_GP - 1)); }
__device__ __forceinline__ int spmv_lane(int tid) { return (tid & 31) / (32 / SP_GP); }

// Resident blocks by slot.  The 16 rows of a warp's SpMV group (items 16 g .. 16 g + 15)
// take their blocks in steps: step j holds block 2 j + h of row r in lane 16 h + r, the
// lane that multiplies it, so that every shared-memory load of the SpMV (a column, one of
// a block's nine values) reads 32 consecutive words, free of bank conflicts.  A group
// has ceil(longest row / 2) steps; the slots past a shorter row's end stay unused.  Slot
// q = 32 (lgb[g] + j) + lane; value c of the block in slot q is at lval[288 (q / 32) + 32 c + q % 32].
__device__ __forceinline__ int blk_slot(const int* lgb, int item, int k) {
  return (lgb[item >> 4] + (k >> 1)) * 32 + 16 * (k & 1) + (item & 15);
}
__device__ __forceinline__ int slot_val(int q, int c) { return (q >> 5) * 288 + 32 * c + (q & 31); }

struct SrLayout {
  float* lws;    // [(ni / PCG_TILE + 1) * 16 * NQ] partial sums per 16-row group (8 per tile)
  TileRef* ltt;  // [ni / PCG_TILE + 1] the CTA's tiles
  int* ltc;      // [ni / PCG_TILE + 1] groups of each tile done in the current SpMV
  int* lrp;      // SR_RES, SR_HALO: [ni + 1] local row pointers (blocks in CTA order)
  int* lgb;      // SR_RES, SR_HALO: [ni / 16 + 1] first slot step of each 16-row group
  int* lcol;     // SR_RES: [nb] columns; SR_HALO: [nb] local columns (own item, or ni + halo index); by slot
  float* lval;   // SR_RES, SR_HALO: [nb * 9] by slot step: nine runs of 32 values
  float* lP;     // SR_RES, SR_STREAM: [ni * 6] inverse (00 01 02 11 12 22 of the symmetric block)
  float *lx, *lr, *lu, *lw, *lp, *ls;  // SR_RES, SR_STREAM: [ni * 3] each (SR_HALO: in registers)
  float4* lu4;   // SR_HALO: [ni + nh] u of the own rows, then of the halo rows (w while it arrives)
  float *hr, *hs, *hP;  // SR_HALO: [nh * 3], [nh * 3], [nh * 6] r, s and inverse of the halo rows
  int* href;     // SR_HALO: [nh] halo rows (slot << HALO_ROW_BITS | row)
};

__host__ __device__ inline size_t up16(size_t b) { return (b + 15) & ~size_t(15); }

// the layout's pieces in carving order (nullptr base: sizes only)
__host__ __device__ inline size_t carve_sr(char* base, int ni, int nb, int nh, int mode, SrLayout* L) {
  const int ntl = ni / PCG_TILE + 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += up16(bytes);
    return p;
  };
  SrLayout l{};
  l.lws = (float*)take(sizeof(float) * ntl * 16 * NQ);
  l.ltc = (int*)take(sizeof(int) * ntl);
  l.ltt = (TileRef*)take(sizeof(TileRef) * ntl);
  if (mode == SR_RES || mode == SR_HALO) {
    l.lrp = (int*)take(sizeof(int) * (ni + 1));
    l.lgb = (int*)take(sizeof(int) * (ni / 16 + 1));
    l.lcol = (int*)take(sizeof(int) * nb);
    l.lval = (float*)take(sizeof(float) * 9 * nb);
  }
  if (mode == SR_RES || mode == SR_STREAM) {
    l.lP = (float*)take(sizeof(float) * 6 * ni);
    float** v[6] = {&l.lx, &l.lr, &l.lu, &l.lw, &l.lp, &l.ls};
    for (float** q : v) *q = (float*)take(sizeof(float) * 3 * ni);
  }
  if (mode == SR_HALO) {
    l.lu4 = (float4*)take(sizeof(float4) * (ni + nh));
    l.hr = (float*)take(sizeof(float) * 3 * nh);
    l.hs = (float*)take(sizeof(float) * 3 * nh);
    l.hP = (float*)take(sizeof(float) * 6 * nh);
    l.href = (int*)take(sizeof(int) * nh);
  }
  if (L) *L = l;
  return off;
}

// ---- the arithmetic every layout shares (explicit rounding, so that all
// layouts, and a halo row and its owner, give the same bits)
// a BSR block times v, accumulated: ax += a[0:3].v, ay += a[3:6].v, az += a[6:9].v
__device__ __forceinline__ void blk_mv(const float* a, float vx, float vy, float vz, float& ax, float& ay,
                                       float& az) {
  ax = __fmaf_rn(a[2], vz, __fmaf_rn(a[1], vy, __fmaf_rn(a[0], vx, ax)));
  ay = __fmaf_rn(a[5], vz, __fmaf_rn(a[4], vy, __fmaf_rn(a[3], vx, ay)));
  az = __fmaf_rn(a[8], vz, __fmaf_rn(a[7], vy, __fmaf_rn(a[6], vx, az)));
}
__device__ __forceinline__ float dot3(float a0, float a1, float a2, float b0, float b1, float b2) {
  return __fmaf_rn(a2, b2, __fmaf_rn(a1, b1, __fmul_rn(a0, b0)));
}
// u = P r, P symmetric, q = its entries 00 01 02 11 12 22
__device__ __forceinline__ void prec6(const float* q, const float* r, float* u) {
  u[0] = dot3(q[0], q[1], q[2], r[0], r[1], r[2]);
  u[1] = dot3(q[1], q[3], q[4], r[0], r[1], r[2]);
  u[2] = dot3(q[2], q[4], q[5], r[0], r[1], r[2]);
}
__device__ __forceinline__ void sym6(const float* P, float* q) {
  q[0] = P[0], q[1] = P[1], q[2] = P[2], q[3] = P[4], q[4] = P[5], q[5] = P[8];
}
// s = w + beta s, r -= alpha s (one component): the part a halo row repeats
__device__ __forceinline__ void upd_sr(float a, float b, float w, float& sv, float& r) {
  sv = __fmaf_rn(b, sv, w);
  r = __fmaf_rn(-a, sv, r);
}
// p = u + beta p, x += alpha p (one component)
__device__ __forceinline__ void upd_px(float a, float b, float u, float& p, float& x) {
  p = __fmaf_rn(b, p, u);
  x = __fmaf_rn(a, p, x);
}
__device__ __forceinline__ void st_relaxed_v2_u64(unsigned long long* p, unsigned long long a, unsigned long long b) {
  asm volatile("st.relaxed.gpu.global.v2.u64 [%0], {%1,%2};" ::"l"(p), "l"(a), "l"(b) : "memory");
}
__device__ __forceinline__ void ld_relaxed_v2_u64(const unsigned long long* p, unsigned long long& a,
                                                  unsigned long long& b) {
  asm volatile("ld.relaxed.gpu.global.v2.u64 {%0,%1}, [%2];" : "=l"(a), "=l"(b) : "l"(p) : "memory");
}

// u of row i: the first four floats of the row's 32-byte record in zrec
__device__ __forceinline__ float* u_ptr(float* zrec, int i) { return zrec + (size_t)i * 8; }
__device__ __forceinline__ void st_f4(float* p, float x, float y, float z) {
  asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(x), "f"(y), "f"(z), "f"(0.0f) : "memory");
}
__device__ __forceinline__ float4 ld_f4_cg(const float* p) {
  float4 v;
  asm volatile("ld.global.cg.v4.f32 {%0,%1,%2,%3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "l"(p));
  return v;
}

// The streamed BSR blocks are read once per SpMV and would evict the vectors
// from L2; they are loaded with an evict-first L2 policy so that the vectors
// (and u, gathered by every CTA) stay resident.
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
  return p;
}
// the same loads at normal L2 priority: a matrix smaller than L2 can stay resident across
// iterations (a batch of small scenes); the tuner chooses per shape class
__device__ __forceinline__ unsigned long long l2_evict_normal() {
  unsigned long long p;
  asm("createpolicy.fractional.L2::evict_normal.b64 %0, 1.0;" : "=l"(p));
  return p;
}
__device__ __forceinline__ float ld_stream(const float* a, unsigned long long pol) {
  float v;
  asm("ld.global.nc.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
  return v;
}
__device__ __forceinline__ int ld_stream(const int* a, unsigned long long pol) {
  int v;
  asm("ld.global.nc.L2::cache_hint.b32 %0, [%1], %2;" : "=r"(v) : "l"(a), "l"(pol));
  return v;
}

// scalar step after the reduction of iteration `it` (it updates done so far):
// stopping tests, then alpha and beta of the next direction, or the exits
__device__ __forceinline__ void sr_step(SState<float>& s, float gam, float del, float rho, float fail, int it,
                                        float tol2, int max_iter) {
  s.rr = rho;
  if (it == 0) {
    s.rr0 = rho;
    s.pfail = fail > 0.0f;
    s.ind = fail > 0.0f;
    s.iters = 0;
    s.hitmax = 0;
    s.nonfinite = !(rho == rho) || !(gam == gam);
    if (s.ind || s.nonfinite || !(rho > 0.0f)) {
      s.done = 1;
      return;
    }
  }
  if (!(rho == rho) || !(gam == gam) || !(del == del)) {
    s.nonfinite = 1;
    s.done = 1;
    return;
  }
  if (it > 0 && rho <= tol2 * s.rr0) {
    s.done = 1;
    return;
  }
  if (it > 0 && s.iters >= max_iter) {
    s.hitmax = 1;
    s.done = 1;
    return;
  }
  const float beta = it > 0 ? gam / s.rz : 0.0f;
  const float d = it > 0 ? del - beta * gam / s.alpha : del;  // p^T A p of the next direction
  s.dq = d;
  if (!(d > 0.0f)) {
    if (!(d == d)) s.nonfinite = 1;
    s.ind = 1;
    s.done = 1;
    return;
  }
  s.beta = beta;
  s.alpha = gam / d;
  s.rz = gam;
}

}  // namespace

size_t pcg_sr_smem_bytes(int ni, int nb, int nh, int mode) { return carve_sr(nullptr, ni, nb, nh, mode, nullptr); }

template <int MODE, bool ONE>
__global__ void __launch_bounds__(NTP, 1)
    k_pcg_sr(const SceneDev<float>* scenes, const TileRef* tiles, int n_tiles, const int* scene_ids,
               int n_scenes_arg, GridBar* bar, int b_from_g, int nb_cap, unsigned long long* flags,
               const int* halo_off, const int* halo_col, const int* halo_ref, int nh_cap, int l2_keep) {
  using W = Words<float>;
  // ONE: a launch of a single scene, whose slot is 0 and which never finishes while another
  // scene runs on (no progress-flag wait); the same operations in the same order
  const int n_scenes = ONE ? 1 : n_scenes_arg;
  constexpr bool HALO = MODE == SR_HALO, RES = MODE == SR_RES || HALO, GV = MODE == SR_GLOBAL;
  constexpr int MS = HALO ? HALO_MAX_SCENES : PCG_MAX_SCENES;  // scenes of one launch
  constexpr int GP = SP_GP;             // lanes per BSR row in the SpMV
  constexpr int RPP = NTP / GP;         // rows per SpMV pass
  // blocks per lane per gather round: from shared memory four (more in flight lengthen the
  // register-bound loop: 4.73 against 4.58 us per CG iteration on the beam), from global
  // memory eight (the streamed SpMV waits on memory latency)
  constexpr int U = RES ? 8 / GP : 16 / GP;
  constexpr int NW = NTP / 32;          // warps
  static_assert(RPP % PCG_TILE == 0 && NTP % PCG_TILE == 0, "passes cover whole tiles");
  static_assert(MS <= NTP, "one thread per scene in the scalar step");
  extern __shared__ __align__(16) char dyn[];
  __shared__ SState<float> st[MS];
  __shared__ SceneLite<float> sl[MS];
  __shared__ float s_sum[MS][NQ];
  __shared__ float s_tol2[MS];  // the scenes' squared relative tolerances, converted once (FP64 -> FP32)
  __shared__ int s_toff[MS];
  __shared__ int s_to, s_lo, s_hi;
  __shared__ unsigned s_seen;
  __shared__ int s_wslot, s_widx;
  __shared__ int s_scan[NW];

  const int tid = threadIdx.x, warp = tid >> 5, lane32 = tid & 31;
  const int grid = (int)gridDim.x;
  const int t0 = (int)(((long long)blockIdx.x * n_tiles) / grid);
  const int t1 = (int)(((long long)(blockIdx.x + 1) * n_tiles) / grid);
  const int ntl = t1 - t0;
  const int n_items = ntl * PCG_TILE;
  SrLayout L;
  carve_sr(dyn, n_items, nb_cap, nh_cap, MODE, &L);
  // SR_HALO: this CTA's first block in halo_col, its halo rows in halo_ref
  const int blk0 = HALO ? halo_off[2 * blockIdx.x] : 0;
  const int h0 = HALO ? halo_off[2 * blockIdx.x + 1] : 0;
  const int nh = HALO ? halo_off[2 * blockIdx.x + 3] - h0 : 0;
  if (tid == 0) {
    s_to = 0;
    s_lo = grid;
    s_hi = -1;
    s_seen = 0;
    s_wslot = s_widx = -1;
  }
  for (int si = tid; si < n_scenes; si += NTP) {
    load_lite(sl[si], scenes[scene_ids[si]]);
    st[si].done = 0;
    s_tol2[si] = (float)sl[si].tol2;
  }
  for (int lt = tid; lt < ntl; lt += NTP) {
    L.ltt[lt] = tiles[t0 + lt];
    L.ltc[lt] = 0;
  }
  __syncthreads();
  if (tid == 0) {
    int o = 0;
    for (int si = 0; si < n_scenes; ++si) {
      s_toff[si] = o;
      o += sl[si].n_ptiles;
    }
  }
  // row of a local item (-1: past the scene's last row) and its slot
  auto row_of = [&](int item, int& slot) -> int {
    const TileRef tr = L.ltt[item / PCG_TILE];
    slot = ONE ? 0 : tr.scene;
    const int i = tr.tile * PCG_TILE + item % PCG_TILE;
    return i < sl[slot].nv ? i : -1;
  };
  __syncthreads();
  // SR_HALO: the CTA's rows fit one SpMV pass, and the lane that forms w of a row in the
  // SpMV (the first of its GP lanes) owns the row: its x, r, p, s, u, w and block-Jacobi
  // inverse stay in that thread's registers for the whole solve (the same values, by the
  // same operations, as the other layouts keep in shared or global memory)
  const int o_item = spmv_row(tid);
  const bool owner = HALO && spmv_lane(tid) == 0 && o_item < n_items;
  int o_slot = 0, o_row = -1;
  if (owner) o_row = row_of(o_item, o_slot);
  float ox[3] = {0.f, 0.f, 0.f}, orr[3] = {0.f, 0.f, 0.f}, op[3] = {0.f, 0.f, 0.f}, os[3] = {0.f, 0.f, 0.f};
  float ou[3] = {0.f, 0.f, 0.f}, ow[3] = {0.f, 0.f, 0.f}, oq[6] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  static_assert(SR_HALO_MAX_ROWS == RPP, "the halo layout's rows fit one SpMV pass");
  if (HALO && n_items > RPP) {  // the planner never builds such a table; refuse it without touching memory
    if (tid == 0) atomicExch(&bar->timeout, 1);
    return;
  }
  // local row pointers (exclusive scan of the row lengths), resident blocks only
  if constexpr (RES) {
    int carry = 0;
    for (int base = 0; base < n_items; base += NTP) {
      const int item = base + tid;
      int len = 0;
      if (item < n_items) {
        int slot;
        const int i = row_of(item, slot);
        if (i >= 0) len = sl[slot].row_ptr[i + 1] - sl[slot].row_ptr[i];
      }
      int v = len;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(0xffffffffu, v, o);
        if (lane32 >= o) v += y;
      }
      if (lane32 == 31) s_scan[warp] = v;
      __syncthreads();
      if (tid < 32) {
        int w = (tid < NW) ? s_scan[tid] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const int y = __shfl_up_sync(0xffffffffu, w, o);
          if (tid >= o) w += y;
        }
        if (tid < NW) s_scan[tid] = w;
      }
      __syncthreads();
      const int excl = carry + v - len + (warp ? s_scan[warp - 1] : 0);
      if (item < n_items) L.lrp[item] = excl;
      const int total = s_scan[NW - 1];
      __syncthreads();
      carry += total;
    }
    if (tid == 0) L.lrp[n_items] = carry;
    __syncthreads();
    // the groups' slot steps (ceil(longest row / 2)), then their first steps; a table
    // the planner sized too small is refused before any block is stored
    const int ng = n_items / 16;
    for (int g = tid; g < ng; g += NTP) {
      int m = 0;
      for (int r = 16 * g; r < 16 * g + 16; ++r) m = max(m, L.lrp[r + 1] - L.lrp[r]);
      L.lgb[g + 1] = (m + 1) >> 1;
    }
    __syncthreads();
    if (tid == 0) {
      L.lgb[0] = 0;
      for (int g = 0; g < ng; ++g) L.lgb[g + 1] += L.lgb[g];
      if (32 * L.lgb[ng] > nb_cap) {
        s_to = 5;
        atomicExch(&bar->timeout, 1);
      }
    }
    __syncthreads();
    if (s_to) return;
  }
  // copy this CTA's blocks (SR_RES; SR_HALO with the local columns); without the halo, the
  // CTAs owning their columns bound the neighbour range of the u flags
  {
    int lo = grid, hi = -1;
    for (int item = warp; item < n_items; item += NW) {
      int slot;
      const int i = row_of(item, slot);
      if (i < 0) continue;
      const SceneLite<float>& S = sl[slot];
      const int kb = S.row_ptr[i], ke = S.row_ptr[i + 1];
      const size_t nb = (size_t)S.nnzb;
      for (int k = kb + lane32; k < ke; k += 32) {
        if constexpr (RES) {
          const int q = blk_slot(L.lgb, item, k - kb);
          L.lcol[q] = HALO ? halo_col[blk0 + L.lrp[item] + (k - kb)] : S.col[k];
#pragma unroll
          for (int c = 0; c < 9; ++c) L.lval[slot_val(q, c)] = S.val[c * nb + k];
        }
        if constexpr (!HALO) {
          const long long gt = s_toff[slot] + S.col[k] / PCG_TILE;  // tile in the launch's table
          const int owner = (int)(((gt + 1) * grid + n_tiles - 1) / n_tiles) - 1;
          lo = min(lo, owner);
          hi = max(hi, owner);
        }
      }
    }
    if constexpr (!HALO) {
      atomicMin(&s_lo, lo);
      atomicMax(&s_hi, hi);
    }
  }
  __syncthreads();

  // ---------------- exchange helpers
  // tile words: quantity k of a tile in parity buffer par is
  // pword[((par * NQ + k) * n_ptiles + tile) * pword_stride(n_ptiles)]
  // SR_HALO: w of the halo rows hb, hb + dh, ... (stamp s, buffer par) into their u slots,
  // which the SpMV has finished reading; one row at a time (two rows' loads in flight
  // measured slower in this register-bound kernel)
  auto halo_w = [&](int hb, int dh, unsigned s, int par) {
    auto rec = [&](int h, int& slot, int& row) -> const unsigned long long* {
      const int ref = L.href[h];
      slot = ONE ? 0 : ref >> HALO_ROW_BITS;
      row = ref & ((1 << HALO_ROW_BITS) - 1);
      if (st[slot].done) return nullptr;
      return reinterpret_cast<const unsigned long long*>(sl[slot].zrec) + ((size_t)par * sl[slot].nv + row) * 4;
    };
    auto wait = [&](const unsigned long long* wr, unsigned long long* w, int slot, int row) {
      for (unsigned spins = 0; !(W::has(w[0], s) && W::has(w[1], s) && W::has(w[2], s)); ++spins) {
        if (spins > kWaitSpins || *(volatile int*)&s_to) {
          if (!s_to) {
            s_to = 3;
            s_seen = (unsigned)((W::has(w[0], s) ? (W::has(w[1], s) ? w[2] : w[1]) : w[0]) >> 32);
            s_wslot = slot;
            s_widx = row;
          }
          break;
        }
        ld_relaxed_v2_u64(wr, w[0], w[1]);
        w[2] = ld_relaxed_u64(wr + 2);
      }
    };
#pragma unroll 1
    for (int h = hb; h < nh; h += dh) {
      int sa, ra;
      const unsigned long long* wa = rec(h, sa, ra);
      unsigned long long a[3];
      if (wa) {
        ld_relaxed_v2_u64(wa, a[0], a[1]);
        a[2] = ld_relaxed_u64(wa + 2);
        wait(wa, a, sa, ra);
        L.lu4[n_items + h] = make_float4(W::join(a), W::join(a + 1), W::join(a + 2), 0.0f);
      }
    }
  };
  // every CTA sums the tile words (buffer par) of quantities [0, nq) of every live scene
  // in tile order.  Once a scene of the launch has finished, a CTA may have no live tile
  // left and post nothing; one warp then also waits until every CTA has started this
  // iteration (progress flag >= s), so that no CTA is ever a whole iteration behind
  // another, which the parity buffers rely on.  (While every scene is live, every CTA
  // posts every iteration and the tile words alone ensure it.)  SR_HALO: the
  // halo's w words are read meanwhile, by the warps without other work when they are at
  // least half of the CTA, else by every warp first.
  auto reduce = [&](int nq, unsigned s, int par) -> bool {
    const int npw = n_scenes * nq + 1;  // warps with words to wait for (the last: the flags)
    if constexpr (HALO) {
      if (npw > NW / 2) halo_w(tid, NTP, s, par);
    }
    for (int x = warp; x < npw; x += NW) {
      if (x == npw - 1) {
        if constexpr (!ONE) {
          bool any_done = false;
          for (int si = 0; si < n_scenes; ++si) any_done |= st[si].done != 0;
          if (any_done)
            PPN_WARP_WAIT_STAMPS(flags, 0, grid - 1, (unsigned long long)s, kWaitSpins, lane32,
                                 *(volatile int*)&s_to, s_to = s_to ? s_to : 4);
        }
        continue;
      }
      const int si = ONE ? 0 : x / nq, q = ONE ? x : x % nq;
      if (st[si].done) continue;  // warp-uniform
      const SceneLite<float>& S = sl[si];
      const int n = S.n_ptiles;
      const size_t ws = (size_t)pword_stride(n);
      const unsigned long long* base = S.pword + (size_t)(par * NQ + q) * n * ws;
      float acc = 0.0f;
      for (int tw = lane32; tw < n; tw += 32 * 8) {
        unsigned long long w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = tw + 32 * u;
          w[u] = t < n ? ld_relaxed_u64(base + t * ws) : W::filler(s);
        }
        for (unsigned spins = 0;; ++spins) {
          bool ready = true;
#pragma unroll
          for (int u = 0; u < 8; ++u) ready &= W::has(w[u], s);
          if (ready) break;
          if (spins > kWaitSpins || *(volatile int*)&s_to) {
            if (!s_to) {
              s_to = 2;
              for (int u = 0; u < 8; ++u)
                if (!W::has(w[u], s)) {
                  s_seen = (unsigned)(w[u] >> 32);
                  s_wslot = si * 4 + q;
                  s_widx = tw + 32 * u;
                  break;
                }
            }
            break;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (!W::has(w[u], s)) w[u] = ld_relaxed_u64(base + (tw + 32 * u) * ws);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (tw + 32 * u < n) acc += W::join(&w[u]);
      }
      acc = warp_sum(acc);
      if (lane32 == 0) s_sum[si][q] = acc;
    }
    if constexpr (HALO) {
      if (npw <= NW / 2 && warp >= npw) halo_w((warp - npw) * 32 + lane32, (NW - npw) * 32, s, par);
    }
    __syncthreads();
    return !s_to;
  };
  // publish this CTA's vector values for its neighbours: release, then the flag
  auto publish_flag = [&](unsigned long long stamp) {
    __syncthreads();
    if (tid == 0) {
      fence_acq_rel();  // release (cumulative over the CTA's writes ordered by the barrier)
      st_relaxed_u64(flags + blockIdx.x, stamp);
    }
  };
  // wait until every CTA of the neighbour range has published `stamp`
  auto wait_flags = [&](unsigned long long stamp) -> bool {
    if (warp == 0) {
      PPN_WARP_WAIT_STAMPS(flags, s_lo, s_hi, stamp, kWaitSpins, lane32, *(volatile int*)&s_to,
                           s_to = s_to ? s_to : 1);
      fence_acq_rel();  // acquire: the neighbours' values before this CTA's gathers
    }
    __syncthreads();
    return !s_to;
  };
  // w = A u over this CTA's rows (GP lanes per row), u gathered from the global array or, in
  // SR_HALO, from shared memory; SR_HALO also stores w as stamped words (stamp s, buffer par)
  const unsigned long long pol = RES ? 0ull : l2_keep ? l2_evict_normal() : l2_evict_first();
  // the tile partials of tile lt (stamp s, buffer par): the fixed tree over its eight
  // 16-row group sums, posted as stamped words
  auto post_tile = [&](int lt, unsigned s, int par, int nq) {
    const TileRef tr = L.ltt[lt];
    const int sc = ONE ? 0 : tr.scene;
    const SceneLite<float>& S = sl[sc];
    if (st[sc].done) return;
    const float* w = L.lws + NQ * 8 * lt;
    const size_t ws = (size_t)pword_stride(S.n_ptiles);
    unsigned long long* wbase = S.pword + ((size_t)par * NQ * S.n_ptiles + tr.tile) * ws;
    for (int q = 0; q < nq; ++q) {
      const float a = (w[q] + w[NQ + q]) + (w[2 * NQ + q] + w[3 * NQ + q]);
      const float b = (w[4 * NQ + q] + w[5 * NQ + q]) + (w[6 * NQ + q] + w[7 * NQ + q]);
      unsigned long long wd[1];
      W::split(a + b, s, wd);
      st_relaxed_u64(wbase + (size_t)q * S.n_ptiles * ws, wd[0]);
    }
  };
  // w = A u; each tile's partials are posted by the warp that completes its last group
  auto spmv = [&](unsigned s, int par, int nq) {
    for (int base = 0; base < n_items; base += RPP) {
      const int row = spmv_row(tid), lane = spmv_lane(tid);
      const int item = base + row;
      float ax = 0.f, ay = 0.f, az = 0.f;
      int slot = 0, i = -1;
      if (item < n_items) i = row_of(item, slot);
      if (i >= 0 && !st[slot].done) {
        const SceneLite<float>& S = sl[slot];
        const float* vb = u_ptr(S.zrec, 0);
        if constexpr (RES) {
          // this lane's blocks lane, lane + 2, ... of the row, in order, by slot step
          const int len = L.lrp[item + 1] - L.lrp[item], g = item >> 4;
          const int j0 = L.lgb[g], nj = L.lgb[g + 1] - j0;
          for (int jb = 0; jb < nj; jb += U) {
            float4 vj[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int j = jb + u;
              if (GP * j + lane < len) {
                const int cl = L.lcol[(j0 + j) * 32 + lane32];
                vj[u] = HALO ? L.lu4[cl] : ld_f4_cg(vb + (size_t)8 * cl);
              }
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int j = jb + u;
              if (GP * j + lane < len) {
                const float* v = L.lval + (j0 + j) * 288 + lane32;
                float a[9];
#pragma unroll
                for (int c = 0; c < 9; ++c) a[c] = v[32 * c];
                blk_mv(a, vj[u].x, vj[u].y, vj[u].z, ax, ay, az);
              }
            }
          }
        } else {
          // blocks from global memory (component-major values), read-only path, evict-first in L2
          const int lb = S.row_ptr[i], le = S.row_ptr[i + 1];
          const size_t nb = (size_t)S.nnzb;
          for (int b0 = lb + lane; b0 < le; b0 += GP * U) {
            float4 vj[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int b = b0 + GP * u;
              if (b < le) vj[u] = ld_f4_cg(vb + (size_t)8 * ld_stream(S.col + b, pol));
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int b = b0 + GP * u;
              if (b < le) {
                float a[9];
#pragma unroll
                for (int c = 0; c < 9; ++c) a[c] = ld_stream(S.val + c * nb + b, pol);
                blk_mv(a, vj[u].x, vj[u].y, vj[u].z, ax, ay, az);
              }
            }
          }
        }
      }
#pragma unroll
      // the row's w in both of its lanes (lane 0 + lane 1, and lane 1 + lane 0: the same bits)
      ax += __shfl_xor_sync(0xffffffffu, ax, 16);
      ay += __shfl_xor_sync(0xffffffffu, ay, 16);
      az += __shfl_xor_sync(0xffffffffu, az, 16);
      if (lane == 0 && item < n_items) {
        if constexpr (GV) {
          if (i >= 0) st_f4(reinterpret_cast<float*>(sl[slot].q + i), ax, ay, az);
        } else if constexpr (HALO) {
          ow[0] = ax, ow[1] = ay, ow[2] = az;
        } else {
          L.lw[3 * item] = ax;
          L.lw[3 * item + 1] = ay;
          L.lw[3 * item + 2] = az;
        }
      }
      // the row's terms: gamma = r.u and rho = r.r in its first lane, delta = w.u in its second
      float x = 0.f, rr = 0.f;
      if (item < n_items && i >= 0 && !st[slot].done) {
        if (lane == 0) {
          float r[3], u[3];
          if constexpr (GV) {
            const float4 rv = ld_f4_cg(reinterpret_cast<const float*>(sl[slot].z + i));
            const float4 uv = ld_f4_cg(u_ptr(sl[slot].zrec, i));
            r[0] = rv.x, r[1] = rv.y, r[2] = rv.z;
            u[0] = uv.x, u[1] = uv.y, u[2] = uv.z;
          } else if constexpr (HALO) {
            unsigned long long w[3];
            W::split(ax, s, w);
            W::split(ay, s, w + 1);
            W::split(az, s, w + 2);
            unsigned long long* wr =
                reinterpret_cast<unsigned long long*>(sl[slot].zrec) + ((size_t)par * sl[slot].nv + i) * 4;
            st_relaxed_v2_u64(wr, w[0], w[1]);
            st_relaxed_u64(wr + 2, w[2]);
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              u[c] = ou[c];
              r[c] = orr[c];
            }
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              r[c] = L.lr[3 * item + c];
              u[c] = L.lu[3 * item + c];
            }
          }
          x = dot3(r[0], r[1], r[2], u[0], u[1], u[2]);
          rr = dot3(r[0], r[1], r[2], r[0], r[1], r[2]);
        } else {
          float u[3];
          if constexpr (GV) {
            const float4 uv = ld_f4_cg(u_ptr(sl[slot].zrec, i));
            u[0] = uv.x, u[1] = uv.y, u[2] = uv.z;
          } else if constexpr (HALO) {
            const float4 uv = L.lu4[item];
            u[0] = uv.x, u[1] = uv.y, u[2] = uv.z;
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) u[c] = L.lu[3 * item + c];
          }
          x = dot3(ax, ay, az, u[0], u[1], u[2]);
        }
      }
      // per group of 16 rows (one warp of the pass), in a fixed order: the tree over the 16
      // rows of warp_sum, lanes 0-15 for gamma and rho, lanes 16-31 for delta
#pragma unroll
      for (int o = 8; o > 0; o >>= 1) {
        x += __shfl_xor_sync(0xffffffffu, x, o);
        rr += __shfl_xor_sync(0xffffffffu, rr, o);
      }
      const int grp = (base >> 4) + warp, lt = grp >> 3;
      float* og = L.lws + NQ * grp;
      if (lane32 == 16) og[1] = x;
      if (lane32 == 0) {
        og[0] = x;
        og[2] = rr;
      }
      __syncwarp();  // (delta's sum, stored by lane 16, before lane 0's count)
      if (lane32 == 0) {
        if (lt < ntl) {  // (the groups past the CTA's tiles of a one-tile CTA post nothing)
          __threadfence_block();  // the group sums before the count
          if (atomicAdd(&L.ltc[lt], 1) == 7) {
            __threadfence_block();  // the other groups' sums after their counts
            L.ltc[lt] = 0;
            post_tile(lt, s, par, nq);
          }
        }
      }
    }
    __syncthreads();
  };

  // a wait ran out: record the first one (iteration, wait) and flag the timeout
  auto fail_out = [&](int it) {
    if (tid == 0) {
      if (atomicCAS(&bar->to_site, 0, s_to) == 0) {
        bar->to_iter = (unsigned)it;
        bar->to_seen = s_seen;
        bar->to_slot = s_wslot;
        bar->to_index = s_widx;
        bar->to_cta = blockIdx.x;
      }
      atomicExch(&bar->timeout, 1);
    }
  };

  // ---------------- set-up: P = block-Jacobi inverse, x = 0, r = b, u = P r
  // right-hand side b of row i: -g (FP64 gradient) or the given r
  auto rhs = [&](const SceneLite<float>& S, int i, float* r) {
    if (b_from_g) {
      const double4 g = ld_d4(S.g + i);
      r[0] = (float)(-g.x);
      r[1] = (float)(-g.y);
      r[2] = (float)(-g.z);
    } else {
      const float4 rv = ld_f4_cg(reinterpret_cast<const float*>(S.r + i));
      r[0] = rv.x;
      r[1] = rv.y;
      r[2] = rv.z;
    }
  };
  if constexpr (HALO) {
    // each owner sets up its row; the failed-block count of a 16-row group (one warp's
    // owners) goes to the group's slot
    float fail = 0.0f;
    if (owner && o_row >= 0) {
      const SceneLite<float>& S = sl[o_slot];
      const int i = o_row;
      float D[9], Pm[9];
      const int bd = blk_slot(L.lgb, o_item, S.diag_idx[i] - S.row_ptr[i]);
#pragma unroll
      for (int c = 0; c < 9; ++c) D[c] = L.lval[slot_val(bd, c)];
      const bool ok = spd_inv3(D, Pm);
      sym6(Pm, oq);
      float* P = S.Pinv + (size_t)9 * i;
#pragma unroll
      for (int c = 0; c < 9; ++c) P[c] = Pm[c];
      rhs(S, i, orr);
      prec6(oq, orr, ou);
      L.lu4[o_item] = make_float4(ou[0], ou[1], ou[2], 0.0f);
      fail = ok ? 0.0f : 1.0f;
    } else if (owner) {
      L.lu4[o_item] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    fail = warp_sum(fail);
    if (lane32 == 0) L.lws[NQ * warp + 3] = fail;
  }
  for (int base = 0; !HALO && base < n_items; base += NTP) {
    const int item = base + tid;
    float fail = 0.0f;
    int slot = 0;
    const int i = item < n_items ? row_of(item, slot) : -1;
    if (i >= 0) {
      const SceneLite<float>& S = sl[slot];
      float D[9];
      if constexpr (RES) {
        const int bd = blk_slot(L.lgb, item, S.diag_idx[i] - S.row_ptr[i]);
#pragma unroll
        for (int c = 0; c < 9; ++c) D[c] = L.lval[slot_val(bd, c)];
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) D[c] = S.val[(size_t)c * S.nnzb + S.diag_idx[i]];
      }
      float Pm[9], q[6];
      const bool ok = spd_inv3(D, Pm);
      sym6(Pm, q);
      float* P = S.Pinv + (size_t)9 * i;
#pragma unroll
      for (int c = 0; c < 9; ++c) P[c] = Pm[c];
      if constexpr (!GV) {
#pragma unroll
        for (int c = 0; c < 6; ++c) L.lP[6 * item + c] = q[c];
      }
      float r[3], u[3];
      rhs(S, i, r);
      prec6(q, r, u);
      if constexpr (GV) {
        st_f4(u_ptr(S.zrec, i), u[0], u[1], u[2]);
        st_f4(reinterpret_cast<float*>(S.z + i), r[0], r[1], r[2]);
        st_f4(reinterpret_cast<float*>(S.dx + i), 0.f, 0.f, 0.f);
        st_f4(reinterpret_cast<float*>(S.d0 + i), 0.f, 0.f, 0.f);
        st_f4(reinterpret_cast<float*>(S.d1 + i), 0.f, 0.f, 0.f);
      } else {
        const int k = 3 * item;
        if constexpr (HALO) {
          L.lu4[item] = make_float4(u[0], u[1], u[2], 0.0f);
        } else {
          st_f4(u_ptr(S.zrec, i), u[0], u[1], u[2]);
#pragma unroll
          for (int c = 0; c < 3; ++c) L.lu[k + c] = u[c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          L.lr[k + c] = r[c];
          L.lx[k + c] = L.lp[k + c] = L.ls[k + c] = 0.0f;
        }
      }
      fail = ok ? 0.0f : 1.0f;
    } else if (HALO && item < n_items) {
      L.lu4[item] = make_float4(0.0f, 0.0f, 0.0f, 0.0f);
    }
    fail = warp_sum(fail);  // the warp's 32 rows: its first 16-row group takes the count
    if (lane32 == 0) {
      L.lws[NQ * ((base >> 4) + 2 * warp) + 3] = fail;
      L.lws[NQ * ((base >> 4) + 2 * warp + 1) + 3] = 0.0f;
    }
  }
  // SR_HALO: the halo rows' state, as their owners set it up (same inputs, same operations)
  if constexpr (HALO) {
    for (int h = tid; h < nh; h += NTP) {
      const int ref = halo_ref[h0 + h];
      L.href[h] = ref;
      const SceneLite<float>& S = sl[ONE ? 0 : ref >> HALO_ROW_BITS];
      const int i = ref & ((1 << HALO_ROW_BITS) - 1);
      float D[9], Pm[9], r[3], u[3];
#pragma unroll
      for (int c = 0; c < 9; ++c) D[c] = S.val[(size_t)c * S.nnzb + S.diag_idx[i]];
      spd_inv3(D, Pm);
      float* q = L.hP + 6 * h;
      sym6(Pm, q);
      rhs(S, i, r);
      prec6(q, r, u);
      L.lu4[n_items + h] = make_float4(u[0], u[1], u[2], 0.0f);
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        L.hr[3 * h + c] = r[c];
        L.hs[3 * h + c] = 0.0f;
      }
    }
  }

  for (int it = 0;; ++it) {
    const unsigned s = W::stamp((unsigned)it + 1);
    if constexpr (HALO) {
      __syncthreads();  // set-up, or the previous update, before the SpMV
      if (tid == 0) st_relaxed_u64(flags + blockIdx.x, (unsigned long long)it + 1);  // progress
    } else {
      // ---- u released to the neighbours (set-up wrote u_0; later iterations below)
      publish_flag((unsigned long long)it + 1);
      if (!wait_flags((unsigned long long)it + 1)) return fail_out(it);
    }
    spmv(s, it & 1, it == 0 ? NQ : 3);  // w = A u, and the tile partials posted
    if (!reduce(it == 0 ? NQ : 3, s, it & 1)) return fail_out(it);
    // one thread per scene (n_scenes <= MS < NTP); the barrier also finds whether all are done
    int done = 1;
    if (tid < n_scenes) {
      if (!st[tid].done)
        sr_step(st[tid], s_sum[tid][0], s_sum[tid][1], s_sum[tid][2], it == 0 ? s_sum[tid][3] : 0.0f, it,
                s_tol2[tid], sl[tid].max_iter);
      done = st[tid].done;
    }
    if (__syncthreads_and(done)) break;
    // ---- p = u + beta p, s = w + beta s; x += alpha p, r -= alpha s, u = M r (published)
    if constexpr (HALO) {
      if (o_row >= 0 && !st[o_slot].done) {
        const float a = st[o_slot].alpha, b = st[o_slot].beta;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          upd_px(a, b, ou[c], op[c], ox[c]);
          upd_sr(a, b, ow[c], os[c], orr[c]);
        }
        prec6(oq, orr, ou);
        L.lu4[o_item] = make_float4(ou[0], ou[1], ou[2], 0.0f);
      }
    }
    for (int item = tid; !HALO && item < n_items; item += NTP) {
      int slot;
      const int i = row_of(item, slot);
      if (i < 0 || st[slot].done) continue;
      const float a = st[slot].alpha, b = st[slot].beta;
      const SceneLite<float>& S = sl[slot];
      float r[3], q[6], u[3];
      if constexpr (GV) {
        const float4 uv = ld_f4_cg(u_ptr(S.zrec, i));
        float4 pv = ld_f4_cg(reinterpret_cast<const float*>(S.d0 + i));
        const float4 wv = ld_f4_cg(reinterpret_cast<const float*>(S.q + i));
        float4 sv = ld_f4_cg(reinterpret_cast<const float*>(S.d1 + i));
        float4 xv = ld_f4_cg(reinterpret_cast<const float*>(S.dx + i));
        const float4 rv = ld_f4_cg(reinterpret_cast<const float*>(S.z + i));
        r[0] = rv.x, r[1] = rv.y, r[2] = rv.z;
        upd_px(a, b, uv.x, pv.x, xv.x);
        upd_px(a, b, uv.y, pv.y, xv.y);
        upd_px(a, b, uv.z, pv.z, xv.z);
        upd_sr(a, b, wv.x, sv.x, r[0]);
        upd_sr(a, b, wv.y, sv.y, r[1]);
        upd_sr(a, b, wv.z, sv.z, r[2]);
        st_f4(reinterpret_cast<float*>(S.d0 + i), pv.x, pv.y, pv.z);
        st_f4(reinterpret_cast<float*>(S.d1 + i), sv.x, sv.y, sv.z);
        st_f4(reinterpret_cast<float*>(S.dx + i), xv.x, xv.y, xv.z);
        st_f4(reinterpret_cast<float*>(S.z + i), r[0], r[1], r[2]);
        const float* P = S.Pinv + (size_t)9 * i;
        q[0] = __ldcg(P), q[1] = __ldcg(P + 1), q[2] = __ldcg(P + 2);
        q[3] = __ldcg(P + 4), q[4] = __ldcg(P + 5), q[5] = __ldcg(P + 8);
      } else {
        const int k = 3 * item;
        float uo[3];
        if constexpr (HALO) {
          const float4 uv = L.lu4[item];
          uo[0] = uv.x, uo[1] = uv.y, uo[2] = uv.z;
        } else {
#pragma unroll
          for (int c = 0; c < 3; ++c) uo[c] = L.lu[k + c];
        }
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          upd_px(a, b, uo[c], L.lp[k + c], L.lx[k + c]);
          r[c] = L.lr[k + c];
          upd_sr(a, b, L.lw[k + c], L.ls[k + c], r[c]);
          L.lr[k + c] = r[c];
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) q[c] = L.lP[6 * item + c];
      }
      prec6(q, r, u);
      if constexpr (HALO) {
        L.lu4[item] = make_float4(u[0], u[1], u[2], 0.0f);
      } else {
        if constexpr (!GV) {
#pragma unroll
          for (int c = 0; c < 3; ++c) L.lu[3 * item + c] = u[c];
        }
        st_f4(u_ptr(S.zrec, i), u[0], u[1], u[2]);
      }
    }
    // SR_HALO: the halo rows repeat their owners' s, r and u updates with the owners' w
    if constexpr (HALO) {
      // every load of a row issued before its arithmetic (the arrays do not alias); the loop
      // is kept rolled (unrolled it measured 1 % slower in this register-bound kernel)
#pragma unroll 1
      for (int h = tid; h < nh; h += NTP) {
        const int slot = ONE ? 0 : L.href[h] >> HALO_ROW_BITS;
        if (st[slot].done) continue;
        const float a = st[slot].alpha, b = st[slot].beta;
        const float4 wv = L.lu4[n_items + h];
        float r[3], sv[3], q[6], u[3];
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          r[c] = L.hr[3 * h + c];
          sv[c] = L.hs[3 * h + c];
        }
#pragma unroll
        for (int c = 0; c < 6; ++c) q[c] = L.hP[6 * h + c];
        upd_sr(a, b, wv.x, sv[0], r[0]);
        upd_sr(a, b, wv.y, sv[1], r[1]);
        upd_sr(a, b, wv.z, sv[2], r[2]);
        prec6(q, r, u);
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          L.hr[3 * h + c] = r[c];
          L.hs[3 * h + c] = sv[c];
        }
        L.lu4[n_items + h] = make_float4(u[0], u[1], u[2], 0.0f);
      }
    }
    for (int si = tid; si < n_scenes; si += NTP)
      if (!st[si].done) st[si].iters += 1;
    // (the barrier at the top of the next iteration orders these updates)
  }

  // x of this CTA's rows to global memory (SR_GLOBAL: already there); CTA 0 publishes the scalars
  if constexpr (HALO) {
    if (o_row >= 0) st_v(sl[o_slot].dx + o_row, mk<float4, float>(ox[0], ox[1], ox[2]));
  } else if constexpr (!GV) {
    for (int item = tid; item < n_items; item += NTP) {
      int slot;
      const int i = row_of(item, slot);
      if (i < 0) continue;
      const float* lx = L.lx + 3 * item;
      st_v(sl[slot].dx + i, mk<float4, float>(lx[0], lx[1], lx[2]));
    }
  }
  if (blockIdx.x == 0)
    for (int si = tid; si < n_scenes; si += NTP) publish(st[si], sl[si].ctl);
}

// One warp waits, through the PCG's flag-wait helper, on n stamped words that
// nothing else writes; out = 1 when the wait ran out.  Exercises the bounded-wait
// path without a second party.
__global__ void k_wait_probe(const unsigned long long* w, int n, unsigned long long stamp, unsigned limit, int* out) {
  __shared__ int s_to;
  if (threadIdx.x == 0) s_to = 0;
  __syncwarp();
  const int lane32 = threadIdx.x & 31;
  PPN_WARP_WAIT_STAMPS(w, 0, n - 1, stamp, limit, lane32, *(volatile int*)&s_to, s_to = 1);
  __syncwarp();
  if (threadIdx.x == 0) *out = s_to ? 1 : 0;
}

cudaError_t launch_wait_probe(const unsigned long long* w, int n, unsigned long long stamp, unsigned limit, int* out,
                              cudaStream_t st) {
  if (n <= 0) return cudaErrorInvalidValue;
  k_wait_probe<<<1, 32, 0, st>>>(w, n, stamp, limit, out);
  return cudaGetLastError();
}

// The kernel of a layout; `one`: a launch of a single scene.  The single-scene forms of
// the layouts without the halo drop the per-scene indexing of their SpMV and update
// (press, global layout, same-box A/B: 50.1 -> 45.5 us per CG iteration, the same bits).
// The halo layout keeps one form: its single-scene form measured 4.48 -> 4.66 us on the
// beam, where the compiler schedules the register-resident rows differently.
static const void* sr_kernel(int mode, bool one) {
  switch (mode) {
    case SR_RES: return one ? (const void*)k_pcg_sr<SR_RES, true> : (const void*)k_pcg_sr<SR_RES, false>;
    case SR_STREAM: return one ? (const void*)k_pcg_sr<SR_STREAM, true> : (const void*)k_pcg_sr<SR_STREAM, false>;
    case SR_GLOBAL: return one ? (const void*)k_pcg_sr<SR_GLOBAL, true> : (const void*)k_pcg_sr<SR_GLOBAL, false>;
    default: return (const void*)k_pcg_sr<SR_HALO, false>;
  }
}

int pcg_sr_max_grid(int device, size_t smem, int mode) {
  // (the multi-scene form; the single-scene forms use no more registers or shared memory, so the
  // same one CTA per SM is co-resident, and the launch sets its own kernel's attribute)
  const void* k = sr_kernel(mode, false);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NTP, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * prop.multiProcessorCount;
}

cudaError_t launch_pcg_sr(const SceneDev<float>* scenes, const PcgLaunch& L, cudaStream_t st) {
  const bool halo = L.sr_mode == SR_HALO;
  if (L.n_scenes <= 0 || L.n_scenes > PCG_MAX_SCENES || L.n_tiles <= 0 || L.grid > XCH_MAX_CTAS || !L.flags ||
      L.sr_mode < SR_RES || L.sr_mode > SR_HALO || (L.sr_mode == SR_RES || halo) != (L.smem_blocks > 0) ||
      (halo && (L.n_scenes > HALO_MAX_SCENES || !L.halo_off || !L.halo_col || !L.halo_ref || L.halo_cap < 0 ||
                (L.n_tiles + L.grid - 1) / L.grid * PCG_TILE > SR_HALO_MAX_ROWS)))
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(L.bar, 0, sizeof(GridBar), st);
  if (e != cudaSuccess) return e;
  // flags and exchange words carry stamps of this launch only
  e = cudaMemsetAsync(L.flags, 0, sizeof(unsigned long long) * L.grid, st);
  if (e != cudaSuccess) return e;
  for (int k = 0; k < L.n_pword; ++k) {
    e = cudaMemsetAsync(L.pword[k], 0, L.pword_bytes[k], st);
    if (e != cudaSuccess) return e;
  }
  for (int k = 0; halo && k < L.n_scenes; ++k) {
    if (!L.zrec[k]) return cudaErrorInvalidValue;
    e = cudaMemsetAsync(L.zrec[k], 0, L.zrec_bytes[k], st);
    if (e != cudaSuccess) return e;
  }
  const TileRef* tiles = L.tiles;
  int n_tiles = L.n_tiles;
  const int* ids = L.scene_ids;
  int n_scenes = L.n_scenes;
  GridBar* bar = L.bar;
  int bg = L.use_b_from_g;
  int nb_cap = L.smem_blocks;
  unsigned long long* flags = L.flags;
  const int* h_off = halo ? L.halo_off : nullptr;
  const int* h_col = halo ? L.halo_col : nullptr;
  const int* h_ref = halo ? L.halo_ref : nullptr;
  int nh_cap = halo ? L.halo_cap : 0;
  int l2_keep = L.l2_keep;
  void* args[] = {(void*)&scenes, (void*)&tiles, (void*)&n_tiles, (void*)&ids,   (void*)&n_scenes,
                  (void*)&bar,    (void*)&bg,    (void*)&nb_cap,  (void*)&flags, (void*)&h_off,
                  (void*)&h_col,  (void*)&h_ref, (void*)&nh_cap, (void*)&l2_keep};
  const void* k = sr_kernel(L.sr_mode, L.n_scenes == 1);
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(k, dim3(L.grid), dim3(NTP), args, L.smem_bytes, st);
}

}  // namespace ppn
