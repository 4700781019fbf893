// Single-reduction block-Jacobi PCG (the linear solve of Algorithm 1; Sec. 4.1
// "Linear Solvers", Sec. 5.1) for the FP32 path: one grid-wide reduction and
// one neighbour-only synchronisation per iteration, instead of the two
// grid-wide reductions of the textbook recurrences.
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
// Data.  Three layouts (SR_RES, SR_STREAM, SR_GLOBAL).  SR_RES and SR_STREAM
// keep each CTA's rows' block-Jacobi inverse and vectors x, r, u, w, p, s in
// shared memory; SR_RES also keeps the rows' BSR blocks there, SR_STREAM
// streams them from global memory (L2 / HBM) every iteration through the
// read-only path.  SR_GLOBAL, for rows that do not fit, keeps the vectors in
// the scene's global PCG arrays as well (x in dx, r in z, w in q, p in d0,
// s in d1, the inverse in Pinv), each row touched only by its own CTA.  In
// every layout only u crosses CTAs, through a global array.
//
// Synchronisation.  A CTA publishes its u values, then a flag with the
// iteration's stamp; before its SpMV it waits only for the flags of the CTAs
// that own the columns of its rows (a contiguous CTA range found at set-up).
// The reduction's tile partials go out as stamped words after the SpMV, and
// every CTA sums them in tile order.  One u array suffices: a CTA overwrites
// it only after it has seen every CTA's partials of the previous iteration,
// which each CTA posts after finishing the SpMV that read the old values.
// All waits are bounded.
#include "pcg_common.cuh"

namespace ppn {

using namespace pcgdev;

namespace {

constexpr int NTP = 512;  // threads per CTA
constexpr int NQ = 4;     // reduction slots: gamma, delta, rho, failed diagonal blocks

struct SrLayout {
  float* lws;    // [(ni / PCG_TILE + 1) * 16 * NQ] partial sums per 16-row group (8 per tile)
  TileRef* ltt;  // [ni / PCG_TILE + 1] the CTA's tiles
  int* lrp;      // SR_RES: [ni + 1] local row pointers
  int* lcol;     // SR_RES: [nb]
  float* lval;   // SR_RES: [nb * 9]
  float* lP;     // SR_RES, SR_STREAM: [ni * 9]
  float *lx, *lr, *lu, *lw, *lp, *ls;  // SR_RES, SR_STREAM: [ni * 3] each
};

__host__ __device__ inline size_t up16(size_t b) { return (b + 15) & ~size_t(15); }

// the layout's pieces in carving order (nullptr base: sizes only)
__host__ __device__ inline size_t carve_sr(char* base, int ni, int nb, int mode, SrLayout* L) {
  const int ntl = ni / PCG_TILE + 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base ? base + off : nullptr;
    off += up16(bytes);
    return p;
  };
  SrLayout l{};
  l.lws = (float*)take(sizeof(float) * ntl * 16 * NQ);
  l.ltt = (TileRef*)take(sizeof(TileRef) * ntl);
  if (mode == SR_RES) {
    l.lrp = (int*)take(sizeof(int) * (ni + 1));
    l.lcol = (int*)take(sizeof(int) * nb);
    l.lval = (float*)take(sizeof(float) * 9 * nb);
  }
  if (mode != SR_GLOBAL) {
    l.lP = (float*)take(sizeof(float) * 9 * ni);
    float** v[6] = {&l.lx, &l.lr, &l.lu, &l.lw, &l.lp, &l.ls};
    for (float** q : v) *q = (float*)take(sizeof(float) * 3 * ni);
  }
  if (L) *L = l;
  return off;
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
                                        double tol2, int max_iter) {
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
  if (it > 0 && rho <= (float)tol2 * s.rr0) {
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

size_t pcg_sr_smem_bytes(int ni, int nb, int mode) { return carve_sr(nullptr, ni, nb, mode, nullptr); }

template <int MODE>
__global__ void __launch_bounds__(NTP, 1)
    k_pcg_sr(const SceneDev<float>* scenes, const TileRef* tiles, int n_tiles, const int* scene_ids,
               int n_scenes, GridBar* bar, int b_from_g, int nb_cap, unsigned long long* flags) {
  using W = Words<float>;
  constexpr bool RES = MODE == SR_RES, GV = MODE == SR_GLOBAL;
  constexpr int GP = 2;                 // lanes per BSR row in the SpMV
  constexpr int RPP = NTP / GP;         // rows per SpMV pass
  constexpr int U = 16 / GP;            // blocks per lane per gather round
  constexpr int NW = NTP / 32;          // warps
  static_assert(RPP % PCG_TILE == 0 && NTP % PCG_TILE == 0, "passes cover whole tiles");
  static_assert(PCG_MAX_SCENES <= NTP, "one thread per scene in the scalar step");
  extern __shared__ __align__(16) char dyn[];
  __shared__ SState<float> st[PCG_MAX_SCENES];
  __shared__ SceneLite<float> sl[PCG_MAX_SCENES];
  __shared__ float s_sum[PCG_MAX_SCENES][NQ];
  __shared__ int s_toff[PCG_MAX_SCENES];
  __shared__ int s_to, s_lo, s_hi;
  __shared__ int s_scan[NW];

  const int tid = threadIdx.x, warp = tid >> 5, lane32 = tid & 31;
  const int grid = (int)gridDim.x;
  const int t0 = (int)(((long long)blockIdx.x * n_tiles) / grid);
  const int t1 = (int)(((long long)(blockIdx.x + 1) * n_tiles) / grid);
  const int ntl = t1 - t0;
  const int n_items = ntl * PCG_TILE;
  SrLayout L;
  carve_sr(dyn, n_items, nb_cap, MODE, &L);
  if (tid == 0) {
    s_to = 0;
    s_lo = grid;
    s_hi = -1;
  }
  for (int si = tid; si < n_scenes; si += NTP) {
    load_lite(sl[si], scenes[scene_ids[si]]);
    st[si].done = 0;
  }
  for (int lt = tid; lt < ntl; lt += NTP) L.ltt[lt] = tiles[t0 + lt];
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
    slot = tr.scene;
    const int i = tr.tile * PCG_TILE + item % PCG_TILE;
    return i < sl[slot].nv ? i : -1;
  };
  __syncthreads();
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
  }
  // copy this CTA's blocks (RES); the CTAs owning their columns bound the neighbour range
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
        const int j = S.col[k];
        if constexpr (RES) {
          const int b = L.lrp[item] + (k - kb);
          L.lcol[b] = j;
#pragma unroll
          for (int c = 0; c < 9; ++c) L.lval[9 * b + c] = S.val[c * nb + k];
        }
        const long long gt = s_toff[slot] + j / PCG_TILE;  // tile in the launch's table
        const int owner = (int)(((gt + 1) * grid + n_tiles - 1) / n_tiles) - 1;
        lo = min(lo, owner);
        hi = max(hi, owner);
      }
    }
    atomicMin(&s_lo, lo);
    atomicMax(&s_hi, hi);
  }
  __syncthreads();

  // ---------------- exchange helpers
  auto post_tile = [&](int lt, int k, float v, unsigned s) {
    const TileRef tr = L.ltt[lt];
    const SceneLite<float>& S = sl[tr.scene];
    unsigned long long w[1];
    W::split(v, s, w);
    st_relaxed_u64(S.pword + (size_t)k * S.n_ptiles + tr.tile, w[0]);
  };
  // every CTA sums the tile words of quantities [0, nq) of every live scene in tile order
  auto reduce = [&](int nq, unsigned s) -> bool {
    for (int x = warp; x < n_scenes * nq; x += NW) {
      const int si = x / nq, q = x % nq;
      if (st[si].done) continue;  // warp-uniform
      const SceneLite<float>& S = sl[si];
      const int n = S.n_ptiles;
      const unsigned long long* base = S.pword + (size_t)q * n;
      float acc = 0.0f;
      for (int tw = lane32; tw < n; tw += 32 * 8) {
        unsigned long long w[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = tw + 32 * u;
          w[u] = t < n ? ld_relaxed_u64(base + t) : W::filler(s);
        }
        for (unsigned spins = 0;; ++spins) {
          bool ready = true;
#pragma unroll
          for (int u = 0; u < 8; ++u) ready &= W::has(w[u], s);
          if (ready) break;
          if (spins > kWaitSpins || *(volatile int*)&s_to) {
            s_to = 1;
            break;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u)
            if (!W::has(w[u], s)) w[u] = ld_relaxed_u64(base + tw + 32 * u);
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (tw + 32 * u < n) acc += W::join(&w[u]);
      }
      acc = warp_sum(acc);
      if (lane32 == 0) s_sum[si][q] = acc;
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
      PPN_WARP_WAIT_STAMPS(flags, s_lo, s_hi, stamp, kWaitSpins, lane32, *(volatile int*)&s_to, s_to = 1);
      fence_acq_rel();  // acquire: the neighbours' values before this CTA's gathers
    }
    __syncthreads();
    return !s_to;
  };
  // w = A u over this CTA's rows, u gathered from the global array (GP lanes per row)
  const unsigned long long pol = RES ? 0ull : l2_evict_first();
  auto spmv = [&]() {
    for (int base = 0; base < n_items; base += RPP) {
      const int row = tid / GP, lane = tid % GP;
      const int item = base + row;
      float ax = 0.f, ay = 0.f, az = 0.f;
      int slot = 0, i = -1;
      if (item < n_items) i = row_of(item, slot);
      if (i >= 0 && !st[slot].done) {
        const SceneLite<float>& S = sl[slot];
        const float* vb = u_ptr(S.zrec, 0);
        if constexpr (RES) {
          const int lb = L.lrp[item], le = L.lrp[item + 1];
          for (int b0 = lb + lane; b0 < le; b0 += GP * U) {
            float4 vj[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int b = b0 + GP * u;
              if (b < le) vj[u] = ld_f4_cg(vb + (size_t)8 * L.lcol[b]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int b = b0 + GP * u;
              if (b < le) {
                const float* a = L.lval + 9 * b;
                ax += a[0] * vj[u].x + a[1] * vj[u].y + a[2] * vj[u].z;
                ay += a[3] * vj[u].x + a[4] * vj[u].y + a[5] * vj[u].z;
                az += a[6] * vj[u].x + a[7] * vj[u].y + a[8] * vj[u].z;
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
                ax += a[0] * vj[u].x + a[1] * vj[u].y + a[2] * vj[u].z;
                ay += a[3] * vj[u].x + a[4] * vj[u].y + a[5] * vj[u].z;
                az += a[6] * vj[u].x + a[7] * vj[u].y + a[8] * vj[u].z;
              }
            }
          }
        }
      }
#pragma unroll
      for (int o = GP / 2; o > 0; o >>= 1) {
        ax += __shfl_down_sync(0xffffffffu, ax, o, GP);
        ay += __shfl_down_sync(0xffffffffu, ay, o, GP);
        az += __shfl_down_sync(0xffffffffu, az, o, GP);
      }
      // w of the row, and its terms of gamma = r.u, delta = w.u, rho = r.r
      float g = 0.f, d = 0.f, rr = 0.f;
      if (lane == 0 && item < n_items) {
        if constexpr (GV) {
          if (i >= 0) st_f4(reinterpret_cast<float*>(sl[slot].q + i), ax, ay, az);
        } else {
          L.lw[3 * item] = ax;
          L.lw[3 * item + 1] = ay;
          L.lw[3 * item + 2] = az;
        }
        if (i >= 0 && !st[slot].done) {
          float r[3], u[3];
          if constexpr (GV) {
            const float4 rv = ld_f4_cg(reinterpret_cast<const float*>(sl[slot].z + i));
            const float4 uv = ld_f4_cg(u_ptr(sl[slot].zrec, i));
            r[0] = rv.x, r[1] = rv.y, r[2] = rv.z;
            u[0] = uv.x, u[1] = uv.y, u[2] = uv.z;
          } else {
#pragma unroll
            for (int c = 0; c < 3; ++c) {
              r[c] = L.lr[3 * item + c];
              u[c] = L.lu[3 * item + c];
            }
          }
          g = r[0] * u[0] + r[1] * u[1] + r[2] * u[2];
          d = ax * u[0] + ay * u[1] + az * u[2];
          rr = r[0] * r[0] + r[1] * r[1] + r[2] * r[2];
        }
      }
      // per group of 16 rows (one warp of the pass), in a fixed order
      g = warp_sum(g);
      d = warp_sum(d);
      rr = warp_sum(rr);
      if (lane32 == 0) {
        float* o = L.lws + NQ * ((base >> 4) + warp);
        o[0] = g;
        o[1] = d;
        o[2] = rr;
      }
    }
    __syncthreads();
  };

  // tile sums of gamma = r.u, delta = w.u, rho = r.r (and failed blocks) from the SpMV's
  // 16-row group sums (8 groups per tile, a fixed tree), posted
  auto post_partials = [&](unsigned stamp, bool with_fail) {
    for (int lt = tid; lt < ntl; lt += NTP) {
      if (st[L.ltt[lt].scene].done) continue;
      const float* w = L.lws + NQ * 8 * lt;
      const int nq = with_fail ? NQ : 3;
      for (int q = 0; q < nq; ++q) {
        const float a = (w[q] + w[NQ + q]) + (w[2 * NQ + q] + w[3 * NQ + q]);
        const float b = (w[4 * NQ + q] + w[5 * NQ + q]) + (w[6 * NQ + q] + w[7 * NQ + q]);
        post_tile(lt, q, a + b, stamp);
      }
    }
  };
  auto fail_out = [&]() {
    if (tid == 0) atomicExch(&bar->timeout, 1);
  };

  // ---------------- set-up: P = block-Jacobi inverse, x = 0, r = b, u = P r
  for (int base = 0; base < n_items; base += NTP) {
    const int item = base + tid;
    float fail = 0.0f;
    int slot = 0;
    const int i = item < n_items ? row_of(item, slot) : -1;
    if (i >= 0) {
      const SceneLite<float>& S = sl[slot];
      float D[9];
      if constexpr (RES) {
        const int bd = L.lrp[item] + (S.diag_idx[i] - S.row_ptr[i]);
#pragma unroll
        for (int c = 0; c < 9; ++c) D[c] = L.lval[9 * bd + c];
      } else {
#pragma unroll
        for (int c = 0; c < 9; ++c) D[c] = S.val[(size_t)c * S.nnzb + S.diag_idx[i]];
      }
      float Pm[9];
      const bool ok = spd_inv3(D, Pm);
      float* P = S.Pinv + (size_t)9 * i;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        P[c] = Pm[c];
        if constexpr (!GV) L.lP[9 * item + c] = Pm[c];
      }
      float r0, r1, r2;
      if (b_from_g) {
        const double4 g = ld_d4(S.g + i);
        r0 = (float)(-g.x);
        r1 = (float)(-g.y);
        r2 = (float)(-g.z);
      } else {
        const float4 rv = ld_f4_cg(reinterpret_cast<const float*>(S.r + i));
        r0 = rv.x;
        r1 = rv.y;
        r2 = rv.z;
      }
      const float u0 = Pm[0] * r0 + Pm[1] * r1 + Pm[2] * r2;
      const float u1 = Pm[3] * r0 + Pm[4] * r1 + Pm[5] * r2;
      const float u2 = Pm[6] * r0 + Pm[7] * r1 + Pm[8] * r2;
      st_f4(u_ptr(S.zrec, i), u0, u1, u2);
      if constexpr (GV) {
        st_f4(reinterpret_cast<float*>(S.z + i), r0, r1, r2);
        st_f4(reinterpret_cast<float*>(S.dx + i), 0.f, 0.f, 0.f);
        st_f4(reinterpret_cast<float*>(S.d0 + i), 0.f, 0.f, 0.f);
        st_f4(reinterpret_cast<float*>(S.d1 + i), 0.f, 0.f, 0.f);
      } else {
        const int k = 3 * item;
        L.lr[k] = r0, L.lr[k + 1] = r1, L.lr[k + 2] = r2;
        L.lu[k] = u0, L.lu[k + 1] = u1, L.lu[k + 2] = u2;
#pragma unroll
        for (int c = 0; c < 3; ++c) L.lx[k + c] = L.lp[k + c] = L.ls[k + c] = 0.0f;
      }
      fail = ok ? 0.0f : 1.0f;
    }
    fail = warp_sum(fail);  // the warp's 32 rows: its first 16-row group takes the count
    if (lane32 == 0) {
      L.lws[NQ * ((base >> 4) + 2 * warp) + 3] = fail;
      L.lws[NQ * ((base >> 4) + 2 * warp + 1) + 3] = 0.0f;
    }
  }

  for (int it = 0;; ++it) {
    // ---- u released to the neighbours (set-up wrote u_0; later iterations below)
    publish_flag((unsigned long long)it + 1);
    if (!wait_flags((unsigned long long)it + 1)) return fail_out();
    spmv();  // w = A u
    const unsigned s = W::stamp((unsigned)it + 1);
    post_partials(s, it == 0);
    if (!reduce(it == 0 ? NQ : 3, s)) return fail_out();
    // one thread per scene (n_scenes <= PCG_MAX_SCENES < NTP); the barrier also finds whether all are done
    int done = 1;
    if (tid < n_scenes) {
      if (!st[tid].done)
        sr_step(st[tid], s_sum[tid][0], s_sum[tid][1], s_sum[tid][2], it == 0 ? s_sum[tid][3] : 0.0f, it,
                sl[tid].tol2, sl[tid].max_iter);
      done = st[tid].done;
    }
    if (__syncthreads_and(done)) break;
    // ---- p = u + beta p, s = w + beta s; x += alpha p, r -= alpha s, u = M r (published)
    for (int item = tid; item < n_items; item += NTP) {
      int slot;
      const int i = row_of(item, slot);
      if (i < 0 || st[slot].done) continue;
      const float a = st[slot].alpha, b = st[slot].beta;
      const SceneLite<float>& S = sl[slot];
      float r[3], P[9];
      if constexpr (GV) {
        const float4 uv = ld_f4_cg(u_ptr(S.zrec, i));
        const float4 pv = ld_f4_cg(reinterpret_cast<const float*>(S.d0 + i));
        const float4 wv = ld_f4_cg(reinterpret_cast<const float*>(S.q + i));
        const float4 sv = ld_f4_cg(reinterpret_cast<const float*>(S.d1 + i));
        const float4 xv = ld_f4_cg(reinterpret_cast<const float*>(S.dx + i));
        const float4 rv = ld_f4_cg(reinterpret_cast<const float*>(S.z + i));
        const float p0 = uv.x + b * pv.x, p1 = uv.y + b * pv.y, p2 = uv.z + b * pv.z;
        const float s0 = wv.x + b * sv.x, s1 = wv.y + b * sv.y, s2 = wv.z + b * sv.z;
        st_f4(reinterpret_cast<float*>(S.d0 + i), p0, p1, p2);
        st_f4(reinterpret_cast<float*>(S.d1 + i), s0, s1, s2);
        st_f4(reinterpret_cast<float*>(S.dx + i), xv.x + a * p0, xv.y + a * p1, xv.z + a * p2);
        r[0] = rv.x - a * s0;
        r[1] = rv.y - a * s1;
        r[2] = rv.z - a * s2;
        st_f4(reinterpret_cast<float*>(S.z + i), r[0], r[1], r[2]);
#pragma unroll
        for (int c = 0; c < 9; ++c) P[c] = __ldcg(S.Pinv + (size_t)9 * i + c);
      } else {
        const int k = 3 * item;
#pragma unroll
        for (int c = 0; c < 3; ++c) {
          const float p = L.lu[k + c] + b * L.lp[k + c];
          const float sv = L.lw[k + c] + b * L.ls[k + c];
          L.lp[k + c] = p;
          L.ls[k + c] = sv;
          L.lx[k + c] += a * p;
          r[c] = L.lr[k + c] - a * sv;
          L.lr[k + c] = r[c];
        }
#pragma unroll
        for (int c = 0; c < 9; ++c) P[c] = L.lP[9 * item + c];
      }
      const float u0 = P[0] * r[0] + P[1] * r[1] + P[2] * r[2];
      const float u1 = P[3] * r[0] + P[4] * r[1] + P[5] * r[2];
      const float u2 = P[6] * r[0] + P[7] * r[1] + P[8] * r[2];
      if constexpr (!GV) {
        const int k = 3 * item;
        L.lu[k] = u0, L.lu[k + 1] = u1, L.lu[k + 2] = u2;
      }
      st_f4(u_ptr(S.zrec, i), u0, u1, u2);
    }
    for (int si = tid; si < n_scenes; si += NTP)
      if (!st[si].done) st[si].iters += 1;
    // (the barrier of the next publish_flag orders these updates)
  }

  // x of this CTA's rows to global memory (SR_GLOBAL: already there); CTA 0 publishes the scalars
  if constexpr (!GV) {
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

static const void* sr_kernel(int mode) {
  return mode == SR_RES ? (const void*)k_pcg_sr<SR_RES>
                        : mode == SR_STREAM ? (const void*)k_pcg_sr<SR_STREAM> : (const void*)k_pcg_sr<SR_GLOBAL>;
}

int pcg_sr_max_grid(int device, size_t smem, int mode) {
  const void* k = sr_kernel(mode);
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
  if (L.n_scenes <= 0 || L.n_scenes > PCG_MAX_SCENES || L.n_tiles <= 0 || L.grid > XCH_MAX_CTAS || !L.flags ||
      L.sr_mode < SR_RES || L.sr_mode > SR_GLOBAL || (L.sr_mode == SR_RES) != (L.smem_blocks > 0))
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
  const TileRef* tiles = L.tiles;
  int n_tiles = L.n_tiles;
  const int* ids = L.scene_ids;
  int n_scenes = L.n_scenes;
  GridBar* bar = L.bar;
  int bg = L.use_b_from_g;
  int nb_cap = L.smem_blocks;
  unsigned long long* flags = L.flags;
  void* args[] = {(void*)&scenes, (void*)&tiles, (void*)&n_tiles, (void*)&ids,  (void*)&n_scenes,
                  (void*)&bar,    (void*)&bg,    (void*)&nb_cap,  (void*)&flags};
  const void* k = sr_kernel(L.sr_mode);
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(k, dim3(L.grid), dim3(NTP), args, L.smem_bytes, st);
}

}  // namespace ppn
