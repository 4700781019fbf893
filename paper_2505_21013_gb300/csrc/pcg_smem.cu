// Shared-memory-resident variant of the cooperative block-Jacobi PCG
// (SolveSPD of Algorithm 1; Sec. 4.1 "Linear Solvers", Sec. 5.1).
//
// Same iteration, scalars and reductions as the global-memory kernel in
// pcg.cu; the difference is where data lives and how CTAs exchange scalars.
//
// Data.  When the BSR rows of a CTA's contiguous tile range fit in shared
// memory, the setup copies them there once per solve (column indices and 3x3
// blocks, row-major per block) with the block-Jacobi inverse, each row's scene
// slot and index, and the per-scene descriptors; the rows' x, r, q, z and d
// vectors stay in shared memory for the whole solve.  Global memory carries
// only what other CTAs need: z and the double-buffered d of every row
// (gathered by neighbouring rows).  Phase A covers RPP rows per pass with G
// lanes per row and issues all neighbour gathers of a lane before using any.
//
// Exchange.  Each tile partial of a reduction crosses the grid as stamped
// 64-bit words (one word for an FP32 partial, hi and lo words for an FP64
// one).  Aligned 64-bit accesses are single-copy atomic, so a word with the
// expected stamp carries that phase's value; no fence is needed between a
// value and its flag.  Per phase: each CTA stores its vector values, then its
// tile partials as stamped words ([quantity][tile] layout per scene); a fence
// before the partials of phase B (and of the set-up) releases the z and d
// values that the next phase A gathers.  Every CTA reads all tile words it
// needs (one warp per scene and quantity, all pending words re-polled together
// each round), sums them in tile order, which gives the same bits in every
// CTA, and applies the same scalar update.  All waits are bounded.
//
// Precision.  The reductions and CG scalars use the vector type T: FP32 in the
// mixed path (FP64 issues at a small fraction of the FP32 rate on this part),
// FP64 in the FP64 path.
#include "pcg_common.cuh"

namespace ppn {

using namespace pcgdev;

namespace {

template <typename T>
struct SmemLayout {
  T* lws;        // [ntl * 16 * 3] per-warp partial sums, summed per tile in fixed order
  int* it_i;     // [ni] row index within its scene (-1: padding row)
  int* it_slot;  // [ni] scene slot
  int* lrp;      // [ni + 1] local row pointers into the block arrays
  int* lcol;     // [nb] global column index
  T* lval;       // [nb * 9] 3x3 blocks, row-major
  T* lP;         // [ni * 9] block-Jacobi inverse
  T* lx;         // [ni * 3]
  T* lr;
  T* lq;
  T* lz;
  T* ld;         // own direction (in place; neighbours read the global copies)
};

__host__ __device__ inline size_t rup16(size_t b) { return (b + 15) & ~size_t(15); }

template <typename T>
__device__ __forceinline__ SmemLayout<T> carve(char* base, int ni, int nb) {
  SmemLayout<T> L;
  const int ntl = ni / PCG_TILE + 1;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    char* p = base + off;
    off += rup16(bytes);
    return p;
  };
  L.lws = (T*)take(sizeof(double) * ntl * 16 * 3);
  L.it_i = (int*)take(sizeof(int) * ni);
  L.it_slot = (int*)take(sizeof(int) * ni);
  L.lrp = (int*)take(sizeof(int) * (ni + 1));
  L.lcol = (int*)take(sizeof(int) * nb);
  L.lval = (T*)take(sizeof(T) * 9 * nb);
  L.lP = (T*)take(sizeof(T) * 9 * ni);
  L.lx = (T*)take(sizeof(T) * 3 * ni);
  L.lr = (T*)take(sizeof(T) * 3 * ni);
  L.lq = (T*)take(sizeof(T) * 3 * ni);
  L.lz = (T*)take(sizeof(T) * 3 * ni);
  L.ld = (T*)take(sizeof(T) * 3 * ni);
  return L;
}


}  // namespace

size_t pcg_smem_bytes(int ni, int nb, int fsize) {
  const size_t ntl = ni / PCG_TILE + 1;
  return rup16(sizeof(double) * ntl * 16 * 3) + 2 * rup16(sizeof(int) * ni) + rup16(sizeof(int) * (ni + 1)) +
         rup16(sizeof(int) * nb) + rup16((size_t)fsize * 9 * nb) + rup16((size_t)fsize * 9 * ni) +
         5 * rup16((size_t)fsize * 3 * ni);
}

constexpr int NTS = 512;  // threads per CTA of the resident kernel (128-register budget)
constexpr int MAXQ = 3;   // quantities exchanged per phase (setup: r.z, r.r, failed blocks)

template <typename T, int G>
__global__ void __launch_bounds__(NTS, 1)
    k_pcg_s(const SceneDev<T>* scenes, const TileRef* tiles, int n_tiles, const int* scene_ids,
            int n_scenes, GridBar* bar, int b_from_g, int nb_cap) {
  using V4 = vec4_t<T>;
  constexpr int RPP = NTS / G;            // rows per SpMV pass
  constexpr int U = 16 / G;               // blocks per lane per gather round
  constexpr int NW = NTS / 32;            // warps
  constexpr int TPP = RPP / PCG_TILE;     // tiles per SpMV pass
  constexpr int WPT = NW / TPP;           // warps per tile in an SpMV pass
  static_assert(RPP % PCG_TILE == 0, "an SpMV pass covers whole reduction tiles");
  static_assert(NW <= 32, "one warp scans the warp totals");
  using W = Words<T>;
  constexpr bool REC = sizeof(T) == 4;    // FP32: z / d_prev records (one 256-bit gather per block)
  constexpr int NWD = W::N;               // words per exchanged value
  extern __shared__ __align__(16) char dyn[];
  __shared__ SState<T> st[PCG_MAX_SCENES];
  __shared__ SceneLite<T> sl[PCG_MAX_SCENES];
  __shared__ T s_sum[PCG_MAX_SCENES][MAXQ];
  __shared__ int s_to, s_all_done;
  __shared__ int s_scan[NW];

  const int tid = threadIdx.x, warp = tid >> 5, lane32 = tid & 31;
  const int t0 = (int)(((long long)blockIdx.x * n_tiles) / gridDim.x);
  const int t1 = (int)(((long long)(blockIdx.x + 1) * n_tiles) / gridDim.x);
  const int ntl = t1 - t0;
  const int n_items = ntl * PCG_TILE;
  const SmemLayout<T> L = carve<T>(dyn, n_items, nb_cap);
  unsigned epoch = 0;
  if (tid == 0) s_to = 0;

  // ---------------- per-scene descriptors and per-row (slot, index) into shared memory;
  // shared memory is not cleared between launches: the scalar state starts live
  for (int si = tid; si < n_scenes; si += NTS) {
    load_lite(sl[si], scenes[scene_ids[si]]);
    st[si].done = 0;
  }
  __syncthreads();
  for (int item = tid; item < n_items; item += NTS) {
    const TileRef tr = tiles[t0 + item / PCG_TILE];
    const int i = tr.tile * PCG_TILE + (item % PCG_TILE);
    L.it_slot[item] = tr.scene;
    L.it_i[item] = i < sl[tr.scene].nv ? i : -1;
  }
  __syncthreads();

  // ---------------- local row pointers (exclusive scan of row lengths)
  {
    int carry = 0;
    for (int base = 0; base < n_items; base += NTS) {
      const int item = base + tid;
      int len = 0;
      if (item < n_items) {
        const int i = L.it_i[item];
        if (i >= 0) {
          const SceneLite<T>& S = sl[L.it_slot[item]];
          len = S.row_ptr[i + 1] - S.row_ptr[i];
        }
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
  // ---------------- copy this CTA's blocks (warp per row, coalesced over blocks)
  for (int item = warp; item < n_items; item += NW) {
    const int i = L.it_i[item];
    if (i < 0) continue;
    const SceneLite<T>& S = sl[L.it_slot[item]];
    const int kb = S.row_ptr[i], ke = S.row_ptr[i + 1], lb = L.lrp[item];
    const size_t nb = (size_t)S.nnzb;
    for (int k = kb + lane32; k < ke; k += 32) {
      const int b = lb + (k - kb);
      L.lcol[b] = S.col[k];
#pragma unroll
      for (int c = 0; c < 9; ++c) L.lval[9 * b + c] = S.val[c * nb + k];
    }
  }
  __syncthreads();

  // ---------------- exchange
  // tile partial k of tile t of a scene: pword[(k * n_ptiles + t) * 2 + h]
  auto post_tile = [&](int lt, int k, T v, unsigned s) {
    const TileRef tr = tiles[t0 + lt];
    const SceneLite<T>& S = sl[tr.scene];
    unsigned long long w[NWD];
    W::split(v, s, w);
    unsigned long long* p = S.pword + NWD * ((size_t)k * S.n_ptiles + tr.tile);
#pragma unroll
    for (int j = 0; j < NWD; ++j) st_relaxed_u64(p + j, w[j]);
  };
  // Every CTA sums quantities ks[0..nq) of every scene from the tile words in
  // the same fixed order (so all CTAs hold bitwise-equal scalars), then applies
  // `update` to each live scene.  Tiles of scenes whose solve has ended are
  // still posted and read, so every CTA waits for every other one at every
  // exchange: a word is rewritten two exchanges later, after every CTA has read
  // it.  One warp per (scene, quantity); each
  // lane polls all of its pending words in one round per L2 round trip.
  // `acquire`: the phase that follows gathers vector values of other CTAs.
  auto exchange = [&](const int* ks, int nq, bool acquire, auto&& update) -> bool {
    const unsigned s = W::stamp(epoch);
    for (int x = warp; x < n_scenes * nq; x += NW) {
      const int si = x / nq, q = x % nq;
      const SceneLite<T>& S = sl[si];
      const int n = S.n_ptiles;
      const unsigned long long* base = S.pword + NWD * (size_t)ks[q] * n;
      T acc = (T)0;
      for (int tw = lane32; tw < n; tw += 32 * 8) {
        unsigned long long w[8][NWD];
#pragma unroll
        for (int u = 0; u < 8; ++u) {
          const int t = tw + 32 * u;
#pragma unroll
          for (int j = 0; j < NWD; ++j) w[u][j] = t < n ? ld_relaxed_u64(base + NWD * t + j) : W::filler(s);
        }
        for (unsigned spins = 0;; ++spins) {
          bool ready = true;
#pragma unroll
          for (int u = 0; u < 8; ++u)
#pragma unroll
            for (int j = 0; j < NWD; ++j) ready &= W::has(w[u][j], s);
          if (ready) break;
          if (spins > kWaitSpins || *(volatile int*)&s_to) {
            s_to = 1;
            break;
          }
#pragma unroll
          for (int u = 0; u < 8; ++u) {
            const int t = tw + 32 * u;
#pragma unroll
            for (int j = 0; j < NWD; ++j)
              if (!W::has(w[u][j], s)) w[u][j] = ld_relaxed_u64(base + NWD * t + j);
          }
        }
#pragma unroll
        for (int u = 0; u < 8; ++u)
          if (tw + 32 * u < n) acc += W::join(w[u]);
      }
      acc = warp_sum(acc);
      if (lane32 == 0) s_sum[si][q] = acc;
    }
    // acquire by the warps that observed stamped words (the barrier below
    // orders the rest of the CTA after them): vector values released before
    // the tile partials are visible to this CTA's gathers
    if (acquire && warp < n_scenes * nq) fence_acq_rel();
    __syncthreads();
    if (s_to) {
      if (tid == 0) atomicExch(&bar->timeout, 1);
      return false;
    }
    for (int si = tid; si < n_scenes; si += NTS)
      if (!st[si].done) update(si);
    __syncthreads();
    return true;
  };

  // ---------------- setup: block-Jacobi inverse, r = b, z = P r, d = 0, x = 0
  for (int base = 0; base < n_items; base += NTS) {
    const int item = base + tid;
    T rz = (T)0, r2 = (T)0, fail = (T)0;
    const int i = item < n_items ? L.it_i[item] : -1;
    if (i >= 0) {
      const SceneLite<T>& S = sl[L.it_slot[item]];
      const int bd = L.lrp[item] + (S.diag_idx[i] - S.row_ptr[i]);
      T Pm[9];
      const bool ok = spd_inv3(L.lval + 9 * bd, Pm);
      T* P = S.Pinv + (size_t)9 * i;
#pragma unroll
      for (int c = 0; c < 9; ++c) {
        P[c] = Pm[c];
        L.lP[9 * item + c] = Pm[c];
      }
      V4 r;
      if (b_from_g) {
        const double4 g = ld_d4(S.g + i);
        r = mk<V4, T>((T)(-g.x), (T)(-g.y), (T)(-g.z));
      } else {
        r = ldcg_v(S.r + i);
      }
      const T z0 = Pm[0] * r.x + Pm[1] * r.y + Pm[2] * r.z;
      const T z1 = Pm[3] * r.x + Pm[4] * r.y + Pm[5] * r.z;
      const T z2 = Pm[6] * r.x + Pm[7] * r.y + Pm[8] * r.z;
      if constexpr (REC) {
        float* rp = rec_ptr(S.zrec, S.nv, 0, i);
        st_rec_half(rp, z0, z1, z2);
        st_rec_half(rp + 4, 0.0f, 0.0f, 0.0f);
      } else {
        st_v(S.z + i, mk<V4, T>(z0, z1, z2));
        st_v(S.d1 + i, mk<V4, T>((T)0, (T)0, (T)0));
      }
      T* lr = L.lr + 3 * item;
      T* lz = L.lz + 3 * item;
      T* lx = L.lx + 3 * item;
      T* ld = L.ld + 3 * item;
      lr[0] = r.x;
      lr[1] = r.y;
      lr[2] = r.z;
      lz[0] = z0;
      lz[1] = z1;
      lz[2] = z2;
      lx[0] = lx[1] = lx[2] = (T)0;
      ld[0] = ld[1] = ld[2] = (T)0;
      rz = r.x * z0 + r.y * z1 + r.z * z2;
      r2 = r.x * r.x + r.y * r.y + r.z * r.z;
      fail = ok ? (T)0 : (T)1;
    }
    rz = warp_sum(rz);
    r2 = warp_sum(r2);
    fail = warp_sum(fail);
    if (lane32 == 0) {
      const int w = (base >> 5) + warp;  // 4 warps per tile (thread per row)
      L.lws[3 * w] = rz;
      L.lws[3 * w + 1] = r2;
      L.lws[3 * w + 2] = fail;
    }
  }
  __syncthreads();
  ++epoch;
  for (int lt = tid; lt < ntl; lt += NTS) {
    const T* w = L.lws + 3 * 4 * lt;
    __threadfence();  // release this CTA's z and d stores before the partials
    post_tile(lt, 0, ((w[0] + w[3]) + w[6]) + w[9], W::stamp(epoch));
    post_tile(lt, 1, ((w[1] + w[4]) + w[7]) + w[10], W::stamp(epoch));
    post_tile(lt, 3, ((w[2] + w[5]) + w[8]) + w[11], W::stamp(epoch));
  }
  {
    const int ks[3] = {0, 1, 3};
    if (!exchange(ks, 3, true, [&](int si) { init_state(st[si], s_sum[si][0], s_sum[si][1], s_sum[si][2]); }))
      return;
  }

  for (;;) {
    if (tid == 0) {
      int all = 1;
      for (int si = 0; si < n_scenes; ++si) all &= st[si].done;
      s_all_done = all;
    }
    __syncthreads();
    if (s_all_done) break;

    // ---------------- phase A: q = H d, d = z + beta d_prev on the fly
    for (int base = 0; base < n_items; base += RPP) {
      const int row = tid / G, lane = tid % G;
      const int item = base + row;
      T ax = 0, ay = 0, az = 0;
      bool live = false;
      int slot = 0, i = -1;
      if (item < n_items) {
        i = L.it_i[item];
        slot = L.it_slot[item];
        live = i >= 0 && !st[slot].done;
        if (live) {
          const SceneLite<T>& S = sl[slot];
          const SState<T>& s = st[slot];
          const T beta = s.beta;
          const V4* dprev = (s.iters & 1) ? S.d0 : S.d1;
          const int lb = L.lrp[item], le = L.lrp[item + 1];
          for (int b0 = lb + lane; b0 < le; b0 += G * U) {
            int j[U];
            bool ok[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
              const int b = b0 + G * u;
              ok[u] = b < le;
              j[u] = ok[u] ? L.lcol[b] : 0;
            }
            if constexpr (REC) {
              const float* rb = rec_ptr(S.zrec, S.nv, s.iters & 1, 0);
              float a[U][8];
#pragma unroll
              for (int u = 0; u < U; ++u)
                if (ok[u]) ld_rec(rb + (size_t)8 * j[u], a[u]);
#pragma unroll
              for (int u = 0; u < U; ++u)
                if (ok[u]) {
                  const T* v = L.lval + 9 * (b0 + G * u);
                  const T dj0 = a[u][0] + beta * a[u][4], dj1 = a[u][1] + beta * a[u][5],
                          dj2 = a[u][2] + beta * a[u][6];
                  ax += v[0] * dj0 + v[1] * dj1 + v[2] * dj2;
                  ay += v[3] * dj0 + v[4] * dj1 + v[5] * dj2;
                  az += v[6] * dj0 + v[7] * dj1 + v[8] * dj2;
                }
            } else {
              V4 zj[U], pj[U];
#pragma unroll
              for (int u = 0; u < U; ++u)
                if (ok[u]) {
                  zj[u] = ldcg_v(S.z + j[u]);
                  pj[u] = ldcg_v(dprev + j[u]);
                }
#pragma unroll
              for (int u = 0; u < U; ++u)
                if (ok[u]) {
                  const T* v = L.lval + 9 * (b0 + G * u);
                  const T dj0 = zj[u].x + beta * pj[u].x, dj1 = zj[u].y + beta * pj[u].y,
                          dj2 = zj[u].z + beta * pj[u].z;
                  ax += v[0] * dj0 + v[1] * dj1 + v[2] * dj2;
                  ay += v[3] * dj0 + v[4] * dj1 + v[5] * dj2;
                  az += v[6] * dj0 + v[7] * dj1 + v[8] * dj2;
                }
            }
          }
        }
      }
      // every lane reaches the same shuffles (fixed tree within each G-lane group)
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        ax += __shfl_down_sync(0xffffffffu, ax, o, G);
        ay += __shfl_down_sync(0xffffffffu, ay, o, G);
        az += __shfl_down_sync(0xffffffffu, az, o, G);
      }
      T dq = (T)0;
      if (lane == 0 && live) {
        const SState<T>& s = st[slot];
        const SceneLite<T>& S = sl[slot];
        const T beta = s.beta;
        V4* dcur = (s.iters & 1) ? S.d1 : S.d0;
        T* ld = L.ld + 3 * item;
        const T* lz = L.lz + 3 * item;
        const T d0 = lz[0] + beta * ld[0], d1 = lz[1] + beta * ld[1], d2 = lz[2] + beta * ld[2];
        ld[0] = d0;
        ld[1] = d1;
        ld[2] = d2;
        if constexpr (REC)
          st_rec_half(rec_ptr(S.zrec, S.nv, (s.iters + 1) & 1, i) + 4, d0, d1, d2);
        else
          st_v(dcur + i, mk<V4, T>(d0, d1, d2));
        T* lq = L.lq + 3 * item;
        lq[0] = ax;
        lq[1] = ay;
        lq[2] = az;
        dq = d0 * ax + d1 * ay + d2 * az;
      }
      dq = warp_sum(dq);  // rows of this warp, fixed tree
      if (lane32 == 0) L.lws[3 * ((base / RPP) * NW + warp)] = dq;
    }
    __syncthreads();
    ++epoch;
    for (int lt = tid; lt < ntl; lt += NTS) {
      // tile lt was covered by pass lt / TPP, warps [WPT * (lt % TPP), + WPT)
      const T* w = L.lws + 3 * ((lt / TPP) * NW + WPT * (lt % TPP));
      T s = (T)0;
#pragma unroll
      for (int k = 0; k < WPT; ++k) s += w[3 * k];
      // no release here: phase B reads no other CTA's vectors, and the fence
      // before the phase-B partials also releases this phase's d stores
      post_tile(lt, 2, s, W::stamp(epoch));
    }
    {
      const int ks[1] = {2};
      if (!exchange(ks, 1, false, [&](int si) { after_dq(st[si], s_sum[si][0]); })) return;
    }

    // ---------------- phase B: x += alpha d, r -= alpha q, z = P r (shared memory)
    for (int base = 0; base < n_items; base += NTS) {
      const int item = base + tid;
      T rz = (T)0, r2 = (T)0;
      const int i = item < n_items ? L.it_i[item] : -1;
      const int slot = item < n_items ? L.it_slot[item] : 0;
      if (i >= 0 && !st[slot].done) {
        const SceneLite<T>& S = sl[slot];
        const T alpha = st[slot].alpha;
        T* lx = L.lx + 3 * item;
        T* lr = L.lr + 3 * item;
        const T* ld = L.ld + 3 * item;
        const T* lq = L.lq + 3 * item;
        const T* P = L.lP + 9 * item;
        lx[0] += alpha * ld[0];
        lx[1] += alpha * ld[1];
        lx[2] += alpha * ld[2];
        const T r0 = lr[0] - alpha * lq[0], r1 = lr[1] - alpha * lq[1], rr2 = lr[2] - alpha * lq[2];
        lr[0] = r0;
        lr[1] = r1;
        lr[2] = rr2;
        const T z0 = P[0] * r0 + P[1] * r1 + P[2] * rr2;
        const T z1 = P[3] * r0 + P[4] * r1 + P[5] * rr2;
        const T z2 = P[6] * r0 + P[7] * r1 + P[8] * rr2;
        T* lz = L.lz + 3 * item;
        lz[0] = z0;
        lz[1] = z1;
        lz[2] = z2;
        if constexpr (REC)
          st_rec_half(rec_ptr(S.zrec, S.nv, (st[slot].iters + 1) & 1, i), z0, z1, z2);
        else
          st_v(S.z + i, mk<V4, T>(z0, z1, z2));
        rz = r0 * z0 + r1 * z1 + rr2 * z2;
        r2 = r0 * r0 + r1 * r1 + rr2 * rr2;
      }
      rz = warp_sum(rz);
      r2 = warp_sum(r2);
      if (lane32 == 0) {
        const int w = (base >> 5) + warp;
        L.lws[3 * w] = rz;
        L.lws[3 * w + 1] = r2;
      }
    }
    __syncthreads();
    ++epoch;
    for (int lt = tid; lt < ntl; lt += NTS) {
      const T* w = L.lws + 3 * 4 * lt;
      __threadfence();  // release this CTA's z and d stores before the partials
      post_tile(lt, 0, ((w[0] + w[3]) + w[6]) + w[9], W::stamp(epoch));
      post_tile(lt, 1, ((w[1] + w[4]) + w[7]) + w[10], W::stamp(epoch));
    }
    {
      const int ks[2] = {0, 1};
      if (!exchange(ks, 2, true, [&](int si) {
            after_rz(st[si], s_sum[si][0], s_sum[si][1], sl[si].tol2, sl[si].max_iter);
          }))
        return;
    }
  }

  // x of this CTA's rows to global memory; CTA 0 publishes the scalars
  for (int item = tid; item < n_items; item += NTS) {
    const int i = L.it_i[item];
    if (i < 0) continue;
    const T* lx = L.lx + 3 * item;
    st_v(sl[L.it_slot[item]].dx + i, mk<V4, T>(lx[0], lx[1], lx[2]));
  }
  if (blockIdx.x == 0)
    for (int si = tid; si < n_scenes; si += NTS) publish(st[si], sl[si].ctl);
}

// G = 2 lanes per row: 512 threads cover two 128-row tiles per pass
template <typename T>
static const void* smem_kernel(int) {
  return (const void*)k_pcg_s<T, 2>;
}

int pcg_smem_max_grid(int group, int device, size_t smem, int fsize) {
  const void* k = fsize == 4 ? smem_kernel<float>(group) : smem_kernel<double>(group);
  if (cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return 0;
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, NTS, smem) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return per_sm * prop.multiProcessorCount;
}

template <typename T>
cudaError_t launch_pcg_smem(const SceneDev<T>* scenes, const PcgLaunch& L, cudaStream_t st) {
  if (L.n_scenes <= 0 || L.n_scenes > PCG_MAX_SCENES || L.n_tiles <= 0 || L.grid > XCH_MAX_CTAS)
    return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(L.bar, 0, sizeof(GridBar), st);
  if (e != cudaSuccess) return e;
  // no stamp of an earlier launch may survive in the exchange words
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
  void* args[] = {(void*)&scenes, (void*)&tiles, (void*)&n_tiles, (void*)&ids, (void*)&n_scenes,
                  (void*)&bar, (void*)&bg, (void*)&nb_cap};
  const void* k = smem_kernel<T>(L.group);
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(k, dim3(L.grid), dim3(NTS), args, L.smem_bytes, st);
}

template cudaError_t launch_pcg_smem<float>(const SceneDev<float>*, const PcgLaunch&, cudaStream_t);
template cudaError_t launch_pcg_smem<double>(const SceneDev<double>*, const PcgLaunch&, cudaStream_t);

}  // namespace ppn
