// Shared-memory-resident variant of the cooperative block-Jacobi PCG
// (SolveSPD of Algorithm 1; Sec. 4.1 "Linear Solvers", Sec. 5.1).
//
// Same iteration, scalars and reductions as the global-memory kernel in
// pcg.cu; the difference is where the data of a CTA's rows lives.  When the
// BSR rows of a CTA's contiguous tile range fit in shared memory, the setup
// copies them there once per solve (column indices and 3x3 blocks, row-major
// per block), together with the block-Jacobi inverse, each row's scene slot
// and index, and the per-scene descriptors; the CTA then keeps its rows' x, r,
// q, z and d vectors in shared memory for the whole solve.  Global memory only
// carries what other CTAs need: z and the double-buffered d of every row
// (gathered by neighbouring rows), the reduction partials and the final x.
// Phase A issues all neighbour gathers of a lane before using any (up to U
// blocks per lane per round).  There is no separate grid barrier: each tile
// publishes its partials as stamped 64-bit words after a release fence, and a
// CTA proceeds once it has read every tile's partial of the current phase,
// which both completes the reduction and guarantees that every vector value
// written before those partials is visible.  A CG iteration thus costs about
// one L2 round trip for the gathers and one for each of the two reductions.
#include "pcg_common.cuh"

namespace ppn {

using namespace pcgdev;

namespace {

template <typename T>
struct SmemLayout {
  double** lpart;  // [ntl] partial record of each local tile
  double* lws;     // [ntl * 16 * 3] per-warp partial sums, summed per tile in fixed order
  int* it_i;       // [ni] row index within its scene (-1: padding row)
  int* it_slot;    // [ni] scene slot
  int* lrp;        // [ni + 1] local row pointers into the block arrays
  int* lcol;       // [nb] global column index
  T* lval;         // [nb * 9] 3x3 blocks, row-major
  T* lP;           // [ni * 9] block-Jacobi inverse
  T* lx;           // [ni * 3]
  T* lr;
  T* lq;
  T* lz;
  T* ld;           // own direction (in place; neighbours read the global copies)
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
  L.lpart = (double**)take(sizeof(double*) * ntl);
  L.lws = (double*)take(sizeof(double) * ntl * 16 * 3);
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

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

}  // namespace

size_t pcg_smem_bytes(int ni, int nb, int fsize) {
  const size_t ntl = ni / PCG_TILE + 1;
  return rup16(sizeof(double*) * ntl) + rup16(sizeof(double) * ntl * 16 * 3) + 2 * rup16(sizeof(int) * ni) +
         rup16(sizeof(int) * (ni + 1)) + rup16(sizeof(int) * nb) + rup16((size_t)fsize * 9 * nb) +
         rup16((size_t)fsize * 9 * ni) + 5 * rup16((size_t)fsize * 3 * ni);
}

constexpr int NTS = 512;  // threads per CTA of the resident kernel (128-register budget, no spills)

template <typename T, int G>
__global__ void __launch_bounds__(NTS, 1)
    k_pcg_s(const SceneDev<T>* scenes, const TileRef* tiles, int n_tiles, const int* scene_ids,
            int n_scenes, GridBar* bar, int b_from_g, int nb_cap, char* xch, unsigned launch_seq) {
  using V4 = vec4_t<T>;
  constexpr int RPP = NTS / G;  // rows per SpMV pass
  constexpr int U = 4;          // blocks per lane per gather round
  constexpr int NW = NTS / 32;  // warps
  static_assert(RPP == PCG_TILE, "one SpMV pass covers exactly one reduction tile");
  static_assert(NW <= 32, "one warp scans the warp totals");
  extern __shared__ __align__(16) char dyn[];
  __shared__ SState st[PCG_MAX_SCENES];
  __shared__ SceneLite<T> sl[PCG_MAX_SCENES];
  __shared__ int s_to, s_all_done;
  __shared__ unsigned long long s_word[SSTATE_WORDS];
  __shared__ int s_scan[NW];

  const int tid = threadIdx.x, warp = tid >> 5, lane32 = tid & 31;
  const int t0 = (int)(((long long)blockIdx.x * n_tiles) / gridDim.x);
  const int t1 = (int)(((long long)(blockIdx.x + 1) * n_tiles) / gridDim.x);
  const int ntl = t1 - t0;
  const int n_items = ntl * PCG_TILE;
  const SmemLayout<T> L = carve<T>(dyn, n_items, nb_cap);
  unsigned epoch = 0;
  if (tid == 0) s_to = 0;

  // ---------------- per-scene descriptors and per-row (slot, index) into shared memory
  for (int si = tid; si < n_scenes; si += NTS) load_lite(sl[si], scenes[scene_ids[si]]);
  __syncthreads();
  for (int item = tid; item < n_items; item += NTS) {
    const TileRef tr = tiles[t0 + item / PCG_TILE];
    const int i = tr.tile * PCG_TILE + (item % PCG_TILE);
    L.it_slot[item] = tr.scene;
    L.it_i[item] = i < sl[tr.scene].nv ? i : -1;
  }
  for (int lt = tid; lt < ntl; lt += NTS) {
    const TileRef tr = tiles[t0 + lt];
    L.lpart[lt] = sl[tr.scene].ppart + 4 * tr.tile;
  }
  __shared__ int s_tb[PCG_MAX_SCENES + 1];  // first launch tile of each slot
  if (tid == 0) {
    int acc = 0;
    for (int si = 0; si < n_scenes; ++si) {
      s_tb[si] = acc;
      acc += sl[si].n_ptiles;
    }
    s_tb[n_scenes] = acc;
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

  // Exchange point (no hot line).  Every CTA posts its tiles' partials and a
  // stamp in its own record; CTA 0 waits for all records, sums each scene's
  // tile partials in tile order, updates the scalars with `update`, and
  // writes a stamped mailbox per CTA (single scene: scalars inline); every
  // other CTA polls only its own mailbox.  All waits are bounded.
  const unsigned long long seq = (unsigned long long)launch_seq << 32;
  auto rec_stamp = [&](int c) { return reinterpret_cast<unsigned long long*>(xch + (size_t)c * XCH_REC_BYTES); };
  char* const boxes = xch + (size_t)XCH_MAX_CTAS * XCH_REC_BYTES;
  auto box_word = [&](int c, int w) {  // w = 0: stamp, 1..9: state words
    return reinterpret_cast<unsigned long long*>(boxes + (size_t)c * XCH_BOX_BYTES + 8 * w);
  };
  unsigned long long* const bcw =
      reinterpret_cast<unsigned long long*>(xch + (size_t)XCH_MAX_CTAS * (XCH_REC_BYTES + XCH_BOX_BYTES));
  auto exchange = [&](auto&& update) -> bool {
    const unsigned long long S = seq | epoch;
    __syncthreads();  // this CTA's record partials are written
    if (tid == 0) {
      __threadfence();
      st_relaxed_u64(rec_stamp(blockIdx.x), S);
    }
    if (blockIdx.x == 0) {
      for (int c = tid; c < (int)gridDim.x; c += NTS) {
        unsigned spins = 0;
        while (ld_relaxed_u64(rec_stamp(c)) != S) {
          if (++spins > kSpinLimit) {
            s_to = 1;
            break;
          }
        }
      }
      fence_acq_rel();
      __syncthreads();
      if (!s_to) {
        for (int si = warp; si < n_scenes; si += NW) update(si);
        __syncthreads();
        if (n_scenes > 1) {
          for (int w = tid; w < n_scenes * SSTATE_WORDS; w += NTS)
            st_relaxed_u64(bcw + w, sword(st[w / SSTATE_WORDS], w % SSTATE_WORDS));
          __syncthreads();
        }
        for (int c = tid; c < (int)gridDim.x; c += NTS) {
          if (n_scenes == 1)
            for (int w = 0; w < SSTATE_WORDS; ++w) st_relaxed_u64(box_word(c, 1 + w), sword(st[0], w));
          __threadfence();
          st_relaxed_u64(box_word(c, 0), S);
        }
      }
    } else {
      if (tid == 0) {
        unsigned spins = 0;
        while (ld_relaxed_u64(box_word(blockIdx.x, 0)) != S) {
          if (++spins > kSpinLimit) {
            s_to = 1;
            break;
          }
        }
        fence_acq_rel();
      }
      __syncthreads();
      if (!s_to) {
        if (n_scenes == 1) {
          if (tid < SSTATE_WORDS) {
            const unsigned long long v = ld_relaxed_u64(box_word(blockIdx.x, 1 + tid));
            s_word[tid] = v;
          }
          __syncthreads();
          if (tid == 0)
            for (int w = 0; w < SSTATE_WORDS; ++w) set_sword(st[0], w, s_word[w]);
        } else {
          for (int si = tid; si < n_scenes; si += NTS)
            for (int w = 0; w < SSTATE_WORDS; ++w) set_sword(st[si], w, ld_relaxed_u64(bcw + si * SSTATE_WORDS + w));
        }
      }
    }
    __syncthreads();
    if (s_to && tid == 0) atomicExch(&bar->timeout, 1);
    return s_to == 0;
  };
  // fixed-order sum of slot k over a scene's tiles (one warp; valid in lane 0)
  auto scene_sum = [&](int si, int k) {
    const double* part = sl[si].ppart;
    const int n = sl[si].n_ptiles;
    double v = 0.0;
#pragma unroll 4
    for (int t = lane32; t < n; t += 32) v += __ldcg(part + 4 * t + k);
    return warp_sum(v);
  };

  // ---------------- setup: block-Jacobi inverse, r = b, z = P r, d = 0, x = 0
  for (int base = 0; base < n_items; base += NTS) {
    const int item = base + tid;
    double rz = 0.0, r2 = 0.0, fail = 0.0;
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
      st_v(S.z + i, mk<V4, T>(z0, z1, z2));
      st_v(S.d1 + i, mk<V4, T>((T)0, (T)0, (T)0));
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
      rz = (double)(r.x * z0 + r.y * z1 + r.z * z2);
      r2 = (double)(r.x * r.x + r.y * r.y + r.z * r.z);
      fail = ok ? 0.0 : 1.0;
    }
    rz = warp_sum(rz);
    r2 = warp_sum(r2);
    fail = warp_sum(fail);
    if (lane32 == 0) {
      const int w = (base >> 5) + warp;  // 4 warps per tile
      L.lws[3 * w] = rz;
      L.lws[3 * w + 1] = r2;
      L.lws[3 * w + 2] = fail;
    }
  }
  __syncthreads();
  for (int lt = tid; lt < ntl; lt += NTS) {
    const double* w = L.lws + 3 * 4 * lt;
    double* p = L.lpart[lt];
    p[0] = ((w[0] + w[3]) + w[6]) + w[9];
    p[1] = ((w[1] + w[4]) + w[7]) + w[10];
    p[3] = ((w[2] + w[5]) + w[8]) + w[11];
  }
  ++epoch;
  if (!exchange([&](int si) {
        const double rz = scene_sum(si, 0), r2 = scene_sum(si, 1), f = scene_sum(si, 3);
        if (lane32 == 0) init_state(st[si], rz, r2, f);
      }))
    return;

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
          const SState& s = st[slot];
          const T beta = (T)s.beta;
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
      // every lane reaches the same shuffles (fixed tree within each G-lane group)
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        ax += __shfl_down_sync(0xffffffffu, ax, o, G);
        ay += __shfl_down_sync(0xffffffffu, ay, o, G);
        az += __shfl_down_sync(0xffffffffu, az, o, G);
      }
      double dq = 0.0;
      if (lane == 0 && live) {
        const SState& s = st[slot];
        const SceneLite<T>& S = sl[slot];
        const T beta = (T)s.beta;
        V4* dcur = (s.iters & 1) ? S.d1 : S.d0;
        T* ld = L.ld + 3 * item;
        const T* lz = L.lz + 3 * item;
        const T d0 = lz[0] + beta * ld[0], d1 = lz[1] + beta * ld[1], d2 = lz[2] + beta * ld[2];
        ld[0] = d0;
        ld[1] = d1;
        ld[2] = d2;
        st_v(dcur + i, mk<V4, T>(d0, d1, d2));
        T* lq = L.lq + 3 * item;
        lq[0] = ax;
        lq[1] = ay;
        lq[2] = az;
        dq = (double)(d0 * ax + d1 * ay + d2 * az);
      }
      dq = warp_sum(dq);  // rows of this warp, fixed tree
      if (lane32 == 0) L.lws[3 * ((base / RPP) * NW + warp)] = dq;
    }
    __syncthreads();
    for (int lt = tid; lt < ntl; lt += NTS) {
      if (st[L.it_slot[lt * PCG_TILE]].done) continue;
      const double* w = L.lws + 3 * NW * lt;
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < NW; ++k) s += w[3 * k];
      L.lpart[lt][2] = s;
    }
    ++epoch;
    if (!exchange([&](int si) {
          if (st[si].done) return;
          const double dq = scene_sum(si, 2);
          if (lane32 == 0) after_dq(st[si], dq);
        }))
      return;

    // ---------------- phase B: x += alpha d, r -= alpha q, z = P r (shared memory)
    for (int base = 0; base < n_items; base += NTS) {
      const int item = base + tid;
      double rz = 0.0, r2 = 0.0;
      const int i = item < n_items ? L.it_i[item] : -1;
      const int slot = item < n_items ? L.it_slot[item] : 0;
      if (i >= 0 && !st[slot].done) {
        const SceneLite<T>& S = sl[slot];
        const T alpha = (T)st[slot].alpha;
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
        st_v(S.z + i, mk<V4, T>(z0, z1, z2));
        rz = (double)(r0 * z0 + r1 * z1 + rr2 * z2);
        r2 = (double)(r0 * r0 + r1 * r1 + rr2 * rr2);
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
    for (int lt = tid; lt < ntl; lt += NTS) {
      if (st[L.it_slot[lt * PCG_TILE]].done) continue;
      const double* w = L.lws + 3 * 4 * lt;
      double* p = L.lpart[lt];
      p[0] = ((w[0] + w[3]) + w[6]) + w[9];
      p[1] = ((w[1] + w[4]) + w[7]) + w[10];
    }
    ++epoch;
    if (!exchange([&](int si) {
          if (st[si].done) return;
          const double rz = scene_sum(si, 0), r2 = scene_sum(si, 1);
          if (lane32 == 0) after_rz(st[si], rz, r2, sl[si].tol2, sl[si].max_iter);
        }))
      return;
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

// rows are split over G = 4 lanes (512 threads cover one 128-row tile per pass)
template <typename T>
static const void* smem_kernel(int) {
  return (const void*)k_pcg_s<T, 4>;
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
  if (L.n_scenes <= 0 || L.n_scenes > PCG_MAX_SCENES || L.n_tiles <= 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(L.bar, 0, sizeof(GridBar), st);
  if (e != cudaSuccess) return e;
  const TileRef* tiles = L.tiles;
  int n_tiles = L.n_tiles;
  const int* ids = L.scene_ids;
  int n_scenes = L.n_scenes;
  GridBar* bar = L.bar;
  int bg = L.use_b_from_g;
  int nb_cap = L.smem_blocks;
  char* xch = reinterpret_cast<char*>(L.bcast);
  unsigned seq = L.launch_seq;
  if (L.grid > XCH_MAX_CTAS) return cudaErrorInvalidValue;
  void* args[] = {(void*)&scenes, (void*)&tiles, (void*)&n_tiles, (void*)&ids, (void*)&n_scenes,
                  (void*)&bar, (void*)&bg, (void*)&nb_cap, (void*)&xch, (void*)&seq};
  const void* k = smem_kernel<T>(L.group);
  e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)L.smem_bytes);
  if (e != cudaSuccess) return e;
  return cudaLaunchCooperativeKernel(k, dim3(L.grid), dim3(NTS), args, L.smem_bytes, st);
}

template cudaError_t launch_pcg_smem<float>(const SceneDev<float>*, const PcgLaunch&, cudaStream_t);
template cudaError_t launch_pcg_smem<double>(const SceneDev<double>*, const PcgLaunch&, cudaStream_t);

}  // namespace ppn
