// Block-Jacobi preconditioned CG with a negative-curvature exit, as one
// persistent cooperative kernel per solve (SolveSPD of Algorithm 1).
//
// Method (Sec. 4.1, "Linear Solvers"; Sec. 5.1): CG from x = 0 on H x = b,
// preconditioned by the inverse 3x3 diagonal blocks; every search direction d
// is checked with d^T H d and the solve stops with ind = true when it is not
// positive, returning the iterate before that direction (the Newton-CG
// iterate); it also stops with ind = true when a diagonal block fails its 3x3
// Cholesky (such a matrix cannot be SPD).  Convergence: ||r|| <= tol ||r0||.
//
// Kernel design.  The launch's PCG_TILE-row tiles (of every scene taking part)
// are split into contiguous ranges, one per CTA.  One CG iteration is two
// phases, each closed by a grid barrier:
//   A: q = H d and d^T q, with d = z + beta d_prev formed on the fly for every
//      gathered neighbour (double-buffered d, so the direction update needs no
//      barrier of its own); G lanes per BSR row, component-major block values;
//   B: x += alpha d, r -= alpha q, z = P r, partial r.z and r.r.
// Each tile writes one partial per quantity (fixed in-tile order).  After a
// barrier every CTA sums each scene's tile partials itself, in tile order, so
// all CTAs reach identical scalars and decisions without further
// communication, and a scene's arithmetic does not depend on the grid size or
// on the other scenes of a batch.  The barrier is one arrival counter that
// only grows within a launch; its waits are bounded and report a timeout.
#include "common.cuh"
#include "kernels.h"

namespace ppn {

namespace {

constexpr unsigned kSpinLimit = 1u << 22;
constexpr int NT = 1024;

__device__ __forceinline__ unsigned ld_relaxed(const unsigned* p) {
  unsigned v;
  asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ float4 ldcg_v(const float4* p) { return __ldcg(p); }
__device__ __forceinline__ double4 ldcg_v(const double4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = __ldcg(q), b = __ldcg(q + 1);
  return make_double4(a.x, a.y, b.x, b.y);
}
__device__ __forceinline__ void st_v(float4* p, float4 v) { *p = v; }
__device__ __forceinline__ void st_v(double4* p, double4 v) { st_d4(p, v); }

template <typename V4, typename T>
__device__ __forceinline__ V4 mk(T x, T y, T z) {
  V4 v;
  v.x = x;
  v.y = y;
  v.z = z;
  v.w = (T)0;
  return v;
}

// Arrive and wait until `target` arrivals (all CTAs of barrier number target/gridDim.x).
__device__ __forceinline__ bool grid_sync(GridBar* bar, unsigned target, int* s_to) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(&bar->count, 1u);
    unsigned spins = 0;
    int to = 0;
    while (ld_relaxed(&bar->count) < target) {
      if (++spins > kSpinLimit) {
        atomicExch(&bar->timeout, 1);
        to = 1;
        break;
      }
    }
    __threadfence();
    *s_to = to;
  }
  __syncthreads();
  return *s_to == 0;
}

// sum of part[4 * t + k] over t in [0, n) by one warp, fixed order; valid in lane 0
__device__ __forceinline__ double warp_tile_sum(const double* part, int n, int k) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
#pragma unroll 4
  for (int t = lane; t < n; t += 32) s += __ldcg(part + 4 * t + k);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  return s;
}

// reduction of one double per thread over aligned groups of PCG_TILE threads
// (4 warps); result valid in the group's first thread
__device__ __forceinline__ double subtile_sum(double v, double* sm) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5;
  if ((threadIdx.x & 31) == 0) sm[w] = v;
  __syncthreads();
  double s = 0.0;
  if ((threadIdx.x & (PCG_TILE - 1)) == 0) {
    const int w0 = threadIdx.x >> 5;
    s = ((sm[w0] + sm[w0 + 1]) + sm[w0 + 2]) + sm[w0 + 3];
  }
  __syncthreads();
  return s;
}

// per-scene solver state, replicated identically in every CTA
struct SState {
  double rz, rr0, rr, alpha, beta, dq;
  int iters, done, ind, pfail, hitmax, nonfinite;
};

}  // namespace

template <typename T, int G>
__global__ void __launch_bounds__(NT, 1)
    k_pcg(const SceneDev<T>* scenes, const TileRef* tiles, int n_tiles, const int* scene_ids,
          int n_scenes, GridBar* bar, int b_from_g) {
  using V4 = vec4_t<T>;
  constexpr int RPP = NT / G;  // rows per SpMV pass
  __shared__ double sm[NT / 32];
  __shared__ double rowv[RPP];
  __shared__ SState st[PCG_MAX_SCENES];
  __shared__ int s_to, s_all_done;

  const int tid = threadIdx.x;
  const int t0 = (int)(((long long)blockIdx.x * n_tiles) / gridDim.x);
  const int t1 = (int)(((long long)(blockIdx.x + 1) * n_tiles) / gridDim.x);
  const int n_items = (t1 - t0) * PCG_TILE;
  unsigned epoch = 0;
  const unsigned grid = gridDim.x;

  // ---------------- setup: block-Jacobi inverse, r = b, z = P r, d_prev = 0, x = 0
  for (int base = 0; base < n_items; base += NT) {
    const int item = base + tid;
    double rz = 0.0, r2 = 0.0, fail = 0.0;
    const int ti = t0 + item / PCG_TILE;
    const bool have = item < n_items;
    TileRef tr{0, 0};
    if (have) tr = tiles[ti];
    if (have) {
      const SceneDev<T>& S = scenes[scene_ids[tr.scene]];
      const int i = tr.tile * PCG_TILE + (item % PCG_TILE);
      if (i < S.nv) {
        T D[9];
        const int kd = S.diag_idx[i];
#pragma unroll
        for (int c = 0; c < 9; ++c) D[c] = S.val[(size_t)c * S.nnzb + kd];
        // Cholesky of the lower triangle, then P = L^-T L^-1
        bool ok = D[0] > (T)0;
        const T l00 = ok ? sqrt(D[0]) : (T)1;
        const T l10 = D[3] / l00, l20 = D[6] / l00;
        const T d11 = D[4] - l10 * l10;
        ok = ok && d11 > (T)0;
        const T l11 = ok ? sqrt(d11) : (T)1;
        const T l21 = (D[7] - l20 * l10) / l11;
        const T d22 = D[8] - l20 * l20 - l21 * l21;
        ok = ok && d22 > (T)0;
        const T l22 = ok ? sqrt(d22) : (T)1;
        const T i00 = (T)1 / l00, i11 = (T)1 / l11, i22 = (T)1 / l22;
        const T i10 = -l10 * i00 * i11;
        const T i21 = -l21 * i11 * i22;
        const T i20 = -(l20 * i00 + l21 * i10) * i22;
        T Pm[9];
        Pm[0] = i00 * i00 + i10 * i10 + i20 * i20;
        Pm[1] = i10 * i11 + i20 * i21;
        Pm[2] = i20 * i22;
        Pm[4] = i11 * i11 + i21 * i21;
        Pm[5] = i21 * i22;
        Pm[8] = i22 * i22;
        Pm[3] = Pm[1];
        Pm[6] = Pm[2];
        Pm[7] = Pm[5];
        T* P = S.Pinv + (size_t)9 * i;
#pragma unroll
        for (int c = 0; c < 9; ++c) P[c] = Pm[c];
        V4 r;
        if (b_from_g) {
          const double4 g = ld_d4(S.g + i);
          r = mk<V4, T>((T)(-g.x), (T)(-g.y), (T)(-g.z));
          st_v(S.r + i, r);
        } else {
          r = ldcg_v(S.r + i);
        }
        const V4 z = mk<V4, T>(Pm[0] * r.x + Pm[1] * r.y + Pm[2] * r.z,
                               Pm[3] * r.x + Pm[4] * r.y + Pm[5] * r.z,
                               Pm[6] * r.x + Pm[7] * r.y + Pm[8] * r.z);
        st_v(S.z + i, z);
        st_v(S.d1 + i, mk<V4, T>((T)0, (T)0, (T)0));
        st_v(S.dx + i, mk<V4, T>((T)0, (T)0, (T)0));
        rz = (double)(r.x * z.x + r.y * z.y + r.z * z.z);
        r2 = (double)(r.x * r.x + r.y * r.y + r.z * r.z);
        fail = ok ? 0.0 : 1.0;
      }
    }
    const double s0 = subtile_sum(rz, sm);
    const double s1 = subtile_sum(r2, sm);
    const double s2 = subtile_sum(fail, sm);
    if ((tid & (PCG_TILE - 1)) == 0 && have) {
      double* p = scenes[scene_ids[tr.scene]].ppart + 4 * tr.tile;
      p[0] = s0;
      p[1] = s1;
      p[3] = s2;
    }
  }
  if (!grid_sync(bar, grid * ++epoch, &s_to)) return;
  for (int si = tid >> 5; si < n_scenes; si += NT / 32) {
    const SceneDev<T>& S = scenes[scene_ids[si]];
    const double rz = warp_tile_sum(S.ppart, S.n_ptiles, 0);
    const double r2 = warp_tile_sum(S.ppart, S.n_ptiles, 1);
    const double f = warp_tile_sum(S.ppart, S.n_ptiles, 3);
    if ((tid & 31) == 0) {
      SState& s = st[si];
      s.rz = rz;
      s.rr0 = r2;
      s.rr = r2;
      s.alpha = 0.0;
      s.beta = 0.0;
      s.dq = 0.0;
      s.iters = 0;
      s.hitmax = 0;
      s.nonfinite = !(r2 == r2) || !(rz == rz);
      s.pfail = f > 0.0;
      s.ind = f > 0.0;
      s.done = (f > 0.0) || !(r2 > 0.0) || s.nonfinite;
    }
  }
  __syncthreads();

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
      int i = 0, slot = 0;
      TileRef tr{0, 0};
      if (item < n_items) {
        tr = tiles[t0 + item / PCG_TILE];
        slot = tr.scene;
        const SceneDev<T>& S = scenes[scene_ids[slot]];
        i = tr.tile * PCG_TILE + (item % PCG_TILE);
        live = !st[slot].done && i < S.nv;
        if (live) {
          const SState& s = st[slot];
          const T beta = (T)s.beta;
          const V4* dprev = (s.iters & 1) ? S.d0 : S.d1;
          const int kb = S.row_ptr[i], ke = S.row_ptr[i + 1];
          const size_t nb = (size_t)S.nnzb;
          for (int k = kb + lane; k < ke; k += G) {
            const int j = __ldg(S.col + k);
            const V4 zj = ldcg_v(S.z + j), pj = ldcg_v(dprev + j);
            const T* v = S.val + k;
            const T v0 = __ldg(v), v1 = __ldg(v + nb), v2 = __ldg(v + 2 * nb), v3 = __ldg(v + 3 * nb),
                    v4 = __ldg(v + 4 * nb), v5 = __ldg(v + 5 * nb), v6 = __ldg(v + 6 * nb),
                    v7 = __ldg(v + 7 * nb), v8 = __ldg(v + 8 * nb);
            const T dj0 = zj.x + beta * pj.x, dj1 = zj.y + beta * pj.y, dj2 = zj.z + beta * pj.z;
            ax += v0 * dj0 + v1 * dj1 + v2 * dj2;
            ay += v3 * dj0 + v4 * dj1 + v5 * dj2;
            az += v6 * dj0 + v7 * dj1 + v8 * dj2;
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
        const SceneDev<T>& S = scenes[scene_ids[slot]];
        const T beta = (T)s.beta;
        const V4* dprev = (s.iters & 1) ? S.d0 : S.d1;
        V4* dcur = (s.iters & 1) ? S.d1 : S.d0;
        const V4 zi = ldcg_v(S.z + i), pi = ldcg_v(dprev + i);
        const V4 di = mk<V4, T>(zi.x + beta * pi.x, zi.y + beta * pi.y, zi.z + beta * pi.z);
        st_v(dcur + i, di);
        st_v(S.q + i, mk<V4, T>(ax, ay, az));
        dq = (double)(di.x * ax + di.y * ay + di.z * az);
      }
      if (lane == 0) rowv[row] = dq;
      __syncthreads();
      const double v = (tid < RPP) ? rowv[tid] : 0.0;
      const double ssum = subtile_sum(v, sm);
      if ((tid & (PCG_TILE - 1)) == 0 && tid < RPP) {
        const int it2 = base + tid;
        if (it2 < n_items) {
          const TileRef tq = tiles[t0 + it2 / PCG_TILE];
          if (!st[tq.scene].done) scenes[scene_ids[tq.scene]].ppart[4 * tq.tile + 2] = ssum;
        }
      }
    }
    if (!grid_sync(bar, grid * ++epoch, &s_to)) return;
    for (int si = tid >> 5; si < n_scenes; si += NT / 32) {
      if (st[si].done) continue;  // warp-uniform
      const SceneDev<T>& S = scenes[scene_ids[si]];
      const double dq = warp_tile_sum(S.ppart, S.n_ptiles, 2);
      if ((tid & 31) == 0) {
        SState& s = st[si];
        s.dq = dq;
        if (!(dq == dq)) {
          s.nonfinite = 1;
          s.done = 1;
        } else if (!(dq > 0.0)) {
          s.ind = 1;
          s.done = 1;
        } else {
          s.alpha = s.rz / dq;
        }
      }
    }
    __syncthreads();

    // ---------------- phase B: x += alpha d, r -= alpha q, z = P r
    for (int base = 0; base < n_items; base += NT) {
      const int item = base + tid;
      double rz = 0.0, r2 = 0.0;
      const bool have = item < n_items;
      TileRef tr{0, 0};
      bool live = false;
      if (have) {
        tr = tiles[t0 + item / PCG_TILE];
        live = !st[tr.scene].done;
      }
      if (live) {
        const SState& s = st[tr.scene];
        const SceneDev<T>& S = scenes[scene_ids[tr.scene]];
        const int i = tr.tile * PCG_TILE + (item % PCG_TILE);
        if (i < S.nv) {
          const T alpha = (T)s.alpha;
          const V4* dcur = (s.iters & 1) ? S.d1 : S.d0;
          const V4 di = ldcg_v(dcur + i), qi = ldcg_v(S.q + i);
          V4 x = ldcg_v(S.dx + i), r = ldcg_v(S.r + i);
          x.x += alpha * di.x;
          x.y += alpha * di.y;
          x.z += alpha * di.z;
          r.x -= alpha * qi.x;
          r.y -= alpha * qi.y;
          r.z -= alpha * qi.z;
          const T* P = S.Pinv + (size_t)9 * i;
          const V4 z = mk<V4, T>(P[0] * r.x + P[1] * r.y + P[2] * r.z, P[3] * r.x + P[4] * r.y + P[5] * r.z,
                                 P[6] * r.x + P[7] * r.y + P[8] * r.z);
          st_v(S.dx + i, x);
          st_v(S.r + i, r);
          st_v(S.z + i, z);
          rz = (double)(r.x * z.x + r.y * z.y + r.z * z.z);
          r2 = (double)(r.x * r.x + r.y * r.y + r.z * r.z);
        }
      }
      const double s0 = subtile_sum(rz, sm);
      const double s1 = subtile_sum(r2, sm);
      if ((tid & (PCG_TILE - 1)) == 0 && live) {
        double* p = scenes[scene_ids[tr.scene]].ppart + 4 * tr.tile;
        p[0] = s0;
        p[1] = s1;
      }
    }
    if (!grid_sync(bar, grid * ++epoch, &s_to)) return;
    for (int si = tid >> 5; si < n_scenes; si += NT / 32) {
      if (st[si].done) continue;
      const SceneDev<T>& S = scenes[scene_ids[si]];
      const double rz = warp_tile_sum(S.ppart, S.n_ptiles, 0);
      const double r2 = warp_tile_sum(S.ppart, S.n_ptiles, 1);
      if ((tid & 31) == 0) {
        SState& s = st[si];
        s.iters += 1;
        s.rr = r2;
        if (!(r2 == r2) || !(rz == rz)) {
          s.nonfinite = 1;
          s.done = 1;
        } else if (r2 <= S.pcg_tol2 * s.rr0) {
          s.done = 1;
        } else if (s.iters >= S.pcg_max_iter) {
          s.hitmax = 1;
          s.done = 1;
        } else {
          s.beta = rz / s.rz;
          s.rz = rz;
        }
      }
    }
    __syncthreads();
  }

  // every CTA holds the same final state; CTA 0 publishes it
  if (blockIdx.x == 0) {
    for (int si = tid; si < n_scenes; si += NT) {
      const SState& s = st[si];
      Ctl* c = scenes[scene_ids[si]].ctl;
      c->pcg_rr0 = s.rr0;
      c->pcg_rr = s.rr;
      c->pcg_rz = s.rz;
      c->pcg_dq = s.dq;
      c->pcg_alpha = s.alpha;
      c->pcg_beta = s.beta;
      c->pcg_iters = s.iters;
      c->pcg_ind = s.ind;
      c->pcg_precond_fail = s.pfail;
      c->pcg_hit_max = s.hitmax;
      c->pcg_done = 1;
      if (s.nonfinite) c->error |= kErrNonFinite;
    }
  }
}

int pcg_max_grid(int group, int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return 0;
  int a = 0, b = 0;
  if (group == 4) {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg<float, 4>, NT, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pcg<double, 4>, NT, 0);
  } else {
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, k_pcg<float, 8>, NT, 0);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_pcg<double, 8>, NT, 0);
  }
  return (a < b ? a : b) * prop.multiProcessorCount;
}

template <typename T>
cudaError_t launch_pcg(const SceneDev<T>* scenes, const PcgLaunch& L, cudaStream_t st) {
  if (L.n_scenes <= 0 || L.n_scenes > PCG_MAX_SCENES || L.n_tiles <= 0) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(L.bar, 0, sizeof(GridBar), st);
  if (e != cudaSuccess) return e;
  const TileRef* tiles = L.tiles;
  int n_tiles = L.n_tiles;
  const int* ids = L.scene_ids;
  int n_scenes = L.n_scenes;
  GridBar* bar = L.bar;
  int bg = L.use_b_from_g;
  void* args[] = {(void*)&scenes, (void*)&tiles, (void*)&n_tiles, (void*)&ids,
                  (void*)&n_scenes, (void*)&bar, (void*)&bg};
  const int grid = L.grid < n_tiles ? L.grid : n_tiles;
  if (L.group == 4)
    return cudaLaunchCooperativeKernel((const void*)k_pcg<T, 4>, dim3(grid), dim3(NT), args, 0, st);
  return cudaLaunchCooperativeKernel((const void*)k_pcg<T, 8>, dim3(grid), dim3(NT), args, 0, st);
}

template cudaError_t launch_pcg<float>(const SceneDev<float>*, const PcgLaunch&, cudaStream_t);
template cudaError_t launch_pcg<double>(const SceneDev<double>*, const PcgLaunch&, cudaStream_t);

}  // namespace ppn
