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
#include "pcg_common.cuh"

namespace ppn {

using namespace pcgdev;


template <typename T, int G>
__global__ void __launch_bounds__(NT, 1)
    k_pcg(const SceneDev<T>* scenes, const TileRef* tiles, int n_tiles, const int* scene_ids,
          int n_scenes, GridBar* bar, int b_from_g) {
  using V4 = vec4_t<T>;
  constexpr int RPP = NT / G;  // rows per SpMV pass
  __shared__ double sm[NT / 32];
  __shared__ double rowv[RPP];
  __shared__ SState<double> st[PCG_MAX_SCENES];
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
        T Pm[9];
        const bool ok = spd_inv3(D, Pm);
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
    if ((tid & 31) == 0) init_state(st[si], rz, r2, f);
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
          const SState<double>& s = st[slot];
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
        const SState<double>& s = st[slot];
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
      if ((tid & 31) == 0) after_dq(st[si], dq);
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
        const SState<double>& s = st[tr.scene];
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
      if ((tid & 31) == 0) after_rz(st[si], rz, r2, S.pcg_tol2, S.pcg_max_iter);
    }
    __syncthreads();
  }

  // every CTA holds the same final state; CTA 0 publishes it
  if (blockIdx.x == 0) {
    for (int si = tid; si < n_scenes; si += NT) publish(st[si], scenes[scene_ids[si]].ctl);
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
