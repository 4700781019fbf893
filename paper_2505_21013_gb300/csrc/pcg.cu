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
// Kernel design.  The CTAs of one cooperative launch own fixed tiles of
// PCG_TILE rows (tile = blockIdx.x + k * gridDim.x) across all scenes in the
// launch.  One CG iteration is two phases separated by grid barriers:
//   A: q = H d and d^T q with d = z + beta d_prev formed on the fly for every
//      gathered neighbour (double-buffered d, so no extra barrier is needed
//      between the direction update and the SpMV); G lanes per BSR row,
//      component-major block values for coalesced loads;
//   B: x += alpha d, r -= alpha q, z = P r, partial r.z and r.r.
// Each tile writes one partial per quantity; the last CTA to reach a barrier
// sums every scene's partials in tile order (so results do not depend on the
// grid size or on the batch a scene runs in), updates the scene's scalars
// (alpha, beta, convergence, ind) and releases the barrier.  Barrier waits are
// bounded: on timeout the kernel records kErrTimeout and returns.
#include "common.cuh"
#include "kernels.h"

namespace ppn {

namespace {

constexpr unsigned kSpinLimit = 1u << 22;

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
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

// Grid barrier; the last CTA to arrive runs `scalar` (all of its threads)
// before releasing the others.  Returns false after a timeout.
template <typename F>
__device__ __forceinline__ bool grid_barrier(GridBar* bar, F&& scalar) {
  __shared__ int s_last;
  __syncthreads();
  if (threadIdx.x == 0) {
    const unsigned gen = ld_acquire(&bar->gen);
    __threadfence();
    const unsigned arrived = atomicAdd(&bar->count, 1u);
    s_last = (arrived == gridDim.x - 1);
    if (!s_last) {
      unsigned spins = 0;
      while (ld_acquire(&bar->gen) == gen) {
        if (++spins > kSpinLimit) {
          atomicExch(&bar->timeout, 1);
          break;
        }
        __nanosleep(64);
      }
    }
    __threadfence();
  }
  __syncthreads();
  if (s_last) {
    scalar();
    __syncthreads();
    if (threadIdx.x == 0) {
      bar->count = 0u;
      __threadfence();
      atomicAdd(&bar->gen, 1u);
    }
  }
  __syncthreads();
  return __ldcg(&bar->timeout) == 0;
}

// sum of part[4 * t + k] over t in [0, n) by one warp, fixed order; valid in lane 0
__device__ __forceinline__ double warp_tile_sum(const double* part, int n, int k) {
  const int lane = threadIdx.x & 31;
  double s = 0.0;
  for (int t = lane; t < n; t += 32) s += __ldcg(part + 4 * t + k);
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
  return s;
}

// reduction of one double per thread over the 128 rows of a sub-tile (4 warps);
// result valid in the sub-tile's first thread
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

}  // namespace

template <typename T, int G>
__global__ void __launch_bounds__(PCG_TILE * G, 1)
    k_pcg(const SceneDev<T>* scenes, const TileRef* tiles, int n_tiles, const int* scene_ids,
          int n_scenes, GridBar* bar, int b_from_g) {
  using V4 = vec4_t<T>;
  constexpr int NT = PCG_TILE * G;
  __shared__ double sm[NT / 32];
  __shared__ double rowv[PCG_TILE];
  __shared__ int s_notdone;

  const int tid = threadIdx.x;
  const int sub = tid / PCG_TILE;  // sub-tile slot in row-wise phases
  const int rr = tid % PCG_TILE;   // row within the sub-tile

  // ---------------- setup: block-Jacobi inverse, r = b, z = P r, d_prev = 0
  for (int k0 = 0;; k0 += G) {
    const int ti = blockIdx.x + (k0 + sub) * gridDim.x;
    if (blockIdx.x + k0 * gridDim.x >= n_tiles) break;
    double rz = 0.0, r2 = 0.0, fail = 0.0;
    int tile = 0;
    const SceneDev<T>* Sp = nullptr;
    if (ti < n_tiles) {
      const TileRef tr = tiles[ti];
      Sp = &scenes[tr.scene];
      tile = tr.tile;
      const SceneDev<T>& S = *Sp;
      const int i = tile * PCG_TILE + rr;
      if (i < S.nv) {
        T D[9];
        const int kd = S.diag_idx[i];
#pragma unroll
        for (int c = 0; c < 9; ++c) D[c] = S.val[(size_t)c * S.nnzb + kd];
        // Cholesky of the lower triangle, then P = L^-T L^-1
        T Pm[9];
        bool ok = D[0] > (T)0;
        T l00 = ok ? sqrt(D[0]) : (T)1;
        T l10 = D[3] / l00, l20 = D[6] / l00;
        T d11 = D[4] - l10 * l10;
        ok = ok && d11 > (T)0;
        T l11 = ok ? sqrt(d11) : (T)1;
        T l21 = (D[7] - l20 * l10) / l11;
        T d22 = D[8] - l20 * l20 - l21 * l21;
        ok = ok && d22 > (T)0;
        T l22 = ok ? sqrt(d22) : (T)1;
        // L^-1 (lower)
        const T i00 = (T)1 / l00, i11 = (T)1 / l11, i22 = (T)1 / l22;
        const T i10 = -l10 * i00 * i11;
        const T i21 = -l21 * i11 * i22;
        const T i20 = -(l20 * i00 + l21 * i10) * i22;
        // P = Linv^T Linv
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
    if (rr == 0 && ti < n_tiles) {
      double* p = Sp->ppart + 4 * tile;
      p[0] = s0;
      p[1] = s1;
      p[2] = s2;
    }
  }

  auto scalar_setup = [&]() {
    if (tid == 0) s_notdone = 0;
    __syncthreads();
    for (int si = tid >> 5; si < n_scenes; si += NT / 32) {
      const SceneDev<T>& S = scenes[scene_ids[si]];
      const double rz = warp_tile_sum(S.ppart, S.n_ptiles, 0);
      const double r2 = warp_tile_sum(S.ppart, S.n_ptiles, 1);
      const double f = warp_tile_sum(S.ppart, S.n_ptiles, 2);
      if ((tid & 31) == 0) {
        Ctl* c = S.ctl;
        c->pcg_iters = 0;
        c->pcg_hit_max = 0;
        c->pcg_rr0 = r2;
        c->pcg_rr = r2;
        c->pcg_rz = rz;
        c->pcg_beta = 0.0;
        c->pcg_alpha = 0.0;
        c->pcg_dq = 0.0;
        c->pcg_precond_fail = f > 0.0;
        c->pcg_ind = f > 0.0;
        const int done = (f > 0.0) || !(r2 > 0.0);
        c->pcg_done = done;
        if (!done) atomicOr(&s_notdone, 1);
      }
    }
    __syncthreads();
    if (tid == 0) bar->all_done = !s_notdone;
    __threadfence();
  };
  if (!grid_barrier(bar, scalar_setup)) return;

  while (!__ldcg(&bar->all_done)) {
    // ---------------- phase A: q = H d, d = z + beta d_prev on the fly
    for (int ti = blockIdx.x; ti < n_tiles; ti += gridDim.x) {
      const TileRef tr = tiles[ti];
      const SceneDev<T>& S = scenes[tr.scene];
      const Ctl* c = S.ctl;
      if (__ldcg(&c->pcg_done)) continue;  // uniform over the CTA
      const int it = __ldcg(&c->pcg_iters);
      const T beta = (T)__ldcg(&c->pcg_beta);
      const V4* dprev = (it & 1) ? S.d0 : S.d1;
      V4* dcur = (it & 1) ? S.d1 : S.d0;
      const int row = tid / G, lane = tid % G;
      const int i = tr.tile * PCG_TILE + row;
      T ax = 0, ay = 0, az = 0;
      if (i < S.nv) {
        const int kb = S.row_ptr[i], ke = S.row_ptr[i + 1];
        for (int k = kb + lane; k < ke; k += G) {
          const int j = S.col[k];
          const V4 zj = ldcg_v(S.z + j), pj = ldcg_v(dprev + j);
          const T dj0 = zj.x + beta * pj.x, dj1 = zj.y + beta * pj.y, dj2 = zj.z + beta * pj.z;
          const T* v = S.val + k;
          const size_t nb = (size_t)S.nnzb;
          ax += v[0] * dj0 + v[nb] * dj1 + v[2 * nb] * dj2;
          ay += v[3 * nb] * dj0 + v[4 * nb] * dj1 + v[5 * nb] * dj2;
          az += v[6 * nb] * dj0 + v[7 * nb] * dj1 + v[8 * nb] * dj2;
        }
      }
#pragma unroll
      for (int o = G / 2; o > 0; o >>= 1) {
        ax += __shfl_down_sync(0xffffffffu, ax, o, G);
        ay += __shfl_down_sync(0xffffffffu, ay, o, G);
        az += __shfl_down_sync(0xffffffffu, az, o, G);
      }
      if (lane == 0) {
        double dq = 0.0;
        if (i < S.nv) {
          const V4 zi = ldcg_v(S.z + i), pi = ldcg_v(dprev + i);
          const V4 di = mk<V4, T>(zi.x + beta * pi.x, zi.y + beta * pi.y, zi.z + beta * pi.z);
          st_v(dcur + i, di);
          st_v(S.q + i, mk<V4, T>(ax, ay, az));
          dq = (double)(di.x * ax + di.y * ay + di.z * az);
        }
        rowv[row] = dq;
      }
      __syncthreads();
      double v = (tid < PCG_TILE) ? rowv[tid] : 0.0;
      const double s = subtile_sum(v, sm);
      if (tid == 0) S.ppart[4 * tr.tile] = s;
    }

    auto scalar_a = [&]() {
      for (int si = tid >> 5; si < n_scenes; si += NT / 32) {
        const SceneDev<T>& S = scenes[scene_ids[si]];
        Ctl* c = S.ctl;
        if (__ldcg(&c->pcg_done)) continue;
        const double dq = warp_tile_sum(S.ppart, S.n_ptiles, 0);
        if ((tid & 31) == 0) {
          c->pcg_dq = dq;
          if (!(dq > 0.0)) {
            c->pcg_ind = 1;
            c->pcg_done = 1;
          } else {
            c->pcg_alpha = __ldcg(&c->pcg_rz) / dq;
          }
        }
      }
      __threadfence();
    };
    if (!grid_barrier(bar, scalar_a)) return;

    // ---------------- phase B: x += alpha d, r -= alpha q, z = P r
    for (int k0 = 0;; k0 += G) {
      if (blockIdx.x + k0 * gridDim.x >= n_tiles) break;
      const int ti = blockIdx.x + (k0 + sub) * gridDim.x;
      double rz = 0.0, r2 = 0.0;
      int tile = -1;
      const SceneDev<T>* Sp = nullptr;
      if (ti < n_tiles) {
        const TileRef tr = tiles[ti];
        Sp = &scenes[tr.scene];
        const SceneDev<T>& S = *Sp;
        const Ctl* c = S.ctl;
        if (!__ldcg(&c->pcg_done)) {
          tile = tr.tile;
          const int it = __ldcg(&c->pcg_iters);
          const T alpha = (T)__ldcg(&c->pcg_alpha);
          const V4* dcur = (it & 1) ? S.d1 : S.d0;
          const int i = tile * PCG_TILE + rr;
          if (i < S.nv) {
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
      }
      const double s0 = subtile_sum(rz, sm);
      const double s1 = subtile_sum(r2, sm);
      if (rr == 0 && tile >= 0) {
        double* p = Sp->ppart + 4 * tile;
        p[0] = s0;
        p[1] = s1;
      }
    }

    auto scalar_b = [&]() {
      if (tid == 0) s_notdone = 0;
      __syncthreads();
      for (int si = tid >> 5; si < n_scenes; si += NT / 32) {
        const SceneDev<T>& S = scenes[scene_ids[si]];
        Ctl* c = S.ctl;
        if (__ldcg(&c->pcg_done)) continue;
        const double rz = warp_tile_sum(S.ppart, S.n_ptiles, 0);
        const double r2 = warp_tile_sum(S.ppart, S.n_ptiles, 1);
        if ((tid & 31) == 0) {
          const int it = __ldcg(&c->pcg_iters) + 1;
          c->pcg_iters = it;
          c->pcg_rr = r2;
          int done = 0;
          if (!(r2 == r2) || !(rz == rz)) {
            c->error |= kErrNonFinite;
            done = 1;
          } else if (r2 <= S.pcg_tol2 * __ldcg(&c->pcg_rr0)) {
            done = 1;
          } else if (it >= S.pcg_max_iter) {
            c->pcg_hit_max = 1;
            done = 1;
          } else {
            c->pcg_beta = rz / __ldcg(&c->pcg_rz);
            c->pcg_rz = rz;
          }
          c->pcg_done = done;
          if (!done) atomicOr(&s_notdone, 1);
        }
      }
      __syncthreads();
      if (tid == 0) bar->all_done = !s_notdone;
      __threadfence();
    };
    if (!grid_barrier(bar, scalar_b)) return;
  }
}

int pcg_max_grid(int group, int device) {
  cudaDeviceProp prop;
  if (cudaGetDeviceProperties(&prop, device) != cudaSuccess) return 0;
  int per_sm = 0;
  if (group == 4)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<float, 4>, PCG_TILE * 4, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pcg<float, 8>, PCG_TILE * 8, 0);
  int per_sm_d = 0;
  if (group == 4)
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_d, k_pcg<double, 4>, PCG_TILE * 4, 0);
  else
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_d, k_pcg<double, 8>, PCG_TILE * 8, 0);
  const int m = per_sm < per_sm_d ? per_sm : per_sm_d;
  return m * prop.multiProcessorCount;
}

template <typename T>
cudaError_t launch_pcg(const SceneDev<T>* scenes, const TileRef* tiles, const PcgLaunch& L,
                       cudaStream_t st) {
  cudaError_t e = cudaMemsetAsync(L.bar, 0, sizeof(GridBar), st);
  if (e != cudaSuccess) return e;
  int n_tiles = L.n_tiles;
  const int* ids = L.scene_ids;
  int n_scenes = L.n_scenes;
  GridBar* bar = L.bar;
  int bg = L.use_b_from_g;
  void* args[] = {(void*)&scenes, (void*)&tiles, (void*)&n_tiles, (void*)&ids,
                  (void*)&n_scenes, (void*)&bar, (void*)&bg};
  const int grid = L.grid;
  if (L.group == 4)
    return cudaLaunchCooperativeKernel((const void*)k_pcg<T, 4>, dim3(grid), dim3(PCG_TILE * 4), args, 0, st);
  return cudaLaunchCooperativeKernel((const void*)k_pcg<T, 8>, dim3(grid), dim3(PCG_TILE * 8), args, 0, st);
}

template cudaError_t launch_pcg<float>(const SceneDev<float>*, const TileRef*, const PcgLaunch&, cudaStream_t);
template cudaError_t launch_pcg<double>(const SceneDev<double>*, const TileRef*, const PcgLaunch&, cudaStream_t);

}  // namespace ppn
