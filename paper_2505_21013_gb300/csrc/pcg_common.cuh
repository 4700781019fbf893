// Helpers shared by the two cooperative PCG kernels (global-memory and
// shared-memory-resident variants): bounded grid barrier, L2-only vector
// loads, fixed-order reductions and the per-scene CG state.
#pragma once

#include "common.cuh"
#include "kernels.h"

namespace ppn {
namespace pcgdev {

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
// The wait is bounded; on timeout the barrier's flag is set and false returned.
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

__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void fence_acq_rel() { asm volatile("fence.acq_rel.gpu;" ::: "memory"); }

template <typename R>
__device__ __forceinline__ R warp_sum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  return v;
}

// ---- stamped words.  A tile partial crosses the grid as N 64-bit words, each
// carrying the phase stamp; stamp 0 is never used (the words are zeroed before
// every launch).  FP32 partials: one word, stamp = the 32-bit phase counter in
// the high half, the value's bits in the low half.  FP64 partials: hi and lo
// words (hi = the value with its 16 low mantissa bits cleared, lo = value - hi,
// exact), stamp in the 16 low bits of each.
template <typename R>
struct Words;
template <>
struct Words<float> {
  static constexpr int N = 1;
  __device__ static unsigned stamp(unsigned epoch) { return epoch; }
  __device__ static unsigned long long filler(unsigned s) { return (unsigned long long)s << 32; }
  __device__ static void split(float v, unsigned s, unsigned long long* w) {
    w[0] = ((unsigned long long)s << 32) | __float_as_uint(v);
  }
  __device__ static bool has(unsigned long long w, unsigned s) { return (unsigned)(w >> 32) == s; }
  __device__ static float join(const unsigned long long* w) { return __uint_as_float((unsigned)w[0]); }
};
template <>
struct Words<double> {
  static constexpr int N = 2;
  __device__ static unsigned stamp(unsigned epoch) { return ((epoch - 1u) % 65535u) + 1u; }
  __device__ static unsigned long long filler(unsigned s) { return s; }
  __device__ static void split(double v, unsigned s, unsigned long long* w) {
    const unsigned long long b = (unsigned long long)__double_as_longlong(v);
    const unsigned long long hb = b & ~0xFFFFull;
    const double lo = v - __longlong_as_double((long long)hb);
    const unsigned long long lb = (unsigned long long)__double_as_longlong(lo) & ~0xFFFFull;
    w[0] = hb | s;
    w[1] = lb | s;
  }
  __device__ static bool has(unsigned long long w, unsigned s) { return (unsigned)(w & 0xFFFFull) == s; }
  __device__ static double join(const unsigned long long* w) {
    return __longlong_as_double((long long)(w[0] & ~0xFFFFull)) +
           __longlong_as_double((long long)(w[1] & ~0xFFFFull));
  }
};
// ---- FP32 z / d_prev records: one 32-byte record {z.xyz, 0, d.xyz, 0} per row
// and parity buffer, so a neighbour gather is one 256-bit load.  Iteration k
// reads buffer k & 1 (z_k, d_{k-1}) and writes d_k and z_{k+1} into the other.
__device__ __forceinline__ void ld_rec(const float* p, float (&a)[8]) {
  asm volatile("ld.global.cg.v8.f32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
               : "=f"(a[0]), "=f"(a[1]), "=f"(a[2]), "=f"(a[3]), "=f"(a[4]), "=f"(a[5]), "=f"(a[6]), "=f"(a[7])
               : "l"(p));
}
__device__ __forceinline__ void st_rec_half(float* p, float x, float y, float z) {
  asm volatile("st.global.v4.f32 [%0], {%1,%2,%3,%4};" ::"l"(p), "f"(x), "f"(y), "f"(z), "f"(0.0f) : "memory");
}
__device__ __forceinline__ float* rec_ptr(float* base, int nv, int parity, int i) {
  return base + ((size_t)parity * nv + i) * 8;
}

// bound of one wait, in polling rounds; a CTA that gives up flags a timeout
constexpr unsigned kWaitSpins = 1u << 20;

// One warp polls the stamped words W[LO..HI] (four per lane per round, LANE the
// lane index) until each is >= STAMP.  It gives up after LIMIT rounds on some
// chunk, or at once when the expression GAVE_UP is true (another warp gave up),
// and then runs GIVE_UP.  A macro, so that the PCG kernels' wait compiles as the
// loop written in place (the kernels sit at the register limit, where an
// out-of-line form measured slower) and the bounded-wait check runs the same text.
#define PPN_WARP_WAIT_STAMPS(W, LO, HI, STAMP, LIMIT, LANE, GAVE_UP, GIVE_UP)      \
  for (int c0 = (LO) + (LANE); c0 <= (HI); c0 += 32 * 4) {                        \
    unsigned long long w_[4];                                                     \
    _Pragma("unroll") for (int u = 0; u < 4; ++u) {                               \
      const int c = c0 + 32 * u;                                                  \
      w_[u] = c <= (HI) ? ld_relaxed_u64((W) + c) : (STAMP);                      \
    }                                                                             \
    for (unsigned spins = 0;; ++spins) {                                          \
      bool ready = true;                                                          \
      _Pragma("unroll") for (int u = 0; u < 4; ++u) ready &= w_[u] >= (STAMP);    \
      if (ready) break;                                                           \
      if (spins > (LIMIT) || (GAVE_UP)) {                                         \
        GIVE_UP;                                                                  \
        break;                                                                    \
      }                                                                           \
      _Pragma("unroll") for (int u = 0; u < 4; ++u) if (w_[u] < (STAMP)) w_[u] =  \
          ld_relaxed_u64((W) + c0 + 32 * u);                                      \
    }                                                                             \
  }

// per-scene fields a PCG kernel needs, copied to shared memory once per solve
// so that no phase chases descriptor pointers through global memory
template <typename T>
struct SceneLite {
  using V4 = vec4_t<T>;
  const int* row_ptr;
  const int* col;
  const T* val;
  const int* diag_idx;
  const double4* g;
  V4* z;
  V4* d0;
  V4* d1;
  V4* q;
  V4* r;
  V4* dx;
  T* Pinv;
  double* ppart;
  unsigned long long* pword;
  T* zrec;
  Ctl* ctl;
  double tol2;
  int nv, nnzb, n_ptiles, max_iter;
};

template <typename T>
__device__ __forceinline__ void load_lite(SceneLite<T>& L, const SceneDev<T>& S) {
  L.row_ptr = S.row_ptr;
  L.col = S.col;
  L.val = S.val;
  L.diag_idx = S.diag_idx;
  L.g = S.g;
  L.z = S.z;
  L.d0 = S.d0;
  L.d1 = S.d1;
  L.q = S.q;
  L.r = S.r;
  L.dx = S.dx;
  L.Pinv = S.Pinv;
  L.ppart = S.ppart;
  L.pword = S.pword;
  L.zrec = S.zrec;
  L.ctl = S.ctl;
  L.tol2 = S.pcg_tol2;
  L.nv = S.nv;
  L.nnzb = S.nnzb;
  L.n_ptiles = S.n_ptiles;
  L.max_iter = S.pcg_max_iter;
}

// per-scene solver state, replicated identically in every CTA.  R is the
// type of the CG scalars: double in the FP64 path, float in the mixed path
// (its vectors are FP32, and FP64 issues at a small fraction of the FP32 rate).
template <typename R>
struct SState {
  R rz, rr0, rr, alpha, beta, dq;
  int iters, done, ind, pfail, hitmax, nonfinite;
};

// 3x3 block-Jacobi inverse through the Cholesky factor of the lower triangle;
// returns false when a pivot is not positive
template <typename T>
__device__ __forceinline__ bool spd_inv3(const T* D, T* Pm) {
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
  Pm[0] = i00 * i00 + i10 * i10 + i20 * i20;
  Pm[1] = i10 * i11 + i20 * i21;
  Pm[2] = i20 * i22;
  Pm[4] = i11 * i11 + i21 * i21;
  Pm[5] = i21 * i22;
  Pm[8] = i22 * i22;
  Pm[3] = Pm[1];
  Pm[6] = Pm[2];
  Pm[7] = Pm[5];
  return ok;
}

// scalar step after phase A: alpha, or the negative-curvature exit
template <typename R>
__device__ __forceinline__ void after_dq(SState<R>& s, R dq) {
  s.dq = dq;
  if (!(dq == dq)) {
    s.nonfinite = 1;
    s.done = 1;
  } else if (!(dq > (R)0)) {
    s.ind = 1;
    s.done = 1;
  } else {
    s.alpha = s.rz / dq;
  }
}

// scalar step after phase B: convergence, iteration cap, beta
template <typename R>
__device__ __forceinline__ void after_rz(SState<R>& s, R rz, R r2, double tol2, int max_iter) {
  s.iters += 1;
  s.rr = r2;
  if (!(r2 == r2) || !(rz == rz)) {
    s.nonfinite = 1;
    s.done = 1;
  } else if (r2 <= (R)tol2 * s.rr0) {
    s.done = 1;
  } else if (s.iters >= max_iter) {
    s.hitmax = 1;
    s.done = 1;
  } else {
    s.beta = rz / s.rz;
    s.rz = rz;
  }
}

constexpr int XCH_MAX_CTAS = 1024;  // CTAs of one resident PCG launch (XCH_MAX_CTAS_HOST in kernels.h)

template <typename R>
__device__ __forceinline__ void init_state(SState<R>& s, R rz, R r2, R f) {
  s.rz = rz;
  s.rr0 = r2;
  s.rr = r2;
  s.alpha = (R)0;
  s.beta = (R)0;
  s.dq = (R)0;
  s.iters = 0;
  s.hitmax = 0;
  s.nonfinite = !(r2 == r2) || !(rz == rz);
  s.pfail = f > (R)0;
  s.ind = f > (R)0;
  s.done = (f > (R)0) || !(r2 > (R)0) || s.nonfinite;
}

template <typename R>
__device__ __forceinline__ void publish(const SState<R>& s, Ctl* c) {
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

}  // namespace pcgdev
}  // namespace ppn
