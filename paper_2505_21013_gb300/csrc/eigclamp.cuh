// Eigenvalue clamping of one tet Hessian through a 9x9 reduced eigenproblem,
// in registers (host-callable for checks).
//
// The projection is the clamping of Sec. 3: H^e = Q D Q^T is replaced by
// Q max(D, eps) Q^T, added to the assembled matrix as the difference
// dH^e = sum_{lambda_i < eps} (eps - lambda_i) q_i q_i^T (Sec. 4.1).  With
// `mirror` the target of such an eigenvalue is max(|lambda_i|, eps) instead
// (eigenvalue mirroring, which the paper compares against clamping, Sec. 5.2).
//
// Reduction.  A linear tet's Hessian is H^e = V B^T A B with B the 9x12 map
// x_e -> vec F built from the shape gradients dN_a (rows of the 4x3 matrix D),
// and A = dP/dF.  Let G = D^T D = L L^T (Cholesky).  With S = D L^-T, whose
// columns are orthonormal, B = B_L T where T x = (sum_a S_aj x_a)_j has
// orthonormal rows and B_L is the same map built from the three columns l_j of
// L instead of the four dN_a.  Hence H^e = T^T M T with the 9x9
//   M = V B_L^T A B_L   (3x3 block (j, l) = the tet Hessian block formula with l_j, l_l),
// so the twelve eigenpairs of H^e are the nine of M, lifted by q_a = sum_j S_aj z_j,
// plus the three rigid translations with eigenvalue exactly 0 (T annihilates
// them).  Clamping those adds eps/4 I to every 3x3 block.  The 9x9 problem is
// solved with Jacobi sweeps of symmetric 2x2 Schur rotations in round-robin order;
// all index arithmetic unrolls at compile time so the matrices live in registers.
#pragma once

#include "tetmath.cuh"

namespace ppn {

PPN_HD constexpr int s9(int r, int c) {
  return r <= c ? r * 9 - (r * (r - 1)) / 2 + (c - r) : c * 9 - (c * (c - 1)) / 2 + (r - c);
}

template <typename T> struct JacobiCfg;
template <> struct JacobiCfg<float> {
  static constexpr float rel_tol = 1e-7f;   // stop when off(M) <= rel_tol ||M||_F
  static constexpr float big_tau = 1e7f;
  static constexpr int max_sweeps = 12;
};
template <> struct JacobiCfg<double> {
  static constexpr double rel_tol = 1e-15;
  static constexpr double big_tau = 1e15;
  static constexpr int max_sweeps = 20;
};

template <typename T>
PPN_HD T rsqrt_t(T x);
template <>
PPN_HD float rsqrt_t<float>(float x) {
#ifdef __CUDA_ARCH__
  return rsqrtf(x);
#else
  return 1.0f / sqrtf(x);
#endif
}
template <>
PPN_HD double rsqrt_t<double>(double x) {
  return 1.0 / sqrt(x);
}

// The symmetric Schur rotation zeroing A(p, q) (Golub & Van Loan, Sec. 8.5): t = tan of
// the angle, c, s its cosine and sine; skip when A(p, q) is already zero.
template <typename T>
struct JRot {
  T app, aqq, apq, t, c, s;
  bool skip;
};
template <typename T, int P, int Q>
PPN_HD JRot<T> jrot_params(const T* A) {
  JRot<T> r;
  r.apq = A[s9(P, Q)];
  r.app = A[s9(P, P)];
  r.aqq = A[s9(Q, Q)];
  r.skip = r.apq == (T)0;
  const T apq = r.skip ? (T)1 : r.apq;
  const T tau = (r.aqq - r.app) / ((T)2 * apq);
  const T at = tau < (T)0 ? -tau : tau;
  T t = at > JacobiCfg<T>::big_tau ? (T)0.5 / at : (T)1 / (at + sqrt((T)1 + at * at));
  if (tau < (T)0) t = -t;
  r.t = t;
  r.c = rsqrt_t<T>((T)1 + t * t);
  r.s = t * r.c;
  return r;
}
// A <- J^T A J and V <- V J for the rotation of (P, Q); V accumulates the eigenvectors (columns)
template <typename T, int P, int Q>
PPN_HD void jrot_apply(T* A, T* V, const JRot<T>& r) {
  if (r.skip) return;
  const T t = r.t, c = r.c, s = r.s;
  A[s9(P, P)] = r.app - t * r.apq;
  A[s9(Q, Q)] = r.aqq + t * r.apq;
  A[s9(P, Q)] = (T)0;
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    if (k == P || k == Q) continue;
    const T akp = A[s9(k, P)], akq = A[s9(k, Q)];
    A[s9(k, P)] = c * akp - s * akq;
    A[s9(k, Q)] = s * akp + c * akq;
  }
#pragma unroll
  for (int k = 0; k < 9; ++k) {
    const T vkp = V[9 * k + P], vkq = V[9 * k + Q];
    V[9 * k + P] = c * vkp - s * vkq;
    V[9 * k + Q] = s * vkp + c * vkq;
  }
}

// Round-robin ordering of the 36 index pairs of a sweep (the circle method for 9
// indices): in round r index x meets (2r - x) mod 9 and index r sits out, so every
// round holds 4 disjoint pairs and every pair meets once in the 9 rounds.  Disjoint
// rotations commute, and a rotation's parameters read only the (p,p), (q,q), (p,q)
// entries of its pair, which the round's other rotations leave unchanged: the four
// parameter computations of a round are independent (four times the work in flight
// of a cyclic-by-row sweep, whose rotations wait for one another).
PPN_HD constexpr int rr_mate(int r, int x) { return ((2 * r - x) % 9 + 9) % 9; }
PPN_HD constexpr int rr_p(int r, int i) {
  int k = 0;
  for (int x = 0; x < 9; ++x)
    if (x != r && x < rr_mate(r, x)) {
      if (k == i) return x;
      ++k;
    }
  return -1;
}
PPN_HD constexpr int rr_q(int r, int i) { return rr_mate(r, rr_p(r, i)); }

template <typename T, int R>
PPN_HD void jround(T* A, T* V) {
  constexpr int p0 = rr_p(R, 0), q0 = rr_q(R, 0), p1 = rr_p(R, 1), q1 = rr_q(R, 1);
  constexpr int p2 = rr_p(R, 2), q2 = rr_q(R, 2), p3 = rr_p(R, 3), q3 = rr_q(R, 3);
  static_assert(p3 >= 0 && q0 > p0 && q1 > p1 && q2 > p2 && q3 > p3, "four pairs per round");
  const JRot<T> r0 = jrot_params<T, p0, q0>(A), r1 = jrot_params<T, p1, q1>(A);
  const JRot<T> r2 = jrot_params<T, p2, q2>(A), r3 = jrot_params<T, p3, q3>(A);
  jrot_apply<T, p0, q0>(A, V, r0);
  jrot_apply<T, p1, q1>(A, V, r1);
  jrot_apply<T, p2, q2>(A, V, r2);
  jrot_apply<T, p3, q3>(A, V, r3);
}

template <typename T, int R>
struct SweepRounds {
  PPN_HD static void run(T* A, T* V) {
    jround<T, R>(A, V);
    if constexpr (R < 8) SweepRounds<T, R + 1>::run(A, V);
  }
};

// Jacobi on the packed symmetric 9x9 A with round-robin sweeps; returns sweeps used
template <typename T>
PPN_HD int jacobi9(T* A, T* V) {
#pragma unroll
  for (int k = 0; k < 81; ++k) V[k] = (k % 10 == 0) ? (T)1 : (T)0;
  T fro2 = 0;
#pragma unroll
  for (int r = 0; r < 9; ++r)
#pragma unroll
    for (int c = r; c < 9; ++c) fro2 += (r == c ? (T)1 : (T)2) * A[s9(r, c)] * A[s9(r, c)];
  const T tol2 = JacobiCfg<T>::rel_tol * JacobiCfg<T>::rel_tol * fro2;
  int sweep = 0;
  for (; sweep < JacobiCfg<T>::max_sweeps; ++sweep) {
    T off2 = 0;
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
      for (int c = r + 1; c < 9; ++c) off2 += (T)2 * A[s9(r, c)] * A[s9(r, c)];
    if (!(off2 > tol2)) break;
    SweepRounds<T, 0>::run(A, V);
  }
  return sweep;
}

// The reduced problem of a tet: M (packed symmetric 9x9, s9 order) and the lift
// S_aj = (L^-1 dN_a)_j.  W = Dm^-1 (row a-1 = dN_a), V = rest volume.
template <typename T>
PPN_HD void reduce9(const TetState<T>& st, const T* W, T Vol, T mu, T lam, T* A, T S[4][3]) {
  T dN[4][3];
  shape_grads(W, dN);
  // G = sum_a dN_a dN_a^T and its Cholesky factor L
  T G[6] = {0, 0, 0, 0, 0, 0};  // (0,0) (1,0) (1,1) (2,0) (2,1) (2,2)
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    G[0] += dN[a][0] * dN[a][0];
    G[1] += dN[a][1] * dN[a][0];
    G[2] += dN[a][1] * dN[a][1];
    G[3] += dN[a][2] * dN[a][0];
    G[4] += dN[a][2] * dN[a][1];
    G[5] += dN[a][2] * dN[a][2];
  }
  const T L00 = sqrt(G[0]);
  const T L10 = G[1] / L00, L20 = G[3] / L00;
  const T L11 = sqrt(G[2] - L10 * L10);
  const T L21 = (G[4] - L20 * L10) / L11;
  const T L22 = sqrt(G[5] - L20 * L20 - L21 * L21);
  const T l[3][3] = {{L00, L10, L20}, {(T)0, L11, L21}, {(T)0, (T)0, L22}};  // columns of L
  T cl[3][3];
#pragma unroll
  for (int j = 0; j < 3; ++j) matvec3(st.C, l[j], cl[j]);

#pragma unroll
  for (int j = 0; j < 3; ++j)
#pragma unroll
    for (int m = j; m < 3; ++m) {
      T blk[9];
      hess_block(st, Vol, mu, lam, l[j], l[m], cl[j], cl[m], blk);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int k = 0; k < 3; ++k)
          if (3 * j + i <= 3 * m + k) A[s9(3 * j + i, 3 * m + k)] = blk[3 * i + k];
    }
  // S_aj = (L^-1 dN_a)_j by forward substitution
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    S[a][0] = dN[a][0] / L00;
    S[a][1] = (dN[a][1] - L10 * S[a][0]) / L11;
    S[a][2] = (dN[a][2] - L20 * S[a][0] - L21 * S[a][1]) / L22;
  }
}

// dH blocks (10 x 9, upper block triangle, tri4 order) of the clamped tet.
// Returns the number of clamped eigenvalues of M (the three translation modes are
// always clamped as well).
template <typename T>
PPN_HD int clamp_tet(const TetState<T>& st, const T* W, T Vol, T mu, T lam, T eps, bool mirror, T* out) {
  T A[45], S[4][3];
  reduce9(st, W, Vol, mu, lam, A, S);
  T Vec[81];
  jacobi9(A, Vec);
  const T e4 = eps * (T)0.25;
#pragma unroll
  for (int b = 0; b < 10; ++b)
#pragma unroll
    for (int k = 0; k < 9; ++k) out[9 * b + k] = (k == 0 || k == 4 || k == 8) ? e4 : (T)0;
  int n_clamped = 0;
#pragma unroll
  for (int p = 0; p < 9; ++p) {
    const T lp = A[s9(p, p)];
    if (lp < eps) {
      ++n_clamped;
      const T w = (mirror ? (-lp > eps ? -lp : eps) : eps) - lp;
      T q[4][3];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int i = 0; i < 3; ++i)
          q[a][i] = S[a][0] * Vec[9 * (0 + i) + p] + S[a][1] * Vec[9 * (3 + i) + p] +
                    S[a][2] * Vec[9 * (6 + i) + p];
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = a; b < 4; ++b)
#pragma unroll
          for (int i = 0; i < 3; ++i)
#pragma unroll
            for (int k = 0; k < 3; ++k) out[9 * tri4(a, b) + 3 * i + k] += w * q[a][i] * q[b][k];
    }
  }
  return n_clamped;
}

}  // namespace ppn
