// Per-tet Stable Neo-Hookean arithmetic in displacement form, shared by the
// element, energy and projection kernels (host-callable for checks).
//
// Model (the paper names Stable Neo-Hookean for 3D tets, Sec. 5.1):
//   psi(F) = mu/2 (tr F^T F - 3) - mu (J - 1) + lam/2 (J - 1)^2,  lam = lam_Lame + mu.
// Everything is written in terms of the displacement gradient H = F - I, which
// is formed from FP64 displacement differences before any rounding to T.  Near
// rest P(F) and psi(F) are O(|H|) and O(|H|^2) quantities; computing them from
// H instead of F avoids the cancellation that would cost FP32 all its digits
// (F - cof F = H + H^T - tr(H) I - cof(H), J - 1 = tr H + I2(H) + det H).
//
// Element Hessian blocks use the closed form of V B^T (dP/dF) B for a linear
// tet with shape-function gradients dN_a (a = 0..3):
//   H_ab = V [ mu (dN_a . dN_b) I + lam (C dN_a)(C dN_b)^T + s [F (dN_a x dN_b)]_eps ],
//   s = lam (J - 1) - mu,  C = cof F,  ([w]_eps)_ik = sum_m eps_ikm w_m.
#pragma once

#include <cuda_runtime.h>

#define PPN_HD __host__ __device__ __forceinline__

namespace ppn {

// index of block (a, b), a <= b, in the 10-block upper triangle of a 4x4 block matrix
PPN_HD constexpr int tri4(int a, int b) { return a * 4 - (a * (a - 1)) / 2 + (b - a); }

template <typename T>
struct TetState {
  T H[9];   // displacement gradient F - I, row-major
  T C[9];   // cof F
  T F[9];   // F
  T Jm1;    // J - 1
  T s;      // lam (J - 1) - mu
};

// cofactor matrix of a general 3x3 (cof = det(A) A^-T)
template <typename T>
PPN_HD void cof3(const T* A, T* C) {
  C[0] = A[4] * A[8] - A[5] * A[7];
  C[1] = A[5] * A[6] - A[3] * A[8];
  C[2] = A[3] * A[7] - A[4] * A[6];
  C[3] = A[2] * A[7] - A[1] * A[8];
  C[4] = A[0] * A[8] - A[2] * A[6];
  C[5] = A[1] * A[6] - A[0] * A[7];
  C[6] = A[1] * A[5] - A[2] * A[4];
  C[7] = A[2] * A[3] - A[0] * A[5];
  C[8] = A[0] * A[4] - A[1] * A[3];
}

// H = E W with E = [u1-u0, u2-u0, u3-u0] formed in double and rounded to T
template <typename T>
PPN_HD void disp_grad(const double* u0, const double* u1, const double* u2, const double* u3,
                      const T* W, T* H) {
  T e[3][3];  // e[c][i] = (u_{c+1} - u_0)_i
  const double* uc[3] = {u1, u2, u3};
  for (int c = 0; c < 3; ++c)
    for (int i = 0; i < 3; ++i) e[c][i] = (T)(uc[c][i] - u0[i]);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) H[3 * i + j] = e[0][i] * W[j] + e[1][i] * W[3 + j] + e[2][i] * W[6 + j];
}

template <typename T>
PPN_HD void tet_state(const T* H, T mu, T lam, TetState<T>& st) {
  T cH[9];
  cof3(H, cH);
  const T trH = H[0] + H[4] + H[8];
  const T I2 = cH[0] + cH[4] + cH[8];  // sum of principal 2x2 minors
  const T detH = H[0] * cH[0] + H[1] * cH[1] + H[2] * cH[2];
  st.Jm1 = trH + I2 + detH;
  for (int a = 0; a < 9; ++a) {
    st.H[a] = H[a];
    st.F[a] = H[a];
  }
  st.F[0] += (T)1;
  st.F[4] += (T)1;
  st.F[8] += (T)1;
  // cof(I + H) = I + tr(H) I - H^T + cof(H)
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) st.C[3 * i + j] = cH[3 * i + j] - H[3 * j + i];
  st.C[0] += (T)1 + trH;
  st.C[4] += (T)1 + trH;
  st.C[8] += (T)1 + trH;
  st.s = lam * st.Jm1 - mu;
}

// energy density from the displacement gradient:
// psi = mu/2 |H|^2 - mu (I2 + det H) + lam/2 (J - 1)^2
template <typename T>
PPN_HD T snh_psi_disp(const T* H, T mu, T lam) {
  T cH[9];
  cof3(H, cH);
  const T trH = H[0] + H[4] + H[8];
  const T I2 = cH[0] + cH[4] + cH[8];
  const T detH = H[0] * cH[0] + H[1] * cH[1] + H[2] * cH[2];
  T n2 = 0;
  for (int a = 0; a < 9; ++a) n2 += H[a] * H[a];
  const T Jm1 = trH + I2 + detH;
  return (T)0.5 * mu * n2 - mu * (I2 + detH) + (T)0.5 * lam * Jm1 * Jm1;
}

// first Piola-Kirchhoff stress: P = mu (F - cof F) + lam (J - 1) cof F
template <typename T>
PPN_HD void snh_pk1_disp(const TetState<T>& st, T mu, T lam, T* P) {
  T cH[9];
  cof3(st.H, cH);
  const T trH = st.H[0] + st.H[4] + st.H[8];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      T fmc = st.H[3 * i + j] + st.H[3 * j + i] - cH[3 * i + j];
      if (i == j) fmc -= trH;
      P[3 * i + j] = mu * fmc + lam * st.Jm1 * st.C[3 * i + j];
    }
}

// shape-function gradients: dN_a = row (a-1) of W for a >= 1, dN_0 = -(sum)
template <typename T>
PPN_HD void shape_grads(const T* W, T dN[4][3]) {
  for (int j = 0; j < 3; ++j) {
    dN[1][j] = W[j];
    dN[2][j] = W[3 + j];
    dN[3][j] = W[6 + j];
    dN[0][j] = -(W[j] + W[3 + j] + W[6 + j]);
  }
}

// One 3x3 Hessian-like block for the generalized "shape vectors" na, nb with
// ca = C na, cb = C nb:  V [mu (na.nb) I + lam ca cb^T + s [F (na x nb)]_eps]
template <typename T>
PPN_HD void hess_block(const TetState<T>& st, T V, T mu, T lam, const T* na, const T* nb,
                       const T* ca, const T* cb, T* out) {
  const T dot = na[0] * nb[0] + na[1] * nb[1] + na[2] * nb[2];
  const T cr[3] = {na[1] * nb[2] - na[2] * nb[1], na[2] * nb[0] - na[0] * nb[2],
                   na[0] * nb[1] - na[1] * nb[0]};
  T w[3];
  for (int m = 0; m < 3; ++m) w[m] = st.F[3 * m] * cr[0] + st.F[3 * m + 1] * cr[1] + st.F[3 * m + 2] * cr[2];
  const T sw0 = st.s * w[0], sw1 = st.s * w[1], sw2 = st.s * w[2];
  const T md = mu * dot;
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) out[3 * i + k] = lam * ca[i] * cb[k];
  out[0] += md;
  out[4] += md;
  out[8] += md;
  // ([w]_eps)_ik = eps_ikm w_m
  out[1] += sw2;
  out[2] -= sw1;
  out[3] -= sw2;
  out[5] += sw0;
  out[6] += sw1;
  out[7] -= sw0;
  for (int a = 0; a < 9; ++a) out[a] *= V;
}

template <typename T>
PPN_HD void matvec3(const T* M, const T* v, T* out) {
  out[0] = M[0] * v[0] + M[1] * v[1] + M[2] * v[2];
  out[1] = M[3] * v[0] + M[4] * v[1] + M[5] * v[2];
  out[2] = M[6] * v[0] + M[7] * v[1] + M[8] * v[2];
}

}  // namespace ppn
