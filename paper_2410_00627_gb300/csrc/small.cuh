// small.cuh -- thread-local small-matrix helpers (register arrays): the
// inverse of a symmetric positive definite matrix, the inverse of the m x m
// measurement covariance, and a bit-pattern test for zero / non-finite values.
#pragma once
#include "grp.cuh"
#include "srtm_internal.cuh"

namespace srtm {

// In-place unpivoted LDL^T of a symmetric NX x NX matrix held row-major in
// memory (only the lower triangle and the diagonal are read): afterwards the
// strictly lower entries hold the unit lower factor L and the diagonal holds
// D, a = L D L^T; the upper entries are left as they were.  D may have either
// sign, so no information of a semidefinite matrix is dropped; a zero pivot
// gives a zero column of L (for a semidefinite matrix that column of a is
// zero too).  One thread, NX reciprocals.
template <int NX, class T>
__device__ __forceinline__ void ldlt_inplace(T* a) {
#pragma unroll
  for (int j = 0; j < NX; ++j) {
    T v[NX > 1 ? NX - 1 : 1];  // v_t = L_jt D_t
    T d = a[j * NX + j];
#pragma unroll
    for (int t = 0; t < j; ++t) {
      v[t] = a[j * NX + t] * a[t * NX + t];
      d = fma(-a[j * NX + t], v[t], d);
    }
    a[j * NX + j] = d;
    if (j + 1 < NX) {
      const T inv = (d != T(0)) ? T(1) / d : T(0);
#pragma unroll
      for (int i = j + 1; i < NX; ++i) {
        T w = a[i * NX + j];
#pragma unroll
        for (int t = 0; t < j; ++t) w = fma(-a[i * NX + t], v[t], w);
        a[i * NX + j] = w * inv;
      }
    }
  }
}

// inverse of a symmetric positive definite matrix by Cholesky (a = L L^T,
// a^-1 = L^-T L^-1).  Only the leading nact x nact block is inverted; the
// rest of inv is set to the identity.  Returns false if a pivot is not
// positive.  logdet (optional): log det of the leading block, 2 sum log L_jj.
template <int N, class T>
__device__ __forceinline__ bool spd_inverse(const T (&a)[N][N], T (&inv)[N][N], int nact = N, T* logdet = nullptr) {
  T Lm[N][N];
  bool ok = true;
  T ld = T(0);
#pragma unroll
  for (int j = 0; j < N; ++j) {
#pragma unroll
    for (int i = 0; i < N; ++i) Lm[i][j] = (i == j) ? T(1) : T(0);
    if (j < nact) {
      T d = a[j][j];
#pragma unroll
      for (int k = 0; k < j; ++k) d = fma(-Lm[j][k], Lm[j][k], d);
      if (!(d > T(0)) || !isfinite(d)) { ok = false; d = T(1); }
      const T ljj = sqrt(d), rinv = T(1) / ljj;
      Lm[j][j] = ljj;
      if (logdet) ld += log(d);
#pragma unroll
      for (int i = j + 1; i < N; ++i) {
        if (i < nact) {
          T s2 = a[i][j];
#pragma unroll
          for (int k = 0; k < j; ++k) s2 = fma(-Lm[i][k], Lm[j][k], s2);
          Lm[i][j] = s2 * rinv;
        }
      }
    }
  }
  T Li[N][N];  // L^-1, lower triangular
#pragma unroll
  for (int i = 0; i < N; ++i) {
#pragma unroll
    for (int j = 0; j < N; ++j) Li[i][j] = (i == j) ? T(1) : T(0);
    if (i < nact) {
      Li[i][i] = T(1) / Lm[i][i];
#pragma unroll
      for (int j = 0; j < i; ++j) {
        T s2 = T(0);
#pragma unroll
        for (int k = j; k < i; ++k) s2 = fma(Lm[i][k], Li[k][j], s2);
        Li[i][j] = -s2 * Li[i][i];
      }
    }
  }
#pragma unroll
  for (int i = 0; i < N; ++i)
#pragma unroll
    for (int j = i; j < N; ++j) {
      T s2 = (i == j) ? T(1) : T(0);
      if (j < nact) {
        s2 = T(0);
#pragma unroll
        for (int k = j; k < N; ++k)
          if (k < nact) s2 = fma(Li[k][i], Li[k][j], s2);
      }
      inv[i][j] = s2;
      inv[j][i] = s2;
    }
  if (logdet) *logdet = ld;
  return ok;
}

// ===========================================================================
// interval setup: for every slow interval k (paper index k+1), from
// p(x_{k-1,l}|y_{1:k-1}) and y_k, the fast-filter blocks it needs (Eq. 17 on
// the blocks of Remark 2) and the parallel IMS element (Eq. 29):
//   X = P C_bar^T, S_y = C_bar X + R_x, kap = S_y^-1 (y - C_bar m),
//   U_i = A^i X + V_i H^T   (U_i = sum_j P^-_{ij} H^T),
//   m^f_i = A^i m + U_i kap,  P^f_{ij} = A^i P A^{jT} + Cov(e_i,e_j) - U_i S_y^-1 U_j^T,
//   P^-_{k+1,1} = A P^f_{ll} A^T + Q,  Z = A^T (P^-_{k+1,1})^-1,
//   E_k = P^f_{1l} Z,  g_k = m^f_1 - E_k A m^f_l,  S_k = P^f_{11} - E_k A (P^f_{1l})^T
// (last interval: E = 0, g = m^f_1, S = P^f_{11}).  The record keeps what the
// recovery reuses.  Runs in TR (float64 except in the float32 mode).
//
// Row split: SG lanes per interval (SG = nx rounded up to a power of two),
// lane r owns row r of every n x n product; the interval's matrices live in
// a shared-memory slot.  The small SPD inverses are formed by every lane of
// the interval from the slot (a warp FP64 instruction costs the same whatever
// its active lanes, so the repetition is free).
// ===========================================================================
// zero, infinite or NaN test on the bit pattern
__device__ __forceinline__ bool bad_value(double x) { return bad_pivot(x); }
__device__ __forceinline__ bool bad_value(float x) { return bad_pivot(x); }

// Inverse of a small symmetric m x m matrix (m <= MY, runtime) held in the
// leading block of a: adjugate for m <= 3 (one division), Cholesky for m = 4.
// The rest of inv is the identity.  Returns false on a singular matrix.
// logdet (optional): log det a, for a positive definite a.
template <class TR>
__device__ __forceinline__ bool small_sym_inverse(const TR (&a)[MY][MY], TR (&inv)[MY][MY], int m,
                                                  TR* logdet = nullptr) {
#pragma unroll
  for (int i = 0; i < MY; ++i)
#pragma unroll
    for (int j = 0; j < MY; ++j) inv[i][j] = (i == j) ? TR(1) : TR(0);
  if (m == 4) return spd_inverse<MY, TR>(a, inv, 4, logdet);
  TR det;
  if (m == 1) {
    det = a[0][0];
  } else if (m == 2) {
    det = a[0][0] * a[1][1] - a[0][1] * a[1][0];
  } else {
    det = a[0][0] * (a[1][1] * a[2][2] - a[1][2] * a[2][1]) - a[0][1] * (a[1][0] * a[2][2] - a[1][2] * a[2][0]) +
          a[0][2] * (a[1][0] * a[2][1] - a[1][1] * a[2][0]);
  }
  if (logdet) *logdet = log(det);
  bool ok = !bad_value(det);
  if (!ok) det = TR(1);
  const TR id = TR(1) / det;
  if (m == 1) {
    inv[0][0] = id;
  } else if (m == 2) {
    inv[0][0] = a[1][1] * id;
    inv[1][1] = a[0][0] * id;
    inv[0][1] = -a[0][1] * id;
    inv[1][0] = -a[1][0] * id;
  } else {
#pragma unroll
    for (int r = 0; r < 3; ++r)
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const int i0 = c == 0 ? 1 : 0, i1 = c == 2 ? 1 : 2, j0 = r == 0 ? 1 : 0, j1 = r == 2 ? 1 : 2;
        TR v = a[i0][j0] * a[i1][j1] - a[i0][j1] * a[i1][j0];
        inv[r][c] = (((r + c) & 1) ? -v : v) * id;
      }
  }
  return ok;
}

// Inverse of the symmetric positive definite d x d matrix a (row-major, ld
// d), one thread: a is overwritten by its LDL^T factors (L below the
// diagonal, D on it) and L^{-1} (above the diagonal, transposed), then
//   a^{-1} = L^{-T} D^{-1} L^{-1}
// is written to inv.  Returns false (inv unset) when a pivot D_j is not
// above rtol times the diagonal entry a_jj it came from (the variable j is
// then determined by the ones before it to within that fraction of its
// variance: the matrix is singular or too ill-conditioned for the inverse to
// keep float64 accuracy) or is not finite.
__device__ inline bool spd_inverse_checked(double* a, int d, double* inv, double rtol) {
  double rd[16];  // 1 / D_k (d <= 16)
  for (int j = 0; j < d; ++j) {
    const double ajj = a[j * d + j];
    double dj = ajj;
    for (int k = 0; k < j; ++k) dj = fma(-a[j * d + k] * a[j * d + k], a[k * d + k], dj);
    if (!(dj > rtol * ajj) || bad_value(dj)) return false;
    a[j * d + j] = dj;
    rd[j] = 1.0 / dj;
    for (int i = j + 1; i < d; ++i) {
      double v = a[i * d + j];
      for (int k = 0; k < j; ++k) v = fma(-a[i * d + k] * a[j * d + k], a[k * d + k], v);
      a[i * d + j] = v * rd[j];
    }
  }
  // X = L^{-1} (unit lower): X_ij = -sum_{k=j}^{i-1} L_ik X_kj, kept at a[j][i]
  for (int j = 0; j < d; ++j)
    for (int i = j + 1; i < d; ++i) {
      double v = -a[i * d + j];
      for (int k = j + 1; k < i; ++k) v = fma(-a[i * d + k], a[j * d + k], v);
      a[j * d + i] = v;
    }
  for (int i = 0; i < d; ++i)
    for (int j = i; j < d; ++j) {
      double v = 0.0;  // sum_{k >= j} X_ki X_kj / D_k, X_kk = 1
      for (int k = j; k < d; ++k) {
        const double xi = k == i ? 1.0 : a[i * d + k], xj = k == j ? 1.0 : a[j * d + k];
        v = fma(xi * xj, rd[k], v);
      }
      inv[i * d + j] = v;
      inv[j * d + i] = v;
    }
  return true;
}

// Is the n x n row-major matrix a (n <= N) a covariance: every entry finite,
// symmetric to within 1e-8 of its largest diagonal entry, and positive
// semi-definite?  The last test is a Cholesky factorisation of the
// symmetric part with a pivot tolerance (the semi-definite Cholesky of
// Higham, "Accuracy and Stability of Numerical Algorithms", 2nd ed.,
// Sec. 10.3): a pivot below -tau fails; a pivot in [-tau, tau] marks a null
// direction, and since every 2 x 2 principal minor of a PSD matrix is
// non-negative, the rest of its column must then vanish to within
// sqrt(tau * s); tau = 1e-10 * n * s, s = max_i a_ii.  One thread (host-callable
// too, for the unit test of the classification).
template <int N>
__host__ __device__ __noinline__ bool psd_check(const double* a, int n) {
  double s = 0.0;
  bool ok = true;
  for (int i = 0; i < n; ++i) s = fmax(s, fabs(a[i * n + i]));
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j) {
      const double v = a[i * n + j];
      if (!isfinite(v) || fabs(v - a[j * n + i]) > 1e-8 * s) ok = false;
    }
  if (!ok) return false;
  const double tau = 1e-10 * n * s, off = sqrt(tau * s);
  double L[N][N];
  for (int j = 0; j < n; ++j) {
    double d = a[j * n + j];
    for (int k = 0; k < j; ++k) d = fma(-L[j][k], L[j][k], d);
    if (d < -tau) return false;
    const bool null_dir = d <= tau;
    const double ljj = null_dir ? 0.0 : sqrt(d);
    L[j][j] = ljj;
    for (int i = j + 1; i < n; ++i) {
      double r = 0.5 * (a[i * n + j] + a[j * n + i]);
      for (int k = 0; k < j; ++k) r = fma(-L[i][k], L[j][k], r);
      if (null_dir) {
        if (fabs(r) > off) return false;
        L[i][j] = 0.0;
      } else {
        L[i][j] = r / ljj;
      }
    }
  }
  return true;
}

}  // namespace srtm
