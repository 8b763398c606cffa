// seq.cuh -- the sequential forms of the slow-rate recursions, one thread per
// sequence: the IMKF (Eq. 9-12) walked forward over k and the IMS backward
// recursion (Eq. 21-22, through the per-interval elements of Eq. 29) walked
// backward.  They are the O(N)-depth counterpart of the two scans and write
// exactly what the scans write (filter results m^f_{k,l}, P^f_{k,l}; the
// smoothing terms Om_k, om_k), so the interval setup and the fast-rate
// recovery are shared with the scan path.
#pragma once
#include <cuda_runtime.h>

#include "small.cuh"
#include "srtm_internal.cuh"

namespace srtm {

constexpr int SEQ_THREADS = 64;

// IMKF step in the decorrelated form behind Eq. (25)-(26): with
// x = x_{k-1,l} ~ N(m, P), y_k = C_bar x + c_k + nu (Cov nu = R_x) and
// x_{k,l} = F x + K (y_k - c_k) + b_{k,l} + eps (Cov eps = D, eps and nu
// independent), F = A^l - K C_bar, D = Q_bar - K (G Q~ M^T)^T.  Conditioning x
// on y_k and propagating gives the Eq. (9)-(12) filter result exactly.
// M = ny (compile-time): loops over the measurement entries run M times.
template <int NX, int M, class TS>
__global__ void __launch_bounds__(SEQ_THREADS) seq_filter_kernel(Ctx c) {
  constexpr int NN = NX * NX, MM = M;
  if (!c.ctr->call_ok) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= c.n_seq) return;
  constexpr int m = M;
  const int N = c.meta.nslow[s];
  const long long off = c.meta.off_slow[s];
  const double* md = c.model + (long long)s * c.ml.stride;
  const double* Fc = md + c.ml.Fc;
  const double* Dc = md + c.ml.Dc;
  const double* Kc = md + c.ml.K;   // n x m
  const double* Cb = md + c.ml.Cb;  // m x n
  const double* Rx = md + c.ml.Rx;  // m x m
  TS* fout = (TS*)c.fout;
  TS mv[NX], P[NX][NX];
#pragma unroll
  for (int r = 0; r < NX; ++r) {
    mv[r] = (TS)md[c.ml.m1 + r];
#pragma unroll
    for (int q = 0; q < NX; ++q) P[r][q] = (TS)md[c.ml.P1 + r * NX + q];
  }
  {
    TS* o = fout + off * (NX + NN);
#pragma unroll
    for (int r = 0; r < NX; ++r) o[r] = mv[r];
#pragma unroll
    for (int e = 0; e < NN; ++e) o[NX + e] = P[e / NX][e % NX];
  }
  bool ok = true;
  for (int k = 1; k < N; ++k) {
    const long long row = off + k;
    const double* yk = c.y + row * m;
    const double* ui = c.uin ? c.uin + row * UIn<NX>::SIZE : nullptr;
    TS yc[MY], CP[MY][NX], S[MY][MY], Si[MY][MY], e[MY];
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      yc[j] = TS(0);
      e[j] = TS(0);
      if (j < m) {
        yc[j] = (TS)(ui ? yk[j] - ui[UIn<NX>::c + j] : yk[j]);
        TS v = yc[j];
#pragma unroll
        for (int q = 0; q < NX; ++q) v = fma(-(TS)__ldg(Cb + j * NX + q), mv[q], v);
        e[j] = v;
      }
    }
    // C_bar P, S = C_bar P C_bar^T + R_x
#pragma unroll
    for (int j = 0; j < MM; ++j)
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        TS v = TS(0);
        if (j < m)
#pragma unroll
          for (int t = 0; t < NX; ++t) v = fma((TS)__ldg(Cb + j * NX + t), P[t][q], v);
        CP[j][q] = v;
      }
#pragma unroll
    for (int i = 0; i < MM; ++i)
#pragma unroll
      for (int j = 0; j < MM; ++j) {
        TS v = (i == j) ? TS(1) : TS(0);
        if (i < m && j < m) {
          v = (TS)__ldg(Rx + i * m + j);
#pragma unroll
          for (int t = 0; t < NX; ++t) v = fma(CP[i][t], (TS)__ldg(Cb + j * NX + t), v);
        }
        S[i][j] = v;
      }
    ok &= small_sym_inverse<TS>(S, Si, m);
    // LT = S^-1 C_bar P  (the transposed gain P C_bar^T S^-1)
    TS LT[MY][NX];
#pragma unroll
    for (int i = 0; i < MM; ++i)
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        TS v = TS(0);
#pragma unroll
        for (int j = 0; j < MM; ++j)
          if (j < m) v = fma(Si[i][j], CP[j][q], v);
        LT[i][q] = v;
      }
    // conditioned on y_k: m+ = m + L e, P+ = P - L C_bar P (upper triangle, mirrored)
    TS mp[NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      TS v = mv[r];
#pragma unroll
      for (int j = 0; j < MM; ++j)
        if (j < m) v = fma(LT[j][r], e[j], v);
      mp[r] = v;
    }
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int q = r; q < NX; ++q) {
        TS v = P[r][q];
#pragma unroll
        for (int j = 0; j < MM; ++j)
          if (j < m) v = fma(-CP[j][r], LT[j][q], v);
        P[r][q] = v;
        P[q][r] = v;
      }
    // propagated: m^f = F m+ + K (y - c) + b_l,  P^f = F P+ F^T + D
    TS FP[NX][NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      TS v = ui ? (TS)ui[UIn<NX>::bl + r] : TS(0);
#pragma unroll
      for (int q = 0; q < NX; ++q) v = fma((TS)__ldg(Fc + r * NX + q), mp[q], v);
#pragma unroll
      for (int j = 0; j < MM; ++j)
        if (j < m) v = fma((TS)__ldg(Kc + r * m + j), yc[j], v);
      mv[r] = v;
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        TS w = TS(0);
#pragma unroll
        for (int t = 0; t < NX; ++t) w = fma((TS)__ldg(Fc + r * NX + t), P[t][q], w);
        FP[r][q] = w;
      }
    }
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int q = r; q < NX; ++q) {
        TS v = (TS)__ldg(Dc + r * NX + q);
#pragma unroll
        for (int t = 0; t < NX; ++t) v = fma(FP[r][t], (TS)__ldg(Fc + q * NX + t), v);
        P[r][q] = v;
        P[q][r] = v;
      }
    TS* o = fout + row * (NX + NN);
#pragma unroll
    for (int r = 0; r < NX; ++r) o[r] = mv[r];
#pragma unroll
    for (int e2 = 0; e2 < NN; ++e2) o[NX + e2] = P[e2 / NX][e2 % NX];
  }
  if (!ok) raise_err(c.ctr, DEVERR_SINGULAR);
}

// Backward IMS recursion (Eq. 21-22) through the elements (E_k, g_k, L_k) of
// Eq. (29): m^s_{k,1} = E_k m^s_{k+1,1} + g_k, P^s_{k,1} = E_k P^s_{k+1,1} E_k^T
// + L_k, started from the last interval's element, accumulated in TR.  Each
// result gives the smoothing terms of the interval before it, as the reverse
// scan's result pass does: Om_{k-1} = Z dP Z^T, om_{k-1} = Z dm with
// dP = P^s_{k,1} - P^-_{k,1}, dm = m^s_{k,1} - A m^f_{k-1,l} - B u_{k-1,l}.
template <int NX, class T, class TR>
__global__ void __launch_bounds__(SEQ_THREADS) seq_smoother_kernel(Ctx c) {
  constexpr int NN = NX * NX;
  using SLy = SL<NX>;
  using RL = Rec<NX>;
  if (!c.ctr->call_ok) return;
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= c.n_seq) return;
  const int N = c.meta.nslow[s];
  const long long off = c.meta.off_slow[s];
  const T* se = (const T*)c.selem;
  const double* A1 = c.model + (long long)s * c.ml.stride + c.ml.Apow + NN;
  TR g[NX], S[NX][NX];
  {
    const T* x = se + (off + N - 1) * SLy::SIZE;
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      g[r] = (TR)x[SLy::g + r];
#pragma unroll
      for (int q = 0; q < NX; ++q) S[r][q] = (TR)x[SLy::S + r * NX + q];
    }
  }
  for (int k = N - 1; k >= 1; --k) {
    if (k < N - 1) {  // fold element k into the running result
      const T* x = se + (off + k) * SLy::SIZE;
      TR E[NX][NX], ng[NX], ES[NX][NX];
#pragma unroll
      for (int r = 0; r < NX; ++r)
#pragma unroll
        for (int q = 0; q < NX; ++q) E[r][q] = (TR)x[SLy::E + r * NX + q];
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        TR v = (TR)x[SLy::g + r];
#pragma unroll
        for (int q = 0; q < NX; ++q) v = fma(E[r][q], g[q], v);
        ng[r] = v;
#pragma unroll
        for (int q = 0; q < NX; ++q) {
          TR w = TR(0);
#pragma unroll
          for (int t = 0; t < NX; ++t) w = fma(E[r][t], S[t][q], w);
          ES[r][q] = w;
        }
      }
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        g[r] = ng[r];
#pragma unroll
        for (int q = r; q < NX; ++q) {
          TR v = (TR)x[SLy::S + r * NX + q];
#pragma unroll
          for (int t = 0; t < NX; ++t) v = fma(ES[r][t], E[q][t], v);
          S[r][q] = v;
          S[q][r] = v;
        }
      }
    }
    // smoothing terms of interval k-1
    const long long row = off + k - 1;
    const TR* rc = (const TR*)c.rec + row * RL::SIZE;
    TR dm[NX], ZdP[NX][NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      TR v = g[r];
#pragma unroll
      for (int q = 0; q < NX; ++q) v = fma(-(TR)__ldg(A1 + r * NX + q), rc[RL::ml + q], v);
      if (c.uin) v -= (TR)c.uin[row * UIn<NX>::SIZE + UIn<NX>::bn + r];
      dm[r] = v;
    }
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        TR w = TR(0);
#pragma unroll
        for (int t = 0; t < NX; ++t) w = fma(rc[RL::Z + r * NX + t], S[t][q] - rc[RL::Pm + t * NX + q], w);
        ZdP[r][q] = w;
      }
    TR* out = (TR*)c.sfin + row * SFin<NX>::SIZE;
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      TR v = TR(0);
#pragma unroll
      for (int q = 0; q < NX; ++q) v = fma(rc[RL::Z + r * NX + q], dm[q], v);
      out[SFin<NX>::om + r] = v;
#pragma unroll
      for (int q = r; q < NX; ++q) {
        TR w = TR(0);
#pragma unroll
        for (int t = 0; t < NX; ++t) w = fma(ZdP[r][t], rc[RL::Z + q * NX + t], w);
        out[SFin<NX>::Om + r * NX + q] = w;
        out[SFin<NX>::Om + q * NX + r] = w;
      }
    }
    ldlt_inplace<NX, TR>(out + SFin<NX>::Om);  // the recovery takes Om as its LDL^T factors
  }
}

}  // namespace srtm
