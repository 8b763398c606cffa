// constants.cuh -- per-model constants (float64), one block per sequence,
// after the blocks that check that every Q, R and P0 is a covariance.
//
// The lifted slow-rate model and the fast-rate blocks (Sec. III-A/B,
// Eq. 7-12, 14-15) and the constant parts of the parallel IMKF elements
// (Eq. 25-26), with e_i = sum_{r<=i} A^{i-r} w_r the noise part of x_{k,i}
// given x_{k-1,l}:
//   A^i (i = 0..l),  Qc_i = Cov(e_i) = sum_{r<i} A^r Q A^rT,
//   S_q = sum_{j<=q} A^j,  V_i = Cov(e_i, sum_j e_j) = A V_{i-1} + Q S_{l-i}^T,
//   Cov(e_i, e_l) = Qc_i A^{(l-i)T},  C_bar = H sum_{i=1..l} A^i,
//   M Q~ M^T = H (sum_i V_i) H^T,  G Q~ M^T = V_l H^T,  Q_bar = Qc_l,
//   R_x = M Q~ M^T + R,  K = G Q~ M^T R_x^-1,  F = A^l - K C_bar,
//   D = Q_bar - K (G Q~ M^T)^T,  J = C_bar^T R_x^-1 C_bar,
// and the first element (m^f_{1,l}, P^f_{1,l}) by one IMKF step from (m0, P0)
// (Eq. 9, 12).  The state size NX is a compile-time constant; the
// measurement size m <= MY is not.
#pragma once
#include "grp.cuh"
#include "small.cuh"
#include "srtm_internal.cuh"

namespace srtm {

constexpr int PRE_THREADS = 256;
constexpr size_t PRE_SMEM_CAP = 200 * 1024;

// out (R x C, row-major, ld C) = alpha op(A) op(B) + ADD over the G lanes of
// one product unit; R <= RM, C <= CM, K <= KM.  op(A) is R x K (TA: A stored
// K x R), op(B) is K x C (TB: B stored C x K).  SYM: only entries r <= c are
// formed and each is written to both (r,c) and (c,r) (for results that are
// symmetric in exact arithmetic).  No barrier.
template <int RM, int CM, int KM, int G, bool TA, bool TB, bool SYM = false>
__device__ __forceinline__ void u_mm(int lane, int R, int K, int C, double* out, const double* A, const double* B,
                                     const double* ADD, double alpha) {
  for (int e = lane; e < RM * CM; e += G) {
    const int r = e / CM, c = e - (e / CM) * CM;
    if (r < R && c < C && (!SYM || r <= c)) {
      double s = 0.0;
#pragma unroll
      for (int k = 0; k < KM; ++k)
        if (k < K) s = fma(TA ? A[k * R + r] : A[r * K + k], TB ? B[c * K + k] : B[k * C + c], s);
      const double v = ADD ? fma(alpha, s, ADD[r * C + c]) : alpha * s;
      out[r * C + c] = v;
      if (SYM) out[c * C + r] = v;
    }
  }
}

// inverse of the symmetric m x m matrix a (ld m) by one unit: every lane
// forms it in registers, lanes write the upper entries, mirrored
template <int G>
__device__ __forceinline__ bool u_sym_inverse(int lane, int m, const double* a, double* inv) {
  double A[MY][MY], Ai[MY][MY];
#pragma unroll
  for (int i = 0; i < MY; ++i)
#pragma unroll
    for (int j = 0; j < MY; ++j) A[i][j] = (i < m && j < m) ? a[i * m + j] : ((i == j) ? 1.0 : 0.0);
  const bool ok = small_sym_inverse<double>(A, Ai, m);
  for (int e = lane; e < MY * MY; e += G) {
    const int i = e / MY, j = e - (e / MY) * MY;
    if (i <= j && j < m) {
      double v = 0.0;
#pragma unroll
      for (int ii = 0; ii < MY; ++ii)
#pragma unroll
        for (int jj = 0; jj < MY; ++jj)
          if (ii == i && jj == j) v = Ai[ii][jj];
      inv[i * m + j] = v;
      inv[j * m + i] = v;
    }
  }
  return ok;
}

// shared-memory layout of the constants kernel (doubles)
template <int NX>
struct PreGeom {
  static constexpr int G = GroupSize<NX>::value;  // lanes per product unit
  static constexpr int NU = PRE_THREADS / G;      // product units per block
  static constexpr int NN = NX * NX, NM = NX * MY, MM = MY * MY;
  // inputs
  static constexpr int A = 0, Q = A + NN, H = Q + NN, R = H + NM, P0 = R + MM, m0 = P0 + NN, y0 = m0 + NX;
  // slow-model constants and first-element work
  static constexpr int T = y0 + MY, Vs = T + NN, HVs = Vs + NN, Rx = HVs + NM, Rxi = Rx + MM, GQM = Rxi + MM,
                       K = GQM + NM, Cr = K + NM, Cb = Cr + NM, Fc = Cb + NM, Dc = Fc + NN, Jc = Dc + NN,
                       AP = Jc + NN, CP = AP + NN, cross = CP + NM, S1 = cross + NM, S1i = S1 + MM, Lg = S1i + MM,
                       innov = Lg + NM, P1 = innov + MY, P1o = P1 + NN, m1 = P1o + NN, bu = m1 + NX,
                       sbu = bu + NX, USCR = sbu + NX;  // bu, sbu: first interval's b_{1,l}, sum_i b_{1,i}
  // two-point recovery: Cov([x_{k+1,1}; y_k] | x_{k,1}) and its inverse, the
  // same for y_k alone, H S_{l-1}
  static constexpr int DD = (NX + MY) * (NX + MY);
  static constexpr int Vb = USCR + NU * NN, Vbi = Vb + DD, Vy = Vbi + DD, Vyi = Vy + MM, HS = Vyi + MM;
  static constexpr int BASE = HS + NM;  // then the tables
  // tables: A^0..A^L, S_0..S_{L-1}, Cov(e_i) terms / prefixes, two V buffers
  __host__ __device__ static size_t tables(int L) { return (size_t)(5 * L + 1) * NN; }
};

// Constants of the two-point recovery of one sequence (float64, by the
// block of its constants kernel, after the model table is written).  Given
// the first state x_{k,1} of an interval, the noise parts of the interval's
// states, eps_i = x_{k,i} - A^{i-1} x_{k,1} (i = 1..l+1, eps_{l+1} for the
// next interval's first state), are jointly distributed as e_{i-1} of the
// lifted model (Sec. III-A; the noise of i - 1 fast steps), so
//   Cov(eps_i) = Qc_{i-1},  Cov(eps_i, eps_{l+1}) = Cov(e_{i-1}, e_l),
//   Cov(eps_i, H sum_j eps_j) = (V_{i-1} - Cov(e_{i-1}, e_l)) H^T,
// and v = [x_{k+1,1}; y_k] has E[v | x_{k,1}] = [A^l; H S_{l-1}] x_{k,1}
// (S_{l-1} = sum_{j<l} A^j) and covariance
//   Vb = [[Qc_l, (V_l - Qc_l) H^T], [., R_x - H V_l H^T - (H V_l H^T)^T + H Qc_l H^T]].
// Conditioning x_{k,i} on (x_{k,1}, v) (the states between two first states
// depend on the rest of the data only through them and y_k):
//   G_i = K_i Vb^{-1},  K_i = Cov(eps_i, v),
//   C2_i = G_i[:, :n],  c3_i = G_i[:, n:],  C1_i = A^{i-1} - G_i [A^l; H S_{l-1}],
//   Sg_i = Qc_{i-1} - G_i K_i^T,
// so that E[x_{k,i} | x_{k,1}, x_{k+1,1}, y_k] = C1_i x_{k,1} + C2_i x_{k+1,1}
// + c3_i y_k with covariance Sg_i.  The last interval conditions on
// (x_{k,1}, y_k) only (C1'_i, c3'_i, Sg'_i from the y block of Vb).  A
// sequence where a pivot of Vb (or of its y block) is below 1e-6 of the
// variance it came from keeps the record form (bflag = 0): singular or
// nearly singular process noise over an interval, where the inverse would
// not keep float64 accuracy.
template <int NX>
__device__ void two_point_constants(const Ctx& c, int s, int l, int m, double* md, double* sm, int tid, int nt) {
  using S = PreGeom<NX>;
  constexpr int NN = NX * NX, BT = 3 * NN + NX * MY, BO = 2 * NN + NX * MY;
  const ModelLayout L = c.ml;
  const int d = NX + m;
  __shared__ int s_bok;
  __syncthreads();  // the model table's tables are complete
  const double* Qcl = md + L.Qc + (size_t)(l - 1) * NN;
  const double* Al = md + L.Apow + (size_t)l * NN;
  const double* H = sm + S::H;
  const double* GQM = sm + S::GQM;
  double *Vb = sm + S::Vb, *Vbi = sm + S::Vbi, *Vy = sm + S::Vy, *Vyi = sm + S::Vyi, *HS = sm + S::HS;
  for (int e = tid; e < d * d; e += nt) {  // upper entries, mirrored
    const int r = e / d, q = e - (e / d) * d;
    if (r > q) continue;
    double v;
    if (q < NX) {
      v = 0.5 * (Qcl[r * NX + q] + Qcl[q * NX + r]);
    } else if (r < NX) {
      const int j = q - NX;
      v = GQM[r * m + j];
      for (int t = 0; t < NX; ++t) v = fma(-Qcl[r * NX + t], H[j * NX + t], v);
    } else {
      const int i = r - NX, j = q - NX;
      v = 0.5 * (sm[S::Rx + i * m + j] + sm[S::Rx + j * m + i]);
      for (int t = 0; t < NX; ++t) v -= H[i * NX + t] * GQM[t * m + j] + H[j * NX + t] * GQM[t * m + i];
      for (int t = 0; t < NX; ++t) {
        double w = 0.0;
        for (int u = 0; u < NX; ++u) w = fma(Qcl[t * NX + u], H[j * NX + u], w);
        v = fma(H[i * NX + t], w, v);
      }
    }
    Vb[r * d + q] = v;
    Vb[q * d + r] = v;
  }
  for (int e = tid; e < m * NX; e += nt) {  // H S_{l-1} = H + C_bar - H A^l
    const int j = e / NX, q = e - (e / NX) * NX;
    double v = H[e] + sm[S::Cb + e];
    for (int t = 0; t < NX; ++t) v = fma(-H[j * NX + t], Al[t * NX + q], v);
    HS[e] = v;
  }
  __syncthreads();
  // the two inverses on two warps at once
  __shared__ int s_ok2[2];
  for (int e = tid; e < m * m; e += nt) Vy[e] = Vb[(NX + e / m) * d + NX + e % m];
  __syncthreads();  // Vy copied before Vb is factorised in place
  if (tid == 0) s_ok2[0] = spd_inverse_checked(Vb, d, Vbi, 1e-6) ? 1 : 0;
  if (tid == 32 % nt) s_ok2[1] = spd_inverse_checked(Vy, m, Vyi, 1e-6) ? 1 : 0;
  __syncthreads();
  if (tid == 0) {
    s_bok = s_ok2[0] && s_ok2[1];
    md[L.bflag] = s_bok ? 1.0 : 0.0;
  }
  __syncthreads();
  const bool ok = s_bok != 0;
  // K_i row q (col < NX the x block, else the y block) into registers
  constexpr int DM = NX + MY;
  auto Krow = [&](int i, int q, double (&K)[DM]) {
    const double* Qlj = md + L.Ql + (size_t)(i - 2) * NN;
    const double* VHj = md + L.VH + (size_t)(i - 2) * NX * m;
#pragma unroll
    for (int col = 0; col < DM; ++col) {
      double v = 0.0;
      if (col < NX) {
        v = Qlj[q * NX + col];
      } else if (col - NX < m) {
        const int j = col - NX;
        v = VHj[q * m + j];
#pragma unroll
        for (int t = 0; t < NX; ++t) v = fma(-Qlj[q * NX + t], H[j * NX + t], v);
      }
      K[col] = v;
    }
  };
  // one thread per entry (i, r, q)
  for (int e = tid; e < l * NN; e += nt) {
    const int i = e / NN + 1, rq = e - (e / NN) * NN, r = rq / NX, q = rq - (rq / NX) * NX;
    double* bt = md + L.BrT + (size_t)(i - 1) * BT;
    double* bo = md + L.BrO + (size_t)(i - 1) * BO;
    const double* Ai = md + L.Apow + (size_t)(i - 1) * NN;
    if (i == 1 || !ok) {  // x_{k,1} itself (and placeholders when the record form is kept)
      const double id = (r == q) ? 1.0 : 0.0;
      bt[rq] = id;
      bt[NN + rq] = 0.0;
      bt[2 * NN + rq] = 0.0;
      bo[rq] = id;
      bo[NN + rq] = 0.0;
      if (q == 0)
        for (int j = 0; j < MY; ++j) {
          bt[3 * NN + r * MY + j] = 0.0;
          bo[2 * NN + r * MY + j] = 0.0;
        }
      continue;
    }
    const double* Qj = md + L.Qc + (size_t)(i - 2) * NN;
    double Kr[DM], Kq[DM], G[DM], Gy[MY];
    Krow(i, r, Kr);
    Krow(i, q, Kq);
#pragma unroll
    for (int col = 0; col < DM; ++col) {
      double v = 0.0;
      if (col < d) {
#pragma unroll
        for (int c2 = 0; c2 < DM; ++c2)
          if (c2 < d) v = fma(Kr[c2], Vbi[c2 * d + col], v);
      }
      G[col] = v;
    }
#pragma unroll
    for (int j = 0; j < MY; ++j) {
      double v = 0.0;
      if (j < m) {
#pragma unroll
        for (int j2 = 0; j2 < MY; ++j2)
          if (j2 < m) v = fma(Kr[NX + j2], Vyi[j2 * m + j], v);
      }
      Gy[j] = v;
    }
    double c1 = Ai[rq], c1o = Ai[rq], sg = Qj[rq], sgo = Qj[rq];
#pragma unroll
    for (int t = 0; t < NX; ++t) {
      c1 = fma(-G[t], Al[t * NX + q], c1);
      sg = fma(-G[t], Kq[t], sg);
    }
#pragma unroll
    for (int j = 0; j < MY; ++j)
      if (j < m) {
        c1 = fma(-G[NX + j], HS[j * NX + q], c1);
        sg = fma(-G[NX + j], Kq[NX + j], sg);
        c1o = fma(-Gy[j], HS[j * NX + q], c1o);
        sgo = fma(-Gy[j], Kq[NX + j], sgo);
      }
    bt[rq] = c1;
    bt[NN + rq] = G[q];
    bt[2 * NN + rq] = sg;
    bo[rq] = c1o;
    bo[NN + rq] = sgo;
    if (q == 0)
#pragma unroll
      for (int j = 0; j < MY; ++j) {
        bt[3 * NN + r * MY + j] = j < m ? G[NX + j] : 0.0;
        bo[2 * NN + r * MY + j] = j < m ? Gy[j] : 0.0;
      }
  }
}

// Per-model constants of one sequence (one block per sequence, after the
// check blocks), float64.
//  1. A^i (i <= l) by doubling: round h forms A^{h+t} = A^h A^t, t = 1..h.
//  2. the terms A^r Q A^{rT} (r < l), one product unit each.
//  3. per entry, the running sums S_q = sum_{j<=q} A^j and
//     Qc_i = Cov(e_i) = sum_{r<i} A^r Q A^{rT}.
//  4. W_i = Q S_{l-i}^T, Cov(e_i, e_l) = Qc_i A^{(l-i)T}, C_bar = H sum A^i.
//  5. V_i = A V_{i-1} + W_i (V_1 = W_1) solved as V_i = sum_{j<=i} A^{i-j} W_j
//     by a log-depth scan: after the round with offset d,
//     X_i <- X_i + A^d X_{i-d} covers the terms j > i - 2d.
//  6. V_i H^T, G Q~ M^T = V_l H^T, M Q~ M^T = H (sum_i V_i) H^T.
//  7. R_x, K, C_bar^T R_x^-1, F, D, J and the first element (one IMKF step
//     from (m0, P0)), independent products on different units.
// The first blocks of the grid check, one thread per matrix, that every
// sequence's Q, R and P0 is a covariance (DEVERR_NOT_PSD); they run beside
// the sequences' blocks and add nothing to their latency.
template <int NX>
__global__ void __launch_bounds__(PRE_THREADS) precompute_kernel(Ctx c, int tables_in_smem) {
  using S = PreGeom<NX>;
  constexpr int G = S::G, NU = S::NU, NN = S::NN;
  extern __shared__ __align__(16) double dsm[];
  __shared__ int s_ok;
  const int check_blocks = (3 * c.n_seq + PRE_THREADS - 1) / PRE_THREADS;
  if (blockIdx.x < check_blocks) {
    const long long item = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (item < 3LL * c.n_seq) {
      const long long q = item / 3;
      const int which = (int)(item - q * 3), n = which == 1 ? c.ny : NX;
      const double* a = which == 0 ? c.Q + q * NN : which == 1 ? c.R + q * c.ny * c.ny : c.P0 + q * NN;
      if (!psd_check<(NX > MY ? NX : MY)>(a, n)) atomicOr(&c.ctr->err, DEVERR_NOT_PSD);
    }
    return;
  }
  if (c.fold_meta) {
    // single sequence (host-validated): this block writes the call metadata
    if (threadIdx.x == 0) {
      const int r = c.uniform_ratio, n = c.uniform_nslow;
      c.ctr->epoch = c.ctr->epoch + 1;
      for (int i = 0; i < 2 * MAXCHUNK; ++i) c.ctr->ticket[i] = 0;
      c.meta.ratio[0] = r;
      c.meta.nslow[0] = n;
      c.meta.off_slow[0] = 0;
      c.meta.off_slow[1] = n;
      c.meta.off_fast[0] = 0;
      c.meta.off_fast[1] = (long long)n * r;
      c.meta.tile_off_f[0] = 0;
      c.meta.tile_off_f[1] = (n + c.tile_f - 1) / c.tile_f;
      c.meta.tile_off_s[0] = 0;
      c.meta.tile_off_s[1] = (n + c.tile_s - 1) / c.tile_s;
      c.ctr->total_tiles_f = (n + c.tile_f - 1) / c.tile_f;
      c.ctr->total_tiles_s = (n + c.tile_s - 1) / c.tile_s;
      c.ctr->call_ok = 1u;
    }
    __syncthreads();
  } else if (!c.ctr->call_ok) {
    return;
  }
  const int s = blockIdx.x - check_blocks;
  const int m = c.ny, l = c.meta.ratio[s];
  const ModelLayout L = c.ml;
  double* md = c.model + (long long)s * L.stride;
  const int tid = threadIdx.x, nt = blockDim.x, unit = tid / G, lane = tid - (tid / G) * G;
  const unsigned umask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << ((tid & 31) & ~(G - 1)));
  double* sm = dsm;
  double* ub = dsm + S::USCR + unit * NN;
  double *Ap, *Sp, *Qp, *X0, *X1;
  if (tables_in_smem) {
    Ap = dsm + S::BASE;
    Sp = Ap + (size_t)(l + 1) * NN;
    Qp = Sp + (size_t)l * NN;
    X0 = Qp + (size_t)l * NN;
    X1 = X0 + (size_t)l * NN;
  } else {
    Ap = md + L.Apow;
    Sp = md + L.Ssc;
    Qp = md + L.Qc;
    X0 = md + L.Vsc;
    X1 = md + L.V2sc;
  }
  {
    const double* F = c.F + (long long)s * NN;
    const double* Q = c.Q + (long long)s * NN;
    const double* H = c.H + (long long)s * m * NX;
    const double* R = c.R + (long long)s * m * m;
    const double* P0 = c.P0 + (long long)s * NN;
    const double* m0 = c.m0 + (long long)s * NX;
    const double* y0 = c.y + c.meta.off_slow[s] * m;
    for (int e = tid; e < NN; e += nt) {
      const int r = e / NX, q = e - (e / NX) * NX;
      sm[S::A + e] = F[e];
      const double qs = 0.5 * (Q[e] + Q[q * NX + r]);
      sm[S::Q + e] = qs;
      md[L.Q + e] = qs;
      sm[S::P0 + e] = P0[e];
      Ap[e] = (r == q) ? 1.0 : 0.0;
      Ap[NN + e] = F[e];
    }
    for (int e = tid; e < m * NX; e += nt) sm[S::H + e] = H[e];
    for (int e = tid; e < m * m; e += nt) sm[S::R + e] = R[e];
    for (int e = tid; e < NX; e += nt) sm[S::m0 + e] = m0[e];
    for (int e = tid; e < m; e += nt) sm[S::y0 + e] = y0[e];
    if (tid == 0) s_ok = 1;
  }
  __syncthreads();
  // 1. powers
  for (int h = 1; h < l; h *= 2) {
    const int cnt = min(h, l - h);
    for (int t = unit; t < cnt; t += NU)
      u_mm<NX, NX, NX, G, false, false>(lane, NX, NX, NX, Ap + (size_t)(h + 1 + t) * NN, Ap + (size_t)h * NN,
                                        Ap + (size_t)(1 + t) * NN, nullptr, 1.0);
    __syncthreads();
  }
  // 2. terms A^r Q A^{rT}
  for (int r = unit; r < l; r += NU) {
    u_mm<NX, NX, NX, G, false, false>(lane, NX, NX, NX, ub, Ap + (size_t)r * NN, sm + S::Q, nullptr, 1.0);
    __syncwarp(umask);
    u_mm<NX, NX, NX, G, false, true, true>(lane, NX, NX, NX, Qp + (size_t)r * NN, ub, Ap + (size_t)r * NN, nullptr,
                                           1.0);
    __syncwarp(umask);
  }
  __syncthreads();
  // 3. running sums per entry
  for (int e = tid; e < NN; e += nt) {
    const int r = e / NX, q = e - (e / NX) * NX;
    double acc = (r == q) ? 1.0 : 0.0;
    Sp[e] = acc;
    for (int j = 1; j < l; ++j) {
      acc += Ap[(size_t)j * NN + e];
      Sp[(size_t)j * NN + e] = acc;
    }
    sm[S::T + e] = acc + Ap[(size_t)l * NN + e] - ((r == q) ? 1.0 : 0.0);
    double qa = 0.0;
    for (int j = 0; j < l; ++j) {
      qa += Qp[(size_t)j * NN + e];
      Qp[(size_t)j * NN + e] = qa;
    }
  }
  __syncthreads();
  // 4. W_i = Q S_{l-i}^T (i = 1..l), Cov(e_i, e_l) = Qc_i A^{(l-i)T}, C_bar = H T
  // known inputs: A^j B and S_j B (j < l), n x nu blocks, into the model table
  if (c.nu > 0) {
    const int nu = c.nu;
    const double* B = c.B + (long long)s * NX * nu;
    for (int e = tid; e < l * NX * nu; e += nt) {
      const int j = e / (NX * nu), rc = e - j * NX * nu, r = rc / nu, q = rc - (rc / nu) * nu;
      double a = 0.0, b = 0.0;
      for (int k = 0; k < NX; ++k) {
        a = fma(Ap[(size_t)j * NN + r * NX + k], B[k * nu + q], a);
        b = fma(Sp[(size_t)j * NN + r * NX + k], B[k * nu + q], b);
      }
      md[L.AB + e] = a;
      md[L.SB + e] = b;
    }
  }
  for (int t = unit; t <= 2 * l; t += NU) {
    if (t < l) {
      const int i = t + 1;
      u_mm<NX, NX, NX, G, false, true>(lane, NX, NX, NX, X0 + (size_t)(i - 1) * NN, sm + S::Q,
                                       Sp + (size_t)(l - i) * NN, nullptr, 1.0);
    } else if (t < 2 * l) {
      const int i = t - l + 1;
      u_mm<NX, NX, NX, G, false, true>(lane, NX, NX, NX, md + L.Ql + (size_t)(i - 1) * NN, Qp + (size_t)(i - 1) * NN,
                                       Ap + (size_t)(l - i) * NN, nullptr, 1.0);
    } else {
      u_mm<MY, NX, NX, G, false, false>(lane, m, NX, NX, sm + S::Cb, sm + S::H, sm + S::T, nullptr, 1.0);
    }
  }
  __syncthreads();
  // 5. V_i = sum_{j<=i} A^{i-j} W_j by doubling offsets
  double* cur = X0;
  double* nxt = X1;
  for (int d = 1; d < l; d *= 2) {
    for (int i = unit + 1; i <= l; i += NU) {
      if (i > d) {
        u_mm<NX, NX, NX, G, false, false>(lane, NX, NX, NX, nxt + (size_t)(i - 1) * NN, Ap + (size_t)d * NN,
                                          cur + (size_t)(i - 1 - d) * NN, cur + (size_t)(i - 1) * NN, 1.0);
      } else {
        for (int e = lane; e < NN; e += G) nxt[(size_t)(i - 1) * NN + e] = cur[(size_t)(i - 1) * NN + e];
      }
    }
    __syncthreads();
    double* x = cur; cur = nxt; nxt = x;
  }
  // 6. V_i H^T, G Q~ M^T = V_l H^T; sum_i V_i (symmetrised) per entry
  for (int t = unit; t <= l; t += NU) {
    if (t < l)
      u_mm<NX, MY, NX, G, false, true>(lane, NX, NX, m, md + L.VH + (size_t)t * NX * m, cur + (size_t)t * NN,
                                       sm + S::H, nullptr, 1.0);
    else
      u_mm<NX, MY, NX, G, false, true>(lane, NX, NX, m, sm + S::GQM, cur + (size_t)(l - 1) * NN, sm + S::H,
                                       nullptr, 1.0);
  }
  for (int e = tid; e < NN; e += nt) {
    const int r = e / NX, q = e - (e / NX) * NX;
    double v = 0.0;
    for (int i = 0; i < l; ++i) v += cur[(size_t)i * NN + r * NX + q] + cur[(size_t)i * NN + q * NX + r];
    sm[S::Vs + e] = 0.5 * v;
  }
  if (tables_in_smem) {
    for (size_t e = tid; e < (size_t)(l + 1) * NN; e += nt) md[L.Apow + e] = Ap[e];
    for (size_t e = tid; e < (size_t)l * NN; e += nt) md[L.Qc + e] = Qp[e];
  }
  // first interval's input terms b_{1,l} = sum_r A^{l-1-r} B u_r and sum_i b_{1,i} = sum_r S_{l-1-r} B u_r
  for (int r = tid; r < NX; r += nt) {
    double b = 0.0, sb = 0.0;
    if (c.nu > 0) {
      const int nu = c.nu;
      const double* u0 = c.u + c.meta.off_fast[s] * nu;
      for (int q = 0; q < l; ++q)
        for (int j = 0; j < nu; ++j) {
          b = fma(md[L.AB + ((size_t)(l - 1 - q) * NX + r) * nu + j], u0[q * nu + j], b);
          sb = fma(md[L.SB + ((size_t)(l - 1 - q) * NX + r) * nu + j], u0[q * nu + j], sb);
        }
    }
    sm[S::bu + r] = b;
    sm[S::sbu + r] = sb;
  }
  __syncthreads();
  for (int e = tid; e < m * NX; e += nt) md[L.Cb + e] = sm[S::Cb + e];
  {  // float copies of A, Qc_1, Cov(e_1, e_l), V_1 H^T for the float32 smoother elements
    float* cf = (float*)(md + L.Cf);
    for (int e = tid; e < NN; e += nt) {
      cf[e] = (float)Ap[NN + e];
      cf[NN + e] = (float)Qp[e];
      cf[2 * NN + e] = (float)md[L.Ql + e];
    }
    for (int e = tid; e < NX * m; e += nt) cf[3 * NN + e] = (float)md[L.VH + e];
  }
  // 7. slow-model constants and the first filter element
  const double* Al = Ap + (size_t)l * NN;
  const double* Qcl = Qp + (size_t)(l - 1) * NN;
  if (unit == 0) u_mm<MY, NX, NX, G, false, false>(lane, m, NX, NX, sm + S::HVs, sm + S::H, sm + S::Vs, nullptr, 1.0);
  if (unit == 1) u_mm<NX, NX, NX, G, false, false>(lane, NX, NX, NX, sm + S::AP, Al, sm + S::P0, nullptr, 1.0);
  if (unit == 2) u_mm<MY, NX, NX, G, false, false>(lane, m, NX, NX, sm + S::CP, sm + S::Cb, sm + S::P0, nullptr, 1.0);
  if (unit == 3)
    for (int j = lane; j < m; j += G) {   // y_1 - C_bar m0 - H sum_i b_{1,i}
      double v = sm[S::y0 + j];
      for (int q = 0; q < NX; ++q) v = fma(-sm[S::Cb + j * NX + q], sm[S::m0 + q], v);
      for (int q = 0; q < NX; ++q) v = fma(-sm[S::H + j * NX + q], sm[S::sbu + q], v);
      sm[S::innov + j] = v;
    }
  __syncthreads();
  if (unit == 0)
    u_mm<MY, MY, NX, G, false, true, true>(lane, m, NX, m, sm + S::Rx, sm + S::HVs, sm + S::H, sm + S::R, 1.0);
  if (unit == 1)
    u_mm<NX, NX, NX, G, false, true, true>(lane, NX, NX, NX, sm + S::P1, sm + S::AP, Al, Qcl, 1.0);
  if (unit == 2)
    u_mm<NX, MY, NX, G, false, true>(lane, NX, NX, m, sm + S::cross, sm + S::AP, sm + S::Cb, sm + S::GQM, 1.0);
  __syncthreads();
  if (unit == 0 && !u_sym_inverse<G>(lane, m, sm + S::Rx, sm + S::Rxi) && lane == 0) s_ok = 0;
  if (unit == 1)
    u_mm<MY, MY, NX, G, false, true, true>(lane, m, NX, m, sm + S::S1, sm + S::CP, sm + S::Cb, sm + S::Rx, 1.0);
  __syncthreads();
  if (unit == 0) u_mm<NX, MY, MY, G, false, false>(lane, NX, m, m, sm + S::K, sm + S::GQM, sm + S::Rxi, nullptr, 1.0);
  if (unit == 1) u_mm<NX, MY, MY, G, true, false>(lane, NX, m, m, sm + S::Cr, sm + S::Cb, sm + S::Rxi, nullptr, 1.0);
  if (unit == 2 && !u_sym_inverse<G>(lane, m, sm + S::S1, sm + S::S1i) && lane == 0) s_ok = 0;
  __syncthreads();
  // F = A^l - K C_bar ; D = Q_bar - K GQM^T ; J = C_bar^T R_x^-1 C_bar ; L = cross S1^-1
  if (unit == 0) u_mm<NX, NX, MY, G, false, false>(lane, NX, m, NX, sm + S::Fc, sm + S::K, sm + S::Cb, Al, -1.0);
  if (unit == 1)
    u_mm<NX, NX, MY, G, false, true, true>(lane, NX, m, NX, sm + S::Dc, sm + S::K, sm + S::GQM, Qcl, -1.0);
  if (unit == 2)
    u_mm<NX, NX, MY, G, false, false, true>(lane, NX, m, NX, sm + S::Jc, sm + S::Cr, sm + S::Cb, nullptr, 1.0);
  if (unit == 3)
    u_mm<NX, MY, MY, G, false, false>(lane, NX, m, m, sm + S::Lg, sm + S::cross, sm + S::S1i, nullptr, 1.0);
  __syncthreads();
  if (unit == 0)
    for (int r = lane; r < NX; r += G) {
      double v = sm[S::bu + r];
      for (int q = 0; q < NX; ++q) v = fma(Al[r * NX + q], sm[S::m0 + q], v);
      for (int j = 0; j < m; ++j) v = fma(sm[S::Lg + r * m + j], sm[S::innov + j], v);
      sm[S::m1 + r] = v;
    }
  if (unit == 1)
    u_mm<NX, NX, MY, G, false, true, true>(lane, NX, m, NX, sm + S::P1o, sm + S::Lg, sm + S::cross, sm + S::P1,
                                           -1.0);
  __syncthreads();
  // results to the model table
  for (int e = tid; e < NN; e += nt) {
    md[L.Fc + e] = sm[S::Fc + e];
    md[L.Dc + e] = sm[S::Dc + e];
    md[L.Jc + e] = sm[S::Jc + e];
    md[L.P1 + e] = sm[S::P1o + e];
    float* cf = (float*)(md + L.Cf) + 3 * NN + 3 * NX * MY;  // float copies for the float32 filter elements
    cf[e] = (float)sm[S::Fc + e];
    cf[NN + e] = (float)sm[S::Dc + e];
    cf[2 * NN + e] = (float)sm[S::Jc + e];
  }
  for (int e = tid; e < NX * m; e += nt) {
    md[L.K + e] = sm[S::K + e];
    md[L.Cr + e] = sm[S::Cr + e];
    float* cf = (float*)(md + L.Cf);  // float copies for the float32 filter elements
    cf[3 * NN + NX * MY + e] = (float)sm[S::K + e];
    cf[3 * NN + 2 * NX * MY + e] = (float)sm[S::Cr + e];
  }
  {  // float copies of C_bar and R_x (the rank-m filter combine, the float32
     // interval setup), A^l and V_l H^T (the float32 interval setup)
    float* cf = (float*)(md + L.Cf) + 6 * NN + 3 * NX * MY;
    for (int e = tid; e < m * NX; e += nt) cf[e] = (float)sm[S::Cb + e];
    for (int e = tid; e < m * m; e += nt) cf[MY * NX + e] = (float)sm[S::Rx + e];
    for (int e = tid; e < NN; e += nt) cf[MY * NX + MY * MY + e] = (float)Al[e];
    for (int e = tid; e < NX * m; e += nt) cf[MY * NX + MY * MY + NN + e] = (float)md[L.VH + (size_t)(l - 1) * NX * m + e];
  }
  for (int e = tid; e < m * m; e += nt) md[L.Rx + e] = sm[S::Rx + e];
  for (int e = tid; e < NX; e += nt) md[L.m1 + e] = sm[S::m1 + e];
  if (c.bridge) two_point_constants<NX>(c, s, l, m, md, sm, tid, nt);
  if (tid == 0 && !s_ok) atomicOr(&c.ctr->err, DEVERR_SINGULAR);
}

template <int NX>
inline void launch_precompute(const Ctx& c, cudaStream_t st) {
  using S = PreGeom<NX>;
  const size_t base = S::BASE * sizeof(double), tab = S::tables(c.max_ratio) * sizeof(double);
  const int in_smem = base + tab <= PRE_SMEM_CAP ? 1 : 0;
  const size_t smem = base + (in_smem ? tab : 0);
  static size_t granted[64] = {};  // per device: the largest size already allowed
  int dev = 0;
  cudaGetDevice(&dev);
  if (smem > 48 * 1024 && (dev < 0 || dev >= 64 || smem > granted[dev])) {
    cudaFuncSetAttribute(precompute_kernel<NX>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (dev >= 0 && dev < 64) granted[dev] = smem;
  }
  const int check_blocks = (3 * c.n_seq + PRE_THREADS - 1) / PRE_THREADS;
  precompute_kernel<NX><<<c.n_seq + check_blocks, PRE_THREADS, smem, st>>>(c, in_smem);
}

}  // namespace srtm
