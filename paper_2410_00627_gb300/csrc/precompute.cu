// precompute.cu -- per-call metadata and per-model constants (float64).
//
// meta_kernel (one block): validates the batch metadata, forms the row and
// tile offsets of every sequence, resets the tickets and bumps the
// call epoch that tags the scans' look-back flags.
//
// precompute_kernel (one block per sequence): the constants of the lifted
// slow-rate model and of the fast-rate blocks (Sec. III-A/B, Eq. 7-12, 14-15)
// and the constant parts of the parallel IMKF elements (Eq. 25-26):
//   A^i (i = 0..l), Qc_i = Cov(e_i) = A Qc_{i-1} A^T + Q,
//   S_q = sum_{j<=q} A^j, V_i = Cov(e_i, sum_j e_j) = A V_{i-1} + Q S_{l-i}^T,
//   Cov(e_i, e_l) = Qc_i A^{(l-i)T},  C_bar = H sum_{i=1..l} A^i,
//   M Q~ M^T = H (sum_i V_i) H^T,  G Q~ M^T = V_l H^T,  Q_bar = Qc_l,
//   R_x = M Q~ M^T + R,  K = G Q~ M^T R_x^-1,  F = A^l - K C_bar,
//   D = Q_bar - K (G Q~ M^T)^T,  J = C_bar^T R_x^-1 C_bar,
// where e_i = sum_{r<=i} A^{i-r} w_r is the noise part of x_{k,i} given
// x_{k-1,l}, and the first element (m^f_{1,l}, P^f_{1,l}) by one IMKF step
// from (m0, P0) (Eq. 9, 12).
#include <cuda_runtime.h>

#include "srtm_internal.cuh"

namespace srtm {

// ---------------------------------------------------------------------------
__global__ void __launch_bounds__(1024) meta_kernel(Ctx c) {
  __shared__ long long sc[4][1024];
  __shared__ int s_bad;
  const int tid = threadIdx.x, nt = blockDim.x;
  if (tid == 0) {
    s_bad = 0;
    c.ctr->epoch = c.ctr->epoch + 1;
    for (int i = 0; i < 4; ++i) c.ctr->ticket[i] = 0;
  }
  __syncthreads();
  const int per = (c.n_seq + nt - 1) / nt;
  const int s0 = min(c.n_seq, tid * per), s1 = min(c.n_seq, s0 + per);
  long long acc[4] = {0, 0, 0, 0};
  int bad = 0;
  for (int s = s0; s < s1; ++s) {
    const int r = c.in_ratio ? c.in_ratio[s] : c.uniform_ratio;
    const int n = c.in_nslow ? c.in_nslow[s] : c.uniform_nslow;
    if (r < 1 || r > c.max_ratio || n < 1) { bad = 1; continue; }
    acc[0] += n;
    acc[1] += (long long)n * r;
    acc[2] += (n + c.tile_f - 1) / c.tile_f;
    acc[3] += (n + c.tile_s - 1) / c.tile_s;
  }
  if (bad) atomicOr(&s_bad, 1);
  for (int q = 0; q < 4; ++q) sc[q][tid] = acc[q];
  __syncthreads();
  // inclusive Hillis-Steele scan of the per-thread sums
  for (int d = 1; d < nt; d <<= 1) {
    long long v[4];
    for (int q = 0; q < 4; ++q) v[q] = (tid >= d) ? sc[q][tid - d] : 0;
    __syncthreads();
    for (int q = 0; q < 4; ++q) sc[q][tid] += v[q];
    __syncthreads();
  }
  long long run[4];
  for (int q = 0; q < 4; ++q) run[q] = (tid > 0) ? sc[q][tid - 1] : 0;
  for (int s = s0; s < s1; ++s) {
    const int r = c.in_ratio ? c.in_ratio[s] : c.uniform_ratio;
    const int n = c.in_nslow ? c.in_nslow[s] : c.uniform_nslow;
    const int rr = max(r, 1), nn = max(n, 1);
    c.meta.ratio[s] = r;
    c.meta.nslow[s] = n;
    c.meta.off_slow[s] = run[0];
    c.meta.off_fast[s] = run[1];
    c.meta.tile_off_f[s] = run[2];
    c.meta.tile_off_s[s] = run[3];
    run[0] += nn;
    run[1] += (long long)nn * rr;
    run[2] += (nn + c.tile_f - 1) / c.tile_f;
    run[3] += (nn + c.tile_s - 1) / c.tile_s;
  }
  __syncthreads();
  if (tid == nt - 1) {
    const bool ok = !s_bad && sc[0][nt - 1] == c.total_slow && sc[1][nt - 1] == c.total_fast;
    c.meta.off_slow[c.n_seq] = sc[0][nt - 1];
    c.meta.off_fast[c.n_seq] = sc[1][nt - 1];
    c.meta.tile_off_f[c.n_seq] = sc[2][nt - 1];
    c.meta.tile_off_s[c.n_seq] = sc[3][nt - 1];
    c.ctr->total_tiles_f = ok ? sc[2][nt - 1] : 0;
    c.ctr->total_tiles_s = ok ? sc[3][nt - 1] : 0;
    c.ctr->call_ok = ok ? 1u : 0u;
    if (!ok) atomicOr(&c.ctr->err, DEVERR_META);
  }
}

// ---------------------------------------------------------------------------
// warp-cooperative small dense products with runtime sizes.
// out (R x C, row-major) = alpha * op(A) op(B) + (ADD ? ADD : 0); op(A) R x K.
// tA: A stored K x R; tB: B stored C x K.  No barrier.
__device__ void w_mm(int R, int K, int C, double* out, const double* A, bool tA, const double* B, bool tB,
                     const double* ADD, double alpha, int lane) {
  for (int e = lane; e < R * C; e += 32) {
    const int r = e / C, c = e - (e / C) * C;
    double s = 0.0;
    for (int k = 0; k < K; ++k) {
      const double a = tA ? A[k * R + r] : A[r * K + k];
      const double b = tB ? B[c * K + k] : B[k * C + c];
      s = fma(a, b, s);
    }
    out[e] = ADD ? fma(alpha, s, ADD[e]) : alpha * s;
  }
}
// in-place symmetrisation of an n x n matrix: upper triangle and mirror take
// the mean of the two entries.  Lanes own (r, c) with r < c; ends with a barrier.
__device__ void w_sym(int n, double* X, int lane) {
  __syncwarp();
  for (int e = lane; e < n * n; e += 32) {
    const int r = e / n, c = e - (e / n) * n;
    if (r < c) {
      const double v = 0.5 * (X[r * n + c] + X[c * n + r]);
      X[r * n + c] = v;
      X[c * n + r] = v;
    }
  }
  __syncwarp();
}

// inverse of an n x n matrix (n <= 8) by Gauss-Jordan with partial pivoting,
// on lane 0 (tiny).  a is overwritten.  Returns false on a zero pivot.
__device__ bool small_inverse(int n, double* a, double* inv) {
  bool ok = true;
  for (int i = 0; i < n * n; ++i) inv[i] = (i / n == i % n) ? 1.0 : 0.0;
  for (int s = 0; s < n; ++s) {
    int p = s;
    for (int r = s + 1; r < n; ++r)
      if (fabs(a[r * n + s]) > fabs(a[p * n + s])) p = r;
    if (!(fabs(a[p * n + s]) > 0.0)) { ok = false; continue; }
    if (p != s)
      for (int c = 0; c < n; ++c) {
        double t = a[s * n + c]; a[s * n + c] = a[p * n + c]; a[p * n + c] = t;
        t = inv[s * n + c]; inv[s * n + c] = inv[p * n + c]; inv[p * n + c] = t;
      }
    const double d = 1.0 / a[s * n + s];
    for (int c = 0; c < n; ++c) { a[s * n + c] *= d; inv[s * n + c] *= d; }
    for (int r = 0; r < n; ++r)
      if (r != s) {
        const double f = a[r * n + s];
        if (f != 0.0)
          for (int c = 0; c < n; ++c) {
            a[r * n + c] = fma(-f, a[s * n + c], a[r * n + c]);
            inv[r * n + c] = fma(-f, inv[s * n + c], inv[r * n + c]);
          }
      }
  }
  return ok;
}

// Shared-memory footprint of precompute_kernel: inputs and per-warp scratch,
// plus the A^i, S_q, Qc_i and V_i tables when they fit.
constexpr int PRE_BASE = 64 + 64 + 32 + 16 + 64 + 8 + 8 + 64 + 4 * 6 * 64;  // doubles
constexpr size_t PRE_SMEM_CAP = 200 * 1024;
inline size_t precompute_table_doubles(int n, int L) { return (size_t)(4 * L + 1) * n * n; }

__global__ void __launch_bounds__(128) precompute_kernel(Ctx c, int tables_in_smem) {
  extern __shared__ __align__(16) double dsm[];
  if (!c.ctr->call_ok) return;
  const int s = blockIdx.x;
  const int n = c.nx, m = c.ny, nn = n * n, l = c.meta.ratio[s];
  const ModelLayout L = c.ml;
  double* md = c.model + (long long)s * L.stride;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, tid = threadIdx.x, nt = blockDim.x;
  double* sA = dsm;
  double* sQ = sA + 64;
  double* sH = sQ + 64;
  double* sR = sH + 32;
  double* sP0 = sR + 16;
  double* sm0 = sP0 + 64;
  double* sy0 = sm0 + 8;
  double* sT = sy0 + 8;          // sum_{i=1..l} A^i
  double* scr = sT + 64;         // per-warp scratch: 6 matrices of 64
  double* wb = scr + warp * 6 * 64;
  double *Ap, *Sp, *Qp, *Vp;
  if (tables_in_smem) {
    Ap = dsm + PRE_BASE;
    Sp = Ap + (size_t)(l + 1) * nn;
    Qp = Sp + (size_t)l * nn;
    Vp = Qp + (size_t)l * nn;
  } else {
    Ap = md + L.Apow;
    Sp = md + L.Ssc;
    Qp = md + L.Qc;
    Vp = md + L.Vsc;
  }
  __shared__ int s_ok;
  {
    const double* F = c.F + (long long)s * nn;
    const double* Q = c.Q + (long long)s * nn;
    const double* H = c.H + (long long)s * m * n;
    const double* R = c.R + (long long)s * m * m;
    const double* P0 = c.P0 + (long long)s * nn;
    const double* m0 = c.m0 + (long long)s * n;
    const double* y0 = c.y + c.meta.off_slow[s] * m;
    for (int e = tid; e < nn; e += nt) {
      const int r = e / n, q = e - (e / n) * n;
      sA[e] = F[e];
      sQ[e] = 0.5 * (Q[e] + Q[q * n + r]);
      md[L.Q + e] = sQ[e];
      sP0[e] = P0[e];
      Ap[e] = (r == q) ? 1.0 : 0.0;
      Ap[nn + e] = F[e];
    }
    for (int e = tid; e < m * n; e += nt) sH[e] = H[e];
    for (int e = tid; e < m * m; e += nt) sR[e] = R[e];
    for (int e = tid; e < n; e += nt) sm0[e] = m0[e];
    for (int e = tid; e < m; e += nt) sy0[e] = y0[e];
    if (tid == 0) s_ok = 1;
  }
  __syncthreads();
  // --- A^i for i = 1..l by doubling: A^{h+t} = A^h A^t, t = 1..h, per round
  for (int h = 1; h < l; h *= 2) {
    const int cnt = min(h, l - h);
    for (int t = warp; t < cnt; t += 4)
      w_mm(n, n, n, Ap + (size_t)(h + 1 + t) * nn, Ap + (size_t)h * nn, false, Ap + (size_t)(1 + t) * nn, false,
           nullptr, 1.0, lane);
    __syncthreads();
  }
  // --- terms A^r Q A^{rT} (r = 0..l-1) into the Qc table, all warps
  for (int r = warp; r < l; r += 4) {
    double* t = wb;
    w_mm(n, n, n, t, Ap + (size_t)r * nn, false, sQ, false, nullptr, 1.0, lane);
    __syncwarp();
    w_mm(n, n, n, Qp + (size_t)r * nn, t, false, Ap + (size_t)r * nn, true, nullptr, 1.0, lane);
    __syncwarp();
  }
  __syncthreads();
  // --- running sums: S_q = sum_{j<=q} A^j (q < l), sum_{i=1..l} A^i, and
  //     Qc_i = sum_{r<i} A^r Q A^rT (symmetric: one thread per upper-triangle pair)
  for (int e = tid; e < nn; e += nt) {
    const int r = e / n, q = e - (e / n) * n;
    double acc = (r == q) ? 1.0 : 0.0;
    Sp[e] = acc;
    for (int j = 1; j < l; ++j) {
      acc += Ap[(size_t)j * nn + e];
      Sp[(size_t)j * nn + e] = acc;
    }
    sT[e] = acc + Ap[(size_t)l * nn + e] - ((r == q) ? 1.0 : 0.0);
  }
  for (int e = tid; e < nn; e += nt) {
    const int r = e / n, q = e - (e / n) * n;
    if (r > q) continue;
    double acc = 0.0;
    for (int j = 0; j < l; ++j) {
      acc += 0.5 * (Qp[(size_t)j * nn + r * n + q] + Qp[(size_t)j * nn + q * n + r]);
      Qp[(size_t)j * nn + r * n + q] = acc;
      Qp[(size_t)j * nn + q * n + r] = acc;
    }
  }
  __syncthreads();
  // --- V chain (warp 0):  V_1 = Q S_{l-1}^T,  V_i = A V_{i-1} + Q S_{l-i}^T
  //     Cov(e_i, e_l) = Qc_i A^{(l-i)T} (warps 1..3);  C_bar = H sum A^i (warp 1)
  if (warp == 0) {
    double* t = wb;
    w_mm(n, n, n, Vp, sQ, false, Sp + (size_t)(l - 1) * nn, true, nullptr, 1.0, lane);
    __syncwarp();
    for (int i = 2; i <= l; ++i) {
      w_mm(n, n, n, t, sA, false, Vp + (size_t)(i - 2) * nn, false, nullptr, 1.0, lane);
      __syncwarp();
      w_mm(n, n, n, Vp + (size_t)(i - 1) * nn, sQ, false, Sp + (size_t)(l - i) * nn, true, t, 1.0, lane);
      __syncwarp();
    }
  } else {
    if (warp == 1) w_mm(m, n, n, md + L.Cb, sH, false, sT, false, nullptr, 1.0, lane);
    for (int i = warp; i <= l; i += 3)
      w_mm(n, n, n, md + L.Ql + (size_t)(i - 1) * nn, Qp + (size_t)(i - 1) * nn, false, Ap + (size_t)(l - i) * nn,
           true, nullptr, 1.0, lane);
  }
  __syncthreads();
  // --- V_i H^T (all warps); tables to global when they were in shared memory
  for (int i = warp + 1; i <= l; i += 4)
    w_mm(n, n, m, md + L.VH + (size_t)(i - 1) * n * m, Vp + (size_t)(i - 1) * nn, false, sH, true, nullptr, 1.0,
         lane);
  if (tables_in_smem) {
    for (size_t e = tid; e < (size_t)(l + 1) * nn; e += nt) md[L.Apow + e] = Ap[e];
    for (size_t e = tid; e < (size_t)l * nn; e += nt) md[L.Qc + e] = Qp[e];
  }
  __syncthreads();
  // --- slow-model constants and the first filter element (warp 0)
  if (warp == 0) {
    double* Vs = wb;          // sum_i V_i = Var(sum e)
    double* t = wb + 64;
    double* MQM = wb + 128;   // m x m
    double* Rxi = wb + 192;
    double* wk = wb + 256;
    double* wk2 = wb + 320;
    for (int e = lane; e < nn; e += 32) {
      double v = 0.0;
      for (int i = 0; i < l; ++i) v += Vp[(size_t)i * nn + e];
      Vs[e] = v;
    }
    w_sym(n, Vs, lane);
    w_mm(m, n, n, t, sH, false, Vs, false, nullptr, 1.0, lane);  // H Vs (m x n)
    __syncwarp();
    w_mm(m, n, m, MQM, t, false, sH, true, sR, 1.0, lane);        // R_x = H Vs H^T + R
    w_sym(m, MQM, lane);
    for (int e = lane; e < m * m; e += 32) md[L.Rx + e] = MQM[e];
    __syncwarp();
    if (lane == 0) {
      for (int e = 0; e < m * m; ++e) wk[e] = MQM[e];
      if (!small_inverse(m, wk, Rxi)) s_ok = 0;
    }
    __syncwarp();
    w_sym(m, Rxi, lane);
    const double* GQM = md + L.VH + (size_t)(l - 1) * n * m;  // G Q~ M^T = V_l H^T
    const double* Al = Ap + (size_t)l * nn;
    const double* Cb = md + L.Cb;
    const double* Qcl = Qp + (size_t)(l - 1) * nn;
    w_mm(n, m, m, md + L.K, GQM, false, Rxi, false, nullptr, 1.0, lane);   // K
    w_mm(n, m, m, md + L.Cr, Cb, true, Rxi, false, nullptr, 1.0, lane);    // C_bar^T R_x^-1
    __syncwarp();
    w_mm(n, m, n, md + L.Fc, md + L.K, false, Cb, false, Al, -1.0, lane);  // A^l - K C_bar
    w_mm(n, m, n, t, md + L.K, false, GQM, true, Qcl, -1.0, lane);
    w_sym(n, t, lane);
    for (int e = lane; e < nn; e += 32) md[L.Dc + e] = t[e];              // Q_bar - K GQM^T
    __syncwarp();
    w_mm(n, m, n, t, md + L.Cr, false, Cb, false, nullptr, 1.0, lane);
    w_sym(n, t, lane);
    for (int e = lane; e < nn; e += 32) md[L.Jc + e] = t[e];              // C_bar^T R_x^-1 C_bar
    __syncwarp();
    // first element: one IMKF step from (m0, P0) with y_1 (Eq. 9, 12)
    double* AP = t;           // A^l P0
    double* cross = wk2;      // A^l P0 C_bar^T + G Q~ M^T   (n x m)
    double* S1 = MQM;         // C_bar P0 C_bar^T + R_x      (m x m)
    double* S1i = Rxi;
    double* CP = wk;          // C_bar P0 (m x n)
    w_mm(n, n, n, AP, Al, false, sP0, false, nullptr, 1.0, lane);
    w_mm(m, n, n, CP, Cb, false, sP0, false, nullptr, 1.0, lane);
    __syncwarp();
    w_mm(n, n, m, cross, AP, false, Cb, true, GQM, 1.0, lane);
    w_mm(m, n, m, S1, CP, false, Cb, true, md + L.Rx, 1.0, lane);
    w_sym(m, S1, lane);
    double* w1 = scr + 1 * 6 * 64;  // warp 1 scratch is free now
    double* Lg = w1;                // n x m gain
    double* tmp = w1 + 64;
    double* innov = w1 + 128;
    double* P1 = w1 + 192;
    double* P1o = w1 + 256;
    if (lane == 0) {
      for (int e = 0; e < m * m; ++e) tmp[e] = S1[e];
      if (!small_inverse(m, tmp, S1i)) s_ok = 0;
    }
    __syncwarp();
    w_mm(n, m, m, Lg, cross, false, S1i, false, nullptr, 1.0, lane);
    for (int j = lane; j < m; j += 32) {
      double v = sy0[j];
      for (int q = 0; q < n; ++q) v = fma(-Cb[j * n + q], sm0[q], v);
      innov[j] = v;
    }
    __syncwarp();
    for (int r = lane; r < n; r += 32) {
      double v = 0.0;
      for (int q = 0; q < n; ++q) v = fma(Al[r * n + q], sm0[q], v);
      for (int j = 0; j < m; ++j) v = fma(Lg[r * m + j], innov[j], v);
      md[L.m1 + r] = v;
    }
    w_mm(n, n, n, P1, AP, false, Al, true, Qcl, 1.0, lane);
    __syncwarp();
    w_mm(n, m, n, P1o, Lg, false, cross, true, P1, -1.0, lane);
    w_sym(n, P1o, lane);
    for (int e = lane; e < nn; e += 32) md[L.P1 + e] = P1o[e];
    __syncwarp();
    if (lane == 0 && !s_ok) atomicOr(&c.ctr->err, DEVERR_SINGULAR);
  }
}

// ev (optional): three events recorded before the metadata kernel, after it
// and after the constants kernel.
int launch_meta_and_precompute(const Ctx& c, cudaStream_t st, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], st);
  meta_kernel<<<1, 1024, 0, st>>>(c);
  if (ev) cudaEventRecord(ev[1], st);
  const size_t tab = precompute_table_doubles(c.nx, c.max_ratio) * sizeof(double);
  const size_t base = PRE_BASE * sizeof(double);
  const int in_smem = base + tab <= PRE_SMEM_CAP ? 1 : 0;
  const size_t smem = base + (in_smem ? tab : 0);
  if (smem > 48 * 1024) cudaFuncSetAttribute(precompute_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  precompute_kernel<<<c.n_seq, 128, smem, st>>>(c, in_smem);
  if (ev) cudaEventRecord(ev[2], st);
  return cudaGetLastError() == cudaSuccess ? SRTM_OK : SRTM_ERR_CUDA;
}

}  // namespace srtm
