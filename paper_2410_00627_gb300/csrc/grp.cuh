// grp.cuh -- small-matrix arithmetic spread over a group of G lanes of one
// warp, with the operands in shared memory.
//
// On sm_103a a float64 warp instruction occupies the FP64 pipe of its
// sub-partition for ~76 cycles whatever its active mask, so a combine
// computed by one lane costs as much issue time as 32 of them.  The scans
// are latency-bound (a chain of dependent combines), so each element is
// owned by G lanes: lane g computes the entries e = g, g+G, ... of every
// product.  G is 4 for nx <= 2, 16 for nx <= 4 and 32 above (entries
// round-robin over the lanes).  Every routine leaves its results in shared
// memory and ends with a group barrier unless stated otherwise.
#pragma once
#include "srtm_internal.cuh"

namespace srtm {

template <int NX>
struct GroupSize {
  static constexpr int value = NX == 1 ? 1 : (NX <= 2 ? 4 : (NX <= 4 ? 16 : 32));
};

template <int G>
struct Grp {
  int lane;
  unsigned mask;
  __device__ __forceinline__ Grp() {
    const int l = threadIdx.x & 31;
    lane = l & (G - 1);
    mask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << (l & ~(G - 1)));
  }
  __device__ __forceinline__ void sync() const { __syncwarp(mask); }
};

// row/column of the u-th entry of the upper triangle (row-major order)
template <int NX>
__device__ __forceinline__ void tri_rc(int u, int& r, int& c) {
  r = 0;
  while (u >= NX - r) { u -= NX - r; ++r; }
  c = r + u;
}

// C = op(A) op(B) (+ ADD), NX x NX, accumulated in TACC.  No barrier.
template <int NX, int G, bool TA, bool TB, class TACC, class TC, class T1, class T2, class T3>
__device__ __forceinline__ void g_mm(const Grp<G>& g, TC* C, const T1* A, const T2* B, const T3* ADD,
                                     TACC sign = TACC(1)) {
  constexpr int NN = NX * NX;
#pragma unroll
  for (int e0 = 0; e0 < NN; e0 += G) {
    const int e = e0 + g.lane;
    if (e < NN) {
      const int r = e / NX, c = e - (e / NX) * NX;
      TACC s = TACC(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) {
        const TACC a = (TACC)(TA ? A[k * NX + r] : A[r * NX + k]);
        const TACC b = (TACC)(TB ? B[c * NX + k] : B[k * NX + c]);
        s = fma(a, b, s);
      }
      C[e] = ADD ? (TC)fma(sign, s, (TACC)ADD[e]) : (TC)(sign * s);
    }
  }
}

// Symmetric result: C = op(A) op(B) + ADD computed on the upper triangle and
// mirrored, so C is exactly symmetric.  No barrier.
template <int NX, int G, bool TA, bool TB, class TACC, class TC, class T1, class T2, class T3>
__device__ __forceinline__ void g_mm_sym(const Grp<G>& g, TC* C, const T1* A, const T2* B, const T3* ADD) {
  constexpr int NT = NX * (NX + 1) / 2;
#pragma unroll
  for (int u0 = 0; u0 < NT; u0 += G) {
    const int u = u0 + g.lane;
    if (u < NT) {
      int r, c;
      tri_rc<NX>(u, r, c);
      TACC s = TACC(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) {
        const TACC a = (TACC)(TA ? A[k * NX + r] : A[r * NX + k]);
        const TACC b = (TACC)(TB ? B[c * NX + k] : B[k * NX + c]);
        s = fma(a, b, s);
      }
      // ADD is symmetric up to rounding; use the mean of its two entries
      const TACC add = ADD ? (TACC)0.5 * ((TACC)ADD[r * NX + c] + (TACC)ADD[c * NX + r]) : TACC(0);
      C[r * NX + c] = (TC)(s + add);
      C[c * NX + r] = (TC)(s + add);
    }
  }
}

// y = op(A) x (+ ADD) on lanes < NX.  No barrier.
template <int NX, int G, bool TA, class TACC, class TY, class T1, class T2, class T3>
__device__ __forceinline__ void g_mv(const Grp<G>& g, TY* y, const T1* A, const T2* x, const T3* ADD,
                                     TACC sign = TACC(1)) {
#pragma unroll
  for (int r0 = 0; r0 < NX; r0 += G) {
    const int r = r0 + g.lane;
    if (r < NX) {
      TACC s = TACC(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) s = fma((TACC)(TA ? A[k * NX + r] : A[r * NX + k]), (TACC)x[k], s);
      y[r] = ADD ? (TY)fma(sign, s, (TACC)ADD[r]) : (TY)(sign * s);
    }
  }
}

template <int NX, int G, class T, class TS>
__device__ __forceinline__ void g_copy(const Grp<G>& g, T* dst, const TS* src, int count) {
  for (int e = g.lane; e < count; e += G) dst[e] = (T)src[e];
}

// Gauss-Jordan elimination with partial pivoting on the augmented NX x 2NX
// matrix Ma = [M | I] (row-major, leading dimension 2NX): on return the right
// half holds M^{-1}.  Every lane of the group reads the pivot column itself,
// so the pivot choice needs no exchange.  Returns false on a zero or
// non-finite pivot (the step then divides by one to stay finite).
template <int NX, int G, class TS>
__device__ __forceinline__ bool g_gauss_jordan(const Grp<G>& g, TS* Ma) {
  constexpr int W = 2 * NX, NE = NX * W, EPL = (NE + G - 1) / G;
  bool ok = true;
#pragma unroll 1
  for (int s = 0; s < NX; ++s) {
    int p = s;
    TS best = fabs(Ma[s * W + s]);
    for (int r = s + 1; r < NX; ++r) {
      const TS v = fabs(Ma[r * W + s]);
      if (v > best) { best = v; p = r; }
    }
    g.sync();
    if (p != s) {
      for (int c = g.lane; c < W; c += G) {
        const TS t = Ma[s * W + c];
        Ma[s * W + c] = Ma[p * W + c];
        Ma[p * W + c] = t;
      }
    }
    g.sync();
    TS piv = Ma[s * W + s];
    if (!(fabs(piv) > TS(0)) || !isfinite(piv)) { ok = false; piv = TS(1); }
    const TS inv = TS(1) / piv;
    TS v[EPL], f[EPL], rs[EPL];
#pragma unroll
    for (int j = 0; j < EPL; ++j) {
      const int e = j * G + g.lane;
      if (e < NE) {
        const int r = e / W, c = e - (e / W) * W;
        v[j] = Ma[e];
        f[j] = Ma[r * W + s] * inv;
        rs[j] = Ma[s * W + c];
      }
    }
    g.sync();
#pragma unroll
    for (int j = 0; j < EPL; ++j) {
      const int e = j * G + g.lane;
      if (e < NE) {
        const int r = e / W;
        Ma[e] = (r == s) ? v[j] * inv : fma(-f[j], rs[j], v[j]);
      }
    }
    g.sync();
  }
  return ok;
}

// ---------------------------------------------------------------------------
// Filter operator of Eq. (27):  o = a (x) b  with a = (F_i,d_i,D_i,eta_i,J_i),
// b = (F_j,...).  With M = I + D_i J_j (so that I + J_j D_i = M^T for
// symmetric D, J) and W = F_j M^{-1}, V = M^{-1} F_i:
//   F_ij = W F_i,                 d_ij = W (d_i + D_i eta_j) + d_j,
//   D_ij = W D_i F_j^T + D_j,     eta_ij = V^T (eta_j - J_j d_i) + eta_i,
//   J_ij = V^T J_j F_i + J_i.
// M, its inverse, W and V are formed in TS (float64 in the mixed mode); the
// rest in T.  D_ij and J_ij are written exactly symmetric.
// prefix=true: a is a prefix that contains the first element (F = 0, eta = 0,
// J = 0 exactly, Eq. 25 with k = 1), so only d_ij, D_ij are formed and F_ij,
// eta_ij, J_ij are zero.
// Scratch: sc (T) 4NN + 2NX, sm (TS) 2NN.
// ---------------------------------------------------------------------------
template <int NX, int G, class T, class TS>
__device__ __forceinline__ bool g_filter_combine(const Grp<G>& g, T* o, const T* a, const T* b, T* sc, TS* Ma,
                                                 bool prefix) {
  using L = FL<NX>;
  constexpr int NN = NX * NX, W2 = 2 * NX, NE = NX * W2;
  T *W = sc, *V = sc + NN, *WD = sc + 2 * NN, *JF = sc + 3 * NN, *t1 = sc + 4 * NN, *t2 = sc + 4 * NN + NX;
  // [I + D_i J_j | I]
#pragma unroll
  for (int e0 = 0; e0 < NE; e0 += G) {
    const int e = e0 + g.lane;
    if (e < NE) {
      const int r = e / W2, c = e - (e / W2) * W2;
      if (c < NX) {
        TS s = (r == c) ? TS(1) : TS(0);
#pragma unroll
        for (int k = 0; k < NX; ++k) s = fma((TS)a[L::D + r * NX + k], (TS)b[L::J + k * NX + c], s);
        Ma[e] = s;
      } else {
        Ma[e] = (r == c - NX) ? TS(1) : TS(0);
      }
    }
  }
  // t1 = d_i + D_i eta_j ;  t2 = eta_j - J_j d_i
  g_mv<NX, G, false, T>(g, t1, a + L::D, b + L::e, a + L::d);
  if (!prefix) g_mv<NX, G, false, T>(g, t2, b + L::J, a + L::d, b + L::e, T(-1));
  g.sync();
  const bool ok = g_gauss_jordan<NX, G, TS>(g, Ma);
  // W = F_j M^{-1} ; V = M^{-1} F_i
#pragma unroll
  for (int e0 = 0; e0 < NN; e0 += G) {
    const int e = e0 + g.lane;
    if (e < NN) {
      const int r = e / NX, c = e - (e / NX) * NX;
      TS s = TS(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) s = fma((TS)b[L::F + r * NX + k], Ma[k * W2 + NX + c], s);
      W[e] = (T)s;
      if (!prefix) {
        TS v = TS(0);
#pragma unroll
        for (int k = 0; k < NX; ++k) v = fma(Ma[r * W2 + NX + k], (TS)a[L::F + k * NX + c], v);
        V[e] = (T)v;
      }
    }
  }
  g.sync();
  g_mm<NX, G, false, false, T>(g, WD, W, a + L::D, (const T*)nullptr);
  if (!prefix) {
    g_mm<NX, G, false, false, T>(g, o + L::F, W, a + L::F, (const T*)nullptr);
    g_mm<NX, G, false, false, T>(g, JF, b + L::J, a + L::F, (const T*)nullptr);
  }
  g.sync();
  g_mv<NX, G, false, T>(g, o + L::d, W, t1, b + L::d);
  g_mm_sym<NX, G, false, true, T>(g, o + L::D, WD, b + L::F, b + L::D);
  if (!prefix) {
    g_mv<NX, G, true, T>(g, o + L::e, V, t2, a + L::e);
    g_mm_sym<NX, G, true, false, T>(g, o + L::J, V, JF, a + L::J);
  } else {
    for (int e = g.lane; e < NN; e += G) { o[L::F + e] = T(0); o[L::J + e] = T(0); }
    for (int e = g.lane; e < NX; e += G) o[L::e + e] = T(0);
  }
  g.sync();
  return ok;
}

// ---------------------------------------------------------------------------
// Smoother operator of Eq. (30):  o = a (x) b  with a = (E_i,g_i,S_i):
//   E_ij = E_i E_j,  g_ij = E_i g_j + g_i,  S_ij = E_i S_j E_i^T + S_i.
// prefix=true: b is a suffix that contains the last element (E_N = 0,
// Eq. 29), so E_ij = 0.  Scratch: sc (T) NN.
// ---------------------------------------------------------------------------
template <int NX, int G, class T>
__device__ __forceinline__ void g_smoother_combine(const Grp<G>& g, T* o, const T* a, const T* b, T* sc,
                                                   bool prefix) {
  using L = SL<NX>;
  constexpr int NN = NX * NX;
  T* ES = sc;
  g_mm<NX, G, false, false, T>(g, ES, a + L::E, b + L::S, (const T*)nullptr);
  g_mv<NX, G, false, T>(g, o + L::g, a + L::E, b + L::g, a + L::g);
  if (!prefix) g_mm<NX, G, false, false, T>(g, o + L::E, a + L::E, b + L::E, (const T*)nullptr);
  else for (int e = g.lane; e < NN; e += G) o[L::E + e] = T(0);
  g.sync();
  g_mm_sym<NX, G, false, true, T>(g, o + L::S, ES, a + L::E, a + L::S);
  g.sync();
}

}  // namespace srtm
