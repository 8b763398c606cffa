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

// |x| as an order-preserving integer (IEEE magnitudes compare like their bit
// patterns), so pivot selection uses the integer pipe, not the FP64 pipe.
__device__ __forceinline__ unsigned long long mag_key(double x) {
  return (unsigned long long)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ unsigned long long mag_key(float x) {
  return (unsigned long long)((unsigned)__float_as_int(x) & 0x7fffffffu);
}
// zero, infinite or NaN pivot, tested on the bit pattern
__device__ __forceinline__ bool bad_pivot(double x) {
  const unsigned long long m = mag_key(x);
  return m == 0ull || m >= 0x7ff0000000000000ull;
}
__device__ __forceinline__ bool bad_pivot(float x) {
  const unsigned long long m = mag_key(x);
  return m == 0ull || m >= 0x7f800000ull;
}

// In-place Gauss-Jordan inversion with partial (row) pivoting of the NX x NX
// matrix a (row-major, shared memory).  Step s swaps the pivot row into place
// and applies
//   a_ss <- 1/p,  a_sc <- a_sc/p,  a_rs <- -a_rs/p,  a_rc <- a_rc - a_rs a_sc/p,
// which leaves (P M)^{-1} after NX steps; undoing the row interchanges on the
// columns (last step first) gives M^{-1}.  Every lane scans the pivot column
// itself, so the choice needs no exchange.  Returns false on a zero or
// non-finite pivot (the step then uses 1 to stay finite).
template <int NX, int G, class TS>
__device__ __forceinline__ bool g_gauss_jordan(const Grp<G>& g, TS* a) {
  constexpr int NN = NX * NX, EPL = (NN + G - 1) / G;
  bool ok = true;
  int pv[NX];
#pragma unroll
  for (int s = 0; s < NX; ++s) {
    int p = s;
    unsigned long long best = mag_key(a[s * NX + s]);
#pragma unroll
    for (int r = s + 1; r < NX; ++r) {
      const unsigned long long v = mag_key(a[r * NX + s]);
      if (v > best) { best = v; p = r; }
    }
    pv[s] = p;
    g.sync();
    if (p != s) {
      for (int c = g.lane; c < NX; c += G) {
        const TS t = a[s * NX + c];
        a[s * NX + c] = a[p * NX + c];
        a[p * NX + c] = t;
      }
    }
    g.sync();
    TS piv = a[s * NX + s];
    if (bad_pivot(piv)) { ok = false; piv = TS(1); }
    const TS inv = TS(1) / piv;
    TS v[EPL], ars[EPL], asc[EPL];
#pragma unroll
    for (int j = 0; j < EPL; ++j) {
      const int e = j * G + g.lane;
      if (e < NN) {
        const int r = e / NX, c = e - (e / NX) * NX;
        v[j] = a[e];
        ars[j] = a[r * NX + s];
        asc[j] = a[s * NX + c];
      }
    }
    g.sync();
#pragma unroll
    for (int j = 0; j < EPL; ++j) {
      const int e = j * G + g.lane;
      if (e < NN) {
        const int r = e / NX, c = e - (e / NX) * NX;
        TS out;
        if (r == s) out = (c == s) ? inv : v[j] * inv;
        else if (c == s) out = -ars[j] * inv;
        else out = fma(-ars[j] * inv, asc[j], v[j]);
        a[e] = out;
      }
    }
    g.sync();
  }
#pragma unroll
  for (int s = NX - 1; s >= 0; --s) {
    if (pv[s] != s) {
      for (int r = g.lane; r < NX; r += G) {
        const TS t = a[r * NX + s];
        a[r * NX + s] = a[r * NX + pv[s]];
        a[r * NX + pv[s]] = t;
      }
      g.sync();
    }
  }
  return ok;
}

// Inverse of an NX x NX matrix, NX <= 4, by the adjugate: entries are
// cofactors over the determinant, so a single division is needed (a pivoted
// elimination needs one per pivot, and a float64 division costs about six
// FMAs on this part).  For NX = 4 the cofactors come from the Laplace
// expansion by complementary 2x2 minors of rows (0,1) and (2,3):
//   s_u = a_0p a_1q - a_1p a_0q,  c_u = a_2p a_3q - a_3p a_2q,
//   (p,q) in (0,1),(0,2),(0,3),(1,2),(1,3),(2,3) for u = 0..5.
// When every lane of the group holds one entry (G >= NX*NX), the
// determinant is the expansion along column 0, det = sum_c a_c0 C_c0, whose
// cofactors C_c0 are the unscaled entries (0, c) of the inverse that lanes
// 0..NX-1 have just formed: one product per lane and a two-level shuffle sum
// instead of a full determinant on every lane (on this part a float64
// instruction costs the same whatever its active lanes).
// In place on a (shared memory); mn holds the 12 minors.  Returns false on
// a zero or non-finite determinant (then divides by one to stay finite).
template <int NX, int G, class TS>
__device__ __forceinline__ bool g_small_inverse(const Grp<G>& g, TS* a, TS* mn) {
  static_assert(NX >= 1 && NX <= 4, "adjugate inverse is for NX <= 4");
  constexpr int NN = NX * NX, EPL = (NN + G - 1) / G;
  constexpr bool SPLIT_DET = (NX >= 3) && (G >= NN) && (G >= 4);
  bool ok = true;
  if (NX == 4) {
    for (int u = g.lane; u < 12; u += G) {
      const int r0 = u < 6 ? 0 : 2, v = u < 6 ? u : u - 6;
      const int p = v < 3 ? 0 : (v < 5 ? 1 : 2);
      const int q = v < 3 ? v + 1 : (v < 5 ? v - 1 : 3);
      mn[u] = fma(a[r0 * 4 + p], a[(r0 + 1) * 4 + q], -a[(r0 + 1) * 4 + p] * a[r0 * 4 + q]);
    }
    g.sync();
  }
  // unscaled inverse entries (cofactors of the transposed positions)
  TS out[EPL];
#pragma unroll
  for (int j = 0; j < EPL; ++j) {
    const int e = j * G + g.lane;
    TS v = TS(0);
    if (e < NN) {
      const int r = e / NX, col = e - (e / NX) * NX;
      if (NX == 1) {
        v = TS(1);
      } else if (NX == 2) {
        v = (r == col) ? a[(1 - r) * 3] : -a[r * 2 + col];
      } else if (NX == 3) {
        // inv[r][col] = cofactor(col, r): minor without row col and column r
        const int i0 = col == 0 ? 1 : 0, i1 = col == 2 ? 1 : 2;
        const int j0 = r == 0 ? 1 : 0, j1 = r == 2 ? 1 : 2;
        v = a[i0 * 3 + j0] * a[i1 * 3 + j1] - a[i0 * 3 + j1] * a[i1 * 3 + j0];
        if ((r + col) & 1) v = -v;
      } else {
        const int arow = col ^ 1;
        const TS* mins = col < 2 ? mn + 6 : mn;
        const int code = r == 0 ? 0x543 : (r == 1 ? 0x521 : (r == 2 ? 0x420 : 0x310));
        const int k0 = r > 0 ? 0 : 1, k1 = r > 1 ? 1 : 2, k2 = r > 2 ? 2 : 3;
        v = a[arow * 4 + k0] * mins[(code >> 8) & 15];
        v = fma(-a[arow * 4 + k1], mins[(code >> 4) & 15], v);
        v = fma(a[arow * 4 + k2], mins[code & 15], v);
        if (((col & 1) != 0) != ((r & 1) != 0)) v = -v;
      }
    }
    out[j] = v;
  }
  TS det;
  if constexpr (SPLIT_DET) {
    // lanes 0..NX-1 hold C_c0 (row 0 of the unscaled inverse, c = lane)
    TS t = (g.lane < NX) ? a[g.lane * NX] * out[0] : TS(0);
    t += __shfl_xor_sync(g.mask, t, 1);
    t += __shfl_xor_sync(g.mask, t, 2);
    det = __shfl_sync(g.mask, t, (int)(threadIdx.x & 31) & ~(G - 1));
  } else if (NX == 4) {
    const TS* sm = mn;
    const TS* cm = mn + 6;
    det = sm[0] * cm[5] - sm[1] * cm[4] + sm[2] * cm[3] + sm[3] * cm[2] - sm[4] * cm[1] + sm[5] * cm[0];
  } else if (NX == 3) {
    det = a[0] * (a[4] * a[8] - a[5] * a[7]) - a[1] * (a[3] * a[8] - a[5] * a[6]) + a[2] * (a[3] * a[7] - a[4] * a[6]);
  } else if (NX == 2) {
    det = a[0] * a[3] - a[1] * a[2];
  } else {
    det = a[0];
  }
  if (bad_pivot(det)) { ok = false; det = TS(1); }
  const TS id = TS(1) / det;
  g.sync();
#pragma unroll
  for (int j = 0; j < EPL; ++j) {
    const int e = j * G + g.lane;
    if (e < NN) a[e] = out[j] * id;
  }
  g.sync();
  return ok;
}

// M^{-1} in place: adjugate for NX <= 4, pivoted Gauss-Jordan above.
template <int NX, int G, class TS>
__device__ __forceinline__ bool g_inverse(const Grp<G>& g, TS* a, TS* mn) {
  if constexpr (NX <= 4) return g_small_inverse<NX, G, TS>(g, a, mn);
  else return g_gauss_jordan<NX, G, TS>(g, a);
}

// ---------------------------------------------------------------------------
// Filter operator of Eq. (27):  o = a (x) b  with a = (F_i,d_i,D_i,eta_i,J_i),
// b = (F_j,...).  With M = I + D_i J_j (so that I + J_j D_i = M^T for
// symmetric D, J) and W = F_j M^{-1}, V = M^{-1} F_i:
//   F_ij = W F_i,                 d_ij = W (d_i + D_i eta_j) + d_j,
//   D_ij = W D_i F_j^T + D_j,     eta_ij = V^T (eta_j - J_j d_i) + eta_i,
//   J_ij = V^T J_j F_i + J_i.
// M is inverted in TS (float64 in the mixed mode): by the adjugate for
// NX <= 4, by pivoted Gauss-Jordan above; everything else is in T.  D_ij and
// J_ij are written exactly symmetric.  (A generic element on the right takes
// the rank-m form of this operator instead, g_filter_combine_rank.)
// prefix=true: a is a prefix that contains the first element (F = 0, eta = 0,
// J = 0 exactly, Eq. 25 with k = 1), so only d_ij, D_ij are formed and F_ij,
// eta_ij, J_ij are zero.
// Scratch: sc (T) 5NN + 2NX, sm (TS) NN + 12.
// ---------------------------------------------------------------------------
template <int NX, int G, class T, class TS>
__device__ __forceinline__ bool g_filter_combine(const Grp<G>& g, T* o, const T* a, const T* b, T* sc, TS* Ma,
                                                 bool prefix) {
  using L = FL<NX>;
  constexpr int NN = NX * NX;
  T *W = sc, *V = sc + NN, *WD = sc + 2 * NN, *JF = sc + 3 * NN, *t1 = sc + 4 * NN, *t2 = sc + 4 * NN + NX;
  T* Mi = sc + 4 * NN + 2 * NX;
  // M = I + D_i J_j, formed in T and held in TS for the solve
#pragma unroll
  for (int e0 = 0; e0 < NN; e0 += G) {
    const int e = e0 + g.lane;
    if (e < NN) {
      const int r = e / NX, c = e - (e / NX) * NX;
      T s = (r == c) ? T(1) : T(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) s = fma(a[L::D + r * NX + k], b[L::J + k * NX + c], s);
      Ma[e] = (TS)s;
    }
  }
  // t1 = d_i + D_i eta_j ;  t2 = eta_j - J_j d_i
  g_mv<NX, G, false, T>(g, t1, a + L::D, b + L::e, a + L::d);
  if (!prefix) g_mv<NX, G, false, T>(g, t2, b + L::J, a + L::d, b + L::e, T(-1));
  g.sync();
  const bool ok = g_inverse<NX, G, TS>(g, Ma, Ma + NN);
  const T* Minv = (const T*)Ma;
  if (sizeof(T) != sizeof(TS)) {  // one rounding of M^{-1} to T
    for (int e = g.lane; e < NN; e += G) Mi[e] = (T)Ma[e];
    g.sync();
    Minv = Mi;
  }
  // W = F_j M^{-1} ; V = M^{-1} F_i
  g_mm<NX, G, false, false, T>(g, W, b + L::F, Minv, (const T*)nullptr);
  if (!prefix) g_mm<NX, G, false, false, T>(g, V, Minv, a + L::F, (const T*)nullptr);
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
