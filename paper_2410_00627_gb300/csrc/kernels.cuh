// kernels.cuh -- templated device path of the SRTM filter/smoother for one
// state size NX: the two associative scans (Eq. 27 and Eq. 30), the
// per-interval setup (fast-filter blocks and smoother elements, Eq. 17, 29)
// and the fast-rate recovery (Eq. 17, 21).  Instantiated per NX in
// inst_nx*.cu so that the translation units compile in parallel.
#pragma once
#include <cuda_runtime.h>

#include <algorithm>

#include "constants.cuh"
#include "grp.cuh"
#include "seq.cuh"
#include "small.cuh"
#include "srtm_internal.cuh"

namespace srtm {

__host__ __device__ constexpr size_t align16(size_t x) { return (x + 15) / 16 * 16; }

template <int NX>
struct SetupGeom {
  static constexpr int SG = NX == 1 ? 1 : (NX == 2 ? 2 : (NX <= 4 ? 4 : 8));
  static constexpr int NN = NX * NX, NM = NX * MY, UA = NM > NN ? NM : NN;
  // slot layout in TR; Aml, AP1 and P11 reuse Pll, AP and Pm, whose last
  // reads precede them, and AP also holds the 2x2 minors of P^- (NX = 4).
  // Everything from Pll on is dead once the record is written; U1 and P1l
  // are the work arrays of smoother elements formed in TR.
  static constexpr int P = 0, mv = P + NN, X = mv + NX, SUl = X + NM, ml = SUl + NM, Pl = ml + NX, Z = Pl + NN,
                       Pll = Z + NN, AP = Pll + NN, Pm = AP + NN, Sy = Pm + NN, ev = Sy + MY * MY, U1 = ev + MY,
                       P1l = U1 + NM, SLOT = P1l + NN;
  static constexpr int Aml = Pll, AP1 = AP, P11 = Pm;
  // float region of a slot (mixed mode: the smoother elements in float32,
  // so U1 and P1l are not needed), laid over the TR entries from Pll on:
  // float copies of P, Pl, X, SUl, Z, m^f_l, m, then U1 (later A P1l^T, so
  // max(NM, NN) entries), P1l, P11, A m^f_l
  static constexpr int FREG = Pll;
  static constexpr int fP = 0, fPl = fP + NN, fX = fPl + NN, fSUl = fX + NM, fZ = fSUl + NM, fml = fZ + NN,
                       fmv = fml + NX, fU1 = fmv + NX, fP1l = fU1 + UA, fP11 = fP1l + NN, fAml = fP11 + NN,
                       SLOTF = fAml + NX;
  static constexpr int SLOT_MIXED_CORE = U1;                                // TR entries the mixed mode uses
  static constexpr int SLOT_MIXED_FLOAT = FREG + (SLOTF * 4 + 7) / 8;       // end of the float region
  static constexpr int SLOT_MIXED = SLOT_MIXED_CORE > SLOT_MIXED_FLOAT ? SLOT_MIXED_CORE : SLOT_MIXED_FLOAT;
  // the float32 setup of two-point sequences (mixed mode): the float region at
  // the slot's start, followed by float S_y (MY x MY) and innovation (MY), then
  // the TR arrays of the P^- solve from TP on: Pll, AP, Pm, Z
  static constexpr int fSy = SLOTF, fev = fSy + MY * MY, TP = (fev + MY + 1) / 2;
  static constexpr int tPll = TP, tAP = tPll + NN, tPm = tAP + NN, tZ = tPm + NN;
  static_assert(tZ + NN <= SLOT_MIXED, "the float32 setup does not fit the mixed-mode slot");
  // the model's float copies (model table, ModelLayout::Cf): A, Qc_1, Cov(e_1, e_l), V_1 H^T
  static constexpr int cA = 0, cQc = NN, cQl = 2 * NN, cVH = 3 * NN;
  template <class T, class TR>
  __host__ __device__ static constexpr size_t slot_bytes() {
    return (((sizeof(T) != sizeof(TR) ? SLOT_MIXED : SLOT) * sizeof(TR) + 15) / 16) * 16;
  }
};

// The per-interval records of sequence s are read by the recovery unless the
// call takes the two-point form for it.
__device__ __forceinline__ bool records_needed(const Ctx& c, int s) {
  return !(c.bridge && c.model[(long long)s * c.ml.stride + c.ml.bflag] != 0.0);
}

// Smoother element of one interval (Eq. 29 with the fast-filter blocks of
// Eq. 17 for i = 1 and i = l), row r by lane r, in the arithmetic type TE:
//   U_1 = A X + V_1 H^T,  m^f_1 = A m + U_1 kap,
//   P^f_11 = A P A^T + Qc_1 - U_1 S_y^-1 U_1^T,
//   P^f_1l = A (P A^{lT}) + Cov(e_1,e_l) - U_1 (S_y^-1 U_l^T),
//   E = P^f_1l Z,  g = m^f_1 - E A m^f_l,  S = P^f_11 - E A (P^f_1l)^T
// (reading A7 for S); with known inputs m^f_1 gains b_{k,1} and the
// prediction A m^f_l gains B u_{k,l} (b1, bnx; NULL without inputs).
// Inputs: P, Pl, X, SUl, Z, ml, mv (slot arrays) and
// the model's A, Qc_1, Cov(e_1,e_l), V_1 H^T (cA, cQc, cQl, cVH; row-major,
// V_1 H^T with row stride m).  Work arrays: U1 (NX x MY), P1l, P11, Aml and
// AP1 (NX x NX, A P1l^T; may alias U1 when that holds NX x NX entries).
template <int NX, int M, class TE, class TC, class T>
__device__ __forceinline__ void setup_elements(int r, bool row, unsigned mask, int m, bool last, const TE* P,
                                               const TE* Pl, const TE* X, const TE* SUl, const TE* Z, const TE* ml,
                                               const TE* mv, const TC* cA, const TC* cQc, const TC* cQl,
                                               const TC* cVH, const TE (&Si)[MY][MY], const TE (&kap)[MY], TE* U1,
                                               TE* P1l, TE* P11, TE* Aml, TE* AP1, T* se, const double* b1,
                                               const double* bnx) {
  using SLy = SL<NX>;
  constexpr int MM = M > 0 ? M : MY;  // loop bound over the measurement dimension
  if constexpr (M > 0) m = M;
  TE U1r[MY], m1 = TE(0);
  if (row) {
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      TE v = TE(0);
      if (j < m) {
        v = (TE)cVH[r * m + j];
#pragma unroll
        for (int q = 0; q < NX; ++q) v = fma((TE)cA[r * NX + q], X[q * MY + j], v);
      }
      U1r[j] = v;
      U1[r * MY + j] = v;
    }
#pragma unroll
    for (int q = 0; q < NX; ++q) m1 = fma((TE)cA[r * NX + q], mv[q], m1);
#pragma unroll
    for (int j = 0; j < MM; ++j)
      if (j < m) m1 = fma(U1r[j], kap[j], m1);
    TE aml = TE(0);
#pragma unroll
    for (int t = 0; t < NX; ++t) aml = fma((TE)cA[r * NX + t], ml[t], aml);
    if (b1) {  // known inputs: b_{k,1} = B u_{k,0} and the prediction's B u_{k,l}
      m1 += (TE)b1[r];
      aml += (TE)bnx[r];
    }
    Aml[r] = aml;
  }
  __syncwarp(mask);
  if (row) {
    TE US[MY], APr[NX];
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      TE v = TE(0);
#pragma unroll
      for (int jj = 0; jj < MM; ++jj)
        if (jj < m && j < m) v = fma(U1r[jj], Si[jj][j], v);
      US[j] = v;
    }
#pragma unroll
    for (int q = 0; q < NX; ++q) {
      TE v = TE(0);
#pragma unroll
      for (int t = 0; t < NX; ++t) v = fma((TE)cA[r * NX + t], P[t * NX + q], v);
      APr[q] = v;
    }
#pragma unroll
    for (int q = 0; q < NX; ++q) {
      if (q >= r) {
        TE v = (TE)cQc[r * NX + q];
#pragma unroll
        for (int t = 0; t < NX; ++t) v = fma(APr[t], (TE)cA[q * NX + t], v);
#pragma unroll
        for (int j = 0; j < MM; ++j)
          if (j < m) v = fma(-US[j], U1[q * MY + j], v);
        P11[r * NX + q] = v;
        P11[q * NX + r] = v;
      }
      TE w = (TE)cQl[r * NX + q];
#pragma unroll
      for (int t = 0; t < NX; ++t) w = fma((TE)cA[r * NX + t], Pl[t * NX + q], w);
#pragma unroll
      for (int j = 0; j < MM; ++j)
        if (j < m) w = fma(-U1r[j], SUl[j * NX + q], w);
      P1l[r * NX + q] = w;
    }
  }
  __syncwarp(mask);
  if (!last) {
    TE Er[NX];
    if (row) {
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        TE v = TE(0);
#pragma unroll
        for (int t = 0; t < NX; ++t) v = fma(P1l[r * NX + t], Z[t * NX + q], v);
        Er[q] = v;
        se[SLy::E + r * NX + q] = (T)v;
      }
      TE g = m1;
#pragma unroll
      for (int q = 0; q < NX; ++q) g = fma(-Er[q], Aml[q], g);
      se[SLy::g + r] = (T)g;
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        TE v = TE(0);
#pragma unroll
        for (int t = 0; t < NX; ++t) v = fma((TE)cA[r * NX + t], P1l[q * NX + t], v);
        AP1[r * NX + q] = v;
      }
    }
    __syncwarp(mask);
    if (row) {
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        if (q >= r) {
          TE v = P11[r * NX + q];
#pragma unroll
          for (int t = 0; t < NX; ++t) v = fma(-Er[t], AP1[t * NX + q], v);
          se[SLy::S + r * NX + q] = (T)v;
          se[SLy::S + q * NX + r] = (T)v;
        }
      }
    }
  } else if (row) {  // last interval: E_N = 0, g = m^f_{N,1}, S = P^f_{N,1}
    se[SLy::g + r] = (T)m1;
#pragma unroll
    for (int q = 0; q < NX; ++q) {
      se[SLy::E + r * NX + q] = T(0);
      se[SLy::S + r * NX + q] = (T)P11[r * NX + q];
    }
  }
}

// P^-_{k+1,1} = A P^f_{k,l} A^T + Q and Z = A^T (P^-_{k+1,1})^{-1} for one
// interval by its SG lanes (lane = row), in TR, from the filter result fk =
// P^f_{k,l} (the fast block ll of Eq. 17 in exact arithmetic); Pll, AP, Pm
// and Z are the slot's work arrays (AP also holds the 2x2 minors of P^- and
// the rows of its inverse).  ok turns false on a singular P^-.  No barrier
// after the last stores of Z.
template <int NX, int SG, class TR>
__device__ __forceinline__ void pminus_z(int lane, unsigned mask, const TR* fk, const double* A1, const double* Qm,
                                         TR* Pll, TR* AP, TR* Pm, TR* Z, bool& ok) {
  const int r = lane;
  const bool row = r < NX;
  if (row) {
#pragma unroll
    for (int q = 0; q < NX; ++q) Pll[r * NX + q] = fk[r * NX + q];
  }
  __syncwarp(mask);
  // A P^f_{ll} (row r)
  if (row) {
#pragma unroll
    for (int q = 0; q < NX; ++q) {
      TR v = TR(0);
#pragma unroll
      for (int t = 0; t < NX; ++t) v = fma((TR)A1[r * NX + t], Pll[t * NX + q], v);
      AP[r * NX + q] = v;
    }
  }
  __syncwarp(mask);
  // P^-_{k+1,1} = (A P^f_{ll}) A^T + Q (row r, upper triangle, mirrored)
  if (row) {
#pragma unroll
    for (int q = 0; q < NX; ++q) {
      if (q >= r) {
        TR v = (TR)Qm[r * NX + q];
#pragma unroll
        for (int t = 0; t < NX; ++t) v = fma(AP[r * NX + t], (TR)A1[q * NX + t], v);
        Pm[r * NX + q] = v;
        Pm[q * NX + r] = v;
      }
    }
  }
  __syncwarp(mask);
  // (P^-)^{-1} by the adjugate for NX <= 4: lane r forms row r of the inverse,
  // the cofactors C_{c,r} of column r, so that det = sum_c P^-_{c,r} C_{c,r}
  // needs no other lane; for NX = 4 the twelve 2x2 minors are shared (three
  // per lane, in the AP slot).  Above NX = 4 every lane forms the whole
  // inverse by Cholesky.  Then Z = A^T (P^-)^{-1} (row r).
  if constexpr (NX <= 4) {
    TR* mn = AP;
    if constexpr (NX == 4) {
      for (int u = lane; u < 12; u += SG) {
        const int r0 = u < 6 ? 0 : 2, v = u < 6 ? u : u - 6;
        const int p = v < 3 ? 0 : (v < 5 ? 1 : 2);
        const int q = v < 3 ? v + 1 : (v < 5 ? v - 1 : 3);
        mn[u] = fma(Pm[r0 * 4 + p], Pm[(r0 + 1) * 4 + q], -Pm[(r0 + 1) * 4 + p] * Pm[r0 * 4 + q]);
      }
      __syncwarp(mask);
    }
    TR cof[NX];
    TR det = TR(0);
    if (row) {
#pragma unroll
      for (int col = 0; col < NX; ++col) {
        TR v;
        if (NX == 1) {
          v = TR(1);
        } else if (NX == 2) {
          v = (r == col) ? Pm[(1 - r) * 3] : -Pm[r * 2 + col];
        } else if (NX == 3) {
          const int i0 = col == 0 ? 1 : 0, i1 = col == 2 ? 1 : 2, j0 = r == 0 ? 1 : 0, j1 = r == 2 ? 1 : 2;
          v = Pm[i0 * 3 + j0] * Pm[i1 * 3 + j1] - Pm[i0 * 3 + j1] * Pm[i1 * 3 + j0];
          if ((r + col) & 1) v = -v;
        } else {
          const int arow = col ^ 1;
          const TR* mins = col < 2 ? mn + 6 : mn;
          const int code = r == 0 ? 0x543 : (r == 1 ? 0x521 : (r == 2 ? 0x420 : 0x310));
          const int k0 = r > 0 ? 0 : 1, k1 = r > 1 ? 1 : 2, k2 = r > 2 ? 2 : 3;
          v = Pm[arow * 4 + k0] * mins[(code >> 8) & 15];
          v = fma(-Pm[arow * 4 + k1], mins[(code >> 4) & 15], v);
          v = fma(Pm[arow * 4 + k2], mins[code & 15], v);
          if (((col & 1) != 0) != ((r & 1) != 0)) v = -v;
        }
        cof[col] = v;
        det = fma(Pm[col * NX + r], v, det);
      }
      if (bad_value(det)) { ok = false; det = TR(1); }
    }
    __syncwarp(mask);  // the minors' last reads
    if (row) {
      const TR id = TR(1) / det;
#pragma unroll
      for (int q = 0; q < NX; ++q) AP[r * NX + q] = cof[q] * id;
    }
    __syncwarp(mask);
    if (row) {
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        TR v = TR(0);
#pragma unroll
        for (int t = 0; t < NX; ++t) v = fma((TR)A1[t * NX + r], AP[t * NX + q], v);
        Z[r * NX + q] = v;
      }
    }
  } else {
    TR Pmv[NX][NX], Pmi[NX][NX];
#pragma unroll
    for (int i = 0; i < NX; ++i)
#pragma unroll
      for (int j = 0; j < NX; ++j) Pmv[i][j] = Pm[i * NX + j];
    ok &= spd_inverse<NX, TR>(Pmv, Pmi);
    if (row) {
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        TR v = TR(0);
#pragma unroll
        for (int t = 0; t < NX; ++t) v = fma((TR)A1[t * NX + r], Pmi[t][q], v);
        Z[r * NX + q] = v;
      }
    }
  }
}

// The interval setup of a sequence that takes the two-point recovery, mixed
// mode (no record is written, and no log likelihood is asked for): the
// fast-filter quantities that only feed the smoother element of Eq. (29)
// (X = P C_bar^T, S_y and its inverse, kap, U_l, S_y^-1 U_l^T, m^f_l,
// P A^{lT}) are formed in float32, as the element itself; P^-_{k+1,1} and its
// inverse stay in float64.  Slot layout: SetupGeom's float region from the
// slot's start, then fSy, fev; the float64 arrays from TP on.
template <int NX, int M, class T, class TR>
__device__ __noinline__ void setup_interval_tp(const Ctx& c, long long gi, int s, long long k, int lane, unsigned mask, TR* sb,
                                  const TR* prev) {
  using Gm = SetupGeom<NX>;
  constexpr int MM = M > 0 ? M : MY;
  constexpr int NN = NX * NX;
  const int r = lane;
  const bool row = r < NX;
  const int N = c.meta.nslow[s], m = M > 0 ? M : c.ny;
  const double* md = c.model + (long long)s * c.ml.stride;
  const double* A1 = md + c.ml.Apow + NN;
  const T* cf = (const T*)(md + c.ml.Cf);
  const T* Cbf = cf + 6 * NN + 3 * NX * MY;  // m x NX
  const T* Rxf = Cbf + MY * NX;               // m x m
  const T* Alf = Rxf + MY * MY;               // NN
  const T* VHlf = Alf + NN;                   // NX x m
  T* sf = (T*)sb;
  bool ok = true;
  // P^f_{k-1,l}, m^f_{k-1,l} in float
  if (row) {
    if (k == 0) {
      sf[Gm::fmv + r] = (T)c.m0[(long long)s * NX + r];
#pragma unroll
      for (int q = 0; q < NX; ++q) sf[Gm::fP + r * NX + q] = (T)c.P0[(long long)s * NN + r * NX + q];
    } else {
      const TR* f = prev ? prev : (const TR*)c.fout + (gi - 1) * (NX + NN);
      sf[Gm::fmv + r] = (T)f[r];
#pragma unroll
      for (int q = 0; q < NX; ++q) sf[Gm::fP + r * NX + q] = (T)f[NX + r * NX + q];
    }
  }
  __syncwarp(mask);
  // X = P C_bar^T (row r)
  if (row) {
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      T v = T(0);
      if (j < m) {
#pragma unroll
        for (int q = 0; q < NX; ++q) v = fma(sf[Gm::fP + r * NX + q], Cbf[j * NX + q], v);
      }
      sf[Gm::fX + r * MY + j] = v;
    }
  }
  __syncwarp(mask);
  // S_y = C_bar X + R_x (upper entries over the lanes, mirrored), innovation
  for (int u = lane; u < MM * MM; u += Gm::SG) {
    const int i = u / MM, j = u - (u / MM) * MM;
    if (i <= j && j < m) {
      T v = Rxf[i * m + j];
#pragma unroll
      for (int q = 0; q < NX; ++q) v = fma(Cbf[i * NX + q], sf[Gm::fX + q * MY + j], v);
      sf[Gm::fSy + i * MY + j] = v;
      sf[Gm::fSy + j * MY + i] = v;
    }
  }
  if (lane < m) {
    T v = (T)c.y[gi * m + lane];
#pragma unroll
    for (int q = 0; q < NX; ++q) v = fma(-Cbf[lane * NX + q], sf[Gm::fmv + q], v);
    sf[Gm::fev + lane] = v;
  }
  __syncwarp(mask);
  T Si[MY][MY], kap[MY];
  {
    T Sy[MY][MY];
#pragma unroll
    for (int i = 0; i < MY; ++i)
#pragma unroll
      for (int j = 0; j < MY; ++j) Sy[i][j] = (i < m && j < m) ? sf[Gm::fSy + i * MY + j] : ((i == j) ? T(1) : T(0));
    ok &= small_sym_inverse<T>(Sy, Si, m);
#pragma unroll
    for (int i = 0; i < MY; ++i) {
      T v = T(0);
#pragma unroll
      for (int j = 0; j < MY; ++j)
        if (i < m && j < m) v = fma(Si[i][j], sf[Gm::fev + j], v);
      kap[i] = i < m ? v : T(0);
#pragma unroll
      for (int j = 0; j < MY; ++j)
        if (!(i < m && j < m)) Si[i][j] = T(0);
    }
  }
  // row r: U_l, S_y^-1 U_l^T (column r), m^f_l, P A^{lT}
  if (row) {
    T Ul[MY];
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      T v = T(0);
      if (j < m) {
        v = VHlf[r * m + j];
#pragma unroll
        for (int q = 0; q < NX; ++q) v = fma(Alf[r * NX + q], sf[Gm::fX + q * MY + j], v);
      }
      Ul[j] = v;
    }
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      T v = T(0);
#pragma unroll
      for (int j = 0; j < MM; ++j)
        if (i < m && j < m) v = fma(Si[i][j], Ul[j], v);
      sf[Gm::fSUl + i * NX + r] = v;
    }
    T v = T(0);
#pragma unroll
    for (int q = 0; q < NX; ++q) v = fma(Alf[r * NX + q], sf[Gm::fmv + q], v);
#pragma unroll
    for (int j = 0; j < MM; ++j)
      if (j < m) v = fma(Ul[j], kap[j], v);
    sf[Gm::fml + r] = v;
#pragma unroll
    for (int q = 0; q < NX; ++q) {
      T w = T(0);
#pragma unroll
      for (int t = 0; t < NX; ++t) w = fma(sf[Gm::fP + r * NX + t], Alf[q * NX + t], w);
      sf[Gm::fPl + r * NX + q] = w;
    }
  }
  // P^-_{k+1,1} and Z in float64, Z rounded once to float
  pminus_z<NX, Gm::SG, TR>(lane, mask, (const TR*)c.fout + gi * (NX + NN) + NX, A1, md + c.ml.Q, sb + Gm::tPll,
                          sb + Gm::tAP, sb + Gm::tPm, sb + Gm::tZ, ok);
  __syncwarp(mask);
  if (row) {
#pragma unroll
    for (int q = 0; q < NX; ++q) sf[Gm::fZ + r * NX + q] = (T)sb[Gm::tZ + r * NX + q];
  }
  __syncwarp(mask);
  T* se = (T*)c.selem + gi * SL<NX>::SIZE;
  const bool last = k >= N - 1 && !c.split_tail_open;
  setup_elements<NX, M, T, T, T>(r, row, mask, m, last, sf + Gm::fP, sf + Gm::fPl, sf + Gm::fX, sf + Gm::fSUl,
                                 sf + Gm::fZ, sf + Gm::fml, sf + Gm::fmv, cf + Gm::cA, cf + Gm::cQc, cf + Gm::cQl,
                                 cf + Gm::cVH, Si, kap, sf + Gm::fU1, sf + Gm::fP1l, sf + Gm::fP11, sf + Gm::fAml,
                                 sf + Gm::fU1, se, nullptr, nullptr);
  if (!ok && lane == 0) raise_err(c.ctr, DEVERR_SINGULAR);
}

// One interval by its SG lanes (lane = row), slot sb in shared memory (with
// its float region sf when the smoother elements are formed in float32).
// prev (optional): p(x_{k-1,l}|y_{1:k-1}) as (m, P) when it is not yet in
// the filter results (the first interval of a scan tile reads it from the
// tile's exclusive prefix).
// M = ny when known at compile time (the setup kernel), 0 = read from c.ny
// (inside the filter scan); loops over the measurement dimension run M times.
template <int NX, int M, class T, class TR>
__device__ void setup_interval(const Ctx& c, long long gi, int lane, unsigned mask, TR* sb, T* sf, const TR* prev) {
  using Gm = SetupGeom<NX>;
  constexpr int MM = M > 0 ? M : MY;
  constexpr int NN = NX * NX;
  using RL = Rec<NX>;
  const int r = lane;
  const bool row = r < NX;
  const int s = find_segment(c.meta.off_slow, c.n_seq, gi);
  const long long k = gi - c.meta.off_slow[s];
  if constexpr (sizeof(T) != sizeof(TR)) {  // mixed mode, a two-point sequence: the float32 setup
    if (c.smoothing && !c.loglik && !records_needed(c, s)) {
      setup_interval_tp<NX, M, T, TR>(c, gi, s, k, lane, mask, sb, prev);
      return;
    }
  }
  const int N = c.meta.nslow[s], l = c.meta.ratio[s], m = M > 0 ? M : c.ny;
  const double* md = c.model + (long long)s * c.ml.stride;
  const double* Apow = md + c.ml.Apow;
  const double* Al = Apow + (long long)l * NN;
  const double* A1 = Apow + NN;
  const double* Cb = md + c.ml.Cb;
  const double* Rx = md + c.ml.Rx;
  bool ok = true;
  // P^f_{k-1,l}, m^f_{k-1,l}
  if (row) {
    if (k == 0) {
      sb[Gm::mv + r] = (TR)c.m0[(long long)s * NX + r];
#pragma unroll
      for (int q = 0; q < NX; ++q) sb[Gm::P + r * NX + q] = (TR)c.P0[(long long)s * NN + r * NX + q];
    } else {
      const TR* f = prev ? prev : (const TR*)c.fout + (gi - 1) * (NX + NN);
      sb[Gm::mv + r] = f[r];
#pragma unroll
      for (int q = 0; q < NX; ++q) sb[Gm::P + r * NX + q] = f[NX + r * NX + q];
    }
  }
  __syncwarp(mask);
  // X = P C_bar^T (row r; columns >= m are zero)
  if (row) {
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      TR v = TR(0);
      if (j < m) {
#pragma unroll
        for (int q = 0; q < NX; ++q) v = fma(sb[Gm::P + r * NX + q], (TR)Cb[j * NX + q], v);
      }
      sb[Gm::X + r * MY + j] = v;
    }
  }
  __syncwarp(mask);
  // S_y = C_bar X + R_x (upper entries spread over the lanes, mirrored) and
  // the innovation e = y_k - C_bar m (lane j < m)
  for (int u = lane; u < MM * MM; u += Gm::SG) {
    const int i = u / MM, j = u - (u / MM) * MM;
    if (i <= j && j < m) {
      TR v = (TR)Rx[i * m + j];
#pragma unroll
      for (int q = 0; q < NX; ++q) v = fma((TR)Cb[i * NX + q], sb[Gm::X + q * MY + j], v);
      sb[Gm::Sy + i * MY + j] = v;
      sb[Gm::Sy + j * MY + i] = v;
    }
  }
  const double* ui = c.uin ? c.uin + gi * UIn<NX>::SIZE : nullptr;
  if (lane < m) {
    const double* yk = c.y + gi * m;
    TR v = (TR)(ui ? yk[lane] - ui[UIn<NX>::c + lane] : yk[lane]);
#pragma unroll
    for (int q = 0; q < NX; ++q) v = fma(-(TR)Cb[lane * NX + q], sb[Gm::mv + q], v);
    sb[Gm::ev + lane] = v;
  }
  __syncwarp(mask);
  // S_y^-1 and kap = S_y^-1 e (every lane)
  TR Si[MY][MY], kap[MY];
  {
    TR Sy[MY][MY];
#pragma unroll
    for (int i = 0; i < MY; ++i)
#pragma unroll
      for (int j = 0; j < MY; ++j) Sy[i][j] = (i < m && j < m) ? sb[Gm::Sy + i * MY + j] : ((i == j) ? TR(1) : TR(0));
    TR logdet = TR(0);  // (the float64 log only when the log likelihood is asked for)
    ok &= small_sym_inverse<TR>(Sy, Si, m, c.loglik ? &logdet : nullptr);
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      TR v = TR(0);
#pragma unroll
      for (int j = 0; j < MM; ++j)
        if (i < m && j < m) v = fma(Si[i][j], sb[Gm::ev + j], v);
      kap[i] = v;
    }
    // log N(y_k; C_bar m^f_{k-1,l}, S_y): this interval's term of log p(y_{1:N})
    if (c.loglik && lane == 0) {
      TR q = TR(0);
#pragma unroll
      for (int j = 0; j < MM; ++j)
        if (j < m) q = fma(sb[Gm::ev + j], kap[j], q);
      c.lterm[gi] = -0.5 * ((double)m * 1.8378770664093454836 + (double)logdet + (double)q);
    }
  }
  // row r: U_l, S_y^-1 U_l^T (column r), m^f_l, P A^{lT}
  TR Ul[MY];
  if (row) {
    const double* VHl = md + c.ml.VH + (long long)(l - 1) * NX * m;
#pragma unroll
    for (int j = 0; j < MM; ++j) {
      TR v = TR(0);
      if (j < m) {
        v = (TR)VHl[r * m + j];
#pragma unroll
        for (int q = 0; q < NX; ++q) v = fma((TR)Al[r * NX + q], sb[Gm::X + q * MY + j], v);
      }
      Ul[j] = v;
    }
#pragma unroll
    for (int i = 0; i < MM; ++i) {
      TR v = TR(0);
#pragma unroll
      for (int j = 0; j < MM; ++j)
        if (i < m && j < m) v = fma(Si[i][j], Ul[j], v);
      sb[Gm::SUl + i * NX + r] = v;
    }
    TR v = ui ? (TR)ui[UIn<NX>::bl + r] : TR(0);
#pragma unroll
    for (int q = 0; q < NX; ++q) v = fma((TR)Al[r * NX + q], sb[Gm::mv + q], v);
#pragma unroll
    for (int j = 0; j < MM; ++j)
      if (j < m) v = fma(Ul[j], kap[j], v);
    sb[Gm::ml + r] = v;
#pragma unroll
    for (int q = 0; q < NX; ++q) {
      TR w = TR(0);
#pragma unroll
      for (int t = 0; t < NX; ++t) w = fma(sb[Gm::P + r * NX + t], (TR)Al[q * NX + t], w);
      sb[Gm::Pl + r * NX + q] = w;
    }
  }
  pminus_z<NX, Gm::SG, TR>(lane, mask, (const TR*)c.fout + gi * (NX + NN) + NX, A1, md + c.ml.Q, sb + Gm::Pll,
                          sb + Gm::AP, sb + Gm::Pm, sb + Gm::Z, ok);
  __syncwarp(mask);
  // record (row r; lane 0 the m-sized parts), which the two-point recovery
  // does not read
  if (records_needed(c, s)) {
    TR* rc = (TR*)c.rec + gi * RL::SIZE;
    if (row) {
      rc[RL::mv + r] = sb[Gm::mv + r];
      rc[RL::ml + r] = sb[Gm::ml + r];
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        rc[RL::P + r * NX + q] = sb[Gm::P + r * NX + q];
        rc[RL::Pl + r * NX + q] = sb[Gm::Pl + r * NX + q];
        rc[RL::Z + r * NX + q] = sb[Gm::Z + r * NX + q];
        rc[RL::Pm + r * NX + q] = sb[Gm::Pm + r * NX + q];
      }
#pragma unroll
      for (int j = 0; j < MM; ++j) {
        rc[RL::X + r * MY + j] = sb[Gm::X + r * MY + j];
        rc[RL::SUl + j * NX + r] = sb[Gm::SUl + j * NX + r];
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < MM; ++i) {
        rc[RL::kap + i] = kap[i];
#pragma unroll
        for (int j = 0; j < MM; ++j) rc[RL::Si + i * MY + j] = Si[i][j];
      }
    }
  }
  if (c.smoothing) {
    T* se = (T*)c.selem + gi * SL<NX>::SIZE;
    const bool last = k >= N - 1 && !c.split_tail_open;
    if constexpr (sizeof(T) == sizeof(TR)) {
      __syncwarp(mask);  // the record's reads of Pm (P11 reuses it)
      setup_elements<NX, M, TR, double, T>(r, row, mask, m, last, sb + Gm::P, sb + Gm::Pl, sb + Gm::X, sb + Gm::SUl,
                                        sb + Gm::Z, sb + Gm::ml, sb + Gm::mv, A1, md + c.ml.Qc, md + c.ml.Ql,
                                        md + c.ml.VH, Si, kap, sb + Gm::U1, sb + Gm::P1l, sb + Gm::P11,
                                        sb + Gm::Aml, sb + Gm::AP1, se, ui ? ui + UIn<NX>::b1 : nullptr,
                                        ui ? ui + UIn<NX>::bn : nullptr);
    } else {
      // float copies of this lane's rows (over the slot's dead TR entries,
      // after every lane's record reads of Pm), then the elements in float32
      __syncwarp(mask);
      if (row) {
#pragma unroll
        for (int q = 0; q < NX; ++q) {
          sf[Gm::fP + r * NX + q] = (T)sb[Gm::P + r * NX + q];
          sf[Gm::fPl + r * NX + q] = (T)sb[Gm::Pl + r * NX + q];
          sf[Gm::fZ + r * NX + q] = (T)sb[Gm::Z + r * NX + q];
        }
#pragma unroll
        for (int j = 0; j < MM; ++j) {
          sf[Gm::fX + r * MY + j] = (T)sb[Gm::X + r * MY + j];
          sf[Gm::fSUl + j * NX + r] = (T)sb[Gm::SUl + j * NX + r];
        }
        sf[Gm::fml + r] = (T)sb[Gm::ml + r];
        sf[Gm::fmv + r] = (T)sb[Gm::mv + r];
      }
      T Sif[MY][MY], kapf[MY];
#pragma unroll
      for (int i = 0; i < MM; ++i) {
        kapf[i] = i < m ? (T)kap[i] : T(0);
#pragma unroll
        for (int j = 0; j < MM; ++j) Sif[i][j] = (i < m && j < m) ? (T)Si[i][j] : T(0);
      }
      __syncwarp(mask);
      const T* cf = (const T*)(md + c.ml.Cf);
      setup_elements<NX, M, T, T, T>(r, row, mask, m, last, sf + Gm::fP, sf + Gm::fPl, sf + Gm::fX, sf + Gm::fSUl,
                                  sf + Gm::fZ, sf + Gm::fml, sf + Gm::fmv, cf + Gm::cA, cf + Gm::cQc, cf + Gm::cQl,
                                  cf + Gm::cVH, Sif, kapf, sf + Gm::fU1, sf + Gm::fP1l, sf + Gm::fP11,
                                  sf + Gm::fAml, sf + Gm::fU1, se, ui ? ui + UIn<NX>::b1 : nullptr,
                                  ui ? ui + UIn<NX>::bn : nullptr);
    }
  }
  if (!ok && lane == 0) raise_err(c.ctr, DEVERR_SINGULAR);
}

// ===========================================================================
// Filter operator of Eq. (27) with a generic element of Eq. (26) on the
// right.  Its J_j = C_bar^T R_x^-1 C_bar has rank m < NX (and eta_j =
// C_bar^T R_x^-1 (y_k - c_k)), so by the matrix inversion lemma
//   (I + D_i J_j)^{-1} = I - K C_bar,   S = R_x + C_bar D_i C_bar^T,
//   K = D_i C_bar^T S^{-1},
// and the n x n solve of the general combine becomes the m x m one of S:
//   u = (I - K C_bar)(d_i + D_i eta_j),          d_ij = F_j u + d_j,
//   D_ij = F_j (D_i - K C_bar D_i) F_j^T + D_j,
//   V = (I - K C_bar) F_i = F_i - K G,  G = C_bar F_i,   F_ij = F_j V,
//   eta_ij = V^T (eta_j - J_j d_i) + eta_i,
//   J_ij = V^T J_j F_i + J_i = G^T S^{-1} G + J_i
// (the last because (I - K C_bar)^T C_bar^T R_x^-1 = C_bar^T S^{-1}).  This
// is the measurement update of the left operand by the interval's
// measurement followed by the element's transition; Eq. (27) is the same map
// for a general right operand.  S^{-1}: for m = 1 the reciprocal of one value
// of type T, correctly rounded in T (which equals the float64 reciprocal
// rounded once to T); for m = 2 the adjugate over det S, with det S (the one
// step that can cancel) formed in TS (float64 in the mixed mode) from the
// exact products of the T entries, and its reciprocal rounded once to T; for
// m > 2 the whole inverse in TS.  Cb (m x NX, ld NX) and Rx (m x m, ld m)
// hold the model's C_bar and R_x in T.  prefix as in g_filter_combine.
// Scratch: sc (T) RankScr<NX>::SIZE.
// ===========================================================================
template <int NX>
struct RankScr {
  static constexpr int NN = NX * NX, NM = NX * MY;
  static constexpr int CD = 0, Kt = CD + NM, Gm = Kt + NM, SiG = Gm + NM, t = SiG + NM, x = t + NX, Ct = x + NX,
                       Si = Ct + MY, Pu = Si + MY * MY, FP = Pu + NN, V = FP + NN, SIZE = V + NN;
};

template <int NX, int G, class T, class TS>
__device__ __forceinline__ bool g_filter_combine_rank(const Grp<G>& g, T* o, const T* a, const T* b, T* sc,
                                                      const T* Cb, const T* Rx, int m, bool prefix) {
  using L = FL<NX>;
  using R = RankScr<NX>;
  constexpr int NN = NX * NX, NT = NX * (NX + 1) / 2;
  T *CD = sc + R::CD, *Kt = sc + R::Kt, *Gm = sc + R::Gm, *SiG = sc + R::SiG, *t = sc + R::t, *x = sc + R::x;
  T *Ct = sc + R::Ct, *Si = sc + R::Si, *Pu = sc + R::Pu, *FP = sc + R::FP, *V = sc + R::V;
  const int mn = m * NX;
  // 1. CD = C_bar D_i, t = d_i + D_i eta_j; without prefix also G = C_bar F_i
  //    and x = eta_j - J_j d_i
  const int n1 = prefix ? mn + NX : 2 * mn + 2 * NX;
  for (int e = g.lane; e < n1; e += G) {
    if (e < mn) {
      const int j = e / NX, q = e - (e / NX) * NX;
      T v = T(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) v = fma(Cb[j * NX + k], a[L::D + k * NX + q], v);
      CD[e] = v;
    } else if (e < mn + NX) {
      const int r = e - mn;
      T v = a[L::d + r];
#pragma unroll
      for (int k = 0; k < NX; ++k) v = fma(a[L::D + r * NX + k], b[L::e + k], v);
      t[r] = v;
    } else if (e < 2 * mn + NX) {
      const int f = e - mn - NX, j = f / NX, q = f - (f / NX) * NX;
      T v = T(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) v = fma(Cb[j * NX + k], a[L::F + k * NX + q], v);
      Gm[f] = v;
    } else {
      const int r = e - 2 * mn - NX;
      T v = b[L::e + r];
#pragma unroll
      for (int k = 0; k < NX; ++k) v = fma(-b[L::J + r * NX + k], a[L::d + k], v);
      x[r] = v;
    }
  }
  g.sync();
  // 2. S = R_x + CD C_bar^T (exactly symmetric) and S^{-1}, on every lane in
  //    registers, stored by lane 0 (ld MY); Ct = C_bar t
  bool ok = true;
  auto rcp = [](T v) -> T {
    if constexpr (sizeof(T) == sizeof(float)) return __frcp_rn(v);
    else return T(1) / v;
  };
  if (m == 1) {
    T s = Rx[0];
#pragma unroll
    for (int k = 0; k < NX; ++k) s = fma(CD[k], Cb[k], s);
    if (bad_value(s)) { ok = false; s = T(1); }
    if (g.lane == 0) Si[0] = rcp(s);
  } else if (m == 2) {
    T s00 = Rx[0], s01 = Rx[1], s11 = Rx[3];
#pragma unroll
    for (int k = 0; k < NX; ++k) {
      s00 = fma(CD[k], Cb[k], s00);
      s01 = fma(CD[k], Cb[NX + k], s01);
      s11 = fma(CD[NX + k], Cb[NX + k], s11);
    }
    const TS t01 = (TS)s01;
    T det = (T)fma((TS)s00, (TS)s11, -(t01 * t01));
    if (bad_value(det)) { ok = false; det = T(1); }
    const T id = rcp(det);
    if (g.lane == 0) {
      Si[0] = s11 * id;
      Si[1] = -s01 * id;
      Si[MY] = -s01 * id;
      Si[MY + 1] = s00 * id;
    }
  } else {
    TS S[MY][MY], Sinv[MY][MY];
#pragma unroll
    for (int i = 0; i < MY; ++i)
#pragma unroll
      for (int j = i; j < MY; ++j) {
        T v = T(0);
        if (j < m) {
          v = Rx[i * m + j];
#pragma unroll
          for (int k = 0; k < NX; ++k) v = fma(CD[i * NX + k], Cb[j * NX + k], v);
        }
        S[i][j] = (TS)v;
        S[j][i] = (TS)v;
      }
    ok = small_sym_inverse<TS>(S, Sinv, m);
    if (g.lane == 0)
#pragma unroll
      for (int i = 0; i < MY; ++i)
#pragma unroll
        for (int j = 0; j < MY; ++j)
          if (i < m && j < m) Si[i * MY + j] = (T)Sinv[i][j];
  }
  for (int j = g.lane; j < m; j += G) {
    T v = T(0);
#pragma unroll
    for (int k = 0; k < NX; ++k) v = fma(Cb[j * NX + k], t[k], v);
    Ct[j] = v;
  }
  g.sync();
  // 3. K^T = S^{-1} CD; without prefix also S^{-1} G
  const int n3 = prefix ? mn : 2 * mn;
  for (int e = g.lane; e < n3; e += G) {
    const bool second = e >= mn;
    const int f = second ? e - mn : e, j = f / NX, q = f - (f / NX) * NX;
    const T* src = second ? Gm : CD;
    T v = T(0);
    for (int i = 0; i < m; ++i) v = fma(Si[j * MY + i], src[i * NX + q], v);
    (second ? SiG : Kt)[f] = v;
  }
  g.sync();
  // 4. u = t - K Ct (over t); P = D_i - K CD (upper, mirrored); without prefix
  //    also J_ij = G^T S^{-1} G + J_i (upper, mirrored) and V = F_i - K G
  const int n4 = prefix ? NX + NT : NX + 2 * NT + NN;
  for (int e = g.lane; e < n4; e += G) {
    if (e < NX) {
      T v = t[e];
      for (int j = 0; j < m; ++j) v = fma(-Kt[j * NX + e], Ct[j], v);
      t[e] = v;
    } else if (e < NX + NT) {
      int r, q;
      tri_rc<NX>(e - NX, r, q);
      T v = a[L::D + r * NX + q];
      for (int j = 0; j < m; ++j) v = fma(-Kt[j * NX + r], CD[j * NX + q], v);
      Pu[r * NX + q] = v;
      Pu[q * NX + r] = v;
    } else if (e < NX + 2 * NT) {
      int r, q;
      tri_rc<NX>(e - NX - NT, r, q);
      T v = a[L::J + r * NX + q];
      for (int j = 0; j < m; ++j) v = fma(Gm[j * NX + r], SiG[j * NX + q], v);
      o[L::J + r * NX + q] = v;
      o[L::J + q * NX + r] = v;
    } else {
      const int f = e - NX - 2 * NT, r = f / NX, q = f - (f / NX) * NX;
      T v = a[L::F + f];
      for (int j = 0; j < m; ++j) v = fma(-Kt[j * NX + r], Gm[j * NX + q], v);
      V[f] = v;
    }
  }
  g.sync();
  // 5. d_ij = F_j u + d_j, FP = F_j P; without prefix also F_ij = F_j V and
  //    eta_ij = V^T x + eta_i
  const int n5 = prefix ? NX + NN : 2 * NX + 2 * NN;
  for (int e = g.lane; e < n5; e += G) {
    if (e < NX) {
      T v = b[L::d + e];
#pragma unroll
      for (int k = 0; k < NX; ++k) v = fma(b[L::F + e * NX + k], t[k], v);
      o[L::d + e] = v;
    } else if (e < NX + 2 * NN) {
      const bool second = e >= NX + NN;
      const int f = e - NX - (second ? NN : 0), r = f / NX, q = f - (f / NX) * NX;
      const T* src = second ? V : Pu;
      T v = T(0);
#pragma unroll
      for (int k = 0; k < NX; ++k) v = fma(b[L::F + r * NX + k], src[k * NX + q], v);
      (second ? o + L::F : FP)[f] = v;
    } else {
      const int r = e - NX - 2 * NN;
      T v = a[L::e + r];
#pragma unroll
      for (int k = 0; k < NX; ++k) v = fma(V[k * NX + r], x[k], v);
      o[L::e + r] = v;
    }
  }
  g.sync();
  // 6. D_ij = FP F_j^T + D_j (upper, mirrored)
  g_mm_sym<NX, G, false, true, T>(g, o + L::D, FP, b + L::F, b + L::D);
  if (prefix) {
    for (int e = g.lane; e < NN; e += G) { o[L::F + e] = T(0); o[L::J + e] = T(0); }
    for (int e = g.lane; e < NX; e += G) o[L::e + e] = T(0);
  }
  g.sync();
  return ok;
}

// ===========================================================================
// scan operators
// ===========================================================================

// Forward scan of the parallel IMKF (Sec. IV): elements a_k of Eq. (25)-(26),
// operator Eq. (27).  Scan position p is the slow step k (0-based).
template <int NX, class T_, class TS_>
struct FilterOp {
  using T = T_;
  using TS = TS_;
  using L = FL<NX>;
  static constexpr int G = GroupSize<NX>::value;
  static constexpr int ES = L::SIZE;
  // group scratch: the combines' work arrays, then the model's C_bar and R_x
  // in T for the rank-m combine (loaded once per tile)
  static constexpr int SCR_GEN = 5 * NX * NX + 2 * NX;
  static constexpr int SCR_OPS = SCR_GEN > RankScr<NX>::SIZE ? SCR_GEN : RankScr<NX>::SIZE;
  static constexpr int CB = SCR_OPS, RX = CB + MY * NX;
  static constexpr int SCR = RX + MY * MY;
  static constexpr int SCRS = NX * NX + 12;
  static constexpr int TICKET = 0;

  __device__ static bool combine(const Grp<G>& g, T* o, const T* left, const T* right, T* sc, TS* scs,
                                 bool prefix) {
    return g_filter_combine<NX, G, T, TS>(g, o, left, right, sc, scs, prefix);
  }
  // the measurement sizes below NX take the rank-m combine for a generic right element
  __device__ static bool rank_form(const Ctx& c) { return c.ny < NX; }
  // before a tile of sequence s: C_bar and R_x into the group scratch (read
  // after the group barrier that precedes the tile's first combine)
  __device__ static void tile_begin(const Grp<G>& g, T* sc, const Ctx& c, int s) {
    if (!rank_form(c)) return;
    const int m = c.ny;
    const double* md = c.model + (long long)s * c.ml.stride;
    if constexpr (sizeof(T) == sizeof(double)) {
      for (int e = g.lane; e < m * NX; e += G) sc[CB + e] = (T)md[c.ml.Cb + e];
      for (int e = g.lane; e < m * m; e += G) sc[RX + e] = (T)md[c.ml.Rx + e];
    } else {
      const float* cf = (const float*)(md + c.ml.Cf) + 6 * NX * NX + 3 * NX * MY;
      for (int e = g.lane; e < m * NX; e += G) sc[CB + e] = cf[e];
      for (int e = g.lane; e < m * m; e += G) sc[RX + e] = cf[MY * NX + e];
    }
  }
  // left (x) right where right is the element loaded for scan position p:
  // every element but the sequence's first one is generic
  __device__ static bool combine_elem(const Grp<G>& g, T* o, const T* left, const T* right, T* sc, TS* scs,
                                      bool prefix, const Ctx& c, long long p) {
    if (rank_form(c) && (p > 0 || c.split_head_generic))
      return g_filter_combine_rank<NX, G, T, TS>(g, o, left, right, sc, sc + CB, sc + RX, c.ny, prefix);
    return g_filter_combine<NX, G, T, TS>(g, o, left, right, sc, scs, prefix);
  }
  __device__ static void identity(const Grp<G>& g, T* x) {  // (I, 0, 0, 0, 0)
    for (int e = g.lane; e < ES; e += G) x[e] = (e < NX * NX && e / NX == e % NX) ? T(1) : T(0);
  }
  // a_1 = (0, m^f_{1,l}, P^f_{1,l}, 0, 0);  a_k = (F, K y_k, D, C_bar^T R_x^-1 y_k, J), k > 1
  // (a range of a split sequence that does not start it has only generic elements)
  __device__ static void load(const Grp<G>& g, T* x, const Ctx& c, int s, long long p, int /*N*/) {
    constexpr int NN = NX * NX;
    const double* md = c.model + (long long)s * c.ml.stride;
    if (p == 0 && !c.split_head_generic) {
      for (int e = g.lane; e < ES; e += G) {
        double v = 0.0;
        if (e >= L::d && e < L::d + NX) v = md[c.ml.m1 + (e - L::d)];
        else if (e >= L::D && e < L::D + NN) v = md[c.ml.P1 + (e - L::D)];
        x[e] = (T)v;
      }
      return;
    }
    if constexpr (sizeof(T) == sizeof(double)) {
      for (int e = g.lane; e < NN; e += G) {
        x[L::F + e] = (T)md[c.ml.Fc + e];
        x[L::D + e] = (T)md[c.ml.Dc + e];
        x[L::J + e] = (T)md[c.ml.Jc + e];
      }
    } else {  // the model's float copies (no float64 conversion per element)
      const float* cfe = (const float*)(md + c.ml.Cf) + 3 * NN + 3 * NX * MY;
      for (int e = g.lane; e < NN; e += G) {
        x[L::F + e] = cfe[e];
        x[L::D + e] = cfe[NN + e];
        x[L::J + e] = cfe[2 * NN + e];
      }
    }
    const int m = c.ny;
    const long long row = c.meta.off_slow[s] + p;
    const double* yk = c.y + row * m;
    // with inputs: y_k - c_k enters K and C_bar^T R_x^-1, and d_k gains b_{k,l};
    // formed in the scan type (float32 elements from the model's float copies
    // of K and C_bar^T R_x^-1 in the mixed and FP32 modes)
    const double* ui = c.uin ? c.uin + row * UIn<NX>::SIZE : nullptr;
    const float* cf = (const float*)(md + c.ml.Cf);
    for (int r = g.lane; r < NX; r += G) {
      T dv = ui ? (T)ui[UIn<NX>::bl + r] : T(0), ev = T(0);
      for (int j = 0; j < m; ++j) {
        const T yj = (T)(ui ? yk[j] - ui[UIn<NX>::c + j] : yk[j]);
        if constexpr (sizeof(T) == sizeof(double)) {
          dv = fma((T)md[c.ml.K + r * m + j], yj, dv);
          ev = fma((T)md[c.ml.Cr + r * m + j], yj, ev);
        } else {
          dv = fma((T)cf[3 * NN + NX * MY + r * m + j], yj, dv);
          ev = fma((T)cf[3 * NN + 2 * NX * MY + r * m + j], yj, ev);
        }
      }
      x[L::d + r] = dv;
      x[L::e + r] = ev;
    }
  }
  // filter result at k: d_k = m^f_{k,l}, D_k = P^f_{k,l}, kept in TS (float64
  // in the mixed mode) for the float64 interval setup
  __device__ static void store(const Grp<G>& g, const T* x, const Ctx& c, int s, long long p, int /*N*/, T*, TS*) {
    constexpr int NN = NX * NX;
    TS* out = (TS*)c.fout + (c.meta.off_slow[s] + p) * (NX + NN);
    for (int e = g.lane; e < NX + NN; e += G) out[e] = (TS)x[L::d + e];  // d then D are contiguous
  }
  __device__ static unsigned char* tile_state(const Ctx& c, long long t) { return c.ftile + t * c.ftile_stride; }
  __device__ static const long long* tile_off(const Ctx& c) { return c.meta.tile_off_f; }
  __device__ static long long total_tiles(const Ctx& c) { return c.ctr->total_tiles_f; }
  __device__ static int tile_elems(const Ctx& c) { return c.tile_f; }

  // After a tile's results are written: the interval setup (fast-filter
  // blocks, smoother elements and recovery records) of the tile's intervals,
  // by the whole block in rounds of blockDim/SG intervals.  The first
  // interval's predecessor result is the tile's exclusive prefix.
  static constexpr bool HAS_EPILOGUE = true;
  static constexpr bool EPILOGUE_ALWAYS = false;  // only while the setup runs inside the filter scan
  // Slots: one per interval of the tile, at most one per SG threads.
  __host__ __device__ static int epilogue_slots(int threads, int tile) {
    const int per = threads / SetupGeom<NX>::SG;
    return per < tile ? per : tile;
  }
  static constexpr bool FLOAT_ELEMENTS = sizeof(T) != sizeof(TS);
  __host__ __device__ static size_t epilogue_bytes(int threads, int tile) {
    using Gm = SetupGeom<NX>;
    return align16((NX + NX * NX) * sizeof(TS)) + (size_t)epilogue_slots(threads, tile) * Gm::template slot_bytes<T, TS>();
  }
  __device__ static void epilogue(const Ctx& c, int s, long long p0, int count, const T* excl, unsigned char* esm) {
    using Gm = SetupGeom<NX>;
    constexpr int SG = Gm::SG, NN = NX * NX;
    TS* prevb = (TS*)esm;
    unsigned char* slots = esm + align16((NX + NN) * sizeof(TS));
    __syncthreads();
    for (int e = threadIdx.x; e < NX + NN; e += blockDim.x) prevb[e] = (TS)excl[L::d + e];
    __syncthreads();
    const int lane = threadIdx.x % SG, slot = threadIdx.x / SG;
    const int per_round = epilogue_slots(blockDim.x, tile_elems(c));
    const unsigned mask = (SG == 32) ? 0xffffffffu : (((1u << SG) - 1u) << ((threadIdx.x & 31) & ~(SG - 1)));
    const long long base_row = c.meta.off_slow[s];
    if (slot < per_round) {
      unsigned char* sl = slots + (size_t)slot * Gm::template slot_bytes<T, TS>();
      TS* sb = (TS*)sl;
      T* sf = FLOAT_ELEMENTS ? (T*)(sb + Gm::FREG) : nullptr;
      // compiled per measurement size, as the separate setup kernel
      for (int j = slot; j < count; j += per_round) {
        const TS* pv = j == 0 ? prevb : nullptr;
        switch (c.ny) {
          case 1: setup_interval<NX, 1, T, TS>(c, base_row + p0 + j, lane, mask, sb, sf, pv); break;
          case 2: setup_interval<NX, 2, T, TS>(c, base_row + p0 + j, lane, mask, sb, sf, pv); break;
          case 3: setup_interval<NX, 3, T, TS>(c, base_row + p0 + j, lane, mask, sb, sf, pv); break;
          default: setup_interval<NX, 4, T, TS>(c, base_row + p0 + j, lane, mask, sb, sf, pv); break;
        }
      }
    }
    __syncthreads();
    // the records' P^f_{k-1,l} as LDL^T factors, one thread per interval
    if (records_needed(c, s))
      for (int j = threadIdx.x; j < count; j += blockDim.x)
        ldlt_inplace<NX, TS>((TS*)c.rec + (base_row + p0 + j) * Rec<NX>::SIZE + Rec<NX>::P);
    __syncthreads();
  }
};

// Reverse scan of the parallel IMS (Sec. IV): elements of Eq. (29) built by
// the interval-setup kernel, operator Eq. (30).  Scan position p is slow step
// k = N-1-p, so the scan-order combine left (x) right is right (x) left in
// the paper's order.  Its result at k is p(x_{k,1} | y_{1:N}) = N(g, S); the
// store step turns it at once into the smoothing terms that the recovery of
// interval k-1 needs (Eq. 21 with G_{k-1,i} = P^f_{k-1,i,l} Z_{k-1}):
//   dm = m^s_{k,1} - A m^f_{k-1,l},  dP = P^s_{k,1} - P^-_{k,1},
//   om_{k-1} = Z dm,  Om_{k-1} = Z dP Z^T,   Z = A^T (P^-_{k,1})^{-1},
// formed by the lane group in TR (float64 except in the float32 mode).
template <int NX, class T_, class TR_>
struct SmootherOp {
  using T = T_;
  using TS = TR_;
  using L = SL<NX>;
  static constexpr int G = GroupSize<NX>::value;
  static constexpr int ES = L::SIZE;
  static constexpr int SCR = NX * NX;
  static constexpr int SCRS = 2 * NX * NX + NX;
  static constexpr int TICKET = 1;

  __device__ static bool combine(const Grp<G>& g, T* o, const T* left, const T* right, T* sc, TS*, bool prefix) {
    g_smoother_combine<NX, G, T>(g, o, right, left, sc, prefix);
    return true;
  }
  __device__ static void tile_begin(const Grp<G>&, T*, const Ctx&, int) {}
  __device__ static bool combine_elem(const Grp<G>& g, T* o, const T* left, const T* right, T* sc, TS* scs,
                                      bool prefix, const Ctx&, long long) {
    return combine(g, o, left, right, sc, scs, prefix);
  }
  __device__ static void identity(const Grp<G>& g, T* x) {  // (I, 0, 0)
    for (int e = g.lane; e < ES; e += G) x[e] = (e < NX * NX && e / NX == e % NX) ? T(1) : T(0);
  }
  __device__ static void load(const Grp<G>& g, T* x, const Ctx& c, int s, long long p, int N) {
    const T* src = (const T*)c.selem + (c.meta.off_slow[s] + (N - 1 - p)) * ES;
    for (int e = g.lane; e < ES; e += G) x[e] = src[e];
  }
  // two-point recovery terms of a sequence whose bflag is set: the result at
  // k is mu0 and (before its LDL^T) L1's source for interval k-1 and mu1 of
  // interval k-1; interval k also takes E_k and S_k of its element (the last
  // interval: L2 = P^s_{k,1})
  __device__ static void store_two_point(const Grp<G>& g, const T* x, const Ctx& c, int s, long long k, int N) {
    constexpr int NN = NX * NX;
    using B = BRec<NX>;
    using TR = TS;
    const long long row = c.meta.off_slow[s] + k;
    TR* b = (TR*)c.brec + row * B::SIZE;
    for (int e = g.lane; e < NX; e += G) b[B::mu0 + e] = (TR)x[L::g + e];
    if (k >= 1) {
      TR* bp = b - B::SIZE;
      for (int e = g.lane; e < NX; e += G) bp[B::mu1 + e] = (TR)x[L::g + e];
      for (int e = g.lane; e < NN; e += G) bp[B::L1 + e] = (TR)x[L::S + e];
    }
    if (k < N - 1) {
      const T* el = (const T*)c.selem + row * ES;
      for (int e = g.lane; e < NN; e += G) {
        b[B::E + e] = (TR)el[L::E + e];
        b[B::L2 + e] = (TR)el[L::S + e];
      }
    } else {
      for (int e = g.lane; e < NN; e += G) b[B::L2 + e] = (TR)x[L::S + e];
    }
  }
  __device__ static bool two_point(const Ctx& c, int s) {
    return c.bridge && c.model[(long long)s * c.ml.stride + c.ml.bflag] != 0.0;
  }
  __device__ static void store(const Grp<G>& g, const T* x, const Ctx& c, int s, long long p, int N, T*, TS* scs) {
    constexpr int NN = NX * NX;
    using RL = Rec<NX>;
    using TR = TS;
    const long long k = N - 1 - p;
    if (two_point(c, s)) {
      store_two_point(g, x, c, s, k, N);
      return;
    }
    if (k == 0) return;
    const long long row = c.meta.off_slow[s] + k - 1;
    const TR* rc = (const TR*)c.rec + row * RL::SIZE;
    const double* A1 = c.model + (long long)s * c.ml.stride + c.ml.Apow + NN;
    TR* dP = scs;
    TR* ZdP = scs + NN;
    TR* dm = scs + 2 * NN;
    TR* out = (TR*)c.sfin + row * SFin<NX>::SIZE;
    for (int e = g.lane; e < NN; e += G) dP[e] = (TR)x[L::S + e] - rc[RL::Pm + e];
    g_mv<NX, G, false, TR>(g, dm, A1, rc + RL::ml, x + L::g, TR(-1));
    if (c.uin)  // the prediction m^-_{k,1} = A m^f_{k-1,l} + B u_{k-1,l}; same lane per entry as g_mv
      for (int e = g.lane; e < NX; e += G) dm[e] -= (TR)c.uin[row * UIn<NX>::SIZE + UIn<NX>::bn + e];
    g.sync();
    g_mm<NX, G, false, false, TR>(g, ZdP, rc + RL::Z, dP, (const TR*)nullptr);
    g_mv<NX, G, false, TR>(g, out + NN, rc + RL::Z, dm, (const TR*)nullptr);
    g.sync();
    g_mm_sym<NX, G, false, true, TR>(g, out, ZdP, rc + RL::Z, (const TR*)nullptr);
    g.sync();
  }
  __device__ static unsigned char* tile_state(const Ctx& c, long long t) { return c.stile + t * c.stile_stride; }
  __device__ static const long long* tile_off(const Ctx& c) { return c.meta.tile_off_s; }
  __device__ static long long total_tiles(const Ctx& c) { return c.ctr->total_tiles_s; }
  __device__ static int tile_elems(const Ctx& c) { return c.tile_s; }
  // After a tile's results are written: the smoothing terms Om of the tile's
  // intervals as LDL^T factors for the recovery, one thread per interval.
  static constexpr bool HAS_EPILOGUE = true;
  static constexpr bool EPILOGUE_ALWAYS = true;
  __host__ __device__ static size_t epilogue_bytes(int, int) { return 0; }
  __device__ static void epilogue(const Ctx& c, int s, long long p0, int count, const T*, unsigned char*) {
    const int N = c.meta.nslow[s];
    __syncthreads();  // every lane group's stores of the tile
    if (two_point(c, s)) {  // the factors this tile's stores wrote: L2 of interval k, L1 of interval k-1
      using B = BRec<NX>;
      for (int j = threadIdx.x; j < 2 * count; j += blockDim.x) {
        const long long k = N - 1 - (p0 + j / 2);
        TR_* b = (TR_*)c.brec + (c.meta.off_slow[s] + k) * B::SIZE;
        if (j & 1) {
          if (k >= 1) ldlt_inplace<NX, TR_>(b - B::SIZE + B::L1);
        } else {
          ldlt_inplace<NX, TR_>(b + B::L2);
        }
      }
      __syncthreads();
      return;
    }
    for (int j = threadIdx.x; j < count; j += blockDim.x) {
      const long long k = N - 1 - (p0 + j);
      if (k >= 1)
        ldlt_inplace<NX, TR_>((TR_*)c.sfin + (c.meta.off_slow[s] + k - 1) * SFin<NX>::SIZE + SFin<NX>::Om);
    }
    __syncthreads();
  }
};

// ===========================================================================
// scan skeleton: persistent blocks take tiles in ticket order; per tile
//   1. each lane group folds E consecutive elements,
//   2. Kogge-Stone scan of the group aggregates in shared memory,
//   3. group 0 resolves the tile prefix by decoupled look-back over the
//      preceding tiles of the same sequence (aggregate / inclusive-prefix
//      flags tagged with the call's epoch),
//   4. each group re-walks its elements from its exclusive prefix and writes
//      the scan results.
// Tickets are taken in increasing order, so every tile waited on belongs to a
// block that is already running and never waits on a later tile: the
// look-back cannot deadlock.  Its waits are still bounded (SPIN_LIMIT).
// ===========================================================================
template <class Op>
struct ScanSmem {
  using T = typename Op::T;
  using TS = typename Op::TS;
  __host__ __device__ static size_t group_bytes() {
    return align16((3 * Op::ES + Op::SCR) * sizeof(T)) + align16((Op::SCRS > 0 ? Op::SCRS : 1) * sizeof(TS));
  }
  // look-back window W: predecessor tiles examined per round (1..MAXWIN)
  static constexpr int MAXWIN = 32;
  // W payloads plus ceil(W/2) for the second buffer of the pairwise fold
  __host__ __device__ static size_t window_bytes(int W) {
    return align16((size_t)(W + (W + 1) / 2) * Op::ES * sizeof(T));
  }
  // layout: [excl | tile id, control | union{ lane-group buffers, group
  // aggregates x2, look-back window ; tile epilogue }]
  __host__ __device__ static size_t scan_part(int NG, int W) {
    return NG * group_bytes() + 2 * align16((size_t)NG * Op::ES * sizeof(T)) + window_bytes(W);
  }
  __host__ __device__ static size_t bytes(int NG, int W, int E, bool epilogue = true) {
    const size_t sp = scan_part(NG, W), ep = epilogue ? Op::epilogue_bytes(NG * Op::G, NG * E) : 0;
    return align16(Op::ES * sizeof(T)) + 32 + (sp > ep ? sp : ep);
  }
  __host__ __device__ static size_t payload_bytes() { return align16(Op::ES * sizeof(T)); }
  __host__ __device__ static size_t tile_state_bytes() { return 16 + 3 * payload_bytes(); }
};

// Tile state: [tile flag | group flag | aggregate | inclusive prefix | group
// aggregate].  Flag words hold (call epoch << 32) | status: tile flag 1 =
// aggregate published, 2 = inclusive prefix published; group flag 3 = the
// group aggregate published.
template <class Op>
__device__ __forceinline__ void publish(const Grp<Op::G>& g, unsigned char* ts, const typename Op::T* x, int slot,
                                        unsigned status, unsigned long long epoch) {
  using T = typename Op::T;
  T* dst = (T*)(ts + 16 + slot * ScanSmem<Op>::payload_bytes());
  for (int e = g.lane; e < Op::ES; e += Op::G) __stcg(dst + e, x[e]);
  __threadfence();
  g.sync();
  if (g.lane == 0)
    st_release_u64((unsigned long long*)(ts + (status == 3u ? 8 : 0)), ((epoch & 0xffffffffull) << 32) | status);
}

// One look-back round over up to W earlier tiles x_q = tile (j_hi - q*step),
// q < w, done by the whole block.  step = 1: the tile's own group, where a
// tile is usable when it has published its aggregate (or its inclusive
// prefix); step = W: the last tiles of earlier groups, usable when they have
// published their group aggregate (or their inclusive prefix, which then
// covers everything up to the end of their group).  The round needs the
// tiles down to the nearest one holding an inclusive prefix (or all w).
// Lane group 0 polls the flags, all threads fetch the payloads, and all lane
// groups fold them pairwise in a tree of log2(w) levels (scan order: the
// older tile is the left operand); group 0 then folds the product into the
// running exclusive prefix, excl <- product (x) excl.  Returns 1 when an
// inclusive prefix ended the walk, 0 when it must go on, -1 on a timed-out
// wait (DEVERR_TIMEOUT latched); `used` receives the number of tiles folded.
template <class Op>
__device__ int lookback_round(const Grp<Op::G>& g, int gid, int NG, const Ctx& c, unsigned long long epoch,
                              long long j_hi, int step, int w, typename Op::T* excl, typename Op::T* tmp,
                              typename Op::T* win, int* ctl, typename Op::T* sc, typename Op::TS* scs, bool& ok,
                              int& used) {
  using T = typename Op::T;
  constexpr int G = Op::G, ES = Op::ES;
  const bool groups = step > 1;
  T* win2 = win + w * ES;
  if (gid == 0) {
    unsigned ready = 0, pref = 0;
    bool timed_out = true;
    int need = w;
    BoundedPoll poll(SPIN_LIMIT);
    while (poll.more()) {
      for (int q = g.lane; q < w; q += G) {
        if (!((ready >> q) & 1u)) {
          const unsigned long long* fl = (const unsigned long long*)Op::tile_state(c, j_hi - (long long)q * step);
          const unsigned long long v = ld_acquire_u64(fl);
          const bool cur = (v >> 32) == (epoch & 0xffffffffull);
          if (cur && (v & 3ull) == 2ull) {
            ready |= 1u << q;
            pref |= 1u << q;
          } else if (!groups) {
            if (cur && (v & 3ull) == 1ull) ready |= 1u << q;
          } else {
            const unsigned long long v2 = ld_acquire_u64(fl + 1);
            if ((v2 >> 32) == (epoch & 0xffffffffull) && (v2 & 3ull) == 3ull) ready |= 1u << q;
          }
        }
      }
      ready = __reduce_or_sync(g.mask, ready);
      pref = __reduce_or_sync(g.mask, pref);
      need = pref ? __ffs(pref) : w;  // tiles q < need
      const unsigned want = (need >= 32) ? 0xffffffffu : ((1u << need) - 1u);
      if ((ready & want) == want) { timed_out = false; break; }
      poll.backoff();
    }
    if (g.lane == 0) {
      ctl[0] = need;
      ctl[1] = pref ? 1 : 0;
      ctl[2] = timed_out ? 1 : 0;
      if (timed_out) raise_err(c.ctr, DEVERR_TIMEOUT);
    }
  }
  __syncthreads();
  const int need = ctl[0];
  const bool found = ctl[1] != 0;
  if (ctl[2]) return -1;
  // payloads: aggregates (group aggregates), the last one a prefix when found
  for (int idx = threadIdx.x; idx < need * ES; idx += blockDim.x) {
    const int q = idx / ES, e = idx - (idx / ES) * ES;
    const int slot = (found && q == need - 1) ? 1 : (groups ? 2 : 0);
    const T* srcp =
        (const T*)(Op::tile_state(c, j_hi - (long long)q * step) + 16 + slot * ScanSmem<Op>::payload_bytes());
    win[idx] = __ldcg(srcp + e);
  }
  __syncthreads();
  // tree: product in scan order x_{need-1} (x) ... (x) x_0
  T* cur = win;
  T* nxt = win2;
  int k = need;
  while (k > 1) {
    const int pairs = k >> 1;
    for (int pi = gid; pi < pairs; pi += NG)
      ok &= Op::combine(g, nxt + pi * ES, cur + (2 * pi + 1) * ES, cur + 2 * pi * ES, sc, scs, false);
    if ((k & 1) && gid == pairs % NG)
      for (int e = g.lane; e < ES; e += G) nxt[pairs * ES + e] = cur[(k - 1) * ES + e];
    __syncthreads();
    T* x = cur; cur = nxt; nxt = x;
    k = pairs + (k & 1);
  }
  if (gid == 0) {
    ok &= Op::combine(g, tmp, cur, excl, sc, scs, false);
    for (int e = g.lane; e < ES; e += G) excl[e] = tmp[e];
    g.sync();
  }
  __syncthreads();
  used = need;
  return found ? 1 : 0;
}

// Two-level decoupled look-back of one tile, done by the whole block.  Tiles
// of a sequence form groups of W consecutive tiles.  A tile first folds the
// earlier tiles of its own group (their aggregates, or down to the nearest
// inclusive prefix).  The last tile of a full group that found no prefix
// there publishes the group aggregate (the product over its group).  The
// walk then goes on over the last tiles of the earlier groups, W at a time,
// taking their group aggregates, down to the nearest inclusive prefix (the
// sequence's first tile always has one).  A tile at depth t of a sequence
// thus folds at most W - 1 + t/W payloads instead of t.  Tickets are taken in
// increasing order, so every tile waited on belongs to a block that is
// already running: the walk cannot deadlock.  Every wait is bounded
// (SPIN_LIMIT polls); past the bound the block latches DEVERR_TIMEOUT and
// finishes with what it has, so the kernel always terminates.
template <class Op>
__device__ bool lookback(const Grp<Op::G>& g, int gid, int NG, int W, const Ctx& c, unsigned long long epoch,
                         long long tile_id, long long t_in_seq, const typename Op::T* agg, typename Op::T* excl,
                         typename Op::T* tmp, typename Op::T* win, int* ctl, typename Op::T* sc,
                         typename Op::TS* scs) {
  unsigned char* ts = Op::tile_state(c, tile_id);
  bool ok = true;
  if (t_in_seq == 0) {
    if (gid == 0) {
      Op::identity(g, excl);
      publish<Op>(g, ts, agg, 1, 2u, epoch);
      g.sync();
    }
    __syncthreads();
    return ok;
  }
  if (gid == 0) {
    publish<Op>(g, ts, agg, 0, 1u, epoch);
    Op::identity(g, excl);
    g.sync();
  }
  __syncthreads();
  const long long j_lo = tile_id - t_in_seq;  // first tile of this sequence
  const int in_grp = (int)(t_in_seq % W);
  const long long g_lo = tile_id - in_grp;    // first tile of this tile's group
  int rc = 0, used = 0;
  // 1. earlier tiles of the own group
  long long j_hi = tile_id - 1;
  while (j_hi >= g_lo) {
    const int w = (int)min((long long)W, j_hi - g_lo + 1);
    rc = lookback_round<Op>(g, gid, NG, c, epoch, j_hi, 1, w, excl, tmp, win, ctl, sc, scs, ok, used);
    if (rc != 0) break;
    j_hi -= used;
  }
  // the last tile of a full group publishes the group aggregate
  if (rc == 0 && in_grp == W - 1) {
    if (gid == 0) {
      ok &= Op::combine(g, tmp, excl, agg, sc, scs, false);
      publish<Op>(g, ts, tmp, 2, 3u, epoch);
      g.sync();
    }
    __syncthreads();
  }
  // 2. the last tiles of the earlier groups
  j_hi = g_lo - 1;
  while (rc == 0 && j_hi >= j_lo) {
    const int w = (int)min((long long)W, (j_hi - j_lo) / W + 1);
    rc = lookback_round<Op>(g, gid, NG, c, epoch, j_hi, W, w, excl, tmp, win, ctl, sc, scs, ok, used);
    if (rc != 0) break;
    j_hi -= (long long)used * W;
  }
  if (gid == 0) {
    ok &= Op::combine(g, tmp, excl, agg, sc, scs, false);
    publish<Op>(g, ts, tmp, 1, 2u, epoch);
    g.sync();
  }
  __syncthreads();
  return ok;
}

template <class Op>
__global__ void __launch_bounds__(256) scan_kernel(Ctx c, int NG, int E, int W) {
  using T = typename Op::T;
  using TS = typename Op::TS;
  constexpr int G = Op::G, ES = Op::ES;
  extern __shared__ __align__(16) unsigned char smem[];
  if (!c.ctr->call_ok) return;  // metadata rejected for this call
  const int gid = threadIdx.x / G;
  const Grp<G> g;
  const size_t gb = ScanSmem<Op>::group_bytes();
  T* excl = (T*)smem;
  long long* s_tile = (long long*)(smem + align16(ES * sizeof(T)));
  int* ctl = (int*)(s_tile + 1);
  unsigned char* uni = (unsigned char*)s_tile + 32;
  unsigned char* gbase = uni + gid * gb;
  T* b0 = (T*)gbase;
  T* b1 = b0 + ES;
  T* b2 = b1 + ES;
  T* sc = b2 + ES;
  TS* scs = (TS*)(gbase + align16((3 * ES + Op::SCR) * sizeof(T)));
  T* ksA = (T*)(uni + NG * gb);
  T* ksB = (T*)((unsigned char*)ksA + align16((size_t)NG * ES * sizeof(T)));
  T* win = (T*)((unsigned char*)ksB + align16((size_t)NG * ES * sizeof(T)));
  unsigned char* esm = uni;  // the tile epilogue reuses the scan buffers

  const unsigned long long epoch = c.ctr->epoch;
  const long long* toff = Op::tile_off(c);
  // tiles of this launch: the whole call, or the sequences of one chunk of a
  // pipelined batch (tickets counted per chunk)
  long long t_lo = 0, total = Op::total_tiles(c);
  if (c.n_chunks > 1) {
    t_lo = toff[c.meta.chunk_seq[c.chunk]];
    total = toff[c.meta.chunk_seq[c.chunk + 1]];
  }
  const int tile_elems = Op::tile_elems(c);
  bool ok = true;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) *s_tile = t_lo + (long long)atomicAdd(&c.ctr->ticket[Op::TICKET + 2 * c.chunk], 1u);
    __syncthreads();
    const long long tile_id = *s_tile;
    if (tile_id >= total) break;
    const int s = find_segment(toff, c.n_seq, tile_id);
    const long long t = tile_id - toff[s];
    const int N = c.meta.nslow[s];
    const long long p0 = t * tile_elems + (long long)gid * E;
    const int cnt = (int)max(0LL, min((long long)E, (long long)N - p0));

    // 1. fold the group's elements
    T* cur = b0;
    T* el = b1;
    T* tmp = b2;
    Op::tile_begin(g, sc, c, s);
    if (cnt == 0) {
      Op::identity(g, cur);
    } else {
      Op::load(g, cur, c, s, p0, N);
      for (int e = 1; e < cnt; ++e) {
        g.sync();
        Op::load(g, el, c, s, p0 + e, N);
        g.sync();
        ok &= Op::combine_elem(g, tmp, cur, el, sc, scs, false, c, p0 + e);
        T* x = cur; cur = tmp; tmp = x;
      }
    }
    g.sync();
    for (int e = g.lane; e < ES; e += G) ksA[gid * ES + e] = cur[e];
    __syncthreads();
    // 2. inclusive scan over the groups of the tile
    T* src = ksA;
    T* dst = ksB;
    for (int d = 1; d < NG; d <<= 1) {
      if (gid >= d) {
        ok &= Op::combine(g, dst + gid * ES, src + (gid - d) * ES, src + gid * ES, sc, scs, false);
      } else {
        for (int e = g.lane; e < ES; e += G) dst[gid * ES + e] = src[gid * ES + e];
      }
      __syncthreads();
      T* x = src; src = dst; dst = x;
    }
    // 3. tile prefix
    ok &= lookback<Op>(g, gid, NG, W, c, epoch, tile_id, t, src + (NG - 1) * ES, excl, b2, win, ctl, sc, scs);
    if (c.reduce_only) {  // only the product of the whole range: the tile holding its last position writes it
      if (t == (long long)(N - 1) / tile_elems && gid == 0) {
        ok &= Op::combine(g, b0, excl, src + (NG - 1) * ES, sc, scs, false);
        for (int e = g.lane; e < ES; e += G) c.agg_out[e] = (double)b0[e];
      }
      continue;
    }
    // 4. results from the exclusive prefixes
    if (cnt > 0) {
      T* st = b0;
      T* nx = b2;
      if (gid == 0) {
        for (int e = g.lane; e < ES; e += G) st[e] = excl[e];
      } else {
        ok &= Op::combine(g, st, excl, src + (gid - 1) * ES, sc, scs, true);
      }
      g.sync();
      for (int e = 0; e < cnt; ++e) {
        Op::load(g, b1, c, s, p0 + e, N);
        g.sync();
        ok &= Op::combine_elem(g, nx, st, b1, sc, scs, true, c, p0 + e);
        T* x = st; st = nx; nx = x;
        Op::store(g, st, c, s, p0 + e, N, sc, scs);
        g.sync();
      }
    }
    if (Op::HAS_EPILOGUE && (Op::EPILOGUE_ALWAYS || !c.setup_separate)) {
      const long long tp0 = t * tile_elems;
      Op::epilogue(c, s, tp0, (int)min((long long)tile_elems, (long long)N - tp0), excl, esm);
    }
  }
  if (!ok && g.lane == 0) raise_err(c.ctr, DEVERR_SINGULAR);
}

// ===========================================================================
// fast-rate recovery (Remarks 1 and 3): one thread per fast step (k, i), a
// flat grid over every fast step of the call.  With the record of interval k
// and the smoothing terms (Om_k, om_k) formed by the smoother scan:
//   U_i    = A^i X + V_i H^T
//   m^f_i  = A^i m + U_i kap
//   P^f_ii = A^i P A^{iT} + Qc_i - (U_i S_y^-1) U_i^T     (P = L D L^T: (A^i L) D (A^i L)^T)
//   P^f_il = A^i (P A^{lT}) + Cov(e_i,e_l) - U_i (S_y^-1 U_l^T)
//   m^s_i  = m^f_i + P^f_il om,   P^s_ii = P^f_ii + P^f_il Om P^f_il^T  (Om = L D L^T)
// which is Eq. (17) and Eq. (21) with G_{k,i} = P^f_{k,i,l} A^T (P^-_{k+1,1})^-1,
// grouped so that no n x n product is repeated per fast step.  The last
// interval is smoothed = filtered (E_N = 0).  Covariances are formed on the
// upper triangle and mirrored (exactly symmetric).
// ===========================================================================
struct FastIdx {
  int s, l, N, i;     // sequence, ratio, slow steps, fast index in the interval (1-based)
  long long k, row;   // interval within the sequence, global slow row
};

__device__ __forceinline__ FastIdx fast_index(const Ctx& c, long long f) {
  FastIdx x;
  x.s = find_segment(c.meta.off_fast, c.n_seq, f);
  x.l = c.meta.ratio[x.s];
  x.N = c.meta.nslow[x.s];
  const long long loc = f - c.meta.off_fast[x.s];
  x.k = loc / x.l;
  x.i = (int)(loc - x.k * x.l) + 1;
  x.row = c.meta.off_slow[x.s] + x.k;
  return x;
}

// filtered moments of fast step x: m^f_i, P^f_ii (upper triangle) and, when
// need_pfl, P^f_il
// M = ny (compile-time): every loop over the measurement dimension runs
// exactly M times (the records keep their MY-padded strides).
template <int NX, int M, class TR>
__device__ __forceinline__ void recover_filtered(const Ctx& c, const FastIdx& x, bool need_pfl, TR (&mf)[NX],
                                                 TR (&Pf)[NX * (NX + 1) / 2], TR (&Pfl)[NX][NX]) {
  constexpr int NN = NX * NX, m = M;
  using RL = Rec<NX>;
  const int i = x.i;
  const double* md = c.model + (long long)x.s * c.ml.stride;
  const TR* rc = (const TR*)c.rec + x.row * RL::SIZE;
  const double* Ai = md + c.ml.Apow + (long long)i * NN;
  const double* VHi = md + c.ml.VH + (long long)(i - 1) * NX * m;
  const double* Qci = md + c.ml.Qc + (long long)(i - 1) * NN;
  const double* Qli = md + c.ml.Ql + (long long)(i - 1) * NN;
  TR a[NX][NX];
#pragma unroll
  for (int r = 0; r < NX; ++r)
#pragma unroll
    for (int q = 0; q < NX; ++q) a[r][q] = (TR)__ldg(Ai + r * NX + q);
  // U_i = A^i X + V_i H^T
  TR U[NX][M];
#pragma unroll
  for (int r = 0; r < NX; ++r)
#pragma unroll
    for (int jj = 0; jj < M; ++jj) {
      TR v = (TR)__ldg(VHi + r * m + jj);
#pragma unroll
      for (int q = 0; q < NX; ++q) v = fma(a[r][q], rc[RL::X + q * MY + jj], v);
      U[r][jj] = v;
    }
  // m^f_i = A^i m + U_i kap (+ b_{k,i} = sum_{q<i} A^{i-1-q} B u_{k,q} with inputs)
#pragma unroll
  for (int r = 0; r < NX; ++r) {
    TR v = TR(0);
#pragma unroll
    for (int q = 0; q < NX; ++q) v = fma(a[r][q], rc[RL::mv + q], v);
#pragma unroll
    for (int jj = 0; jj < M; ++jj) v = fma(U[r][jj], rc[RL::kap + jj], v);
    mf[r] = v;
  }
  if (c.nu > 0) {
    const int nu = c.nu;
    const double* uk = c.u + (c.meta.off_fast[x.s] + x.k * x.l) * nu;
    const double* AB = md + c.ml.AB;
    for (int q = 0; q < i; ++q)
      for (int j = 0; j < nu; ++j) {
        const double uq = __ldg(uk + q * nu + j);
        const double* ab = AB + ((long long)(i - 1 - q) * NX) * nu + j;
#pragma unroll
        for (int r = 0; r < NX; ++r) mf[r] = fma((TR)__ldg(ab + r * nu), (TR)uq, mf[r]);
      }
  }
  // P^f_il = A^i Pl + Cov(e_i,e_l) - U_i SUl
  if (need_pfl) {
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        TR v = (TR)__ldg(Qli + r * NX + q);
#pragma unroll
        for (int t = 0; t < NX; ++t) v = fma(a[r][t], rc[RL::Pl + t * NX + q], v);
#pragma unroll
        for (int jj = 0; jj < M; ++jj) v = fma(-U[r][jj], rc[RL::SUl + jj * NX + q], v);
        Pfl[r][q] = v;
      }
  }
  // P^f_ii (upper triangle)
  {
    TR US[NX][M], B[NX][NX], BD[NX][NX];
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int jj = 0; jj < M; ++jj) {
        TR v = TR(0);
#pragma unroll
        for (int j2 = 0; j2 < M; ++j2) v = fma(U[r][j2], rc[RL::Si + j2 * MY + jj], v);
        US[r][jj] = v;
      }
    // A^i P A^iT with P = L D L^T (the record's factors): B = A^i L, then
    // (B D) B^T on the upper triangle
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        TR v = a[r][q];
#pragma unroll
        for (int t = q + 1; t < NX; ++t) v = fma(a[r][t], rc[RL::P + t * NX + q], v);
        B[r][q] = v;
        BD[r][q] = v * rc[RL::P + q * NX + q];
      }
    int u = 0;
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int q = r; q < NX; ++q) {
        TR v = (TR)__ldg(Qci + r * NX + q);
#pragma unroll
        for (int t = 0; t < NX; ++t) v = fma(BD[r][t], B[q][t], v);
#pragma unroll
        for (int jj = 0; jj < M; ++jj) v = fma(-US[r][jj], U[q][jj], v);
        Pf[u++] = v;
      }
  }
}

// smoothing update in place: m += P^f_il om, P += P^f_il Om P^f_il^T (upper)
// with Om = L D L^T given by its factors (L below the diagonal, D on it):
// B = P^f_il L, then (B D) B^T
template <int NX, class TR>
__device__ __forceinline__ void recover_smooth(const TR* Om, const TR* om, TR (&mf)[NX], TR (&Pf)[NX * (NX + 1) / 2],
                                               const TR (&Pfl)[NX][NX]) {
  TR B[NX][NX], BD[NX][NX];
#pragma unroll
  for (int r = 0; r < NX; ++r)
#pragma unroll
    for (int q = 0; q < NX; ++q) {
      TR v = Pfl[r][q];
#pragma unroll
      for (int t = q + 1; t < NX; ++t) v = fma(Pfl[r][t], Om[t * NX + q], v);
      B[r][q] = v;
      BD[r][q] = v * Om[q * NX + q];
    }
  int u = 0;
#pragma unroll
  for (int r = 0; r < NX; ++r)
#pragma unroll
    for (int q = r; q < NX; ++q) {
      TR v = Pf[u];
#pragma unroll
      for (int t = 0; t < NX; ++t) v = fma(BD[r][t], B[q][t], v);
      Pf[u++] = v;
    }
#pragma unroll
  for (int r = 0; r < NX; ++r) {
    TR v = mf[r];
#pragma unroll
    for (int t = 0; t < NX; ++t) v = fma(Pfl[r][t], om[t], v);
    mf[r] = v;
  }
}

// P += (W Lf) Df (W Lf)^T on the upper triangle, with Lf Df Lf^T given by
// its factors f (Lf below the diagonal, Df on it)
template <int NX, class TR>
__device__ __forceinline__ void add_factored_quad(const TR (&W)[NX][NX], const TR* f, TR (&P)[NX * (NX + 1) / 2]) {
  TR B[NX][NX], BD[NX][NX];
#pragma unroll
  for (int r = 0; r < NX; ++r)
#pragma unroll
    for (int q = 0; q < NX; ++q) {
      TR v = W[r][q];
#pragma unroll
      for (int t = q + 1; t < NX; ++t) v = fma(W[r][t], f[t * NX + q], v);
      B[r][q] = v;
      BD[r][q] = v * f[q * NX + q];
    }
  int u = 0;
#pragma unroll
  for (int r = 0; r < NX; ++r)
#pragma unroll
    for (int q = r; q < NX; ++q) {
      TR v = P[u];
#pragma unroll
      for (int t = 0; t < NX; ++t) v = fma(BD[r][t], B[q][t], v);
      P[u++] = v;
    }
}

// Two-point recovery of fast step x (a sequence whose bflag is set), from
// the interval's terms (BRec) and the constants of fast index i:
//   m^s_{k,i} = C1_i mu0 + C2_i mu1 + c3_i y_k,
//   P^s_{k,ii} = Sg_i + [C1_i C2_i] J_k [C1_i C2_i]^T,
// J_k the smoothed joint covariance of (x_{k,1}, x_{k+1,1}).  With
// x_{k,1} = E_k x_{k+1,1} + (independent part of covariance S_k),
//   [C1 C2] J [C1 C2]^T = (C1 E_k + C2) P^s_{k+1,1} (C1 E_k + C2)^T + C1 S_k C1^T,
// each quadratic form from its LDL^T factors.  The last interval conditions
// on (x_{k,1}, y_k) only: Sg'_i + C1'_i P^s_{k,1} C1'_i^T.
template <int NX, int M, class TR>
__device__ __forceinline__ void recover_two_point(const Ctx& c, const FastIdx& x, TR (&mf)[NX],
                                                  TR (&Pf)[NX * (NX + 1) / 2]) {
  constexpr int NN = NX * NX, BT = 3 * NN + NX * MY, BO = 2 * NN + NX * MY;
  using B = BRec<NX>;
  const double* md = c.model + (long long)x.s * c.ml.stride;
  const TR* b = (const TR*)c.brec + x.row * B::SIZE;
  const bool two = x.k < x.N - 1;
  const double* K = md + (two ? c.ml.BrT + (long long)(x.i - 1) * BT : c.ml.BrO + (long long)(x.i - 1) * BO);
  const double* Sg = K + (two ? 2 * NN : NN);
  const double* c3 = K + (two ? 3 * NN : 2 * NN);
  const double* yk = c.y + x.row * M;
  TR C1[NX][NX];
#pragma unroll
  for (int r = 0; r < NX; ++r)
#pragma unroll
    for (int q = 0; q < NX; ++q) C1[r][q] = (TR)__ldg(K + r * NX + q);
#pragma unroll
  for (int r = 0; r < NX; ++r) {
    TR v = TR(0);
#pragma unroll
    for (int q = 0; q < NX; ++q) v = fma(C1[r][q], b[B::mu0 + q], v);
#pragma unroll
    for (int j = 0; j < M; ++j) v = fma((TR)__ldg(c3 + r * MY + j), (TR)__ldg(yk + j), v);
    mf[r] = v;
  }
  {
    int u = 0;
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int q = r; q < NX; ++q) Pf[u++] = (TR)__ldg(Sg + r * NX + q);
  }
  if (two) {
    const double* C2 = K + NN;
    TR W[NX][NX];
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      TR v = mf[r];
#pragma unroll
      for (int q = 0; q < NX; ++q) {
        const TR c2 = (TR)__ldg(C2 + r * NX + q);
        v = fma(c2, b[B::mu1 + q], v);
        TR w = c2;
#pragma unroll
        for (int t = 0; t < NX; ++t) w = fma(C1[r][t], b[B::E + t * NX + q], w);
        W[r][q] = w;
      }
      mf[r] = v;
    }
    add_factored_quad<NX, TR>(W, b + B::L1, Pf);
  }
  add_factored_quad<NX, TR>(C1, b + B::L2, Pf);
}

// Output stores of the recovery.  The fast rows of a warp (32 consecutive
// fast steps) are contiguous in the outputs, so each lane first puts its mean
// and mirrored covariance into the warp's shared-memory slab and the warp then
// writes the block out with consecutive lanes on consecutive words: every
// store instruction covers whole cache lines (this matters most when the
// outputs are pinned host memory written over the CPU-GPU link).  The slow
// row (i == l, one fast step in l) is written by its own thread.
template <int NX>
struct RecSlab {
  static constexpr int NN = NX * NX, ROW = NX + NN;
  static constexpr int MEAN = 0, COV = 32 * NX;  // offsets in the warp's slab (doubles)
  static constexpr int WARP_DOUBLES = 32 * ROW;
};

// cnt consecutive doubles from shared memory to global memory: as 16-byte
// stores (the odd last one by lane 0) when both dst and src are 16-byte
// aligned, else as 8-byte stores
__device__ __forceinline__ void warp_copy_out(double* dst, const double* src, int cnt, int lane) {
  if ((reinterpret_cast<uintptr_t>(dst) | reinterpret_cast<uintptr_t>(src)) & 15) {
    for (int e = lane; e < cnt; e += 32) dst[e] = src[e];
    return;
  }
  const int pairs = cnt >> 1;
  double2* d2 = reinterpret_cast<double2*>(dst);
  const double2* s2 = reinterpret_cast<const double2*>(src);
  for (int e = lane; e < pairs; e += 32) d2[e] = s2[e];
  if ((cnt & 1) && lane == 0) dst[cnt - 1] = src[cnt - 1];
}

// The warp's 32 rows f0 .. f0+31 (f0 a multiple of 32) go through the slab;
// rows v0 .. v1-1 of them are this launch's and are written.
template <int NX, class TR>
__device__ __forceinline__ void warp_store_fast(double* slab, int lane, long long f0, int v0, int v1, bool active,
                                                double* mo, double* co, const TR* mv, const TR* Pu) {
  using SB = RecSlab<NX>;
  constexpr int NN = NX * NX;
  if (!mo && !co) return;  // uniform over the warp
  __syncwarp();
  if (active) {
#pragma unroll
    for (int r = 0; r < NX; ++r) slab[SB::MEAN + lane * NX + r] = (double)mv[r];
    int u = 0;
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int q = r; q < NX; ++q) {
        const double v = (double)Pu[u++];
        slab[SB::COV + lane * NN + r * NX + q] = v;
        slab[SB::COV + lane * NN + q * NX + r] = v;
      }
  }
  __syncwarp();
  // f0 is a multiple of 32, so dst and src offsets have the same parity and a
  // 16-byte aligned output base gives 16-byte stores
  if (mo) warp_copy_out(mo + (f0 + v0) * NX, slab + SB::MEAN + v0 * NX, (v1 - v0) * NX, lane);
  if (co) warp_copy_out(co + (f0 + v0) * NN, slab + SB::COV + v0 * NN, (v1 - v0) * NN, lane);
}

template <int NX, class TR>
__device__ __forceinline__ void store_slow(long long row, double* smo, double* sco, const TR* mv, const TR* Pu) {
  constexpr int NN = NX * NX;
  if (smo) {
#pragma unroll
    for (int r = 0; r < NX; ++r) smo[row * NX + r] = (double)mv[r];
  }
  if (sco) {
    double* dst = sco + row * NN;
    int u = 0;
#pragma unroll
    for (int r = 0; r < NX; ++r)
#pragma unroll
      for (int q = r; q < NX; ++q) {
        const double v = (double)Pu[u++];
        dst[r * NX + q] = v;
        dst[q * NX + r] = v;
      }
  }
}

// dynamic shared memory of the recovery: one slab per warp
template <int NX>
__host__ __device__ inline size_t recover_smem_bytes(int threads) {
  return (size_t)((threads + 31) / 32) * RecSlab<NX>::WARP_DOUBLES * sizeof(double);
}

// PHASE 0: the whole recovery after the smoother scan.  PHASE 1 / 2: the two
// halves of a split recovery.  PHASE 1 needs only the filter scan and the
// interval setup, so it runs on a second stream while the smoother scan runs:
// it forms the filtered moments (and P^f_il), writes the filtered outputs the
// caller asked for and keeps the moments in c.rscr.  PHASE 2 runs after the
// smoother scan: it reads them back, applies the smoothing terms and writes
// the smoothed outputs.  The arithmetic and its order are those of PHASE 0,
// so for the same scan results the outputs are identical.
template <int NX, int M, class TR, int PHASE>
__global__ void __launch_bounds__(128, 3) recover_kernel(Ctx c) {
  constexpr int NT = NX * (NX + 1) / 2, NN = NX * NX;
  using RS = RecScr<NX>;
  extern __shared__ __align__(16) double rslab[];
  if (!c.ctr->call_ok) return;
  // fast steps of this launch: the whole call, or one chunk of a pipelined batch
  long long f_lo = 0, f_hi = c.total_fast;
  if (c.n_chunks > 1) {
    f_lo = c.meta.off_fast[c.meta.chunk_seq[c.chunk]];
    f_hi = c.meta.off_fast[c.meta.chunk_seq[c.chunk + 1]];
  }
  const int lane = threadIdx.x & 31;
  double* slab = rslab + (size_t)(threadIdx.x >> 5) * RecSlab<NX>::WARP_DOUBLES;
  const long long grid_warps = ((long long)gridDim.x * blockDim.x) >> 5;
  // warps take aligned blocks of 32 fast rows (f0 = 32 wb) that meet
  // [f_lo, f_hi); with a grid of one thread per fast step each warp makes one
  // trip, a smaller grid loops
  for (long long wb = (f_lo >> 5) + ((blockIdx.x * (long long)blockDim.x + threadIdx.x) >> 5); wb * 32 < f_hi;
       wb += grid_warps) {
    const long long f0 = wb * 32, f = f0 + lane;
    const int v0 = (int)max(0LL, f_lo - f0), v1 = (int)min(32LL, f_hi - f0);
    const bool active = lane >= v0 && lane < v1;
    FastIdx x;
    bool last_i = false, smooth_k = false;
    TR mf[NX], Pf[NT], Pfl[NX][NX];
    if (active) {
      x = fast_index(c, f);
      last_i = x.i == x.l;
      smooth_k = c.smoothing && (x.k < x.N - 1 || c.split_tail_open);
      if (PHASE == 0 && c.bridge && c.model[(long long)x.s * c.ml.stride + c.ml.bflag] != 0.0) {
        recover_two_point<NX, M, TR>(c, x, mf, Pf);  // the smoothed moments themselves
        smooth_k = false;
      } else if (PHASE < 2) {
        recover_filtered<NX, M, TR>(c, x, smooth_k, mf, Pf, Pfl);
      } else {  // component-major: a warp reads 32 consecutive words per component
        const TR* src = (const TR*)c.rscr + f;
        const long long T = c.total_fast;
#pragma unroll
        for (int r = 0; r < NX; ++r) mf[r] = src[(RS::mf + r) * T];
#pragma unroll
        for (int u = 0; u < NT; ++u) Pf[u] = src[(RS::Pf + u) * T];
        if (smooth_k)
#pragma unroll
          for (int e = 0; e < NN; ++e) Pfl[e / NX][e % NX] = src[(RS::Pfl + e) * T];
      }
    }
    // filtered outputs (the call's outputs for a filter, the optional extras for a smoother)
    if (!c.smoothing) {
      warp_store_fast<NX, TR>(slab, lane, f0, v0, v1, active, c.fast_mean, c.fast_cov, mf, Pf);
      if (active && last_i) store_slow<NX, TR>(x.row, c.slow_mean, c.slow_cov, mf, Pf);
      continue;
    }
    if (PHASE < 2) {
      warp_store_fast<NX, TR>(slab, lane, f0, v0, v1, active, c.ffast_mean, c.ffast_cov, mf, Pf);
      if (active && last_i) store_slow<NX, TR>(x.row, c.fslow_mean, c.fslow_cov, mf, Pf);
    }
    if (PHASE == 1) {
      if (active) {  // component-major, as read back
        TR* dst = (TR*)c.rscr + f;
        const long long T = c.total_fast;
#pragma unroll
        for (int r = 0; r < NX; ++r) dst[(RS::mf + r) * T] = mf[r];
#pragma unroll
        for (int u = 0; u < NT; ++u) dst[(RS::Pf + u) * T] = Pf[u];
        if (smooth_k)
#pragma unroll
          for (int e = 0; e < NN; ++e) dst[(RS::Pfl + e) * T] = Pfl[e / NX][e % NX];
      }
      continue;
    }
    if (active && smooth_k) {
      const TR* Om = (const TR*)c.sfin + x.row * SFin<NX>::SIZE;
      recover_smooth<NX, TR>(Om + SFin<NX>::Om, Om + SFin<NX>::om, mf, Pf, Pfl);
    }
    warp_store_fast<NX, TR>(slab, lane, f0, v0, v1, active, c.fast_mean, c.fast_cov, mf, Pf);
    if (active && last_i) store_slow<NX, TR>(x.row, c.slow_mean, c.slow_cov, mf, Pf);
  }
}

// ===========================================================================
// per-interval input terms (known inputs only): one thread per interval,
// from the model's A^j B and S_j B tables (ld nu, j < l):
//   b_{k,l} = sum_q A^{l-1-q} B u_{k,q},   b_{k,1} = B u_{k,0},
//   B u_{k,l} = B u_{k+1,0} (0 for the last interval),
//   c_k = H sum_i b_{k,i} = H sum_q S_{l-1-q} B u_{k,q}
// ===========================================================================
template <int NX>
__global__ void __launch_bounds__(128) input_kernel(Ctx c) {
  using UI = UIn<NX>;
  if (!c.ctr->call_ok) return;
  const long long gi = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (gi >= c.total_slow) return;
  const int s = find_segment(c.meta.off_slow, c.n_seq, gi);
  const long long k = gi - c.meta.off_slow[s];
  const int l = c.meta.ratio[s], N = c.meta.nslow[s], nu = c.nu, m = c.ny;
  const double* md = c.model + (long long)s * c.ml.stride;
  const double* B = c.B + (long long)s * NX * nu;
  const double* H = c.H + (long long)s * m * NX;
  const double* uk = c.u + (c.meta.off_fast[s] + k * l) * nu;
  double bl[NX], sb[NX], b1[NX], bn[NX];
#pragma unroll
  for (int r = 0; r < NX; ++r) bl[r] = sb[r] = b1[r] = bn[r] = 0.0;
  for (int q = 0; q < l; ++q)
    for (int j = 0; j < nu; ++j) {
      const double uq = uk[q * nu + j];
      const double* ab = md + c.ml.AB + ((long long)(l - 1 - q) * NX) * nu + j;
      const double* sbt = md + c.ml.SB + ((long long)(l - 1 - q) * NX) * nu + j;
#pragma unroll
      for (int r = 0; r < NX; ++r) {
        bl[r] = fma(ab[r * nu], uq, bl[r]);
        sb[r] = fma(sbt[r * nu], uq, sb[r]);
      }
    }
  for (int j = 0; j < nu; ++j) {
    const double u0 = uk[j], un = (k < N - 1) ? uk[l * nu + j] : 0.0;
#pragma unroll
    for (int r = 0; r < NX; ++r) {
      b1[r] = fma(B[r * nu + j], u0, b1[r]);
      bn[r] = fma(B[r * nu + j], un, bn[r]);
    }
  }
  double* out = c.uin + gi * UI::SIZE;
#pragma unroll
  for (int r = 0; r < NX; ++r) {
    out[UI::bl + r] = bl[r];
    out[UI::b1 + r] = b1[r];
    out[UI::bn + r] = bn[r];
  }
  for (int i = 0; i < MY; ++i) {
    double v = 0.0;
    if (i < m)
#pragma unroll
      for (int r = 0; r < NX; ++r) v = fma(H[i * NX + r], sb[r], v);
    out[UI::c + i] = v;
  }
}

// ===========================================================================
// interval setup as its own kernel (after the filter scan): blocks of 128
// threads, SG lanes per interval, one interval per lane group.
// ===========================================================================
template <int NX, int M, class T, class TS>
__global__ void __launch_bounds__(128) setup_kernel(Ctx c) {
  using Gm = SetupGeom<NX>;
  constexpr int SG = Gm::SG;
  extern __shared__ __align__(16) unsigned char ssm[];
  if (!c.ctr->call_ok) return;
  const int lane = threadIdx.x % SG, slot = threadIdx.x / SG, per = blockDim.x / SG;
  // intervals of this launch: the whole call, or one chunk of a pipelined batch
  long long g_lo = 0, g_hi = c.total_slow;
  if (c.n_chunks > 1) {
    g_lo = c.meta.off_slow[c.meta.chunk_seq[c.chunk]];
    g_hi = c.meta.off_slow[c.meta.chunk_seq[c.chunk + 1]];
  }
  const unsigned mask = (SG == 32) ? 0xffffffffu : (((1u << SG) - 1u) << ((threadIdx.x & 31) & ~(SG - 1)));
  unsigned char* sl = ssm + (size_t)slot * Gm::template slot_bytes<T, TS>();
  T* sf = (sizeof(T) != sizeof(TS)) ? (T*)((TS*)sl + Gm::FREG) : nullptr;
  // rounds of `per` intervals, one per lane group (uniform over the block),
  // then the round's records' P^f_{k-1,l} as LDL^T factors, one thread each
  for (long long base = g_lo + (long long)blockIdx.x * per; base < g_hi; base += (long long)gridDim.x * per) {
    if (base + slot < g_hi) setup_interval<NX, M, T, TS>(c, base + slot, lane, mask, (TS*)sl, sf, nullptr);
    __syncthreads();
    const long long gi = base + threadIdx.x;
    if (threadIdx.x < per && gi < g_hi && (!c.bridge || records_needed(c, find_segment(c.meta.off_slow, c.n_seq, gi))))
      ldlt_inplace<NX, TS>((TS*)c.rec + gi * Rec<NX>::SIZE + Rec<NX>::P);
    __syncthreads();
  }
}

// ===========================================================================
// host-side launch of the templated stages
// ===========================================================================
template <int NX, int M, class T, class TS>
struct SetupTag {};
template <int NX, int M, class TR, int PHASE>
struct RecoverTag {};

// Raises (never lowers) a kernel's dynamic shared-memory limit on the current
// device: launches with other shapes may still need a larger limit.
template <class Op>
inline void set_smem_attr(const void* fn, size_t bytes) {
  static size_t granted[64] = {};
  int dev = 0;
  cudaGetDevice(&dev);
  if (bytes > 48 * 1024 && (dev < 0 || dev >= 64 || bytes > granted[dev])) {
    cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes);
    if (dev >= 0 && dev < 64) granted[dev] = bytes;
  }
}

// The recovery is compiled per measurement size (M = ny = 1..4); the
// smoothing half of a split recovery does not depend on it (one variant).
template <int NX, class TR, int PHASE>
inline void set_recover_smem(size_t bytes) {
  set_smem_attr<RecoverTag<NX, 1, TR, PHASE>>((const void*)recover_kernel<NX, 1, TR, PHASE>, bytes);
  if constexpr (PHASE != 2) {
    set_smem_attr<RecoverTag<NX, 2, TR, PHASE>>((const void*)recover_kernel<NX, 2, TR, PHASE>, bytes);
    set_smem_attr<RecoverTag<NX, 3, TR, PHASE>>((const void*)recover_kernel<NX, 3, TR, PHASE>, bytes);
    set_smem_attr<RecoverTag<NX, 4, TR, PHASE>>((const void*)recover_kernel<NX, 4, TR, PHASE>, bytes);
  }
}

template <int NX, class TR, int PHASE>
inline void launch_recover(const Ctx& c, unsigned blocks, int threads, size_t smem, cudaStream_t st) {
  if constexpr (PHASE == 2) {
    recover_kernel<NX, 1, TR, PHASE><<<blocks, threads, smem, st>>>(c);
  } else {
    switch (c.ny) {
      case 1: recover_kernel<NX, 1, TR, PHASE><<<blocks, threads, smem, st>>>(c); break;
      case 2: recover_kernel<NX, 2, TR, PHASE><<<blocks, threads, smem, st>>>(c); break;
      case 3: recover_kernel<NX, 3, TR, PHASE><<<blocks, threads, smem, st>>>(c); break;
      default: recover_kernel<NX, 4, TR, PHASE><<<blocks, threads, smem, st>>>(c); break;
    }
  }
}

template <int NX, class T, class TS, class TR>
int query_shapes_t(int scan_groups, int scan_elems, int window, int recover_threads, int setup_separate,
                   int sm_count, long long total_slow, int n_seq, Shapes* sh) {
  using FOp = FilterOp<NX, T, TS>;
  using SOp = SmootherOp<NX, T, TR>;
  constexpr int G = FOp::G;
  const int NG = scan_groups;
  const int threads = NG * G;
  if (threads < 32 || threads > 256 || window < 1 || window > ScanSmem<FOp>::MAXWIN) return SRTM_ERR_ARG;
  sh->scan_groups_f = sh->scan_groups_s = NG;
  sh->scan_elems_f = sh->scan_elems_s = scan_elems;
  sh->window_f = sh->window_s = window;
  sh->smem_f = ScanSmem<FOp>::bytes(NG, window, scan_elems, !setup_separate);
  sh->smem_s = ScanSmem<SOp>::bytes(NG, window, scan_elems);
  set_smem_attr<FOp>((const void*)scan_kernel<FOp>, sh->smem_f);
  set_smem_attr<SOp>((const void*)scan_kernel<SOp>, sh->smem_s);
  int nb = 0;
  const long long tiles = total_slow / ((long long)NG * scan_elems) + n_seq;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, scan_kernel<FOp>, threads, sh->smem_f);
  sh->blocks_per_sm_f = std::max(nb, 1);
  sh->grid_f = (int)std::max(1LL, std::min((long long)sh->blocks_per_sm_f * sm_count, tiles));
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, scan_kernel<SOp>, threads, sh->smem_s);
  sh->blocks_per_sm_s = std::max(nb, 1);
  sh->grid_s = (int)std::max(1LL, std::min((long long)sh->blocks_per_sm_s * sm_count, tiles));
  sh->grid_setup = (int)((total_slow + 128 / SetupGeom<NX>::SG - 1) / (128 / SetupGeom<NX>::SG));
  sh->smem_setup = setup_separate ? (size_t)(128 / SetupGeom<NX>::SG) * SetupGeom<NX>::template slot_bytes<T, TS>() : 0;
  if (setup_separate) {  // the setup kernel is compiled per measurement size
    set_smem_attr<SetupTag<NX, 1, T, TS>>((const void*)setup_kernel<NX, 1, T, TS>, sh->smem_setup);
    set_smem_attr<SetupTag<NX, 2, T, TS>>((const void*)setup_kernel<NX, 2, T, TS>, sh->smem_setup);
    set_smem_attr<SetupTag<NX, 3, T, TS>>((const void*)setup_kernel<NX, 3, T, TS>, sh->smem_setup);
    set_smem_attr<SetupTag<NX, 4, T, TS>>((const void*)setup_kernel<NX, 4, T, TS>, sh->smem_setup);
  }
  sh->recover_threads = recover_threads;
  set_recover_smem<NX, TR, 0>(recover_smem_bytes<NX>(recover_threads));
  set_recover_smem<NX, TR, 1>(recover_smem_bytes<NX>(recover_threads));
  set_recover_smem<NX, TR, 2>(recover_smem_bytes<NX>(recover_threads));
  if (cudaGetLastError() != cudaSuccess) return SRTM_ERR_CUDA;
  return SRTM_OK;
}

template <int NX>
int query_shapes(srtm_precision prec, int scan_groups, int scan_elems, int window, int recover_threads,
                 int setup_separate, int sm_count, long long total_slow, int n_seq, Shapes* sh) {
  switch (prec) {
    case SRTM_FP64:
      return query_shapes_t<NX, double, double, double>(scan_groups, scan_elems, window, recover_threads,
                                                         setup_separate, sm_count, total_slow, n_seq, sh);
    case SRTM_MIXED:
      return query_shapes_t<NX, float, double, double>(scan_groups, scan_elems, window, recover_threads,
                                                        setup_separate, sm_count, total_slow, n_seq, sh);
    case SRTM_FP32:
      return query_shapes_t<NX, float, float, float>(scan_groups, scan_elems, window, recover_threads,
                                                      setup_separate, sm_count, total_slow, n_seq, sh);
  }
  return SRTM_ERR_ARG;
}

// The last interval of a range of a split sequence that does not end it (one
// lane group, after the interval setup, before the smoother scan): with the
// smoothed x_{N,1} = N(next_mean, next_cov) that follows the range (formed
// from the later ranges' smoother aggregates, Eq. 30),
//   its smoothing terms Om, om for the recovery (as the smoother scan's result
//   pass forms them for every other interval), and
//   its smoother element b_{N-1} <- b_{N-1} (x) (0, next_mean, next_cov), so
//   that the range's suffix scan yields the smoothed x_{k,1} of the whole
//   sequence (Sec. II: the operator is associative).
template <int NX, class T, class TR>
__global__ void __launch_bounds__(32) split_tail_kernel(Ctx c) {
  using SOp = SmootherOp<NX, T, TR>;
  using L = SL<NX>;
  constexpr int G = SOp::G, ES = SOp::ES, NN = NX * NX;
  __shared__ T x[ES], b[ES], o[ES], sc[NN];
  __shared__ TR scs[SOp::SCRS];
  if (!c.ctr->call_ok || threadIdx.x >= G) return;
  const Grp<G> g;
  const long long N = c.total_slow;
  for (int e = g.lane; e < NN; e += G) {
    x[L::E + e] = T(0);
    x[L::S + e] = (T)c.next_cov[e];
  }
  for (int e = g.lane; e < NX; e += G) x[L::g + e] = (T)c.next_mean[e];
  g.sync();
  SOp::store(g, x, c, 0, -1, (int)N, sc, scs);  // scan position -1 is slow step N: terms of interval N-1
  if (g.lane == 0) ldlt_inplace<NX, TR>((TR*)c.sfin + (N - 1) * SFin<NX>::SIZE + SFin<NX>::Om);
  T* el = (T*)c.selem + (N - 1) * ES;
  for (int e = g.lane; e < ES; e += G) b[e] = el[e];
  g.sync();
  g_smoother_combine<NX, G, T>(g, o, b, x, sc, true);  // x is a suffix with E = 0
  for (int e = g.lane; e < ES; e += G) el[e] = o[e];
}

template <int NX, class T, class TS>
inline void launch_setup(const Ctx& c, unsigned grid, size_t smem, cudaStream_t st) {
  switch (c.ny) {
    case 1: setup_kernel<NX, 1, T, TS><<<grid, 128, smem, st>>>(c); break;
    case 2: setup_kernel<NX, 2, T, TS><<<grid, 128, smem, st>>>(c); break;
    case 3: setup_kernel<NX, 3, T, TS><<<grid, 128, smem, st>>>(c); break;
    default: setup_kernel<NX, 4, T, TS><<<grid, 128, smem, st>>>(c); break;
  }
}

// A batch in chunks of whole sequences (after the metadata, constants and
// input kernels): on `st` the filter scan, interval setup and smoother scan of
// chunk q; on the library's second stream the fast-rate recovery of chunk q,
// which waits for chunk q's scans and runs while `st` goes on with the scans
// of chunk q+1 (Remark 1: the recovery of an interval needs only that
// interval's scan results).  The chunks' rows are disjoint, so the launches
// share the workspace without conflict.  Stage events (optional): ev[1..3]
// after the last chunk's scans, ev[4] after the last recovery, ev[8+2q] and
// ev[9+2q] around the recovery of chunk q (on the second stream).
template <int NX, class T, class TS, class TR>
int launch_chunks(const Ctx& c, const Shapes& sh, cudaStream_t st, cudaEvent_t* ev, const SideStream* side) {
  using FOp = FilterOp<NX, T, TS>;
  using SOp = SmootherOp<NX, T, TR>;
  constexpr int G = FOp::G;
  const size_t rsmem = recover_smem_bytes<NX>(sh.recover_threads);
  for (int q = 0; q < c.n_chunks; ++q) {
    Ctx cq = c;
    cq.chunk = q;
    scan_kernel<FOp><<<sh.grid_f_chunk, sh.scan_groups_f * G, sh.smem_f, st>>>(cq, sh.scan_groups_f, sh.scan_elems_f,
                                                                             sh.window_f);
    if (c.setup_separate) launch_setup<NX, T, TS>(cq, (unsigned)sh.grid_setup_chunk, sh.smem_setup, st);
    if (c.smoothing)
      scan_kernel<SOp><<<sh.grid_s_chunk, sh.scan_groups_s * G, sh.smem_s, st>>>(cq, sh.scan_groups_s, sh.scan_elems_s,
                                                                               sh.window_s);
    cudaEventRecord(side->fork, st);
    cudaStreamWaitEvent(side->st, side->fork, 0);
    if (ev) cudaEventRecord(ev[8 + 2 * q], side->st);
    launch_recover<NX, TR, 0>(cq, (unsigned)sh.grid_recover_chunk, sh.recover_threads, rsmem, side->st);
    if (ev) cudaEventRecord(ev[9 + 2 * q], side->st);
  }
  if (ev)
    for (int i = 1; i <= 3; ++i) cudaEventRecord(ev[i], st);
  cudaEventRecord(side->join, side->st);
  cudaStreamWaitEvent(st, side->join, 0);
  launch_loglik(c, st);
  if (ev) cudaEventRecord(ev[4], st);
  return cudaGetLastError() == cudaSuccess ? SRTM_OK : SRTM_ERR_CUDA;
}

// ev (optional): five events recorded after the constants, the filter scan,
// the interval setup, the smoother scan and the recovery; with a split
// recovery also ev[5] before its smoothing half and ev[6], ev[7] around its
// filtered half (second stream).
template <int NX, class T, class TS, class TR>
int launch_t(const Ctx& c, const Shapes& sh, cudaStream_t st, cudaEvent_t* ev, const SideStream* side) {
  using FOp = FilterOp<NX, T, TS>;
  using SOp = SmootherOp<NX, T, TR>;
  constexpr int G = FOp::G;
  launch_precompute<NX>(c, st);
  if (c.uin) input_kernel<NX><<<(unsigned)((c.total_slow + 127) / 128), 128, 0, st>>>(c);
  if (ev) cudaEventRecord(ev[0], st);
  if (c.n_chunks > 1 && side) return launch_chunks<NX, T, TS, TR>(c, sh, st, ev, side);
  if (c.split_mode == 1) {  // the filter aggregate of a range of a split sequence: a reducing scan only
    Ctx cr = c;
    cr.reduce_only = 1;
    scan_kernel<FOp><<<sh.grid_f, sh.scan_groups_f * G, sh.smem_f, st>>>(cr, sh.scan_groups_f, sh.scan_elems_f,
                                                                        sh.window_f);
    if (ev)
      for (int i = 1; i <= 4; ++i) cudaEventRecord(ev[i], st);
    return cudaGetLastError() == cudaSuccess ? SRTM_OK : SRTM_ERR_CUDA;
  }
  const unsigned seq_blocks = (unsigned)((c.n_seq + SEQ_THREADS - 1) / SEQ_THREADS);
  if (c.sequential) {
    switch (c.ny) {
      case 1: seq_filter_kernel<NX, 1, TS><<<seq_blocks, SEQ_THREADS, 0, st>>>(c); break;
      case 2: seq_filter_kernel<NX, 2, TS><<<seq_blocks, SEQ_THREADS, 0, st>>>(c); break;
      case 3: seq_filter_kernel<NX, 3, TS><<<seq_blocks, SEQ_THREADS, 0, st>>>(c); break;
      default: seq_filter_kernel<NX, 4, TS><<<seq_blocks, SEQ_THREADS, 0, st>>>(c); break;
    }
  } else
    scan_kernel<FOp><<<sh.grid_f, sh.scan_groups_f * G, sh.smem_f, st>>>(c, sh.scan_groups_f, sh.scan_elems_f, sh.window_f);
  if (ev) cudaEventRecord(ev[1], st);
  if (c.setup_separate) launch_setup<NX, T, TS>(c, (unsigned)sh.grid_setup, sh.smem_setup, st);
  launch_loglik(c, st);
  if (ev) cudaEventRecord(ev[2], st);  // otherwise the interval setup runs inside the filter scan
  if (c.split_mode == 2) {  // the smoother aggregate of a range of a split sequence
    Ctx cr = c;
    cr.reduce_only = 1;
    scan_kernel<SOp><<<sh.grid_s, sh.scan_groups_s * G, sh.smem_s, st>>>(cr, sh.scan_groups_s, sh.scan_elems_s,
                                                                        sh.window_s);
    if (ev)
      for (int i = 3; i <= 4; ++i) cudaEventRecord(ev[i], st);
    return cudaGetLastError() == cudaSuccess ? SRTM_OK : SRTM_ERR_CUDA;
  }
  if (c.split_mode == 3 && c.next_mean) split_tail_kernel<NX, T, TR><<<1, SOp::G, 0, st>>>(c);
  const unsigned rblocks = (unsigned)((c.total_fast + sh.recover_threads - 1) / sh.recover_threads);
  const size_t rsmem = recover_smem_bytes<NX>(sh.recover_threads);
  const bool split = c.smoothing && c.recover_split && side;
  // split recovery: the smoother scan is issued first, so that its blocks are
  // placed before the filtered half fills the remaining room
  if (split) cudaEventRecord(side->fork, st);
  if (c.smoothing && c.sequential)
    seq_smoother_kernel<NX, T, TR><<<seq_blocks, SEQ_THREADS, 0, st>>>(c);
  else if (c.smoothing)
    scan_kernel<SOp><<<sh.grid_s, sh.scan_groups_s * G, sh.smem_s, st>>>(c, sh.scan_groups_s, sh.scan_elems_s, sh.window_s);
  if (split) {
    cudaStreamWaitEvent(side->st, side->fork, 0);
    if (ev) cudaEventRecord(ev[6], side->st);
    launch_recover<NX, TR, 1>(c, rblocks, sh.recover_threads, rsmem, side->st);
    if (ev) cudaEventRecord(ev[7], side->st);
    cudaEventRecord(side->join, side->st);
  }
  if (ev) cudaEventRecord(ev[3], st);
  if (split) {
    cudaStreamWaitEvent(st, side->join, 0);
    if (ev) cudaEventRecord(ev[5], st);
    launch_recover<NX, TR, 2>(c, rblocks, sh.recover_threads, rsmem, st);
  } else {
    launch_recover<NX, TR, 0>(c, rblocks, sh.recover_threads, rsmem, st);
  }
  if (ev) cudaEventRecord(ev[4], st);
  return cudaGetLastError() == cudaSuccess ? SRTM_OK : SRTM_ERR_CUDA;
}

// Product in float64 of n filter (op 0, Eq. 27) or smoother (op 1, Eq. 30)
// elements in the paper's order, in[0] (x) in[1] (x) ... (x) in[n-1], by one
// lane group; the symmetric blocks of the result (D and J, or S) are written
// as the mean of the matrix and its transpose.  The exchange step of a
// sequence split over several GPUs: the prefix of the earlier ranges'
// filter aggregates, the suffix of the later ranges' smoother aggregates.
template <int NX>
__global__ void __launch_bounds__(32) split_combine_kernel(int op, const double* in, int n, double* out,
                                                           Counters* ctr) {
  using FOp = FilterOp<NX, double, double>;
  constexpr int G = FOp::G, ESF = FL<NX>::SIZE, ESS = SL<NX>::SIZE, NN = NX * NX;
  constexpr int ES = ESF > ESS ? ESF : ESS;
  __shared__ double acc[ES], nxt[ES], el[ES], sc[FOp::SCR], scs[FOp::SCRS];
  if (threadIdx.x >= G) return;
  const Grp<G> g;
  const int es = op == 0 ? ESF : ESS;
  bool ok = true;
  for (int e = g.lane; e < es; e += G) acc[e] = in[e];
  for (int i = 1; i < n; ++i) {
    g.sync();
    for (int e = g.lane; e < es; e += G) el[e] = in[(long long)i * es + e];
    g.sync();
    if (op == 0) ok &= g_filter_combine<NX, G, double, double>(g, nxt, acc, el, sc, scs, false);
    else g_smoother_combine<NX, G, double>(g, nxt, acc, el, sc, false);
    g.sync();
    for (int e = g.lane; e < es; e += G) acc[e] = nxt[e];
  }
  g.sync();
  for (int e = g.lane; e < es; e += G) {
    double v = acc[e];
    const int blk = op == 0 ? ((e >= FL<NX>::D && e < FL<NX>::D + NN) ? FL<NX>::D
                                                                        : ((e >= FL<NX>::J) ? FL<NX>::J : -1))
                            : ((e >= SL<NX>::S) ? SL<NX>::S : -1);
    if (blk >= 0) {
      const int r = (e - blk) / NX, q = (e - blk) % NX;
      v = 0.5 * (acc[blk + r * NX + q] + acc[blk + q * NX + r]);
    }
    out[e] = v;
  }
  if (!ok && g.lane == 0) raise_err(ctr, DEVERR_SINGULAR);
}

template <int NX>
int launch_split_combine(int op, const double* in, int n, double* out, Counters* ctr, cudaStream_t st) {
  split_combine_kernel<NX><<<1, 32, 0, st>>>(op, in, n, out, ctr);
  return cudaGetLastError() == cudaSuccess ? SRTM_OK : SRTM_ERR_CUDA;
}

template <int NX>
int launch_device_path(const Ctx& c, srtm_precision prec, const Shapes& sh, cudaStream_t st, cudaEvent_t* ev,
                       const SideStream* side) {
  switch (prec) {
    case SRTM_FP64: return launch_t<NX, double, double, double>(c, sh, st, ev, side);
    case SRTM_MIXED: return launch_t<NX, float, double, double>(c, sh, st, ev, side);
    case SRTM_FP32: return launch_t<NX, float, float, float>(c, sh, st, ev, side);
  }
  return SRTM_ERR_ARG;
}

}  // namespace srtm

#define SRTM_INSTANTIATE(NXV)                                                                                \
  template int srtm::launch_device_path<NXV>(const srtm::Ctx&, srtm_precision, const srtm::Shapes&,          \
                                             cudaStream_t, cudaEvent_t*, const srtm::SideStream*);           \
  template int srtm::query_shapes<NXV>(srtm_precision, int, int, int, int, int, int, long long, int, srtm::Shapes*); \
  template int srtm::launch_split_combine<NXV>(int, const double*, int, double*, srtm::Counters*, cudaStream_t);
