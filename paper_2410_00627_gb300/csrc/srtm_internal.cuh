// srtm_internal.cuh -- shared definitions of the sm_103a SRTM library:
// the launch context, device-workspace layouts and memory-ordering helpers.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "srtm.h"

namespace srtm {

constexpr int MAXNX = 8;  // compiled state sizes 1..8
constexpr int MY = 4;     // measurement sizes 1..4 (padded to 4 in per-interval records)
// A batch may be processed in up to MAXCHUNK chunks of whole sequences: the
// scans of chunk c+1 run while the fast-rate recovery of chunk c runs.
constexpr int MAXCHUNK = 16;

enum DevErr : unsigned { DEVERR_TIMEOUT = 1u, DEVERR_SINGULAR = 2u, DEVERR_META = 4u, DEVERR_NOT_PSD = 8u };

// Look-back wait bound: polls with exponential __nanosleep back-off capped at
// 2 us, so the bound is a few seconds of wall time.
constexpr long long SPIN_LIMIT = 2000000;

// Device-side control block at offset 0 of the workspace.
struct Counters {
  unsigned long long epoch;   // bumped once per call by the metadata kernel
  unsigned int ticket[2 * MAXCHUNK];  // tile tickets of chunk q: 2q filter scan, 2q+1 smoother scan
  unsigned int err;           // DevErr bits, sticky until srtm_status()
  unsigned int call_ok;       // 1 when this call's metadata passed validation
  long long total_tiles_f, total_tiles_s;
  unsigned long long never_set;  // stays 0: the flag of the bounded-wait self-test
};

// Per-sequence metadata (SoA, written by the metadata kernel).
struct SeqMeta {
  int* ratio;
  int* nslow;
  long long* off_slow;        // [n_seq+1] row offsets of y / slow outputs
  long long* off_fast;        // [n_seq+1] row offsets of fast outputs
  long long* tile_off_f;      // [n_seq+1] filter-scan tile offsets
  long long* tile_off_s;      // [n_seq+1] smoother-scan tile offsets
  int* chunk_seq;             // [n_chunks+1] first sequence of each chunk (batches)
};

// Per-model constant table (float64), offsets in doubles.  L is the largest
// ratio of the call; sequence s uses its own l <= L.
struct ModelLayout {
  long long Apow;  // (L+1) n^2   A^0..A^L
  long long VH;    // L n m       V_i H^T,  V_i = Cov(e_i, sum_j e_j)
  long long Qc;    // L n^2       Qc_i = Cov(e_i) = sum_{r<i} A^r Q A^rT
  long long Ql;    // L n^2       Cov(e_i, e_l) = Qc_i A^{(l-i)T}
  long long Ssc;   // L n^2       scratch: S_q = sum_{j<=q} A^j
  long long Vsc;   // L n^2       scratch: V_i
  long long V2sc;  // L n^2       scratch: second buffer of the V_i scan
  long long Cb;    // m n         C_bar = H sum_{i=1..l} A^i
  long long Rx;    // m m         M Q~ M^T + R
  long long Fc;    // n^2         A^l - K C_bar
  long long Dc;    // n^2         Q_bar - K (G Q~ M^T)^T
  long long Jc;    // n^2         C_bar^T R_x^-1 C_bar
  long long K;     // n m         G Q~ M^T R_x^-1
  long long Cr;    // n m         C_bar^T R_x^-1
  long long m1;    // n           m^f_{1,l}
  long long P1;    // n^2         P^f_{1,l}
  long long Q;     // n^2         copy of Q
  long long Cf;    // float copies of A, Qc_1, Cov(e_1,e_l) (n^2 each), V_1 H^T, K and C_bar^T R_x^-1
                   // (n x m each, ld m, at n x MY strides), then F, D, J of the generic element (n^2 each),
                   // C_bar (m x n, at an MY x n stride), R_x (m x m, ld m, at an MY x MY stride), A^l (n^2)
                   // and V_l H^T (n x m, ld m)
  long long BrT;   // L (3n^2 + n MY)  two-point recovery constants per fast index i: C1_i, C2_i, Sg_i (n^2 each),
                   //                  c3_i (n x m, ld MY)                      [two-point recovery]
  long long BrO;   // L (2n^2 + n MY)  the same for the last interval: C1'_i, Sg'_i, c3'_i
  long long bflag; // 1              1.0: the sequence takes the two-point recovery
  long long AB;    // L n MU      A^j B   (j = 0..L-1), n x nu blocks (ld nu)      [inputs]
  long long SB;    // L n MU      S_j B = sum_{i<=j} A^i B                         [inputs]
  long long stride;
};

__host__ __device__ inline ModelLayout make_model_layout(int n, int m, int L) {
  ModelLayout ml;
  long long o = 0, nn = (long long)n * n;
  ml.Apow = o; o += (L + 1) * nn;
  ml.VH = o;   o += (long long)L * n * m;
  ml.Qc = o;   o += L * nn;
  ml.Ql = o;   o += L * nn;
  ml.Ssc = o;  o += L * nn;
  ml.Vsc = o;  o += L * nn;
  ml.V2sc = o; o += L * nn;
  ml.Cb = o;   o += (long long)m * n;
  ml.Rx = o;   o += (long long)m * m;
  ml.Fc = o;   o += nn;
  ml.Dc = o;   o += nn;
  ml.Jc = o;   o += nn;
  ml.K = o;    o += (long long)n * m;
  ml.Cr = o;   o += (long long)n * m;
  ml.m1 = o;   o += n;
  ml.P1 = o;   o += nn;
  ml.Q = o;    o += nn;
  ml.Cf = o;   o += (7 * nn + 5LL * n * MY + MY * MY + 1) / 2;
  ml.BrT = o;  o += (long long)L * (3 * nn + (long long)n * MY);
  ml.BrO = o;  o += (long long)L * (2 * nn + (long long)n * MY);
  ml.bflag = o; o += 1;
  ml.AB = o;   o += (long long)L * n * SRTM_MAX_NU;
  ml.SB = o;   o += (long long)L * n * SRTM_MAX_NU;
  ml.stride = (o + 31) / 32 * 32;
  return ml;
}

// Per-interval record written by the interval-setup kernel, read by the
// recovery (units of TR).  Sizes use the padded measurement dimension MY.
template <int NX>
struct Rec {
  static constexpr int NN = NX * NX;
  static constexpr int P = 0;                 // P^f_{k-1,l} as LDL^T NN (L below the diagonal, D on it)
  static constexpr int mv = P + NN;           // m^f_{k-1,l}          NX
  static constexpr int X = mv + NX;           // P C_bar^T            NX*MY
  static constexpr int Si = X + NX * MY;      // S_y^-1               MY*MY
  static constexpr int kap = Si + MY * MY;    // S_y^-1 (y - C_bar m) MY
  static constexpr int Pl = kap + MY;         // P A^{lT}             NN
  static constexpr int SUl = Pl + NN;         // S_y^-1 U_l^T         MY*NX
  static constexpr int Z = SUl + MY * NX;     // A^T (P^-_{k+1,1})^-1 NN
  static constexpr int ml = Z + NN;           // m^f_{k,l}            NX
  static constexpr int Pm = ml + NX;          // P^-_{k+1,1}          NN
  // padded to 32 entries (256 B in float64): records start on cache-line
  // boundaries and no cache sector holds parts of two of them
  static constexpr int SIZE = (Pm + NN + 31) / 32 * 32;
};

// Per-interval input terms (with x_{k,i} = A^i x_{k-1,l} + b_{k,i} + noise,
// b_{k,i} = sum_{r<i} A^{i-1-r} B u_{k,r}):  b_{k,l}, b_{k,1} = B u_{k,0},
// B u_{k+1,0} (the input of the smoother's prediction m^-_{k+1,1}), and
// c_k = H sum_i b_{k,i} (the input part of the predicted measurement).
template <int NX>
struct UIn {
  static constexpr int bl = 0, b1 = NX, bn = 2 * NX, c = 3 * NX, SIZE = 3 * NX + MY;
};

// Per-interval terms of the two-point recovery (recovery type), written by
// the smoother scan: E_k (the smoother gain of Eq. 29), the LDL^T factors of
// P^s_{k+1,1} (L1) and of the element's S_k = Cov(x_{k,1} | x_{k+1,1}, y_{1:k})
// (L2; for the last interval of P^s_{k,1}), and the smoothed means
// mu0 = m^s_{k,1}, mu1 = m^s_{k+1,1}; padded to 32 entries.
template <int NX>
struct BRec {
  static constexpr int NN = NX * NX;
  static constexpr int E = 0, L1 = NN, L2 = 2 * NN, mu0 = 3 * NN, mu1 = 3 * NN + NX;
  static constexpr int SIZE = (3 * NN + 2 * NX + 31) / 32 * 32;
};

// Per-interval smoothing terms (Om_k as its LDL^T factors: L below the
// diagonal, D on it; om_k), padded like the record.
template <int NX>
struct SFin {
  static constexpr int Om = 0, om = NX * NX, SIZE = (NX * NX + NX + 31) / 32 * 32;
};

// Filter element (F, d, D, eta, J) and smoother element (E, g, S) layouts.
template <int NX>
struct FL {
  static constexpr int NN = NX * NX;
  static constexpr int F = 0, d = NN, D = NN + NX, e = 2 * NN + NX, J = 2 * NN + 2 * NX;
  static constexpr int SIZE = 3 * NN + 2 * NX;
};
template <int NX>
struct SL {
  static constexpr int NN = NX * NX;
  static constexpr int E = 0, g = NN, S = NN + NX;
  static constexpr int SIZE = 2 * NN + NX;
};

// Everything a kernel needs; passed by value.
struct Ctx {
  int n_seq, nx, ny, max_ratio;
  int smoothing;                      // 1: smoother call, 0: filter only
  int fold_meta;                      // 1: single sequence, metadata written by the constants kernel
  int uniform_ratio, uniform_nslow;   // used when in_ratio/in_nslow are NULL
  long long total_slow, total_fast;   // declared totals (validated on the device)
  const int* in_ratio;
  const int* in_nslow;
  const double *F, *Q, *H, *R, *m0, *P0, *y;
  int nu;                 // known inputs (0: none)
  const double *B, *u;    // B per sequence (nx x nu), u per fast step (rows in sequence order)
  // outputs of the call (smoothed, or filtered for a filter-only call)
  double *fast_mean, *fast_cov, *slow_mean, *slow_cov;
  // filtered outputs requested alongside a smoother call
  double *ffast_mean, *ffast_cov, *fslow_mean, *fslow_cov;
  // workspace
  Counters* ctr;
  SeqMeta meta;
  double* model;
  ModelLayout ml;
  unsigned char* ftile;  long long ftile_stride;  // filter scan tile states
  unsigned char* stile;  long long stile_stride;  // smoother scan tile states
  void* fout;   // [total_slow][NX + NN] filter results m^f_{k,l}, P^f_{k,l}   (solve type)
  void* rec;    // [total_slow][Rec::SIZE] per-interval records              (recovery type)
  void* selem;  // [total_slow][SL::SIZE]  smoother elements                  (scan type)
  void* sfin;   // [total_slow][NN + NX]   per-interval smoothing terms Om_k, om_k (recovery type)
  double* lterm;   // [total_slow] per-interval terms of log p(y_{1:N})
  double* uin;     // [total_slow][UIn::SIZE] per-interval input terms (NULL without inputs)
  double* loglik;  // caller's output: log p(y_{1:N}) per sequence (NULL: not computed)
  // launch shapes
  int tile_f, tile_s;    // elements per scan tile
  int setup_separate;    // 1: the interval setup runs as its own kernel after the filter scan
  int sequential;        // 1: the slow-rate recursions run sequentially (one thread per sequence)
  int recover_split;     // 1: filtered half of the recovery concurrent with the smoother scan
  int n_chunks;          // > 1: a batch processed in chunks of whole sequences, pipelined
  int chunk;             // the chunk a launch works on (0 when n_chunks == 1)
  // one sequence split over several GPUs in contiguous slow-step ranges (the
  // call works on one range): 1 filter aggregate, 2 smoother aggregate,
  // 3 range smoother; 0 otherwise
  int split_mode;
  int split_head_generic;  // the range does not start the sequence: its first filter element is generic
  int split_tail_open;     // the range does not end the sequence: its last interval is not terminal
  int reduce_only;         // this scan launch forms only the range's aggregate (written to agg_out)
  double* agg_out;         // float64 aggregate of the range (filter: FL layout, smoother: SL layout)
  const double *next_mean, *next_cov;  // smoothed x_{k+1,1} after the range's last interval (mode 3)
  void* rscr;            // [RecScr::SIZE][total_fast] filtered moments between the two halves (recovery type)
  // two-point recovery: the fast-rate smoothed moments of an interval from
  // the smoothed joint of its first state and the next interval's first state
  // and its measurement, for the sequences whose bflag is set
  int bridge;            // 1: the call forms the two-point constants and terms
  void* brec;            // [total_slow][BRec::SIZE] (recovery type)
};

// Filtered moments of one fast step kept between the two halves of a split
// recovery: m^f_i, P^f_ii (upper triangle), P^f_il; stored component-major
// (component c of fast step f at c * total_fast + f).
template <int NX>
struct RecScr {
  static constexpr int NT = NX * (NX + 1) / 2;
  static constexpr int mf = 0, Pf = NX, Pfl = NX + NT, SIZE = NX + NT + NX * NX;
};

// The library's second stream of the current GPU and the two events that fork
// work onto it and join it back (split recovery).
struct SideStream {
  cudaStream_t st;
  cudaEvent_t fork, join;
};

// ---------------------------------------------------------------------------
// memory-ordering helpers (look-back protocol)
// ---------------------------------------------------------------------------
__device__ __forceinline__ unsigned long long ld_acquire_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// index s with off[s] <= x < off[s+1]; off has n+1 nondecreasing entries.
__device__ __forceinline__ int find_segment(const long long* off, int n, long long x) {
  int lo = 0, hi = n;  // invariant off[lo] <= x < off[hi]
  while (hi - lo > 1) {
    int mid = (lo + hi) >> 1;
    if (__ldg(off + mid) <= x) lo = mid; else hi = mid;
  }
  return lo;
}

__device__ __forceinline__ void raise_err(Counters* c, unsigned bits) { atomicOr(&c->err, bits); }

// Bounded polling for every device-side wait: at most `limit` polls, with an
// exponential __nanosleep back-off (32 ns doubling up to 1 us) between them.
// A wait that runs out returns with its condition unmet and the caller
// latches DEVERR_TIMEOUT, so no wait can hang a kernel.
struct BoundedPoll {
  long long left;
  unsigned ns;
  __device__ explicit BoundedPoll(long long limit) : left(limit), ns(32) {}
  __device__ bool more() const { return left > 0; }
  __device__ void backoff() {
    --left;
    __nanosleep(ns);
    if (ns < 1024) ns <<= 1;
  }
};

// ---------------------------------------------------------------------------
// host-side launch entry points (defined per nx in inst_nx*.cu)
// ---------------------------------------------------------------------------
struct Shapes {  // resolved launch shapes for one call
  int scan_groups_f, scan_elems_f, scan_groups_s, scan_elems_s;
  int window_f, window_s;  // look-back window (tiles per round)
  int recover_threads;
  int grid_f, grid_s, grid_setup;
  int blocks_per_sm_f, blocks_per_sm_s;  // resident scan blocks per SM
  size_t smem_f, smem_s, smem_setup;
  // per-chunk launches of a pipelined batch (set by the caller of the launch)
  int grid_f_chunk, grid_s_chunk, grid_setup_chunk, grid_recover_chunk;
};

template <int NX>
int launch_device_path(const Ctx& c, srtm_precision prec, const Shapes& sh, cudaStream_t st, cudaEvent_t* ev,
                       const SideStream* side);

// sums the per-interval terms into the caller's log-likelihood output (meta.cu)
int launch_loglik(const Ctx& c, cudaStream_t st);
// bounded wait on a flag that nothing sets (failure-detection self-test, meta.cu)
int launch_wait_probe(Counters* ctr, long long polls, cudaStream_t st);

// float64 product of n filter (op 0) or smoother (op 1) elements (kernels.cuh)
template <int NX>
int launch_split_combine(int op, const double* in, int n, double* out, Counters* ctr, cudaStream_t st);

template <int NX>
int query_shapes(srtm_precision prec, int scan_groups, int scan_elems, int window, int recover_threads,
                 int setup_separate, int sm_count, long long total_slow, int n_seq, Shapes* sh);

}  // namespace srtm
