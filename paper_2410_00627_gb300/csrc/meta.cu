// meta.cu -- per-call metadata: meta_kernel (one block) validates the batch
// metadata, forms the row and tile offsets of every sequence and the chunks
// of a pipelined batch, resets the scan tickets and bumps the call epoch that
// tags the scans' look-back flags.
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
    for (int i = 0; i < 2 * MAXCHUNK; ++i) c.ctr->ticket[i] = 0;
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
  // chunks of a pipelined batch: chunk q starts at the first sequence whose
  // fast rows begin at or after q/n_chunks of the batch's fast steps, so that
  // the chunks hold nearly equal recovery work (empty chunks are allowed)
  if (c.n_chunks > 1) {
    __syncthreads();  // the offsets above are visible to the whole block
    for (int q = tid; q <= c.n_chunks; q += nt) {
      int first;
      if (q == 0) {
        first = 0;
      } else if (q == c.n_chunks) {
        first = c.n_seq;
      } else {
        const long long want = (c.total_fast * q) / c.n_chunks;
        int lo = 0, hi = c.n_seq;  // smallest s with off_fast[s] >= want
        while (lo < hi) {
          const int mid = (lo + hi) >> 1;
          if (c.meta.off_fast[mid] >= want) hi = mid; else lo = mid + 1;
        }
        first = lo;
      }
      c.meta.chunk_seq[q] = first;
    }
  }
}

// Failure-detection self-test: one thread waits, with the bounded polling of
// the scans' look-back, on a control-block flag that nothing sets; after
// `polls` polls it latches DEVERR_TIMEOUT and returns.
__global__ void wait_probe_kernel(Counters* ctr, long long polls) {
  BoundedPoll poll(polls);
  bool seen = false;
  while (poll.more()) {
    if (ld_acquire_u64(&ctr->never_set) != 0ull) { seen = true; break; }
    poll.backoff();
  }
  if (!seen) raise_err(ctr, DEVERR_TIMEOUT);
}

int launch_wait_probe(Counters* ctr, long long polls, cudaStream_t st) {
  wait_probe_kernel<<<1, 1, 0, st>>>(ctr, polls);
  return cudaGetLastError() == cudaSuccess ? SRTM_OK : SRTM_ERR_CUDA;
}

// ev (optional): two events recorded before and after the metadata kernel.
// A single sequence needs no scan over sequences: its metadata is written by
// the constants kernel instead (c.fold_meta), saving this launch.
int launch_meta(const Ctx& c, cudaStream_t st, cudaEvent_t* ev) {
  if (ev) cudaEventRecord(ev[0], st);
  if (!c.fold_meta) meta_kernel<<<1, 1024, 0, st>>>(c);
  if (ev) cudaEventRecord(ev[1], st);
  return cudaGetLastError() == cudaSuccess ? SRTM_OK : SRTM_ERR_CUDA;
}

// log p(y_{1:N}) of each sequence: the sum of its intervals' terms, one block
// per sequence in a fixed order (strided partial sums, then a tree), so that
// repeated calls give identical values.
__global__ void __launch_bounds__(256) loglik_kernel(Ctx c) {
  __shared__ double part[256];
  if (!c.ctr->call_ok) return;
  const int s = blockIdx.x;
  const long long lo = c.meta.off_slow[s], hi = c.meta.off_slow[s + 1];
  double acc = 0.0;
  for (long long k = lo + threadIdx.x; k < hi; k += blockDim.x) acc += c.lterm[k];
  part[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) part[threadIdx.x] += part[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) c.loglik[s] = part[0];
}

int launch_loglik(const Ctx& c, cudaStream_t st) {
  if (!c.loglik) return SRTM_OK;
  loglik_kernel<<<c.n_seq, 256, 0, st>>>(c);
  return cudaGetLastError() == cudaSuccess ? SRTM_OK : SRTM_ERR_CUDA;
}

}  // namespace srtm
