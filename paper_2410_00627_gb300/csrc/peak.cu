// peak.cu -- throughput calibration (the paper has no counterpart): the
// float64 and float32 FMA rates of this GPU, measured by a kernel of
// independent FMA chains on every SM (the denominators of the roofline
// fractions the benchmark reports for the FP64-bound fast-rate recovery and
// the float32 scans), and the CPU-GPU link's rate for pinned host memory.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>

#include "srtm_internal.cuh"

namespace srtm {
namespace {

constexpr int PEAK_THREADS = 256;
constexpr int PEAK_CHAINS = 8;   // independent accumulators per thread
constexpr int PEAK_UNROLL = 16;  // FMAs per chain per loop trip

// Every thread runs PEAK_CHAINS independent chains a <- a * b + c for
// `trips` * PEAK_UNROLL steps (|b| < 1, so the values stay finite) and writes
// their sum, so that nothing is optimised away.  FLOPs = 2 * threads * trips *
// PEAK_UNROLL * PEAK_CHAINS.
template <class T>
__global__ void __launch_bounds__(PEAK_THREADS) fma_peak_kernel(T* out, long long trips, T b, T c) {
  const long long tid = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  T a[PEAK_CHAINS];
#pragma unroll
  for (int j = 0; j < PEAK_CHAINS; ++j) a[j] = T(tid & 7) * T(0.125) + T(j);
  for (long long t = 0; t < trips; ++t) {
#pragma unroll
    for (int u = 0; u < PEAK_UNROLL; ++u)
#pragma unroll
      for (int j = 0; j < PEAK_CHAINS; ++j) a[j] = fma(a[j], b, c);
  }
  T s = T(0);
#pragma unroll
  for (int j = 0; j < PEAK_CHAINS; ++j) s += a[j];
  out[tid] = s;
}

template <class T>
int measure(float target_ms, double* gflops, float* ms_out, cudaStream_t st) {
  int dev = 0, sms = 0, per_sm = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SRTM_ERR_CUDA;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fma_peak_kernel<T>, PEAK_THREADS, 0) != cudaSuccess ||
      per_sm < 1)
    return SRTM_ERR_CUDA;
  const long long blocks = (long long)sms * per_sm;  // one full wave: every SM at its occupancy limit
  const long long threads = blocks * PEAK_THREADS;
  T* out = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SRTM_OK;
  if (cudaMallocAsync((void**)&out, sizeof(T) * threads, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
      cudaEventCreate(&e1) != cudaSuccess)
    rc = SRTM_ERR_CUDA;
  const T b = T(0.9999), c = T(1e-3);
  auto run = [&](long long trips, float* ms) -> int {
    cudaEventRecord(e0, st);
    fma_peak_kernel<T><<<(unsigned)blocks, PEAK_THREADS, 0, st>>>(out, trips, b, c);
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess)
      return SRTM_ERR_CUDA;
    return SRTM_OK;
  };
  float ms = 0.f;
  long long trips = 64;
  // grow the launch until it lasts at least a tenth of the target, then size
  // the timed launches to the target
  for (int i = 0; rc == SRTM_OK && i < 24; ++i) {
    rc = run(trips, &ms);
    if (rc || ms >= 0.1f * target_ms) break;
    trips *= 4;
  }
  if (rc == SRTM_OK && ms > 0.f) trips = (long long)((double)trips * target_ms / ms) + 1;
  double best = 0.0;
  float best_ms = 0.f;
  for (int r = 0; rc == SRTM_OK && r < 3; ++r) {  // the fastest of three timed launches
    rc = run(trips, &ms);
    const double fl = 2.0 * (double)threads * (double)trips * PEAK_UNROLL * PEAK_CHAINS;
    const double g = fl / ((double)ms * 1e-3) / 1e9;
    if (rc == SRTM_OK && g > best) { best = g; best_ms = ms; }
  }
  if (out) cudaFreeAsync(out, st);
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  if (rc == SRTM_OK && cudaGetLastError() != cudaSuccess) rc = SRTM_ERR_CUDA;
  *gflops = best;
  if (ms_out) *ms_out = best_ms;
  return rc;
}

// consecutive 16-byte stores of a grid-stride loop (the pattern of the
// library's copy-out kernel)
__global__ void __launch_bounds__(256) link_store_kernel(double2* dst, const double2* src, long long n) {
  const long long stride = (long long)gridDim.x * blockDim.x;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) dst[i] = __ldcs(src + i);
}

}  // namespace
}  // namespace srtm

extern "C" int srtm_measure_link(int kind, double gib, double* gbps, srtm_stream_t stream) {
  if (!gbps || kind < 0 || kind > 3 || !(gib >= 0.0625 && gib <= 64.0)) return SRTM_ERR_ARG;
  const size_t bytes = (size_t)(gib * (double)(1ull << 30)) / 256 * 256;
  cudaStream_t st = (cudaStream_t)stream;
  void *h = nullptr, *hd = nullptr, *d = nullptr;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  int rc = SRTM_OK, dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return SRTM_ERR_CUDA;
  const unsigned flags = kind == 3 ? cudaHostRegisterMapped : cudaHostAllocMapped;
  if (kind == 3) {  // pageable memory made page-locked by registration
    h = malloc(bytes);
    if (!h || cudaHostRegister(h, bytes, flags) != cudaSuccess) rc = SRTM_ERR_CUDA;
  } else if (cudaHostAlloc(&h, bytes, flags) != cudaSuccess) {
    rc = SRTM_ERR_CUDA;
  }
  if (rc == SRTM_OK && (cudaHostGetDevicePointer(&hd, h, 0) != cudaSuccess || cudaMalloc(&d, bytes) != cudaSuccess ||
                        cudaMemsetAsync(d, 0, bytes, st) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
                        cudaEventCreate(&e1) != cudaSuccess))
    rc = SRTM_ERR_CUDA;
  auto once = [&](float* ms) -> int {
    cudaEventRecord(e0, st);
    if (kind == 0) cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, st);
    else if (kind == 2) cudaMemcpyAsync(d, h, bytes, cudaMemcpyHostToDevice, st);
    else srtm::link_store_kernel<<<2 * sms, 256, 0, st>>>((double2*)hd, (const double2*)d, (long long)(bytes / 16));
    cudaEventRecord(e1, st);
    if (cudaEventSynchronize(e1) != cudaSuccess || cudaEventElapsedTime(ms, e0, e1) != cudaSuccess) return SRTM_ERR_CUDA;
    return SRTM_OK;
  };
  double best = 0.0;
  for (int r = 0; rc == SRTM_OK && r < 4; ++r) {  // the first run warms up; the fastest of the others
    float ms = 0.f;
    rc = once(&ms);
    if (rc == SRTM_OK && r > 0 && ms > 0.f) best = std::max(best, (double)bytes / (ms * 1e-3) / 1e9);
  }
  if (e0) cudaEventDestroy(e0);
  if (e1) cudaEventDestroy(e1);
  cudaStreamSynchronize(st);
  if (d) cudaFree(d);
  if (h) {
    if (kind == 3) { cudaHostUnregister(h); free(h); }
    else cudaFreeHost(h);
  }
  if (rc == SRTM_OK && cudaGetLastError() != cudaSuccess) rc = SRTM_ERR_CUDA;
  *gbps = best;
  return rc;
}

extern "C" int srtm_measure_peak(int kind, float target_ms, double* gflops, float* ms, srtm_stream_t stream) {
  if (!gflops || (kind != 0 && kind != 1) || !(target_ms >= 1.f && target_ms <= 5000.f)) return SRTM_ERR_ARG;
  return kind == 0 ? srtm::measure<double>(target_ms, gflops, ms, (cudaStream_t)stream)
                   : srtm::measure<float>(target_ms, gflops, ms, (cudaStream_t)stream);
}
