// srtm_api.cu -- the C-ABI entry points declared in include/srtm.h: argument
// validation, the cached per-GPU workspace, launch of the device path, the
// host-buffer entry point and the device error latch.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "srtm_internal.cuh"

namespace srtm {
int launch_meta(const Ctx& c, cudaStream_t st, cudaEvent_t* ev);
}
using namespace srtm;

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

constexpr int NSTAGE = 6;  // metadata, constants, filter scan, interval setup, smoother scan, recovery
// stage-timing events: 0..NSTAGE bound the stages in launch order; with a
// split recovery NSTAGE+1 marks the start of its smoothing half (main stream)
// and NSTAGE+2, NSTAGE+3 bound its filtered half (second stream)
// and NSTAGE+4+2q, NSTAGE+5+2q bound the recovery of chunk q of a chunked batch
constexpr int NEVENT = NSTAGE + 4 + 2 * MAXCHUNK;
struct DevState {
  void* ws = nullptr;
  size_t ws_bytes = 0;
  void* stage = nullptr;
  size_t stage_bytes = 0;
  void* hstage = nullptr;            // pinned host buffer: the host entry's packed small inputs
  size_t hstage_bytes = 0;
  cudaEvent_t hstage_ev = nullptr;   // recorded after the copy out of hstage
  int sms = 0;
  cudaEvent_t ev[NEVENT] = {};  // stage-timing events (created on first use)
  bool ev_split = false;        // the timed call split its recovery
  int ev_chunks = 1;            // chunks of the timed call
  cudaStream_t ev_stream = nullptr;
  bool ev_valid = false;
  // placement of the scan tile-state regions used by the previous call
  size_t last_ftile = 0, last_ftile_bytes = 0, last_stile = 0, last_stile_bytes = 0;
  long long last_fstride = 0, last_sstride = 0;
  int last_launches = 0;  // kernel launches of the last call
  SideStream side = {};   // second stream + fork/join events (split recovery), created on first use
};
constexpr int MAXDEV = 64;
std::mutex g_mu;
DevState g_dev[MAXDEV];
srtm_tuning g_tune[MAXNX + 1][3];  // zero fields = built-in choice
bool g_timing = false;

int group_size(int nx) { return nx == 1 ? 1 : (nx <= 2 ? 4 : (nx <= 4 ? 16 : 32)); }

srtm_tuning effective_tuning(int nx, srtm_precision prec) {
  srtm_tuning t;
  const int G = group_size(nx);
  t.scan_groups = std::max(1, 128 / G);
  t.scan_elems = 4;
  t.recover_threads = 128;
  t.lookback_window = 16;
  t.setup_mode = 1;
  t.recover_split = 1;
  t.batch_chunks = 1;
  t.chunk_recover_bps = 0;
  t.chunk_scan_bps = 0;
  t.recover_form = 2;
  const srtm_tuning& u = g_tune[nx][prec];
  if (u.scan_groups) t.scan_groups = u.scan_groups;
  if (u.scan_elems) t.scan_elems = u.scan_elems;
  if (u.recover_threads) t.recover_threads = u.recover_threads;
  if (u.lookback_window) t.lookback_window = u.lookback_window;
  if (u.setup_mode) t.setup_mode = u.setup_mode;
  if (u.recover_split) t.recover_split = u.recover_split;
  if (u.batch_chunks) t.batch_chunks = u.batch_chunks;
  if (u.chunk_recover_bps) t.chunk_recover_bps = u.chunk_recover_bps;
  if (u.chunk_scan_bps) t.chunk_scan_bps = u.chunk_scan_bps;
  if (u.recover_form) t.recover_form = u.recover_form;
  return t;
}

// Mapped pinned host memory: the address the device uses for it (with unified
// addressing the host address itself), or NULL for any other pointer.
void* mapped_host_ptr(const void* p) {
  if (!p) return nullptr;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

size_t a256(size_t x) { return (x + 255) / 256 * 256; }
size_t a16(size_t x) { return (x + 15) / 16 * 16; }

struct Layout {
  size_t ctr, ratio, nslow, off_slow, off_fast, tile_f, tile_s, chunks, model, ftile, stile, fout, rec, selem, sfin,
      lterm, uin, rscr, brec, total;
  long long ftile_stride, stile_stride;
  ModelLayout ml;
};

// bytes of the split recovery's per-fast-step moments (RecScr)
size_t split_scratch_bytes(int nx, srtm_precision prec, long long total_fast) {
  const size_t sR = prec == SRTM_FP32 ? 4 : 8;
  return sR * (size_t)(nx + nx * (nx + 1) / 2 + nx * nx) * (size_t)total_fast;
}
constexpr size_t SPLIT_SCRATCH_MAX = (size_t)4 << 30;

Layout make_layout(int nx, int ny, int max_ratio, int n_seq, long long total_slow, srtm_precision prec, int tile_f,
                   int tile_s, int nu, size_t rscr_bytes, bool two_point = false) {
  Layout L;
  const size_t sT = prec == SRTM_FP64 ? 8 : 4, sR = prec == SRTM_FP32 ? 4 : 8;
  const long long nn = (long long)nx * nx;
  const long long FE = 3 * nn + 2 * nx, SE = 2 * nn + nx;
  // record and smoothing-term strides, padded to 32 entries (Rec, SFin)
  const long long REC = (4 * nn + 2 * nx + 2LL * nx * MY + MY * MY + MY + 31) / 32 * 32;
  const long long SFN = (nn + nx + 31) / 32 * 32;
  L.ml = make_model_layout(nx, ny, max_ratio);
  // tile state: two flag words, aggregate, inclusive prefix, group aggregate
  L.ftile_stride = 16 + 3 * (long long)a16(FE * sT);
  L.stile_stride = 16 + 3 * (long long)a16(SE * sT);
  const long long tiles_f = total_slow / tile_f + n_seq, tiles_s = total_slow / tile_s + n_seq;
  size_t o = 0;
  auto take = [&](size_t bytes) { const size_t at = a256(o); o = at + bytes; return at; };
  L.ctr = take(sizeof(Counters));
  L.ratio = take(sizeof(int) * n_seq);
  L.nslow = take(sizeof(int) * n_seq);
  L.off_slow = take(sizeof(long long) * (n_seq + 1));
  L.off_fast = take(sizeof(long long) * (n_seq + 1));
  L.tile_f = take(sizeof(long long) * (n_seq + 1));
  L.tile_s = take(sizeof(long long) * (n_seq + 1));
  L.chunks = take(sizeof(int) * (MAXCHUNK + 1));
  L.model = take(sizeof(double) * (size_t)L.ml.stride * n_seq);
  L.ftile = take((size_t)L.ftile_stride * tiles_f);
  L.stile = take((size_t)L.stile_stride * tiles_s);
  L.fout = take(sR * (size_t)(nx + nn) * total_slow);
  L.rec = take(sR * (size_t)REC * total_slow);
  L.selem = take(sT * (size_t)SE * total_slow);
  L.sfin = take(sR * (size_t)SFN * total_slow);
  L.lterm = take(sizeof(double) * (size_t)total_slow);
  L.uin = take(nu > 0 ? sizeof(double) * (size_t)(3 * nx + MY) * total_slow : 0);
  L.rscr = take(rscr_bytes);
  L.brec = take(two_point ? sR * (size_t)((3 * nn + 2 * nx + 31) / 32 * 32) * total_slow : 0);
  L.total = a256(o);
  return L;
}

// Launch shapes depend on (nx, precision, tuning) and the GPU; the scan grids
// also on the tile count.  The occupancy queries and attribute settings are
// made once per key and device and cached (caller holds g_mu).
struct ShapeKey {
  int dev, nx, prec, sg, se, rt, w, sm;
  bool operator==(const ShapeKey& o) const {
    return dev == o.dev && nx == o.nx && prec == o.prec && sg == o.sg && se == o.se && rt == o.rt && w == o.w &&
           sm == o.sm;
  }
};
constexpr int SHAPE_CACHE = 64;
ShapeKey g_shape_key[SHAPE_CACHE];
Shapes g_shape_val[SHAPE_CACHE];
int g_shape_n = 0, g_shape_next = 0;

int query_shapes_for(int nx, srtm_precision prec, const srtm_tuning& t, int sms, long long total_slow, int n_seq,
                     Shapes* sh);

int shapes_for(int nx, srtm_precision prec, const srtm_tuning& t, int sms, long long total_slow, int n_seq,
               Shapes* sh) {
  int dev = 0;
  cudaGetDevice(&dev);
  const ShapeKey key{dev, nx, (int)prec, t.scan_groups, t.scan_elems, t.recover_threads, t.lookback_window,
                     t.setup_mode};
  int hit = -1;
  for (int i = 0; i < g_shape_n; ++i)
    if (g_shape_key[i] == key) { hit = i; break; }
  if (hit < 0) {
    const int rc = query_shapes_for(nx, prec, t, sms, total_slow, n_seq, sh);
    if (rc) return rc;
    hit = g_shape_next;
    g_shape_key[hit] = key;
    g_shape_val[hit] = *sh;
    g_shape_next = (g_shape_next + 1) % SHAPE_CACHE;
    if (g_shape_n < SHAPE_CACHE) ++g_shape_n;
  }
  *sh = g_shape_val[hit];
  const long long tiles = total_slow / ((long long)sh->scan_groups_f * sh->scan_elems_f) + n_seq;
  sh->grid_f = (int)std::max(1LL, std::min((long long)sh->blocks_per_sm_f * sms, tiles));
  sh->grid_s = (int)std::max(1LL, std::min((long long)sh->blocks_per_sm_s * sms, tiles));
  const int sg = nx == 1 ? 1 : (nx == 2 ? 2 : (nx <= 4 ? 4 : 8)), per = 128 / sg;  // lanes per setup interval
  sh->grid_setup = (int)((total_slow + per - 1) / per);
  return SRTM_OK;
}

int query_shapes_for(int nx, srtm_precision prec, const srtm_tuning& t, int sms, long long total_slow, int n_seq,
                     Shapes* sh) {
#define SRTM_Q(N) \
  case N:                                                                                               \
    return query_shapes<N>(prec, t.scan_groups, t.scan_elems, t.lookback_window, t.recover_threads,              \
                           t.setup_mode == 2 ? 1 : 0, sms, total_slow, n_seq, sh);
  switch (nx) {
    SRTM_Q(1) SRTM_Q(2) SRTM_Q(3) SRTM_Q(4) SRTM_Q(5) SRTM_Q(6) SRTM_Q(7) SRTM_Q(8)
  }
#undef SRTM_Q
  return SRTM_ERR_UNSUPPORTED;
}

int launch_for(int nx, const Ctx& c, srtm_precision prec, const Shapes& sh, cudaStream_t st, cudaEvent_t* ev,
               const SideStream* side) {
#define SRTM_L(N) \
  case N: return launch_device_path<N>(c, prec, sh, st, ev, side);
  switch (nx) {
    SRTM_L(1) SRTM_L(2) SRTM_L(3) SRTM_L(4) SRTM_L(5) SRTM_L(6) SRTM_L(7) SRTM_L(8)
  }
#undef SRTM_L
  return SRTM_ERR_UNSUPPORTED;
}

// Launch grids of the per-chunk kernels of a pipelined batch.  The host does
// not know the chunks' sizes (they are formed on the device), so the grids are
// sized for an even split and the kernels loop over whatever their chunk holds.
void chunk_grids(const Ctx& c, const srtm_tuning& t, int sms, Shapes* sh) {
  const int C = c.n_chunks;
  const int bf = t.chunk_scan_bps > 0 ? std::min(t.chunk_scan_bps, sh->blocks_per_sm_f) : sh->blocks_per_sm_f;
  const int bs = t.chunk_scan_bps > 0 ? std::min(t.chunk_scan_bps, sh->blocks_per_sm_s) : sh->blocks_per_sm_s;
  const long long tiles = c.total_slow / ((long long)sh->scan_groups_f * sh->scan_elems_f) / C + c.n_seq / C + 1;
  sh->grid_f_chunk = (int)std::max(1LL, std::min((long long)bf * sms, tiles));
  sh->grid_s_chunk = (int)std::max(1LL, std::min((long long)bs * sms, tiles));
  const int sg = c.nx == 1 ? 1 : (c.nx == 2 ? 2 : (c.nx <= 4 ? 4 : 8)), per = 128 / sg;
  sh->grid_setup_chunk = (int)std::max(1LL, (c.total_slow / C + per - 1) / per);
  const long long even = (c.total_fast / C + sh->recover_threads - 1) / sh->recover_threads;
  sh->grid_recover_chunk =
      (int)std::max(1LL, t.chunk_recover_bps > 0 ? std::min((long long)t.chunk_recover_bps * sms, even) : even);
}

// Runs the device path for a fully validated context (sizes in `c` set).
// host_outputs: some output is pinned host memory written over the CPU-GPU
// link; the recovery then stays one kernel, so that those slower stores
// overlap all of its arithmetic instead of only the smoothing half.
int run(Ctx c, srtm_precision prec, cudaStream_t st, bool host_outputs = false) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV)
    return fail(SRTM_ERR_CUDA, "no usable CUDA device");
  std::lock_guard<std::mutex> lk(g_mu);
  DevState& d = g_dev[dev];
  if (!d.sms && cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return fail(SRTM_ERR_CUDA, "cudaDeviceGetAttribute failed");
  srtm_tuning t = effective_tuning(c.nx, prec);
  if (c.sequential) t.setup_mode = 2;  // no filter scan to carry the setup
  Shapes sh;
  int rc = shapes_for(c.nx, prec, t, d.sms, c.total_slow, c.n_seq, &sh);
  if (rc) return fail(rc, "launch shape query failed (%d)", rc);
  const int tile_f = sh.scan_groups_f * sh.scan_elems_f, tile_s = sh.scan_groups_s * sh.scan_elems_s;
  // split recovery: smoother calls of the scan path whose moments fit the bound
  const size_t rscr_bytes = split_scratch_bytes(c.nx, prec, c.total_fast);
  c.recover_split = (t.recover_split == 2 && c.smoothing && !c.sequential && !host_outputs &&
                     rscr_bytes <= SPLIT_SCRATCH_MAX && (c.split_mode == 0 || c.split_mode == 3))
                        ? 1
                        : 0;
  // two-point recovery: smoothed outputs only, no known inputs, not a range
  // of a split sequence; the whole recovery then follows the smoother scan
  c.bridge = (t.recover_form == 2 && c.smoothing && !c.sequential && c.split_mode == 0 && c.nu == 0 &&
              !c.ffast_mean && !c.ffast_cov && !c.fslow_mean && !c.fslow_cov)
                 ? 1
                 : 0;
  if (c.bridge) c.recover_split = 0;
  // a batch in chunks: the scans of one chunk beside the recovery of the one before
  c.n_chunks = 1;
  c.chunk = 0;
  if (!c.fold_meta && !c.sequential && t.batch_chunks > 1) {
    c.n_chunks = std::min(std::min(t.batch_chunks, MAXCHUNK), c.n_seq);
    if (c.n_chunks > 1) c.recover_split = 0;
  }
  if ((c.recover_split || c.n_chunks > 1) && !d.side.st) {
    int lo = 0, hi = 0;
    cudaDeviceGetStreamPriorityRange(&lo, &hi);  // the filtered half at the lowest priority
    if (cudaStreamCreateWithPriority(&d.side.st, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&d.side.fork, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&d.side.join, cudaEventDisableTiming) != cudaSuccess)
      return fail(SRTM_ERR_CUDA, "second stream creation failed");
  }
  const Layout L = make_layout(c.nx, c.ny, c.max_ratio, c.n_seq, c.total_slow, prec, tile_f, tile_s, c.nu,
                               c.recover_split ? rscr_bytes : 0, c.bridge != 0);
  if (d.ws_bytes < L.total) {
    if (d.ws) {
      cudaDeviceSynchronize();
      cudaFree(d.ws);
      d.ws = nullptr;
      d.ws_bytes = 0;
    }
    if (cudaMalloc(&d.ws, L.total) != cudaSuccess) {
      cudaGetLastError();
      return fail(SRTM_ERR_CUDA, "workspace cudaMalloc of %zu bytes failed", L.total);
    }
    if (cudaMemset(d.ws, 0, L.total) != cudaSuccess) return fail(SRTM_ERR_CUDA, "workspace memset failed");
    d.ws_bytes = L.total;
    d.last_ftile = d.last_ftile_bytes = d.last_stile = d.last_stile_bytes = 0;
    d.last_fstride = d.last_sstride = 0;
  }
  unsigned char* w = (unsigned char*)d.ws;
  // The look-back flags carry the call epoch, so flags left by earlier calls
  // never match.  When the tile-state regions move or change stride, other
  // data may now sit where flags are read: clear the regions first.
  const size_t fbytes = L.stile - L.ftile, sbytes = L.fout - L.stile;
  if (L.ftile != d.last_ftile || fbytes != d.last_ftile_bytes || L.stile != d.last_stile ||
      sbytes != d.last_stile_bytes || L.ftile_stride != d.last_fstride || L.stile_stride != d.last_sstride) {
    if (cudaMemsetAsync(w + L.ftile, 0, fbytes + sbytes, st) != cudaSuccess)
      return fail(SRTM_ERR_CUDA, "tile-state clear failed");
    d.last_ftile = L.ftile; d.last_ftile_bytes = fbytes; d.last_stile = L.stile; d.last_stile_bytes = sbytes;
    d.last_fstride = L.ftile_stride; d.last_sstride = L.stile_stride;
  }
  c.ctr = (Counters*)(w + L.ctr);
  c.meta.ratio = (int*)(w + L.ratio);
  c.meta.nslow = (int*)(w + L.nslow);
  c.meta.off_slow = (long long*)(w + L.off_slow);
  c.meta.off_fast = (long long*)(w + L.off_fast);
  c.meta.tile_off_f = (long long*)(w + L.tile_f);
  c.meta.tile_off_s = (long long*)(w + L.tile_s);
  c.meta.chunk_seq = (int*)(w + L.chunks);
  c.model = (double*)(w + L.model);
  c.ml = L.ml;
  c.ftile = w + L.ftile;
  c.ftile_stride = L.ftile_stride;
  c.stile = w + L.stile;
  c.stile_stride = L.stile_stride;
  c.fout = w + L.fout;
  c.rec = w + L.rec;
  c.selem = w + L.selem;
  c.sfin = w + L.sfin;
  c.lterm = (double*)(w + L.lterm);
  c.uin = c.nu > 0 ? (double*)(w + L.uin) : nullptr;
  c.rscr = c.recover_split ? (void*)(w + L.rscr) : nullptr;
  c.brec = c.bridge ? (void*)(w + L.brec) : nullptr;
  c.tile_f = tile_f;
  c.tile_s = tile_s;
  c.setup_separate = t.setup_mode == 2 ? 1 : 0;
  if (c.n_chunks > 1) chunk_grids(c, t, d.sms, &sh);
  const int per_chunk = 2 + (c.smoothing ? 1 : 0) + c.setup_separate;  // scans, setup, recovery
  d.last_launches = (c.fold_meta ? 0 : 1) + 1 + per_chunk * c.n_chunks + (c.loglik ? 1 : 0) + (c.nu > 0 ? 1 : 0) +
                    c.recover_split;
  if (c.split_mode == 1) d.last_launches = 2;                                    // constants, reducing filter scan
  if (c.split_mode == 2) d.last_launches -= 1;                                   // no recovery
  if (c.split_mode == 3 && c.next_mean) d.last_launches += 1;                    // the range's tail
  cudaEvent_t* ev = nullptr;
  if (g_timing) {
    if (!d.ev[0])
      for (int i = 0; i < NEVENT; ++i) cudaEventCreate(&d.ev[i]);
    ev = d.ev;
    d.ev_split = c.recover_split != 0;
    d.ev_chunks = c.n_chunks;
    d.ev_stream = st;
    d.ev_valid = true;
  }
  rc = launch_meta(c, st, ev);
  if (rc) return fail(rc, "launch of the metadata kernel failed: %s", cudaGetErrorString(cudaGetLastError()));
  rc = launch_for(c.nx, c, prec, sh, st, ev ? ev + 2 : nullptr, (c.recover_split || c.n_chunks > 1) ? &d.side : nullptr);
  if (rc) return fail(rc, "launch of the constants/scan/recovery kernels failed (scan smem %zu/%zu bytes)", sh.smem_f,
                      sh.smem_s);
  return SRTM_OK;
}

int check_dims(int nx, int ny) {
  if (nx < 1 || nx > MAXNX) return fail(SRTM_ERR_UNSUPPORTED, "nx=%d outside 1..%d", nx, MAXNX);
  if (ny < 1 || ny > MY) return fail(SRTM_ERR_UNSUPPORTED, "ny=%d outside 1..%d", ny, MY);
  return SRTM_OK;
}

int check_outputs(const srtm_output* o, const char* what) {
  if (!o) return SRTM_OK;
  const double* ps[5] = {o->fast_mean, o->fast_cov, o->slow_mean, o->slow_cov, o->loglik};
  const char* nm[5] = {"fast_mean", "fast_cov", "slow_mean", "slow_cov", "loglik"};
  for (int i = 0; i < 5; ++i)
    if (ps[i] && !is_device_ptr(ps[i]) && mapped_host_ptr(ps[i]) != ps[i])
      return fail(SRTM_ERR_ARG, "%s.%s is neither device memory nor mapped pinned host memory", what, nm[i]);
  return SRTM_OK;
}

int check_inputs(const double* F, const double* Q, const double* H, const double* R, const double* m0,
                 const double* P0, const double* y) {
  const double* ps[7] = {F, Q, H, R, m0, P0, y};
  const char* nm[7] = {"F", "Q", "H", "R", "m0", "P0", "y"};
  for (int i = 0; i < 7; ++i) {
    if (!ps[i]) return fail(SRTM_ERR_ARG, "%s is NULL", nm[i]);
    if (!is_device_ptr(ps[i]) && mapped_host_ptr(ps[i]) != ps[i])
      return fail(SRTM_ERR_ARG, "%s is not a device pointer (nor mapped pinned host memory)", nm[i]);
  }
  return SRTM_OK;
}

// Known inputs: nu in 0..SRTM_MAX_NU; with nu > 0, B and u are device arrays.
int check_controls(int nu, const double* B, const double* u) {
  if (nu < 0 || nu > SRTM_MAX_NU) return fail(SRTM_ERR_UNSUPPORTED, "nu=%d outside 0..%d", nu, SRTM_MAX_NU);
  if (nu == 0) return SRTM_OK;
  if (!B || !u) return fail(SRTM_ERR_ARG, "nu=%d needs B and u", nu);
  for (const double* q : {B, u})
    if (!is_device_ptr(q) && mapped_host_ptr(q) != q)
      return fail(SRTM_ERR_ARG, "B and u must be device pointers (or mapped pinned host memory)");
  return SRTM_OK;
}

// true when some fast or slow output is (mapped pinned) host memory
bool any_host_output(const srtm_output* out, const srtm_output* extra) {
  for (const srtm_output* o : {out, extra})
    if (o)
      for (const double* q : {o->fast_mean, o->fast_cov, o->slow_mean, o->slow_cov})
        if (q && !is_device_ptr(q)) return true;
  return false;
}

void set_outputs(Ctx& c, const srtm_output* main, const srtm_output* extra) {
  c.fast_mean = main ? main->fast_mean : nullptr;
  c.fast_cov = main ? main->fast_cov : nullptr;
  c.slow_mean = main ? main->slow_mean : nullptr;
  c.slow_cov = main ? main->slow_cov : nullptr;
  c.ffast_mean = extra ? extra->fast_mean : nullptr;
  c.ffast_cov = extra ? extra->fast_cov : nullptr;
  c.fslow_mean = extra ? extra->slow_mean : nullptr;
  c.fslow_cov = extra ? extra->slow_cov : nullptr;
  c.loglik = (main && main->loglik) ? main->loglik : (extra ? extra->loglik : nullptr);
}

int single(const srtm_problem* p, srtm_precision prec, const srtm_output* out, const srtm_output* extra,
           int smoothing, srtm_stream_t stream, int sequential = 0) {
  if (!p) return fail(SRTM_ERR_ARG, "problem is NULL");
  if (prec < SRTM_FP64 || prec > SRTM_FP32) return fail(SRTM_ERR_ARG, "unknown precision %d", (int)prec);
  int rc = check_dims(p->nx, p->ny);
  if (rc) return rc;
  if (p->ratio < 1) return fail(SRTM_ERR_ARG, "ratio=%d < 1", p->ratio);
  if (p->n_slow < 1) return fail(SRTM_ERR_ARG, "n_slow=%d < 1", p->n_slow);
  if ((rc = check_inputs(p->F, p->Q, p->H, p->R, p->m0, p->P0, p->y))) return rc;
  if ((rc = check_controls(p->nu, p->B, p->u))) return rc;
  if ((rc = check_outputs(out, "output")) || (rc = check_outputs(extra, "filtered output"))) return rc;
  Ctx c;
  memset(&c, 0, sizeof c);
  c.nu = p->nu;
  c.B = p->nu ? p->B : nullptr;
  c.u = p->nu ? p->u : nullptr;
  c.n_seq = 1;
  c.fold_meta = 1;
  c.nx = p->nx;
  c.ny = p->ny;
  c.max_ratio = p->ratio;
  c.smoothing = smoothing;
  c.sequential = sequential;
  c.uniform_ratio = p->ratio;
  c.uniform_nslow = p->n_slow;
  c.total_slow = p->n_slow;
  c.total_fast = (long long)p->n_slow * p->ratio;
  c.F = p->F; c.Q = p->Q; c.H = p->H; c.R = p->R; c.m0 = p->m0; c.P0 = p->P0; c.y = p->y;
  set_outputs(c, out, extra);
  return run(c, prec, (cudaStream_t)stream, any_host_output(out, extra));
}

int batch(const srtm_batch* b, srtm_precision prec, const srtm_output* out, const srtm_output* extra, int smoothing,
          srtm_stream_t stream, int sequential = 0) {
  if (!b) return fail(SRTM_ERR_ARG, "batch is NULL");
  if (prec < SRTM_FP64 || prec > SRTM_FP32) return fail(SRTM_ERR_ARG, "unknown precision %d", (int)prec);
  int rc = check_dims(b->nx, b->ny);
  if (rc) return rc;
  if (b->n_seq < 1) return fail(SRTM_ERR_ARG, "n_seq=%d < 1", b->n_seq);
  if (b->max_ratio < 1) return fail(SRTM_ERR_ARG, "max_ratio=%d < 1", b->max_ratio);
  if (b->total_slow < b->n_seq || b->total_fast < b->total_slow)
    return fail(SRTM_ERR_ARG, "total_slow=%lld / total_fast=%lld inconsistent with n_seq=%d", b->total_slow,
                b->total_fast, b->n_seq);
  if (!is_device_ptr(b->ratio) || !is_device_ptr(b->n_slow))
    return fail(SRTM_ERR_ARG, "ratio and n_slow must be device int arrays");
  if ((rc = check_inputs(b->F, b->Q, b->H, b->R, b->m0, b->P0, b->y))) return rc;
  if ((rc = check_controls(b->nu, b->B, b->u))) return rc;
  if ((rc = check_outputs(out, "output")) || (rc = check_outputs(extra, "filtered output"))) return rc;
  Ctx c;
  memset(&c, 0, sizeof c);
  c.nu = b->nu;
  c.B = b->nu ? b->B : nullptr;
  c.u = b->nu ? b->u : nullptr;
  c.n_seq = b->n_seq;
  c.nx = b->nx;
  c.ny = b->ny;
  c.max_ratio = b->max_ratio;
  c.smoothing = smoothing;
  c.total_slow = b->total_slow;
  c.total_fast = b->total_fast;
  c.sequential = sequential;
  c.in_ratio = b->ratio;
  c.in_nslow = b->n_slow;
  c.F = b->F; c.Q = b->Q; c.H = b->H; c.R = b->R; c.m0 = b->m0; c.P0 = b->P0; c.y = b->y;
  set_outputs(c, out, extra);
  return run(c, prec, (cudaStream_t)stream, any_host_output(out, extra));
}

}  // namespace

extern "C" {

int srtm_filter(const srtm_problem* p, srtm_precision prec, const srtm_output* filt, srtm_stream_t stream) {
  return single(p, prec, filt, nullptr, 0, stream);
}

int srtm_smoother(const srtm_problem* p, srtm_precision prec, const srtm_output* smooth, const srtm_output* filt,
                  srtm_stream_t stream) {
  return single(p, prec, smooth, filt, 1, stream);
}

int srtm_filter_batch(const srtm_batch* b, srtm_precision prec, const srtm_output* filt, srtm_stream_t stream) {
  return batch(b, prec, filt, nullptr, 0, stream);
}

int srtm_smoother_batch(const srtm_batch* b, srtm_precision prec, const srtm_output* smooth,
                        const srtm_output* filt, srtm_stream_t stream) {
  return batch(b, prec, smooth, filt, 1, stream);
}

int srtm_filter_sequential(const srtm_problem* p, srtm_precision prec, const srtm_output* filt,
                           srtm_stream_t stream) {
  return single(p, prec, filt, nullptr, 0, stream, 1);
}

int srtm_smoother_sequential(const srtm_problem* p, srtm_precision prec, const srtm_output* smooth,
                             const srtm_output* filt, srtm_stream_t stream) {
  return single(p, prec, smooth, filt, 1, stream, 1);
}

int srtm_filter_batch_sequential(const srtm_batch* b, srtm_precision prec, const srtm_output* filt,
                                 srtm_stream_t stream) {
  return batch(b, prec, filt, nullptr, 0, stream, 1);
}

int srtm_smoother_batch_sequential(const srtm_batch* b, srtm_precision prec, const srtm_output* smooth,
                                   const srtm_output* filt, srtm_stream_t stream) {
  return batch(b, prec, smooth, filt, 1, stream, 1);
}

}  // extern "C"

namespace {

// One range of a sequence split over several GPUs (contiguous slow steps),
// validated as a single-sequence call; known inputs are not supported here.
int split_range(const srtm_problem* p, srtm_precision prec, int mode, int head_generic, int tail_open, double* agg,
                const double* next_mean, const double* next_cov, const srtm_output* out, const srtm_output* extra,
                srtm_stream_t stream) {
  if (!p) return fail(SRTM_ERR_ARG, "problem is NULL");
  if (prec < SRTM_FP64 || prec > SRTM_FP32) return fail(SRTM_ERR_ARG, "unknown precision %d", (int)prec);
  int rc = check_dims(p->nx, p->ny);
  if (rc) return rc;
  if (p->ratio < 1) return fail(SRTM_ERR_ARG, "ratio=%d < 1", p->ratio);
  if (p->n_slow < 1) return fail(SRTM_ERR_ARG, "n_slow=%d < 1", p->n_slow);
  if (p->nu != 0) return fail(SRTM_ERR_UNSUPPORTED, "a split sequence takes no known inputs (nu=%d)", p->nu);
  if ((rc = check_inputs(p->F, p->Q, p->H, p->R, p->m0, p->P0, p->y))) return rc;
  if (mode != 3 && !is_device_ptr(agg)) return fail(SRTM_ERR_ARG, "agg must be device memory");
  if (mode == 3) {
    if ((next_mean == nullptr) != (next_cov == nullptr))
      return fail(SRTM_ERR_ARG, "next_mean and next_cov must both be given or both be NULL");
    if (next_mean && (!is_device_ptr(next_mean) || !is_device_ptr(next_cov)))
      return fail(SRTM_ERR_ARG, "next_mean and next_cov must be device memory");
    if ((rc = check_outputs(out, "output")) || (rc = check_outputs(extra, "filtered output"))) return rc;
  }
  Ctx c;
  memset(&c, 0, sizeof c);
  c.n_seq = 1;
  c.fold_meta = 1;
  c.nx = p->nx;
  c.ny = p->ny;
  c.max_ratio = p->ratio;
  c.smoothing = mode == 1 ? 0 : 1;
  c.uniform_ratio = p->ratio;
  c.uniform_nslow = p->n_slow;
  c.total_slow = p->n_slow;
  c.total_fast = (long long)p->n_slow * p->ratio;
  c.F = p->F; c.Q = p->Q; c.H = p->H; c.R = p->R; c.m0 = p->m0; c.P0 = p->P0; c.y = p->y;
  c.split_mode = mode;
  c.split_head_generic = head_generic;
  c.split_tail_open = tail_open;
  c.agg_out = agg;
  c.next_mean = next_mean;
  c.next_cov = next_cov;
  if (mode == 3) set_outputs(c, out, extra);
  return run(c, prec, (cudaStream_t)stream, mode == 3 && any_host_output(out, extra));
}

}  // namespace

extern "C" {

int srtm_split_filter_aggregate(const srtm_problem* p, int starts_sequence, srtm_precision prec, double* agg,
                                srtm_stream_t stream) {
  return split_range(p, prec, 1, starts_sequence ? 0 : 1, 0, agg, nullptr, nullptr, nullptr, nullptr, stream);
}

int srtm_split_smoother_aggregate(const srtm_problem* p, int ends_sequence, srtm_precision prec, double* agg,
                                  srtm_stream_t stream) {
  return split_range(p, prec, 2, 0, ends_sequence ? 0 : 1, agg, nullptr, nullptr, nullptr, nullptr, stream);
}

int srtm_split_smoother(const srtm_problem* p, const double* next_mean, const double* next_cov, srtm_precision prec,
                        const srtm_output* smooth, const srtm_output* filt, srtm_stream_t stream) {
  return split_range(p, prec, 3, 0, next_mean ? 1 : 0, nullptr, next_mean, next_cov, smooth, filt, stream);
}

int srtm_split_combine(int op, int nx, const double* elems, int n, double* out, srtm_stream_t stream) {
  if (op != 0 && op != 1) return fail(SRTM_ERR_ARG, "op=%d is neither 0 (filter) nor 1 (smoother)", op);
  if (nx < 1 || nx > MAXNX) return fail(SRTM_ERR_UNSUPPORTED, "nx=%d outside 1..%d", nx, MAXNX);
  if (n < 1) return fail(SRTM_ERR_ARG, "n=%d < 1", n);
  if (!is_device_ptr(elems) || !is_device_ptr(out)) return fail(SRTM_ERR_ARG, "elems and out must be device memory");
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return fail(SRTM_ERR_CUDA, "no device");
  std::lock_guard<std::mutex> lk(g_mu);
  DevState& d = g_dev[dev];
  if (!d.ws) {  // the error latch lives in the control block at the start of the workspace
    const size_t bytes = 4096;
    if (cudaMalloc(&d.ws, bytes) != cudaSuccess) {
      cudaGetLastError();
      d.ws = nullptr;
      return fail(SRTM_ERR_CUDA, "workspace cudaMalloc failed");
    }
    if (cudaMemset(d.ws, 0, bytes) != cudaSuccess) return fail(SRTM_ERR_CUDA, "workspace memset failed");
    d.ws_bytes = bytes;
  }
  d.last_launches = 1;
  Counters* ctr = (Counters*)d.ws;
  int rc = SRTM_ERR_UNSUPPORTED;
  cudaStream_t st = (cudaStream_t)stream;
  switch (nx) {
    case 1: rc = launch_split_combine<1>(op, elems, n, out, ctr, st); break;
    case 2: rc = launch_split_combine<2>(op, elems, n, out, ctr, st); break;
    case 3: rc = launch_split_combine<3>(op, elems, n, out, ctr, st); break;
    case 4: rc = launch_split_combine<4>(op, elems, n, out, ctr, st); break;
    case 5: rc = launch_split_combine<5>(op, elems, n, out, ctr, st); break;
    case 6: rc = launch_split_combine<6>(op, elems, n, out, ctr, st); break;
    case 7: rc = launch_split_combine<7>(op, elems, n, out, ctr, st); break;
    case 8: rc = launch_split_combine<8>(op, elems, n, out, ctr, st); break;
  }
  if (rc) return fail(rc, "launch of the combine kernel failed");
  return SRTM_OK;
}

int srtm_selftest_wait(long long polls, srtm_stream_t stream) {
  if (polls < 1 || polls > SPIN_LIMIT) return fail(SRTM_ERR_ARG, "polls=%lld outside 1..%lld", polls, SPIN_LIMIT);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return fail(SRTM_ERR_CUDA, "no device");
  std::lock_guard<std::mutex> lk(g_mu);
  DevState& d = g_dev[dev];
  if (!d.ws) {  // the control block lives at the start of the workspace
    const size_t bytes = 4096;
    if (cudaMalloc(&d.ws, bytes) != cudaSuccess) {
      cudaGetLastError();
      d.ws = nullptr;
      return fail(SRTM_ERR_CUDA, "workspace cudaMalloc failed");
    }
    if (cudaMemset(d.ws, 0, bytes) != cudaSuccess) return fail(SRTM_ERR_CUDA, "workspace memset failed");
    d.ws_bytes = bytes;
  }
  d.last_launches = 1;
  if (launch_wait_probe((Counters*)d.ws, polls, (cudaStream_t)stream))
    return fail(SRTM_ERR_CUDA, "launch of the wait probe failed");
  return SRTM_OK;
}

int srtm_status(srtm_stream_t stream) {
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
    return fail(SRTM_ERR_CUDA, "stream synchronize failed: %s", cudaGetErrorString(cudaGetLastError()));
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return fail(SRTM_ERR_CUDA, "no device");
  std::lock_guard<std::mutex> lk(g_mu);
  DevState& d = g_dev[dev];
  if (!d.ws) return SRTM_OK;
  unsigned err = 0;
  unsigned* perr = (unsigned*)((unsigned char*)d.ws + offsetof(Counters, err));
  if (cudaMemcpy(&err, perr, sizeof err, cudaMemcpyDeviceToHost) != cudaSuccess)
    return fail(SRTM_ERR_CUDA, "reading the device error latch failed");
  if (!err) return SRTM_OK;
  cudaMemset(perr, 0, sizeof err);
  if (err & DEVERR_META) return fail(SRTM_ERR_META, "batch metadata disagrees with the declared sizes");
  if (err & DEVERR_TIMEOUT) return fail(SRTM_ERR_TIMEOUT, "a scan look-back wait exceeded its bound");
  if (err & DEVERR_NOT_PSD) return fail(SRTM_ERR_NOT_PSD, "Q, R or P0 is not a covariance matrix");
  return fail(SRTM_ERR_SINGULAR, "a solve met a zero, negative or non-finite pivot");
}

int srtm_smoother_host(const srtm_problem* hp, srtm_precision prec, const srtm_output* hout, srtm_stream_t stream) {
  if (!hp || !hout) return fail(SRTM_ERR_ARG, "problem and output must not be NULL");
  int rc = check_dims(hp->nx, hp->ny);
  if (rc) return rc;
  if (hp->ratio < 1 || hp->n_slow < 1) return fail(SRTM_ERR_ARG, "ratio and n_slow must be >= 1");
  if (hp->nu < 0 || hp->nu > SRTM_MAX_NU) return fail(SRTM_ERR_UNSUPPORTED, "nu=%d outside 0..%d", hp->nu, SRTM_MAX_NU);
  const int n_in = hp->nu > 0 ? 9 : 7;
  const double* in[9] = {hp->F, hp->Q, hp->H, hp->R, hp->m0, hp->P0, hp->y, hp->B, hp->u};
  for (int i = 0; i < n_in; ++i)
    if (!in[i]) return fail(SRTM_ERR_ARG, "input %d is NULL", i);
  const long long nx = hp->nx, ny = hp->ny, N = hp->n_slow, l = hp->ratio, nu = hp->nu;
  const size_t in_cnt[9] = {(size_t)(nx * nx), (size_t)(nx * nx), (size_t)(ny * nx), (size_t)(ny * ny),
                            (size_t)nx,        (size_t)(nx * nx), (size_t)(N * ny),  (size_t)(nx * nu),
                            (size_t)(N * l * nu)};
  const size_t out_cnt[5] = {(size_t)(N * l * nx), (size_t)(N * l * nx * nx), (size_t)(N * nx), (size_t)(N * nx * nx),
                             1};
  double* hout_p[5] = {hout->fast_mean, hout->fast_cov, hout->slow_mean, hout->slow_cov, hout->loglik};
  // outputs in mapped pinned host memory are written by the kernels directly
  // (over the CPU-GPU link); the others are staged and copied back
  double* direct[5];
  for (int i = 0; i < 5; ++i) {
    direct[i] = (double*)mapped_host_ptr(hout_p[i]);
    if (direct[i] != hout_p[i]) direct[i] = nullptr;  // only where the device uses the host address
  }
  // the model arrays (F, Q, H, R, m0, P0, B) are packed on the host into one
  // pinned buffer and copied in one transfer; the per-step arrays y and u are
  // read by the kernels directly when they are mapped pinned host memory
  const bool small[9] = {true, true, true, true, true, true, false, true, false};
  const double* bulk_direct[9] = {};
  size_t off[14], o = 0;
  for (int i = 0; i < n_in; ++i)
    if (small[i]) { off[i] = o; o += a256(in_cnt[i] * sizeof(double)); }
  const size_t small_bytes = o;
  for (int i = 0; i < n_in; ++i) {
    if (small[i]) continue;
    if (mapped_host_ptr(in[i]) == (const void*)in[i]) {
      bulk_direct[i] = in[i];
    } else {
      off[i] = o;
      o += a256(in_cnt[i] * sizeof(double));
    }
  }
  for (int i = 0; i < 5; ++i) {
    off[9 + i] = o;
    o += (hout_p[i] && !direct[i]) ? a256(out_cnt[i] * sizeof(double)) : 0;
  }
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return fail(SRTM_ERR_CUDA, "no device");
  unsigned char* stg = nullptr;
  unsigned char* hst = nullptr;
  cudaEvent_t hev = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    DevState& d = g_dev[dev];
    if (!d.hstage_ev && cudaEventCreateWithFlags(&d.hstage_ev, cudaEventDisableTiming) != cudaSuccess)
      return fail(SRTM_ERR_CUDA, "event creation failed");
    if (d.hstage_bytes < small_bytes) {
      if (d.hstage) { cudaEventSynchronize(d.hstage_ev); cudaFreeHost(d.hstage); d.hstage = nullptr; d.hstage_bytes = 0; }
      if (cudaHostAlloc(&d.hstage, small_bytes, cudaHostAllocDefault) != cudaSuccess) {
        cudaGetLastError();
        d.hstage = nullptr;
        return fail(SRTM_ERR_CUDA, "pinned staging allocation of %zu bytes failed", small_bytes);
      }
      d.hstage_bytes = small_bytes;
    }
    hst = (unsigned char*)d.hstage;
    hev = d.hstage_ev;
    if (d.stage_bytes < o) {
      if (d.stage) { cudaDeviceSynchronize(); cudaFree(d.stage); d.stage = nullptr; d.stage_bytes = 0; }
      if (cudaMalloc(&d.stage, o) != cudaSuccess) {
        cudaGetLastError();
        return fail(SRTM_ERR_CUDA, "staging cudaMalloc of %zu bytes failed", o);
      }
      d.stage_bytes = o;
    }
    stg = (unsigned char*)d.stage;
  }
  cudaStream_t st = (cudaStream_t)stream;
  // the previous call's copy out of the pinned buffer must be done before it is rewritten
  if (cudaEventSynchronize(hev) != cudaSuccess) return fail(SRTM_ERR_CUDA, "staging event wait failed");
  for (int i = 0; i < n_in; ++i)
    if (small[i]) memcpy(hst + off[i], in[i], in_cnt[i] * sizeof(double));
  if (cudaMemcpyAsync(stg, hst, small_bytes, cudaMemcpyHostToDevice, st) != cudaSuccess ||
      cudaEventRecord(hev, st) != cudaSuccess)
    return fail(SRTM_ERR_CUDA, "model input copy failed");
  for (int i = 0; i < n_in; ++i)
    if (!small[i] && !bulk_direct[i] &&
        cudaMemcpyAsync(stg + off[i], in[i], in_cnt[i] * sizeof(double), cudaMemcpyDefault, st) != cudaSuccess)
      return fail(SRTM_ERR_CUDA, "input copy %d failed", i);
  auto at = [&](int i) { return bulk_direct[i] ? bulk_direct[i] : (const double*)(stg + off[i]); };
  srtm_problem dp = *hp;
  dp.F = at(0); dp.Q = at(1); dp.H = at(2); dp.R = at(3); dp.m0 = at(4); dp.P0 = at(5); dp.y = at(6);
  dp.B = n_in > 7 ? at(7) : nullptr;
  dp.u = n_in > 7 ? at(8) : nullptr;
  srtm_output dout;
  double** dsl[5] = {&dout.fast_mean, &dout.fast_cov, &dout.slow_mean, &dout.slow_cov, &dout.loglik};
  for (int i = 0; i < 5; ++i) *dsl[i] = direct[i] ? direct[i] : (hout_p[i] ? (double*)(stg + off[9 + i]) : nullptr);
  rc = srtm_smoother(&dp, prec, &dout, nullptr, stream);
  if (rc) return rc;
  for (int i = 0; i < 5; ++i)
    if (hout_p[i] && !direct[i] &&
        cudaMemcpyAsync(hout_p[i], *dsl[i], out_cnt[i] * sizeof(double), cudaMemcpyDefault, st) != cudaSuccess)
      return fail(SRTM_ERR_CUDA, "output copy %d failed", i);
  return srtm_status(stream);
}

int srtm_last_error_detail(char* buf, int len) {
  const int n = (int)strlen(g_err);
  if (buf && len > 0) {
    strncpy(buf, g_err, (size_t)len - 1);
    buf[len - 1] = '\0';
  }
  return n;
}

void g_noalloc_forget(int dev);

int srtm_release(void) {
  std::lock_guard<std::mutex> lk(g_mu);
  int cur = 0;
  cudaGetDevice(&cur);
  for (int d = 0; d < MAXDEV; ++d) {
    g_noalloc_forget(d);  // looked up again by the next call (e.g. after a context reset)
    if (!g_dev[d].ws && !g_dev[d].stage && !g_dev[d].hstage && !g_dev[d].side.st) continue;
    cudaSetDevice(d);
    cudaDeviceSynchronize();
    if (g_dev[d].ws) cudaFree(g_dev[d].ws);
    if (g_dev[d].stage) cudaFree(g_dev[d].stage);
    if (g_dev[d].hstage) cudaFreeHost(g_dev[d].hstage);
    if (g_dev[d].hstage_ev) cudaEventDestroy(g_dev[d].hstage_ev);
    if (g_dev[d].side.st) cudaStreamDestroy(g_dev[d].side.st);
    if (g_dev[d].side.fork) cudaEventDestroy(g_dev[d].side.fork);
    if (g_dev[d].side.join) cudaEventDestroy(g_dev[d].side.join);


    for (int i = 0; i < NEVENT; ++i)
      if (g_dev[d].ev[i]) cudaEventDestroy(g_dev[d].ev[i]);
    g_dev[d] = DevState();
  }
  cudaSetDevice(cur);
  return SRTM_OK;
}

int srtm_set_tuning(int nx, srtm_precision prec, const srtm_tuning* t) {
  if (nx < 1 || nx > MAXNX || prec < SRTM_FP64 || prec > SRTM_FP32 || !t) return fail(SRTM_ERR_ARG, "bad tuning key");
  const int G = group_size(nx);
  if (t->scan_groups && (t->scan_groups < 1 || t->scan_groups > 256 || (t->scan_groups & (t->scan_groups - 1)) ||
                         t->scan_groups * G < 32 || t->scan_groups * G > 256))
    return fail(SRTM_ERR_ARG, "scan_groups=%d invalid for nx=%d", t->scan_groups, nx);
  if (t->scan_elems && (t->scan_elems < 1 || t->scan_elems > 64)) return fail(SRTM_ERR_ARG, "scan_elems out of range");
  if (t->recover_threads && (t->recover_threads < 32 || t->recover_threads > 128 || t->recover_threads % 32))
    return fail(SRTM_ERR_ARG, "recover_threads out of range");
  if (t->lookback_window && (t->lookback_window < 1 || t->lookback_window > 32))
    return fail(SRTM_ERR_ARG, "lookback_window out of range");
  if (t->setup_mode < 0 || t->setup_mode > 2) return fail(SRTM_ERR_ARG, "setup_mode out of range");
  if (t->recover_split < 0 || t->recover_split > 2) return fail(SRTM_ERR_ARG, "recover_split out of range");
  if (t->batch_chunks < 0 || t->batch_chunks > MAXCHUNK) return fail(SRTM_ERR_ARG, "batch_chunks out of range");
  if (t->chunk_recover_bps < 0 || t->chunk_recover_bps > 3) return fail(SRTM_ERR_ARG, "chunk_recover_bps out of range");
  if (t->chunk_scan_bps < 0 || t->chunk_scan_bps > 8) return fail(SRTM_ERR_ARG, "chunk_scan_bps out of range");
  if (t->recover_form < 0 || t->recover_form > 2) return fail(SRTM_ERR_ARG, "recover_form out of range");
  std::lock_guard<std::mutex> lk(g_mu);
  g_tune[nx][prec] = *t;
  return SRTM_OK;
}

int srtm_get_tuning(int nx, srtm_precision prec, srtm_tuning* t) {
  if (nx < 1 || nx > MAXNX || prec < SRTM_FP64 || prec > SRTM_FP32 || !t) return fail(SRTM_ERR_ARG, "bad tuning key");
  std::lock_guard<std::mutex> lk(g_mu);
  *t = effective_tuning(nx, prec);
  return SRTM_OK;
}

}  // extern "C"

namespace {

// Times `call` under each candidate tuning of (nx, prec); see srtm_autotune.
template <class Call>
int autotune_impl(int nx, srtm_precision prec, int reps, Call call, srtm_tuning* best, float* best_ms,
                  cudaStream_t st, bool batched = false) {
  if (reps < 1) return fail(SRTM_ERR_ARG, "reps=%d < 1", reps);
  srtm_tuning saved;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    saved = g_tune[nx][prec];
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  cudaStream_t cs = nullptr;  // the candidates' graphs are captured and replayed here
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess ||
      cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking) != cudaSuccess) {
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    return fail(SRTM_ERR_CUDA, "event or stream creation failed");
  }
  bool timing;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    timing = g_timing;
    g_timing = false;  // no stage events inside the captured candidates
  }
  auto restore = [&](int rc) {
    std::lock_guard<std::mutex> lk(g_mu);
    g_tune[nx][prec] = saved;
    return rc;
  };
  // A candidate runs once directly on the caller's stream (workspace, shapes,
  // errors), is then captured into a CUDA graph on a private stream and the
  // graph replayed `reps` times between events: the score is device time
  // without host launch cost, as for graph-captured production calls.
  auto score = [&](const srtm_tuning& t, float* ms) -> int {
    {
      std::lock_guard<std::mutex> lk(g_mu);
      g_tune[nx][prec] = t;
    }
    int rc = call(st);
    if (!rc) rc = srtm_status(st);
    if (rc) return rc;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeRelaxed) != cudaSuccess)
      return fail(SRTM_ERR_CUDA, "stream capture failed to start");
    rc = call(cs);
    const cudaError_t ce = cudaStreamEndCapture(cs, &graph);
    if (!rc && ce != cudaSuccess) rc = fail(SRTM_ERR_CUDA, "stream capture failed: %s", cudaGetErrorString(ce));
    if (!rc && cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) rc = fail(SRTM_ERR_CUDA, "graph instantiation failed");
    float bestr = 0.f;
    for (int r = 0; r < reps && !rc; ++r) {
      cudaEventRecord(e0, cs);
      if (cudaGraphLaunch(exec, cs) != cudaSuccess) rc = fail(SRTM_ERR_CUDA, "graph launch failed");
      cudaEventRecord(e1, cs);
      const int rs = srtm_status(cs);
      if (!rc) rc = rs;
      float v = 0.f;
      if (!rc && cudaEventElapsedTime(&v, e0, e1) != cudaSuccess) rc = fail(SRTM_ERR_CUDA, "event timing failed");
      if (!rc && (r == 0 || v < bestr)) bestr = v;
    }
    if (exec) cudaGraphExecDestroy(exec);
    if (graph) cudaGraphDestroy(graph);
    cudaGetLastError();
    *ms = bestr;
    return rc;
  };
  const int G = group_size(nx);
  srtm_tuning cur = effective_tuning(nx, prec);
  float cur_ms = 0.f;
  bool have = false;
  int rc = SRTM_OK;
  auto consider = [&](const srtm_tuning& t) {
    float ms = 0.f;
    rc = score(t, &ms);
    if (!rc && (!have || ms < cur_ms)) { cur = t; cur_ms = ms; have = true; }
    return rc;
  };
  const int elems[] = {1, 2, 4, 8, 16, 32};
  for (int sg = 1; sg * G <= 256 && !rc; sg *= 2) {
    if (sg * G < 32) continue;
    for (int e : elems) {
      srtm_tuning t = cur;
      t.scan_groups = sg;
      t.scan_elems = e;
      if (consider(t)) break;
    }
  }
  const int windows[] = {4, 8, 16, 32};
  for (int w : windows) {
    if (rc || w == cur.lookback_window) continue;
    srtm_tuning t = cur;
    t.lookback_window = w;
    consider(t);
  }
  const int threads[] = {32, 64, 96, 128};
  for (int th : threads) {
    if (rc || th == cur.recover_threads) continue;
    srtm_tuning t = cur;
    t.recover_threads = th;
    consider(t);
  }
  for (int md = 1; md <= 2; ++md) {  // interval setup in the filter scan / as its own kernel
    if (rc || md == cur.setup_mode) continue;
    srtm_tuning t = cur;
    t.setup_mode = md;
    consider(t);
  }
  // recovery: record form in one kernel / with its filtered half beside the
  // smoother scan, two-point form (which has no filtered half)
  const int forms[3][2] = {{1, 1}, {1, 2}, {2, 1}};
  for (const auto& fs : forms) {
    if (rc || (fs[0] == cur.recover_form && (fs[0] == 2 || fs[1] == cur.recover_split))) continue;
    srtm_tuning t = cur;
    t.recover_form = fs[0];
    t.recover_split = fs[1];
    consider(t);
  }
  if (batched) {  // a batch in chunks: the scans of one chunk beside the recovery of the one before
    const int chunks[] = {2, 4, 8, 16};
    for (int q : chunks) {
      if (rc || q == cur.batch_chunks) continue;
      srtm_tuning t = cur;
      t.batch_chunks = q;
      consider(t);
    }
    if (cur.batch_chunks > 1) {
      for (int b = 0; b <= 3; ++b) {
        if (rc || b == cur.chunk_recover_bps) continue;
        srtm_tuning t = cur;
        t.chunk_recover_bps = b;
        consider(t);
      }
      const int sbps[] = {0, 1, 2, 4};
      for (int b : sbps) {
        if (rc || b == cur.chunk_scan_bps) continue;
        srtm_tuning t = cur;
        t.chunk_scan_bps = b;
        consider(t);
      }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaStreamDestroy(cs);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_timing = timing;
  }
  if (rc) return restore(rc);
  {
    std::lock_guard<std::mutex> lk(g_mu);
    g_tune[nx][prec] = cur;
  }
  if (best) *best = cur;
  if (best_ms) *best_ms = cur_ms;
  return SRTM_OK;
}

}  // namespace

extern "C" {

int srtm_autotune(const srtm_problem* p, srtm_precision prec, const srtm_output* smooth, int reps,
                  srtm_tuning* best, float* best_ms, srtm_stream_t stream) {
  if (!p) return fail(SRTM_ERR_ARG, "problem is NULL");
  int rc = check_dims(p->nx, p->ny);
  if (rc) return rc;
  if (prec < SRTM_FP64 || prec > SRTM_FP32) return fail(SRTM_ERR_ARG, "unknown precision %d", (int)prec);
  return autotune_impl(
      p->nx, prec, reps, [&](cudaStream_t s) { return srtm_smoother(p, prec, smooth, nullptr, (srtm_stream_t)s); },
      best, best_ms, (cudaStream_t)stream);
}

int srtm_autotune_batch(const srtm_batch* b, srtm_precision prec, const srtm_output* smooth, int reps,
                        srtm_tuning* best, float* best_ms, srtm_stream_t stream) {
  if (!b) return fail(SRTM_ERR_ARG, "batch is NULL");
  int rc = check_dims(b->nx, b->ny);
  if (rc) return rc;
  if (prec < SRTM_FP64 || prec > SRTM_FP32) return fail(SRTM_ERR_ARG, "unknown precision %d", (int)prec);
  return autotune_impl(
      b->nx, prec, reps,
      [&](cudaStream_t s) { return srtm_smoother_batch(b, prec, smooth, nullptr, (srtm_stream_t)s); }, best, best_ms,
      (cudaStream_t)stream, true);
}

int srtm_launches_per_call(int smoothing, int batched) { return (smoothing ? 4 : 3) + (batched ? 1 : 0); }

int srtm_last_call_launches(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return 0;
  std::lock_guard<std::mutex> lk(g_mu);
  return g_dev[dev].last_launches;
}

int srtm_set_stage_timing(int enable) {
  std::lock_guard<std::mutex> lk(g_mu);
  g_timing = enable != 0;
  return SRTM_OK;
}

int srtm_stage_times(float* ms, int n) {
  int dev = 0;
  if (!ms || n < 1) return fail(SRTM_ERR_ARG, "ms must hold at least one value");
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV) return fail(SRTM_ERR_CUDA, "no device");
  std::lock_guard<std::mutex> lk(g_mu);
  DevState& d = g_dev[dev];
  if (!d.ev_valid) return fail(SRTM_ERR_ARG, "no call was timed on this device (srtm_set_stage_timing(1) first)");
  if (cudaEventSynchronize(d.ev[NSTAGE]) != cudaSuccess) return fail(SRTM_ERR_CUDA, "event synchronize failed");
  for (int i = 0; i < n && i < NSTAGE + 1; ++i) {
    if (i == NSTAGE - 1 && d.ev_chunks > 1) {  // the chunks' recovery launches, summed
      ms[i] = 0.f;
      for (int q = 0; q < d.ev_chunks; ++q) {
        float v = 0.f;
        if (cudaEventElapsedTime(&v, d.ev[NSTAGE + 4 + 2 * q], d.ev[NSTAGE + 5 + 2 * q]) != cudaSuccess)
          return fail(SRTM_ERR_CUDA, "event timing failed");
        ms[i] += v;
      }
      continue;
    }
    cudaEvent_t a = d.ev[i], b = d.ev[i + 1];
    if (i == NSTAGE - 1 && d.ev_split) a = d.ev[NSTAGE + 1];  // smoothing half only
    if (i == NSTAGE) {  // filtered half of a split recovery
      if (!d.ev_split) { ms[i] = 0.f; continue; }
      a = d.ev[NSTAGE + 2];
      b = d.ev[NSTAGE + 3];
    }
    if (cudaEventElapsedTime(&ms[i], a, b) != cudaSuccess) return fail(SRTM_ERR_CUDA, "event timing failed");
  }
  return SRTM_OK;
}

}  // extern "C"

// ===========================================================================
// Allocation-free smoother.
//
// Some callers must not allocate device memory at all: a process whose HBM
// is already reserved by another allocator (a new cudaMalloc could fail or
// fragment that pool), or a latency-bound loop that cannot absorb the
// device-wide synchronisation that cudaMalloc/cudaFree imply.  For them,
// srtm_smoother_noalloc runs the same device path as srtm_smoother with its
// scratch (metadata, model tables, look-back tile states, per-interval
// records) in the file-scope array below instead of the cached workspace.
// The array is reserved on every GPU that loads this library, for as long as
// the library stays loaded.
// ===========================================================================
namespace {
constexpr size_t NOALLOC_SCRATCH_BYTES = 32ull << 20;  // 32 MiB
}
static __device__ __align__(256) unsigned char g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
namespace {
// Device address of g_noalloc_scratch per GPU.  In host code the symbol is
// only a host-side stand-in, so the address is fetched once per device.
void* g_noalloc_addr[MAXDEV] = {};
}
// Drops the cached address of GPU dev (srtm_release; the caller holds g_mu).
void g_noalloc_forget(int dev) {
  if (dev >= 0 && dev < MAXDEV) g_noalloc_addr[dev] = nullptr;
}

extern "C" int srtm_smoother_noalloc(const srtm_problem* p, srtm_precision prec, const srtm_output* smooth,
                                     srtm_stream_t stream) {
  if (!p) return fail(SRTM_ERR_ARG, "problem is NULL");
  if (prec < SRTM_FP64 || prec > SRTM_FP32) return fail(SRTM_ERR_ARG, "unknown precision %d", (int)prec);
  int rc = check_dims(p->nx, p->ny);
  if (rc) return rc;
  if (p->ratio < 1) return fail(SRTM_ERR_ARG, "ratio=%d < 1", p->ratio);
  if (p->n_slow < 1) return fail(SRTM_ERR_ARG, "n_slow=%d < 1", p->n_slow);
  if ((rc = check_inputs(p->F, p->Q, p->H, p->R, p->m0, p->P0, p->y))) return rc;
  if ((rc = check_controls(p->nu, p->B, p->u))) return rc;
  if ((rc = check_outputs(smooth, "output"))) return rc;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= MAXDEV)
    return fail(SRTM_ERR_CUDA, "no usable CUDA device");
  cudaStream_t st = (cudaStream_t)stream;
  Ctx c;
  memset(&c, 0, sizeof c);
  c.nu = p->nu;
  c.B = p->nu ? p->B : nullptr;
  c.u = p->nu ? p->u : nullptr;
  c.n_seq = 1;
  c.fold_meta = 1;
  c.nx = p->nx;
  c.ny = p->ny;
  c.max_ratio = p->ratio;
  c.smoothing = 1;
  c.uniform_ratio = p->ratio;
  c.uniform_nslow = p->n_slow;
  c.total_slow = p->n_slow;
  c.total_fast = (long long)p->n_slow * p->ratio;
  c.F = p->F; c.Q = p->Q; c.H = p->H; c.R = p->R; c.m0 = p->m0; c.P0 = p->P0; c.y = p->y;
  set_outputs(c, smooth, nullptr);
  unsigned char* w = nullptr;
  Layout L;
  {
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_noalloc_addr[dev]) {
      void* addr = nullptr;
      const cudaError_t e = cudaGetSymbolAddress(&addr, g_noalloc_scratch);
      if (e != cudaSuccess || !addr)
        return fail(SRTM_ERR_CUDA, "cudaGetSymbolAddress of the static scratch failed: %s", cudaGetErrorString(e));
      g_noalloc_addr[dev] = addr;
    }
    w = (unsigned char*)g_noalloc_addr[dev];
    DevState& d = g_dev[dev];
    if (!d.sms && cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return fail(SRTM_ERR_CUDA, "cudaDeviceGetAttribute failed");
    const srtm_tuning t = effective_tuning(c.nx, prec);
    Shapes sh;
    rc = shapes_for(c.nx, prec, t, d.sms, c.total_slow, c.n_seq, &sh);
    if (rc) return fail(rc, "launch shape query failed (%d)", rc);
    const int tile_f = sh.scan_groups_f * sh.scan_elems_f, tile_s = sh.scan_groups_s * sh.scan_elems_s;
    L = make_layout(c.nx, c.ny, c.max_ratio, c.n_seq, c.total_slow, prec, tile_f, tile_s, c.nu, 0);
    if (L.total > NOALLOC_SCRATCH_BYTES)
      return fail(SRTM_ERR_ARG, "this problem needs %zu bytes of scratch; the static scratch holds %zu bytes",
                  L.total, NOALLOC_SCRATCH_BYTES);
    // The array keeps the previous call's contents: the control block and
    // the look-back flags must start at zero.
    if (cudaMemsetAsync(w + L.ctr, 0, sizeof(Counters), st) != cudaSuccess ||
        cudaMemsetAsync(w + L.ftile, 0, L.fout - L.ftile, st) != cudaSuccess)
      return fail(SRTM_ERR_CUDA, "clearing the static scratch failed");
    c.ctr = (Counters*)(w + L.ctr);
    c.meta.ratio = (int*)(w + L.ratio);
    c.meta.nslow = (int*)(w + L.nslow);
    c.meta.off_slow = (long long*)(w + L.off_slow);
    c.meta.off_fast = (long long*)(w + L.off_fast);
    c.meta.tile_off_f = (long long*)(w + L.tile_f);
    c.meta.tile_off_s = (long long*)(w + L.tile_s);
    c.model = (double*)(w + L.model);
    c.ml = L.ml;
    c.ftile = w + L.ftile;
    c.ftile_stride = L.ftile_stride;
    c.stile = w + L.stile;
    c.stile_stride = L.stile_stride;
    c.fout = w + L.fout;
    c.rec = w + L.rec;
    c.selem = w + L.selem;
    c.sfin = w + L.sfin;
    c.lterm = (double*)(w + L.lterm);
    c.uin = c.nu > 0 ? (double*)(w + L.uin) : nullptr;
    c.bridge = 0;  // the record form: the static scratch holds no two-point terms
    c.brec = nullptr;
    c.tile_f = tile_f;
    c.tile_s = tile_s;
    c.setup_separate = t.setup_mode == 2 ? 1 : 0;
    rc = launch_meta(c, st, nullptr);
    if (rc) return fail(rc, "launch of the metadata kernel failed");
    rc = launch_for(c.nx, c, prec, sh, st, nullptr, nullptr);
    if (rc) return fail(rc, "launch of the scan/recovery kernels failed");
  }
  // Device-side errors of this call live in the static scratch: read them on
  // the caller's stream and wait for that stream only.
  unsigned err = 0;
  const cudaError_t ce = cudaMemcpyAsync(&err, w + L.ctr + offsetof(Counters, err), sizeof err,
                                         cudaMemcpyDeviceToHost, st);
  const cudaError_t se = cudaStreamSynchronize(st);
  if (ce != cudaSuccess || se != cudaSuccess)
    return fail(SRTM_ERR_CUDA, "reading the device error latch failed: %s",
                cudaGetErrorString(ce != cudaSuccess ? ce : se));
  if (err & DEVERR_TIMEOUT) return fail(SRTM_ERR_TIMEOUT, "a scan look-back wait exceeded its bound");
  if (err & DEVERR_NOT_PSD) return fail(SRTM_ERR_NOT_PSD, "Q, R or P0 is not a covariance matrix");
  if (err & DEVERR_SINGULAR) return fail(SRTM_ERR_SINGULAR, "a solve met a zero, negative or non-finite pivot");
  return SRTM_OK;
}
