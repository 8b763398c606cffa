/*
 * srtm.h -- C-ABI of the GB300 (sm_103a) parallel-in-time filter and smoother
 * for linear Gaussian systems with slow-rate integrated measurements (SRTM),
 * after Yaghoobi & Sarkka, "Parallel state estimation for systems with
 * integrated measurements" (arXiv 2410.00627).
 *
 * Model (Sec. III, Eq. (5)-(6)), one sequence:
 *     x_{k,i} = F x_{k,i-1} + w,          w ~ N(0, Q),   x_{k,0} = x_{k-1,l}
 *     y_k     = H sum_{i=1..l} x_{k,i} + v_k,  v_k ~ N(0, R),  x_{0,l} ~ N(m0, P0)
 * for slow steps k = 1..N and fast steps i = 1..l (l = ratio).  H multiplies
 * the SUM of the l fast states; the paper's C (which multiplies their average)
 * is l*H.
 *
 * Every entry point runs the whole method on the GPU: per-model constants
 * (Eq. 7-12, 25-26), the forward filter scan with the (F,d,D,eta,J) operator
 * (Eq. 27), the per-interval smoother elements (Eq. 29), the reverse smoother
 * scan with the (E,g,S) operator (Eq. 30), and the fast-rate recovery inside
 * each slow interval (Eq. 17 and 21, Remarks 1 and 3).  No CPU fallback exists.
 *
 * Conventions for all entry points
 *   - Matrices are row-major IEEE float64.  Device entry points take DEVICE
 *     pointers (cudaMalloc'd or managed); inputs and outputs may also be
 *     mapped pinned host memory (cudaHostAlloc'd or registered, addressed by
 *     the device at its host address), which the kernels then read or write
 *     directly over the CPU-GPU link.  Any other host pointer returns
 *     SRTM_ERR_ARG.  The caller owns every input and output buffer.
 *   - Calls are asynchronous on `stream` (NULL = legacy default stream).
 *     Errors found on the device (a look-back wait that exceeded its bound,
 *     Q, R or P0 that is not a covariance, a singular solve, inconsistent
 *     batch metadata) are latched on the device and returned by
 *     srtm_status(), which synchronizes the stream.
 *   - The library owns one cached device workspace per GPU.  A call whose
 *     problem needs more workspace than any earlier call allocates it (a
 *     synchronizing cudaMalloc); make one such call before capturing calls
 *     into a CUDA graph.  srtm_release() frees it.  Calls that share a GPU
 *     must be issued on one stream (or be otherwise serialized): they share
 *     the workspace.
 *   - Limits: 1 <= nx <= 8, 1 <= ny <= 4, ratio >= 1, n_slow >= 1.
 *   - Output index convention: the fast state x_{k,i} (paper index, 1-based k
 *     and i) is row (k-1)*ratio + (i-1) of the fast outputs; the slow outputs
 *     hold x_{k,l} (the last fast state of interval k) in row k-1.  Each
 *     covariance row is a full nx*nx row-major matrix (exactly symmetric).
 */
#ifndef SRTM_H
#define SRTM_H

#ifdef __cplusplus
extern "C" {
#endif

/* Same type as cudaStream_t. */
typedef struct CUstream_st *srtm_stream_t;

typedef enum {
  SRTM_FP64 = 0,  /* everything in float64                                       */
  SRTM_MIXED = 1, /* both scans and their elements (Eq. 25-26, 29) in float32;
                     the (I + D_i J_j) solves of Eq. 27, the per-interval
                     fast-filter blocks and predicted-covariance solve
                     (Eq. 17, 21), covariance symmetrisation and the fast-rate
                     recovery in float64                                          */
  SRTM_FP32 = 2   /* everything after the per-model constants in float32          */
} srtm_precision;

enum {
  SRTM_OK = 0,
  SRTM_ERR_ARG = -1,         /* bad size, NULL required pointer, host pointer   */
  SRTM_ERR_NOT_PSD = -2,     /* Q, R or P0 not a covariance: a non-finite entry,
                                asymmetric beyond 1e-8 of its largest diagonal
                                entry, or indefinite beyond a pivot tolerance of
                                1e-10 * n * that entry (semi-definite Cholesky in
                                the constants kernel; singular matrices pass)    */
  SRTM_ERR_SINGULAR = -3,    /* a solve met a zero or non-finite pivot          */
  SRTM_ERR_TIMEOUT = -4,     /* a scan look-back wait exceeded its bound        */
  SRTM_ERR_CUDA = -5,        /* a CUDA runtime call failed                      */
  SRTM_ERR_UNSUPPORTED = -6, /* nx or ny outside the compiled range             */
  SRTM_ERR_META = -7         /* batch metadata inconsistent with declared sizes */
};

/* One sequence.  All pointers are device pointers to float64 (or mapped
 * pinned host memory, see the conventions above).
 *   F  nx*nx   fast transition (the paper's A)
 *   Q  nx*nx   fast process-noise covariance
 *   H  ny*nx   integrated-measurement matrix (applies to the sum of l states)
 *   R  ny*ny   measurement-noise covariance
 *   m0 nx, P0 nx*nx   prior of x_0
 *   y  n_slow*ny      y_k in row k-1
 * Known inputs (Sec. II: x_{t+1} = F x_t + B u_t + w_t), optional:
 *   nu                number of inputs, 0..SRTM_MAX_NU (0: no inputs, B and u
 *                     are ignored)
 *   B  nx*nu          input matrix
 *   u  n_slow*ratio*nu  u_t in row t (t = 0 .. n_slow*ratio-1); row t drives
 *                     x_{t+1}, so interval k uses rows (k-1)*ratio .. k*ratio-1 */
#define SRTM_MAX_NU 4
typedef struct {
  int nx, ny, ratio, n_slow;
  const double *F, *Q, *H, *R, *m0, *P0;
  const double *y;
  int nu;
  const double *B, *u;
} srtm_problem;

/* Caller-allocated outputs; any pointer may be NULL (that output is skipped).
 *   fast_mean n_slow*ratio*nx,  fast_cov n_slow*ratio*nx*nx
 *   slow_mean n_slow*nx,        slow_cov n_slow*nx*nx
 *   loglik    one value per sequence: log p(y_{1:N}), the sum over the slow
 *             steps of log N(y_k; C_bar m^f_{k-1,l}, S_k) with the IMKF's
 *             predicted measurement and innovation covariance (Eq. 9-12; the
 *             prediction-error decomposition of the marginal likelihood).
 *             Formed in float64 from the filter results; costs one more
 *             launch.  In a smoother call it may be given in either struct.  */
typedef struct {
  double *fast_mean, *fast_cov, *slow_mean, *slow_cov;
  double *loglik;
} srtm_output;

/* A ragged batch of independent sequences with common nx and ny.
 *   ratio[s], n_slow[s]   DEVICE int arrays of length n_seq
 *   F,Q,R,P0 ... packed per sequence: sequence s uses F + s*nx*nx, Q + s*nx*nx,
 *              H + s*ny*nx, R + s*ny*ny, m0 + s*nx, P0 + s*nx*nx
 *   y          rows of all sequences concatenated in order (total_slow rows)
 *   max_ratio  host-side upper bound of ratio[]
 *   total_slow host-side sum of n_slow[]; total_fast = sum of n_slow[s]*ratio[s]
 *   nu, B, u   optional known inputs: B packed per sequence (B + s*nx*nu), u
 *              rows of all sequences concatenated in order (total_fast rows)
 * Outputs are concatenated the same way (fast rows in sequence order, then
 * slow rows in sequence order).  Metadata that disagrees with total_slow,
 * total_fast or max_ratio is detected on the device: nothing is computed and
 * srtm_status() returns SRTM_ERR_META.                                         */
typedef struct {
  int n_seq, nx, ny, max_ratio;
  long long total_slow, total_fast;
  const int *ratio, *n_slow;
  const double *F, *Q, *H, *R, *m0, *P0;
  const double *y;
  int nu;
  const double *B, *u;
} srtm_batch;

/* Filtering p(x_{k,i} | y_{1:k}): slow IMKF by the parallel scan (Eq. 25-27)
 * and fast-rate filtering per interval (Eq. 17, Remark 1).                     */
int srtm_filter(const srtm_problem *p, srtm_precision prec, const srtm_output *filt,
                srtm_stream_t stream);

/* Smoothing p(x_{k,i} | y_{1:N}) (Eq. 21, 29-30).  `filt` (may be NULL)
 * additionally receives the filtering results computed on the way.  A call
 * with `filt` NULL and no known inputs forms the fast-rate moments in the
 * two-point form by default (srtm_tuning.recover_form): the same posterior,
 * from the smoothed joint of each interval's first state and the next one. */
int srtm_smoother(const srtm_problem *p, srtm_precision prec, const srtm_output *smooth,
                  const srtm_output *filt, srtm_stream_t stream);

/* Ragged-batch forms: every sequence of the batch in the same launches.       */
int srtm_filter_batch(const srtm_batch *b, srtm_precision prec, const srtm_output *filt,
                      srtm_stream_t stream);
int srtm_smoother_batch(const srtm_batch *b, srtm_precision prec, const srtm_output *smooth,
                        const srtm_output *filt, srtm_stream_t stream);

/* Sequential forms (the O(N)-depth comparator of the scans): the same
 * arguments, outputs and errors as the four calls above, with the slow-rate
 * recursions run one step after another, one GPU thread per sequence -- the
 * IMKF (Eq. 9-12) forward over k and the IMS recursion (Eq. 21-22) backward.
 * The per-interval work (Eq. 17 blocks, Eq. 29 elements) and the fast-rate
 * recovery (Remarks 1, 3) run as in the scan path.  Results agree with the
 * scan path up to rounding.  Tuning: setup_mode is ignored (always its own
 * kernel); the scan shapes do not apply.                                      */
int srtm_filter_sequential(const srtm_problem *p, srtm_precision prec, const srtm_output *filt,
                           srtm_stream_t stream);
int srtm_smoother_sequential(const srtm_problem *p, srtm_precision prec, const srtm_output *smooth,
                             const srtm_output *filt, srtm_stream_t stream);
int srtm_filter_batch_sequential(const srtm_batch *b, srtm_precision prec, const srtm_output *filt,
                                 srtm_stream_t stream);
int srtm_smoother_batch_sequential(const srtm_batch *b, srtm_precision prec, const srtm_output *smooth,
                                   const srtm_output *filt, srtm_stream_t stream);

/* One sequence split over several GPUs (Sec. II: the filter operator of
 * Eq. (27) and the smoother operator of Eq. (30) are associative, so a scan
 * over the whole sequence is a scan over each range combined with the
 * product of the ranges before it (filter) or after it (smoother); Sec. IV:
 * the span stays logarithmic).  Each GPU holds a contiguous range of slow
 * steps k = s..e (its y rows in p->y, p->n_slow = e-s+1; F, Q, H, R as for
 * the whole sequence; known inputs are not supported: p->nu must be 0,
 * else SRTM_ERR_UNSUPPORTED) and makes, in this order:
 *   1. srtm_split_filter_aggregate: agg_f = a_s (x) ... (x) a_e (Eq. 25-27);
 *      the first range (starts_sequence = 1) has a_1 from p->m0, p->P0; the
 *      others have generic elements only (m0, P0 are read but do not enter).
 *   2. exchange: gather every range's agg_f; with srtm_split_combine(0, ...)
 *      over the aggregates of the EARLIER ranges, (d, D) of the product is
 *      the filtered x_{s-1,l} ~ N(m_in, P_in) (the first range keeps m0, P0).
 *   3. srtm_split_smoother_aggregate with p->m0, p->P0 = m_in, P_in:
 *      agg_s = b_s (x) ... (x) b_e (Eq. 29-30), where b_e is the generic
 *      element unless ends_sequence (then E_e = 0, Eq. 29 with k = N).
 *   4. exchange: gather every range's agg_s; with srtm_split_combine(1, ...)
 *      over the aggregates of the LATER ranges, (g, S) of the product is the
 *      smoothed x_{e+1,1} ~ N(next_mean, next_cov) (the last range has none).
 *   5. srtm_split_smoother with p->m0, p->P0 = m_in, P_in and next_mean,
 *      next_cov (NULL for the last range): the range's fast- and slow-rate
 *      smoothed (and optionally filtered) outputs, rows relative to the range,
 *      equal to those of the whole sequence's srtm_smoother up to rounding.
 *      Its loglik output is the range's share of log p(y_{1:N}) (the sum over
 *      the ranges is the sequence's).
 * Aggregates are float64 device arrays: a filter element (F, d, D, eta, J)
 * holds 3 nx^2 + 2 nx values in that order (matrices row-major), a smoother
 * element (E, g, S) 2 nx^2 + nx.  In the mixed and FP32 modes they carry the
 * float32 scans' rounding.  The calls are asynchronous on `stream`; errors
 * are those of srtm_smoother (device errors through srtm_status).  The
 * exchange itself (an all-gather of 3 nx^2 + 2 nx values per range, then of
 * 2 nx^2 + nx) is the caller's: NCCL between GPUs, or any transport.        */
int srtm_split_filter_aggregate(const srtm_problem *p, int starts_sequence, srtm_precision prec, double *agg,
                                srtm_stream_t stream);
int srtm_split_smoother_aggregate(const srtm_problem *p, int ends_sequence, srtm_precision prec, double *agg,
                                  srtm_stream_t stream);
int srtm_split_smoother(const srtm_problem *p, const double *next_mean, const double *next_cov,
                        srtm_precision prec, const srtm_output *smooth, const srtm_output *filt,
                        srtm_stream_t stream);
/* The float64 product elems[0] (x) elems[1] (x) ... (x) elems[n-1] of n >= 1
 * filter elements (op 0, Eq. 27) or smoother elements (op 1, Eq. 30), each
 * laid out as above and stored one after another, written to out (one
 * element; its symmetric blocks D and J, or S, as the mean of the matrix and
 * its transpose).  Device pointers; asynchronous on `stream`; a singular
 * solve is latched for srtm_status().  Errors: SRTM_ERR_ARG,
 * SRTM_ERR_UNSUPPORTED (nx), SRTM_ERR_CUDA.                                   */
int srtm_split_combine(int op, int nx, const double *elems, int n, double *out, srtm_stream_t stream);

/* srtm_smoother with HOST buffers (pageable or pinned) for every input and
 * output.  The model arrays (F, Q, H, R, m0, P0, B) are packed into a
 * library-owned pinned buffer and copied to the device in one transfer.  The
 * per-step arrays (y, u) and the outputs, where they are pinned host memory
 * the device can address (cudaHostAlloc'd or registered, unified addressing),
 * are read and written by the kernels directly over the CPU-GPU link; where
 * they are not, they are staged on the device and copied.  Synchronizes the
 * stream and returns the final status (as srtm_status).                       */
int srtm_smoother_host(const srtm_problem *host_p, srtm_precision prec,
                       const srtm_output *host_smooth, srtm_stream_t stream);

/* Synchronizes `stream`, then returns and clears the device-side error latch of
 * the current GPU: SRTM_OK, SRTM_ERR_META, SRTM_ERR_TIMEOUT, SRTM_ERR_NOT_PSD
 * or SRTM_ERR_SINGULAR (the first that applies, in that order).               */
int srtm_status(srtm_stream_t stream);

/* Failure-detection self-test (the paper has no counterpart).  Launches one
 * GPU thread on `stream` that waits, with the bounded polling every device-side
 * wait of this library uses (the scans' look-back), on a control-block flag
 * that nothing sets.  After `polls` polls (1..2000000; back-off 32 ns doubling
 * to 1 us, so about polls microseconds) the wait gives up, latches the
 * device error that the next srtm_status() returns as SRTM_ERR_TIMEOUT, and
 * the kernel returns: the context stays usable.  Returns SRTM_ERR_ARG for
 * polls out of range, SRTM_ERR_CUDA if the launch fails.                      */
int srtm_selftest_wait(long long polls, srtm_stream_t stream);

/* Copies a NUL-terminated description of the last host-side error of this
 * thread into buf (at most len bytes).  Returns the length of the message.    */
int srtm_last_error_detail(char *buf, int len);

/* Frees the cached device workspace, the staging buffers and the library's
 * second streams and events of every GPU.                                     */
int srtm_release(void);

/* Tuning of the launch shapes (lane groups per scan block, elements per lane
 * group, recovery block size, look-back depth, setup placement, recovery
 * split, batch pipelining) for one (nx, precision).  Zero values keep the
 * built-in choice (128/lanes-per-group groups, 4 elements, 128 threads,
 * window 16, setup inside the filter scan, one recovery kernel, batches in
 * one chunk, two-point recovery form).  Returns SRTM_ERR_ARG for
 * out-of-range values.  The setting is process-wide and applies to the calls
 * issued after it.                                                            */
typedef struct {
  int scan_groups;      /* lane groups per scan block: a power of two such that
                           groups x lanes-per-group (1, 4, 16 or 32 by nx) is
                           32..256                                              */
  int scan_elems;       /* elements per lane group per tile (1..64)            */
  int recover_threads;  /* recovery block size (32..128, multiple of 32)       */
  int lookback_window;  /* scan look-back depth: preceding tiles examined per
                           round of the decoupled look-back (1..32)            */
  int setup_mode;       /* interval setup (smoother elements and recovery
                           records): 1 = inside the filter scan, after each
                           tile's results; 2 = its own kernel after the filter
                           scan (one more launch)                            */
  int recover_split;    /* fast-rate recovery of smoother calls: 1 = one kernel
                           after the smoother scan; 2 = split in two: the
                           filtered half on a library-owned second stream,
                           concurrently with the smoother scan, the smoothing
                           half after it (one more launch; needs
                           total_fast*(nx + nx(nx+1)/2 + nx^2) recovery-type
                           words of workspace and is used only while that is
                           at most 4 GiB and every output is device memory,
                           else 1 applies)                                   */
  int batch_chunks;     /* batches (scan method) only: 1 = every stage over the
                           whole batch; 2..16 = the batch is processed in that
                           many chunks of whole sequences with nearly equal
                           fast steps, the fast-rate recovery of chunk q on a
                           library-owned second stream while the scans of
                           chunk q+1 run (replaces recover_split)             */
  int chunk_recover_bps;/* recovery grid of a chunked batch: 0 = one thread per
                           fast step of the chunk; 1..3 = that many resident
                           blocks per SM, each thread looping over fast steps */
  int chunk_scan_bps;   /* scan grid of a chunked batch: 0 = as many blocks per
                           SM as fit; 1..8 = at most that many per SM        */
  int recover_form;     /* fast-rate recovery of smoother calls: 1 = record
                           form (filtered fast-rate moments of the interval,
                           Remarks 1 and 3, then the smoothing terms of Eq.
                           21); 2 = two-point form for the calls that ask for
                           smoothed outputs only, without known inputs (not
                           the range calls of a split sequence nor
                           srtm_smoother_noalloc): every fast-rate smoothed
                           moment from the smoothed joint of the interval's
                           first state and the next interval's first state,
                           conditioned on the interval's measurement (the
                           same posterior, about 15% fewer float64
                           operations per fast step at ny = 1; one record of
                           3 nx^2 + 2 nx recovery-type words per slow step
                           more workspace).  A sequence whose covariance of
                           (next first state, measurement) given the
                           interval's first state is singular or nearly so (a
                           pivot below 1e-6 of the variance it came from, e.g.
                           no process noise) keeps the record form inside a
                           two-point call.                                  */
} srtm_tuning;
int srtm_set_tuning(int nx, srtm_precision prec, const srtm_tuning *t);
int srtm_get_tuning(int nx, srtm_precision prec, srtm_tuning *t);

/* Autotuner (the paper has no counterpart; launch shapes are a property of
 * this implementation).  Runs srtm_smoother on the caller's problem with a
 * sequence of candidate tunings and keeps the fastest for (p->nx, prec) as if
 * by srtm_set_tuning: first the grid of scan_groups (every valid power of
 * two) x scan_elems (1, 2, 4, 8, 16, 32), then lookback_window (4, 8, 16, 32)
 * recover_threads (32, 64, 96, 128) and setup_mode (1, 2) one at a time
 * from the best so far, then the recovery as (recover_form, recover_split)
 * in (1, 1), (1, 2), (2, 1).
 * Each candidate is run once untimed on `stream`, then captured into a CUDA
 * graph on a private stream and the graph replayed `reps` times (reps >= 1),
 * timed by CUDA events around each replay (device time without host launch
 * cost); its score is the fastest of the reps.  Inputs and `smooth` are as
 * for srtm_smoother (device buffers owned by the caller); `smooth` is
 * overwritten by every run.  The streams are synchronized after each run.  On success *best (if not NULL) receives the
 * chosen tuning and *best_ms (if not NULL) its time in milliseconds.  Errors:
 * those of srtm_smoother and srtm_status (the first failing candidate stops
 * the search and the previous tuning is restored).                          */
int srtm_autotune(const srtm_problem *p, srtm_precision prec, const srtm_output *smooth, int reps,
                  srtm_tuning *best, float *best_ms, srtm_stream_t stream);
/* The same for a batch (srtm_smoother_batch; tuning key (b->nx, prec)), whose
 * search then also tries batch_chunks (1, 2, 4, 8, 16) and, for the best
 * chunk count above 1, chunk_recover_bps (0..3) and chunk_scan_bps (0, 1, 2,
 * 4) one at a time.                                                          */
int srtm_autotune_batch(const srtm_batch *b, srtm_precision prec, const srtm_output *smooth, int reps,
                        srtm_tuning *best, float *best_ms, srtm_stream_t stream);

/* Kernel launches of a plain call (for reporting): constants, filter scan
 * (which also forms the per-interval smoother elements), smoother scan
 * (smoother calls only) and fast-rate recovery, plus the metadata kernel for
 * batches.                                                                    */
int srtm_launches_per_call(int smoothing, int batched);
/* Kernel launches of the last call issued on the current GPU (0 before any):
 * srtm_launches_per_call plus one for each of a separate setup kernel, a
 * split recovery, known inputs and the log likelihood; a batch in C chunks
 * launches its scans, setup and recovery once per chunk.                      */
int srtm_last_call_launches(void);

/* Stage timing.  While enabled, every call records CUDA events on its stream
 * around each of its launches.  srtm_stage_times() waits for the last timed
 * call of the current GPU and writes up to n durations in milliseconds, in
 * launch order: metadata, model constants, filter scan, interval setup,
 * smoother scan (0 for a filter call), fast-rate recovery (with a split
 * recovery: its smoothing half), then the filtered half of a split recovery
 * (run beside the smoother scan on the second stream; 0 without a split).
 * A batch in chunks reports as "filter scan" the time from the end of the
 * constants to the end of the last chunk's smoother scan (all chunks' scans,
 * overlapping the recoveries of the earlier chunks), 0 for the setup and the
 * smoother scan, and as "recovery" the summed durations of the chunks'
 * recovery launches (each timed on the second stream; they overlap scans).  */
int srtm_set_stage_timing(int enable);
int srtm_stage_times(float *ms, int n);

/* Arithmetic-throughput calibration (the paper has no counterpart; used for
 * the roofline denominators of the benchmark).  Runs a kernel of independent
 * FMA chains (8 per thread, a <- a*b + c) on every SM of the current GPU at its
 * occupancy limit, in float64 (kind 0) or float32 (kind 1), sized so that one
 * launch lasts about target_ms milliseconds (1..5000), and writes the fastest
 * of three timed launches (CUDA events on `stream`) to *gflops (GFLOP/s, an
 * FMA counted as 2 flops) and its duration to *ms (may be NULL).  Allocates a
 * small output buffer with cudaMallocAsync on `stream` and synchronizes it.
 * Errors: SRTM_ERR_ARG (kind, target_ms or gflops invalid), SRTM_ERR_CUDA.   */
int srtm_measure_peak(int kind, float target_ms, double *gflops, float *ms, srtm_stream_t stream);
/* CPU-GPU link calibration (the paper has no counterpart; it explains the
 * end-to-end numbers of the benchmark): moves `gib` GiB (1/16..64) between a
 * device buffer and page-locked host memory and writes the fastest of three
 * timed moves (after one untimed) in GB/s to *gbps.  kind 0: device to host
 * by cudaMemcpyAsync (copy engine) into cudaHostAlloc'd memory; 1: device to
 * host by a kernel of consecutive 16-byte stores into the same kind of
 * memory; 2: host to device by cudaMemcpyAsync; 3: as 1 into malloc'd memory
 * registered with cudaHostRegister.  Allocates and frees its buffers
 * (cudaMalloc, cudaHostAlloc or malloc + cudaHostRegister) and synchronizes
 * `stream`.  Errors: SRTM_ERR_ARG, SRTM_ERR_CUDA.                            */
int srtm_measure_link(int kind, double gib, double *gbps, srtm_stream_t stream);

/* srtm_smoother for callers that must not allocate device memory (the paper
 * has no counterpart; this is a deployment variant).  Such callers include a
 * process whose GPU memory is already reserved by another allocator, where a
 * new cudaMalloc could fail or fragment that pool, and latency-bound loops
 * that cannot absorb the device-wide synchronisation of cudaMalloc/cudaFree.
 * This entry point calls no cudaMalloc, cudaFree or other allocating routine:
 * its scratch is a 32 MiB static device array that every GPU loading this
 * library reserves until the library is unloaded.  Inputs and outputs are the
 * caller's device buffers, as for srtm_smoother (filtered extras are not
 * offered).  A problem whose scratch would exceed 32 MiB (for nx=4 in float64
 * about 2*10^4 slow steps) returns SRTM_ERR_ARG with the needed size in
 * srtm_last_error_detail().  The first call on a GPU looks up the array's
 * device address on that GPU (make it before any stream capture); the address
 * is kept until srtm_release(), after which the next call looks it up again
 * (so release after resetting the device).  All calls share the array: calls
 * whose work overlaps on the GPU (other streams or threads) race and must be
 * serialized by the caller.  The call reads its device-side status on
 * `stream`, synchronizes that stream (only), and returns the status directly
 * (SRTM_OK, SRTM_ERR_TIMEOUT, SRTM_ERR_NOT_PSD or SRTM_ERR_SINGULAR).         */
int srtm_smoother_noalloc(const srtm_problem *p, srtm_precision prec, const srtm_output *smooth,
                          srtm_stream_t stream);

#ifdef __cplusplus
}
#endif
#endif /* SRTM_H */
