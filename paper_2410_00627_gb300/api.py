"""ctypes binding of ``libsrtm.so`` (see include/srtm.h).

Argument marshalling only: every step of the filter/smoother runs in the
library's CUDA kernels.  Tensors are torch CUDA float64 tensors (row-major,
contiguous); PyTorch provides device memory and streams.  There is no CPU
fallback: if the library is missing, every call raises.
"""
from __future__ import annotations

import ctypes
import os
from ctypes import c_int, c_longlong, c_void_p

from . import build as _build

PRECISION = {"fp64": 0, "mixed": 1, "fp32": 2}
ERRORS = {0: "SRTM_OK", -1: "SRTM_ERR_ARG", -2: "SRTM_ERR_NOT_PSD", -3: "SRTM_ERR_SINGULAR", -4: "SRTM_ERR_TIMEOUT",
          -5: "SRTM_ERR_CUDA", -6: "SRTM_ERR_UNSUPPORTED", -7: "SRTM_ERR_META"}
OUTPUT_KEYS = ("fast_mean", "fast_cov", "slow_mean", "slow_cov")   # the default outputs
ALL_OUTPUTS = OUTPUT_KEYS + ("loglik",)                               # + log p(y_1:N) per sequence

# every entry point declared in include/srtm.h
SYMBOLS = ("srtm_filter", "srtm_smoother", "srtm_filter_batch", "srtm_smoother_batch",
           "srtm_smoother_host", "srtm_status", "srtm_last_error_detail", "srtm_release",
           "srtm_set_tuning", "srtm_get_tuning", "srtm_launches_per_call", "srtm_set_stage_timing",
           "srtm_stage_times", "srtm_smoother_noalloc", "srtm_autotune", "srtm_autotune_batch",
           "srtm_last_call_launches", "srtm_filter_sequential", "srtm_smoother_sequential",
           "srtm_filter_batch_sequential", "srtm_smoother_batch_sequential", "srtm_selftest_wait",
           "srtm_measure_peak", "srtm_split_filter_aggregate", "srtm_split_smoother_aggregate",
           "srtm_split_smoother", "srtm_split_combine", "srtm_measure_link")
METHODS = {"scan": "", "sequential": "_sequential"}  # entry-point suffix per method
STAGES = ("metadata", "constants", "filter_scan", "interval_setup", "smoother_scan", "recovery",
          "recovery_filtered_half")


class Problem(ctypes.Structure):
    _fields_ = [("nx", c_int), ("ny", c_int), ("ratio", c_int), ("n_slow", c_int),
                ("F", c_void_p), ("Q", c_void_p), ("H", c_void_p), ("R", c_void_p),
                ("m0", c_void_p), ("P0", c_void_p), ("y", c_void_p),
                ("nu", c_int), ("B", c_void_p), ("u", c_void_p)]


class Output(ctypes.Structure):
    _fields_ = [(k, c_void_p) for k in ALL_OUTPUTS]


class Batch(ctypes.Structure):
    _fields_ = [("n_seq", c_int), ("nx", c_int), ("ny", c_int), ("max_ratio", c_int),
                ("total_slow", c_longlong), ("total_fast", c_longlong),
                ("ratio", c_void_p), ("n_slow", c_void_p),
                ("F", c_void_p), ("Q", c_void_p), ("H", c_void_p), ("R", c_void_p),
                ("m0", c_void_p), ("P0", c_void_p), ("y", c_void_p),
                ("nu", c_int), ("B", c_void_p), ("u", c_void_p)]


class Tuning(ctypes.Structure):
    _fields_ = [("scan_groups", c_int), ("scan_elems", c_int), ("recover_threads", c_int),
                ("lookback_window", c_int), ("setup_mode", c_int), ("recover_split", c_int),
                ("batch_chunks", c_int), ("chunk_recover_bps", c_int), ("chunk_scan_bps", c_int),
                ("recover_form", c_int)]


class SRTMError(RuntimeError):
    def __init__(self, code: int, detail: str):
        super().__init__(f"{ERRORS.get(code, code)}: {detail}")
        self.code = code


_lib = None


def lib_path() -> str:
    return _build.LIB


def load():
    """Load libsrtm.so (built by ``paper_2410_00627_gb300.build.build()``)."""
    global _lib
    if _lib is not None:
        return _lib
    path = lib_path()
    if not os.path.exists(path):
        raise RuntimeError(f"{path} is missing: build it with paper_2410_00627_gb300.build.build() "
                           "(there is no CPU fallback)")
    lib = ctypes.CDLL(path)
    P, O, B, T = ctypes.POINTER(Problem), ctypes.POINTER(Output), ctypes.POINTER(Batch), ctypes.POINTER(Tuning)
    sig = {
        "srtm_filter": [P, c_int, O, c_void_p],
        "srtm_smoother": [P, c_int, O, O, c_void_p],
        "srtm_filter_batch": [B, c_int, O, c_void_p],
        "srtm_smoother_batch": [B, c_int, O, O, c_void_p],
        "srtm_smoother_host": [P, c_int, O, c_void_p],
        "srtm_status": [c_void_p],
        "srtm_last_error_detail": [ctypes.c_char_p, c_int],
        "srtm_release": [],
        "srtm_set_tuning": [c_int, c_int, T],
        "srtm_get_tuning": [c_int, c_int, T],
        "srtm_launches_per_call": [c_int, c_int],
        "srtm_last_call_launches": [],
        "srtm_set_stage_timing": [c_int],
        "srtm_stage_times": [ctypes.POINTER(ctypes.c_float), c_int],
        "srtm_smoother_noalloc": [P, c_int, O, c_void_p],
        "srtm_autotune": [P, c_int, O, c_int, T, ctypes.POINTER(ctypes.c_float), c_void_p],
        "srtm_autotune_batch": [B, c_int, O, c_int, T, ctypes.POINTER(ctypes.c_float), c_void_p],
        "srtm_filter_sequential": [P, c_int, O, c_void_p],
        "srtm_smoother_sequential": [P, c_int, O, O, c_void_p],
        "srtm_filter_batch_sequential": [B, c_int, O, c_void_p],
        "srtm_smoother_batch_sequential": [B, c_int, O, O, c_void_p],
        "srtm_selftest_wait": [c_longlong, c_void_p],
        "srtm_measure_peak": [c_int, ctypes.c_float, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_float),
                              c_void_p],
        "srtm_split_filter_aggregate": [P, c_int, c_int, c_void_p, c_void_p],
        "srtm_split_smoother_aggregate": [P, c_int, c_int, c_void_p, c_void_p],
        "srtm_split_smoother": [P, c_void_p, c_void_p, c_int, O, O, c_void_p],
        "srtm_split_combine": [c_int, c_int, c_void_p, c_int, c_void_p, c_void_p],
        "srtm_measure_link": [c_int, ctypes.c_double, ctypes.POINTER(ctypes.c_double), c_void_p],
    }
    for name, args in sig.items():
        f = getattr(lib, name)
        f.argtypes = args
        f.restype = c_int
    _lib = lib
    return lib


def last_error_detail() -> str:
    buf = ctypes.create_string_buffer(512)
    load().srtm_last_error_detail(buf, 512)
    return buf.value.decode(errors="replace")


def _check(rc: int) -> None:
    if rc != 0:
        raise SRTMError(rc, last_error_detail())


def _stream_handle(stream):
    import torch
    s = torch.cuda.current_stream() if stream is None else stream
    return c_void_p(s.cuda_stream)


def _dev_tensor(t, name, shape):
    import torch
    if not (isinstance(t, torch.Tensor) and t.is_cuda and t.dtype == torch.float64 and t.is_contiguous()):
        raise TypeError(f"{name} must be a contiguous CUDA float64 tensor")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
    return c_void_p(t.data_ptr())


def _out_tensor(t, name, shape):
    """Outputs: CUDA tensors, or pinned host tensors (the kernels write those
    directly; with unified addressing the device uses the host address)."""
    import torch
    if isinstance(t, torch.Tensor) and not t.is_cuda:
        if not (t.is_pinned() and t.dtype == torch.float64 and t.is_contiguous()):
            raise TypeError(f"{name} must be a CUDA tensor or a contiguous pinned float64 host tensor")
        if tuple(t.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(t.shape)}, expected {tuple(shape)}")
        return c_void_p(t.data_ptr())
    return _dev_tensor(t, name, shape)


def _alloc_outputs(keys, device, rows_fast, rows_slow, nx, out=None, n_seq=1):
    import torch
    res = {}
    shapes = {"fast_mean": (rows_fast, nx), "fast_cov": (rows_fast, nx, nx),
              "slow_mean": (rows_slow, nx), "slow_cov": (rows_slow, nx, nx), "loglik": (n_seq,)}
    for k in keys:
        if k not in shapes:
            raise ValueError(f"unknown output {k}")
        t = None if out is None else out.get(k)
        if t is None:
            t = torch.empty(shapes[k], dtype=torch.float64, device=device)
        _out_tensor(t, k, shapes[k])
        res[k] = t
    o = Output(*[c_void_p(res[k].data_ptr()) if k in res else None for k in ALL_OUTPUTS])
    return res, o


def _problem(F, Q, H, R, m0, P0, y, ratio, B=None, u=None):
    nx, ny = F.shape[0], H.shape[0]
    n_slow = y.shape[0]
    nu, pB, pu = 0, None, None
    if B is not None:
        nu = B.shape[1]
        pB, pu = _dev_tensor(B, "B", (nx, nu)), _dev_tensor(u, "u", (n_slow * int(ratio), nu))
    return Problem(nx, ny, int(ratio), n_slow, _dev_tensor(F, "F", (nx, nx)), _dev_tensor(Q, "Q", (nx, nx)),
                   _dev_tensor(H, "H", (ny, nx)), _dev_tensor(R, "R", (ny, ny)), _dev_tensor(m0, "m0", (nx,)),
                   _dev_tensor(P0, "P0", (nx, nx)), _dev_tensor(y, "y", (n_slow, ny)), nu, pB, pu)


def _entry(name, method):
    if method not in METHODS:
        raise ValueError(f"method must be one of {tuple(METHODS)}, got {method!r}")
    return getattr(load(), name + METHODS[method])


def smoother(F, Q, H, R, m0, P0, y, ratio, precision="fp64", outputs=OUTPUT_KEYS, filtered=(),
             stream=None, out=None, out_filtered=None, B=None, u=None, method="scan"):
    """p(x_{k,i} | y_{1:N}) for one sequence.  Returns (smoothed, filtered) dicts
    of CUDA tensors keyed by fast_mean / fast_cov / slow_mean / slow_cov (and
    loglik when asked for).  B (nx, nu) and u (n_slow*ratio, nu): optional
    known inputs, x_{t+1} = F x_t + B u_t + w_t.  method: "scan" (the
    parallel scans, srtm_smoother) or "sequential" (srtm_smoother_sequential)."""
    prob = _problem(F, Q, H, R, m0, P0, y, ratio, B, u)
    rows_fast, rows_slow = prob.n_slow * prob.ratio, prob.n_slow
    sm, so = _alloc_outputs(outputs, y.device, rows_fast, rows_slow, prob.nx, out)
    fi, fo = _alloc_outputs(filtered, y.device, rows_fast, rows_slow, prob.nx, out_filtered)
    rc = _entry("srtm_smoother", method)(ctypes.byref(prob), PRECISION[precision], ctypes.byref(so),
                                         ctypes.byref(fo) if filtered else None, _stream_handle(stream))
    _check(rc)
    return sm, fi


def filter(F, Q, H, R, m0, P0, y, ratio, precision="fp64", outputs=OUTPUT_KEYS, stream=None, out=None,  # noqa: A001
           B=None, u=None, method="scan"):
    """p(x_{k,i} | y_{1:k}) for one sequence (method as for smoother)."""
    prob = _problem(F, Q, H, R, m0, P0, y, ratio, B, u)
    res, o = _alloc_outputs(outputs, y.device, prob.n_slow * prob.ratio, prob.n_slow, prob.nx, out)
    _check(_entry("srtm_filter", method)(ctypes.byref(prob), PRECISION[precision], ctypes.byref(o),
                                         _stream_handle(stream)))
    return res


def make_batch(F, Q, H, R, m0, P0, y, ratio, n_slow, max_ratio, total_slow, total_fast, B=None, u=None):
    """Batch descriptor over packed CUDA tensors: F (S,nx,nx), Q, H (S,ny,nx), R, m0 (S,nx),
    P0, y (total_slow, ny) and CUDA int32 tensors ratio (S,), n_slow (S,); optional
    inputs B (S,nx,nu) and u (total_fast, nu)."""
    import torch
    S, nx, ny = F.shape[0], F.shape[1], H.shape[1]
    for t, nm in ((ratio, "ratio"), (n_slow, "n_slow")):
        if not (t.is_cuda and t.dtype == torch.int32 and t.is_contiguous() and tuple(t.shape) == (S,)):
            raise TypeError(f"{nm} must be a contiguous CUDA int32 tensor of shape ({S},)")
    nu, pB, pu = 0, None, None
    if B is not None:
        nu = B.shape[2]
        pB, pu = _dev_tensor(B, "B", (S, nx, nu)), _dev_tensor(u, "u", (int(total_fast), nu))
    b = Batch(S, nx, ny, int(max_ratio), int(total_slow), int(total_fast),
              c_void_p(ratio.data_ptr()), c_void_p(n_slow.data_ptr()),
              _dev_tensor(F, "F", (S, nx, nx)), _dev_tensor(Q, "Q", (S, nx, nx)),
              _dev_tensor(H, "H", (S, ny, nx)), _dev_tensor(R, "R", (S, ny, ny)),
              _dev_tensor(m0, "m0", (S, nx)), _dev_tensor(P0, "P0", (S, nx, nx)),
              _dev_tensor(y, "y", (int(total_slow), ny)), nu, pB, pu)
    # the descriptor holds raw device pointers: keep the tensors alive with it
    b._tensors = (F, Q, H, R, m0, P0, y, ratio, n_slow, B, u)
    return b


def smoother_batch(batch: Batch, precision="fp64", outputs=OUTPUT_KEYS, filtered=(), stream=None,
                   device=None, out=None, out_filtered=None, method="scan"):
    """Ragged batch: every sequence of ``batch`` in one set of launches."""
    import torch
    device = device or torch.device("cuda", torch.cuda.current_device())
    sm, so = _alloc_outputs(outputs, device, batch.total_fast, batch.total_slow, batch.nx, out, batch.n_seq)
    fi, fo = _alloc_outputs(filtered, device, batch.total_fast, batch.total_slow, batch.nx, out_filtered, batch.n_seq)
    _check(_entry("srtm_smoother_batch", method)(ctypes.byref(batch), PRECISION[precision], ctypes.byref(so),
                                                 ctypes.byref(fo) if filtered else None, _stream_handle(stream)))
    return sm, fi


def filter_batch(batch: Batch, precision="fp64", outputs=OUTPUT_KEYS, stream=None, device=None, out=None,
                 method="scan"):
    import torch
    device = device or torch.device("cuda", torch.cuda.current_device())
    res, o = _alloc_outputs(outputs, device, batch.total_fast, batch.total_slow, batch.nx, out, batch.n_seq)
    _check(_entry("srtm_filter_batch", method)(ctypes.byref(batch), PRECISION[precision], ctypes.byref(o),
                                               _stream_handle(stream)))
    return res


def smoother_host(F, Q, H, R, m0, P0, y, ratio, precision="fp64", out=None, stream=None, loglik=False, B=None,
                  u=None):
    """Host-buffer entry point: numpy float64 inputs/outputs (pinned or pageable
    memory); the library copies to the GPU, runs the smoother, copies back and
    synchronizes.  ``out`` may hold preallocated (e.g. pinned) output arrays;
    B (nx, nu) and u (n_slow*ratio, nu) are optional known inputs."""
    import numpy as np

    def host(a, name, shape):
        if not (isinstance(a, np.ndarray) and a.dtype == np.float64 and a.flags.c_contiguous):
            raise TypeError(f"{name} must be a C-contiguous float64 numpy array")
        if tuple(a.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {a.shape}, expected {shape}")
        return c_void_p(a.ctypes.data)

    nx, ny, N = F.shape[0], H.shape[0], y.shape[0]
    nu, pB, pu = 0, None, None
    if B is not None:
        nu = B.shape[1]
        pB, pu = host(B, "B", (nx, nu)), host(u, "u", (N * int(ratio), nu))
    prob = Problem(nx, ny, int(ratio), N, host(F, "F", (nx, nx)), host(Q, "Q", (nx, nx)), host(H, "H", (ny, nx)),
                   host(R, "R", (ny, ny)), host(m0, "m0", (nx,)), host(P0, "P0", (nx, nx)), host(y, "y", (N, ny)),
                   nu, pB, pu)
    shapes = {"fast_mean": (N * ratio, nx), "fast_cov": (N * ratio, nx, nx), "slow_mean": (N, nx),
              "slow_cov": (N, nx, nx)}
    if loglik:
        shapes["loglik"] = (1,)
    res = {}
    for k, s in shapes.items():
        a = None if out is None else out.get(k)
        res[k] = np.empty(s) if a is None else a
        host(res[k], k, s)
    o = Output(*[c_void_p(res[k].ctypes.data) if k in res else None for k in ALL_OUTPUTS])
    s = c_void_p(0) if stream is None else c_void_p(stream.cuda_stream)
    _check(load().srtm_smoother_host(ctypes.byref(prob), PRECISION[precision], ctypes.byref(o), s))
    return res


def selftest_wait(polls: int, stream=None) -> None:
    """Launch the bounded wait on a flag that nothing sets (srtm_selftest_wait);
    the next status() raises SRTMError SRTM_ERR_TIMEOUT."""
    _check(load().srtm_selftest_wait(int(polls), _stream_handle(stream)))


def status(stream=None) -> None:
    """Synchronize the stream and raise if the device latched an error."""
    _check(load().srtm_status(_stream_handle(stream)))


def set_tuning(nx: int, precision: str, scan_groups=0, scan_elems=0, recover_threads=0, lookback_window=0,
               setup_mode=0, recover_split=0, batch_chunks=0, chunk_recover_bps=0, chunk_scan_bps=0,
               recover_form=0):
    _check(load().srtm_set_tuning(nx, PRECISION[precision], ctypes.byref(
        Tuning(scan_groups, scan_elems, recover_threads, lookback_window, setup_mode, recover_split, batch_chunks,
               chunk_recover_bps, chunk_scan_bps, recover_form))))


def get_tuning(nx: int, precision: str) -> dict:
    t = Tuning()
    _check(load().srtm_get_tuning(nx, PRECISION[precision], ctypes.byref(t)))
    return {k: getattr(t, k) for k, _ in Tuning._fields_}


def autotune(F, Q, H, R, m0, P0, y, ratio, precision="mixed", reps=2, stream=None, out=None, B=None, u=None):
    """Search the launch shapes for this problem (srtm_autotune) and keep the
    fastest for (nx, precision).  Returns (tuning dict, milliseconds per call)."""
    prob = _problem(F, Q, H, R, m0, P0, y, ratio, B, u)
    _, so = _alloc_outputs(OUTPUT_KEYS, y.device, prob.n_slow * prob.ratio, prob.n_slow, prob.nx, out)
    t, ms = Tuning(), ctypes.c_float()
    _check(load().srtm_autotune(ctypes.byref(prob), PRECISION[precision], ctypes.byref(so), int(reps),
                                ctypes.byref(t), ctypes.byref(ms), _stream_handle(stream)))
    return {k: getattr(t, k) for k, _ in Tuning._fields_}, float(ms.value)


def autotune_batch(batch: Batch, precision="mixed", reps=2, stream=None, device=None, out=None):
    """srtm_autotune_batch: the same search for a ragged batch."""
    import torch
    device = device or torch.device("cuda", torch.cuda.current_device())
    _, so = _alloc_outputs(OUTPUT_KEYS, device, batch.total_fast, batch.total_slow, batch.nx, out)
    t, ms = Tuning(), ctypes.c_float()
    _check(load().srtm_autotune_batch(ctypes.byref(batch), PRECISION[precision], ctypes.byref(so), int(reps),
                                      ctypes.byref(t), ctypes.byref(ms), _stream_handle(stream)))
    return {k: getattr(t, k) for k, _ in Tuning._fields_}, float(ms.value)


def last_call_launches() -> int:
    """Kernel launches of the last call issued on the current GPU."""
    return load().srtm_last_call_launches()


def launches_per_call(smoothing: bool = True, batched: bool = False) -> int:
    return load().srtm_launches_per_call(1 if smoothing else 0, 1 if batched else 0)


def set_stage_timing(enable: bool) -> None:
    _check(load().srtm_set_stage_timing(1 if enable else 0))


def stage_times() -> dict:
    """Durations (ms) of each launch of the last timed call on this GPU."""
    buf = (ctypes.c_float * len(STAGES))()
    _check(load().srtm_stage_times(buf, len(STAGES)))
    return dict(zip(STAGES, list(buf)))


def filter_element_size(nx: int) -> int:
    """Values of a filter element (F, d, D, eta, J) of Eq. 27."""
    return 3 * nx * nx + 2 * nx


def smoother_element_size(nx: int) -> int:
    """Values of a smoother element (E, g, S) of Eq. 30."""
    return 2 * nx * nx + nx


def split_filter_aggregate(F, Q, H, R, m0, P0, y, ratio, starts_sequence: bool, precision="mixed", stream=None):
    """srtm_split_filter_aggregate: the filter aggregate of this range of a
    split sequence (a float64 CUDA tensor of filter_element_size(nx))."""
    import torch
    prob = _problem(F, Q, H, R, m0, P0, y, ratio)
    agg = torch.empty(filter_element_size(prob.nx), dtype=torch.float64, device=y.device)
    _check(load().srtm_split_filter_aggregate(ctypes.byref(prob), 1 if starts_sequence else 0, PRECISION[precision],
                                              c_void_p(agg.data_ptr()), _stream_handle(stream)))
    return agg


def split_smoother_aggregate(F, Q, H, R, m_in, P_in, y, ratio, ends_sequence: bool, precision="mixed", stream=None):
    """srtm_split_smoother_aggregate: the smoother aggregate of this range
    (prior m_in, P_in = the filtered state before the range)."""
    import torch
    prob = _problem(F, Q, H, R, m_in, P_in, y, ratio)
    agg = torch.empty(smoother_element_size(prob.nx), dtype=torch.float64, device=y.device)
    _check(load().srtm_split_smoother_aggregate(ctypes.byref(prob), 1 if ends_sequence else 0, PRECISION[precision],
                                                c_void_p(agg.data_ptr()), _stream_handle(stream)))
    return agg


def split_smoother(F, Q, H, R, m_in, P_in, y, ratio, next_mean=None, next_cov=None, precision="mixed",
                   outputs=OUTPUT_KEYS, filtered=(), stream=None, out=None, out_filtered=None):
    """srtm_split_smoother: this range's smoothed (and filtered) outputs, given
    the filtered state before it and the smoothed x_{e+1,1} after it (None for
    the range that ends the sequence).  Returns (smoothed, filtered) dicts."""
    prob = _problem(F, Q, H, R, m_in, P_in, y, ratio)
    nx = prob.nx
    pm = pc = None
    if next_mean is not None:
        pm, pc = _dev_tensor(next_mean, "next_mean", (nx,)), _dev_tensor(next_cov, "next_cov", (nx, nx))
    rows_fast, rows_slow = prob.n_slow * prob.ratio, prob.n_slow
    sm, so = _alloc_outputs(outputs, y.device, rows_fast, rows_slow, nx, out)
    fi, fo = _alloc_outputs(filtered, y.device, rows_fast, rows_slow, nx, out_filtered)
    _check(load().srtm_split_smoother(ctypes.byref(prob), pm, pc, PRECISION[precision], ctypes.byref(so),
                                      ctypes.byref(fo) if filtered else None, _stream_handle(stream)))
    return sm, fi


def split_combine(op: str, elems, stream=None):
    """srtm_split_combine: the float64 product elems[0] (x) ... (x) elems[n-1]
    of filter (op "filter", Eq. 27) or smoother (op "smoother", Eq. 30)
    elements, given as a contiguous CUDA float64 tensor of shape (n, size)."""
    import torch
    n, size = elems.shape
    nx = {filter_element_size(k): k for k in range(1, 9)}.get(size) if op == "filter" else \
        {smoother_element_size(k): k for k in range(1, 9)}.get(size)
    if nx is None:
        raise ValueError(f"element size {size} matches no state size for op {op!r}")
    _dev_tensor(elems, "elems", (n, size))
    out = torch.empty(size, dtype=torch.float64, device=elems.device)
    _check(load().srtm_split_combine({"filter": 0, "smoother": 1}[op], nx, c_void_p(elems.data_ptr()), n,
                                     c_void_p(out.data_ptr()), _stream_handle(stream)))
    return out


def measure_peak(kind: str = "fp64", target_ms: float = 200.0, stream=None) -> tuple[float, float]:
    """FMA throughput of the current GPU (srtm_measure_peak): kind "fp64" or
    "fp32"; returns (GFLOP/s, milliseconds of the fastest timed launch)."""
    g, ms = ctypes.c_double(), ctypes.c_float()
    _check(load().srtm_measure_peak({"fp64": 0, "fp32": 1}[kind], float(target_ms), ctypes.byref(g), ctypes.byref(ms),
                                    _stream_handle(stream)))
    return float(g.value), float(ms.value)


LINK_KINDS = {"d2h_copy_engine": 0, "d2h_kernel_stores": 1, "h2d_copy_engine": 2, "d2h_kernel_stores_registered": 3}


def measure_link(kind: str, gib: float = 4.0, stream=None) -> float:
    """CPU-GPU link rate in GB/s (srtm_measure_link); kind is a key of LINK_KINDS."""
    g = ctypes.c_double()
    _check(load().srtm_measure_link(LINK_KINDS[kind], float(gib), ctypes.byref(g), _stream_handle(stream)))
    return float(g.value)


def release() -> None:
    load().srtm_release()
