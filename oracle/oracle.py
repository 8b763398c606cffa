"""ctypes wrapper around ``oracle.c`` (plain FP64 C, compiled with gcc).

TEST INFRASTRUCTURE ONLY: this is the independent checker of the CUDA
library.  It shares no code with ``paper_2410_00627_gb300``; inputs come from
the seeded generators and are passed to both sides.

Functions take any object with attributes F, Q, H, R, m0, P0, y, ratio (the
paper's A, Q, C/l, R, m0, P0, y_{1:N}, l).  Arrays are float64, row-major.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
SO = os.path.join(HERE, "liboracle.so")

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def build(force: bool = False) -> str:
    """Compile oracle.c into oracle/liboracle.so (gcc -O2, no fast-math)."""
    if not force and os.path.exists(SO) and os.path.getmtime(SO) >= os.path.getmtime(SRC):
        return SO
    tmp = SO + f".{os.getpid()}.tmp"
    subprocess.check_call(["gcc", "-O2", "-std=c99", "-shared", "-fPIC", "-o", tmp, SRC, "-lm"])
    os.replace(tmp, SO)
    return SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(SO)
        i = ctypes.c_int
        lib.oracle_srtm_sequential.argtypes = [i, i, i, i] + [_dp] * 7 + [i, i] + [_dp] * 8 + [i, _dp, _dp]
        lib.oracle_srtm_parallel.argtypes = [i, i, i, i] + [_dp] * 7 + [i, i] + [_dp] * 4 + [i, _dp, _dp]
        lib.oracle_filter_op.argtypes = [i, _dp, _dp, _dp]
        lib.oracle_smoother_op.argtypes = [i, _dp, _dp, _dp]
        lib.oracle_lifted.argtypes = [i, i, i] + [_dp] * 8
        lib.oracle_loglik.argtypes = [i, i, i, i] + [_dp] * 9 + [i, _dp, _dp]
        for f in (lib.oracle_srtm_sequential, lib.oracle_srtm_parallel, lib.oracle_filter_op,
                  lib.oracle_smoother_op, lib.oracle_lifted, lib.oracle_loglik):
            f.restype = ctypes.c_int
        _lib = lib
    return _lib


def _p(a):
    if a is None:
        return None
    assert a.dtype == np.float64 and a.flags.c_contiguous
    return a.ctypes.data_as(_dp)


def _inputs(prob):
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
    return [c(prob.F), c(prob.Q), c(prob.H), c(prob.R), c(prob.m0), c(prob.P0), c(prob.y)]


def _controls(prob):
    """(nu, B, u) of the known inputs, or (0, None, None)."""
    B, u = getattr(prob, "B", None), getattr(prob, "u", None)
    if B is None or u is None:
        return 0, None, None
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
    B, u = c(B), c(u)
    return B.shape[1], B, u


def sequential(prob, k_lo: int = 0, k_hi: int | None = None, fast: bool = True,
               smooth: bool = True, slow: bool = True) -> dict:
    """Sequential IMKF + fast filter + the paper's sequential smoother.

    Returns dict with (when requested) slow_filt_mean/cov (x_{k,l}|y_{1:k}),
    first_smooth_mean/cov (x_{k,1}|y_{1:N}), fast_filt_mean/cov and
    fast_smooth_mean/cov for intervals [k_lo, k_hi) with shape
    ((k_hi-k_lo)*l, nx) / (..., nx, nx)."""
    lib = _load()
    n, m, l, N = prob.F.shape[0], prob.H.shape[0], int(prob.ratio), prob.y.shape[0]
    k_hi = N if k_hi is None else k_hi
    nf = (k_hi - k_lo) * l
    out = {}
    z = lambda *s: np.zeros(s)  # noqa: E731
    if slow:
        out["slow_filt_mean"], out["slow_filt_cov"] = z(N, n), z(N, n, n)
    if smooth:
        out["first_smooth_mean"], out["first_smooth_cov"] = z(N, n), z(N, n, n)
    if fast:
        out["fast_filt_mean"], out["fast_filt_cov"] = z(nf, n), z(nf, n, n)
        if smooth:
            out["fast_smooth_mean"], out["fast_smooth_cov"] = z(nf, n), z(nf, n, n)
    keys = ["slow_filt_mean", "slow_filt_cov", "first_smooth_mean", "first_smooth_cov",
            "fast_filt_mean", "fast_filt_cov", "fast_smooth_mean", "fast_smooth_cov"]
    ins = _inputs(prob)
    nu, B, u = _controls(prob)
    rc = lib.oracle_srtm_sequential(n, m, l, N, *[_p(a) for a in ins], k_lo, k_hi,
                                    *[_p(out.get(k)) for k in keys], nu, _p(B), _p(u))
    if rc != 0:
        raise RuntimeError(f"oracle_srtm_sequential failed rc={rc}")
    return out


def parallel(prob, order: int = 0, flags: int = 0) -> dict:
    """The paper's parallel-form elements/operators folded on the CPU
    (order 0: sequential fold, 1: doubling bracketing).  flags=1 uses the
    printed (untransposed) S_k formula."""
    lib = _load()
    n, m, l, N = prob.F.shape[0], prob.H.shape[0], int(prob.ratio), prob.y.shape[0]
    out = {k: np.zeros(s) for k, s in [("slow_filt_mean", (N, n)), ("slow_filt_cov", (N, n, n)),
                                       ("first_smooth_mean", (N, n)), ("first_smooth_cov", (N, n, n))]}
    ins = _inputs(prob)
    nu, B, u = _controls(prob)
    rc = lib.oracle_srtm_parallel(n, m, l, N, *[_p(a) for a in ins], order, flags,
                                  *[_p(out[k]) for k in ["slow_filt_mean", "slow_filt_cov",
                                                         "first_smooth_mean", "first_smooth_cov"]],
                                  nu, _p(B), _p(u))
    if rc != 0:
        raise RuntimeError(f"oracle_srtm_parallel failed rc={rc}")
    return out


def _pack_filter(e, n):
    return np.concatenate([np.ravel(e["F"]), e["d"], np.ravel(e["D"]), e["eta"], np.ravel(e["J"])])


def _unpack_filter(v, n):
    nn = n * n
    return {"F": v[:nn].reshape(n, n), "d": v[nn:nn + n], "D": v[nn + n:2 * nn + n].reshape(n, n),
            "eta": v[2 * nn + n:2 * nn + 2 * n], "J": v[2 * nn + 2 * n:].reshape(n, n)}


def filter_op(ai: dict, aj: dict) -> dict:
    """Eq. (27) on elements given as dicts with F, d, D, eta, J."""
    lib = _load()
    n = ai["F"].shape[0]
    a, b = _pack_filter(ai, n), _pack_filter(aj, n)
    o = np.zeros_like(a)
    rc = lib.oracle_filter_op(n, _p(a), _p(b), _p(o))
    if rc != 0:
        raise RuntimeError("oracle_filter_op: singular")
    return _unpack_filter(o, n)


def smoother_op(ai: dict, aj: dict) -> dict:
    """Eq. (30) on elements given as dicts with E, g, S."""
    lib = _load()
    n = ai["E"].shape[0]
    pk = lambda e: np.concatenate([np.ravel(e["E"]), e["g"], np.ravel(e["S"])])  # noqa: E731
    a, b = pk(ai), pk(aj)
    o = np.zeros_like(a)
    lib.oracle_smoother_op(n, _p(a), _p(b), _p(o))
    nn = n * n
    return {"E": o[:nn].reshape(n, n), "g": o[nn:nn + n], "S": o[nn + n:].reshape(n, n)}


def lifted(F, Q, H, ratio: int) -> dict:
    """Slow-rate lifted model of Sec. III-A: Abar, Qbar, Cbar, MQM (= M Q~ M^T),
    GQM (= G Q~ M^T)."""
    lib = _load()
    n, m = F.shape[0], H.shape[0]
    out = {"Abar": np.zeros((n, n)), "Qbar": np.zeros((n, n)), "Cbar": np.zeros((m, n)),
           "MQM": np.zeros((m, m)), "GQM": np.zeros((n, m))}
    c = lambda a: np.ascontiguousarray(a, dtype=np.float64)  # noqa: E731
    Fc, Qc, Hc = c(F), c(Q), c(H)
    lib.oracle_lifted(n, m, int(ratio), _p(Fc), _p(Qc), _p(Hc),
                      *[_p(out[k]) for k in ["Abar", "Qbar", "Cbar", "MQM", "GQM"]])
    return out


def loglik(prob, terms: bool = False):
    """log p(y_{1:N}) by the prediction-error decomposition of the slow-rate
    IMKF (Eq. 9-12); with terms=True also the N per-interval terms."""
    lib = _load()
    n, m, l, N = prob.F.shape[0], prob.H.shape[0], int(prob.ratio), prob.y.shape[0]
    t = np.zeros(N) if terms else None
    total = np.zeros(1)
    nu, B, u = _controls(prob)
    rc = lib.oracle_loglik(n, m, l, N, *[_p(a) for a in _inputs(prob)], _p(t), _p(total), nu, _p(B), _p(u))
    if rc != 0:
        raise RuntimeError(f"oracle_loglik failed rc={rc}")
    return (float(total[0]), t) if terms else float(total[0])
