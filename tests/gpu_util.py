"""Helpers for the GPU parity tests: run a problem through the C-ABI
(via the ctypes binding) and compare with the FP64 oracle."""
from __future__ import annotations

import numpy as np

TOL = {  # (means, covariances) relative tolerances of the paper-method outputs vs the FP64 oracle
    "fp64": (1e-9, 1e-8),
    "mixed": (1e-4, 1e-3),
}


def to_dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a, dtype=np.float64), device="cuda")


def controls(prob):
    """Known inputs of a problem as keyword arguments of the binding (none without)."""
    if getattr(prob, "B", None) is None:
        return {}
    return {"B": to_dev(prob.B), "u": to_dev(prob.u)}


def run_smoother(prob, precision="fp64", filtered=True):
    import torch

    from paper_2410_00627_gb300 import api
    args = [to_dev(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    sm, fi = api.smoother(*args, prob.ratio, precision=precision,
                          filtered=api.OUTPUT_KEYS if filtered else (), **controls(prob))
    api.status()
    torch.cuda.synchronize()
    return ({k: v.cpu().numpy() for k, v in sm.items()}, {k: v.cpu().numpy() for k, v in fi.items()})


def run_filter(prob, precision="fp64"):
    from paper_2410_00627_gb300 import api
    args = [to_dev(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    out = api.filter(*args, prob.ratio, precision=precision, **controls(prob))
    api.status()
    return {k: v.cpu().numpy() for k, v in out.items()}


# Two calls on the same inputs agree to rounding, not bit for bit: the scans'
# decoupled look-back folds the nearest prefix already published by an earlier
# tile, so the association order of the combines depends on timing.
SAME_CALL_TOL = {"fp64": 1e-12, "mixed": 1e-5, "fp32": 1e-5}


def assert_same_to_rounding(a, b, precision, label=""):
    """a, b: arrays or tensors from two calls on the same inputs."""
    a = a.cpu().numpy() if hasattr(a, "cpu") else np.asarray(a)
    b = b.cpu().numpy() if hasattr(b, "cpu") else np.asarray(b)
    assert a.shape == b.shape, (label, a.shape, b.shape)
    e = rel_err(a, b)
    assert e <= SAME_CALL_TOL[precision], f"{label}: calls differ by {e:.3e}"


def rel_err(a, b):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


def compare(gpu, ref, tol_m, tol_c, label=""):
    """gpu / ref: dicts of arrays with *_mean / *_cov keys; every key of ref
    must be in gpu (an output the GPU path did not write fails); returns the
    errors."""
    errs = {}
    for k in ref:
        assert k in gpu, f"{label}: output {k} missing from the GPU results"
        assert k.endswith("mean") or k.endswith("cov") or k == "loglik", f"{label}: unknown output {k}"
        e = rel_err(gpu[k], ref[k])
        errs[k] = e
        tol = tol_c if k.endswith("cov") else tol_m   # means and the log likelihood at the mean tolerance
        assert e <= tol, f"{label} {k}: rel err {e:.3e} > {tol:.1e}"
    return errs


def oracle_views(o, l):
    """Oracle outputs in the library's layout (smoothed, filtered)."""
    sm = {"fast_mean": o["fast_smooth_mean"], "fast_cov": o["fast_smooth_cov"],
          "slow_mean": o["fast_smooth_mean"][l - 1::l], "slow_cov": o["fast_smooth_cov"][l - 1::l]}
    fi = {"fast_mean": o["fast_filt_mean"], "fast_cov": o["fast_filt_cov"],
          "slow_mean": o["slow_filt_mean"], "slow_cov": o["slow_filt_cov"]}
    return sm, fi
