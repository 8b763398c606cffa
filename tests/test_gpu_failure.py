"""Failure detection on the GPU without a fault: a bounded device-side wait on
a flag that nothing sets gives up, latches the timeout, and the host reads it
through srtm_status; the context stays usable for the next call."""
import time

import numpy as np
import pytest

from paper_2410_00627_gb300 import synth
from tests.gpu_util import TOL, compare, oracle_views, run_smoother, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00627_gb300 import api, build
    build.build()
    api.load()


def test_wait_that_runs_out_is_reported_and_the_context_survives(oracle_mod):
    from paper_2410_00627_gb300 import api
    api.status()  # nothing latched before
    t0 = time.perf_counter()
    api.selftest_wait(2000)
    with pytest.raises(api.SRTMError) as err:
        api.status()
    elapsed = time.perf_counter() - t0
    assert err.value.code == -4  # SRTM_ERR_TIMEOUT
    assert elapsed < 5.0, elapsed
    api.status()  # the latch was cleared by the read
    prob = synth.random_model(71, 3, 2, 5, 40)
    sm, fi = run_smoother(prob, "fp64")
    ref_sm, ref_fi = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    compare(sm, ref_sm, *TOL["fp64"], label="after timeout")
    compare(fi, ref_fi, *TOL["fp64"], label="after timeout")


def test_timeout_latch_is_per_read_and_repeatable():
    from paper_2410_00627_gb300 import api
    for _ in range(3):
        api.selftest_wait(50)
        with pytest.raises(api.SRTMError):
            api.status()
        api.status()
    assert np.isfinite(api.last_call_launches())


def test_singular_model_is_reported_and_the_next_call_is_clean(oracle_mod):
    """No process or measurement noise and an exactly known prior: the
    measurement covariance R_x = M Q~ M^T + R is zero, the solves meet a zero
    pivot, the latch reports SRTM_ERR_SINGULAR (the kernels divide by one
    instead and stay finite), and the next call is unaffected."""
    from paper_2410_00627_gb300 import api
    nx, ny, l, N = 2, 1, 3, 20
    F = np.eye(nx)
    Q = np.zeros((nx, nx))
    H = np.array([[1.0, 0.0]])
    R = np.zeros((ny, ny))
    m0 = np.zeros(nx)
    P0 = np.zeros((nx, nx))
    y = np.zeros((N, ny))
    args = [to_dev(a) for a in (F, Q, H, R, m0, P0, y)]
    api.smoother(*args, l, precision="fp64")
    with pytest.raises(api.SRTMError) as err:
        api.status()
    assert err.value.code == -3  # SRTM_ERR_SINGULAR
    api.status()
    prob = synth.random_model(72, 2, 1, 3, 30)
    sm, _ = run_smoother(prob, "fp64")
    ref_sm, _ = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    compare(sm, ref_sm, *TOL["fp64"], label="after a singular call")


def _with(prob, **over):
    return [to_dev(np.asarray(over.get(k, getattr(prob, k)), dtype=np.float64))
            for k in ("F", "Q", "H", "R", "m0", "P0", "y")]


def _indefinite_q(nx):
    """A covariance with one eigenvalue pushed to -1e-3 of the largest."""
    rng = np.random.default_rng(5)
    V, _ = np.linalg.qr(rng.standard_normal((nx, nx)))
    ev = np.linspace(1.0, 0.1, nx)
    ev[-1] = -1e-3
    return 1e-2 * (V * ev) @ V.T


BAD = {  # name -> overrides of a (nx=3, ny=2) model that are not covariances
    "Q_indefinite": lambda p: {"Q": _indefinite_q(3)},
    "Q_indefinite_behind_a_zero_pivot": lambda p: {"Q": np.array([[0.0, 1e-3, 0], [1e-3, 1e-2, 0], [0, 0, 1e-2]])},
    "R_asymmetric": lambda p: {"R": p.R + np.array([[0.0, 1e-3 * p.R[0, 0]], [0.0, 0.0]])},
    "R_negative_diagonal": lambda p: {"R": np.diag([-1e-2, 1e-2])},
    "P0_nan": lambda p: {"P0": np.where(np.eye(3) > 0, np.nan, 0.0)},
    "P0_inf_offdiagonal": lambda p: {"P0": p.P0 + np.array([[0, np.inf, 0], [np.inf, 0, 0], [0, 0, 0]])},
}

GOOD = {  # covariances the check must accept (singular ones included)
    "Q_rank_one": lambda p: {"Q": 1e-2 * np.outer([1.0, -2.0, 0.5], [1.0, -2.0, 0.5])},
    "Q_zero": lambda p: {"Q": np.zeros((3, 3))},
    "P0_zero": lambda p: {"P0": np.zeros((3, 3))},
    "R_asymmetric_to_rounding": lambda p: {"R": p.R + np.array([[0.0, 1e-15 * p.R[0, 0]], [0.0, 0.0]])},
}
# With no process noise at all the backward pass in any RTS form, the
# oracle's included, multiplies by the inverse of the contracting transition
# (Z = A^T (A P A^T)^-1) a hundred times: the early smoothed covariances are
# lost to rounding on both sides.  The filter has no such step.
FILTER_ONLY = {"Q_zero"}


@pytest.mark.parametrize("method", ["scan", "sequential"])
@pytest.mark.parametrize("bad", sorted(BAD))
def test_non_covariance_input_is_reported_and_the_next_call_is_clean(oracle_mod, bad, method):
    """Q, R or P0 that is not a covariance (indefinite, asymmetric, non-finite)
    latches SRTM_ERR_NOT_PSD in the constants kernel; the next call is exact."""
    from paper_2410_00627_gb300 import api
    prob = synth.random_model(73, 3, 2, 4, 25)
    api.status()
    api.smoother(*_with(prob, **BAD[bad](prob)), prob.ratio, precision="fp64", method=method)
    with pytest.raises(api.SRTMError) as err:
        api.status()
    assert err.value.code == -2, err.value  # SRTM_ERR_NOT_PSD
    api.status()
    sm, _ = run_smoother(prob, "fp64")
    ref_sm, _ = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    compare(sm, ref_sm, *TOL["fp64"], label=f"after {bad}")


@pytest.mark.parametrize("good", sorted(GOOD))
def test_singular_covariances_pass_the_check_and_match_the_oracle(oracle_mod, good):
    """Positive semi-definite but singular Q or P0 (noise on a subspace, a
    known initial state) and rounding-level asymmetry are accepted; the
    results match the oracle on the same inputs."""
    from paper_2410_00627_gb300 import api
    prob = synth.random_model(74, 3, 2, 4, 25)
    for k, v in GOOD[good](prob).items():
        setattr(prob, k, v)
    sm, fi = run_smoother(prob, "fp64")
    api.status()
    ref_sm, ref_fi = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    if good not in FILTER_ONLY:
        compare(sm, ref_sm, *TOL["fp64"], label=good)
    compare(fi, ref_fi, *TOL["fp64"], label=good)


def test_one_bad_sequence_in_a_batch_is_reported():
    import torch

    from paper_2410_00627_gb300 import api
    probs = [synth.random_model(75 + i, 3, 2, 3, 10 + i) for i in range(5)]
    probs[3].Q = _indefinite_q(3)
    pk = synth.pack(probs)
    t = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    b = api.make_batch(t(pk["F"]), t(pk["Q"]), t(pk["H"]), t(pk["R"]), t(pk["m0"]), t(pk["P0"]), t(pk["y"]),
                       t(pk["ratio"]), t(pk["n_slow"]), pk["max_ratio"], pk["total_slow"], pk["total_fast"])
    api.smoother_batch(b, precision="mixed")
    with pytest.raises(api.SRTMError) as err:
        api.status()
    assert err.value.code == -2
    api.status()
