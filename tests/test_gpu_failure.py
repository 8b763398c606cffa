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
