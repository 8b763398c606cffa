"""Failure detection on the GPU without a fault: a bounded device-side wait on
a flag that nothing sets gives up, latches the timeout, and the host reads it
through srtm_status; the context stays usable for the next call."""
import time

import numpy as np
import pytest

from paper_2410_00627_gb300 import synth
from tests.gpu_util import TOL, compare, oracle_views, run_smoother

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
