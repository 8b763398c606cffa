"""The allocation-free smoother entry point, srtm_smoother_noalloc.

It serves callers that must not allocate GPU memory (their memory is owned by
another allocator, or they cannot afford the device-wide synchronisation of
cudaMalloc/cudaFree): the same device path runs with its scratch in a static
device array.  This file is collected last so that a run stopping at the
first failure has already run every other test; it also passes on its own in
a fresh process.
"""
import ctypes

import numpy as np
import pytest

from paper_2410_00627_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00627_gb300 import api, build
    build.build()
    return api.load()


def _device_problem(prob):
    import torch

    from paper_2410_00627_gb300 import api
    ts = {k: torch.as_tensor(np.ascontiguousarray(getattr(prob, k)), dtype=torch.float64, device="cuda")
          for k in ("F", "Q", "H", "R", "m0", "P0", "y")}
    p = api.Problem(prob.nx, prob.ny, prob.ratio, prob.n_slow,
                    *[ctypes.c_void_p(ts[k].data_ptr()) for k in ("F", "Q", "H", "R", "m0", "P0", "y")])
    return p, ts


def _outputs(prob):
    import torch

    from paper_2410_00627_gb300 import api
    nf, ns, n = prob.n_slow * prob.ratio, prob.n_slow, prob.nx
    o = {"fast_mean": torch.full((nf, n), np.nan, dtype=torch.float64, device="cuda"),
         "fast_cov": torch.full((nf, n, n), np.nan, dtype=torch.float64, device="cuda"),
         "slow_mean": torch.full((ns, n), np.nan, dtype=torch.float64, device="cuda"),
         "slow_cov": torch.full((ns, n, n), np.nan, dtype=torch.float64, device="cuda")}
    return o, api.Output(*[ctypes.c_void_p(o[k].data_ptr()) for k in api.OUTPUT_KEYS])


@pytest.mark.parametrize("precision,tol", [(0, (1e-9, 1e-8)), (1, (1e-4, 1e-3))])
def test_noalloc_matches_smoother_on_two_calls(lib, precision, tol):
    import torch

    from paper_2410_00627_gb300 import api
    prob = synth.chain4(seed=31, n_slow=700, keep_states=False)
    p, _keep = _device_problem(prob)
    ref, ref_o = _outputs(prob)
    assert lib.srtm_smoother(ctypes.byref(p), precision, ctypes.byref(ref_o), None, None) == 0
    assert lib.srtm_status(None) == 0
    for _ in range(2):  # the static scratch keeps the previous call's contents
        got, got_o = _outputs(prob)
        rc = lib.srtm_smoother_noalloc(ctypes.byref(p), precision, ctypes.byref(got_o), None)
        assert rc == 0, api.last_error_detail()
        torch.cuda.synchronize()
        for k in api.OUTPUT_KEYS:
            a, b = got[k].cpu().numpy(), ref[k].cpu().numpy()
            err = np.max(np.abs(a - b)) / np.max(np.abs(b))
            assert err <= (tol[0] if k.endswith("mean") else tol[1]), (k, err)


def test_noalloc_rejects_problems_beyond_its_scratch(lib):
    from paper_2410_00627_gb300 import api
    prob = synth.chain4(seed=32, n_slow=60_000, keep_states=False)
    p, _keep = _device_problem(prob)
    out = api.Output(None, None, None, None)
    assert lib.srtm_smoother_noalloc(ctypes.byref(p), 0, ctypes.byref(out), None) == -1
    assert "static scratch holds" in api.last_error_detail()
