"""The single-sequence workloads at their full sizes (network8: 10^5 slow /
5*10^6 fast steps, nx = 8; stiff_chain6: l = 100, 10^6 fast steps): every
slow-rate output and the fast-rate outputs of the first and last three
intervals against the FP64 oracle.  FP64 and mixed are gated at the stated
tolerances; the pure-FP32 mode is reported, not gated."""
import pytest

from tests.gpu_util import TOL

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["ab_kinetics", "chain4", "network8", "stiff_chain6"])
def test_full_size_errors_within_tolerance(name):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import bench
    rep = bench.report_errors(name)
    print(rep)
    for prec in ("fp64", "mixed"):
        tm, tc = TOL[prec]
        for key, e in rep["errors"][prec].items():
            tol = tm if "mean" in key else tc
            assert e <= tol, f"{name} {prec} {key}: {e:.3e} > {tol:.0e}"
    assert "fp32" in rep["errors"]  # reported, not gated
