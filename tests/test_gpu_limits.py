"""GPU parity at limits of the model: measurements that carry no information
(R = 10^14 I, the smoother returns the prior marginals), and the same model in
non-orthogonal state and measurement coordinates (every mean maps to T m,
every covariance to T P T^T).  The CUDA path through the C-ABI against the
FP64 oracle on the same inputs, at the tolerances of the other parity tests."""
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


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", [(86, 4, 2, 20, 90, 0), (87, 3, 1, 6, 70, 2)], ids=["n4m2", "n3m1u2"])
def test_uninformative_measurements(oracle_mod, case, precision):
    seed, nx, ny, l, N, nu = case
    prob = synth.random_model(seed, nx, ny, l, N, nu=nu)
    prob.R = 1e14 * np.eye(ny)
    ref_sm, ref_fi = oracle_views(oracle_mod.sequential(prob), l)
    sm, fi = run_smoother(prob, precision)
    compare(sm, ref_sm, *TOL[precision], label=f"smoothed {precision}")
    compare(fi, ref_fi, *TOL[precision], label=f"filtered {precision}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_change_of_coordinates(oracle_mod, precision):
    prob = synth.random_model(88, 4, 2, 8, 120)
    rng = np.random.default_rng(88)
    T = np.eye(4) + 0.6 * rng.standard_normal((4, 4))
    S = np.eye(2) + 0.6 * rng.standard_normal((2, 2))
    Ti = np.linalg.inv(T)
    prob.F, prob.Q, prob.H = T @ prob.F @ Ti, T @ prob.Q @ T.T, S @ prob.H @ Ti
    prob.R, prob.m0, prob.P0, prob.y = S @ prob.R @ S.T, T @ prob.m0, T @ prob.P0 @ T.T, prob.y @ S.T
    ref_sm, ref_fi = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    sm, fi = run_smoother(prob, precision)
    compare(sm, ref_sm, *TOL[precision], label=f"smoothed {precision}")
    compare(fi, ref_fi, *TOL[precision], label=f"filtered {precision}")
