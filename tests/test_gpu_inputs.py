"""GPU parity with known inputs, x_{t+1} = F x_t + B u_t + w_t (Sec. II):
the CUDA path through the C-ABI against the FP64 oracle, element by element.

The inputs enter the filter elements (b_{k,l} in d_k, c_k = H sum_i b_{k,i}
subtracted from y_k), the smoother's one-step prediction (B u_{k+1,0}), the
fast-rate recovery (b_{k,i}) and the log likelihood.  Cases span nx = 1..8,
nu = 1..4, several scan tiles with a ragged tail, a 100-step ratio, and a
ragged batch.  Tolerances are the ones of the input-free parity tests.
"""
import numpy as np
import pytest

from paper_2410_00627_gb300 import synth
from tests.gpu_util import TOL, compare, controls, oracle_views, run_filter, run_smoother, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00627_gb300 import api, build
    build.build()
    api.load()


CASES = [  # (seed, nx, ny, ratio, n_slow, nu)
    (21, 1, 1, 3, 70, 1),
    (22, 2, 1, 1, 300, 2),
    (23, 3, 2, 4, 97, 1),
    (24, 4, 2, 20, 161, 2),
    (25, 4, 1, 5, 2, 4),
    (26, 5, 3, 6, 50, 3),
    (27, 6, 2, 100, 20, 3),
    (28, 7, 1, 3, 33, 2),
    (29, 8, 3, 4, 67, 4),
    (30, 3, 3, 2, 1, 1),
    (36, 8, 4, 5, 30, 4),   # largest state, measurement and input sizes
]

ARGS = ("F", "Q", "H", "R", "m0", "P0", "y")


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n{1}m{2}l{3}N{4}u{5}".format(*c))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_smoother_with_inputs_matches_oracle(oracle_mod, case, precision):
    seed, nx, ny, l, N, nu = case
    prob = synth.random_model(seed, nx, ny, l, N, nu=nu)
    ref_sm, ref_fi = oracle_views(oracle_mod.sequential(prob), l)
    sm, fi = run_smoother(prob, precision)
    tm, tc = TOL[precision]
    compare(sm, ref_sm, tm, tc, f"smoothed {precision}")
    compare(fi, ref_fi, tm, tc, f"filtered {precision}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_filter_call_with_inputs_matches_oracle(oracle_mod, precision):
    from paper_2410_00627_gb300 import api
    prob = synth.random_model(31, 4, 2, 10, 140, nu=2)
    _, ref_fi = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    args = [to_dev(getattr(prob, k)) for k in ARGS]
    api.filter(*args, prob.ratio, precision=precision)
    plain_launches = api.last_call_launches()
    got = run_filter(prob, precision)
    assert api.last_call_launches() == plain_launches + 1  # the input-terms kernel
    compare(got, ref_fi, *TOL[precision], label=f"filter {precision}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_loglik_with_inputs_matches_oracle(oracle_mod, precision):
    from paper_2410_00627_gb300 import api
    for seed, nx, ny, l, N, nu in CASES[:6]:
        prob = synth.random_model(seed, nx, ny, l, N, nu=nu)
        args = [to_dev(getattr(prob, k)) for k in ARGS]
        sm, _ = api.smoother(*args, l, precision=precision, outputs=("slow_mean", "loglik"), **controls(prob))
        api.status()
        want = oracle_mod.loglik(prob)
        got = float(sm["loglik"].cpu().item())
        tol = 1e-9 if precision == "fp64" else 1e-4
        assert abs(got - want) <= tol * max(1.0, abs(want)), (prob.name, got, want)


def test_inputs_change_the_means_but_not_the_covariances(oracle_mod):
    """Known inputs shift every mean and leave every covariance as it is
    (the gains do not depend on u); zero inputs reproduce the input-free path."""
    from paper_2410_00627_gb300 import api
    prob = synth.random_model(32, 5, 2, 7, 90, nu=2)
    args = [to_dev(getattr(prob, k)) for k in ARGS]
    with_u, _ = api.smoother(*args, prob.ratio, **controls(prob))
    plain, _ = api.smoother(*args, prob.ratio)
    zero, _ = api.smoother(*args, prob.ratio, B=to_dev(prob.B), u=to_dev(np.zeros_like(prob.u)))
    api.status()
    w, p, z = ({k: v.cpu().numpy() for k, v in d.items()} for d in (with_u, plain, zero))
    assert np.max(np.abs(w["fast_mean"] - p["fast_mean"])) > 1e-3
    for k in ("fast_cov", "slow_cov"):
        assert np.max(np.abs(w[k] - p[k])) <= 1e-13 * np.max(np.abs(p[k])), k
    for k in p:
        assert np.max(np.abs(z[k] - p[k])) <= 1e-13 * np.max(np.abs(p[k])), k


def test_ragged_batch_with_inputs_matches_per_sequence_oracle(oracle_mod):
    import torch

    from paper_2410_00627_gb300 import api
    shapes = [(3, 40), (7, 1), (5, 90), (1, 55), (20, 12), (4, 3)]
    probs = [synth.random_model(40 + i, 4, 2, l, N, nu=3) for i, (l, N) in enumerate(shapes)]
    pk = synth.pack(probs)
    t = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    for precision in ("fp64", "mixed"):
        b = api.make_batch(t(pk["F"]), t(pk["Q"]), t(pk["H"]), t(pk["R"]), t(pk["m0"]), t(pk["P0"]), t(pk["y"]),
                           t(pk["ratio"]), t(pk["n_slow"]), pk["max_ratio"], pk["total_slow"], pk["total_fast"],
                           B=t(pk["B"]), u=t(pk["u"]))
        sm, fi = api.smoother_batch(b, precision=precision, outputs=api.ALL_OUTPUTS, filtered=api.OUTPUT_KEYS)
        api.status()
        sm = {k: v.cpu().numpy() for k, v in sm.items()}
        fi = {k: v.cpu().numpy() for k, v in fi.items()}
        fo = so = 0
        for s, p in enumerate(probs):
            l, N = p.ratio, p.n_slow
            ref_sm, ref_fi = oracle_views(oracle_mod.sequential(p), l)
            cut = lambda d: {"fast_mean": d["fast_mean"][fo:fo + N * l], "fast_cov": d["fast_cov"][fo:fo + N * l],  # noqa: E731
                             "slow_mean": d["slow_mean"][so:so + N], "slow_cov": d["slow_cov"][so:so + N]}
            compare(cut(sm), ref_sm, *TOL[precision], label=f"batch {p.name} {precision}")
            compare(cut(fi), ref_fi, *TOL[precision], label=f"batch {p.name} {precision}")
            want = oracle_mod.loglik(p)
            tol = 1e-9 if precision == "fp64" else 1e-4
            assert abs(sm["loglik"][s] - want) <= tol * max(1.0, abs(want)), (p.name, sm["loglik"][s], want)
            fo += N * l
            so += N


def test_long_sequence_with_inputs(oracle_mod):
    """3000 slow steps of a 4-state model at ratio 20 (many scan tiles)."""
    prob = synth.random_model(33, 4, 1, 20, 3000, nu=2)
    ref_sm, ref_fi = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    for precision in ("fp64", "mixed"):
        sm, fi = run_smoother(prob, precision)
        compare(sm, ref_sm, *TOL[precision], label=f"smoothed {precision}")
        compare(fi, ref_fi, *TOL[precision], label=f"filtered {precision}")


def test_host_entry_point_with_inputs(oracle_mod):
    from paper_2410_00627_gb300 import api
    prob = synth.random_model(34, 3, 2, 6, 80, nu=2)
    res = api.smoother_host(*[np.ascontiguousarray(getattr(prob, k)) for k in ARGS], prob.ratio,
                            precision="fp64", loglik=True, B=np.ascontiguousarray(prob.B),
                            u=np.ascontiguousarray(prob.u))
    ref_sm, _ = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    compare({k: res[k] for k in ref_sm}, ref_sm, *TOL["fp64"], label="host entry")
    want = oracle_mod.loglik(prob)
    assert abs(res["loglik"][0] - want) <= 1e-9 * abs(want)


def test_too_many_inputs_rejected():
    from paper_2410_00627_gb300 import api
    prob = synth.random_model(35, 3, 1, 2, 5, nu=1)
    args = [to_dev(getattr(prob, k)) for k in ARGS]
    B = to_dev(np.ones((3, 5)))
    u = to_dev(np.ones((10, 5)))
    with pytest.raises(api.SRTMError):
        api.smoother(*args, prob.ratio, B=B, u=u)
    api.status()
