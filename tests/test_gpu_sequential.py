"""GPU parity of the sequential forms (srtm_*_sequential: the IMKF of
Eq. 9-12 walked forward and the IMS recursion of Eq. 21-22 walked backward,
one thread per sequence) against the FP64 oracle, element by element, and
against the scan path.  Tolerances are those of the scan path's tests."""
import numpy as np
import pytest

from paper_2410_00627_gb300 import synth
from tests.gpu_util import TOL, compare, controls, oracle_views, to_dev

pytestmark = pytest.mark.gpu

ARGS = ("F", "Q", "H", "R", "m0", "P0", "y")


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00627_gb300 import api, build
    build.build()
    api.load()


CASES = [  # (seed, nx, ny, ratio, n_slow, nu)
    (51, 1, 1, 3, 70, 0),
    (52, 2, 1, 1, 300, 0),
    (53, 3, 2, 4, 97, 1),
    (54, 4, 2, 20, 161, 0),
    (55, 4, 4, 7, 65, 2),
    (56, 5, 3, 6, 50, 0),
    (57, 6, 2, 100, 20, 3),
    (58, 7, 1, 3, 33, 0),
    (59, 8, 3, 4, 67, 4),
    (60, 2, 2, 2, 1, 0),
    (63, 8, 4, 3, 30, 2),
]


def _run(prob, precision, method, filtered=True):
    from paper_2410_00627_gb300 import api
    args = [to_dev(getattr(prob, k)) for k in ARGS]
    sm, fi = api.smoother(*args, prob.ratio, precision=precision, outputs=api.ALL_OUTPUTS,
                          filtered=api.OUTPUT_KEYS if filtered else (), method=method, **controls(prob))
    api.status()
    return ({k: v.cpu().numpy() for k, v in sm.items()}, {k: v.cpu().numpy() for k, v in fi.items()})


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n{1}m{2}l{3}N{4}u{5}".format(*c))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_sequential_smoother_matches_oracle(oracle_mod, case, precision):
    seed, nx, ny, l, N, nu = case
    prob = synth.random_model(seed, nx, ny, l, N, nu=nu)
    ref_sm, ref_fi = oracle_views(oracle_mod.sequential(prob), l)
    sm, fi = _run(prob, precision, "sequential")
    tm, tc = TOL[precision]
    compare(sm, ref_sm, tm, tc, f"smoothed {precision}")
    compare(fi, ref_fi, tm, tc, f"filtered {precision}")
    want = oracle_mod.loglik(prob)
    tol = 1e-9 if precision == "fp64" else 1e-4
    assert abs(sm["loglik"][0] - want) <= tol * max(1.0, abs(want))


def test_sequential_and_scan_agree_to_rounding():
    prob = synth.chain4(seed=3, n_slow=2000, keep_states=False)
    seq, _ = _run(prob, "fp64", "sequential", filtered=False)
    scan, _ = _run(prob, "fp64", "scan", filtered=False)
    compare(seq, scan, 1e-12, 1e-11, "sequential vs scan")


def test_sequential_filter_call(oracle_mod):
    from paper_2410_00627_gb300 import api
    prob = synth.random_model(61, 4, 2, 10, 140, nu=2)
    _, ref_fi = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    args = [to_dev(getattr(prob, k)) for k in ARGS]
    out = api.filter(*args, prob.ratio, method="sequential", **controls(prob))
    api.status()
    # constants, input terms, sequential filter, interval setup, recovery
    assert api.last_call_launches() == 5
    compare({k: v.cpu().numpy() for k, v in out.items()}, ref_fi, *TOL["fp64"], label="sequential filter")


def test_sequential_ragged_batch_matches_per_sequence_oracle(oracle_mod):
    import torch

    from paper_2410_00627_gb300 import api
    probs = synth.ragged_chains(seed=12, n_seq=150, n_min=1, n_max=150)
    pk = synth.pack(probs)
    t = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    b = api.make_batch(t(pk["F"]), t(pk["Q"]), t(pk["H"]), t(pk["R"]), t(pk["m0"]), t(pk["P0"]), t(pk["y"]),
                       t(pk["ratio"]), t(pk["n_slow"]), pk["max_ratio"], pk["total_slow"], pk["total_fast"])
    for precision in ("fp64", "mixed"):
        sm, fi = api.smoother_batch(b, precision=precision, outputs=api.ALL_OUTPUTS, filtered=api.OUTPUT_KEYS,
                                    method="sequential")
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
            assert abs(sm["loglik"][s] - want) <= tol * max(1.0, abs(want))
            fo += N * l
            so += N


def test_unknown_method_rejected():
    from paper_2410_00627_gb300 import api
    prob = synth.random_model(62, 2, 1, 2, 4)
    args = [to_dev(getattr(prob, k)) for k in ARGS]
    with pytest.raises(ValueError):
        api.smoother(*args, prob.ratio, method="parallel-ish")
