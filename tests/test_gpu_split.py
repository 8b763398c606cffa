"""GPU parity of one sequence split over several ranges (the cross-GPU
decomposition of the filter and smoother scans, Sec. II associativity of
Eq. 27 and Eq. 30): every range's smoothed and filtered outputs, fast and
slow, and the log likelihood, against the FP64 oracle of the whole sequence.

The ranges run on one GPU: one after another in one process (each phase for
every range before the next phase, as the ranks would), and as two processes
exchanging the aggregates over gloo with both processes on cuda:0 (their
kernels never wait on one another: the exchange is on the host between
launches).  Tolerances are those of the other parity tests."""
import os
import socket

import numpy as np
import pytest

from paper_2410_00627_gb300 import synth
from tests.gpu_util import TOL, compare, oracle_views, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00627_gb300 import api, build
    build.build()
    api.load()


def _model(prob):
    return [to_dev(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0")]


def _check_ranges(oracle_mod, prob, res, parts, precision, label, filtered=True):
    from paper_2410_00627_gb300 import split
    l = prob.ratio
    ref_sm, ref_fi = oracle_views(oracle_mod.sequential(prob), l)
    for r, (lo, hi) in enumerate(split.ranges(prob.n_slow, parts)):
        sm, fi = ({k: v.cpu().numpy() for k, v in d.items()} for d in res[r])
        cut = {k: (v[lo * l:hi * l] if k.startswith("fast") else v[lo:hi]) for k, v in ref_sm.items()}
        compare(sm, cut, *TOL[precision], label=f"{label} range {r} smoothed")
        if filtered:
            cut = {k: (v[lo * l:hi * l] if k.startswith("fast") else v[lo:hi]) for k, v in ref_fi.items()}
            compare(fi, cut, *TOL[precision], label=f"{label} range {r} filtered")
    # the ranges' shares of log p(y_1:N) add up to the sequence's
    if "loglik" in res[0][0]:
        tot = sum(float(res[r][0]["loglik"].cpu().numpy()[0]) for r in range(parts))
        want = oracle_mod.loglik(prob)
        tol = 1e-9 if precision == "fp64" else 1e-4
        assert abs(tot - want) <= tol * max(1.0, abs(want)), (label, tot, want)


CASES = [  # (seed, nx, ny, ratio, n_slow, parts)
    (1, 2, 1, 5, 40, 2), (2, 4, 2, 3, 300, 3), (3, 3, 1, 1, 130, 4), (4, 8, 3, 4, 90, 2), (5, 5, 2, 7, 61, 5),
    (6, 4, 1, 6, 8, 8)]


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: f"nx{c[1]}ny{c[2]}l{c[3]}N{c[4]}p{c[5]}")
def test_split_sequence_matches_oracle(oracle_mod, case, precision):
    from paper_2410_00627_gb300 import api, split
    seed, nx, ny, ratio, n_slow, parts = case
    prob = synth.random_model(seed, nx, ny, ratio, n_slow)
    res = split.smoother_split_serial(*_model(prob), to_dev(prob.y), ratio, parts, precision,
                                      outputs=api.ALL_OUTPUTS, filtered=api.OUTPUT_KEYS)
    api.status()
    _check_ranges(oracle_mod, prob, res, parts, precision, f"split {prob.name}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_network8_split_over_four_ranges(oracle_mod, precision):
    """network8's model (nx=8, ny=3, l=50) over 4 ranges of 400 slow steps:
    many scan tiles per range."""
    from paper_2410_00627_gb300 import api, split
    prob = synth.network8(seed=3, n_slow=400)
    res = split.smoother_split_serial(*_model(prob), to_dev(prob.y), prob.ratio, 4, precision,
                                      filtered=api.OUTPUT_KEYS)
    api.status()
    _check_ranges(oracle_mod, prob, res, 4, precision, "network8")


def test_one_range_is_the_whole_sequence(oracle_mod):
    """parts = 1: the first range is also the last (no exchange)."""
    from paper_2410_00627_gb300 import api, split
    prob = synth.chain4(seed=4, n_slow=150)
    res = split.smoother_split_serial(*_model(prob), to_dev(prob.y), prob.ratio, 1, "fp64", filtered=api.OUTPUT_KEYS)
    api.status()
    _check_ranges(oracle_mod, prob, res, 1, "fp64", "one range")


def test_split_combine_is_the_operator_product(oracle_mod):
    """srtm_split_combine against the oracle's operators (Eq. 27, Eq. 30) on
    random elements, folded left to right."""
    import torch

    from paper_2410_00627_gb300 import api
    rng = np.random.default_rng(5)
    for nx in (1, 3, 4, 6, 8):
        def spd():
            a = rng.standard_normal((nx, nx))
            return a @ a.T / nx + 0.1 * np.eye(nx)
        fe = [{"F": 0.5 * rng.standard_normal((nx, nx)), "d": rng.standard_normal(nx), "D": spd(),
               "eta": rng.standard_normal(nx), "J": spd()} for _ in range(4)]
        flat = np.stack([np.concatenate([e["F"].ravel(), e["d"], e["D"].ravel(), e["eta"], e["J"].ravel()])
                         for e in fe])
        got = api.split_combine("filter", torch.as_tensor(flat, device="cuda")).cpu().numpy()
        want = fe[0]
        for e in fe[1:]:
            want = oracle_mod.filter_op(want, e)
        w = np.concatenate([want["F"].ravel(), want["d"], want["D"].ravel(), want["eta"], want["J"].ravel()])
        assert np.max(np.abs(got - w)) <= 1e-12 * max(1.0, np.max(np.abs(w))), nx
        se = [{"E": 0.5 * rng.standard_normal((nx, nx)), "g": rng.standard_normal(nx), "S": spd()} for _ in range(3)]
        flat = np.stack([np.concatenate([e["E"].ravel(), e["g"], e["S"].ravel()]) for e in se])
        got = api.split_combine("smoother", torch.as_tensor(flat, device="cuda")).cpu().numpy()
        want = se[0]
        for e in se[1:]:
            want = oracle_mod.smoother_op(want, e)
        w = np.concatenate([want["E"].ravel(), want["g"], want["S"].ravel()])
        assert np.max(np.abs(got - w)) <= 1e-12 * max(1.0, np.max(np.abs(w))), nx
    api.status()


def test_split_rejects_inputs_and_bad_arguments():
    import ctypes

    import torch

    from paper_2410_00627_gb300 import api
    lib = api.load()
    prob = synth.random_model(7, 3, 1, 2, 10, nu=1)
    args = _model(prob)
    y = to_dev(prob.y)
    with pytest.raises(api.SRTMError, match="UNSUPPORTED"):
        p = api._problem(*args, y, prob.ratio, to_dev(prob.B), to_dev(prob.u))
        agg = torch.empty(api.filter_element_size(3), dtype=torch.float64, device="cuda")
        api._check(lib.srtm_split_filter_aggregate(ctypes.byref(p), 1, 0, ctypes.c_void_p(agg.data_ptr()), None))
    nm = torch.zeros(3, dtype=torch.float64, device="cuda")
    p = api._problem(*args, y, prob.ratio)
    assert lib.srtm_split_smoother(ctypes.byref(p), ctypes.c_void_p(nm.data_ptr()), None, 0, None, None, None) == -1
    host = np.zeros(api.filter_element_size(3))
    assert lib.srtm_split_filter_aggregate(ctypes.byref(p), 1, 0, ctypes.c_void_p(host.ctypes.data), None) == -1
    assert lib.srtm_split_combine(2, 3, None, 1, None, None) == -1
    assert lib.srtm_split_combine(0, 9, None, 1, None, None) == -6


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys

    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_2410_00627_gb300 import api, split
    from paper_2410_00627_gb300 import synth as sy
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        torch.cuda.set_device(0)
        api.load()
        prob = sy.chain4(seed=8, n_slow=240)
        lo, hi = split.ranges(prob.n_slow, world)[rank]
        dev = lambda a: torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")  # noqa: E731
        model = [dev(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0")]
        sm, fi = split.smoother_split(*model, dev(prob.y[lo:hi]), prob.ratio, "fp64", outputs=api.ALL_OUTPUTS,
                                      filtered=api.OUTPUT_KEYS)
        api.status()
        q.put((rank, {k: v.cpu().numpy() for k, v in sm.items()}, {k: v.cpu().numpy() for k, v in fi.items()}))
    finally:
        dist.destroy_process_group()


def test_two_processes_exchange_aggregates_over_gloo(oracle_mod):
    """smoother_split on two processes (gloo all-gathers), both on cuda:0."""
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        r, sm, fi = q.get(timeout=300)
        got[r] = (sm, fi)
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    prob = synth.chain4(seed=8, n_slow=240)

    class _T:  # numpy results in the shape _check_ranges expects
        def __init__(self, a):
            self.a = a

        def cpu(self):
            return self

        def numpy(self):
            return self.a
    res = [({k: _T(v) for k, v in got[r][0].items()}, {k: _T(v) for k, v in got[r][1].items()}) for r in range(2)]
    _check_ranges(oracle_mod, prob, res, 2, "fp64", "gloo")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_chain4_split_boundaries(oracle_mod, precision):
    """chain4 at 10^4 slow steps over 4 ranges (many scan tiles per range): the
    fast outputs of the two intervals on each side of every range boundary,
    the sequence's first and last intervals, and every smoothed x_{k,1},
    against the oracle of the whole sequence."""
    from paper_2410_00627_gb300 import api, split
    prob = synth.chain4(seed=9, n_slow=10_000, keep_states=False)
    l, N = prob.ratio, prob.n_slow
    parts = 4
    res = split.smoother_split_serial(*_model(prob), to_dev(prob.y), l, parts, precision,
                                      filtered=api.OUTPUT_KEYS)
    api.status()
    rg = split.ranges(N, parts)
    sm = {k: np.concatenate([res[r][0][k].cpu().numpy() for r in range(parts)]) for k in api.OUTPUT_KEYS}
    fi = {k: np.concatenate([res[r][1][k].cpu().numpy() for r in range(parts)]) for k in api.OUTPUT_KEYS}
    tm, tc = TOL[precision]
    windows = [(0, 2), (N - 2, N)] + [(hi - 2, hi + 2) for _, hi in rg[:-1]]
    for k0, k1 in windows:
        o = oracle_mod.sequential(prob, k_lo=k0, k_hi=k1, slow=False)
        sl = slice(k0 * l, k1 * l)
        compare({"fast_mean": sm["fast_mean"][sl], "fast_cov": sm["fast_cov"][sl]},
                {"fast_mean": o["fast_smooth_mean"], "fast_cov": o["fast_smooth_cov"]}, tm, tc, f"smoothed {k0}")
        compare({"fast_mean": fi["fast_mean"][sl], "fast_cov": fi["fast_cov"][sl]},
                {"fast_mean": o["fast_filt_mean"], "fast_cov": o["fast_filt_cov"]}, tm, tc, f"filtered {k0}")
    seq = oracle_mod.sequential(prob, fast=False)
    compare({"first_mean": sm["fast_mean"][0::l], "first_cov": sm["fast_cov"][0::l]},
            {"first_mean": seq["first_smooth_mean"], "first_cov": seq["first_smooth_cov"]}, tm, tc, "x_(k,1)")
    compare({"slow_mean": fi["slow_mean"], "slow_cov": fi["slow_cov"]},
            {"slow_mean": seq["slow_filt_mean"], "slow_cov": seq["slow_filt_cov"]}, tm, tc, "filtered slow")
