"""GPU parity: the CUDA path (through the C-ABI) against the FP64 oracle.

Small cases compare every output element by element; they span several scan
tiles with a ragged tail (scan tiles hold 16-128 slow steps depending on nx).
Full-size cases (chain4 at 10^4 slow steps, the benchmark's workload and
launch configuration) compare sampled windows of fast outputs plus every
slow output against the oracle.  Tolerances: FP64 1e-9 (means) / 1e-8
(covariances, relative to max |P|); mixed 1e-4 / 1e-3.
"""
import numpy as np
import pytest

from paper_2410_00627_gb300 import synth
from tests.gpu_util import TOL, assert_same_to_rounding, compare, oracle_views, run_filter, run_smoother, to_dev

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00627_gb300 import api, build
    build.build()
    api.load()


CASES = [  # (seed, nx, ny, ratio, n_slow)
    (1, 1, 1, 3, 70),
    (2, 2, 1, 1, 300),
    (3, 3, 2, 4, 97),
    (4, 4, 2, 20, 161),
    (5, 4, 4, 7, 65),
    (6, 5, 3, 6, 50),
    (7, 6, 2, 5, 49),
    (8, 7, 1, 3, 33),
    (9, 8, 3, 4, 67),
    (10, 2, 2, 2, 1),
    (11, 4, 1, 5, 2),
    (12, 3, 3, 1, 17),
    (13, 8, 4, 3, 40),     # largest state and measurement sizes
    (14, 7, 4, 1, 25),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n{1}m{2}l{3}N{4}".format(*c))
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_smoother_matches_oracle(oracle_mod, case, precision):
    seed, nx, ny, l, N = case
    prob = synth.random_model(seed, nx, ny, l, N)
    ref_sm, ref_fi = oracle_views(oracle_mod.sequential(prob), l)
    sm, fi = run_smoother(prob, precision)
    tm, tc = TOL[precision]
    compare(sm, ref_sm, tm, tc, f"smoothed {precision}")
    compare(fi, ref_fi, tm, tc, f"filtered {precision}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("name,n_slow", [("ab_kinetics", 100), ("chain4", 257), ("stiff_chain6", 40)])
def test_workloads_small_match_oracle(oracle_mod, name, n_slow, precision):
    prob = synth.WORKLOADS[name](seed=11, n_slow=n_slow, keep_states=False)
    ref_sm, ref_fi = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    sm, fi = run_smoother(prob, precision)
    tm, tc = TOL[precision]
    compare(sm, ref_sm, tm, tc, f"{name} smoothed {precision}")
    compare(fi, ref_fi, tm, tc, f"{name} filtered {precision}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_filter_call_matches_oracle(oracle_mod, precision):
    prob = synth.random_model(21, 4, 2, 6, 131)
    o = oracle_mod.sequential(prob, smooth=False)
    out = run_filter(prob, precision)
    from paper_2410_00627_gb300 import api
    assert api.last_call_launches() == 3   # constants, filter scan, recovery
    l = prob.ratio
    ref = {"fast_mean": o["fast_filt_mean"], "fast_cov": o["fast_filt_cov"],
           "slow_mean": o["slow_filt_mean"], "slow_cov": o["slow_filt_cov"]}
    compare(out, ref, *TOL[precision], label=f"filter {precision}")
    assert np.array_equal(out["slow_mean"], out["fast_mean"][l - 1::l])


def test_fp32_mode_runs_and_is_close(oracle_mod):
    prob = synth.chain4(seed=2, n_slow=120, keep_states=False)
    ref_sm, _ = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    sm, _ = run_smoother(prob, "fp32", filtered=False)
    errs = compare(sm, ref_sm, 1e-2, 1e-1, "fp32")
    assert all(np.isfinite(v) for v in errs.values())


def test_outputs_exactly_symmetric_and_last_interval(oracle_mod):
    prob = synth.chain4(seed=3, n_slow=50, keep_states=False)
    sm, fi = run_smoother(prob, "fp64")
    P = sm["fast_cov"]
    assert np.array_equal(P, np.swapaxes(P, 1, 2))
    l = prob.ratio
    assert np.array_equal(sm["fast_mean"][-l:], fi["fast_mean"][-l:])
    assert np.array_equal(sm["fast_cov"][-l:], fi["fast_cov"][-l:])


def test_repeated_calls_agree_to_rounding():
    prob = synth.chain4(seed=4, n_slow=3000, keep_states=False)
    for precision in ("fp64", "mixed"):
        a, _ = run_smoother(prob, precision, filtered=False)
        b, _ = run_smoother(prob, precision, filtered=False)
        for k in a:
            assert_same_to_rounding(a[k], b[k], precision, k)


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_full_size_chain4_sampled(oracle_mod, precision):
    """chain4 at its full size (10^4 slow steps, 2*10^5 fast steps) in the
    benchmark's launch configuration (shapes chosen by the autotuner): every
    slow output, and fast outputs of sampled windows (start, two interior
    windows, end)."""
    from paper_2410_00627_gb300 import api
    prob = synth.chain4(seed=0, n_slow=10_000, keep_states=False)
    l, N = prob.ratio, prob.n_slow
    args = [to_dev(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    try:
        api.autotune(*args, l, precision=precision, reps=1)   # the benchmark's shapes
        sm, fi = run_smoother(prob, precision)
    finally:
        api.set_tuning(4, precision)
    seq = oracle_mod.sequential(prob, fast=False)
    tm, tc = TOL[precision]
    windows = [(0, 3), (4093, 4099), (7770, 7772), (N - 3, N)]
    for k0, k1 in windows:
        o = oracle_mod.sequential(prob, k_lo=k0, k_hi=k1, slow=False)
        sl = slice(k0 * l, k1 * l)
        compare({"fast_mean": sm["fast_mean"][sl], "fast_cov": sm["fast_cov"][sl]},
                {"fast_mean": o["fast_smooth_mean"], "fast_cov": o["fast_smooth_cov"]}, tm, tc, f"window {k0}")
        compare({"fast_mean": fi["fast_mean"][sl], "fast_cov": fi["fast_cov"][sl]},
                {"fast_mean": o["fast_filt_mean"], "fast_cov": o["fast_filt_cov"]}, tm, tc, f"window {k0}")
    compare({"slow_mean": fi["slow_mean"], "slow_cov": fi["slow_cov"]},
            {"slow_mean": seq["slow_filt_mean"], "slow_cov": seq["slow_filt_cov"]}, tm, tc, "slow filtered")
    compare({"first_mean": sm["fast_mean"][0::l], "first_cov": sm["fast_cov"][0::l]},
            {"first_mean": seq["first_smooth_mean"], "first_cov": seq["first_smooth_cov"]}, tm, tc, "first smoothed")


def test_ragged_batch_matches_per_sequence_oracle(oracle_mod):
    import torch

    from paper_2410_00627_gb300 import api
    from tests.gpu_util import to_dev
    probs = synth.ragged_chains(seed=5, n_seq=9, n_min=1, n_max=120)
    probs[3] = synth.ragged_chains(seed=6, n_seq=1, n_min=1, n_max=1)[0]   # a length-1 sequence
    S = len(probs)
    stack = lambda k: to_dev(np.stack([getattr(p, k) for p in probs]))  # noqa: E731
    y = to_dev(np.concatenate([p.y for p in probs]))
    ratio = torch.tensor([p.ratio for p in probs], dtype=torch.int32, device="cuda")
    n_slow = torch.tensor([p.n_slow for p in probs], dtype=torch.int32, device="cuda")
    tot_s = sum(p.n_slow for p in probs)
    tot_f = sum(p.n_slow * p.ratio for p in probs)
    for precision in ("fp64", "mixed"):
        b = api.make_batch(stack("F"), stack("Q"), stack("H"), stack("R"), stack("m0"), stack("P0"), y,
                           ratio, n_slow, max(p.ratio for p in probs), tot_s, tot_f)
        sm, fi = api.smoother_batch(b, precision=precision, filtered=api.OUTPUT_KEYS)
        api.status()
        sm = {k: v.cpu().numpy() for k, v in sm.items()}
        fi = {k: v.cpu().numpy() for k, v in fi.items()}
        fo = so = 0
        for p in probs:
            l, N = p.ratio, p.n_slow
            ref_sm, ref_fi = oracle_views(oracle_mod.sequential(p), l)
            got_sm = {"fast_mean": sm["fast_mean"][fo:fo + N * l], "fast_cov": sm["fast_cov"][fo:fo + N * l],
                      "slow_mean": sm["slow_mean"][so:so + N], "slow_cov": sm["slow_cov"][so:so + N]}
            got_fi = {"fast_mean": fi["fast_mean"][fo:fo + N * l], "fast_cov": fi["fast_cov"][fo:fo + N * l],
                      "slow_mean": fi["slow_mean"][so:so + N], "slow_cov": fi["slow_cov"][so:so + N]}
            compare(got_sm, ref_sm, *TOL[precision], label=f"batch {p.name} {precision}")
            compare(got_fi, ref_fi, *TOL[precision], label=f"batch {p.name} {precision}")
            fo += N * l
            so += N


def test_batch_metadata_mismatch_is_reported_not_computed():
    import torch

    from paper_2410_00627_gb300 import api
    from tests.gpu_util import to_dev
    probs = synth.ragged_chains(seed=7, n_seq=3, n_min=5, n_max=9)
    stack = lambda k: to_dev(np.stack([getattr(p, k) for p in probs]))  # noqa: E731
    y = to_dev(np.concatenate([p.y for p in probs]))
    ratio = torch.tensor([p.ratio for p in probs], dtype=torch.int32, device="cuda")
    n_slow = torch.tensor([p.n_slow for p in probs], dtype=torch.int32, device="cuda")
    tot_s = sum(p.n_slow for p in probs)
    tot_f = sum(p.n_slow * p.ratio for p in probs)
    # declared total_fast one row short of the metadata: rejected on the device
    b = api.make_batch(stack("F"), stack("Q"), stack("H"), stack("R"), stack("m0"), stack("P0"), y,
                       ratio, n_slow, 20, tot_s, tot_f - 1)
    api.smoother_batch(b, precision="fp64")
    with pytest.raises(api.SRTMError) as ei:
        api.status()
    assert ei.value.code == -7
    # a ratio above the declared max_ratio is rejected the same way
    b = api.make_batch(stack("F"), stack("Q"), stack("H"), stack("R"), stack("m0"), stack("P0"), y,
                       ratio, n_slow, 4, tot_s, tot_f)
    api.smoother_batch(b, precision="fp64")
    with pytest.raises(api.SRTMError):
        api.status()
    api.status()  # latch cleared


def test_host_pointer_rejected():
    import ctypes

    from paper_2410_00627_gb300 import api
    prob = synth.random_model(1, 2, 1, 2, 3)
    F = np.ascontiguousarray(prob.F)
    p = api.Problem(2, 1, 2, 3, *[ctypes.c_void_p(np.ascontiguousarray(getattr(prob, k)).ctypes.data)
                                  for k in ("F", "Q", "H", "R", "m0", "P0", "y")])
    assert F.size == 4
    out = api.Output(None, None, None, None)
    assert api.load().srtm_smoother(ctypes.byref(p), 0, ctypes.byref(out), None, None) == -1
    assert "not a device pointer" in api.last_error_detail()


def test_host_entry_point_matches_device_entry_point():
    from paper_2410_00627_gb300 import api
    prob = synth.chain4(seed=8, n_slow=200, keep_states=False)
    dev, _ = run_smoother(prob, "mixed", filtered=False)
    host = api.smoother_host(*[np.ascontiguousarray(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")],
                             prob.ratio, precision="mixed")
    for k in dev:
        assert_same_to_rounding(host[k], dev[k], "fp64", k)


def test_stage_timing_reports_every_stage():
    from paper_2410_00627_gb300 import api
    prob = synth.chain4(seed=9, n_slow=500, keep_states=False)
    api.set_stage_timing(True)
    times = {}
    try:
        for split in (1, 2):   # (the record form: the two-point form has no filtered half)
            api.set_tuning(4, "fp64", recover_split=split, recover_form=1)
            run_smoother(prob, "fp64", filtered=False)
            times[split] = api.stage_times()
    finally:
        api.set_stage_timing(False)
        api.set_tuning(4, "fp64")
    for split, t in times.items():
        assert set(t) == set(api.STAGES)
        assert all(v > 0 for k, v in t.items() if k != "recovery_filtered_half"), (split, t)
    assert times[1]["recovery_filtered_half"] == 0.0
    assert times[2]["recovery_filtered_half"] > 0.0


SHAPES = [  # (scan_groups, scan_elems, recover_threads, lookback_window, setup_mode, recover_split), nx=4
    (2, 1, 32, 1, 1, 1),      # smallest tiles, serial look-back
    (16, 32, 128, 32, 2, 2),  # largest tiles and window, setup as its own kernel, split recovery
    (8, 4, 64, 4, 2, 1),
    (4, 2, 96, 2, 1, 2),
]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "g{}e{}t{}w{}s{}r{}".format(*s))
def test_launch_shapes_do_not_change_results(oracle_mod, shape):
    from paper_2410_00627_gb300 import api
    prob = synth.chain4(seed=5, n_slow=613, keep_states=False)
    ref_sm, ref_fi = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    try:
        for precision in ("fp64", "mixed"):
            api.set_tuning(4, precision, *shape)
            sm, fi = run_smoother(prob, precision)
            tm, tc = TOL[precision]
            compare(sm, ref_sm, tm, tc, f"smoothed {precision} {shape}")
            compare(fi, ref_fi, tm, tc, f"filtered {precision} {shape}")
    finally:
        api.set_tuning(4, "fp64")
        api.set_tuning(4, "mixed")


def test_autotune_keeps_a_valid_tuning_and_results_still_match(oracle_mod):
    from paper_2410_00627_gb300 import api
    prob = synth.chain4(seed=6, n_slow=900, keep_states=False)
    args = [to_dev(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    try:
        tuned, ms = api.autotune(*args, prob.ratio, precision="mixed", reps=1)
        assert ms > 0
        assert tuned == api.get_tuning(4, "mixed")
        assert tuned["scan_groups"] in (2, 4, 8, 16) and 1 <= tuned["scan_elems"] <= 32
        assert tuned["recover_threads"] in (32, 64, 96, 128) and tuned["lookback_window"] in (4, 8, 16, 32)
        assert tuned["setup_mode"] in (1, 2)
        ref_sm, ref_fi = oracle_views(oracle_mod.sequential(prob), prob.ratio)
        sm, fi = run_smoother(prob, "mixed")
        tm, tc = TOL["mixed"]
        compare(sm, ref_sm, tm, tc, "smoothed after autotune")
        compare(fi, ref_fi, tm, tc, "filtered after autotune")
    finally:
        api.set_tuning(4, "mixed")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("case", CASES[:9], ids=lambda c: "n{1}m{2}l{3}N{4}".format(*c))
def test_loglik_matches_oracle(oracle_mod, case, precision):
    """log p(y_1:N) (the loglik output) against the oracle's prediction-error
    decomposition; the other outputs are unchanged by asking for it."""
    from paper_2410_00627_gb300 import api
    seed, nx, ny, l, N = case
    prob = synth.random_model(seed, nx, ny, l, N)
    args = [to_dev(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    sm, _ = api.smoother(*args, l, precision=precision, outputs=api.ALL_OUTPUTS)
    api.status()
    assert api.last_call_launches() == 5
    want = oracle_mod.loglik(prob)
    got = float(sm["loglik"].cpu().item())
    tol = 1e-9 if precision == "fp64" else 1e-4
    assert abs(got - want) <= tol * max(1.0, abs(want)), (got, want)
    plain, _ = api.smoother(*args, l, precision=precision)
    assert_same_to_rounding(plain["fast_cov"], sm["fast_cov"], precision, "fast_cov")


def test_loglik_full_size_chain4_and_filter_call(oracle_mod):
    from paper_2410_00627_gb300 import api
    prob = synth.chain4(seed=0, n_slow=10_000, keep_states=False)
    args = [to_dev(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    want = oracle_mod.loglik(prob)
    for precision, tol in (("fp64", 1e-9), ("mixed", 1e-4)):
        out = api.filter(*args, prob.ratio, precision=precision, outputs=("slow_mean", "loglik"))
        api.status()
        got = float(out["loglik"].cpu().item())
        assert abs(got - want) <= tol * abs(want), (precision, got, want)


def test_loglik_per_sequence_in_a_batch(oracle_mod):
    import torch

    from paper_2410_00627_gb300 import api
    probs = synth.ragged_chains(seed=9, n_seq=7, n_min=1, n_max=90)
    pk = synth.pack(probs)
    t = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    b = api.make_batch(t(pk["F"]), t(pk["Q"]), t(pk["H"]), t(pk["R"]), t(pk["m0"]), t(pk["P0"]), t(pk["y"]),
                       t(pk["ratio"]), t(pk["n_slow"]), pk["max_ratio"], pk["total_slow"], pk["total_fast"])
    sm, _ = api.smoother_batch(b, precision="fp64", outputs=("slow_mean", "loglik"))
    api.status()
    got = sm["loglik"].cpu().numpy()
    want = np.array([oracle_mod.loglik(p) for p in probs])
    assert np.all(np.abs(got - want) <= 1e-9 * np.maximum(1.0, np.abs(want)))


def test_loglik_through_host_entry_point(oracle_mod):
    from paper_2410_00627_gb300 import api
    prob = synth.chain4(seed=8, n_slow=200, keep_states=False)
    res = api.smoother_host(*[np.ascontiguousarray(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")],
                            prob.ratio, precision="fp64", loglik=True)
    want = oracle_mod.loglik(prob)
    assert abs(res["loglik"][0] - want) <= 1e-9 * abs(want)


def test_batch_descriptor_keeps_its_tensors_alive(oracle_mod):
    """make_batch over temporaries: the descriptor holds only raw pointers, so
    it must keep the tensors alive; freed blocks are reused by new tensors."""
    import gc

    import torch

    from paper_2410_00627_gb300 import api
    probs = synth.ragged_chains(seed=13, n_seq=20, n_min=1, n_max=60)
    pk = synth.pack(probs)
    t = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    b = api.make_batch(t(pk["F"]), t(pk["Q"]), t(pk["H"]), t(pk["R"]), t(pk["m0"]), t(pk["P0"]), t(pk["y"]),
                       t(pk["ratio"]), t(pk["n_slow"]), pk["max_ratio"], pk["total_slow"], pk["total_fast"])
    gc.collect()
    junk = [torch.full((pk[k].size,), 7, dtype=torch.int32 if k in ("ratio", "n_slow") else torch.float64,
                       device="cuda") for k in ("F", "Q", "H", "R", "m0", "P0", "y", "ratio", "n_slow")]
    sm, _ = api.smoother_batch(b, precision="fp64", outputs=("slow_mean",))
    api.status()
    del junk
    got = sm["slow_mean"].cpu().numpy()
    so = 0
    for p in probs:
        ref = oracle_mod.sequential(p)["fast_smooth_mean"][p.ratio - 1::p.ratio]
        compare({"slow_mean": got[so:so + p.n_slow]}, {"slow_mean": ref}, *TOL["fp64"], label=p.name)
        so += p.n_slow


def test_host_entry_point_direct_pinned_outputs_match_staged():
    """Pinned host outputs are written by the kernels directly; pageable ones
    are staged and copied: both agree with the device path to rounding."""
    import torch

    from paper_2410_00627_gb300 import api
    prob = synth.chain4(seed=21, n_slow=300, keep_states=False)
    host_in = [np.ascontiguousarray(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    n_fast, nx = prob.n_slow * prob.ratio, prob.nx
    shapes = {"fast_mean": (n_fast, nx), "fast_cov": (n_fast, nx, nx), "slow_mean": (prob.n_slow, nx),
              "slow_cov": (prob.n_slow, nx, nx)}
    pinned = {k: torch.full(s, np.nan, dtype=torch.float64, pin_memory=True).numpy() for k, s in shapes.items()}
    for precision in ("fp64", "mixed"):
        direct = api.smoother_host(*host_in, prob.ratio, precision=precision, out=pinned)
        staged = api.smoother_host(*host_in, prob.ratio, precision=precision)
        dev, _ = api.smoother(*[to_dev(a) for a in host_in], prob.ratio, precision=precision)
        api.status()
        for k in shapes:
            want = dev[k].cpu().numpy()
            assert_same_to_rounding(direct[k], want, precision, f"direct {k}")
            assert_same_to_rounding(staged[k], want, precision, f"staged {k}")


def test_host_entry_point_reads_pinned_inputs_directly():
    """Pinned y (and u) are read by the kernels in place; results agree with
    the device path's to rounding, with and without known inputs."""
    import torch

    from paper_2410_00627_gb300 import api

    def pin(a):
        t = torch.empty(a.shape, dtype=torch.float64, pin_memory=True)
        t.numpy()[...] = a
        return t.numpy()

    for prob in (synth.chain4(seed=22, n_slow=200, keep_states=False), synth.random_model(23, 3, 2, 5, 90, nu=2)):
        keys = ("F", "Q", "H", "R", "m0", "P0", "y")
        host_in = [pin(np.ascontiguousarray(getattr(prob, k))) for k in keys]
        extra = {} if prob.B is None else {"B": pin(prob.B), "u": pin(prob.u)}
        got = api.smoother_host(*host_in, prob.ratio, precision="fp64", loglik=True, **extra)
        dev_extra = {} if prob.B is None else {"B": to_dev(prob.B), "u": to_dev(prob.u)}
        want, _ = api.smoother(*[to_dev(getattr(prob, k)) for k in keys], prob.ratio, precision="fp64",
                               outputs=api.ALL_OUTPUTS, **dev_extra)
        api.status()
        for k in api.ALL_OUTPUTS:
            assert_same_to_rounding(got[k], want[k], "fp64", f"{prob.name} {k}")


def test_outputs_at_8_byte_offsets():
    """Output buffers that are only 8-byte aligned (views one double into a
    larger tensor) take the 8-byte store path and give the same results."""
    import torch

    from paper_2410_00627_gb300 import api
    prob = synth.random_model(24, 3, 2, 5, 37)
    args = [to_dev(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    n_fast, nx = prob.n_slow * prob.ratio, prob.nx
    base = {"fast_mean": n_fast * nx, "fast_cov": n_fast * nx * nx, "slow_mean": prob.n_slow * nx,
            "slow_cov": prob.n_slow * nx * nx}
    shapes = {"fast_mean": (n_fast, nx), "fast_cov": (n_fast, nx, nx), "slow_mean": (prob.n_slow, nx),
              "slow_cov": (prob.n_slow, nx, nx)}
    odd = {k: torch.empty(n + 1, dtype=torch.float64, device="cuda")[1:].view(shapes[k]) for k, n in base.items()}
    assert all(v.data_ptr() % 16 == 8 for v in odd.values())
    got, _ = api.smoother(*args, prob.ratio, out=odd)
    want, _ = api.smoother(*args, prob.ratio)
    api.status()
    for k in shapes:
        assert_same_to_rounding(got[k], want[k], "fp64", k)


def test_split_recovery_matches_one_kernel():
    """The two halves of a split recovery do the one-kernel arithmetic in the
    same order: smoothed, filtered extras and log likelihood agree (to the
    rounding that separates any two calls); the call makes one more launch.
    Also for a ragged batch."""
    import torch

    from paper_2410_00627_gb300 import api
    prob = synth.random_model(25, 4, 2, 6, 300, nu=2)
    args = [to_dev(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    ctl = {"B": to_dev(prob.B), "u": to_dev(prob.u)}
    probs = synth.ragged_chains(seed=14, n_seq=12, n_min=1, n_max=80)
    pk = synth.pack(probs)
    t = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    b = api.make_batch(t(pk["F"]), t(pk["Q"]), t(pk["H"]), t(pk["R"]), t(pk["m0"]), t(pk["P0"]), t(pk["y"]),
                       t(pk["ratio"]), t(pk["n_slow"]), pk["max_ratio"], pk["total_slow"], pk["total_fast"])
    try:
        for precision in ("fp64", "mixed", "fp32"):
            res, launches = {}, {}
            for split in (1, 2):
                api.set_tuning(4, precision, recover_split=split)
                sm, fi = api.smoother(*args, prob.ratio, precision=precision, outputs=api.ALL_OUTPUTS,
                                      filtered=api.OUTPUT_KEYS, **ctl)
                api.status()
                launches[split] = api.last_call_launches()
                bs, _ = api.smoother_batch(b, precision=precision)
                api.status()
                res[split] = ({k: v.cpu() for k, v in sm.items()}, {k: v.cpu() for k, v in fi.items()},
                              {k: v.cpu() for k, v in bs.items()})
            assert launches[2] == launches[1] + 1
            for part in range(3):
                for k in res[1][part]:
                    assert_same_to_rounding(res[2][part][k], res[1][part][k], precision, f"{part} {k}")
    finally:
        for p in ("fp64", "mixed", "fp32"):
            api.set_tuning(4, p)


def test_pinned_host_output_tensors_through_the_device_api():
    """Outputs may be pinned host tensors (the kernels write them directly):
    equal to the device outputs, for a single sequence and a batch."""
    import torch

    from paper_2410_00627_gb300 import api
    prob = synth.random_model(27, 4, 2, 6, 120)
    args = [to_dev(getattr(prob, k)) for k in ("F", "Q", "H", "R", "m0", "P0", "y")]
    n_fast, nx = prob.n_slow * prob.ratio, prob.nx
    host = {"fast_cov": torch.empty((n_fast, nx, nx), dtype=torch.float64, pin_memory=True),
            "slow_mean": torch.empty((prob.n_slow, nx), dtype=torch.float64, pin_memory=True)}
    got, _ = api.smoother(*args, prob.ratio, precision="mixed", out=host)
    want, _ = api.smoother(*args, prob.ratio, precision="mixed")
    api.status()
    assert not got["fast_cov"].is_cuda
    for k in host:
        assert_same_to_rounding(got[k], want[k], "mixed", k)
    with pytest.raises(TypeError):  # pageable host memory is not accepted
        api.smoother(*args, prob.ratio, out={"slow_mean": torch.empty((prob.n_slow, nx), dtype=torch.float64)})
    probs = synth.ragged_chains(seed=15, n_seq=9, n_min=1, n_max=70)
    pk = synth.pack(probs)
    t = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    b = api.make_batch(t(pk["F"]), t(pk["Q"]), t(pk["H"]), t(pk["R"]), t(pk["m0"]), t(pk["P0"]), t(pk["y"]),
                       t(pk["ratio"]), t(pk["n_slow"]), pk["max_ratio"], pk["total_slow"], pk["total_fast"])
    hs = {"slow_cov": torch.empty((pk["total_slow"], 4, 4), dtype=torch.float64, pin_memory=True)}
    got, _ = api.smoother_batch(b, precision="fp64", out=hs)
    want, _ = api.smoother_batch(b, precision="fp64")
    api.status()
    assert_same_to_rounding(got["slow_cov"], want["slow_cov"], "fp64", "batch slow_cov")
