"""GPU parity of a batch processed in chunks of whole sequences (tuning field
batch_chunks): the scans of chunk q+1 run while the fast-rate recovery of
chunk q runs on a second stream.  Every output of every sequence is compared
with the FP64 oracle (tolerances of the other parity tests), for several chunk
counts and launch grids, with chunks that are empty (one sequence holding most
of the batch), more chunks than sequences, known inputs and the log
likelihood, a filter-only call, host-pinned outputs, and the launch count."""
import numpy as np
import pytest

from paper_2410_00627_gb300 import synth
from tests.gpu_util import TOL, assert_same_to_rounding, compare, oracle_views

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2410_00627_gb300 import api, build
    build.build()
    api.load()
    yield
    for nx in range(1, 9):
        for p in ("fp64", "mixed", "fp32"):
            api.set_tuning(nx, p)


def _batch(probs):
    import torch

    from paper_2410_00627_gb300 import api
    pk = synth.pack(probs)
    t = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    extra = {"B": t(pk["B"]), "u": t(pk["u"])} if "B" in pk else {}
    return api.make_batch(t(pk["F"]), t(pk["Q"]), t(pk["H"]), t(pk["R"]), t(pk["m0"]), t(pk["P0"]), t(pk["y"]),
                          t(pk["ratio"]), t(pk["n_slow"]), pk["max_ratio"], pk["total_slow"], pk["total_fast"],
                          **extra)


def _check_against_oracle(oracle_mod, probs, sm, fi, precision, label, loglik=False):
    sm = {k: v.cpu().numpy() for k, v in sm.items()}
    fi = {k: v.cpu().numpy() for k, v in fi.items()}
    fo = so = 0
    for s, p in enumerate(probs):
        l, N = p.ratio, p.n_slow
        ref_sm, ref_fi = oracle_views(oracle_mod.sequential(p), l)

        def cut(d):
            return {k: (d[k][fo:fo + N * l] if k.startswith("fast") else d[k][so:so + N])
                    for k in ("fast_mean", "fast_cov", "slow_mean", "slow_cov") if k in d}
        compare(cut(sm), ref_sm, *TOL[precision], label=f"{label} smoothed {p.name}")
        if fi:
            compare(cut(fi), ref_fi, *TOL[precision], label=f"{label} filtered {p.name}")
        if loglik:
            want = oracle_mod.loglik(p)
            tol = 1e-9 if precision == "fp64" else 1e-4
            assert abs(sm["loglik"][s] - want) <= tol * max(1.0, abs(want)), (label, p.name, sm["loglik"][s], want)
        fo += N * l
        so += N


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("chunks,rec_bps,scan_bps,setup_mode", [
    (2, 0, 0, 1), (3, 2, 1, 1), (8, 1, 2, 2), (16, 3, 0, 1)])
def test_chunked_batch_matches_oracle(oracle_mod, precision, chunks, rec_bps, scan_bps, setup_mode):
    from paper_2410_00627_gb300 import api
    probs = synth.ragged_chains(seed=71, n_seq=37, n_min=1, n_max=400)
    probs[5] = synth.ragged_chains(seed=72, n_seq=1, n_min=1, n_max=1)[0]   # a length-1 sequence
    b = _batch(probs)
    api.set_tuning(4, precision, batch_chunks=chunks, chunk_recover_bps=rec_bps, chunk_scan_bps=scan_bps,
                   setup_mode=setup_mode)
    sm, fi = api.smoother_batch(b, precision=precision, filtered=api.OUTPUT_KEYS)
    api.status()
    _check_against_oracle(oracle_mod, probs, sm, fi, precision, f"chunks={chunks}")


def test_empty_chunks_and_more_chunks_than_sequences(oracle_mod):
    """One sequence holding most of the fast steps leaves middle chunks empty;
    a batch of three sequences asked for 16 chunks runs in three."""
    from paper_2410_00627_gb300 import api
    big = synth.ragged_chains(seed=81, n_seq=1, n_min=3000, n_max=3000)
    small = synth.ragged_chains(seed=82, n_seq=6, n_min=2, n_max=20)
    for probs in (big + small, small[:3]):
        b = _batch(probs)
        api.set_tuning(4, "fp64", batch_chunks=16)
        sm, _ = api.smoother_batch(b, precision="fp64")
        api.status()
        _check_against_oracle(oracle_mod, probs, sm, {}, "fp64", f"empty chunks S={len(probs)}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_chunked_batch_with_inputs_and_loglik(oracle_mod, precision):
    from paper_2410_00627_gb300 import api
    shapes = [(3, 40), (7, 1), (5, 90), (1, 55), (20, 12), (4, 3), (10, 70), (2, 200)]
    probs = [synth.random_model(90 + i, 3, 2, l, N, nu=2) for i, (l, N) in enumerate(shapes)]
    b = _batch(probs)
    api.set_tuning(3, precision, batch_chunks=4)
    sm, fi = api.smoother_batch(b, precision=precision, outputs=api.ALL_OUTPUTS, filtered=api.OUTPUT_KEYS)
    api.status()
    _check_against_oracle(oracle_mod, probs, sm, fi, precision, "chunks with inputs", loglik=True)


def test_chunked_filter_batch_and_launch_count(oracle_mod):
    from paper_2410_00627_gb300 import api
    probs = synth.ragged_chains(seed=91, n_seq=20, n_min=5, n_max=300)
    b = _batch(probs)
    api.set_tuning(4, "fp64", batch_chunks=4)
    out = api.filter_batch(b, precision="fp64")
    api.status()
    assert api.last_call_launches() == 1 + 1 + 4 * 2   # metadata, constants, (filter scan, recovery) per chunk
    got = {k: v.cpu().numpy() for k, v in out.items()}
    fo = so = 0
    for p in probs:
        l, N = p.ratio, p.n_slow
        _, ref_fi = oracle_views(oracle_mod.sequential(p), l)
        cut = {k: (got[k][fo:fo + N * l] if k.startswith("fast") else got[k][so:so + N]) for k in got}
        compare(cut, ref_fi, *TOL["fp64"], label=f"chunked filter {p.name}")
        fo += N * l
        so += N
    api.set_tuning(4, "fp64", batch_chunks=4, setup_mode=2)
    api.smoother_batch(b, precision="fp64")
    api.status()
    assert api.last_call_launches() == 1 + 1 + 4 * 4   # + (setup, smoother scan) per chunk


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_chunked_equals_one_chunk_to_rounding(precision):
    """A larger batch (200 sequences up to 3000 slow steps, many scan tiles per
    sequence): chunked and unchunked calls agree to the rounding that
    separates any two calls; so do device and pinned host outputs."""
    import torch

    from paper_2410_00627_gb300 import api
    probs = synth.ragged_chains(seed=95, n_seq=200, n_min=100, n_max=3000)
    b = _batch(probs)
    api.set_tuning(4, precision, batch_chunks=1)
    want, _ = api.smoother_batch(b, precision=precision)
    api.status()
    api.set_tuning(4, precision, batch_chunks=8)
    got, _ = api.smoother_batch(b, precision=precision)
    api.status()
    for k in want:
        assert_same_to_rounding(got[k], want[k], precision, f"chunked {k}")
    host = {k: torch.empty(v.shape, dtype=torch.float64, pin_memory=True) for k, v in want.items()}
    api.smoother_batch(b, precision=precision, out=host)
    api.status()
    for k in want:
        assert_same_to_rounding(host[k], want[k], precision, f"chunked pinned host {k}")
    assert np.all(np.isfinite(host["fast_cov"].numpy()))


@pytest.mark.parametrize("chunks", [1, 5])
def test_batch_host_outputs_written_over_the_link(oracle_mod, chunks):
    """Pinned host outputs of a batch (smoothed and filtered, fast and slow,
    and the log likelihood), written by the kernels over the CPU-GPU link, in
    one piece and in chunks: every output of every sequence against the
    oracle, also when the host buffers start 8 bytes past a 16-byte boundary."""
    import torch

    from paper_2410_00627_gb300 import api
    probs = synth.ragged_chains(seed=97, n_seq=23, n_min=1, n_max=250)
    b = _batch(probs)
    api.set_tuning(4, "fp64", batch_chunks=chunks)
    pk = synth.pack(probs)
    nf, ns, n = pk["total_fast"], pk["total_slow"], 4
    shapes = {"fast_mean": (nf, n), "fast_cov": (nf, n, n), "slow_mean": (ns, n), "slow_cov": (ns, n, n)}

    def pinned(shape, shift):
        raw = torch.full((int(np.prod(shape)) + 2,), np.nan, dtype=torch.float64, pin_memory=True)
        return raw[shift:shift + int(np.prod(shape))].view(shape)
    for shift in (0, 1):
        sm_h = {k: pinned(s, shift) for k, s in shapes.items()}
        fi_h = {k: pinned(s, shift) for k, s in shapes.items()}
        sm_h["loglik"] = pinned((len(probs),), shift)
        sm, fi = api.smoother_batch(b, precision="fp64", outputs=api.ALL_OUTPUTS, filtered=api.OUTPUT_KEYS,
                                    out=sm_h, out_filtered=fi_h)
        api.status()
        assert sm["fast_cov"].data_ptr() == sm_h["fast_cov"].data_ptr()
        _check_against_oracle(oracle_mod, probs, sm, fi, "fp64", f"host outputs chunks={chunks} shift={shift}",
                              loglik=True)
