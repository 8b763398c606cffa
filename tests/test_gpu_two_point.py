"""GPU parity of the two-point form of the fast-rate recovery (tuning field
recover_form = 2).  A smoother call that asks for smoothed outputs only
takes every fast-rate smoothed moment of interval k from the smoothed joint
of x_{k,1} and x_{k+1,1} (the smoother scan's results and the gain E_k of
its element, Eq. 29), conditioned on y_k through per-model constants.  The
outputs are compared with the FP64 oracle for every state size, several
measurement sizes and ratios (ratio 1 and a single slow step included), in
FP64 and mixed precision, next to the record form of the same call; in a
batch where a sequence whose process noise is confined to a subspace keeps
the record form; in a chunked batch; and with filtered outputs asked for
(the record form, the same bits as recover_form = 1)."""
import numpy as np
import pytest

from paper_2410_00627_gb300 import synth
from tests.gpu_util import TOL, compare, oracle_views, run_smoother

pytestmark = pytest.mark.gpu

CASES = [(1, 1, 5, 30), (2, 1, 3, 40), (3, 2, 4, 25), (4, 1, 20, 50), (4, 2, 10, 40), (5, 3, 6, 20),
         (6, 2, 8, 15), (7, 1, 4, 12), (8, 3, 5, 12), (4, 1, 1, 30), (3, 2, 4, 1), (4, 4, 3, 20)]


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


def _smoothed(prob, precision, form):
    from paper_2410_00627_gb300 import api
    api.set_tuning(prob.nx, precision, recover_form=form)
    sm, _ = run_smoother(prob, precision, filtered=False)
    api.status()
    return {k: np.asarray(v) for k, v in sm.items()}, api.last_call_launches()


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nx,ny,l,N", CASES)
def test_two_point_matches_oracle(oracle_mod, nx, ny, l, N, precision):
    prob = synth.random_model(200 + 10 * nx + ny, nx, ny, l, N)
    ref, _ = oracle_views(oracle_mod.sequential(prob), l)
    got2, n2 = _smoothed(prob, precision, 2)
    got1, n1 = _smoothed(prob, precision, 1)
    compare(got2, ref, *TOL[precision], label=f"two-point {prob.name} {precision}")
    compare(got1, ref, *TOL[precision], label=f"record form {prob.name} {precision}")
    assert n1 == n2   # the same launches (the record form without the split recovery)
    assert np.all(np.isfinite(got2["fast_cov"]))


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nx,ny,l,N", [(4, 1, 10, 60), (3, 2, 4, 45), (6, 2, 5, 20)])
def test_two_point_with_the_setup_as_its_own_kernel(oracle_mod, nx, ny, l, N, precision):
    """setup_mode 2: the interval setup (float32 for two-point sequences in the
    mixed mode) runs as its own kernel after the filter scan."""
    from paper_2410_00627_gb300 import api
    prob = synth.random_model(500 + nx, nx, ny, l, N)
    ref, _ = oracle_views(oracle_mod.sequential(prob), l)
    api.set_tuning(nx, precision, setup_mode=2, recover_form=2)
    sm, _ = run_smoother(prob, precision, filtered=False)
    api.status()
    compare({k: np.asarray(v) for k, v in sm.items()}, ref, *TOL[precision], label=f"setup kernel {prob.name}")


def test_two_point_fp32_runs_within_the_mixed_bound(oracle_mod):
    """The FP32 mode (everything after the model constants in float32, not
    gated elsewhere) takes the two-point form too; on a well-conditioned model
    it stays within the mixed tolerances."""
    prob = synth.random_model(611, 4, 2, 8, 40)
    ref, _ = oracle_views(oracle_mod.sequential(prob), prob.ratio)
    got, _ = _smoothed(prob, "fp32", 2)
    compare(got, ref, *TOL["mixed"], label=f"two-point fp32 {prob.name}")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_two_point_ragged_chains_and_chunks(oracle_mod, precision):
    import torch

    from paper_2410_00627_gb300 import api
    probs = synth.ragged_chains(seed=61, n_seq=24, n_min=1, n_max=300)
    pk = synth.pack(probs)
    t = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    b = api.make_batch(t(pk["F"]), t(pk["Q"]), t(pk["H"]), t(pk["R"]), t(pk["m0"]), t(pk["P0"]), t(pk["y"]),
                       t(pk["ratio"]), t(pk["n_slow"]), pk["max_ratio"], pk["total_slow"], pk["total_fast"])
    for chunks in (1, 4):
        api.set_tuning(4, precision, recover_form=2, batch_chunks=chunks)
        sm, _ = api.smoother_batch(b, precision=precision)
        api.status()
        got = {k: v.cpu().numpy() for k, v in sm.items()}
        fo = so = 0
        for p in probs:
            l, N = p.ratio, p.n_slow
            ref, _ = oracle_views(oracle_mod.sequential(p), l)
            cut = {k: (got[k][fo:fo + N * l] if k.startswith("fast") else got[k][so:so + N]) for k in got}
            compare(cut, ref, *TOL[precision], label=f"two-point batch chunks={chunks} {p.name}")
            fo += N * l
            so += N


def test_sequence_without_full_interval_noise_keeps_the_record_form(oracle_mod):
    """Process noise on two of four states of a diagonal transition: the
    covariance of x_{k+1,1} given x_{k,1} is singular, so that sequence keeps
    the record form (its outputs are the record form's bits) while the
    others of the batch take the two-point form; all match the oracle."""
    import torch

    from paper_2410_00627_gb300 import api
    probs = [synth.random_model(300 + i, 4, 1, 4, 20) for i in range(3)]
    sub = probs[1]
    sub.F = np.diag([0.99, 0.98, 0.995, 0.99])
    sub.Q = np.diag([0.02, 0.03, 0.0, 0.0])   # (the measurements stay those of the generated model)
    pk = synth.pack(probs)
    t = lambda a: torch.as_tensor(a, device="cuda")  # noqa: E731
    b = api.make_batch(t(pk["F"]), t(pk["Q"]), t(pk["H"]), t(pk["R"]), t(pk["m0"]), t(pk["P0"]), t(pk["y"]),
                       t(pk["ratio"]), t(pk["n_slow"]), pk["max_ratio"], pk["total_slow"], pk["total_fast"])
    outs = {}
    for form in (1, 2):
        api.set_tuning(4, "fp64", recover_form=form)
        sm, _ = api.smoother_batch(b, precision="fp64")
        api.status()
        outs[form] = {k: v.cpu().numpy() for k, v in sm.items()}
    fo = so = 0
    for s, p in enumerate(probs):
        l, N = p.ratio, p.n_slow
        ref, _ = oracle_views(oracle_mod.sequential(p), l)
        for form in (1, 2):
            got = outs[form]
            cut = {k: (got[k][fo:fo + N * l] if k.startswith("fast") else got[k][so:so + N]) for k in got}
            compare(cut, ref, *TOL["fp64"], label=f"form {form} seq {s}")
        if s == 1:
            for k in outs[1]:
                a = outs[1][k][fo:fo + N * l] if k.startswith("fast") else outs[1][k][so:so + N]
                c = outs[2][k][fo:fo + N * l] if k.startswith("fast") else outs[2][k][so:so + N]
                assert np.array_equal(a, c), k
        fo += N * l
        so += N


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_filtered_outputs_take_the_record_form(precision):
    """With filtered outputs asked for, recover_form = 2 runs the record form:
    the same bits as recover_form = 1."""
    from paper_2410_00627_gb300 import api
    prob = synth.random_model(411, 4, 2, 6, 35)
    res = {}
    for form in (1, 2):
        api.set_tuning(4, precision, recover_form=form, recover_split=1)
        sm, fi = run_smoother(prob, precision, filtered=True)
        api.status()
        res[form] = ({k: np.asarray(v) for k, v in sm.items()}, {k: np.asarray(v) for k, v in fi.items()})
    for part in (0, 1):
        for k in res[1][part]:
            assert np.array_equal(res[1][part][k], res[2][part][k]), (part, k)
