"""The ragged batch at its full size (4096 ragged sequences, ~4*10^7 slow and ~5*10^8
fast steps) in the launch configuration the benchmark times: shapes chosen by
the autotuner on the first 512 sequences, the batched call captured in a CUDA
graph and replayed.  Sampled sequences (the shortest, the longest, the first,
the last and three drawn at random) are compared in full with the FP64
oracle, for the mixed and the FP64 modes."""
import os

import numpy as np
import pytest

from paper_2410_00627_gb300 import synth
from tests.gpu_util import TOL, compare, oracle_views

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def full_batch():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    probs = synth.ragged_chains(seed=0, n_seq=4096, workers=max(1, min(16, os.cpu_count() or 1)))
    return probs, synth.pack(probs)


def test_ragged_chains_full_batch_sampled(oracle_mod, full_batch):
    import torch

    import bench
    from paper_2410_00627_gb300 import api, build
    build.build()
    api.load()
    probs, pk = full_batch
    dev = torch.device("cuda", torch.cuda.current_device())
    batch, ten = bench.upload_batch(pk, api, torch, dev)
    outs = bench.batch_outputs(torch, dev, pk["total_fast"], pk["total_slow"], 4)
    n = pk["n_slow"]
    rng = np.random.default_rng(1)
    pick = sorted({int(np.argmin(n)), int(np.argmax(n)), 0, len(probs) - 1, *rng.integers(0, len(probs), 3).tolist()})
    off_s = np.concatenate([[0], np.cumsum(n.astype(np.int64))])
    off_f = np.concatenate([[0], np.cumsum(n.astype(np.int64) * pk["ratio"])])
    refs = {s: oracle_views(oracle_mod.sequential(probs[s]), probs[s].ratio)[0] for s in pick}
    sub = synth.pack(probs[:512])
    sb, sten = bench.upload_batch(sub, api, torch, dev)
    so = bench.batch_outputs(torch, dev, sub["total_fast"], sub["total_slow"], 4)
    stream = torch.cuda.Stream()
    try:
        for precision in ("mixed", "fp64"):
            api.autotune_batch(sb, precision=precision, reps=1, out=so)
            with torch.cuda.stream(stream):
                api.smoother_batch(batch, precision=precision, out=outs, stream=stream)
                api.status(stream)
            g = torch.cuda.CUDAGraph()
            with torch.cuda.graph(g, stream=stream, capture_error_mode="relaxed"):
                api.smoother_batch(batch, precision=precision, out=outs, stream=stream)
            # the poison fill and the replay on one stream: a fill on another
            # stream may run beside the replay's persistent scans and land
            # after the recovery's stores
            with torch.cuda.stream(stream):   # replay() launches on the current stream
                for v in outs.values():
                    v.fill_(float("nan"))
                g.replay()
            stream.synchronize()
            api.status(stream)
            for s in pick:
                fs, ff = slice(int(off_s[s]), int(off_s[s + 1])), slice(int(off_f[s]), int(off_f[s + 1]))
                got = {"fast_mean": outs["fast_mean"][ff].cpu().numpy(), "fast_cov": outs["fast_cov"][ff].cpu().numpy(),
                       "slow_mean": outs["slow_mean"][fs].cpu().numpy(), "slow_cov": outs["slow_cov"][fs].cpu().numpy()}
                compare(got, refs[s], *TOL[precision], label=f"ragged_chains seq {s} (N={n[s]}, l={pk['ratio'][s]}) {precision}")
            assert not torch.isnan(outs["slow_cov"]).any()
            del g
    finally:
        api.set_tuning(4, "mixed")
        api.set_tuning(4, "fp64")
