"""The benchmark's host logic: the multi-rank aggregation (no collective on the
data path) on two gloo ranks on the CPU: the whole-job step time is the
slowest rank's, and the units are summed; the split of the batch over ranks;
and the reference arm's JSON line (the oracle on the host cores)."""
import os
import socket

import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    import sys
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms = [3.0, 5.5][rank]
        units = [200_000, 150_000][rank]
        q.put((rank, bench.reduce_over_ranks(ms, units, dist, "cpu")))
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_two_gloo_ranks():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    got = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(2):
        assert got[r] == pytest.approx((5.5, 350_000.0))


def test_reduce_over_ranks_single_process():
    import bench
    assert bench.reduce_over_ranks(2.0, 10, None, "cpu") == (2.0, 10.0)


def test_bench_arguments_default_to_one_gpu_ragged_batch():
    import bench
    a = bench.parse([])
    assert a.gpus == 1 and a.workload == "ragged_chains" and a.n_seq == 4096 and a.warmup >= 3 and a.impl == "ours"
    b = bench.parse(["--workload", "chain4", "--steps", "3"])
    assert b.workload == "chain4" and b.n_slow == 10_000 and b.steps == 3


def test_batch_partition_over_ranks_balances_fast_steps():
    """Under torchrun the batch is split into contiguous sequence ranges of
    nearly equal fast steps; the ranges tile the batch and the shapes used to
    split it are those of the generated sequences."""
    import numpy as np

    from paper_2410_00627_gb300 import synth
    r, n = synth.ragged_shapes(0, 4096)
    f = r * n
    for world in (2, 4, 8):
        rng = synth.balanced_ranges(f, world)
        assert rng[0][0] == 0 and rng[-1][1] == 4096
        assert all(a[1] == b[0] for a, b in zip(rng[:-1], rng[1:]))
        share = np.array([f[lo:hi].sum() for lo, hi in rng]) / f.sum()
        assert np.all(np.abs(share - 1.0 / world) <= f.max() / f.sum() + 1e-12), (world, share)
    probs = synth.ragged_chains(0, 12, seq_range=(4, 9))
    r12, n12 = synth.ragged_shapes(0, 12)
    assert [(p.ratio, p.n_slow) for p in probs] == list(zip(r12[4:9], n12[4:9]))


def test_reference_arm_line_on_the_cpu():
    """`bench.py --impl reference` (the oracle on the host cores) prints one JSON
    line with the contract's keys, on the same metric and workload as the GPU arm."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--workload", "chain4",
                          "--n-slow", "100", "--steps", "2", "--warmup", "1"], capture_output=True, text=True,
                         timeout=300, check=True)
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    import bench
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["metric"] == bench.METRIC and d["unit"] == bench.UNIT
    assert d["higher_is_better"] is True and d["value"] > 0 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == 1
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["config"]["workload"].startswith("chain4") and d["config"]["n_slow"] == 100
