"""The benchmark's host logic: the multi-rank aggregation (weak scaling: every rank runs its
own workload, no collective on the data path) on two gloo ranks on the CPU:
the whole-job step time is the slowest rank's, and the units are summed; and
the reference arm's JSON line (the oracle on the host cores)."""
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


def test_bench_arguments_default_to_one_gpu_chain4():
    import bench
    a = bench.parse([])
    assert a.gpus == 1 and a.workload == "chain4" and a.warmup >= 3 and a.impl == "ours"
    b = bench.parse(["--workload", "ragged_chains", "--steps", "3"])
    assert b.workload == "ragged_chains" and b.n_seq == 4096 and b.steps == 3


def test_reference_arm_line_on_the_cpu():
    """`bench.py --impl reference` (the oracle on the host cores) prints one JSON
    line with the contract's keys, on the same metric and workload as the GPU arm."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--n-slow", "100",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, check=True)
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
