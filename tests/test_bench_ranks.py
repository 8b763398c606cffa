"""The benchmark's multi-rank aggregation (weak scaling: every rank runs its
own workload, no collective on the data path) on two gloo ranks on the CPU:
the whole-job step time is the slowest rank's, and the units are summed."""
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
