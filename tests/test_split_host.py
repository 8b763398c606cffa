"""Host logic of the cross-GPU split of one sequence (paper_2410_00627_gb300.split)
on CPU gloo ranks, with the library's calls replaced at the exchange boundary
by fakes that only record what they receive: every rank gathers every
aggregate, combines the EARLIER ranks' filter aggregates in rank order into its
prior, the LATER ranks' smoother aggregates in rank order into the state after
its range, and hands both to its range smoother; the first rank keeps m0, P0
and the last rank has no following state."""
import os
import socket

import pytest


def test_ranges_tile_the_sequence():
    from paper_2410_00627_gb300 import split
    for n, parts in ((10, 1), (10, 3), (7, 7), (10_000, 8), (101, 4)):
        rg = split.ranges(n, parts)
        assert rg[0][0] == 0 and rg[-1][1] == n and len(rg) == parts
        assert all(a[1] == b[0] for a, b in zip(rg[:-1], rg[1:]))
        sizes = [hi - lo for lo, hi in rg]
        assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        split.ranges(3, 4)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _fake_api(api, torch, nx, rank):
    """Aggregates carry the producing rank's id; a combine encodes the order of
    the ranks it received as the decimal digits (rank + 1) of its mean part."""
    def filt(F, Q, H, R, m0, P0, y, ratio, starts, precision, stream):
        assert starts == (rank == 0)
        return torch.full((api.filter_element_size(nx),), float(rank))

    def smagg(F, Q, H, R, m_in, P_in, y, ratio, ends, precision, stream):
        return torch.full((api.smoother_element_size(nx),), float(rank) + 100.0 * float(m_in[0]))

    def combine(op, elems, stream=None):
        n, size = elems.shape
        code = 0.0
        for i in range(n):
            code = code * 10 + (float(elems[i, 0]) % 100.0) + 1
        out = torch.zeros(size)
        out[nx * nx:nx * nx + nx] = code if op == "filter" else -code
        return out

    def final(F, Q, H, R, m_in, P_in, y, ratio, nm, nc, precision, outputs, filtered, stream):
        return {"m_in": m_in.clone(), "next": None if nm is None else nm.clone()}, {}

    api.split_filter_aggregate = filt
    api.split_smoother_aggregate = smagg
    api.split_combine = combine
    api.split_smoother = final


def _rank_main(rank, world, port, q):
    import sys

    import torch
    import torch.distributed as dist
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    from paper_2410_00627_gb300 import api, split
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        nx = 3
        _fake_api(api, torch, nx, rank)
        m0 = torch.full((nx,), -7.0)
        P0 = torch.eye(nx)
        sm, _ = split.smoother_split(torch.zeros(nx, nx), None, None, None, m0, P0, torch.zeros(5, 1), 4, "fp64")
        q.put((rank, sm["m_in"].tolist(), None if sm["next"] is None else sm["next"].tolist()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_each_rank_combines_the_right_aggregates_in_order(world):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    got = {}
    for _ in procs:
        r, m_in, nxt = q.get(timeout=120)
        got[r] = (m_in, nxt)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in range(world):
        m_in, nxt = got[r]
        if r == 0:
            assert m_in == [-7.0] * 3                       # the first range keeps m0
        else:                                               # filter aggregates of ranks 0..r-1, in order
            want = 0.0
            for k in range(r):
                want = want * 10 + k + 1
            assert m_in == [want] * 3
        if r == world - 1:
            assert nxt is None                              # the last range ends the sequence
        else:                                               # smoother aggregates of ranks r+1..world-1, in order
            want = 0.0
            for k in range(r + 1, world):
                want = want * 10 + k + 1
            assert nxt == [-want] * 3
