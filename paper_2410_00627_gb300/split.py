"""One long sequence split over several GPUs (one rank per GPU).

The filter operator of Eq. (27) and the smoother operator of Eq. (30) are
associative (Sec. II), so each rank scans its own contiguous range of slow
steps and the ranks exchange one aggregate element per scan:

  1. every rank reduces its range's filter elements to one aggregate
     (srtm_split_filter_aggregate) and the aggregates are all-gathered;
  2. the product of the earlier ranks' aggregates (srtm_split_combine) is the
     filtered state before the range, its prior;
  3. with that prior every rank forms its smoother elements and reduces them
     to one aggregate (srtm_split_smoother_aggregate); all-gather;
  4. the product of the later ranks' aggregates is the smoothed first state
     after the range;
  5. every rank runs its range's scans and fast-rate recovery with the prior
     and that state (srtm_split_smoother).

The two all-gathers move 3 nx^2 + 2 nx and 2 nx^2 + nx float64 values per
rank; everything else stays on the rank's GPU.  This module only orders the
calls and moves the aggregates: every arithmetic step runs in the library's
kernels.  The exchange is torch.distributed's all_gather (NCCL between GPUs;
gloo moves CPU copies).
"""
from __future__ import annotations

import numpy as np

from . import api


def ranges(n_slow: int, parts: int) -> list[tuple[int, int]]:
    """Contiguous slow-step ranges [lo, hi) of the sequence, one per rank,
    whose lengths differ by at most one (every range holds at least one step)."""
    if parts < 1 or n_slow < parts:
        raise ValueError(f"{n_slow} slow steps cannot be split into {parts} non-empty ranges")
    cuts = np.linspace(0, n_slow, parts + 1).round().astype(int)
    return [(int(a), int(b)) for a, b in zip(cuts[:-1], cuts[1:])]


def _state(elem, nx):
    """(mean, covariance) part of a combined element: (d, D) of a filter
    element, (g, S) of a smoother element; both start at offset nx^2."""
    return elem[nx * nx:nx * nx + nx].contiguous(), elem[nx * nx + nx:nx * nx + nx + nx * nx].reshape(nx, nx).contiguous()


def prior_from(aggs_before, m0, P0):
    """The filtered state before a range: (d, D) of the product of the earlier
    ranges' filter aggregates (Eq. 27), or (m0, P0) for the first range."""
    if len(aggs_before) == 0:
        return m0, P0
    import torch
    return _state(api.split_combine("filter", torch.stack(list(aggs_before))), m0.shape[0])


def next_from(aggs_after, nx):
    """The smoothed first state after a range: (g, S) of the product of the
    later ranges' smoother aggregates (Eq. 30), or (None, None) for the range
    that ends the sequence."""
    if len(aggs_after) == 0:
        return None, None
    import torch
    return _state(api.split_combine("smoother", torch.stack(list(aggs_after))), nx)


def all_gather(t, group=None):
    """torch.distributed all_gather of a small CUDA tensor (through CPU copies
    when the process group's backend is gloo)."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    cpu = dist.get_backend(group) == "gloo"
    src = t.cpu() if cpu else t
    parts = [torch.empty_like(src) for _ in range(world)]
    dist.all_gather(parts, src, group=group)
    return [p.to(t.device) for p in parts] if cpu else parts


def smoother_split(F, Q, H, R, m0, P0, y_range, ratio, precision="mixed", outputs=api.OUTPUT_KEYS, filtered=(),
                   group=None, stream=None, exchange=None):
    """The smoother for this rank's range of a sequence split over the ranks of
    ``group`` in rank order (rank r holds the r-th range; ``ranges`` gives an
    even split).  F, Q, H, R, m0, P0 are the whole sequence's model (CUDA
    float64 tensors on this rank's GPU), y_range the range's measurements.
    Returns (smoothed, filtered) dicts of the range's outputs, rows relative to
    the range, as the single-GPU srtm_smoother would give them for those rows.
    ``exchange(t) -> list`` replaces the all-gather (default: all_gather)."""
    import torch.distributed as dist
    rank, world = dist.get_rank(group), dist.get_world_size(group)
    gather = exchange or (lambda t: all_gather(t, group))
    nx = F.shape[0]
    agg_f = api.split_filter_aggregate(F, Q, H, R, m0, P0, y_range, ratio, rank == 0, precision, stream)
    all_f = gather(agg_f)
    m_in, P_in = prior_from(all_f[:rank], m0, P0)
    agg_s = api.split_smoother_aggregate(F, Q, H, R, m_in, P_in, y_range, ratio, rank == world - 1, precision, stream)
    all_s = gather(agg_s)
    nm, nc = next_from(all_s[rank + 1:], nx)
    return api.split_smoother(F, Q, H, R, m_in, P_in, y_range, ratio, nm, nc, precision, outputs, filtered, stream)


def smoother_split_serial(F, Q, H, R, m0, P0, y, ratio, parts, precision="mixed", outputs=api.OUTPUT_KEYS,
                          filtered=(), stream=None):
    """The same decomposition with ``parts`` ranges run one after another on
    the current GPU (each phase for every range before the next phase, as
    the ranks would run it): a check of the split on one GPU.  Returns a list
    of (smoothed, filtered) per range."""
    rg = ranges(y.shape[0], parts)
    ys = [y[lo:hi].contiguous() for lo, hi in rg]
    nx = F.shape[0]
    all_f = [api.split_filter_aggregate(F, Q, H, R, m0, P0, ys[r], ratio, r == 0, precision, stream)
             for r in range(parts)]
    priors = [prior_from(all_f[:r], m0, P0) for r in range(parts)]
    all_s = [api.split_smoother_aggregate(F, Q, H, R, *priors[r], ys[r], ratio, r == parts - 1, precision, stream)
             for r in range(parts)]
    res = []
    for r in range(parts):
        nm, nc = next_from(all_s[r + 1:], nx)
        res.append(api.split_smoother(F, Q, H, R, *priors[r], ys[r], ratio, nm, nc, precision, outputs, filtered,
                                      stream))
    return res
