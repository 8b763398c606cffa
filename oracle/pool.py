"""The oracle over many independent sequences on every host core.

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: the CPU baseline of
a batch of sequences (the benchmark's CPU leg).  Each task is one call of
``oracle.sequential`` on one sequence, untouched; sequences are independent,
so they are spread over worker processes.  Workers are started with the
"spawn" method: a process forked from one that has already used the GPU can
hang.  A worker returns only the number of fast steps it solved, never the
outputs.
"""
from __future__ import annotations

import multiprocessing as mp
import os
import time
import types
from concurrent.futures import FIRST_COMPLETED, ProcessPoolExecutor, wait

FIELDS = ("F", "Q", "H", "R", "m0", "P0", "y", "ratio", "B", "u")


def _ready(_=None) -> int:
    from . import oracle
    oracle._load()
    return os.getpid()


def _one(fields: dict) -> int:
    from . import oracle
    p = types.SimpleNamespace(**fields)
    oracle.sequential(p)
    return int(p.y.shape[0]) * int(p.ratio)


def host_cores() -> int:
    try:
        return len(os.sched_getaffinity(0))
    except AttributeError:
        return os.cpu_count() or 1


class SequencePool:
    """``workers`` spawned processes, each with the oracle library loaded."""

    def __init__(self, workers: int | None = None):
        from . import oracle
        oracle.build()   # compiled once here, loaded by every worker
        self.workers = workers or host_cores()
        self._ex = ProcessPoolExecutor(self.workers, mp_context=mp.get_context("spawn"))
        list(self._ex.map(_ready, range(self.workers)))   # start-up outside any timed region

    def run(self, probs, seconds: float) -> dict:
        """Solve probs[0], probs[1], ... in order until ``seconds`` have passed
        (tasks already started finish).  Returns the fast steps and sequences
        solved, the wall time and the worker count."""
        todo = iter(probs)
        pending, done_steps, used = set(), 0, 0
        t0 = time.perf_counter()
        while True:
            while len(pending) < 2 * self.workers and time.perf_counter() - t0 < seconds:
                p = next(todo, None)
                if p is None:
                    break
                pending.add(self._ex.submit(_one, {k: getattr(p, k, None) for k in FIELDS}))
                used += 1
            if not pending:
                break
            finished, pending = wait(pending, return_when=FIRST_COMPLETED)
            done_steps += sum(f.result() for f in finished)
        elapsed = time.perf_counter() - t0
        return {"fast_steps": done_steps, "sequences": used, "seconds": elapsed, "workers": self.workers}

    def close(self):
        self._ex.shutdown()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
