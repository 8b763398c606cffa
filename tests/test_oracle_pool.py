"""The batch CPU baseline's worker pool (oracle/pool.py): spawned workers run
the oracle on whole sequences in order and report the fast steps solved."""
import numpy as np

from paper_2410_00627_gb300 import synth


def test_pool_solves_every_sequence_in_order():
    from oracle.pool import SequencePool
    probs = [synth.random_model(90 + i, 3, 2, 2 + i, 5 + 3 * i, nu=i % 2) for i in range(5)]
    with SequencePool(2) as pool:
        r = pool.run(probs, seconds=60.0)
    assert r["workers"] == 2 and r["sequences"] == 5
    assert r["fast_steps"] == sum(p.n_slow * p.ratio for p in probs)
    assert np.isfinite(r["seconds"]) and r["seconds"] > 0


def test_pool_stops_submitting_after_its_time():
    from oracle.pool import SequencePool
    probs = [synth.random_model(95, 2, 1, 3, 40)] * 200
    with SequencePool(2) as pool:
        r = pool.run(probs, seconds=0.0)
    assert r["sequences"] == 0 and r["fast_steps"] == 0
