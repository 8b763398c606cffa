"""The oracle against a second, independent algorithm: the augmented-state
Kalman filter + RTS smoother of ``oracle/augmented.py`` (the state augmented
with the running sum of the interval's fast states, the alternative the paper
names in the footnote to its dual-rate reformulation, Sec. II).  Unlike the
brute-force joint posterior it scales to hundreds of slow steps, so it pins
the oracle at the sizes the GPU parity tests use."""
import numpy as np
import pytest

from paper_2410_00627_gb300 import synth
from oracle.augmented import augmented

CASES = [  # (seed, nx, ny, ratio, n_slow, nu)
    (81, 1, 1, 3, 40, 0),
    (82, 2, 1, 1, 60, 0),
    (83, 2, 2, 4, 50, 1),
    (84, 3, 2, 6, 30, 0),
    (85, 4, 1, 5, 40, 2),
    (86, 4, 3, 2, 45, 0),
    (87, 3, 1, 7, 1, 1),
]

KEYS = ("fast_filt_mean", "fast_filt_cov", "slow_filt_mean", "slow_filt_cov", "fast_smooth_mean", "fast_smooth_cov")


def rel(a, b):
    return float(np.max(np.abs(a - b)) / max(float(np.max(np.abs(b))), 1e-300))


@pytest.mark.parametrize("case", CASES, ids=lambda c: "n{1}m{2}l{3}N{4}u{5}".format(*c))
def test_oracle_matches_augmented_state_smoother(oracle_mod, case):
    seed, nx, ny, l, N, nu = case
    prob = synth.random_model(seed, nx, ny, l, N, nu=nu)
    want = augmented(prob)
    got = oracle_mod.sequential(prob)
    for k in KEYS:
        assert rel(got[k], want[k]) < 1e-9, (k, rel(got[k], want[k]))
    assert abs(oracle_mod.loglik(prob) - want["loglik"]) <= 1e-9 * max(1.0, abs(want["loglik"]))


@pytest.mark.parametrize("name,n_slow", [("ab_kinetics", 100), ("chain4", 100)])
def test_oracle_matches_augmented_state_smoother_workloads(oracle_mod, name, n_slow):
    prob = synth.WORKLOADS[name](seed=4, n_slow=n_slow, keep_states=False)
    want = augmented(prob)
    got = oracle_mod.sequential(prob)
    for k in KEYS:
        assert rel(got[k], want[k]) < 1e-9, (k, rel(got[k], want[k]))
    assert abs(oracle_mod.loglik(prob) - want["loglik"]) <= 1e-9 * abs(want["loglik"])


def test_augmented_detects_a_planted_oracle_mistake(oracle_mod):
    """Measurement on the mean instead of the sum (H/l): the kind of slip the
    lifted constants could hide; the augmented posterior rejects it."""
    prob = synth.random_model(88, 3, 2, 4, 20)
    want = augmented(prob)
    wrong = synth.Problem(prob.F, prob.Q, prob.H / prob.ratio, prob.R, prob.m0, prob.P0, prob.y, prob.ratio)
    got = oracle_mod.sequential(wrong)
    assert rel(got["fast_smooth_mean"], want["fast_smooth_mean"]) > 1e-3
