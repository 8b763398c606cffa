"""Pins of the seeded input generators (they hold no estimator arithmetic)."""
import numpy as np
import scipy.linalg

from paper_2410_00627_gb300 import synth


def test_ab_kinetics_transition_is_bateman_closed_form():
    """F = expm(K dt) for A->B kinetics has the Bateman closed form."""
    p = synth.ab_kinetics(seed=0, n_slow=5)
    k1, k2, dt = 0.5, 0.2, 0.1
    e1, e2 = np.exp(-k1 * dt), np.exp(-k2 * dt)
    F = np.array([[e1, 0.0], [k1 * (e1 - e2) / (k2 - k1), e2]])
    assert np.allclose(p.F, F, rtol=0, atol=1e-15)


def test_simulation_matches_stepwise_recursion():
    """The vectorised simulator equals the step-by-step loop driven by the same draws."""
    p = synth.random_model(9, 3, 2, 4, 7)
    rng = np.random.default_rng(9)
    # replay the generator's draw order: model draws, then x0, w, v
    n, m, l, N = 3, 2, 4, 7
    rng.standard_normal((n, n)); rng.standard_normal((n, n)); rng.standard_normal((m, m))
    rng.standard_normal((m, n)); rng.standard_normal(n); rng.standard_normal((n, n))
    x0 = p.m0 + np.linalg.cholesky(p.P0) @ rng.standard_normal(n)
    w = rng.standard_normal((N, l, n)) @ np.linalg.cholesky(p.Q).T
    v = rng.standard_normal((N, m)) @ np.linalg.cholesky(p.R).T
    x = [x0]
    y = np.zeros((N, m))
    for k in range(N):
        s = np.zeros(n)
        for i in range(l):
            x.append(p.F @ x[-1] + w[k, i])
            s += x[-1]
        y[k] = p.H @ s + v[k]
    assert np.allclose(np.array(x), p.x, atol=1e-12)
    assert np.allclose(y, p.y, atol=1e-12)


def test_workload_shapes_and_structure():
    p2 = synth.chain4(seed=0, n_slow=50)
    assert p2.F.shape == (4, 4) and p2.H.shape == (2, 4) and p2.ratio == 20
    K = p2.meta["K"]
    assert np.allclose(np.triu(K, 1), 0) and np.allclose(np.tril(K, -2), 0)
    assert np.all((p2.meta["rates"] >= 0.05) & (p2.meta["rates"] <= 1.0))
    p3 = synth.network8(seed=0, n_slow=10)
    K3 = p3.meta["K"]
    assert np.max(np.linalg.eigvalsh(K3 + K3.T)) < 0
    assert np.max(np.real(np.linalg.eigvals(K3))) < 0
    p5 = synth.stiff_chain6(seed=0, n_slow=10)
    assert p5.ratio == 100 and p5.F.shape == (6, 6)
    assert np.allclose(p5.F, scipy.linalg.expm(p5.meta["K"] * 0.01))
    b = synth.ragged_chains(seed=0, n_seq=8, n_min=10, n_max=30)
    assert len(b) == 8 and all(q.ratio in (5, 10, 20) for q in b)
    assert all(10 <= q.n_slow <= 30 for q in b) and all(q.H.shape == (1, 4) for q in b)


def test_ragged_chains_parallel_build_equals_serial_and_packs():
    a = synth.ragged_chains(seed=3, n_seq=12, n_min=5, n_max=40)
    b = synth.ragged_chains(seed=3, n_seq=12, n_min=5, n_max=40, workers=2)
    assert len(a) == len(b) == 12
    for p, q in zip(a, b):
        assert p.ratio == q.ratio and np.array_equal(p.y, q.y) and np.array_equal(p.F, q.F)
    pk = synth.pack(a)
    assert pk["F"].shape == (12, 4, 4) and pk["H"].shape == (12, 1, 4) and pk["m0"].shape == (12, 4)
    assert pk["y"].shape == (pk["total_slow"], 1) and pk["ratio"].dtype == np.int32
    assert pk["total_fast"] == sum(p.n_slow * p.ratio for p in a)
    off = np.concatenate([[0], np.cumsum(pk["n_slow"])])
    for s, p in enumerate(a):
        assert np.array_equal(pk["y"][off[s]:off[s + 1]], p.y)


def test_simulation_with_inputs_matches_stepwise_recursion():
    """x_{t+1} = F x_t + B u_t + w_t: the vectorised simulator equals the step loop."""
    p = synth.random_model(17, 3, 2, 4, 6, nu=2)
    n, m, l, N = 3, 2, 4, 6
    y, x = synth.simulate(np.random.default_rng(5), p.F, p.Q, p.H, p.R, p.m0, p.P0, l, N, True, p.B, p.u)
    rng = np.random.default_rng(5)
    x0 = p.m0 + np.linalg.cholesky(p.P0) @ rng.standard_normal(n)
    w = (rng.standard_normal((N * l, n)) @ np.linalg.cholesky(p.Q).T)
    v = rng.standard_normal((N, m)) @ np.linalg.cholesky(p.R).T
    xs, yy = [x0], np.zeros((N, m))
    for t in range(N * l):
        xs.append(p.F @ xs[-1] + p.B @ p.u[t] + w[t])
        if (t + 1) % l == 0:
            yy[t // l] = p.H @ np.sum(xs[-l:], axis=0) + v[t // l]
    assert np.allclose(x, np.array(xs), rtol=0, atol=1e-12)
    assert np.allclose(y, yy, rtol=0, atol=1e-12)
