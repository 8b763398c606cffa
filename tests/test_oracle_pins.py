"""Pins of the FP64 CPU oracle against things other than itself.

Each pin is chosen so that a plausible slip in the oracle (a dropped term, a
wrong sign or index, a transposed operand) fails at least one of them:

* brute-force dense joint-Gaussian posteriors over all stacked fast states
  (tests/brute.py) for the filter (Eq. 17), the slow IMKF (Eq. 12), the
  sequential smoother (Eq. 21, 22) and the parallel form (Eq. 25-30);
* the textbook Kalman filter + RTS smoother when the ratio l is 1 (Sec. III-C
  notes that l=1 is the standard RTS case);
* the lifted slow-rate constants (Eq. 7-11) read off the joint prior;
* with no process noise (Q = 0), the filter equals the linear-regression
  posterior of x_0 on the stacked measurements, pushed through A^t;
* with uninformative measurements (R = 10^14 I) every filtered and smoothed
  moment equals the prior marginal of its fast state;
* on data drawn from the model, the normalised squared error of every fast
  state averages nx (filtered and smoothed), tying the generator to the oracle;
* a non-orthogonal change of state and measurement coordinates maps every
  mean and covariance as it must, and shifts the log likelihood by the
  Jacobian term -N log |det S|;
* the discrete algebraic Riccati equation with cross term (scipy) as the
  steady state of the slow filter covariance;
* associativity and the identity of both operators (Eq. 27, 30), and each
  operator against what its elements mean (Gaussian conditioning and
  marginalisation written out in information form);
* invariants: symmetry, PSD, smoothed == filtered on the last interval
  (E_N = 0, Eq. 29), smoothed covariance <= filtered covariance;
* a planted mistake (the printed S_k without the transpose) must fail the
  brute-force pin.
"""
import numpy as np
import pytest
import scipy.linalg

from paper_2410_00627_gb300 import synth
from tests import brute


def rel_mean(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


def rel_cov(a, b):
    return np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-300)


TINY = [
    dict(seed=1, nx=1, ny=1, ratio=3, n_slow=4),
    dict(seed=2, nx=2, ny=1, ratio=1, n_slow=5),
    dict(seed=3, nx=3, ny=2, ratio=4, n_slow=5),
    dict(seed=4, nx=2, ny=2, ratio=2, n_slow=1),
    dict(seed=5, nx=3, ny=1, ratio=5, n_slow=3),
    dict(seed=6, nx=4, ny=3, ratio=2, n_slow=4),
]


@pytest.mark.parametrize("kw", TINY, ids=lambda k: "n{nx}m{ny}l{ratio}N{n_slow}".format(**k))
def test_sequential_matches_brute_force(oracle_mod, kw):
    prob = synth.random_model(kw["seed"], kw["nx"], kw["ny"], kw["ratio"], kw["n_slow"])
    ref = brute.posteriors(prob)
    out = oracle_mod.sequential(prob)
    l, n = prob.ratio, prob.nx
    for key in ["fast_filt_mean", "fast_smooth_mean"]:
        assert rel_mean(out[key], ref[key]) < 1e-11, key
    for key in ["fast_filt_cov", "fast_smooth_cov"]:
        assert rel_cov(out[key], ref[key]) < 1e-11, key
    # slow IMKF (Eq. 12) = x_{k,l} | y_{1:k};  first smoothed state (Eq. 22) = x_{k,1} | y_{1:N}
    last = np.arange(prob.n_slow) * l + (l - 1)
    first = np.arange(prob.n_slow) * l
    assert rel_mean(out["slow_filt_mean"], ref["fast_filt_mean"][last]) < 1e-11
    assert rel_cov(out["slow_filt_cov"], ref["fast_filt_cov"][last]) < 1e-11
    assert rel_mean(out["first_smooth_mean"], ref["fast_smooth_mean"][first]) < 1e-11
    assert rel_cov(out["first_smooth_cov"], ref["fast_smooth_cov"][first]) < 1e-11
    assert out["fast_filt_cov"].shape == (prob.n_slow * l, n, n)


@pytest.mark.parametrize("kw", TINY, ids=lambda k: "n{nx}m{ny}l{ratio}N{n_slow}".format(**k))
@pytest.mark.parametrize("order", [0, 1])
def test_parallel_form_matches_brute_force(oracle_mod, kw, order):
    prob = synth.random_model(kw["seed"], kw["nx"], kw["ny"], kw["ratio"], kw["n_slow"])
    ref = brute.posteriors(prob)
    out = oracle_mod.parallel(prob, order=order)
    l = prob.ratio
    last = np.arange(prob.n_slow) * l + (l - 1)
    first = np.arange(prob.n_slow) * l
    assert rel_mean(out["slow_filt_mean"], ref["fast_filt_mean"][last]) < 1e-10
    assert rel_cov(out["slow_filt_cov"], ref["fast_filt_cov"][last]) < 1e-10
    assert rel_mean(out["first_smooth_mean"], ref["fast_smooth_mean"][first]) < 1e-10
    assert rel_cov(out["first_smooth_cov"], ref["fast_smooth_cov"][first]) < 1e-10


def test_printed_sk_without_transpose_fails_brute_force(oracle_mod):
    """Plants the printed S_k = P^f_{k,1} - E_k A P^f_{k,1,l} (no transpose) in the
    oracle's parallel smoother and shows the brute-force pin rejects it, while
    the transposed reading passes (the reading this build takes, Eq. 29)."""
    prob = synth.random_model(3, 3, 2, 4, 5)
    ref = brute.posteriors(prob)
    first = np.arange(prob.n_slow) * prob.ratio
    good = oracle_mod.parallel(prob, order=0, flags=0)
    bad = oracle_mod.parallel(prob, order=0, flags=1)
    assert rel_cov(good["first_smooth_cov"], ref["fast_smooth_cov"][first]) < 1e-10
    assert rel_cov(bad["first_smooth_cov"], ref["fast_smooth_cov"][first]) > 1e-4


def textbook_kf_rts(F, Q, H, R, m0, P0, y):
    """Standard Kalman filter + RTS smoother (x_k = F x_{k-1} + w, y_k = H x_k + v)."""
    N, n = y.shape[0], F.shape[0]
    mf = np.zeros((N, n)); Pf = np.zeros((N, n, n))
    mp = np.zeros((N, n)); Pp = np.zeros((N, n, n))
    m, P = m0, P0
    for k in range(N):
        m, P = F @ m, F @ P @ F.T + Q
        mp[k], Pp[k] = m, P
        S = H @ P @ H.T + R
        K = np.linalg.solve(S, H @ P).T
        m = m + K @ (y[k] - H @ m)
        P = P - K @ S @ K.T
        mf[k], Pf[k] = m, P
    ms = mf.copy(); Ps = Pf.copy()
    for k in range(N - 2, -1, -1):
        G = np.linalg.solve(Pp[k + 1], F @ Pf[k]).T
        ms[k] = mf[k] + G @ (ms[k + 1] - mp[k + 1])
        Ps[k] = Pf[k] + G @ (Ps[k + 1] - Pp[k + 1]) @ G.T
    return mf, Pf, ms, Ps


@pytest.mark.parametrize("seed,nx,ny", [(11, 2, 1), (12, 3, 2), (13, 4, 4)])
def test_ratio_one_is_textbook_kalman_rts(oracle_mod, seed, nx, ny):
    prob = synth.random_model(seed, nx, ny, 1, 60)
    mf, Pf, ms, Ps = textbook_kf_rts(prob.F, prob.Q, prob.H, prob.R, prob.m0, prob.P0, prob.y)
    out = oracle_mod.sequential(prob)
    assert rel_mean(out["fast_filt_mean"], mf) < 1e-11
    assert rel_cov(out["fast_filt_cov"], Pf) < 1e-11
    assert rel_mean(out["slow_filt_mean"], mf) < 1e-11
    assert rel_mean(out["fast_smooth_mean"], ms) < 1e-10
    assert rel_cov(out["fast_smooth_cov"], Ps) < 1e-10
    par = oracle_mod.parallel(prob, order=1)
    assert rel_mean(par["first_smooth_mean"], ms) < 1e-10
    assert rel_cov(par["first_smooth_cov"], Ps) < 1e-10


@pytest.mark.parametrize("seed,nx,ny,l", [(21, 2, 1, 3), (22, 3, 2, 5), (23, 4, 2, 20)])
def test_lifted_constants_from_joint_prior(oracle_mod, seed, nx, ny, l):
    """With x_{k-1,l} known, (x_{k,l}, y_k) has covariance [[Qbar, GQM],[GQM^T, MQM+R]]
    and means (Abar x, Cbar x): read them off the joint prior of one interval."""
    prob = synth.random_model(seed, nx, ny, l, 1)
    lift = oracle_mod.lifted(prob.F, prob.Q, prob.H, l)
    n = nx
    mu, S = brute.joint_prior(prob.F, prob.Q, np.zeros(n), np.zeros((n, n)), l)
    Hz = brute.meas_matrix(prob.H, n, l, 1)
    xl = slice(l * n, (l + 1) * n)
    assert np.allclose(lift["Qbar"], S[xl, xl], rtol=0, atol=1e-13 * np.abs(S).max())
    assert np.allclose(lift["MQM"], Hz @ S @ Hz.T, rtol=0, atol=1e-13 * np.abs(Hz @ S @ Hz.T).max())
    assert np.allclose(lift["GQM"], S[xl] @ Hz.T, rtol=0, atol=1e-13 * np.abs(S[xl] @ Hz.T).max())
    # means are linear in x_0: use the transition maps of the unrolled prior
    e = np.eye(n)
    Ab = np.stack([brute.joint_prior(prob.F, prob.Q, e[j], np.zeros((n, n)), l)[0][xl] for j in range(n)], 1)
    Cb = np.stack([Hz @ brute.joint_prior(prob.F, prob.Q, e[j], np.zeros((n, n)), l)[0] for j in range(n)], 1)
    assert np.allclose(lift["Abar"], Ab, atol=1e-13)
    assert np.allclose(lift["Cbar"], Cb, atol=1e-12 * max(1, np.abs(Cb).max()))


@pytest.mark.parametrize("name", ["ab_kinetics", "chain4"])
def test_slow_filter_reaches_dare(oracle_mod, name):
    """The IMKF covariance converges to the DARE solution with cross term
    S = G Q~ M^T:  X = A X A^T + Qbar - (A X C^T + S)(C X C^T + R_x)^{-1}(.)^T."""
    prob = synth.WORKLOADS[name](seed=0, n_slow=400, keep_states=False)
    lift = oracle_mod.lifted(prob.F, prob.Q, prob.H, prob.ratio)
    X = scipy.linalg.solve_discrete_are(lift["Abar"].T, lift["Cbar"].T, lift["Qbar"],
                                        lift["MQM"] + prob.R, s=lift["GQM"])
    out = oracle_mod.sequential(prob, fast=False, smooth=False)
    assert rel_cov(out["slow_filt_cov"][-1], X) < 1e-9


def _random_filter_element(rng, n):
    G1, G2 = rng.standard_normal((n, n)), rng.standard_normal((n, n))
    return {"F": rng.standard_normal((n, n)) * 0.7, "d": rng.standard_normal(n),
            "D": G1 @ G1.T / n, "eta": rng.standard_normal(n), "J": G2 @ G2.T / n}


@pytest.mark.parametrize("n", [1, 2, 4, 6])
def test_filter_operator_associative_with_identity(oracle_mod, n):
    rng = np.random.default_rng(n)
    a, b, c = (_random_filter_element(rng, n) for _ in range(3))
    left = oracle_mod.filter_op(oracle_mod.filter_op(a, b), c)
    right = oracle_mod.filter_op(a, oracle_mod.filter_op(b, c))
    for k in left:
        assert np.allclose(left[k], right[k], rtol=1e-10, atol=1e-10), k
    ident = {"F": np.eye(n), "d": np.zeros(n), "D": np.zeros((n, n)), "eta": np.zeros(n), "J": np.zeros((n, n))}
    for x in (oracle_mod.filter_op(ident, a), oracle_mod.filter_op(a, ident)):
        for k in x:
            assert np.allclose(x[k], a[k], rtol=1e-13, atol=1e-13), k


@pytest.mark.parametrize("n", [1, 3, 8])
def test_smoother_operator_associative_with_identity(oracle_mod, n):
    rng = np.random.default_rng(100 + n)

    def el():
        G = rng.standard_normal((n, n))
        return {"E": rng.standard_normal((n, n)) * 0.5, "g": rng.standard_normal(n), "S": G @ G.T}

    a, b, c = el(), el(), el()
    left = oracle_mod.smoother_op(oracle_mod.smoother_op(a, b), c)
    right = oracle_mod.smoother_op(a, oracle_mod.smoother_op(b, c))
    for k in left:
        assert np.allclose(left[k], right[k], rtol=1e-12, atol=1e-12), k
    ident = {"E": np.eye(n), "g": np.zeros(n), "S": np.zeros((n, n))}
    for x in (oracle_mod.smoother_op(ident, a), oracle_mod.smoother_op(a, ident)):
        for k in x:
            assert np.allclose(x[k], a[k], atol=1e-14), k


@pytest.mark.parametrize("name,n_slow", [("ab_kinetics", 100), ("chain4", 150)])
def test_parallel_equals_sequential_midsize(oracle_mod, name, n_slow):
    """The paper states the parallel and sequential forms give identical results."""
    prob = synth.WORKLOADS[name](seed=3, n_slow=n_slow, keep_states=False)
    seq = oracle_mod.sequential(prob, fast=False)
    for order in (0, 1):
        par = oracle_mod.parallel(prob, order=order)
        for k in ["slow_filt_mean", "first_smooth_mean"]:
            assert rel_mean(par[k], seq[k]) < 1e-10, (k, order)
        for k in ["slow_filt_cov", "first_smooth_cov"]:
            assert rel_cov(par[k], seq[k]) < 1e-10, (k, order)


@pytest.mark.parametrize("name", ["ab_kinetics", "chain4"])
def test_invariants(oracle_mod, name):
    prob = synth.WORKLOADS[name](seed=5, n_slow=60, keep_states=False)
    out = oracle_mod.sequential(prob)
    l = prob.ratio
    for key in ["fast_filt_cov", "fast_smooth_cov", "slow_filt_cov", "first_smooth_cov"]:
        P = out[key]
        assert np.max(np.abs(P - np.swapaxes(P, 1, 2))) <= 1e-12 * np.abs(P).max(), key
        ev = np.linalg.eigvalsh(0.5 * (P + np.swapaxes(P, 1, 2)))
        assert ev.min() >= -1e-12 * np.abs(P).max(), key
    # last interval: smoothed == filtered (E_N = 0)
    assert np.array_equal(out["fast_smooth_mean"][-l:], out["fast_filt_mean"][-l:])
    assert np.array_equal(out["fast_smooth_cov"][-l:], out["fast_filt_cov"][-l:])
    # smoothing never increases uncertainty
    d = out["fast_filt_cov"] - out["fast_smooth_cov"]
    ev = np.linalg.eigvalsh(0.5 * (d + np.swapaxes(d, 1, 2)))
    assert ev.min() >= -1e-10 * np.abs(out["fast_filt_cov"]).max()
    # slow IMKF == last block of the fast filter (two derivations of the same quantity)
    assert rel_mean(out["slow_filt_mean"], out["fast_filt_mean"][l - 1::l]) < 1e-12
    assert rel_cov(out["slow_filt_cov"], out["fast_filt_cov"][l - 1::l]) < 1e-11


def test_sampled_fast_range_matches_full(oracle_mod):
    prob = synth.chain4(seed=7, n_slow=30, keep_states=False)
    full = oracle_mod.sequential(prob)
    part = oracle_mod.sequential(prob, k_lo=10, k_hi=13)
    l = prob.ratio
    for k in ["fast_filt_mean", "fast_filt_cov", "fast_smooth_mean", "fast_smooth_cov"]:
        assert np.array_equal(part[k], full[k][10 * l:13 * l]), k


# --------------------------------------------------------------------------- log marginal likelihood
@pytest.mark.parametrize("kw", TINY, ids=lambda k: "n{nx}m{ny}l{ratio}N{n_slow}".format(**k))
def test_loglik_matches_dense_joint_density(oracle_mod, kw):
    """log p(y_{1:N}) from the IMKF's prediction-error decomposition equals the
    log density of the stacked measurements under the dense joint prior."""
    prob = synth.random_model(kw["seed"], kw["nx"], kw["ny"], kw["ratio"], kw["n_slow"])
    total, terms = oracle_mod.loglik(prob, terms=True)
    ref = brute.loglik(prob)
    assert abs(total - ref) <= 1e-10 * max(1.0, abs(ref))
    assert np.isclose(terms.sum(), total, rtol=0, atol=1e-12 * max(1.0, abs(total)))


def test_loglik_first_term_is_the_prior_predictive(oracle_mod):
    """The k = 1 term is log N(y_1; C_bar m0, C_bar P0 C_bar^T + M Q~ M^T + R): with
    n = m = 1 every piece is a scalar written out by hand."""
    prob = synth.random_model(31, 1, 1, 3, 2)
    a, q, h, r = prob.F[0, 0], prob.Q[0, 0], prob.H[0, 0], prob.R[0, 0]
    l = prob.ratio
    # y_1 = h (x_1 + x_2 + x_3) + v with x_i = a^i x_0 + sum_{s<i} a^{i-1-s} w_s
    c = h * sum(a ** i for i in range(1, l + 1))
    var_w = q * h * h * sum(sum(a ** (i - 1 - s) for i in range(s + 1, l + 1)) ** 2 for s in range(l))
    mean = c * prob.m0[0]
    var = c * c * prob.P0[0, 0] + var_w + r
    want = -0.5 * (np.log(2 * np.pi * var) + (prob.y[0, 0] - mean) ** 2 / var)
    _, terms = oracle_mod.loglik(prob, terms=True)
    assert abs(terms[0] - want) <= 1e-12 * max(1.0, abs(want))


def test_planted_loglik_mistake_fails_the_dense_pin(oracle_mod):
    """A total that drops the normalising constant -N m log(2 pi) / 2 (a
    plausible slip) is rejected by the dense pin that the oracle passes."""
    prob = synth.random_model(3, 3, 2, 4, 5)
    total, terms = oracle_mod.loglik(prob, terms=True)
    ref = brute.loglik(prob)
    assert abs(total - ref) < 1e-10 * abs(ref)
    N, m = prob.y.shape
    assert abs((total + 0.5 * N * m * np.log(2 * np.pi)) - ref) > 1e-3 * abs(ref)


# --------------------------------------------------------------------------- known inputs (B u)
TINY_U = [
    dict(seed=41, nx=2, ny=1, ratio=3, n_slow=4, nu=1),
    dict(seed=42, nx=3, ny=2, ratio=4, n_slow=5, nu=2),
    dict(seed=43, nx=1, ny=1, ratio=1, n_slow=6, nu=1),
    dict(seed=44, nx=4, ny=3, ratio=2, n_slow=3, nu=3),
]


@pytest.mark.parametrize("kw", TINY_U, ids=lambda k: "n{nx}m{ny}l{ratio}N{n_slow}u{nu}".format(**k))
def test_inputs_sequential_and_parallel_match_brute_force(oracle_mod, kw):
    """With x_{t+1} = F x_t + B u_t + w_t the filter, the smoother, their
    parallel forms and log p(y_1:N) match the dense joint posterior."""
    prob = synth.random_model(kw["seed"], kw["nx"], kw["ny"], kw["ratio"], kw["n_slow"], nu=kw["nu"])
    ref = brute.posteriors(prob)
    out = oracle_mod.sequential(prob)
    for key in ["fast_filt_mean", "fast_smooth_mean"]:
        assert rel_mean(out[key], ref[key]) < 1e-11, key
    for key in ["fast_filt_cov", "fast_smooth_cov"]:
        assert rel_cov(out[key], ref[key]) < 1e-11, key
    l = prob.ratio
    par = oracle_mod.parallel(prob, order=1)
    assert rel_mean(par["slow_filt_mean"], ref["fast_filt_mean"][l - 1::l]) < 1e-11
    assert rel_mean(par["first_smooth_mean"], ref["fast_smooth_mean"][0::l]) < 1e-11
    assert abs(oracle_mod.loglik(prob) - brute.loglik(prob)) < 1e-10 * abs(brute.loglik(prob))


def test_zero_inputs_equal_no_inputs(oracle_mod):
    prob = synth.random_model(45, 3, 2, 4, 6, nu=2)
    base = synth.random_model(45, 3, 2, 4, 6, nu=2)
    base.u = np.zeros_like(base.u)
    plain = synth.Problem(base.F, base.Q, base.H, base.R, base.m0, base.P0, base.y, base.ratio)
    a, b = oracle_mod.sequential(base), oracle_mod.sequential(plain)
    for k in a:
        assert np.array_equal(a[k], b[k]), k
    assert oracle_mod.loglik(base) == oracle_mod.loglik(plain)
    # and the inputs matter when they are not zero
    assert rel_mean(oracle_mod.sequential(prob)["fast_smooth_mean"], b["fast_smooth_mean"]) > 1e-3


@pytest.mark.parametrize("seed,nx,ny,l,N", [(74, 3, 2, 4, 25), (76, 2, 1, 7, 12)])
def test_noise_free_dynamics_filter_is_regression_on_x0(oracle_mod, seed, nx, ny, l, N):
    """With Q = 0 every fast state is A^t x_0, so p(x_{k,i} | y_{1:k}) is the
    Gaussian linear-regression posterior of x_0 on the stacked y_1..y_k
    (y_j = H sum_i A^{(j-1)l+i} x_0 + v_j), pushed through A^t.  The fast-rate
    filter (Eq. 17) and the slow IMKF (Eq. 9-12) must reproduce it."""
    prob = synth.random_model(seed, nx, ny, l, N)
    prob.Q = np.zeros((nx, nx))
    A, H, R = prob.F, prob.H, prob.R
    o = oracle_mod.sequential(prob)
    Ap = [np.eye(nx)]
    for _ in range(N * l):
        Ap.append(A @ Ap[-1])
    C = np.vstack([H @ sum(Ap[(j - 1) * l + i] for i in range(1, l + 1)) for j in range(1, N + 1)])
    for k in range(1, N + 1):
        Ck, Rk = C[:k * ny], np.kron(np.eye(k), R)
        S = Ck @ prob.P0 @ Ck.T + Rk
        G = np.linalg.solve(S, Ck @ prob.P0).T
        mx = prob.m0 + G @ (prob.y[:k].reshape(-1) - Ck @ prob.m0)
        Px = prob.P0 - G @ Ck @ prob.P0
        for i in range(1, l + 1):
            t = (k - 1) * l + i
            assert rel_mean(o["fast_filt_mean"][t - 1], Ap[t] @ mx) < 1e-10, (k, i)
            assert rel_cov(o["fast_filt_cov"][t - 1], Ap[t] @ Px @ Ap[t].T) < 1e-9, (k, i)
        assert rel_cov(o["slow_filt_cov"][k - 1], Ap[k * l] @ Px @ Ap[k * l].T) < 1e-9, k


def _similarity(prob, T, S):
    """The same model in state coordinates x' = T x and measurement
    coordinates y' = S y (inputs enter through B' = T B)."""
    import copy
    Ti = np.linalg.inv(T)
    q = copy.copy(prob)
    q.F, q.Q, q.H = T @ prob.F @ Ti, T @ prob.Q @ T.T, S @ prob.H @ Ti
    q.R, q.m0, q.P0 = S @ prob.R @ S.T, T @ prob.m0, T @ prob.P0 @ T.T
    q.y = prob.y @ S.T
    if getattr(prob, "B", None) is not None:
        q.B = T @ prob.B
    return q


@pytest.mark.parametrize("seed,nx,ny,l,N,nu", [(81, 4, 2, 5, 60, 0), (82, 3, 3, 7, 40, 2), (83, 6, 1, 3, 50, 1)])
def test_posterior_transforms_under_a_change_of_coordinates(oracle_mod, seed, nx, ny, l, N, nu):
    """Filtering and smoothing commute with an invertible, non-orthogonal change
    of state coordinates T and of measurement coordinates S: every mean maps to
    T m and every covariance to T P T^T (a misplaced transpose of a
    non-symmetric factor such as A or H breaks this), and log p(y'_{1:N}) = log p(y_{1:N}) -
    N log |det S| (the Jacobian of y' = S y)."""
    prob = synth.random_model(seed, nx, ny, l, N, nu=nu)
    rng = np.random.default_rng(seed)
    T = np.eye(nx) + 0.6 * rng.standard_normal((nx, nx))
    S = np.eye(ny) + 0.6 * rng.standard_normal((ny, ny))
    assert min(abs(np.linalg.det(T)), abs(np.linalg.det(S))) > 0.05
    a = oracle_mod.sequential(prob)
    b = oracle_mod.sequential(_similarity(prob, T, S))
    for k in ("slow_filt", "first_smooth", "fast_filt", "fast_smooth"):
        assert rel_mean(b[k + "_mean"], a[k + "_mean"] @ T.T) < 1e-10, k
        assert rel_cov(b[k + "_cov"], np.einsum("ij,tjk,lk->til", T, a[k + "_cov"], T)) < 1e-10, k
    la = oracle_mod.loglik(prob)
    lb = oracle_mod.loglik(_similarity(prob, T, S))
    assert abs(lb - (la - N * np.log(abs(np.linalg.det(S))))) < 1e-9 * max(1.0, abs(la))


@pytest.mark.parametrize("seed,nx,ny,l,N,nu", [(84, 4, 2, 20, 40, 0), (85, 3, 1, 6, 30, 2)])
def test_uninformative_measurements_give_the_prior_marginals(oracle_mod, seed, nx, ny, l, N, nu):
    """With R = 10^14 I the measurements carry no information (relative weight
    ~1e-13): filtered and smoothed moments of every fast state equal the prior
    marginals m_t = A m_{t-1} + B u_{t-1}, P_t = A P_{t-1} A^T + Q from (m0, P0)."""
    prob = synth.random_model(seed, nx, ny, l, N, nu=nu)
    prob.R = 1e14 * np.eye(ny)
    o = oracle_mod.sequential(prob)
    m, P = prob.m0.copy(), prob.P0.copy()
    pm, pP = [], []
    for t in range(N * l):
        m = prob.F @ m + (prob.B @ prob.u[t] if nu else 0.0)
        P = prob.F @ P @ prob.F.T + prob.Q
        pm.append(m)
        pP.append(P)
    pm, pP = np.array(pm), np.array(pP)
    for k in ("fast_filt", "fast_smooth"):
        assert rel_mean(o[k + "_mean"], pm) < 1e-9, k
        assert rel_cov(o[k + "_cov"], pP) < 1e-9, k
    assert rel_cov(o["slow_filt_cov"], pP[l - 1::l]) < 1e-9


@pytest.mark.parametrize("make", [lambda: synth.chain4(seed=3, n_slow=2000),
                                  lambda: synth.random_model(61, 3, 2, 5, 2000, nu=2),
                                  lambda: synth.ab_kinetics(seed=2, n_slow=3000)],
                         ids=["chain4", "random_inputs", "ab_kinetics"])
def test_posterior_is_calibrated_against_the_simulated_states(oracle_mod, make):
    """On data drawn from the model itself, the normalised squared error of
    every fast state, (x - m)^T P^-1 (x - m), averages nx for the filtered and
    the smoothed posteriors (a consistent estimator), and smoothing lowers the
    mean squared error.  Ties the generator's model (H on the sum, noise
    scales, input timing) to the oracle's: reading H as acting on the mean
    gives a ratio near 200 on chain4, halving Q a ratio near 2."""
    p = make()
    o = oracle_mod.sequential(p)
    x = p.x[1:]                       # x_{k,i} in the fast-output row order
    mse = {}
    for k in ("fast_filt", "fast_smooth"):
        e = x - o[k + "_mean"]
        nees = np.einsum("ti,tij,tj->t", e, np.linalg.inv(o[k + "_cov"]), e)
        assert 0.9 < nees.mean() / p.nx < 1.1, (k, nees.mean() / p.nx)
        mse[k] = np.mean(e ** 2)
    assert mse["fast_smooth"] < mse["fast_filt"]


@pytest.mark.parametrize("n", [1, 2, 4, 6])
def test_filter_operator_is_gaussian_conditioning_and_marginalisation(oracle_mod, n):
    """Eq. (27) from what an element means: a_k = (F, d, D, eta, J) holds
    p(x_k | x_{k-1}) = N(F x_{k-1} + d, D) and the likelihood of its
    measurements as a function of x_{k-1}, exp(-x^T J x / 2 + eta^T x).  For
    a_i (x_{i-1} -> x_i) then a_j (x_i -> x_j), textbook Gaussian algebra gives
    p(x_j | x_{i-1}): condition x_i ~ N(F_i x + d_i, D_i) on the factor of a_j
    (precision D_i^-1 + J_j), push it through F_j and add D_j; and the
    likelihood of x_{i-1}: a_i's factor times the Gaussian integral over x_i.
    The combined element must reproduce both for any x_{i-1}."""
    rng = np.random.default_rng(300 + n)
    ai, aj = _random_filter_element(rng, n), _random_filter_element(rng, n)
    ai["D"] = ai["D"] + 0.3 * np.eye(n)   # the information form below inverts D_i: keep it well conditioned
    c = oracle_mod.filter_op(ai, aj)
    Di_inv = np.linalg.inv(ai["D"])
    Lam = Di_inv + aj["J"]
    Sig = np.linalg.inv(Lam)

    def log_lik(x):   # log of a_i's factor times the integral over x_i, up to a constant
        m = ai["F"] @ x + ai["d"]
        h = Di_inv @ m + aj["eta"]
        return (-0.5 * x @ ai["J"] @ x + ai["eta"] @ x
                + 0.5 * h @ Sig @ h - 0.5 * m @ Di_inv @ m)

    base = log_lik(np.zeros(n))
    for _ in range(5):
        x = rng.standard_normal(n)
        mu = Sig @ (Di_inv @ (ai["F"] @ x + ai["d"]) + aj["eta"])
        assert np.allclose(c["F"] @ x + c["d"], aj["F"] @ mu + aj["d"], rtol=1e-10, atol=1e-10)
        want = -0.5 * x @ c["J"] @ x + c["eta"] @ x
        assert abs((log_lik(x) - base) - want) < 1e-9 * max(1.0, abs(want))
    assert np.allclose(c["D"], aj["F"] @ Sig @ aj["F"].T + aj["D"], rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("n", [1, 3, 5])
def test_smoother_operator_is_backward_conditional_composition(oracle_mod, n):
    """Eq. (30) from what an element means: a_k = (E, g, S) holds
    p(x_k | x_{k+1}) = N(E x_{k+1} + g, S).  Composing a_i (x_i | x_j) with
    a_j (x_j | x_k) by marginalising x_j gives N(E_i (E_j x + g_j) + g_i,
    E_i S_j E_i^T + S_i), which the combined element must be."""
    rng = np.random.default_rng(400 + n)

    def el():
        G = rng.standard_normal((n, n))
        return {"E": rng.standard_normal((n, n)) * 0.5, "g": rng.standard_normal(n), "S": G @ G.T}

    ai, aj = el(), el()
    c = oracle_mod.smoother_op(ai, aj)
    for _ in range(3):
        x = rng.standard_normal(n)
        assert np.allclose(c["E"] @ x + c["g"], ai["E"] @ (aj["E"] @ x + aj["g"]) + ai["g"], rtol=1e-12, atol=1e-12)
    assert np.allclose(c["S"], ai["E"] @ aj["S"] @ ai["E"].T + ai["S"], rtol=1e-12, atol=1e-12)
