"""Seeded synthetic SRTM workloads (linear kinetics) shared by the oracle tests,
the CUDA parity tests and the benchmark.

This module only builds models and simulates data from them: it draws rate
constants, forms the fast transition ``F = expm(K dt)``, and simulates the
fast-rate linear Gaussian system with slow-rate integrated measurements

    x_{t+1} = F x_t + w_t,            w_t ~ N(0, Q)
    y_k     = H sum_{i=1..l} x_{k,i} + v_k,   v_k ~ N(0, R)

(the dual-rate model of Sec. III, with the measurement matrix ``H`` applied
to the *sum* of the ``l`` fast states of interval ``k``; the paper's ``C``
applies to their average, so ``C = l H``).  It contains no filtering or
smoothing arithmetic.

The paper's own benchmark (a CSTR case study whose parameters live in a cited
paper) is not available; these five synthetic families stand in for it:

1. 2-state A->B kinetics, l=10, N=100 (small reference case).
2. 4-species first-order chain, rates log-U[0.05,1], dt=0.05, l=20, ny=2.
3. 8-state random stable network K=-(D+S), l=50, ny=3, dense random H.
4. 4096 ragged chains (nx=4, ny=1), l in {5,10,20}, N ~ U[100,20000].
5. Stiff 6-species chain, rates log-U[1e-3,1e2], dt=0.01, l=100, ny=2.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg


@dataclass
class Problem:
    """One SRTM sequence: model, prior and slow-rate measurements (all float64).

    F: (nx,nx) fast transition.  Q: (nx,nx) fast process-noise covariance.
    H: (ny,nx) applied to the sum of the ``ratio`` fast states of a slow interval.
    R: (ny,ny) measurement-noise covariance.  m0, P0: prior of x_0.
    y: (n_slow, ny) measurements; row k is y_{k+1} in the paper's 1-based index.
    x: optional (n_slow*ratio+1, nx) simulated fast states x_0, x_{1,1}, ..., x_{N,l}.
    B, u: optional known inputs, x_{t+1} = F x_t + B u_t + w_t (Sec. II).
    """

    F: np.ndarray
    Q: np.ndarray
    H: np.ndarray
    R: np.ndarray
    m0: np.ndarray
    P0: np.ndarray
    y: np.ndarray
    ratio: int
    x: np.ndarray | None = None
    name: str = ""
    meta: dict = field(default_factory=dict)
    B: np.ndarray | None = None   # (nx, nu) input matrix, or None
    u: np.ndarray | None = None   # (n_slow*ratio, nu) inputs; row t drives x_{t+1}

    @property
    def nx(self) -> int:
        return self.F.shape[0]

    @property
    def ny(self) -> int:
        return self.H.shape[0]

    @property
    def n_slow(self) -> int:
        return self.y.shape[0]


def chain_rates_matrix(rates: np.ndarray) -> np.ndarray:
    """Lower-bidiagonal first-order chain X1 -> X2 -> ... -> Xn -> (out)."""
    n = len(rates)
    K = np.zeros((n, n))
    for j in range(n):
        K[j, j] = -rates[j]
        if j + 1 < n:
            K[j + 1, j] = rates[j]
    return K


def log_uniform(rng: np.random.Generator, lo: float, hi: float, size) -> np.ndarray:
    return np.exp(rng.uniform(np.log(lo), np.log(hi), size=size))


def simulate(rng: np.random.Generator, F, Q, H, R, m0, P0, ratio: int, n_slow: int,
             keep_states: bool = True, B=None, u=None):
    """Draw x_0 ~ N(m0,P0), run x_{t+1} = F x_t + w_t for n_slow*ratio fast steps
    and form y_k = H sum_{i=1..ratio} x_{k,i} + v_k.

    The fast recursion is evaluated interval by interval, vectorised over the
    intervals: the within-interval noise response e_{k,i} = F e_{k,i-1} + w
    for all k at once, the interval end states by repeated doubling with
    F^ratio, then x_{k,i} = F^i x_{k-1,l} + e_{k,i}.  This is the same sample
    path as the step-by-step loop driven by the same noise draws.
    """
    nx = F.shape[0]
    ny = H.shape[0]
    l, N = ratio, n_slow
    Lq = np.linalg.cholesky(Q)
    Lr = np.linalg.cholesky(R)
    x0 = m0 + np.linalg.cholesky(P0) @ rng.standard_normal(nx)
    w = (rng.standard_normal((N * l, nx)) @ Lq.T).reshape(N, l, nx)   # w[k, i-1]: noise into x_{k,i}
    if B is not None:   # known inputs enter like the noise: B u_t + w_t drives x_{t+1}
        w = w + (u @ B.T).reshape(N, l, nx)
    v = rng.standard_normal((N, ny)) @ Lr.T
    # e[k, i-1] = sum_{r<=i} F^{i-r} w[k, r-1]
    e = np.empty_like(w)
    acc = np.zeros((N, nx))
    for i in range(l):
        acc = acc @ F.T + w[:, i]
        e[:, i] = acc
    # interval end states: z_k = F^l z_{k-1} + e[k, l-1], z_0 = x0  (doubling scan)
    Fl = np.linalg.matrix_power(F, l)
    z = np.concatenate([x0[None], e[:, l - 1]], axis=0)   # z[0]=x0, z[k]=e_k
    Fd = Fl.copy()
    d = 1
    while d < N + 1:
        z[d:] = z[d:] + z[:-d] @ Fd.T
        Fd = Fd @ Fd
        d *= 2
    # fast states x_{k,i} = F^i z_{k-1} + e[k, i-1]
    Fpow = np.empty((l, nx, nx))
    P = np.eye(nx)
    for i in range(l):
        P = F @ P
        Fpow[i] = P
    xs = (z[:-1] @ Fpow.reshape(l * nx, nx).T).reshape(N, l, nx) + e   # (N, l, nx)
    y = xs.sum(axis=1) @ H.T + v
    x = None
    if keep_states:
        x = np.concatenate([x0[None], xs.reshape(N * l, nx)], axis=0)
    return y, x


def ab_kinetics(seed: int = 0, n_slow: int = 100, keep_states: bool = True) -> Problem:
    """2-state A->B kinetics: K=[[-k1,0],[k1,-k2]], k1=.5, k2=.2, dt=.1, l=10,
    Q=.01 I, m0=[1,0], P0=.1 I, y = [0,1] * sum of 10 fast states + N(0, 0.1)."""
    rng = np.random.default_rng(seed)
    k1, k2, dt = 0.5, 0.2, 0.1
    K = np.array([[-k1, 0.0], [k1, -k2]])
    F = scipy.linalg.expm(K * dt)
    Q = 0.01 * np.eye(2)
    H = np.array([[0.0, 1.0]])
    R = np.array([[0.1]])
    m0 = np.array([1.0, 0.0])
    P0 = 0.1 * np.eye(2)
    y, x = simulate(rng, F, Q, H, R, m0, P0, 10, n_slow, keep_states)
    return Problem(F, Q, H, R, m0, P0, y, 10, x, "ab_kinetics", {"K": K, "dt": dt})


def chain4(seed: int = 0, n_slow: int = 10_000, keep_states: bool = True) -> Problem:
    """4-species chain, rates log-U[0.05,1], dt=.05, l=20, H=[e3;e4], Q=1e-3 I,
    R=.05 I, m0=e1, P0=.1 I."""
    rng = np.random.default_rng(seed)
    rates = log_uniform(rng, 0.05, 1.0, 4)
    K = chain_rates_matrix(rates)
    dt = 0.05
    F = scipy.linalg.expm(K * dt)
    Q = 1e-3 * np.eye(4)
    H = np.zeros((2, 4)); H[0, 2] = 1.0; H[1, 3] = 1.0
    R = 0.05 * np.eye(2)
    m0 = np.eye(4)[0]
    P0 = 0.1 * np.eye(4)
    y, x = simulate(rng, F, Q, H, R, m0, P0, 20, n_slow, keep_states)
    return Problem(F, Q, H, R, m0, P0, y, 20, x, "chain4", {"K": K, "dt": dt, "rates": rates})


def network8(seed: int = 0, n_slow: int = 100_000, keep_states: bool = False) -> Problem:
    """8-state stable network K = -(D+S): D diag log-U[.01,2], S 20%-dense N(0,1)
    scaled so ||S||_2 <= 0.5 min(D) (then K+K^T < 0).  l=50, H (3x8) iid N(0,1),
    Q=1e-4 I, R=.01 I, dt=.05, m0=e1, P0=.1 I."""
    rng = np.random.default_rng(seed)
    n = 8
    D = np.diag(log_uniform(rng, 0.01, 2.0, n))
    S = rng.standard_normal((n, n)) * (rng.uniform(size=(n, n)) < 0.2)
    np.fill_diagonal(S, 0.0)
    s2 = np.linalg.norm(S, 2)
    if s2 > 0:
        S *= 0.5 * np.min(np.diag(D)) / s2
    K = -(D + S)
    dt = 0.05
    F = scipy.linalg.expm(K * dt)
    Q = 1e-4 * np.eye(n)
    H = rng.standard_normal((3, n))
    R = 0.01 * np.eye(3)
    m0 = np.eye(n)[0]
    P0 = 0.1 * np.eye(n)
    y, x = simulate(rng, F, Q, H, R, m0, P0, 50, n_slow, keep_states)
    return Problem(F, Q, H, R, m0, P0, y, 50, x, "network8", {"K": K, "dt": dt})


def _ragged_one(seed: int, s: int, n_min: int, n_max: int, ratios, keep_states: bool) -> Problem:
    rng = np.random.default_rng([seed, s])
    rates = log_uniform(rng, 0.05, 1.0, 4)
    K = chain_rates_matrix(rates)
    F = scipy.linalg.expm(K * 0.05)
    Q = 1e-3 * np.eye(4)
    H = np.zeros((1, 4)); H[0, 3] = 1.0
    R = np.array([[0.05]])
    m0 = np.eye(4)[0]
    P0 = 0.1 * np.eye(4)
    l = int(rng.choice(ratios))
    N = int(rng.integers(n_min, n_max + 1))
    y, x = simulate(rng, F, Q, H, R, m0, P0, l, N, keep_states)
    return Problem(F, Q, H, R, m0, P0, y, l, x, f"ragged_chains[{s}]", {"K": K})


def _ragged_chunk(args):
    seed, lo, hi, n_min, n_max, ratios, keep_states = args
    return [_ragged_one(seed, s, n_min, n_max, ratios, keep_states) for s in range(lo, hi)]


def ragged_shapes(seed: int = 0, n_seq: int = 4096, n_min: int = 100, n_max: int = 20_000,
                  ratios=(5, 10, 20)) -> tuple[np.ndarray, np.ndarray]:
    """(ratio, n_slow) of every sequence of ``ragged_chains`` without building
    them: the same draws from each sequence's generator, up to its length."""
    ratios = tuple(int(r) for r in ratios)
    rs, ns = np.empty(n_seq, dtype=np.int64), np.empty(n_seq, dtype=np.int64)
    for s in range(n_seq):
        rng = np.random.default_rng([seed, s])
        log_uniform(rng, 0.05, 1.0, 4)
        rs[s] = int(rng.choice(ratios))
        ns[s] = int(rng.integers(n_min, n_max + 1))
    return rs, ns


def balanced_ranges(fast_steps: np.ndarray, parts: int) -> list[tuple[int, int]]:
    """Contiguous index ranges [lo, hi) of nearly equal total ``fast_steps``
    (range r starts at the first index whose preceding sum reaches r/parts of
    the total); ranges may be empty when one entry outweighs a share."""
    cum = np.concatenate([[0], np.cumsum(fast_steps, dtype=np.int64)])
    cuts = [0] + [int(np.searchsorted(cum, cum[-1] * r / parts, side="left")) for r in range(1, parts)] + [len(fast_steps)]
    cuts = [min(max(c, 0), len(fast_steps)) for c in cuts]
    for i in range(1, len(cuts)):
        cuts[i] = max(cuts[i], cuts[i - 1])
    return [(cuts[i], cuts[i + 1]) for i in range(parts)]


def ragged_chains(seed: int = 0, n_seq: int = 4096, n_min: int = 100, n_max: int = 20_000,
            ratios=(5, 10, 20), keep_states: bool = False, workers: int = 1,
            seq_range: tuple[int, int] | None = None) -> list[Problem]:
    """Ragged batch: per sequence a 4-species chain as in chain4 (dt=.05),
    ratio drawn from {5,10,20}, n_slow ~ U[n_min, n_max], ny=1 observing
    species 4, Q=1e-3 I, R=.05, m0=e1, P0=.1 I.

    Sequence s draws from its own generator seeded with (seed, s), so the
    batch is the same whether it is built serially or by ``workers`` processes
    (a pool started with the ``spawn`` method, safe after CUDA has been used).
    ``seq_range`` = (lo, hi) builds only sequences lo .. hi-1 of the batch.
    """
    ratios = tuple(int(r) for r in ratios)
    lo, hi = (0, n_seq) if seq_range is None else (int(seq_range[0]), int(seq_range[1]))
    if workers <= 1 or hi - lo < 2 * workers:
        return _ragged_chunk((seed, lo, hi, n_min, n_max, ratios, keep_states))
    import multiprocessing as mp
    import os
    bounds = np.linspace(lo, hi, 4 * workers + 1).astype(int)
    jobs = [(seed, int(a), int(b), n_min, n_max, ratios, keep_states) for a, b in zip(bounds[:-1], bounds[1:]) if b > a]
    # one BLAS thread per worker process (the workers already fill the cores)
    keys = ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS")
    saved = {k: os.environ.get(k) for k in keys}
    os.environ.update({k: "1" for k in keys})
    try:
        with mp.get_context("spawn").Pool(workers) as pool:
            parts = pool.map(_ragged_chunk, jobs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
    return [p for part in parts for p in part]


def pack(probs: list[Problem]) -> dict:
    """A list of same-size sequences as the batch layout of the C-ABI: stacked
    F, Q, H, R, m0, P0, the measurements concatenated in sequence order, and
    per-sequence ratio / n_slow (int32) with the batch totals; with known
    inputs also B stacked (S, nx, nu) and u concatenated (total_fast, nu)."""
    out = {k: np.ascontiguousarray(np.stack([getattr(p, k) for p in probs])) for k in ("F", "Q", "H", "R", "m0", "P0")}
    out["y"] = np.ascontiguousarray(np.concatenate([p.y for p in probs]))
    if probs[0].B is not None:
        out["B"] = np.ascontiguousarray(np.stack([p.B for p in probs]))
        out["u"] = np.ascontiguousarray(np.concatenate([p.u for p in probs]))
    out["ratio"] = np.array([p.ratio for p in probs], dtype=np.int32)
    out["n_slow"] = np.array([p.n_slow for p in probs], dtype=np.int32)
    out["max_ratio"] = int(out["ratio"].max())
    out["total_slow"] = int(out["n_slow"].sum(dtype=np.int64))
    out["total_fast"] = int((out["n_slow"].astype(np.int64) * out["ratio"]).sum())
    return out


def stiff_chain6(seed: int = 0, n_slow: int = 10_000, keep_states: bool = False) -> Problem:
    """Stiff 6-species chain, rates log-U[1e-3,1e2], dt=.01, l=100, observing the
    last two species, Q=1e-6 I, R=1e-3 I, m0=e1, P0=.1 I."""
    rng = np.random.default_rng(seed)
    rates = log_uniform(rng, 1e-3, 1e2, 6)
    K = chain_rates_matrix(rates)
    dt = 0.01
    F = scipy.linalg.expm(K * dt)
    Q = 1e-6 * np.eye(6)
    H = np.zeros((2, 6)); H[0, 4] = 1.0; H[1, 5] = 1.0
    R = 1e-3 * np.eye(2)
    m0 = np.eye(6)[0]
    P0 = 0.1 * np.eye(6)
    y, x = simulate(rng, F, Q, H, R, m0, P0, 100, n_slow, keep_states)
    return Problem(F, Q, H, R, m0, P0, y, 100, x, "stiff_chain6", {"K": K, "dt": dt, "rates": rates})


def random_model(seed: int, nx: int, ny: int, ratio: int, n_slow: int,
                 q_scale: float = 0.05, r_scale: float = 0.1, nu: int = 0) -> Problem:
    """Small generic model with dense (non-diagonal) Q, R and P0, a random
    stable F and random H; used for pins and edge cases at tiny sizes.  With
    nu > 0 also a random input matrix B and inputs u_t (a sinusoid plus noise)."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((nx, nx))
    A *= 0.9 / max(1e-12, np.max(np.abs(np.linalg.eigvals(A))))
    G = rng.standard_normal((nx, nx))
    Q = q_scale * (G @ G.T / nx + 0.2 * np.eye(nx))
    Gr = rng.standard_normal((ny, ny))
    R = r_scale * (Gr @ Gr.T / ny + 0.5 * np.eye(ny))
    H = rng.standard_normal((ny, nx))
    m0 = rng.standard_normal(nx)
    Gp = rng.standard_normal((nx, nx))
    P0 = 0.2 * (Gp @ Gp.T / nx + 0.3 * np.eye(nx))
    B = u = None
    if nu > 0:
        B = rng.standard_normal((nx, nu)) * 0.5
        t = np.arange(n_slow * ratio)[:, None]
        u = np.sin(0.07 * t + np.arange(nu)[None, :]) + 0.3 * rng.standard_normal((n_slow * ratio, nu))
    y, x = simulate(rng, A, Q, H, R, m0, P0, ratio, n_slow, True, B, u)
    return Problem(A, Q, H, R, m0, P0, y, ratio, x, f"rand{nx}x{ny}l{ratio}N{n_slow}u{nu}", B=B, u=u)


# single-sequence workloads by name (ragged_chains returns a batch)
WORKLOADS = {"ab_kinetics": ab_kinetics, "chain4": chain4, "network8": network8, "stiff_chain6": stiff_chain6}
