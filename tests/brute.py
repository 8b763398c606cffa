"""Brute-force dense joint-Gaussian posterior over all stacked fast states.

Independent of the paper's recursions: the prior of z = (x_0, x_1, ..., x_T),
T = N*l, is built from x_t = A^t x_0 + sum_{s<t} A^{t-1-s} w_s; the
measurements y_k = H sum_{i=1..l} x_{(k-1)l+i} + v_k are linear in z, and
every filtering / smoothing marginal is plain Gaussian conditioning of that
joint on y_{1:K}.  Tiny sizes only ((T+1)*nx up to a few hundred).
"""
from __future__ import annotations

import numpy as np


def joint_prior(F, Q, m0, P0, T, B=None, u=None):
    n = F.shape[0]
    Apow = [np.eye(n)]
    for _ in range(T):
        Apow.append(Apow[-1] @ F)
    # z = Phi xi, xi = (x_0, w_0, ..., w_{T-1}) with cov blockdiag(P0, Q, ..., Q)
    Phi = np.zeros(((T + 1) * n, (T + 1) * n))
    for t in range(T + 1):
        Phi[t * n:(t + 1) * n, 0:n] = Apow[t]
        for s in range(t):
            Phi[t * n:(t + 1) * n, (1 + s) * n:(2 + s) * n] = Apow[t - 1 - s]
    Cxi = np.zeros_like(Phi)
    Cxi[:n, :n] = P0
    for s in range(T):
        Cxi[(1 + s) * n:(2 + s) * n, (1 + s) * n:(2 + s) * n] = Q
    mu = np.concatenate([Apow[t] @ m0 for t in range(T + 1)])
    if B is not None:   # known inputs: x_t gains sum_{s<t} A^{t-1-s} B u_s
        for t in range(1, T + 1):
            mu[t * n:(t + 1) * n] += sum(Apow[t - 1 - s] @ (B @ u[s]) for s in range(t))
    return mu, Phi @ Cxi @ Phi.T


def meas_matrix(H, n, l, N):
    m = H.shape[0]
    Hz = np.zeros((N * m, (N * l + 1) * n))
    for k in range(N):
        for i in range(1, l + 1):
            t = k * l + i
            Hz[k * m:(k + 1) * m, t * n:(t + 1) * n] = H
    return Hz


def condition(mu, S, Hz, R, y, K):
    """Posterior of z given y_{1:K} (K measurements)."""
    m = R.shape[0]
    if K == 0:
        return mu, S
    Hk = Hz[:K * m]
    Rk = np.kron(np.eye(K), R)
    Sy = Hk @ S @ Hk.T + Rk
    G = np.linalg.solve(Sy, Hk @ S).T
    return mu + G @ (y[:K].ravel() - Hk @ mu), S - G @ Hk @ S


def posteriors(prob):
    """Returns dict with fast_filt_mean/cov (x_{k,i}|y_{1:k}), fast_smooth_mean/cov
    (x_{k,i}|y_{1:N}) in the library's row order (k*l + i-1)."""
    F, Q, H, R, m0, P0, y, l = prob.F, prob.Q, prob.H, prob.R, prob.m0, prob.P0, prob.y, prob.ratio
    n, N = F.shape[0], y.shape[0]
    mu, S = joint_prior(F, Q, m0, P0, N * l, getattr(prob, "B", None), getattr(prob, "u", None))
    Hz = meas_matrix(H, n, l, N)
    ffm = np.zeros((N * l, n)); ffc = np.zeros((N * l, n, n))
    for k in range(N):
        mk, Sk = condition(mu, S, Hz, R, y, k + 1)
        for i in range(1, l + 1):
            t = k * l + i
            ffm[k * l + i - 1] = mk[t * n:(t + 1) * n]
            ffc[k * l + i - 1] = Sk[t * n:(t + 1) * n, t * n:(t + 1) * n]
    ms, Ss = condition(mu, S, Hz, R, y, N)
    fsm = np.zeros((N * l, n)); fsc = np.zeros((N * l, n, n))
    for t in range(1, N * l + 1):
        fsm[t - 1] = ms[t * n:(t + 1) * n]
        fsc[t - 1] = Ss[t * n:(t + 1) * n, t * n:(t + 1) * n]
    return {"fast_filt_mean": ffm, "fast_filt_cov": ffc, "fast_smooth_mean": fsm, "fast_smooth_cov": fsc}


def loglik(prob):
    """log p(y_{1:N}) of the stacked measurements under the dense joint prior:
    y = Hz z + v, so y ~ N(Hz mu, Hz S Hz^T + I_N (x) R)."""
    F, Q, H, R, m0, P0, y, l = prob.F, prob.Q, prob.H, prob.R, prob.m0, prob.P0, prob.y, prob.ratio
    n, N, m = F.shape[0], y.shape[0], H.shape[0]
    mu, S = joint_prior(F, Q, m0, P0, N * l, getattr(prob, "B", None), getattr(prob, "u", None))
    Hz = meas_matrix(H, n, l, N)
    Sy = Hz @ S @ Hz.T + np.kron(np.eye(N), R)
    r = y.ravel() - Hz @ mu
    sign, logdet = np.linalg.slogdet(Sy)
    assert sign > 0
    return float(-0.5 * (N * m * np.log(2 * np.pi) + logdet + r @ np.linalg.solve(Sy, r)))
