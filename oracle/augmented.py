"""Augmented-state cross-check of the SRTM posteriors (numpy, float64).

TEST INFRASTRUCTURE ONLY, like the rest of ``oracle/``: only the test-suite
may import it.  It shares no code with the CUDA library, nor with
``oracle.c``: a second, independent algorithm for the same posteriors.

The paper notes (Sec. II, footnote to the dual-rate reformulation) that the
integrated measurement could instead be handled by augmenting the state with
the running sum of the fast states, and adopts the lifted form for its lower
cost.  This module takes the augmented route literally, on the fast time
grid: the state is z = [x; p], where p is the sum of the fast states already
seen in the current slow interval (p = 0 at its first step), so that

    first step of an interval:  x' = A x + B u + w,  p' = 0
    later steps:                x' = A x + B u + w,  p' = p + x
    last step of interval k:    y_k = H (p + x) + v        (H on the sum)

with w ~ N(0, Q), v ~ N(0, R), x_0 ~ N(m0, P0).  A textbook Kalman filter
over the T = N l fast steps (a measurement update at the last step of each
interval only) and a Rauch-Tung-Striebel backward pass then give

    p(x_t | y_{1:N})        the RTS pass over the whole grid,
    p(x_{k,l} | y_{1:k})    the filter right after the update of interval k,
    p(x_{k,i} | y_{1:k})    the RTS pass run back from that update over the
                            steps of interval k alone (no data in between),
    log p(y_{1:N})          the sum of the update steps' innovation densities.

At the first step of an interval the predicted covariance has an exactly zero
p-block; the RTS gain then inverts the x-block only (the p-part of that state
is the constant 0, so it carries no information back).
"""
from __future__ import annotations

import numpy as np


def _inputs(prob):
    B, u = getattr(prob, "B", None), getattr(prob, "u", None)
    if B is None or u is None:
        return None, None
    return np.asarray(B, dtype=np.float64), np.asarray(u, dtype=np.float64)


def augmented(prob) -> dict:
    """Kalman filter + RTS smoother on the augmented state z = [x; p].

    Returns fast_filt_mean/cov (p(x_{k,i}|y_{1:k}), rows k*l + i - 1),
    slow_filt_mean/cov (p(x_{k,l}|y_{1:k})), fast_smooth_mean/cov
    (p(x_{k,i}|y_{1:N})) and loglik (log p(y_{1:N}))."""
    A = np.asarray(prob.F, dtype=np.float64)
    Q = np.asarray(prob.Q, dtype=np.float64)
    H = np.asarray(prob.H, dtype=np.float64)
    R = np.asarray(prob.R, dtype=np.float64)
    y = np.asarray(prob.y, dtype=np.float64)
    l = int(prob.ratio)
    n, m, N = A.shape[0], H.shape[0], y.shape[0]
    T = N * l
    B, u = _inputs(prob)
    I, O = np.eye(n), np.zeros((n, n))
    phi_first = np.block([[A, O], [O, O]])   # x' = A x (+ B u + w), p' = 0
    phi_later = np.block([[A, O], [I, I]])   # x' = A x (+ B u + w), p' = p + x
    Qz = np.block([[Q, O], [O, O]])
    Cz = np.hstack([H, H])                    # y_k = H (p + x) + v at the last step

    m_z = np.concatenate([np.asarray(prob.m0, dtype=np.float64), np.zeros(n)])
    P_z = np.block([[np.asarray(prob.P0, dtype=np.float64), O], [O, O]])
    pred_m = np.zeros((T, 2 * n))
    pred_P = np.zeros((T, 2 * n, 2 * n))
    filt_m = np.zeros((T, 2 * n))
    filt_P = np.zeros((T, 2 * n, 2 * n))
    loglik = 0.0
    for t in range(T):
        i = t % l + 1
        phi = phi_first if i == 1 else phi_later
        mp = phi @ m_z
        if B is not None:
            mp[:n] += B @ u[t]
        Pp = phi @ P_z @ phi.T + Qz
        pred_m[t], pred_P[t] = mp, Pp
        if i == l:
            k = t // l
            S = Cz @ Pp @ Cz.T + R
            e = y[k] - Cz @ mp
            K = np.linalg.solve(S, Cz @ Pp).T        # Pp Cz^T S^-1 (S symmetric)
            m_z = mp + K @ e
            P_z = Pp - K @ S @ K.T
            P_z = 0.5 * (P_z + P_z.T)
            _, logdet = np.linalg.slogdet(S)
            loglik += -0.5 * (m * np.log(2.0 * np.pi) + logdet + e @ np.linalg.solve(S, e))
        else:
            m_z, P_z = mp, Pp
        filt_m[t], filt_P[t] = m_z, P_z

    def gain(t):
        """RTS gain from step t to step t + 1: Cov(z_t, z_{t+1}) times the
        (pseudo-)inverse of the predicted covariance of step t + 1."""
        i_next = (t + 1) % l + 1
        phi = phi_first if i_next == 1 else phi_later
        C = filt_P[t] @ phi.T
        if i_next == 1:   # predicted p-block is exactly zero
            G = np.zeros((2 * n, 2 * n))
            G[:, :n] = np.linalg.solve(pred_P[t + 1][:n, :n], C[:, :n].T).T
            return G
        return np.linalg.solve(pred_P[t + 1], C.T).T

    def rts_step(t, ms_next, Ps_next):
        G = gain(t)
        ms = filt_m[t] + G @ (ms_next - pred_m[t + 1])
        Ps = filt_P[t] + G @ (Ps_next - pred_P[t + 1]) @ G.T
        return ms, 0.5 * (Ps + Ps.T)

    # whole-grid RTS pass: p(z_t | y_{1:N})
    sm_m = np.zeros((T, 2 * n))
    sm_P = np.zeros((T, 2 * n, 2 * n))
    sm_m[T - 1], sm_P[T - 1] = filt_m[T - 1], filt_P[T - 1]
    for t in range(T - 2, -1, -1):
        sm_m[t], sm_P[t] = rts_step(t, sm_m[t + 1], sm_P[t + 1])

    # per interval: back from its update over its own steps, p(z_t | y_{1:k})
    ff_m = np.zeros((T, 2 * n))
    ff_P = np.zeros((T, 2 * n, 2 * n))
    for k in range(N):
        t_end = k * l + l - 1
        ff_m[t_end], ff_P[t_end] = filt_m[t_end], filt_P[t_end]
        for t in range(t_end - 1, k * l - 1, -1):
            ff_m[t], ff_P[t] = rts_step(t, ff_m[t + 1], ff_P[t + 1])

    x = slice(0, n)
    return {
        "fast_filt_mean": ff_m[:, x].copy(), "fast_filt_cov": ff_P[:, x, x].copy(),
        "slow_filt_mean": filt_m[l - 1::l, x].copy(), "slow_filt_cov": filt_P[l - 1::l, x, x].copy(),
        "fast_smooth_mean": sm_m[:, x].copy(), "fast_smooth_cov": sm_P[:, x, x].copy(),
        "loglik": float(loglik),
    }
