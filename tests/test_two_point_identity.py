"""The identity behind the two-point form of the fast-rate recovery, checked
against the brute-force joint posterior over all stacked fast states (no
GPU, no library code): the states inside an interval depend on the rest of
the data only through the interval's first state x_{k,1}, the next
interval's first state x_{k+1,1} and the interval's measurement y_k, so

  m^s_{k,i} = C1_i m^s_{k,1} + C2_i m^s_{k+1,1} + c3_i y_k,
  P^s_{k,ii} = Sg_i + [C1_i C2_i] Cov([x_{k,1}; x_{k+1,1}] | y_{1:N}) [C1_i C2_i]^T,

with the constants of Gaussian conditioning on v = [x_{k+1,1}; y_k] given
x_{k,1}, formed from the lifted model's noise covariances (Sec. III-A):
Cov(e_j) = Qc_j, Cov(e_j, e_l), V_j = Cov(e_j, sum_t e_t) and
R_x = H (sum_j V_j) H^T + R; the last interval conditions on (x_{k,1}, y_k).
These are the formulas the constants kernel evaluates (restated here in
numpy); the GPU outputs themselves are checked against the oracle by the
GPU tests."""
import numpy as np
import pytest

from paper_2410_00627_gb300 import synth
from tests import brute


def _lifted(F, Q, H, R, l):
    n = F.shape[0]
    Ap = [np.linalg.matrix_power(F, i) for i in range(l + 1)]
    Qc = [sum((Ap[r] @ Q @ Ap[r].T for r in range(j)), np.zeros((n, n))) for j in range(l + 1)]

    def cov(j, t):  # Cov(e_j, e_t)
        return Qc[j] @ Ap[t - j].T if j <= t else Ap[j - t] @ Qc[t]
    V = [sum(cov(j, t) for t in range(1, l + 1)) for j in range(l + 1)]
    Rx = H @ sum(V[1:]) @ H.T + R
    return Ap, Qc, [cov(j, l) for j in range(l + 1)], V, sum(Ap[1:]), Rx


def _constants(F, Q, H, R, l):
    n, m = F.shape[0], H.shape[0]
    Ap, Qc, Ql, V, T, Rx = _lifted(F, Q, H, R, l)
    Vb = np.block([[Qc[l], (V[l] - Qc[l]) @ H.T],
                   [H @ (V[l] - Qc[l]).T, Rx - H @ V[l] @ H.T - H @ V[l].T @ H.T + H @ Qc[l] @ H.T]])
    HS = H @ (np.eye(n) + T - Ap[l])   # H sum_{j<l} A^j
    two, one = [], []
    for i in range(1, l + 1):
        K = np.zeros((n, n + m)) if i == 1 else np.hstack([Ql[i - 1], (V[i - 1] - Ql[i - 1]) @ H.T])
        G = K @ np.linalg.inv(Vb)
        two.append((Ap[i - 1] - G[:, :n] @ Ap[l] - G[:, n:] @ HS, G[:, :n], G[:, n:], Qc[i - 1] - G @ K.T))
        Gy = K[:, n:] @ np.linalg.inv(Vb[n:, n:])
        one.append((Ap[i - 1] - Gy @ HS, Gy, Qc[i - 1] - Gy @ K[:, n:].T))
    return two, one


@pytest.mark.parametrize("n,m,l,N", [(3, 2, 4, 5), (2, 1, 3, 4), (4, 1, 5, 3), (3, 1, 1, 4), (2, 2, 6, 2),
                                     (3, 2, 3, 1)])
def test_two_point_identity_against_the_joint_posterior(n, m, l, N):
    prob = synth.random_model(100 + n + 7 * l, n, m, l, N)
    mu, S = brute.joint_prior(prob.F, prob.Q, prob.m0, prob.P0, N * l)
    ms, Ss = brute.condition(mu, S, brute.meas_matrix(prob.H, n, l, N), prob.R, prob.y, N)
    two, one = _constants(prob.F, prob.Q, prob.H, prob.R, l)
    blk = lambda t: slice(t * n, (t + 1) * n)  # noqa: E731  (x_{k,i} is z index k*l + i)
    for k in range(N):
        t0 = k * l + 1
        for i in range(1, l + 1):
            t = k * l + i
            if k < N - 1:
                C1, C2, c3, Sg = two[i - 1]
                t1 = t0 + l
                idx = np.r_[blk(t0), blk(t1)]
                mean = C1 @ ms[blk(t0)] + C2 @ ms[blk(t1)] + c3 @ prob.y[k]
                CC = np.hstack([C1, C2])
                cov = Sg + CC @ Ss[np.ix_(idx, idx)] @ CC.T
            else:
                C1, c3, Sg = one[i - 1]
                mean = C1 @ ms[blk(t0)] + c3 @ prob.y[k]
                cov = Sg + C1 @ Ss[blk(t0), blk(t0)] @ C1.T
            assert np.max(np.abs(mean - ms[blk(t)])) <= 1e-12 * np.max(np.abs(ms)), (k, i)
            assert np.max(np.abs(cov - Ss[blk(t), blk(t)])) <= 1e-12 * np.max(np.abs(Ss)), (k, i)
    # i = 1 is x_{k,1} itself
    C1, C2, c3, Sg = two[0]
    assert np.array_equal(C1, np.eye(n)) and not C2.any() and not c3.any() and not Sg.any()
