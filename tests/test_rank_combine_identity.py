"""The identity behind the rank-m form of the filter combine, checked in
float64 on random operands (no GPU, no library code).  For a generic element
of Eq. (26) on the right, J_j = C_bar^T R_x^-1 C_bar and
eta_j = C_bar^T R_x^-1 (y - c), and with S = R_x + C_bar D_i C_bar^T,
K = D_i C_bar^T S^-1, G = C_bar F_i the combine of Eq. (27) equals

  u = (I - K C_bar)(d_i + D_i eta_j),            d_ij = F_j u + d_j,
  D_ij = F_j (D_i - K C_bar D_i) F_j^T + D_j,
  V = F_i - K G,  F_ij = F_j V,  eta_ij = V^T (eta_j - J_j d_i) + eta_i,
  J_ij = G^T S^-1 G + J_i,

the arithmetic of the rank-m combine kernel (restated here in numpy); the
m = 2 inverse of S is its adjugate over its determinant.  The general form is
Eq. (27) with M = I + D_i J_j inverted."""
import numpy as np
import pytest


def _general(a, b):
    n = a["F"].shape[0]
    Mi = np.linalg.inv(np.eye(n) + a["D"] @ b["J"])
    W, V = b["F"] @ Mi, Mi @ a["F"]
    return {"F": W @ a["F"], "d": W @ (a["d"] + a["D"] @ b["e"]) + b["d"], "D": W @ a["D"] @ b["F"].T + b["D"],
            "e": V.T @ (b["e"] - b["J"] @ a["d"]) + a["e"], "J": V.T @ b["J"] @ a["F"] + a["J"]}


def _rank(a, b, Cb, Rx):
    m = Cb.shape[0]
    CD = Cb @ a["D"]
    S = Rx + CD @ Cb.T
    if m == 2:   # adjugate over the determinant
        Si = np.array([[S[1, 1], -S[0, 1]], [-S[1, 0], S[0, 0]]]) / (S[0, 0] * S[1, 1] - S[0, 1] * S[1, 0])
    else:
        Si = np.linalg.inv(S)
    Kt = Si @ CD                      # K^T
    t = a["d"] + a["D"] @ b["e"]
    G = Cb @ a["F"]
    x = b["e"] - b["J"] @ a["d"]
    u = t - Kt.T @ (Cb @ t)
    P = a["D"] - Kt.T @ CD
    V = a["F"] - Kt.T @ G
    return {"F": b["F"] @ V, "d": b["F"] @ u + b["d"], "D": b["F"] @ P @ b["F"].T + b["D"],
            "e": V.T @ x + a["e"], "J": G.T @ Si @ G + a["J"]}


def _spd(rng, k, scale=1.0):
    A = rng.standard_normal((k, k))
    return scale * (A @ A.T + 0.5 * k * np.eye(k))


@pytest.mark.parametrize("n,m", [(2, 1), (3, 1), (4, 1), (4, 2), (5, 3), (6, 2), (8, 3), (8, 4)])
@pytest.mark.parametrize("seed", [0, 1, 2])
def test_rank_form_equals_eq27(n, m, seed):
    rng = np.random.default_rng(100 * n + 10 * m + seed)
    a = {"F": rng.standard_normal((n, n)), "d": rng.standard_normal(n), "D": _spd(rng, n),
         "e": rng.standard_normal(n), "J": _spd(rng, n, 0.3)}
    Cb = rng.standard_normal((m, n))
    Rx = _spd(rng, m, 0.2)
    y = rng.standard_normal(m)
    b = {"F": rng.standard_normal((n, n)), "d": rng.standard_normal(n), "D": _spd(rng, n),
         "J": Cb.T @ np.linalg.solve(Rx, Cb), "e": Cb.T @ np.linalg.solve(Rx, y)}
    want, got = _general(a, b), _rank(a, b, Cb, Rx)
    for k in want:
        assert np.max(np.abs(got[k] - want[k])) <= 1e-10 * max(1.0, np.max(np.abs(want[k]))), k


def test_prefix_case_is_a_measurement_update_then_the_transition():
    """With a prefix on the left (F_i = 0, eta_i = 0, J_i = 0) the rank form is
    the Kalman update of (d_i, D_i) by y followed by the element's transition."""
    rng = np.random.default_rng(7)
    n, m = 4, 1
    Cb, Rx, y = rng.standard_normal((m, n)), _spd(rng, m, 0.2), rng.standard_normal(m)
    a = {"F": np.zeros((n, n)), "d": rng.standard_normal(n), "D": _spd(rng, n), "e": np.zeros(n),
         "J": np.zeros((n, n))}
    b = {"F": rng.standard_normal((n, n)), "d": rng.standard_normal(n), "D": _spd(rng, n),
         "J": Cb.T @ np.linalg.solve(Rx, Cb), "e": Cb.T @ np.linalg.solve(Rx, y)}
    got = _rank(a, b, Cb, Rx)
    S = Cb @ a["D"] @ Cb.T + Rx
    K = a["D"] @ Cb.T @ np.linalg.inv(S)
    m_upd = a["d"] + K @ (y - Cb @ a["d"])
    P_upd = a["D"] - K @ S @ K.T
    assert np.allclose(got["d"], b["F"] @ m_upd + b["d"], rtol=0, atol=1e-11)
    assert np.allclose(got["D"], b["F"] @ P_upd @ b["F"].T + b["D"], rtol=0, atol=1e-10)
    assert not np.any(got["F"]) and not np.any(got["e"]) and not np.any(got["J"])
