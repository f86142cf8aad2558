"""Pins of the tube, tightening and conformal-radius oracle (oracle/tubes.py, paper Sec. 4.2
eq. of_optimization_tightening1/2, Sec. 4.4): the tube is the worst case of the simulated closed
loop over unit-ball disturbances (reached by the maximising disturbance, never exceeded by random
ones), the margins of unit-vector constraints are the tube's rows, and the radius is the stated
order statistic, with the conformal coverage it promises."""
import math

import numpy as np

from oracle import tubes
from test_oracle_sls import _closed_loop_system, simulate_observer_controller


def _deviation(s, w_hat, e_hat):
    """states and controls of the simulated closed loop for the unit disturbances w = E w_hat,
    e = F e_hat from x_0 = 0"""
    w = np.einsum("jab,jb->ja", s["E"], w_hat)
    e = np.einsum("jab,jb->ja", s["F"], e_hat)
    return simulate_observer_controller(s, np.zeros(s["A"].shape[1]), w, e)


def test_tube_is_the_worst_case_of_the_simulated_closed_loop():
    n, p, m, N = 4, 3, 2, 5
    s = _closed_loop_system(21)
    XW, UW, XE, UE = s["maps"]
    tau = tubes.tube_widths(XW, UW, XE, UE, s["E"], s["F"], N)
    rng = np.random.default_rng(22)
    for k in (1, 3, N):
        for r in range(n + m):
            # the maximising disturbance of row r at time k: each w_j, e_j along its row's gradient
            w_hat, e_hat = np.zeros((N, n)), np.zeros((N, p))
            for j in range(k):
                g = (np.vstack([XW, UW])[_row(k, r, n, m, N)], np.vstack([XE, UE])[_row(k, r, n, m, N)])
                gw = g[0][(j + 1) * n:(j + 2) * n] @ s["E"][j]
                ge = g[1][(j + 1) * p:(j + 2) * p] @ s["F"][j]
                w_hat[j] = _unit(gw)
                e_hat[j] = _unit(ge)
            xs, us = _deviation(s, w_hat, e_hat)
            dev = (xs[k * n + r] if r < n else us[k * m + r - n])
            assert abs(dev - tau[k, r]) <= 1e-10 * max(1.0, tau[k, r]), (k, r)
        for _ in range(50):
            w_hat = rng.normal(size=(N, n))
            w_hat /= np.maximum(1.0, np.linalg.norm(w_hat, axis=1))[:, None]
            e_hat = rng.normal(size=(N, p))
            e_hat /= np.maximum(1.0, np.linalg.norm(e_hat, axis=1))[:, None]
            xs, us = _deviation(s, w_hat, e_hat)
            dev = np.concatenate([xs[k * n:(k + 1) * n], us[k * m:(k + 1) * m]])
            assert np.all(np.abs(dev) <= tau[k] + 1e-12)
    assert np.all(tau[0] == 0)                       # nothing has entered at time 0


def _unit(g):
    """g / |g| (zero when g is: a disturbance that cannot reach the row)"""
    nrm = np.linalg.norm(g)
    return g / nrm if nrm > 0 else np.zeros_like(g)


def _row(k, r, n, m, N):
    """row index of [x_k; u_k][r] in the stacked [Phi^x*; Phi^u*]"""
    return k * n + r if r < n else (N + 1) * n + k * m + (r - n)


def test_margins_of_coordinate_constraints_are_the_tube_rows():
    n, p, m, N = 4, 3, 2, 5
    s = _closed_loop_system(23)
    XW, UW, XE, UE = s["maps"]
    tau = tubes.tube_widths(XW, UW, XE, UE, s["E"], s["F"], N)
    rng = np.random.default_rng(24)
    z, v = rng.normal(size=(N + 1, n)), rng.normal(size=(N, m))
    Ccon = np.vstack([np.eye(n + m), -np.eye(n + m)])
    bcon = rng.normal(size=2 * (n + m))
    mg = tubes.constraint_margins(XW, UW, XE, UE, s["E"], s["F"], N, Ccon, bcon, z, v)
    for k in range(N):
        zk = np.concatenate([z[k], v[k]])
        assert np.allclose(mg[k, :n + m], -bcon[:n + m] - zk - tau[k], atol=1e-12)
        assert np.allclose(mg[k, n + m:], -bcon[n + m:] + zk - tau[k], atol=1e-12)


def test_margin_of_a_general_constraint_is_its_simulated_worst_case():
    """For c = a random row over [x; u]: the maximising disturbances drive c^T (deviation) to the
    tightening term exactly."""
    n, p, m, N = 4, 3, 2, 5
    s = _closed_loop_system(25)
    XW, UW, XE, UE = s["maps"]
    rng = np.random.default_rng(26)
    c = rng.normal(size=(1, n + m))
    z, v = np.zeros((N + 1, n)), np.zeros((N, m))
    k = 4
    mg = tubes.constraint_margins(XW, UW, XE, UE, s["E"], s["F"], N, c, np.zeros(1), z, v)
    Sx, Su = np.zeros((n + m, (N + 1) * n)), np.zeros((n + m, (N + 1) * m))
    Sx[:n, k * n:(k + 1) * n] = np.eye(n)
    Su[n:, k * m:(k + 1) * m] = np.eye(m)
    row_w = c @ (Sx @ XW + Su @ UW)
    row_e = c @ (Sx @ XE + Su @ UE)
    w_hat, e_hat = np.zeros((N, n)), np.zeros((N, p))
    for j in range(k):
        gw = row_w[0, (j + 1) * n:(j + 2) * n] @ s["E"][j]
        ge = row_e[0, (j + 1) * p:(j + 2) * p] @ s["F"][j]
        w_hat[j], e_hat[j] = _unit(gw), _unit(ge)
    xs, us = _deviation(s, w_hat, e_hat)
    worst = c[0] @ np.concatenate([xs[k * n:(k + 1) * n], us[k * m:(k + 1) * m]])
    assert abs(-mg[k, 0] - worst) <= 1e-10 * abs(worst)


def test_conformal_radius_order_statistic():
    s = np.array([0.5, 0.1, 0.9, 0.3, 0.7, 0.2, 0.8, 0.4, 0.6])
    # (n + 1)(1 - delta/T) = 9 -> the largest; 5 -> the median; 9.5 -> past n: +inf
    assert tubes.conformal_radius(s, 0.2, 2) == 0.9
    assert tubes.conformal_radius(s, 0.5, 1) == 0.5
    assert math.isinf(tubes.conformal_radius(s, 0.05, 1))
    assert tubes.conformal_radius(s, 0.8, 1) == 0.2       # index 2: the second smallest
    q = np.array([[0.0, 3.0], [1.0, 1.0]])
    assert np.allclose(tubes.conformal_scores(q, np.zeros((2, 2))), [3.0, np.sqrt(2.0)])


def test_conformal_radius_covers_with_the_stated_probability():
    """Exchangeable scores: the next score falls within the radius with probability at least
    1 - delta/T and at most 1 - delta/T + 1/(n + 1) (checked over 4000 seeded draws)."""
    rng = np.random.default_rng(27)
    n, delta, T = 99, 0.4, 4
    hits = 0
    trials = 4000
    for _ in range(trials):
        s = rng.exponential(size=n + 1)
        hits += s[-1] <= tubes.conformal_radius(s[:-1], delta, T)
    cover = hits / trials
    lo, hi = 1 - delta / T, 1 - delta / T + 1 / (n + 1)
    sd = math.sqrt(lo * (1 - lo) / trials)
    assert lo - 4 * sd <= cover <= hi + 4 * sd
