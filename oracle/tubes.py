"""FP64 oracle of the reachable tubes, the constraint tightening and the conformal radius
(arxiv 2606.14188, Sec. 4.2 eq. of_optimization_tightening1/2; Sec. 4.4).

TEST INFRASTRUCTURE ONLY (see oracle/sim.py).

Inputs are the closed-loop maps of oracle/sls.py (dense block lower-triangular arrays over times
0..N, block (k, j) mapping the disturbance that enters at time j to time k: delta_{j+1} = w_j for
the process disturbance, the observation disturbance e_j entering Phihat^y's block j + 1).

Readings:
  * The sums of eq. of_optimization_tightening1/2 run over the disturbances w_j, e_j injected at
    j = 0..k-1, which reach time k through the blocks (k, j + 1) of Phi^w = [Phi^xw; Phi^uw] and
    Phi^e = [Phi^xe; Phi^ue] (the initial estimation error is the Kalman recursion's Xi and is not
    in the printed sums).
  * The tube tau_k is a vector over the rows of [x_k; u_k]: the row-wise 2-norms summed over j.
  * A constraint i is the row c_i of [x; u] with offset b_i; its tightened margin at time k is
    -b_i - c_i^T [z_k; v_k] - sum_j (|c_i^T Phi^w_{k,j+1} E_j|_2 + |c_i^T Phi^e_{k,j+1} F_j|_2),
    k = 0..N-1 (the times that carry a nominal control); the constraint holds robustly when it
    is >= 0.
  * The conformal radius takes the ceil((n + 1)(1 - delta / T))-th smallest score, +inf when that
    index exceeds n (Sec. 4.4).
"""
from __future__ import annotations

import math

import numpy as np


def _block(M, k, j, r, c):
    return M[k * r:(k + 1) * r, j * c:(j + 1) * c]


def tube_widths(PXW, PUW, PXE, PUE, E, F, N):
    """tau [N+1][n+m]: tau_k = sum_{j<k} ||[Phi^xw; Phi^uw]_{k,j+1} E_j||_{2,r}
    + ||[Phi^xe; Phi^ue]_{k,j+1} F_j||_{2,r}."""
    E, F = np.asarray(E, dtype=np.float64), np.asarray(F, dtype=np.float64)
    n, m, p = E.shape[1], PUW.shape[0] // (N + 1), F.shape[1]
    tau = np.zeros((N + 1, n + m))
    for k in range(N + 1):
        for j in range(k):
            W = np.vstack([_block(PXW, k, j + 1, n, n), _block(PUW, k, j + 1, m, n)]) @ E[j]
            V = np.vstack([_block(PXE, k, j + 1, n, p), _block(PUE, k, j + 1, m, p)]) @ F[j]
            tau[k] += np.linalg.norm(W, axis=1) + np.linalg.norm(V, axis=1)
    return tau


def constraint_margins(PXW, PUW, PXE, PUE, E, F, N, Ccon, bcon, z, v):
    """margin [N][nc] of eq. of_optimization_tightening1 for the nominal states z [N+1][n] and
    controls v [N][m]."""
    E, F = np.asarray(E, dtype=np.float64), np.asarray(F, dtype=np.float64)
    Ccon, bcon = np.asarray(Ccon, dtype=np.float64), np.asarray(bcon, dtype=np.float64)
    n, m, p = E.shape[1], PUW.shape[0] // (N + 1), F.shape[1]
    out = np.zeros((N, Ccon.shape[0]))
    for k in range(N):
        s = np.zeros(Ccon.shape[0])
        for j in range(k):
            W = Ccon @ np.vstack([_block(PXW, k, j + 1, n, n), _block(PUW, k, j + 1, m, n)]) @ E[j]
            V = Ccon @ np.vstack([_block(PXE, k, j + 1, n, p), _block(PUE, k, j + 1, m, p)]) @ F[j]
            s += np.linalg.norm(W, axis=1) + np.linalg.norm(V, axis=1)
        out[k] = -bcon - Ccon @ np.concatenate([z[k], v[k]]) - s
    return out


def conformal_scores(q_next, f_pred):
    """s_i = ||qbar_i^+ - f(qbar_i, u_i)||_2."""
    d = np.asarray(q_next, dtype=np.float64) - np.asarray(f_pred, dtype=np.float64)
    return np.sqrt(np.sum(d * d, axis=1))


def conformal_radius(scores, delta, T):
    """s_(ceil((n + 1)(1 - delta / T))) of the sorted scores (1-based), +inf past n."""
    s = np.sort(np.asarray(scores, dtype=np.float64))
    n = s.size
    idx = math.ceil((n + 1) * (1.0 - delta / T))
    return float("inf") if idx > n else float(s[max(idx, 1) - 1])
