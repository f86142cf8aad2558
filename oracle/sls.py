"""FP64 oracle of the output-feedback SLS observer stage (arxiv 2606.14188, Sec. 4.2).

TEST INFRASTRUCTURE ONLY (see oracle/sim.py).

The stage takes the linearisation of the dynamics and of the observation model along one nominal
trajectory and returns the Kalman covariances and gains, the observer's closed-loop responses
Phihat^x, Phihat^y and the closed-loop maps Phi^xw, Phi^uw, Phi^xe, Phi^ue.  Times run 0..N:

    A_j (n x n), C_j (p x n), E_j (n x nw), F_j (p x ne)   for j = 0..N-1,    Xi (n x n0).

Functions:
  kalman_recursion     eq. kalman_recursions, step by step in j;
  scan_element, prior_element, combine, kalman_scan
                       eq. combination_rules with eq. initialization: the same covariances by an
                       associative scan;
  observer_responses   eq. backward_propagations;
  closed_loop_maps     the assembly of Phi^xw, Phi^uw, Phi^xe, Phi^ue from the state-feedback
                       responses Phibar^x, Phibar^u and M = I - Z A.

Block lower-triangular operators over times 0..N are dense arrays of (N+1) x (N+1) blocks (block
(k, j) at rows k*r.., columns j*c..), so that the tests can check them with dense algebra.

Readings (the paper's indices are garbled here; each reading is the one under which the printed
relations hold together):
  * Pi and L do not depend on the injection time k: nothing on the right of eq. kalman_recursions
    does, so Pi_{k,j} = Pi_j and L_{k,j} = L_j.
  * The gain that eq. kalman_recursions computes from (Pi_j, A_j, C_j) carries the label j+1.  The
    propagation through A_j uses that gain, Phihat^x_{k,j} = Phihat^x_{k,j+1} (A_j + L_{j+1}^T C_j),
    and Phihat^y_{k,j} = Phihat^x_{k,j} L_j^T for j >= 1, Phihat^y_{k,0} = 0 (there is no L_0).
    Under these labels Phihat satisfies the observer half of eq. phi_equation,
    Phihat^x (I - Z A) - Phihat^y Z C = I, and the error covariance it implies is Pi.
  * The scan's elements are the prior (Atil, Dtil, Ptil) = (0, 0, Xi Xi^T) and, for step j,
    (A_j^T, C_j^T (F_j F_j^T)^{-1} C_j, E_j E_j^T) (eq. initialization, whose step element carries
    the label (j+1, j)).  Pi_j is the composition e_{j-1} (x) ... (x) e_0 (x) prior, the later step
    on the left: the left operand of eq. combination_rules is the pair (i, m), the right (m, l).
"""
from __future__ import annotations

import numpy as np


# ---------------------------------------------------------------------------------------------
# eq. kalman_recursions
# ---------------------------------------------------------------------------------------------

def kalman_recursion(A, C, E, F, Xi):
    """Pi_0 = Xi Xi^T and, for j = 0..N-1,
        L_{j+1}  = -(F_j F_j^T + C_j Pi_j C_j^T)^{-1} C_j Pi_j A_j^T,
        Pi_{j+1} = E_j E_j^T + A_j Pi_j A_j^T + A_j Pi_j C_j^T L_{j+1}.
    Returns Pi (N+1, n, n) and L (N, p, n) with L[j] = L_{j+1}."""
    A, C, E, F, Xi = (np.asarray(x, dtype=np.float64) for x in (A, C, E, F, Xi))
    N, n = A.shape[0], A.shape[1]
    p = C.shape[1]
    Pi = np.zeros((N + 1, n, n))
    L = np.zeros((N, p, n))
    Pi[0] = Xi @ Xi.T
    for j in range(N):
        S = F[j] @ F[j].T + C[j] @ Pi[j] @ C[j].T
        L[j] = -np.linalg.solve(S, C[j] @ Pi[j] @ A[j].T)
        Pi[j + 1] = E[j] @ E[j].T + A[j] @ Pi[j] @ A[j].T + A[j] @ Pi[j] @ C[j].T @ L[j]
    return Pi, L


# ---------------------------------------------------------------------------------------------
# eq. combination_rules, eq. initialization
# ---------------------------------------------------------------------------------------------

def scan_element(A_j, C_j, E_j, F_j):
    """The step-j element (Atil, Dtil, Ptil) = (A_j^T, C_j^T (F_j F_j^T)^{-1} C_j, E_j E_j^T)."""
    R = F_j @ F_j.T
    return (np.array(A_j.T, dtype=np.float64), C_j.T @ np.linalg.solve(R, C_j), E_j @ E_j.T)


def prior_element(Xi):
    """The prior element (0, 0, Xi Xi^T)."""
    n = Xi.shape[0]
    return (np.zeros((n, n)), np.zeros((n, n)), Xi @ Xi.T)


def combine(left, right):
    """(Atil, Dtil, Ptil)_{i,l} = (i, m) (x) (m, l):
        Ptil_{i,l} = Atil_{i,m}^T (I + Ptil_{m,l} Dtil_{i,m})^{-1} Ptil_{m,l} Atil_{i,m} + Ptil_{i,m}
        Atil_{i,l} = Atil_{m,l} (I + Dtil_{i,m} Ptil_{m,l})^{-1} Atil_{i,m}
        Dtil_{i,l} = Atil_{m,l} (I + Dtil_{i,m} Ptil_{m,l})^{-1} Dtil_{i,m} Atil_{m,l}^T + Dtil_{m,l}."""
    A1, D1, P1 = left
    A2, D2, P2 = right
    I = np.eye(A1.shape[0])
    P = A1.T @ np.linalg.solve(I + P2 @ D1, P2 @ A1) + P1
    X = np.linalg.solve(I + D1 @ P2, np.hstack([A1, D1 @ A2.T]))
    n = A1.shape[0]
    return (A2 @ X[:, :n], A2 @ X[:, n:] + D2, P)


def kalman_scan(A, C, E, F, Xi, order="fold"):
    """Pi_0..Pi_N from the scan elements.  order "fold": Pi_{j+1} = e_j (x) (composition up to j);
    order "tree": each prefix composed as a balanced binary tree of the elements (the grouping of a
    parallel scan), which equals the fold by associativity."""
    N = A.shape[0]
    elems = [prior_element(np.asarray(Xi, dtype=np.float64))]
    elems += [scan_element(*(np.asarray(x[j], dtype=np.float64) for x in (A, C, E, F))) for j in range(N)]
    out = [elems[0][2]]
    if order == "fold":
        acc = elems[0]
        for j in range(N):
            acc = combine(elems[j + 1], acc)
            out.append(acc[2])
    elif order == "tree":
        def compose(seq):                 # seq ordered from the latest element to the earliest
            if len(seq) == 1:
                return seq[0]
            h = len(seq) // 2
            return combine(compose(seq[:h]), compose(seq[h:]))
        for j in range(1, N + 1):
            out.append(compose(elems[j::-1])[2])
    else:
        raise ValueError(order)
    return np.stack(out)


# ---------------------------------------------------------------------------------------------
# eq. backward_propagations
# ---------------------------------------------------------------------------------------------

def observer_responses(A, C, L):
    """Phihat^x_{k,k} = I; Phihat^x_{k,j} = Phihat^x_{k,j+1} (A_j + L_{j+1}^T C_j) for j < k;
    Phihat^y_{k,j} = Phihat^x_{k,j} L_j^T for 1 <= j <= k.  Dense ((N+1) n, (N+1) n) and
    ((N+1) n, (N+1) p) block lower-triangular arrays."""
    A, C, L = (np.asarray(x, dtype=np.float64) for x in (A, C, L))
    N, n, p = A.shape[0], A.shape[1], C.shape[1]
    PX = np.zeros(((N + 1) * n, (N + 1) * n))
    PY = np.zeros(((N + 1) * n, (N + 1) * p))
    for k in range(N + 1):
        blk = np.eye(n)
        PX[k * n:(k + 1) * n, k * n:(k + 1) * n] = blk
        for j in range(k - 1, -1, -1):
            blk = blk @ (A[j] + L[j].T @ C[j])
            PX[k * n:(k + 1) * n, j * n:(j + 1) * n] = blk
        for j in range(1, k + 1):
            PY[k * n:(k + 1) * n, j * p:(j + 1) * p] = PX[k * n:(k + 1) * n, j * n:(j + 1) * n] @ L[j - 1].T
    return PX, PY


# ---------------------------------------------------------------------------------------------
# The closed-loop maps
# ---------------------------------------------------------------------------------------------

def downshift(blocks, rows, cols):
    """Z X for the block-diagonal X = diag(X_0..X_{N-1}, 0): X_j at block (j+1, j), over times
    0..N.  blocks (N, rows, cols)."""
    N = blocks.shape[0]
    out = np.zeros(((N + 1) * rows, (N + 1) * cols))
    for j in range(N):
        out[(j + 1) * rows:(j + 2) * rows, j * cols:(j + 1) * cols] = blocks[j]
    return out


def closed_loop_maps(A, PBX, PBU, PX, PY):
    """M = I - Z A and
        Phi^xw = Phibar^x + Phihat^x - Phibar^x M Phihat^x,    Phi^uw = Phibar^u (I - M Phihat^x),
        Phi^xe = Phihat^y - Phibar^x M Phihat^y,               Phi^ue = -Phibar^u M Phihat^y."""
    A = np.asarray(A, dtype=np.float64)
    n = A.shape[1]
    M = np.eye(PX.shape[0]) - downshift(A, n, n)
    MX, MY = M @ PX, M @ PY
    return (PBX + PX - PBX @ MX, PBU - PBU @ MX, PY - PBX @ MY, -PBU @ MY)


def state_feedback_responses(A, Bm, K):
    """Phibar^x = (I - Z (A + B K))^{-1}, Phibar^u = K Phibar^x with K = diag(K_0..K_N): the
    responses of the state feedback u_k = K_k x_k, which satisfy (I - Z A) Phibar^x - Z B Phibar^u
    = I.  An input of the closed-loop maps (the state-feedback stage is not this stage's)."""
    A, Bm, K = (np.asarray(x, dtype=np.float64) for x in (A, Bm, K))
    N, n, m = A.shape[0], A.shape[1], Bm.shape[2]
    Acl = np.stack([A[j] + Bm[j] @ K[j] for j in range(N)])
    PX = np.linalg.inv(np.eye((N + 1) * n) - downshift(Acl, n, n))
    Kd = np.zeros(((N + 1) * m, (N + 1) * n))
    for k in range(N + 1):
        Kd[k * m:(k + 1) * m, k * n:(k + 1) * n] = K[k]
    return PX, Kd @ PX
