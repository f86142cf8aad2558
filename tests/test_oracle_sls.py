"""Pins of the SLS observer oracle (oracle/sls.py, paper Sec. 4.2) against results fixed outside it:
Gaussian conditioning by brute force, the discrete algebraic Riccati equation, the affine constraints
of eq. phi_equation, the error covariance that the observer's responses imply, and the degenerate
case without measurements."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import sls


def _system(seed, n, p, N, nw=None, ne=None, rho=0.95):
    """A time-varying system with every matrix different at every step (an index slip changes the
    result)."""
    rng = np.random.default_rng(seed)
    nw = n if nw is None else nw
    ne = p if ne is None else ne
    A = np.stack([rho * sla.expm(0.3 * rng.normal(size=(n, n))) / np.exp(0.3 * np.sqrt(n) / 2)
                  + 0.1 * rng.normal(size=(n, n)) for _ in range(N)])
    C = rng.normal(size=(N, p, n))
    E = 0.3 * rng.normal(size=(N, n, nw))
    F = 0.2 * rng.normal(size=(N, p, ne)) + 0.3 * np.eye(p, ne)[None]
    Xi = 0.5 * rng.normal(size=(n, n))
    return A, C, E, F, Xi


def test_covariances_equal_gaussian_conditioning_by_brute_force():
    """Pi_j is the covariance of x_j given y_0..y_{j-1} for x_{j+1} = A_j x_j + w_j, y_j = C_j x_j +
    e_j, x_0 ~ N(0, Xi Xi^T), w_j ~ N(0, E_j E_j^T), e_j ~ N(0, F_j F_j^T): computed here from the
    joint covariance of all variables, as one linear map of the independent sources."""
    n, p, N = 3, 2, 4
    A, C, E, F, Xi = _system(1, n, p, N)
    Pi, _ = sls.kalman_recursion(A, C, E, F, Xi)
    n0, nw, ne = Xi.shape[1], E.shape[2], F.shape[2]
    ns = n0 + N * nw + N * ne                          # sources: x_0 noise, w_0.., e_0..
    X = [np.zeros((n, ns))]
    X[0][:, :n0] = Xi
    for j in range(N):
        Xn = A[j] @ X[j]
        Xn[:, n0 + j * nw:n0 + (j + 1) * nw] += E[j]
        X.append(Xn)
    Y = []
    for j in range(N):
        Yj = C[j] @ X[j]
        Yj[:, n0 + N * nw + j * ne:n0 + N * nw + (j + 1) * ne] += F[j]
        Y.append(Yj)
    for j in range(N + 1):
        if j == 0:
            cond = X[0] @ X[0].T
        else:
            Yo = np.vstack(Y[:j])
            Sxy = X[j] @ Yo.T
            cond = X[j] @ X[j].T - Sxy @ np.linalg.solve(Yo @ Yo.T, Sxy.T)
        assert np.allclose(Pi[j], cond, rtol=1e-10, atol=1e-12), j


def test_time_invariant_covariance_reaches_the_riccati_solution():
    """With constant (A, C, E, F) and a stable A, Pi_j converges to the stabilising solution of the
    filter's discrete algebraic Riccati equation (scipy's solver, with the duality A -> A^T,
    B -> C^T)."""
    n, p, N = 4, 2, 400
    A1, C1, E1, F1, Xi = _system(2, n, p, 1)
    A = np.repeat(A1, N, 0)
    C = np.repeat(C1, N, 0)
    E = np.repeat(E1, N, 0)
    F = np.repeat(F1, N, 0)
    Pi, L = sls.kalman_recursion(A, C, E, F, Xi)
    X = sla.solve_discrete_are(A1[0].T, C1[0].T, E1[0] @ E1[0].T, F1[0] @ F1[0].T)
    assert np.allclose(Pi[-1], X, rtol=1e-9, atol=1e-11)
    # the gain in its textbook predictor form K = A X C^T (C X C^T + R)^{-1}, x^+ = A x^ + K (y - C x^)
    K = sla.solve((C1[0] @ X @ C1[0].T + F1[0] @ F1[0].T).T, (A1[0] @ X @ C1[0].T).T).T
    assert np.allclose(-L[-1].T, K, rtol=1e-8, atol=1e-10)


@pytest.mark.parametrize("order", ["fold", "tree"])
def test_associative_scan_reproduces_the_recursion(order):
    n, p, N = 5, 3, 9
    A, C, E, F, Xi = _system(3, n, p, N)
    Pi, _ = sls.kalman_recursion(A, C, E, F, Xi)
    Ps = sls.kalman_scan(A, C, E, F, Xi, order=order)
    for j in range(N + 1):
        assert np.allclose(Ps[j], Pi[j], rtol=1e-10, atol=1e-12 * np.abs(Pi[j]).max()), j


def test_combination_rule_is_associative_on_generic_elements():
    rng = np.random.default_rng(4)
    n = 4

    def elem():
        G, H = rng.normal(size=(n, n)), rng.normal(size=(n, n))
        return (rng.normal(size=(n, n)), G @ G.T, H @ H.T)

    a, b, c = elem(), elem(), elem()
    x = sls.combine(sls.combine(a, b), c)
    y = sls.combine(a, sls.combine(b, c))
    for u, v in zip(x, y):
        assert np.allclose(u, v, rtol=1e-10, atol=1e-10)


def test_swapped_operands_of_the_combination_are_caught():
    """A plausible slip, composing the earlier step on the left, changes Pi_2 (the pins would fail
    on it)."""
    n, p, N = 3, 2, 2
    A, C, E, F, Xi = _system(5, n, p, N)
    Pi, _ = sls.kalman_recursion(A, C, E, F, Xi)
    e0 = sls.scan_element(A[0], C[0], E[0], F[0])
    e1 = sls.scan_element(A[1], C[1], E[1], F[1])
    pr = sls.prior_element(Xi)
    right = sls.combine(e1, sls.combine(e0, pr))[2]
    wrong = sls.combine(e0, sls.combine(e1, pr))[2]
    assert np.allclose(right, Pi[2], rtol=1e-10)
    assert not np.allclose(wrong, Pi[2], rtol=1e-3)


def _dense_C(C):
    N, p, n = C.shape
    return sls.downshift(C, p, n)


def test_observer_responses_satisfy_the_observer_constraint():
    """Phihat^x (I - Z A) - Phihat^y Z C = I (the observer half of eq. phi_equation), and Phihat^x
    is block lower triangular with identity diagonal blocks."""
    n, p, N = 4, 3, 6
    A, C, E, F, Xi = _system(6, n, p, N)
    _, L = sls.kalman_recursion(A, C, E, F, Xi)
    PX, PY = sls.observer_responses(A, C, L)
    I = np.eye((N + 1) * n)
    M = I - sls.downshift(A, n, n)
    R = PX @ M - PY @ _dense_C(C)
    assert np.allclose(R, I, atol=1e-11)
    assert np.allclose(np.triu(PX, 1)[np.kron(np.triu(np.ones((N + 1, N + 1)), 1), np.ones((n, n))) > 0], 0)


def test_observer_responses_imply_the_kalman_covariance():
    """The estimation error e_k = sum_j Phihat^x_{k,j} dx_j + sum_j Phihat^y_{k,j} dy_j with the
    independent disturbances dx_0 ~ N(0, Xi Xi^T), dx_{j+1} = w_j, dy_{j+1} = e_j has covariance
    Pi_k: the responses and the recursion agree only if the gains and their labels are right."""
    n, p, N = 4, 2, 7
    A, C, E, F, Xi = _system(7, n, p, N)
    Pi, L = sls.kalman_recursion(A, C, E, F, Xi)
    PX, PY = sls.observer_responses(A, C, L)
    for k in range(N + 1):
        S = PX[k * n:(k + 1) * n, 0:n] @ Xi @ Xi.T @ PX[k * n:(k + 1) * n, 0:n].T
        for j in range(1, k + 1):
            bx = PX[k * n:(k + 1) * n, j * n:(j + 1) * n]
            by = PY[k * n:(k + 1) * n, j * p:(j + 1) * p]
            S = S + bx @ E[j - 1] @ E[j - 1].T @ bx.T + by @ F[j - 1] @ F[j - 1].T @ by.T
        assert np.allclose(S, Pi[k], rtol=1e-10, atol=1e-12), k


def test_without_measurements_the_observer_is_the_open_loop():
    """C = 0: no gain, Phihat^x = (I - Z A)^{-1} and Pi follows the Lyapunov recursion."""
    n, p, N = 3, 2, 5
    A, C, E, F, Xi = _system(8, n, p, N)
    C = np.zeros_like(C)
    Pi, L = sls.kalman_recursion(A, C, E, F, Xi)
    assert np.all(L == 0)
    PX, PY = sls.observer_responses(A, C, L)
    assert np.allclose(PX, np.linalg.inv(np.eye((N + 1) * n) - sls.downshift(A, n, n)), atol=1e-12)
    assert np.all(PY == 0)
    P = Xi @ Xi.T
    for j in range(N):
        P = A[j] @ P @ A[j].T + E[j] @ E[j].T
        assert np.allclose(Pi[j + 1], P, rtol=1e-12)


def test_closed_loop_maps_satisfy_both_affine_constraints():
    """With Phibar from a state feedback, the assembled maps satisfy eq. phi_equation:
    [I - ZA, -ZB] Phi = [I, 0] and Phi [I - ZA; -ZC] = [I; 0]."""
    n, p, m, N = 4, 3, 2, 5
    A, C, E, F, Xi = _system(9, n, p, N)
    rng = np.random.default_rng(10)
    Bm = rng.normal(size=(N, n, m))
    K = 0.2 * rng.normal(size=(N + 1, m, n))
    PBX, PBU = sls.state_feedback_responses(A, Bm, K)
    I = np.eye((N + 1) * n)
    M = I - sls.downshift(A, n, n)
    ZB = sls.downshift(Bm, n, m)
    assert np.allclose(M @ PBX - ZB @ PBU, I, atol=1e-11)
    _, L = sls.kalman_recursion(A, C, E, F, Xi)
    PX, PY = sls.observer_responses(A, C, L)
    XW, UW, XE, UE = sls.closed_loop_maps(A, PBX, PBU, PX, PY)
    Phi = np.block([[XW, XE], [UW, UE]])
    left = np.hstack([M, -ZB]) @ Phi
    assert np.allclose(left, np.hstack([I, np.zeros(((N + 1) * n, (N + 1) * p))]), atol=1e-10)
    right = Phi @ np.vstack([M, -_dense_C(C)])
    assert np.allclose(right, np.vstack([I, np.zeros(((N + 1) * m, (N + 1) * n))]), atol=1e-10)


def _closed_loop_system(seed, n=4, p=3, m=2, N=5):
    A, C, E, F, Xi = _system(seed, n, p, N)
    rng = np.random.default_rng(seed + 100)
    Bm = rng.normal(size=(N, n, m))
    K = 0.2 * rng.normal(size=(N + 1, m, n))
    PBX, PBU = sls.state_feedback_responses(A, Bm, K)
    Pi, L = sls.kalman_recursion(A, C, E, F, Xi)
    PX, PY = sls.observer_responses(A, C, L)
    return dict(A=A, C=C, E=E, F=F, Bm=Bm, K=K, L=L,
                maps=sls.closed_loop_maps(A, PBX, PBU, PX, PY))


def simulate_observer_controller(s, x0, w, e):
    """The observer-based controller u_k = K_k xhat_k with the predictor xhat_{j+1} = A_j xhat_j
    + B_j u_j - L_{j+1}^T (y_j - C_j xhat_j), y_j = C_j x_j + e_j, on x_{j+1} = A_j x_j + B_j u_j
    + w_j, xhat_0 = 0: states x_0..x_N and controls u_0..u_N."""
    A, C, Bm, K, L = s["A"], s["C"], s["Bm"], s["K"], s["L"]
    N = A.shape[0]
    x, xh, xs, us = x0, np.zeros_like(x0), [x0], []
    for j in range(N):
        u = K[j] @ xh
        y = C[j] @ x + e[j]
        xh = A[j] @ xh + Bm[j] @ u - L[j].T @ (y - C[j] @ xh)
        x = A[j] @ x + Bm[j] @ u + w[j]
        xs.append(x)
        us.append(u)
    us.append(K[N] @ xh)
    return np.concatenate(xs), np.concatenate(us)


def test_closed_loop_maps_reproduce_the_observer_based_controller():
    """The assembled maps are the responses of the controller u = K xhat with the Kalman predictor:
    simulating that controller under random disturbances gives x = Phi^xw dx + Phi^xe dy and
    u = Phi^uw dx + Phi^ue dy (dx_0 = x_0, dx_{j+1} = w_j, dy_{j+1} = e_j)."""
    n, p, N = 4, 3, 5
    s = _closed_loop_system(11)
    rng = np.random.default_rng(12)
    x0, w, e = rng.normal(size=n), rng.normal(size=(N, n)), rng.normal(size=(N, p))
    xs, us = simulate_observer_controller(s, x0, w, e)
    XW, UW, XE, UE = s["maps"]
    dx = np.concatenate([x0, w.ravel()])
    dy = np.concatenate([np.zeros(p), e.ravel()])
    assert np.allclose(XW @ dx + XE @ dy, xs, atol=1e-12)
    assert np.allclose(UW @ dx + UE @ dy, us, atol=1e-12)
