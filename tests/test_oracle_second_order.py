"""Pins of the second-order (inertial) oracle, oracle/second_order.py (CPU only).

The inertial step M (x+ - x - dt v)/dt^2 + D (x+ - x)/dt + dE(x+) = tau + J^T lam, v+ = (x+ - x)/dt,
is checked against: the paper's quasi-static step it reduces to at v = 0, D = 0 (eq. dynamics); the
implicit Euler recurrence of a linear spring chain solved by a dense linear solve; the closed-form
period and per-step decay of the implicit Euler oscillator; the discrete energy balance of a linear
chain; bounded energy with damping and contact off; and central differences of its Jacobians and of
a rollout gradient.
"""
import copy

import numpy as np
import pytest

from oracle import sim, second_order as so
from paper_2606_14188_b300 import scenes

from tests.test_oracle_pins import rope


def _chain(n, L, *, k_s, k_b, m, D, dt=0.01, alpha=0.0, beta=0.0, grasp=(0, None)):
    """A straight chain along x with spacing L, gravity off, no obstacles; grasped nodes held by
    grippers at their rest positions (the HARD grasp: stiffness D within r_grasp)."""
    X0 = np.stack([np.arange(n) * L, np.zeros(n), np.zeros(n)], axis=1)
    gn = (grasp[0], n - 1 if grasp[1] is None else grasp[1])
    sc, q = rope(n, X0, k_s=k_s, k_b=k_b, D=D, m=m, dt=dt, gravity=(0, 0, 0), grasp_nodes=gn)
    sc.p["damp_alpha"], sc.p["damp_beta"] = alpha, beta
    return sc, q


def _axial_matrices(sc):
    """The chain's axial stiffness (springs) and the grasp stiffness, n x n, written from the
    spring list: the 1-D linear elasticity of a straight chain moving along its axis."""
    n = sc.nv
    Ks = np.zeros((n, n))
    for a, b, k in zip(sc.a, sc.b, sc.k):
        Ks[a, a] += k; Ks[b, b] += k; Ks[a, b] -= k; Ks[b, a] -= k
    Kg = np.zeros((n, n))
    for j in sc.grasp:
        Kg[j, j] += sc.p["D_max"]
    return Ks, Kg


def test_reduces_to_the_quasi_static_step():
    """v = 0 and no damping: the inertial step is eq. (dynamics) itself, on a rope step with
    contact, in both modes; v+ is the displacement over dt."""
    w = scenes.workload(1)
    sc = sim.Scene(w["scene"]["params"], w["scene"]["rest_x"])
    q, U = w["q0"][0], w["U"][0]
    for t in range(10):
        for mode in (sim.HARD, sim.SMOOTH):
            qa, sta = sim.step(sc, q, U[t], mode)
            q2, st2 = so.step2(sc, so.lift(sc, q), U[t], mode)
            x2, v2, g2 = so.split_q2(sc, q2)
            xa, ga = sim.split_q(sc, qa)
            x0, _ = sim.split_q(sc, q)
            assert sta == st2 == 0
            assert np.max(np.abs(x2 - xa)) <= 1e-13
            np.testing.assert_array_equal(g2, ga)
            np.testing.assert_allclose(v2, (x2 - x0) / sc.dt, rtol=0, atol=1e-10)
        q, _ = sim.step(sc, q, U[t], sim.HARD)


@pytest.mark.parametrize("alpha,beta", [(0.0, 0.0), (0.8, 0.0), (0.0, 0.01), (0.5, 0.02)])
def test_linear_chain_is_the_implicit_euler_recurrence(alpha, beta):
    """A straight 4-node chain moving along its axis is a linear system: springs are linear in
    the axial displacement, the axial Rayleigh stiffness is the chain's stiffness matrix.  Its
    step is (M/dt^2 + D/dt + K) x+ = M/dt^2 (x + dt v) + D/dt x + K_g x_g + (springs at rest), a
    dense 4 x 4 solve; the oracle's 3-D Newton solve must follow it to rounding."""
    n, L, m, dt = 4, 0.1, 0.05, 0.01
    sc, q = _chain(n, L, k_s=200.0, k_b=20.0, m=m, D=1e3, dt=dt, alpha=alpha, beta=beta)
    Ks, Kg = _axial_matrices(sc)
    rest = np.arange(n) * L
    xg = rest.copy()                                      # the grippers hold their nodes' rest positions
    D = alpha * m * np.eye(n) + beta * Ks
    x0 = rest + np.array([0.0, 0.01, -0.005, 0.0])
    v0 = np.array([0.0, -0.3, 0.2, 0.1])
    X0 = np.stack([x0, np.zeros(n), np.zeros(n)], axis=1)
    V0 = np.stack([v0, np.zeros(n), np.zeros(n)], axis=1)
    _, _, g = so.split_q2(sc, so.lift(sc, q))
    q2 = so.join_q2(X0, V0, g)
    x, v = x0.copy(), v0.copy()
    Amat = m / dt ** 2 * np.eye(n) + D / dt + Ks + Kg
    for step in range(40):
        q2, st = so.step2(sc, q2, np.zeros(6), sim.HARD)
        assert st == 0
        rhs = m / dt ** 2 * (x + dt * v) + D @ x / dt + Ks @ rest + Kg @ xg
        xn = np.linalg.solve(Amat, rhs)
        v, x = (xn - x) / dt, xn
        X, V, _ = so.split_q2(sc, q2)
        np.testing.assert_allclose(X[:, 0], x, rtol=0, atol=1e-12)
        np.testing.assert_allclose(V[:, 0], v, rtol=0, atol=1e-9)
        assert np.max(np.abs(X[:, 1:])) == 0.0 and np.max(np.abs(V[:, 1:])) == 0.0


def test_linear_chain_energy_balance():
    """For a quadratic potential with stiffness K and constant D the implicit Euler step loses
    exactly  E_n - E_{n+1} = m |v+ - v|^2/2 + dt v+^T D v+ + dt^2 v+^T K v+/2  (kinetic + elastic +
    grasp springs): a check of every term of the step (inertia, both damping parts, potential)."""
    n, L, m, dt = 4, 0.1, 0.05, 0.01
    alpha, beta = 0.6, 0.015
    sc, q = _chain(n, L, k_s=200.0, k_b=20.0, m=m, D=1e3, dt=dt, alpha=alpha, beta=beta)
    Ks, Kg = _axial_matrices(sc)
    D = alpha * m * np.eye(n) + beta * Ks
    rest = np.arange(n) * L
    X0 = np.stack([rest + np.array([0.0, 0.02, -0.01, 0.0]), np.zeros(n), np.zeros(n)], axis=1)
    _, _, g = so.split_q2(sc, so.lift(sc, q))
    q2 = so.join_q2(X0, np.zeros((n, 3)), g)

    def E(q2):
        X, V, G = so.split_q2(sc, q2)
        e = 0.5 * m * float(np.sum(V * V)) + sim.elastic_energy(sc, X)
        for i, j in enumerate(sc.grasp):
            e += 0.5 * sc.p["D_max"] * float(np.sum((X[j] - G[i]) ** 2))
        return e

    e0 = E(q2)
    for step in range(30):
        q2n, st = so.step2(sc, q2, np.zeros(6), sim.HARD)
        _, V, _ = so.split_q2(sc, q2)
        _, Vn, _ = so.split_q2(sc, q2n)
        v, vn = V[:, 0], Vn[:, 0]
        loss = 0.5 * m * np.sum((vn - v) ** 2) + dt * vn @ D @ vn + 0.5 * dt ** 2 * vn @ (Ks + Kg) @ vn
        assert abs((E(q2) - E(q2n)) - loss) <= 1e-12 * e0
        q2 = q2n


def test_spring_mass_period_and_decay():
    """One node on a spring to a rigidly held node (grasp stiffness 1e9 against k = 100): the
    implicit Euler oscillator x+ = (x + dt v)/(1 + w^2 dt^2) has eigenvalues 1/(1 -+ i w dt), so it
    turns by atan(w dt) per step (period 2 pi/atan(w dt) steps) and shrinks by (1 + w^2 dt^2)^-1/2."""
    m, k, dt, L, A0 = 1.0, 100.0, 0.01, 0.1, 0.004
    sc, q = _chain(2, L, k_s=k, k_b=0.0, m=m, D=1e9, dt=dt, grasp=(0, 0))
    w = np.sqrt(k / m)
    X0 = np.array([[0.0, 0.0, 0.0], [L + A0, 0.0, 0.0]])
    _, _, g = so.split_q2(sc, so.lift(sc, q))
    q2 = so.join_q2(X0, np.zeros((2, 3)), g)
    xi = [A0]
    for _ in range(300):
        q2, st = so.step2(sc, q2, np.zeros(6), sim.HARD)
        assert st == 0
        X, _, _ = so.split_q2(sc, q2)
        xi.append(X[1, 0] - L)
    xi = np.array(xi)
    # upward zero crossings, linearly interpolated
    up = [i + xi[i] / (xi[i] - xi[i + 1]) for i in range(len(xi) - 1) if xi[i] < 0.0 <= xi[i + 1]]
    period = np.mean(np.diff(up))
    assert len(up) >= 3
    assert abs(period - 2 * np.pi / np.arctan(w * dt)) <= 2e-3 * period
    # amplitude decay over whole periods: |lambda| per step
    rho = 1.0 / np.sqrt(1.0 + (w * dt) ** 2)
    r = np.hypot(xi[1:], (xi[1:] - xi[:-1]) / (w * dt))      # a phase-plane radius
    n1, n2 = 40, 240
    assert abs(np.log(r[n2] / r[n1]) / (n2 - n1) - np.log(rho)) <= 0.02 * abs(np.log(rho))


def test_energy_bounded_with_damping_and_contact_off():
    """A sagging 3-D rope under gravity, ends held still, no obstacles, Rayleigh damping on:
    kinetic + elastic + gravity + grasp energy never rises above its start and falls overall."""
    w = scenes.workload(1)
    p = copy.deepcopy(w["scene"]["params"])
    p["obstacles"] = []
    p["damp_alpha"], p["damp_beta"] = 0.5, 0.01
    sc = sim.Scene(p, w["scene"]["rest_x"])
    q2 = so.lift(sc, w["q0"][0])

    def E(q2):
        X, V, G = so.split_q2(sc, q2)
        e = so.energy(sc, q2)
        for i, j in enumerate(sc.grasp):
            e += 0.5 * p["D_max"] * float(np.sum((X[j] - G[i]) ** 2))
        return e

    es = [E(q2)]
    for _ in range(80):
        q2, st = so.step2(sc, q2, np.zeros(6), sim.HARD)
        assert st == 0
        es.append(E(q2))
    es = np.array(es)
    scale = abs(es[0]) + 1.0
    assert np.all(es <= es[0] + 1e-12 * scale)
    assert es[-1] < es[0] - 1e-6 * scale
    assert np.all(np.diff(es) <= 1e-10 * scale)


def _damped_scene():
    w = scenes.workload(1)
    p = copy.deepcopy(w["scene"]["params"])
    p["damp_alpha"], p["damp_beta"] = 0.5, 0.02
    return sim.Scene(p, w["scene"]["rest_x"]), w


def test_inertial_step_jacobians_match_central_differences():
    """A_t, B_t of the smooth inertial step (forward-mode tangents through both stages, the damping's
    dependence on the step start included) against central differences of the step, at steps with
    and without contact; the adjoint is their transpose."""
    sc, w = _damped_scene()
    q0, U = w["q0"][0], w["U"][0]
    traj, st = so.rollout2(sc, so.lift(sc, q0), U, sim.SMOOTH)
    assert st == 0
    rng = np.random.default_rng(3)
    m2 = so.nq2(sc)
    for t in (3, 6, 9):                   # the grasp offset c is nonzero (|c| is not smooth at 0)
        jac = so.SmoothStepJacobian2(sc, traj[t], U[t])
        assert jac.defined
        A, B = jac.jacobians()
        dq, du = rng.standard_normal(m2), rng.standard_normal(6)
        errs = []
        for h in (1e-6, 1e-7):
            fp, _ = so.step2(sc, traj[t] + h * dq, U[t] + h * du, sim.SMOOTH, x_start=jac.xs)
            fm, _ = so.step2(sc, traj[t] - h * dq, U[t] - h * du, sim.SMOOTH, x_start=jac.xs)
            fd = (fp - fm) / (2 * h)
            errs.append(np.linalg.norm(fd - (A @ dq + B @ du)) / np.linalg.norm(fd))
        assert min(errs) <= 1e-6, (t, errs)
        qb = rng.standard_normal(m2)
        vq, vu = jac.vjp(qb)
        np.testing.assert_allclose(vq, A.T @ qb, rtol=0, atol=1e-9 * np.abs(A).max() * np.abs(qb).max() * m2)
        np.testing.assert_allclose(vu, B.T @ qb, rtol=0, atol=1e-9 * np.abs(B).max() * np.abs(qb).max() * m2)


def test_inertial_rollout_gradient_matches_central_differences():
    """dL/du of a smooth (consistent) inertial rollout of 6 steps against central differences of
    L along random control directions."""
    sc, w = _damped_scene()
    q20 = so.lift(sc, w["q0"][0])
    U = w["U"][0][:6].copy()
    r = so.rollout_vjp2(sc, q20, U, "consistent")
    assert r["status"] == 0
    rng = np.random.default_rng(5)
    for _ in range(3):
        dU = rng.standard_normal(U.shape)
        h = 1e-6
        Lp = so.rollout_vjp2(sc, q20, U + h * dU, "consistent")["L"]
        Lm = so.rollout_vjp2(sc, q20, U - h * dU, "consistent")["L"]
        fd = (Lp - Lm) / (2 * h)
        an = float(np.sum(r["dL_du"] * dU))
        assert abs(fd - an) <= 1e-5 * max(abs(fd), abs(an)), (fd, an)
