"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks the oracle against something other than itself: a closed form, an invariant,
a limit, a finite difference, a complex-step derivative, an independent library solver, or a
structural number the paper prints.  A plausible mistake in the oracle (a dropped term, a sign,
a wrong index, a transposed operand) fails at least one of them.
"""
import os

import numpy as np
import pytest
from scipy.optimize import minimize

from oracle import sim, grad
from paper_2606_14188_b300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def rope(n, X0, *, k_s=500.0, k_b=25.0, D=1e4, m=0.01, dt=0.01, obstacles=(), rest=None,
         grippers=None, grasp_nodes=None, mu=0.5, kappa_c=1e-4, gravity=(0, 0, -9.81)):
    """A custom rope scene: node positions X0 [n,3]; rest positions `rest` (default X0);
    gripper positions (default on the grasped nodes)."""
    p = scenes.default_params("rope")
    p.update(n_nodes=n, node_mass=m, dt=dt, k_stretch=k_s, k_bend=k_b, D_max=D,
             obstacles=list(obstacles), mu=mu, kappa_c=kappa_c, gravity=gravity,
             grasp_nodes=grasp_nodes if grasp_nodes is not None else (0, n - 1))
    X0 = np.asarray(X0, dtype=np.float64)
    sc = sim.Scene(p, X0 if rest is None else rest)
    g = X0[list(p["grasp_nodes"])] if grippers is None else np.asarray(grippers, dtype=np.float64)
    return sc, sim.join_q(X0, g)


FAR = [[10.0, 10.0, 10.0], [-10.0, -10.0, 10.0]]   # grippers out of grasp range: d = 0 (HARD)


# ------------------------------------------------------------------------------------------
# stage 1 closed forms
# ------------------------------------------------------------------------------------------

def test_free_fall_exact():
    """No springs, no grasp, no contact: q_{k+1} = q_k + dt^2 g exactly (eq. dynamics with
    E = 0 and lambda = 0), so z_k = z_0 - k g dt^2."""
    X0 = np.array([[0.0, 0.0, 1.0], [0.3, 0.0, 1.0], [0.6, 0.1, 0.9]])
    sc, q = rope(3, X0, k_s=0.0, k_b=0.0, grippers=FAR)
    U = np.zeros((20, 6))
    traj, st, counts = sim.rollout(sc, q, U, sim.HARD)
    assert st == 0
    for k in range(21):
        x, _ = sim.split_q(sc, traj[k])
        np.testing.assert_allclose(x[:, 2], X0[:, 2] - k * 9.81 * 0.01 ** 2, atol=1e-13)
        np.testing.assert_allclose(x[:, :2], X0[:, :2], atol=1e-14)


def test_single_spring_to_anchor_closed_form():
    """Node 0 held rigidly by gripper 0 at height a; node 1 hangs on one spring (k, L).
    Stage 1 in 1-D: z+ = (w z + k (a - L) - m g)/(w + k), w = m/dt^2, a geometric approach to
    z_eq = a - L - m g/k with ratio w/(w + k)."""
    m, dt, k, L, a = 0.02, 0.01, 50.0, 0.1, 1.0
    X0 = np.array([[0.0, 0.0, a], [0.0, 0.0, a - L]])
    sc, q = rope(2, X0, k_s=k, k_b=0.0, D=1e12, m=m, dt=dt,
                 grippers=[[0.0, 0.0, a], [5.0, 5.0, 5.0]])
    w = m / dt ** 2
    z = a - L
    traj, st, _ = sim.rollout(sc, q, np.zeros((15, 6)), sim.HARD)
    for t in range(1, 16):
        z = (w * z + k * (a - L) - m * 9.81) / (w + k)
        x, _ = sim.split_q(sc, traj[t])
        assert abs(x[1, 2] - z) < 1e-10, (t, x[1, 2], z)
    z_eq = a - L - m * 9.81 / k
    r = w / (w + k)
    assert abs((z - z_eq) - r ** 15 * ((a - L) - z_eq)) < 1e-12


def test_grasp_spring_closed_form():
    """One free node pulled by a kinematic gripper through the grasp spring (zero rest length,
    stiffness D_max while |c| <= r_grasp): x+ = (w x + d (g + u) + m grav)/(w + d)."""
    m, dt, D = 0.01, 0.01, 300.0
    X0 = np.array([[0.0, 0.0, 0.5], [1.0, 0.0, 0.5]])
    g0 = np.array([[0.002, -0.001, 0.5], [9.0, 9.0, 9.0]])
    sc, q = rope(2, X0, k_s=0.0, k_b=0.0, D=D, m=m, dt=dt, grippers=g0)
    u = np.array([0.001, 0.002, -0.003, 0.0, 0.0, 0.0])
    qp, st = sim.step(sc, q, u, sim.HARD)
    w = m / dt ** 2
    expect = (w * X0[0] + D * (g0[0] + u[:3]) + m * np.array([0, 0, -9.81])) / (w + D)
    x, g = sim.split_q(sc, qp)
    np.testing.assert_allclose(x[0], expect, atol=1e-14)
    np.testing.assert_allclose(g[0], g0[0] + u[:3], atol=0)


def test_hanging_chain_parabola():
    """Zero-rest-length linear springs, both ends held: the fixed point of the quasi-static map
    is the static equilibrium, a parabola z_j = z_0 + (m g/2k) j (j - n) with x linear in j."""
    n_nodes, k, m = 11, 200.0, 0.002
    nlast = n_nodes - 1
    X0 = np.stack([np.linspace(0, 1, n_nodes), np.zeros(n_nodes),
                   np.full(n_nodes, 0.5) + 0.01 * np.sin(np.arange(n_nodes))], axis=1)
    X0[0, 2] = X0[-1, 2] = 0.5
    rest = np.zeros((n_nodes, 3))               # every spring has rest length 0
    sc, q = rope(n_nodes, X0, k_s=k, k_b=0.0, D=1e12, m=m, rest=rest,
                 grippers=[[0, 0, 0.5], [1, 0, 0.5]])
    for _ in range(400):
        qn, st = sim.step(sc, q, np.zeros(6), sim.HARD)
        if np.max(np.abs(qn - q)) < 1e-15:
            break
        q = qn
    x, _ = sim.split_q(sc, q)
    j = np.arange(n_nodes)
    z_expect = 0.5 + (m * 9.81 / (2 * k)) * j * (j - nlast)
    np.testing.assert_allclose(x[:, 2], z_expect, atol=1e-10)
    np.testing.assert_allclose(x[:, 0], j / nlast, atol=1e-10)


def test_vertical_chain_stretch():
    """A chain hanging from one end: spring j carries the weight of the nodes below it, so its
    length is L + (#nodes below) m g/k at equilibrium."""
    n_nodes, k, m, L = 6, 80.0, 0.01, 0.05
    X0 = np.stack([np.zeros(n_nodes), np.zeros(n_nodes), 1.0 - L * np.arange(n_nodes)], axis=1)
    sc, q = rope(n_nodes, X0, k_s=k, k_b=0.0, D=1e12, m=m,
                 grippers=[[0, 0, 1.0], [3.0, 3.0, 3.0]])
    for _ in range(2000):
        qn, _ = sim.step(sc, q, np.zeros(6), sim.HARD)
        if np.max(np.abs(qn - q)) < 1e-15:
            break
        q = qn
    x, _ = sim.split_q(sc, q)
    lengths = np.linalg.norm(np.diff(x, axis=0), axis=1)
    below = n_nodes - 1 - np.arange(n_nodes - 1)
    np.testing.assert_allclose(lengths, L + below * m * 9.81 / k, atol=1e-9)


def test_proximal_descent_invariant():
    """With contact off and the grasp stiffness fixed (HARD), each step minimises
    Psi(y) = |y - x|_M^2/(2 dt^2) + Pi(y), so Pi(q+) + |x+ - x|_M^2/(2 dt^2) <= Pi(q): the
    quasi-static map never increases the potential energy (no energy drift)."""
    w = scenes.workload(1)
    sc0 = w["scene"]
    p = dict(sc0["params"]); p["obstacles"] = []
    sc = sim.Scene(p, sc0["rest_x"])
    q = w["q0"][0].copy()

    def Pi(qq, gstar, d):
        x, _ = sim.split_q(sc, qq)
        v = sim.elastic_energy(sc, x) - sc.m * float(np.sum(x @ sc.grav))
        for i in range(2):
            v += 0.5 * d[i] * float(np.sum((gstar[i] - x[sc.grasp[i]]) ** 2))
        return v

    for t in range(15):
        x, g = sim.split_q(sc, q)
        d = sim.grasp_stiffness(sc, x, g, sim.HARD)
        qn, st = sim.step(sc, q, np.zeros(6), sim.HARD)
        xn, _ = sim.split_q(sc, qn)
        lhs = Pi(qn, g, d) + 0.5 * sc.w * float(np.sum((xn - x) ** 2))
        assert lhs <= Pi(q, g, d) + 1e-14
        q = qn


def test_translation_and_rotation_equivariance():
    """With no obstacles, a rigid translation of (q, rest state) commutes with the step;
    a rotation about z (gravity along -z) commutes with it too."""
    w = scenes.workload(1)
    p = dict(w["scene"]["params"]); p["obstacles"] = []
    sc = sim.Scene(p, w["scene"]["rest_x"])
    q = w["q0"][0]
    u = w["U"][0, 0]
    traj, _, _ = sim.rollout(sc, q, w["U"][0, :3], sim.SMOOTH)
    q = traj[-1]
    qn, _ = sim.step(sc, q, u, sim.SMOOTH)
    T = np.array([0.3, -0.2, 0.7])
    qT = q + np.tile(T, sc.nq // 3)
    qTn, _ = sim.step(sc, qT, u, sim.SMOOTH)
    np.testing.assert_allclose(qTn, qn + np.tile(T, sc.nq // 3), atol=1e-12)
    th = 0.7
    R = np.array([[np.cos(th), -np.sin(th), 0], [np.sin(th), np.cos(th), 0], [0, 0, 1]])
    qR = (q.reshape(-1, 3) @ R.T).ravel()
    uR = (u.reshape(-1, 3) @ R.T).ravel()
    qRn, _ = sim.step(sc, qR, uR, sim.SMOOTH)
    np.testing.assert_allclose(qRn, (qn.reshape(-1, 3) @ R.T).ravel(), atol=1e-12)


# ------------------------------------------------------------------------------------------
# stage 2
# ------------------------------------------------------------------------------------------

def _falling_node_scene(kappa_c=1e-4, mu=0.0):
    # node 0 falls from just above the ground through it in one step (dt large)
    X0 = np.array([[0.0, 0.0, 0.006], [1.0, 0.0, 0.5]])
    sc, q = rope(2, X0, k_s=0.0, k_b=0.0, m=0.01, dt=0.05, grippers=FAR,
                 obstacles=[scenes.plane((0, 0, 1), 0.0)], mu=mu, kappa_c=kappa_c)
    return sc, q


def test_stage2_single_node_hard_projection():
    """Diagonal P, one node through the plane: the SOCP solution projects the node back onto
    the plane, z+ = h + r (frictionless and, for an isotropic P, frictional alike)."""
    for mu in (0.0, 0.5):
        sc, q = _falling_node_scene(mu=mu)
        info = {}
        qp, st = sim.step(sc, q, np.zeros(6), sim.HARD, info=info)
        assert st == 0 and info["phi"][0, 0] < 0
        x, _ = sim.split_q(sc, qp)
        phi = info["phi"][0, 0]
        # the SOCP is solved along the barrier's central path down to kappa_hard, whose
        # solution is D = (-phi + sqrt(phi^2 + 4 kappa_hard/w))/2 = -phi + O(kappa_hard)
        kh = sc.p["kappa_hard"]
        D = (-phi + np.sqrt(phi * phi + 4 * kh / sc.w)) / 2
        assert abs(info["Delta"][0, 2] - D) < 1e-13
        assert abs(x[0, 2] - sc.p["node_radius"]) < 2 * kh / (sc.w * abs(phi))
        assert abs(x[0, 0]) < 1e-12 and abs(x[0, 1]) < 1e-12


def test_stage2_single_node_smooth_closed_form():
    """Smooth stage 2, P = w I, frictionless: min w/2 D^2 - kappa log(phi + D) gives
    D = (-phi + sqrt(phi^2 + 4 kappa/w))/2; with friction the tangential part vanishes by
    symmetry, so the same D holds, and s^T lambda = kappa exactly."""
    for mu in (0.0, 0.5):
        sc, q = _falling_node_scene(mu=mu)
        info = {}
        qp, st = sim.step(sc, q, np.zeros(6), sim.SMOOTH, info=info)
        phi = info["phi"][0, 0]
        kap = sc.p["kappa_c"]
        D = (-phi + np.sqrt(phi * phi + 4 * kap / sc.w)) / 2
        assert abs(info["Delta"][0, 2] - D) < 1e-13
        lam = sim.contact_force(info["sig"], info["n"], kap, mu)
        np.testing.assert_allclose((lam * info["sig"]).sum(-1), kap, rtol=1e-12)


def _contact_case(mu):
    """A 3-node rope dragged sideways into the ground: coupled P, friction matters."""
    X0 = np.array([[0.0, 0.0, 0.02], [0.05, 0.0, 0.01], [0.10, 0.0, 0.02]])
    sc, q = rope(3, X0, k_s=50.0, k_b=5.0, m=0.01, dt=0.05, D=200.0,
                 obstacles=[scenes.plane((0, 0, 1), 0.0)], mu=mu, kappa_c=1e-4)
    u = np.array([0.02, 0.01, -0.03, 0.03, 0.0, -0.03])
    return sc, q, u


@pytest.mark.parametrize("mu", [0.0, 0.3, 1.0])
def test_stage2_hard_kkt_and_independent_solver(mu):
    """The nonsmooth stage 2 solution satisfies the KKT conditions of eq. (dynamics-second-stage)
    (P Delta = sum J^T lambda, lambda in F_mu, s in F*_mu, s.lambda ~ 0) and matches an
    independent general-purpose solver (SciPy SLSQP) on the same small SOCP."""
    sc, q, u = _contact_case(mu)
    sc.p["kappa_hard"] = 1e-10          # the FP64 oracle can follow the path this far here
    info = {}
    qp, st = sim.step(sc, q, u, sim.HARD, info=info)
    assert st == 0
    phi, n, Delta, sig, xs, d = (info[k] for k in ("phi", "n", "Delta", "sig", "xs", "d"))
    assert np.any(phi < 0)
    kap = sc.p["kappa_hard"]
    lam = sim.contact_force(sig, n, kap, mu)
    s = Delta[:, None, :] + phi[..., None] * n
    sn = (s * n).sum(-1)
    st_norm = np.linalg.norm(s - sn[..., None] * n, axis=-1)
    ln = (lam * n).sum(-1)
    lt_norm = np.linalg.norm(lam - ln[..., None] * n, axis=-1)
    assert np.all(sn >= mu * st_norm - 1e-12)
    assert np.all(mu * ln >= lt_norm - 1e-12)
    assert np.all(np.abs((s * lam).sum(-1)) <= 1.01 * kap)
    PD = sim.stage1_hessian_vec(sc, xs, d, Delta)
    np.testing.assert_allclose(PD, lam.sum(axis=1), atol=1e-9)
    # independent solve
    P = np.zeros((sc.n, sc.n))
    for j in range(sc.n):
        e = np.zeros((sc.nv, 3)); e.reshape(-1)[j] = 1.0
        P[:, j] = sim.stage1_hessian_vec(sc, xs, d, e).ravel()
    cons = []
    for j in range(sc.nv):
        for o in range(phi.shape[1]):
            def cfun(z, j=j, o=o):
                sv = z.reshape(-1, 3)[j] + phi[j, o] * n[j, o]
                a = sv @ n[j, o]
                t = sv - a * n[j, o]
                return a - mu * np.sqrt(t @ t + 1e-30)
            cons.append(dict(type="ineq", fun=cfun))
    res = minimize(lambda z: 0.5 * z @ P @ z, np.abs(phi.min()) * np.tile([0, 0, 1.0], sc.nv),
                   jac=lambda z: P @ z, constraints=cons, method="SLSQP",
                   options=dict(ftol=1e-15, maxiter=500))
    # SLSQP meets the nonsmooth cone constraints only to ~1e-6, so the two agree to that; the
    # KKT checks above pin the interior-point solution itself
    np.testing.assert_allclose(Delta.ravel(), res.x, atol=2e-6)
    # the default end of the path (kappa_hard = 1e-6 N m) is within O(kappa_hard / lam_n)
    sc.p["kappa_hard"] = 1e-6
    info2 = {}
    sim.step(sc, q, u, sim.HARD, info=info2)
    lam_min = max(1e-3, float(np.min(np.linalg.norm(lam.sum(1), axis=1)[phi.min(1) < 0])))
    assert np.max(np.abs(info2["Delta"] - Delta)) <= 10 * 1e-6 / lam_min


def test_hard_contact_limit():
    """As kappa_c -> 0 the smooth step tends to the nonsmooth one, with error O(kappa)."""
    sc, q, u = _contact_case(0.5)
    sc.p["kappa_hard"] = 1e-11             # the nonsmooth reference, far down the path
    qh, _ = sim.step(sc, q, u, sim.HARD)
    errs = []
    for kap in (1e-4, 1e-5, 1e-6, 1e-7):
        sc.p["kappa_c"] = kap
        qs, st = sim.step(sc, q, u, sim.SMOOTH)
        assert st == 0
        errs.append(np.max(np.abs(qs - qh)))
    errs = np.array(errs)
    assert np.all(np.diff(errs) < 0)
    ratio = errs[:-1] / errs[1:]
    assert np.all(ratio > 3.0), errs            # ~10x per decade: first order in kappa


# ------------------------------------------------------------------------------------------
# element derivatives and geometry
# ------------------------------------------------------------------------------------------

def test_elastic_gradient_and_hessian_by_complex_step():
    rng = np.random.default_rng(1)
    w = scenes.workload(1)
    sc = sim.Scene(w["scene"]["params"], w["scene"]["rest_x"])
    X = w["scene"]["rest_x"] + 0.01 * rng.normal(size=(sc.nv, 3))
    G = sim.elastic_gradient(sc, X)
    for j in (0, 5, 19):
        for al in range(3):
            Xc = X.astype(complex); Xc[j, al] += 1e-30j
            d = Xc[sc.b] - Xc[sc.a]
            l = np.sqrt((d * d).sum(1))
            E = 0.5 * np.sum(sc.k * (l - sc.L) ** 2)
            assert abs(np.imag(E) / 1e-30 - G[j, al]) < 1e-12 * max(1, abs(G[j, al]))
    v = rng.normal(size=(sc.nv, 3))
    Hv = sim.stage1_hessian_vec(sc, X, np.zeros(2), v) - sc.w * v
    # directional derivative of the gradient
    Xc = X + 1e-30j * v
    d = Xc[sc.b] - Xc[sc.a]
    l = np.sqrt((d * d).sum(1))
    f = (sc.k * (l - sc.L) / l)[:, None] * d
    Gc = np.zeros_like(Xc); np.add.at(Gc, sc.b, f); np.add.at(Gc, sc.a, -f)
    np.testing.assert_allclose(np.imag(Gc) / 1e-30, Hv, atol=1e-9)


def test_band_hessian_matches_matvec():
    w = scenes.workload(3, B=1)
    sc = sim.Scene(w["scene"]["params"], w["scene"]["rest_x"])
    rng = np.random.default_rng(2)
    X = w["scene"]["rest_x"] + 0.002 * rng.normal(size=(sc.nv, 3))
    d = np.array([3.0, 7.0])
    ab = sim.stage1_hessian_band(sc, X, d)
    v = rng.normal(size=(sc.nv, 3))
    # band matvec
    n, bw = sc.n, sc.bw
    vv = v.ravel()
    out = ab[0] * vv
    for k in range(1, bw + 1):
        out[k:] += ab[k, : n - k] * vv[: n - k]
        out[: n - k] += ab[k, : n - k] * vv[k:]
    np.testing.assert_allclose(out, sim.stage1_hessian_vec(sc, X, d, v).ravel(), atol=1e-9)


def test_obstacle_sdf_and_normal():
    """Signed distances at points with known answers, and n = grad phi (complex step)."""
    bx = scenes.box((0.0, 0.0, 0.0), (0.1, 0.2, 0.3))
    pts = np.array([[0.5, 0.0, 0.0], [0.0, 0.0, -0.1], [0.4, 0.6, 0.0], [0.2, 0.4, 0.5],
                    [0.05, 0.0, 0.0]])
    phi, n = sim.obstacle_phi_normal(bx, pts, 0.0)
    np.testing.assert_allclose(phi, [0.4, -0.1, 0.5, np.sqrt(0.1 ** 2 + 0.2 ** 2 + 0.2 ** 2),
                                     -0.05], atol=1e-14)
    sp_ = scenes.sphere((0.1, 0.2, 0.3), 0.2)
    pts2 = np.array([[0.1, 0.2, 0.8], [0.4, 0.6, 0.3]])
    phi2, _ = sim.obstacle_phi_normal(sp_, pts2, 0.01)
    np.testing.assert_allclose(phi2, [0.5 - 0.2 - 0.01, 0.5 - 0.2 - 0.01], atol=1e-14)
    rng = np.random.default_rng(3)
    for ob in (bx, sp_, scenes.plane((0.3, 0.1, 1.0), 0.2)):
        P = rng.normal(size=(40, 3)) * 0.4
        _, nn = sim.obstacle_phi_normal(ob, P, 0.0)
        gradphi = grad.complex_step_jac(lambda z: sim.obstacle_phi_normal(ob, z, 0.0)[0][..., None], P)[:, 0, :]
        np.testing.assert_allclose(gradphi, nn, atol=1e-12)


def test_contact_force_is_barrier_gradient_and_W_its_jacobian():
    rng = np.random.default_rng(4)
    n = rng.normal(size=(10, 3)); n /= np.linalg.norm(n, axis=1, keepdims=True)
    mu, kap = 0.4, 1e-3
    sig = n * 0.5 + 0.05 * rng.normal(size=(10, 3))
    assert sim.in_cone_interior(sig, n, mu)
    bfun = lambda z: -kap / 2 * np.log((1 + mu * mu) * ((z * n).sum(-1)) ** 2 - mu * mu * (z * z).sum(-1))
    gb = grad.complex_step_jac(lambda z: bfun(z)[..., None], sig)[:, 0, :]
    np.testing.assert_allclose(sim.contact_force(sig, n, kap, mu), -gb, atol=1e-13)
    Jl = grad.complex_step_jac(lambda z: sim.contact_force(z, n, kap, mu), sig)
    np.testing.assert_allclose(sim.contact_force_jacobian(sig, n, kap, mu), -Jl, atol=1e-11)
    # lambda lies in the friction cone F_mu and s.lambda = kappa
    lam = sim.contact_force(sig, n, kap, mu)
    ln = (lam * n).sum(-1)
    lt = np.linalg.norm(lam - ln[:, None] * n, axis=1)
    assert np.all(mu * ln >= lt)
    np.testing.assert_allclose((lam * sig).sum(-1), kap, rtol=1e-12)


# ------------------------------------------------------------------------------------------
# gradients
# ------------------------------------------------------------------------------------------

def _rope20_state(t=9):
    w = scenes.workload(1)
    sc = sim.Scene(w["scene"]["params"], w["scene"]["rest_x"])
    traj, _, _ = sim.rollout(sc, w["q0"][0], w["U"][0, :t], sim.HARD)
    return sc, traj[-1], w["U"][0, t], w


def test_step_jacobian_vs_central_differences():
    """Implicit differentiation (eq. diff-sim, with the total derivative) against central
    differences of the smooth step, at a state with an active contact."""
    sc, q, u, _ = _rope20_state()
    J = grad.SmoothStepJacobian(sc, q, u)
    A, B = J.jacobians()
    h = 1e-6
    for k in list(range(0, sc.nq, 7)) + [sc.nq - 1]:
        e = np.zeros(sc.nq); e[k] = h
        col = (sim.step(sc, q + e, u, sim.SMOOTH)[0] - sim.step(sc, q - e, u, sim.SMOOTH)[0]) / (2 * h)
        np.testing.assert_allclose(A[:, k], col, atol=2e-7)
    for k in range(6):
        e = np.zeros(6); e[k] = h
        col = (sim.step(sc, q, u + e, sim.SMOOTH)[0] - sim.step(sc, q, u - e, sim.SMOOTH)[0]) / (2 * h)
        np.testing.assert_allclose(B[:, k], col, atol=2e-7)


def test_adjoint_dot_product():
    sc, q, u, _ = _rope20_state(6)
    J = grad.SmoothStepJacobian(sc, q, u)
    rng = np.random.default_rng(5)
    for _ in range(3):
        v, du, wv = rng.normal(size=sc.nq), rng.normal(size=6), rng.normal(size=sc.nq)
        qb, ub = J.vjp(wv)
        lhs = wv @ J.jvp(v, du)
        assert abs(lhs - (qb @ v + ub @ du)) < 1e-12 * max(1.0, abs(lhs))


def test_rollout_gradient_vs_central_differences():
    """dL/du of the whole rollout (CONSISTENT mode: smooth forward) against central
    differences of the planning loss."""
    w = scenes.workload(1)
    sc = sim.Scene(w["scene"]["params"], w["scene"]["rest_x"])
    q0, U = w["q0"][0], w["U"][0]
    r = grad.rollout_vjp(sc, q0, U, "consistent")

    def Lof(Uc):
        tr, _, _ = sim.rollout(sc, q0, Uc, sim.SMOOTH)
        return grad.loss_and_seeds(sc, tr, Uc)[0]

    for (t, k) in [(0, 0), (2, 4), (5, 2), (9, 5)]:
        E = np.zeros_like(U); E[t, k] = 1e-6
        fd = (Lof(U + E) - Lof(U - E)) / 2e-6
        assert abs(fd - r["dL_du"][t, k]) < 1e-7 * max(1.0, abs(fd)), (t, k, fd, r["dL_du"][t, k])


def test_linear_chain_jacobian_closed_form():
    """Zero-rest-length springs, no grasp, no contact: the step is linear,
    x+ = (w I + K)^{-1} (w x + f), so A_xx = (w I + K)^{-1} w exactly."""
    n_nodes, k, m, dt = 7, 40.0, 0.01, 0.01
    X0 = np.stack([np.linspace(0, 0.6, n_nodes), 0.01 * np.arange(n_nodes), np.full(n_nodes, 0.4)], 1)
    sc, q = rope(n_nodes, X0, k_s=k, k_b=3.0, D=0.0, m=m, dt=dt, rest=np.zeros((n_nodes, 3)),
                 grippers=FAR)
    A, B = grad.SmoothStepJacobian(sc, q, np.zeros(6)).jacobians()
    Lap = np.zeros((n_nodes, n_nodes))
    for a_, b_, kk in zip(sc.a, sc.b, sc.k):
        Lap[a_, a_] += kk; Lap[b_, b_] += kk; Lap[a_, b_] -= kk; Lap[b_, a_] -= kk
    w = m / dt ** 2
    Axx = np.kron(np.linalg.inv(w * np.eye(n_nodes) + Lap) * w, np.eye(3))
    np.testing.assert_allclose(A[: sc.n, : sc.n], Axx, atol=1e-13)
    np.testing.assert_allclose(A[sc.n:, sc.n:], np.eye(6), atol=0)
    np.testing.assert_allclose(B[sc.n:], np.eye(6), atol=0)


# ------------------------------------------------------------------------------------------
# structural numbers printed in the paper
# ------------------------------------------------------------------------------------------

def test_state_dimensions_printed_in_paper():
    """n_q = 3 n_v + n_u with two 3-D grippers (Sec. 4.1): the 8x8 cloth has 198 states
    (App. B.2), the drag-rope MPC tubes show 66 states (App. D) and the output-feedback rope 39
    (App. E); the fixture lists (nodes, n_q) with their sources."""
    rows = []
    with open(os.path.join(GOLDEN, "state_dims.txt")) as f:
        for line in f:
            line = line.split("#")[0].strip()
            if line:
                kind, a, b, nq = line.split()
                rows.append((kind, int(a), int(b), int(nq)))
    assert rows
    for kind, a, b, nq in rows:
        if kind == "cloth":
            p = scenes.default_params("cloth"); p.update(rows=a, cols=b, n_nodes=a * b)
            rest = np.stack(np.meshgrid(np.arange(a), np.arange(b), [0.0], indexing="ij"), -1).reshape(-1, 3) * 0.05
        else:
            p = scenes.default_params("rope"); p.update(n_nodes=a)
            rest = np.stack([np.arange(a) * 0.05, np.zeros(a), np.zeros(a)], 1)
        p["grasp_nodes"] = (0, 1)
        assert sim.Scene(p, rest).nq == nq


# ------------------------------------------------------------------------------------------
# second-order cone machinery of the stage-2 interior point
# ------------------------------------------------------------------------------------------

def _random_cone_pairs(seed, k=20):
    rng = np.random.default_rng(seed)
    s = np.concatenate([np.ones((k, 1)), 0.6 * rng.uniform(-1, 1, (k, 2))], axis=1) * rng.uniform(0.1, 3, (k, 1))
    z = np.concatenate([np.ones((k, 1)), 0.6 * rng.uniform(-1, 1, (k, 2))], axis=1) * rng.uniform(0.1, 3, (k, 1))
    return s, z


def test_tangent_frame_orthonormal():
    rng = np.random.default_rng(7)
    n = rng.normal(size=(200, 3))
    n[:5] = [[0, 0, 1], [0, 0, -1], [1, 0, 0], [0, -1, 0], [0, 0, -1 + 1e-12]]
    n /= np.linalg.norm(n, axis=1, keepdims=True)
    t1, t2 = sim.tangent_frame(n)
    F = np.stack([n, t1, t2], axis=1)
    np.testing.assert_allclose(F @ np.swapaxes(F, 1, 2), np.broadcast_to(np.eye(3), F.shape), atol=1e-12)


def test_nesterov_todd_scaling_properties():
    """W is symmetric positive definite with W z = W^{-1} s (the defining NT property)."""
    s, z = _random_cone_pairs(8)
    W, Winv, lam = sim.nt_scaling(s, z)
    np.testing.assert_allclose(np.einsum("kab,kb->ka", W, z), np.einsum("kab,kb->ka", Winv, s), atol=1e-12)
    np.testing.assert_allclose(W @ Winv, np.broadcast_to(np.eye(3), W.shape), atol=1e-12)
    assert np.all(np.linalg.eigvalsh(W) > 0)


def test_jordan_algebra_and_step_to_boundary():
    s, z = _random_cone_pairs(9)
    r = np.random.default_rng(10).normal(size=s.shape)
    v = sim.jordan_solve(s, r)
    np.testing.assert_allclose(sim.jordan(s, v), r, atol=1e-12)
    np.testing.assert_allclose(sim.jordan(s, sim.jordan_inverse(s)), np.tile([1.0, 0, 0], (len(s), 1)), atol=1e-12)
    d = np.random.default_rng(11).normal(size=s.shape)
    a = sim.max_step(s, d)
    fin = np.isfinite(a)
    edge = s[fin] + a[fin, None] * d[fin]
    np.testing.assert_allclose(sim.soc_det(edge), 0.0, atol=1e-10)
    assert np.all(edge[:, 0] >= -1e-12)
    # just inside / outside
    assert sim.soc_interior(s[fin] + 0.999 * a[fin, None] * d[fin])
    big = s[~fin] + 1e6 * d[~fin]
    assert np.all(big[:, 0] >= np.linalg.norm(big[:, 1:], axis=1) - 1e-6)


def test_central_point_scaling_equals_barrier_hessian():
    """On the central path s o z = kappa e, A^T W^{-2} A is the Hessian of the relaxed
    complementarity barrier and A^T z its force: the primal-dual iteration and the smoothed
    model share one definition."""
    rng = np.random.default_rng(12)
    n = rng.normal(size=(15, 3)); n /= np.linalg.norm(n, axis=1, keepdims=True)
    for mu in (0.2, 0.5, 1.3):
        A = sim.cone_frames(n, mu)
        tang = rng.normal(size=(15, 3))
        tang -= (tang * n).sum(1, keepdims=True) * n
        tang *= (0.6 * 0.01 / mu) / np.linalg.norm(tang, axis=1, keepdims=True)
        sig = n * 0.01 + tang
        s = np.einsum("iab,ib->ia", A, sig)
        assert sim.soc_interior(s)
        kap = 3e-4
        z = kap * sim.jordan_inverse(s)
        _, Winv, _ = sim.nt_scaling(s, z)
        AMA = np.einsum("iba,ibc,icd->iad", A, Winv @ Winv, A)
        np.testing.assert_allclose(AMA, sim.contact_force_jacobian(sig, n, kap, mu), rtol=1e-10, atol=1e-12)
        np.testing.assert_allclose(np.einsum("iab,ia->ib", A, z), sim.contact_force(sig, n, kap, mu), atol=1e-14)


def test_infeasible_cone_set_is_flagged():
    """A node pushed deep between two obstacles whose friction cones do not meet has no stage-2
    solution: the step is flagged CS_ST_CONTACT quickly instead of running to the cap."""
    X0 = np.array([[0.0, 0.0, 0.0], [0.3, 0.0, 0.3]])
    obs = [scenes.sphere((0.03, 0.0, 0.0), 0.04), scenes.sphere((-0.03, 0.0, 0.0), 0.04)]
    sc, q = rope(2, X0, k_s=0.0, k_b=0.0, m=0.01, dt=0.05, D=1e4, obstacles=obs, mu=0.8,
                 grippers=[[0.0, 0.0, 0.0], [5.0, 5.0, 5.0]])
    info = {}
    qp, st = sim.step(sc, q, np.zeros(6), sim.HARD, info=info)
    assert st & sim.ST_CONTACT
    assert info["ipm_it"] < 60


def test_saddle_root_has_no_defined_step_jacobian():
    """Three nodes on a line, the end nodes held, no gravity, the grippers pushed towards each
    other: by symmetry stage 1 returns the straight, compressed chain, whose transverse stiffness
    w + 2 k (1 - L/l) is negative once the compression is large enough (Euler buckling): the root
    is a saddle of the potential, dF/dq* is indefinite and the step's Jacobian is reported as
    undefined (ST_NOTPD), never as numbers."""
    L0, k, m, dt = 0.4, 500.0, 1e-3, 0.01
    X0 = np.array([[0.0, 0.0, 1.0], [L0, 0.0, 1.0], [2 * L0, 0.0, 1.0]])
    sc, q = rope(3, X0, k_s=k, k_b=0.0, m=m, dt=dt, gravity=(0, 0, 0))
    delta = 0.02
    u = np.array([delta, 0.0, 0.0, -delta, 0.0, 0.0])
    jac = grad.SmoothStepJacobian(sc, q, u)
    x, _ = sim.split_q(sc, jac.q_next)
    assert np.allclose(x[:, 1:], X0[:, 1:], atol=1e-12)             # still straight
    l = x[1, 0] - x[0, 0]
    assert l < L0 and sc.w + 2 * k * (1 - L0 / l) < 0                 # transverse saddle
    assert not jac.defined and (jac.status & sim.ST_NOTPD)
    r = grad.rollout_vjp(sc, q, u[None, :], "consistent")
    assert (r["status"] & sim.ST_NOTPD) and np.isnan(r["L"])
    # a small push keeps the chain stable: defined Jacobian
    jac2 = grad.SmoothStepJacobian(sc, q, u * 1e-3)
    assert jac2.defined and jac2.status == 0


# ------------------------------------------------------------------------------------------
# cloth stage 1
# ------------------------------------------------------------------------------------------

def _cloth_params(rows, cols, **kw):
    p = scenes.default_params("cloth")
    p.update(rows=rows, cols=cols, n_nodes=rows * cols, obstacles=[])
    p.update(kw)
    return p


def test_one_row_cloth_is_a_rope():
    """A cloth of one row has exactly the rope's springs (structural along the row = stretch,
    distance-2 along the row = bend); on a well-posed step (both roots minimisers) the cloth's
    shifted Newton and the rope's Newton reach the same root."""
    n = 9
    X0 = np.stack([np.linspace(0.0, 0.4, n), np.zeros(n), np.full(n, 0.3)], axis=1)
    prm = dict(node_mass=0.01, dt=0.01, k_stretch=500.0, k_bend=25.0, D_max=1e4,
               grasp_nodes=(0, n - 1), gravity=(0, 0, -9.81))
    pr = scenes.default_params("rope"); pr.update(n_nodes=n, obstacles=[], **prm)
    pc = _cloth_params(1, n, **prm)
    sr, sc = sim.Scene(pr, X0), sim.Scene(pc, X0)
    assert sorted(zip(sr.a, sr.b, sr.k)) == sorted(zip(sc.a, sc.b, sc.k))
    q0 = sim.join_q(X0, X0[[0, n - 1]])
    U = np.tile([0.01, 0.0, 0.0, -0.01, 0.0, 0.0], (4, 1))      # pull the ends apart: taut
    tr, st_r, _ = sim.rollout(sr, q0, U, sim.HARD)
    tc, st_c, _ = sim.rollout(sc, q0, U, sim.HARD)
    assert st_r == 0 and st_c == 0
    np.testing.assert_allclose(tc, tr, rtol=0, atol=1e-12)


def test_cloth_linear_springs_equilibrium_is_a_linear_solve():
    """Zero rest lengths make every spring linear, E = sum k/2 |x_b - x_a|^2, so stage 1 is the
    linear system (w I + K + D_g) x* = w x + m g + D_g g*, with K the spring-weighted graph
    Laplacian of the grid.  The test enumerates the grid's springs itself (4-neighbour
    structural, both diagonals of every cell shear, distance-2 along rows and columns bend)."""
    R, C = 4, 5
    n = R * C
    rng = np.random.default_rng(3)
    X0 = rng.normal(0.0, 0.05, size=(n, 3)) + np.array([0.0, 0.0, 0.3])
    rest = np.zeros((n, 3))                     # every rest length 0
    ks, ksh, kb, m, dt, D = 40.0, 20.0, 5.0, 0.01, 0.01, 300.0
    p = _cloth_params(R, C, node_mass=m, dt=dt, k_stretch=ks, k_shear=ksh, k_bend=kb, D_max=D,
                      grasp_nodes=(0, C - 1), gravity=(0, 0, -9.81))
    sc = sim.Scene(p, rest)
    g = X0[[0, C - 1]]
    u = np.array([0.01, 0.02, -0.01, -0.02, 0.0, 0.01])
    q1, st = sim.step(sc, sim.join_q(X0, g), u, sim.HARD)
    assert st == 0
    Kl = np.zeros((n, n))
    def spring(i, j, k):
        Kl[i, i] += k; Kl[j, j] += k; Kl[i, j] -= k; Kl[j, i] -= k
    idx = lambda r, c: r * C + c
    for r in range(R):
        for c in range(C):
            if c + 1 < C: spring(idx(r, c), idx(r, c + 1), ks)
            if r + 1 < R: spring(idx(r, c), idx(r + 1, c), ks)
            if r + 1 < R and c + 1 < C:
                spring(idx(r, c), idx(r + 1, c + 1), ksh); spring(idx(r, c + 1), idx(r + 1, c), ksh)
            if c + 2 < C: spring(idx(r, c), idx(r, c + 2), kb)
            if r + 2 < R: spring(idx(r, c), idx(r + 2, c), kb)
    w = m / dt ** 2
    A = w * np.eye(n) + Kl
    rhs = w * X0 + m * np.array([0.0, 0.0, -9.81])
    gs = g + u.reshape(2, 3)
    for i, j in enumerate((0, C - 1)):          # both grippers grasp (|c| = 0 <= r_grasp)
        A[j, j] += D
        rhs[j] += D * gs[i]
    x_ref = np.linalg.solve(A, rhs)
    x1, g1 = sim.split_q(sc, q1)
    np.testing.assert_allclose(x1, x_ref, rtol=0, atol=1e-12)
    np.testing.assert_allclose(g1, gs, rtol=0, atol=0)


def test_cloth_root_is_a_local_minimiser():
    """On a slack 16 x 16 cloth the shifted Newton ends at a point where F = 0 and dF/dq* is positive definite (it stops only on an unshifted step):
    a local minimiser of Psi, i.e. a stable quasi-static equilibrium."""
    sc_ = scenes.cloth_scene(16, 16, n_spheres=0, seed=5)
    sc = sim.Scene(sc_["params"], sc_["rest_x"])
    u = scenes.controls_normal_clear(sc_, 1, 1, seed=9)[0, 0]
    x, g = sim.split_q(sc, sc_["q0"])
    d = sim.grasp_stiffness(sc, x, g, sim.HARD)
    gs = g + u.reshape(2, 3)
    X0 = x.copy()
    for i in range(2):
        X0[sc.grasp[i]] += u[3 * i:3 * i + 3]
    xs, it, st = sim.stage1_solve(sc, x, gs, d, x_start=X0)
    assert st == 0 and it > 1
    F = sim.stage1_residual(sc, xs, x, gs, d)
    assert np.abs(F).max() <= 1e-9 * np.abs(sim.stage1_residual(sc, X0, x, gs, d)).max()
    ev = np.linalg.eigvalsh(_dense_from_band(sim.stage1_hessian_band(sc, xs, d)))
    assert ev.min() > 0.0


def _dense_from_band(ab):
    bw, n = ab.shape[0] - 1, ab.shape[1]
    A = np.zeros((n, n))
    for k in range(bw + 1):
        i = np.arange(n - k)
        A[i + k, i] = ab[k, : n - k]
        A[i, i + k] = ab[k, : n - k]
    return A


# ------------------------------------------------------------------------------------------
# grasp stiffness values, the planning loss value, the surrogate composition, the stage-1 start
# ------------------------------------------------------------------------------------------

def test_grasp_stiffness_values():
    """Sec. 4.1 Contact Smoothing: the smooth grasp stiffness D_max exp(-|c|/kappa) and the
    indicator-like nonsmooth one D_max 1[|c| <= r_grasp], at hand-chosen offsets (D_max 1e4 N/m,
    kappa_h 0.01 m, r_grasp 0.01 m): |c| = 0.005 m gives 1e4 e^(-1/2) = 6065.306597126334,
    |c| = 0.01 m gives 1e4 e^(-1) = 3678.7944117144234 and |c| = 0.0101 m 1e4 e^(-1.01) =
    3642.1897957152332 (a grasp smoothed with kappa_c = 1e-4, or with |c|^2, gives other values)."""
    p = scenes.default_params("rope")
    p.update(n_nodes=2, node_mass=0.01, grasp_nodes=(0, 1), D_max=1e4, kappa_h=0.01, r_grasp=0.01)
    sc = sim.Scene(p, np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0]]))
    c = np.array([[0.003, 0.004, 0.0], [0.0, 0.006, 0.008], [0.0, 0.0, 0.0101]])
    np.testing.assert_allclose(sim.grasp_stiffness_of_c(sc, c, sim.SMOOTH),
                               [6065.306597126334, 3678.7944117144234, 3642.1897957152332], rtol=1e-14)
    np.testing.assert_array_equal(sim.grasp_stiffness_of_c(sc, c, sim.HARD), [1e4, 1e4, 0.0])


def test_smooth_grasp_spring_closed_form():
    """The smooth stiffness enters stage 1 at the old state (eq. dynamics-first-stage uses c_i(q)):
    one free node, gripper offset c = (0.003, 0.004, 0) (|c| = 0.005 m), D_max = 300 N/m,
    kappa_h = 0.01 m, so d = 300 e^(-1/2); then x+ = (w x + d (g + u) + m grav)/(w + d) =
    (0.0025813550224302265, 0.00387203253364534, 0.49771606105242844) for w = 100."""
    m, dt, D = 0.01, 0.01, 300.0
    X0 = np.array([[0.0, 0.0, 0.5], [1.0, 0.0, 0.5]])
    g0 = np.array([[0.003, 0.004, 0.5], [9.0, 9.0, 9.0]])
    sc, q = rope(2, X0, k_s=0.0, k_b=0.0, D=D, m=m, dt=dt, grippers=g0)
    sc.p["kappa_h"] = 0.01
    u = np.array([0.001, 0.002, -0.003, 0.0, 0.0, 0.0])
    qp, st = sim.step(sc.__class__({**sc.p, "obstacles": []}, X0), q, u, sim.SMOOTH)
    x, _ = sim.split_q(sc, qp)
    np.testing.assert_allclose(x[0], [0.0025813550224302265, 0.00387203253364534, 0.49771606105242844],
                               rtol=0, atol=1e-15)


def _loss_scene():
    """Three nodes, a table plane z = 0 and a sphere (centre 0, radius 0.1 m); node radius 5 mm,
    margin 0.02 m, w_pen 100, goal node 2 at (0.5, 0, 0.3) with w_goal 1, w_u 0.01."""
    X0 = np.array([[0.0, 0.0, 1.0], [0.3, 0.0, 1.0], [0.6, 0.0, 1.0]])
    sc, _ = rope(3, X0, obstacles=[scenes.plane(), scenes.sphere((0.0, 0.0, 0.0), 0.1)])
    sc.p["loss"] = dict(goal_nodes=(2,), goal_pos=np.array([[0.5, 0.0, 0.3]]), w_goal=1.0,
                        w_pen=100.0, pen_margin=0.02, w_u=0.01)
    g = np.zeros(6)
    traj = np.array([
        np.concatenate([[0.105, 0, 0], [1, 0, 1], [2, 0, 1], g]),         # t = 0: not penalised
        np.concatenate([[0, 0.11, 0], [0, 0, -0.12], [1, 1, 1], g]),      # t = 1: node 1 below the table
        np.concatenate([[1, 0, 1], [0.3, 0, 0.4], [0.5, 0.1, 0.2], g]),   # t = 2 = H: goal error
    ], dtype=np.float64)
    U = np.array([[0.01, 0, 0, 0, 0.02, 0], [0, 0, 0, 0, 0, 0.03]], dtype=np.float64)
    return sc, traj, U


def test_loss_value_by_hand():
    """The planning loss on a 3-node, 2-step trajectory computed by hand:
      t = 1 node 0: phi_sphere = 0.11 - 0.1 - 0.005 = 0.005, 100 (0.02 - 0.005)^2 = 0.0225;
      t = 1 node 1: phi_sphere = 0.12 - 0.105 = 0.015, 100 (0.02 - 0.015)^2 = 0.0025
                    (its plane term, 100 (0.02 + 0.125)^2 = 2.1025, is excluded);
      t = 0 node 0 touches the sphere (0.04 if t = 0 were penalised): excluded;
      goal: |(0.5, 0.1, 0.2) - (0.5, 0, 0.3)|^2 = 0.02;  effort: 0.01 (1e-4 + 4e-4 + 9e-4) = 1.4e-5.
    L = 0.045014; seeds dL/dx_0(1) = -2 100 0.015 (0, 1, 0), dL/dx_1(1) = -2 100 0.005 (0, 0, -1),
    dL/dx_2(2) = 2 (0, 0.1, -0.1), dL/du = 0.02 u."""
    sc, traj, U = _loss_scene()
    L, seeds, dU = grad.loss_and_seeds(sc, traj, U)
    assert abs(L - 0.045014) < 1e-15
    expect = np.zeros_like(traj)
    expect[1, 0:3] = [0.0, -3.0, 0.0]
    expect[1, 3:6] = [0.0, 0.0, 1.0]
    expect[2, 6:9] = [0.0, 0.2, -0.2]
    np.testing.assert_allclose(seeds, expect, rtol=0, atol=1e-14)
    np.testing.assert_allclose(dU, 0.02 * U, rtol=0, atol=0)


def _contact_rope6():
    """Six nodes along x at z = 0.3 m, ends held, resting on a sphere (centre (0.125, 0, 0.2),
    radius 0.1 m) that the middle nodes penetrate by about 2 mm: a contact step from t = 0."""
    X0 = np.stack([np.linspace(0.0, 0.25, 6), np.zeros(6), np.full(6, 0.3)], axis=1)
    sc, q = rope(6, X0, m=0.1 / 6, obstacles=[scenes.plane(), scenes.sphere((0.125, 0.0, 0.2), 0.1)])
    sc.p["loss"] = dict(goal_nodes=(2, 3), goal_pos=X0[[2, 3]] + [0.0, 0.0, 0.05], w_goal=1.0,
                        w_pen=100.0, pen_margin=0.02, w_u=0.01)
    U = np.array([[0.002, 0, 0.003, -0.001, 0, 0.002],
                  [0.001, 0.001, 0.002, 0, -0.001, 0.003],
                  [0, 0.002, 0.001, 0.001, 0, 0.002]], dtype=np.float64)
    return sc, q, U


def test_surrogate_gradient_is_the_smooth_step_chain_at_the_hard_states():
    """The surrogate gradient (Sec. 4.1 Contact Smoothing): the nonsmooth rollout's loss,
    differentiated with the SMOOTH step's Jacobians evaluated at the NONSMOOTH trajectory's
    states.  Here those Jacobians come from central differences of the smooth step map at each
    (q_t, u_t) of the nonsmooth rollout (no implicit differentiation), chained by hand:
      lam_H = dL/dq_H;  dL/du_t = B_t^T lam_{t+1} + dL_u/du_t;  lam_t = A_t^T lam_{t+1} + dL/dq_t.
    The consistent gradient (smooth forward) differs from it by far more than the tolerance, so
    evaluating the Jacobians on the smooth trajectory, or one step off, fails."""
    sc, q0, U = _contact_rope6()
    H = U.shape[0]
    r = grad.rollout_vjp(sc, q0, U, "surrogate")
    traj, st, _ = sim.rollout(sc, q0, U, sim.HARD)
    assert st == 0 and r["status"] == 0
    phi, _ = sim.contact_geometry(sc, sim.split_q(sc, traj[1])[0])
    assert np.min(phi) < 0.05 * sc.p["node_radius"]          # the rollout is in contact
    L, seeds, dU = grad.loss_and_seeds(sc, traj, U)
    assert abs(L - r["L"]) < 1e-14
    h = 1e-6
    lam = seeds[H].copy()
    g_u = np.zeros_like(U)
    for t in range(H - 1, -1, -1):
        info = {}
        sim.step(sc, traj[t], U[t], sim.SMOOTH, info=info)
        xs0 = info["xs"]

        def f(qq, uu):
            return sim.step(sc, qq, uu, sim.SMOOTH, x_start=xs0)[0]

        A = np.zeros((sc.nq, sc.nq))
        for k in range(sc.nq):
            e = np.zeros(sc.nq); e[k] = h
            A[:, k] = (f(traj[t] + e, U[t]) - f(traj[t] - e, U[t])) / (2 * h)
        Bm = np.zeros((sc.nq, 6))
        for k in range(6):
            e = np.zeros(6); e[k] = h
            Bm[:, k] = (f(traj[t], U[t] + e) - f(traj[t], U[t] - e)) / (2 * h)
        g_u[t] = Bm.T @ lam + dU[t]
        lam = A.T @ lam + seeds[t]
    scale = np.max(np.abs(g_u))
    assert np.max(np.abs(g_u - r["dL_du"])) < 2e-6 * scale, (g_u, r["dL_du"])
    rc = grad.rollout_vjp(sc, q0, U, "consistent")
    assert np.max(np.abs(rc["dL_du"] - r["dL_du"])) > 1e-3 * scale


def test_surrogate_equals_consistent_without_contact_in_the_grasp_limit():
    """No obstacles and the grasp held (|c| stays far below r_grasp): with kappa_h large the
    smooth grasp stiffness equals D_max to 1e-9 and its slope is negligible, so the smooth and
    nonsmooth models coincide and the surrogate gradient must equal the consistent (exact)
    gradient of the same rollout."""
    X0 = np.stack([np.linspace(0.0, 0.3, 6), np.zeros(6), np.full(6, 0.3)], axis=1)
    sc, q0 = rope(6, X0, m=0.1 / 6)
    sc.p["kappa_h"] = 1e6
    sc.p["loss"] = dict(goal_nodes=(2, 3), goal_pos=X0[[2, 3]] + [0.0, 0.0, 0.05], w_goal=1.0,
                        w_pen=100.0, pen_margin=0.02, w_u=0.01)
    U = scenes.controls_normal(1, 5, sigma=0.005, seed=7)[0]
    rs = grad.rollout_vjp(sc, q0, U, "surrogate")
    rc = grad.rollout_vjp(sc, q0, U, "consistent")
    assert rs["status"] == 0 and rc["status"] == 0
    for t in range(U.shape[0] + 1):
        c = sim.grasp_offsets(sc, *sim.split_q(sc, rs["traj"][t]))
        assert np.max(np.linalg.norm(c, axis=1)) < 0.1 * sc.p["r_grasp"]
    assert abs(rs["L"] - rc["L"]) < 1e-12
    scale = np.max(np.abs(rc["dL_du"]))
    assert np.max(np.abs(rs["dL_du"] - rc["dL_du"])) < 1e-8 * scale
    np.testing.assert_allclose(rs["dL_dq0"], rc["dL_dq0"], rtol=0, atol=1e-8 * np.max(np.abs(rc["dL_dq0"])))


def _stage1_from(sc, q, u, moved, maxit=100):
    x, g = sim.split_q(sc, q)
    gstar = g + np.asarray(u).reshape(2, 3)
    d = sim.grasp_stiffness(sc, x, g, sim.HARD)
    xs0 = x.copy()
    if moved:
        for i in range(2):
            xs0[sc.grasp[i]] += gstar[i] - g[i]
    xs, _, st = sim.stage1_solve(sc, x, gstar, d, maxit=maxit, x_start=xs0)
    try:
        sim.band_factor(sim.stage1_hessian_band(sc, xs, d))
        pd = True
    except Exception:
        pd = False
    return xs, st, pd


def test_stage1_start_reaches_the_minimising_root():
    """Which root stage 1 returns (Sec. 4.1: "solved using Newton's method", start unstated).
    The iteration accepts a root only on a step taken with the exact Hessian, so the root is a
    local minimiser of the stage-1 potential (a stable equilibrium: stage 2's QP is convex there
    and dF/dq* of the adjoint positive definite).  The start is q with each grasped node moved
    with its gripper: the start at which the grasp offsets c_i are those of q, i.e. the linearised
    holonomic constraint J_i (q* - q) + c_i(q) = c_i(q) holds.  On the 1024 x 64-node rope
    workload, Newton from q itself does not converge within the cap of 100 iterations at the first
    step of rollouts 267, 384 and 727 (it wanders near saddles of the potential: the chain
    compressed between a moved gripper and its unmoved node), and where it converges given 2000
    iterations (rollout 384, after 385) it reaches the root of the moved start, which converges
    in 19-25.  On sampled rollouts both starts reach the same root to 1e-10 (all 50 steps)."""
    wl = scenes.workload(2)
    sc = sim.Scene(wl["scene"]["params"], wl["scene"]["rest_x"])
    U, q0 = wl["U"], wl["q0"]
    for b in (267, 384, 727):
        xa, sa, pda = _stage1_from(sc, q0[b], U[b, 0], moved=False)
        xb, sb, pdb = _stage1_from(sc, q0[b], U[b, 0], moved=True)
        assert sa == sim.ST_NEWTON and not pda, b
        assert sb == 0 and pdb, b
    xa, sa, pda = _stage1_from(sc, q0[384], U[384, 0], moved=False, maxit=2000)
    xb, sb, pdb = _stage1_from(sc, q0[384], U[384, 0], moved=True)
    assert sa == 0 and pda and np.max(np.abs(xa - xb)) < 1e-10
    for b in (0, 100, 521):
        q = q0[b]
        for t in range(U.shape[1]):
            xa, sa, pda = _stage1_from(sc, q, U[b, t], moved=False)
            xb, sb, pdb = _stage1_from(sc, q, U[b, t], moved=True)
            assert sb == 0 and pdb
            if sa == 0:
                assert np.max(np.abs(xa - xb)) < 1e-10, (b, t)
            q, _ = sim.step(sc, q, U[b, t], sim.HARD)
