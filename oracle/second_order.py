"""FP64 oracle of the second-order (inertial) variant of the rope step.

TEST INFRASTRUCTURE ONLY (see oracle/sim.py).

The paper's step, eq. (dynamics), is quasi-static: M (q+ - q)/dt^2 + dE/dq(q+) = tau(u) + sum J^T lam.
Its inertial form keeps the node velocity v and Rayleigh damping D:

    M (x+ - x - dt v)/dt^2 + D (x+ - x)/dt + dE/dx(x+) = tau + sum J^T lam,    v+ = (x+ - x)/dt,

the implicit Euler step of M a = f - D v, the form of the fully dynamic simulator the paper compares
against (Sec. 5).  It is the paper's step when v = 0 and D = 0.  Readings (silent in the paper):

* State q2 = [x_1..x_nv, v_1..v_nv, g_1, g_2]: six values per node (the 240-dimensional state of a
  40-node rope), then the two kinematic grippers, g+ = g + u as in the quasi-static step.
* D = alpha M + beta K_ax(x), Rayleigh damping with the springs' axial stiffness
  K_ax = sum_s k_s u_s u_s^T (u_s the unit spring vector at the step start x): symmetric positive
  semidefinite and smooth in x (the full elastic Hessian is indefinite in compression).  D is
  fixed during a step, so stage 1 is still the root of the gradient of a potential,
      Psi2(z) = |z - x - dt v|_M^2/(2 dt^2) + (z - x)^T D (z - x)/(2 dt) + E(z) - tau^T z + grasp,
  found by the same damped Newton method, and stage 2 keeps P = dF/dq* (now with D/dt).
* Stage 1 starts at the inertial predictor x + dt v, the grasped nodes moved with their grippers.
* Contact, grasp and smoothing are those of the quasi-static step (oracle/sim.py).
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import LinAlgError

from . import sim
from .sim import HARD, SMOOTH, TOL_X, NEWTON_MAX, ST_NEWTON, ST_NONFINITE, ST_NOTPD


def nq2(sc: sim.Scene):
    return 2 * sc.n + 6


def split_q2(sc: sim.Scene, q2):
    q2 = np.asarray(q2, dtype=np.float64)
    n = sc.n
    return q2[:n].reshape(sc.nv, 3), q2[n:2 * n].reshape(sc.nv, 3), q2[2 * n:].reshape(2, 3)


def join_q2(x, v, g):
    return np.concatenate([x.ravel(), v.ravel(), g.ravel()])


def axial_blocks(sc: sim.Scene, x):
    """k_s u_s u_s^T per spring at node positions x [nv, 3] (complex-safe)."""
    d = x[sc.b] - x[sc.a]
    l2 = (d * d).sum(axis=1)
    return sc.k[:, None, None] * d[:, :, None] * d[:, None, :] / l2[:, None, None]


class Damping:
    """D/dt for one step, D = alpha M + beta K_ax(x) at the step start x: its band (lower band
    storage of oracle/sim.py), its node diagonal blocks and its product."""

    def __init__(self, sc: sim.Scene, x):
        p = sc.p
        self.sc = sc
        self.alpha = float(p.get("damp_alpha", 0.0))
        self.beta = float(p.get("damp_beta", 0.0))
        dt = sc.dt
        self.Kax = self.beta * axial_blocks(sc, x) / dt
        self.cm = self.alpha * sc.m / dt
        self.band = sim.band_zeros(sc)
        self.band[0, :] += self.cm
        sim.band_add_springs(sc, self.band, self.Kax)
        diag = np.zeros((sc.nv, 3, 3))
        diag[:, [0, 1, 2], [0, 1, 2]] = self.cm
        np.add.at(diag, sc.a, self.Kax)
        np.add.at(diag, sc.b, self.Kax)
        self.diag = diag

    def band_dense(self):
        """D/dt as a dense N x N matrix."""
        sc = self.sc
        N = sc.n
        M = np.zeros((N, N))
        for k in range(self.band.shape[0]):
            idx = np.arange(N - k)
            M[idx + k, idx] += self.band[k, :N - k]
            if k:
                M[idx, idx + k] += self.band[k, :N - k]
        return M

    def vec(self, V):
        sc = self.sc
        f = np.einsum("sij,sj->si", self.Kax, V[sc.b] - V[sc.a])
        out = self.cm * V
        np.add.at(out, sc.b, f)
        np.add.at(out, sc.a, -f)
        return out

    def psi(self, Y, Dl):
        """(Y + Dl)^T (D/dt) (Y + Dl)/2 - Y^T (D/dt) Y/2, written in the step Dl itself."""
        return float(np.sum(Dl * self.vec(Y + 0.5 * Dl)))


def stage1_solve2(sc: sim.Scene, x, xt, gstar, d, damp: Damping, tol=TOL_X, maxit=NEWTON_MAX, x_start=None):
    """Damped Newton for the root of F2(z) = dPsi2/dz (the quasi-static residual with the inertial
    anchor xt = x + dt v, plus D (z - x)/dt), the rules of sim.stage1_solve for a rope: the exact
    Hessian, the projected one where the exact one is not positive definite, an Armijo search on
    Psi2, and a stop only on an exact-Hessian step below tol."""
    X = np.array(x_start, dtype=np.float64)
    for it in range(maxit):
        F = sim.stage1_residual(sc, X, xt, gstar, d) + damp.vec(X - x)
        if not np.all(np.isfinite(F)):
            return X, it, ST_NONFINITE
        exact = True
        try:
            cb = sim.band_factor(sim.stage1_hessian_band(sc, X, d) + damp.band)
        except LinAlgError:
            cb = sim.band_factor(sim.stage1_hessian_band(sc, X, d, project=True) + damp.band)
            exact = False
        p = -sim.band_solve(cb, F)
        if np.max(np.abs(p)) <= tol and exact:
            return X + p, it + 1, 0
        slope = float(np.sum(F * p))
        alpha = 1.0
        for _ in range(60):
            dpsi = sim.psi_difference(sc, X, alpha * p, xt, gstar, d) + damp.psi(X - x, alpha * p)
            if dpsi <= 1e-4 * alpha * slope:
                break
            alpha *= 0.5
        X = X + alpha * p
    return X, maxit, ST_NEWTON


def step2(sc: sim.Scene, q2, u, mode, tol=TOL_X, info=None, x_start=None, Delta_start=None):
    """(q2, u) -> q2+ of the inertial step: stage 1 for x*, stage 2 (eq. dynamics-second-stage with
    P = dF2/dq*), x+ = x* + Delta, v+ = (x+ - x)/dt, g+ = g + u."""
    x, v, g = split_q2(sc, q2)
    gstar = g + np.asarray(u, dtype=np.float64).reshape(2, 3)
    xt = x + sc.dt * v
    if x_start is None:
        x_start = xt.copy()
        for i in range(2):
            x_start[sc.grasp[i]] = x[sc.grasp[i]] + gstar[i] - g[i]
    d = sim.grasp_stiffness(sc, x, g, mode)
    damp = Damping(sc, x)
    xs, it1, st1 = stage1_solve2(sc, x, xt, gstar, d, damp, tol, x_start=x_start)
    phi, n = sim.contact_geometry(sc, xs)
    if mode == HARD and np.all(phi >= 0.0):
        Delta, sig, it2, st2 = np.zeros((sc.nv, 3)), None, 0, 0
    else:
        kf = sc.p["kappa_hard"] if mode == HARD else None
        Delta, sig, it2, st2 = sim.stage2_ipm(sc, xs, d, phi, n, sc.p["kappa_c"], kf, tol,
                                              Delta_start=Delta_start, extra=damp)
    xp = xs + Delta
    if info is not None:
        info.update(xs=xs, Delta=Delta, sig=sig, phi=phi, n=n, d=d, gstar=gstar, damp=damp,
                    newton_it=it1, ipm_it=it2, status=st1 | st2)
    return join_q2(xp, (xp - x) / sc.dt, gstar), st1 | st2


def rollout2(sc: sim.Scene, q20, U, mode, tol=TOL_X, xs_out=None):
    """q2_0 .. q2_H (traj [H+1, 6 nv + 6]), status; stage 2 warm-started as sim.rollout."""
    H = U.shape[0]
    traj = np.zeros((H + 1, nq2(sc)))
    traj[0] = q20
    status = 0
    D_prev = None
    for t in range(H):
        info = {}
        traj[t + 1], st = step2(sc, traj[t], U[t], mode, tol, info, Delta_start=D_prev)
        D_prev = info["Delta"] if np.any(info["Delta"] != 0.0) else None
        status |= st
        if xs_out is not None:
            xs_out.append(info["xs"])
    return traj, status


def lift(sc: sim.Scene, q):
    """A quasi-static state [x, g] as the inertial state [x, 0, g] (at rest)."""
    x, g = sim.split_q(sc, q)
    return join_q2(x, np.zeros_like(x), g)


def energy(sc: sim.Scene, q2):
    """Kinetic + elastic + gravitational energy of the nodes (grasp springs excluded)."""
    x, v, _ = split_q2(sc, q2)
    return 0.5 * sc.m * float(np.sum(v * v)) + sim.elastic_energy(sc, x) - sc.m * float(np.sum(x @ sc.grav))


# ------------------------------------------------------------------------------------------
# derivatives of the smooth inertial step (the implicit function theorem on F2 = 0 and on the
# reduced stage-2 optimality, as oracle/grad.py does for the quasi-static step)
# ------------------------------------------------------------------------------------------

def _spring_block_jac(sc: sim.Scene, fn, X):
    """Sparse N x N Jacobian of the node field sum_s (+f_s at b, -f_s at a), f_s = fn(d_s), d_s =
    X_b - X_a, from the 3 x 3 complex-step Jacobians of fn."""
    from .grad import complex_step_jac, _blocks_to_sparse
    N = sc.n
    J = complex_step_jac(fn, X[sc.b] - X[sc.a])
    return (_blocks_to_sparse(sc.b, sc.b, J, (N, N)) + _blocks_to_sparse(sc.a, sc.a, J, (N, N))
            - _blocks_to_sparse(sc.b, sc.a, J, (N, N)) - _blocks_to_sparse(sc.a, sc.b, J, (N, N)))


class SmoothStepJacobian2:
    """The smooth inertial step's Jacobian at (q2, u), both ways: theta = (x, v, g, u)."""

    def __init__(self, sc: sim.Scene, q2, u, tol=TOL_X, x_start=None, Delta_start=None):
        from .grad import complex_step_jac, _blocks_to_sparse
        self.sc = sc
        info = {}
        self.q_next, st = step2(sc, q2, u, SMOOTH, tol, info, x_start=x_start, Delta_start=Delta_start)
        self.status = st
        self.counts = (info["newton_it"], info["ipm_it"])
        x, v, g = split_q2(sc, q2)
        xs, Delta, sig, phi, n, d, gstar, damp = (info[k] for k in
                                                 ("xs", "Delta", "sig", "phi", "n", "d", "gstar", "damp"))
        self.xs, self.Delta = xs, Delta
        p = sc.p
        kc, mu = p["kappa_c"], p["mu"]
        nv, N = sc.nv, sc.n
        self.defined = False
        try:
            ab1 = sim.stage1_hessian_band(sc, xs, d) + damp.band
            self.cb1 = sim.band_factor(ab1)
            ab2 = ab1.copy()
            if sig is not None and sig.shape[1]:
                W = sim.contact_force_jacobian(sig, n, kc, mu)
                sim.band_add_node_blocks(sc, ab2, np.arange(nv), W.sum(axis=1))
            self.cb2 = sim.band_factor(ab2)
        except LinAlgError:
            self.status |= ST_NOTPD
            return
        self.defined = True
        # dR/dq*: the spring third derivatives acting on Delta, and the contact forces at fixed Delta
        dlt = Delta[sc.b] - Delta[sc.a]
        Rx = _spring_block_jac(sc, lambda dd: np.einsum("sij,sj->si", sim.spring_hessian_d(sc.k, sc.L, dd), dlt), xs)
        r = p["node_radius"]
        for ob in sc.obstacles:
            def lam_of_x(xc, ob=ob):
                ph, nn = sim.obstacle_phi_normal(ob, xc, r)
                return sim.contact_force(Delta + ph[:, None] * nn, nn, kc, mu)
            Jl = complex_step_jac(lam_of_x, xs)
            Rx = Rx - _blocks_to_sparse(np.arange(nv), np.arange(nv), Jl, (N, N))
        self.Rx = Rx.tocsr()
        # the damping's dependence on the step-start x: d/dx [(D/dt) Y] for Y = x* - x (in F2) and
        # Y = Delta (in P Delta of R)
        bt = damp.beta / sc.dt

        def dD_of(Y):
            dY = Y[sc.b] - Y[sc.a]
            return _spring_block_jac(
                sc, lambda dd: bt * sc.k[:, None] * dd * ((dd * dY).sum(axis=1) / (dd * dd).sum(axis=1))[:, None], x)

        dDF = dD_of(xs - x).toarray()
        dDR = dD_of(Delta).toarray()
        # grasp stiffness gradients
        c = sim.grasp_offsets(sc, x, g)
        rho = np.linalg.norm(c, axis=1)
        gd = complex_step_jac(lambda cc: sim.grasp_stiffness_of_c(sc, cc, SMOOTH)[..., None], c)[:, 0, :]
        gd[rho == 0.0] = 0.0
        m2 = nq2(sc)
        xc, vc, gc, uc = slice(0, N), slice(N, 2 * N), slice(2 * N, m2), slice(m2, m2 + 6)
        # dF2/dtheta and dR/dq2
        Ft = np.zeros((N, m2 + 6))
        Ft[:, xc] = -sc.w * np.eye(N) - damp.band_dense() + dDF
        Ft[:, vc] = -sc.w * sc.dt * np.eye(N)
        Rq = np.zeros((N, m2))
        Rq[:, xc] = dDR
        for i in range(2):
            a = sc.grasp[i]
            ra = slice(3 * a, 3 * a + 3)
            gcols = slice(2 * N + 3 * i, 2 * N + 3 * i + 3)
            ucols = slice(m2 + 3 * i, m2 + 3 * i + 3)
            xa = slice(3 * a, 3 * a + 3)
            off = xs[a] - gstar[i]
            Ft[ra, gcols] += -d[i] * np.eye(3) + np.outer(off, gd[i])
            Ft[ra, xa] += np.outer(off, -gd[i])
            Ft[ra, ucols] += -d[i] * np.eye(3)
            Rq[ra, gcols] += np.outer(Delta[a], gd[i])
            Rq[ra, xa] += np.outer(Delta[a], -gd[i])
        self.Ft, self.Rq = Ft, Rq
        self.slices = (xc, vc, gc, uc)

    def jacobians(self):
        """A = dq2+/dq2 [6 nv + 6, 6 nv + 6] and B = dq2+/du [6 nv + 6, 6]."""
        sc = self.sc
        N, m2 = sc.n, nq2(sc)
        th = np.eye(m2 + 6)
        dxs = -sim.band_solve_cols(self.cb1, self.Ft @ th)
        dD = -sim.band_solve_cols(self.cb2, self.Rx @ dxs + self.Rq @ th[:m2])
        dxp = dxs + dD
        J = np.zeros((m2, m2 + 6))
        J[:N] = dxp
        J[N:2 * N] = (dxp - th[:N]) / sc.dt
        J[2 * N:, 2 * N:m2] = np.eye(6)
        J[2 * N:, m2:] = np.eye(6)
        return J[:, :m2], J[:, m2:]

    def vjp(self, qbar_next):
        """(q2bar, ubar) given the adjoint of q2+."""
        sc = self.sc
        N, m2 = sc.n, nq2(sc)
        xb = qbar_next[:N] + qbar_next[N:2 * N] / sc.dt
        gb = qbar_next[2 * N:]
        mu = sim.band_solve_cols(self.cb2, xb)
        nu = sim.band_solve_cols(self.cb1, xb - self.Rx.T @ mu)
        tbar = -(self.Ft.T @ nu)
        tbar[:m2] -= self.Rq.T @ mu
        tbar[:N] -= qbar_next[N:2 * N] / sc.dt
        tbar[2 * N:m2] += gb
        tbar[m2:] += gb
        return tbar[:m2], tbar[m2:]


def linearize2(sc: sim.Scene, Z, V, tol=TOL_X):
    """A_t, B_t of the smooth inertial step at each nominal (z_t, v_t), stage 1 started at the
    nominal next positions (as oracle/grad.linearize)."""
    H = V.shape[0]
    m2 = nq2(sc)
    A = np.zeros((H, m2, m2))
    Bm = np.zeros((H, m2, 6))
    for t in range(H):
        jac = SmoothStepJacobian2(sc, Z[t], V[t], tol, x_start=np.asarray(Z[t + 1])[: sc.n].reshape(sc.nv, 3))
        if jac.defined:
            A[t], Bm[t] = jac.jacobians()
        else:
            A[t], Bm[t] = np.nan, np.nan
    return A, Bm


def rollout_vjp2(sc: sim.Scene, q20, U, grad_mode="surrogate", tol=TOL_X):
    """Forward rollout of the inertial step and the adjoint of the planning loss of oracle/grad.py
    (a function of the positions and grippers; the velocities enter through the dynamics only).
    Returns dict(traj, L, dL_du, dL_dq0, status)."""
    from .grad import loss_and_seeds
    fwd = HARD if grad_mode == "surrogate" else SMOOTH
    xs_fwd = []
    traj, status = rollout2(sc, q20, U, fwd, tol, xs_out=xs_fwd)
    H = U.shape[0]
    N = sc.n
    pos = np.concatenate([traj[:, :N], traj[:, 2 * N:]], axis=1)
    L, seeds1, dU = loss_and_seeds(sc, pos, U)
    seeds = np.zeros_like(traj)
    seeds[:, :N] = seeds1[:, :N]
    seeds[:, 2 * N:] = seeds1[:, N:]
    qbar = seeds[H].copy()
    dL_du = np.zeros_like(U)
    for t in range(H - 1, -1, -1):
        D_fwd = traj[t + 1][:N].reshape(sc.nv, 3) - xs_fwd[t]
        jac = SmoothStepJacobian2(sc, traj[t], U[t], tol, x_start=xs_fwd[t], Delta_start=D_fwd)
        status |= jac.status
        if not jac.defined:
            L, dL_du[:], qbar = np.nan, np.nan, np.full_like(qbar, np.nan)
            break
        qb, ub = jac.vjp(qbar)
        dL_du[t] = ub + dU[t]
        qbar = qb + seeds[t]
    return dict(traj=traj, L=L, dL_du=dL_du, dL_dq0=qbar, status=status)
