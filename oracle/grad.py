"""FP64 oracle: implicit differentiation of the simulator step, the planning loss, rollout
adjoints and the per-step linearisation.

TEST INFRASTRUCTURE ONLY (see oracle/sim.py).

Sec. 4.1 "Differentiating Through Simulation": with theta = (q, u),
    dq*/dtheta = -(dF/dq*)^{-1} dF/dtheta                          (stage 1, implicit function)
    dq+/dq*    = -[I 0] K^{-1} dG/dq*                               (stage 2, KKT system)
and eq. (diff-sim) composes the two.  Stage 2 is differentiated through its reduced optimality
condition  R(Delta; q*, q) = P(q*, q) Delta - sum_i E_j lam_i(Delta_j + phi_i(q*) n_i(q*), n_i(q*)),
whose Jacobian in Delta is the barrier Newton matrix H2 = P + sum_i E_j W_i E_j^T; eliminating the
multipliers from K gives the same solve.  The total derivative keeps every dependence the paper's
compact formula leaves implicit: dP/dq* (third derivatives of E), dn/dq* and dphi/dq* of the
contact frames, and the direct dependence of P and F on q through the grasp stiffness d_i(q).

Derivative checks use the complex-step method (Squire & Trapp 1998): for a real-analytic f,
f'(x) = Im f(x + i h)/h to rounding for h = 1e-30.  Local element functions (a spring's Hessian
action, a contact force, a grasp stiffness) are differentiated this way; the stage solves use the
analytic F and dF/dq*.

Surrogate gradients (Sec. 4.1 "Contact Smoothing"): the gradient of a nonsmooth rollout is the
product of the SMOOTH step's Jacobians evaluated at the states of the nonsmooth trajectory.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
from numpy.linalg import LinAlgError

from . import sim
from .sim import SMOOTH, HARD

CS_H = 1e-30


def complex_step_jac(f, x0):
    """J[..., :, k] = d f / d x0[..., k] for x0 of shape (..., 3) (f maps (..., 3) -> (..., m))."""
    cols = []
    for k in range(x0.shape[-1]):
        xc = x0.astype(np.complex128)
        xc[..., k] += 1j * CS_H
        cols.append(np.imag(f(xc)) / CS_H)
    return np.stack(cols, axis=-1)


def _blocks_to_sparse(rows, cols, blocks, shape):
    """Assemble 3x3 blocks at node rows/cols into a sparse matrix."""
    r_idx, c_idx, vals = [], [], []
    for al in range(3):
        for be in range(3):
            r_idx.append(3 * rows + al)
            c_idx.append(3 * cols + be)
            vals.append(blocks[:, al, be])
    return sp.coo_matrix((np.concatenate(vals), (np.concatenate(r_idx), np.concatenate(c_idx))),
                         shape=shape).tocsr()


class SmoothStepJacobian:
    """Everything needed to apply the smooth step's Jacobian at (q, u), both ways."""

    def __init__(self, sc: sim.Scene, q, u, tol=sim.TOL_X, x_start=None, Delta_start=None):
        self.sc = sc
        info = {}
        qp, st = sim.step(sc, q, u, SMOOTH, tol, info, x_start=x_start, Delta_start=Delta_start)
        self.q_next = qp
        self.counts = (info["newton_it"], info["ipm_it"])
        self.status = st
        x, g = sim.split_q(sc, q)
        self.x, self.g = x, g
        xs, Delta, sig = info["xs"], info["Delta"], info["sig"]
        phi, n, d, gstar = info["phi"], info["n"], info["d"], info["gstar"]
        self.xs, self.Delta, self.sig, self.d, self.gstar = xs, Delta, sig, d, gstar
        p = sc.p
        kc, mu = p["kappa_c"], p["mu"]
        nv, N = sc.nv, sc.n

        # factorizations of dF/dq* and of the stage-2 Newton matrix H2 at the solution.  When
        # either is not positive definite (the stage-1 root is a saddle of the potential: an
        # unstable, buckled equilibrium) the step's Jacobian is reported as undefined (ST_NOTPD).
        self.defined = False
        try:
            self.cb1 = sim.band_factor(sim.stage1_hessian_band(sc, xs, d))
            W = sim.contact_force_jacobian(sig, n, kc, mu)
            ab2 = sim.stage1_hessian_band(sc, xs, d)
            sim.band_add_node_blocks(sc, ab2, np.arange(nv), W.sum(axis=1))
            self.cb2 = sim.band_factor(ab2)
        except LinAlgError:
            self.status |= sim.ST_NOTPD
            return
        self.defined = True

        # dR/dq*: spring third-derivative part
        dS = xs[sc.b] - xs[sc.a]
        dlt = Delta[sc.b] - Delta[sc.a]
        Jy = complex_step_jac(
            lambda dd: np.einsum("sij,sj->si", sim.spring_hessian_d(sc.k, sc.L, dd), dlt), dS)
        Rx = _blocks_to_sparse(sc.b, sc.b, Jy, (N, N)) + _blocks_to_sparse(sc.a, sc.a, Jy, (N, N)) \
            - _blocks_to_sparse(sc.b, sc.a, Jy, (N, N)) - _blocks_to_sparse(sc.a, sc.b, Jy, (N, N))
        # dR/dq*: contact part, lam_i(Delta_j + phi_i(x) n_i(x), n_i(x)) at fixed Delta
        r = p["node_radius"]
        for o, ob in enumerate(sc.obstacles):
            def lam_of_x(xc, ob=ob):
                ph, nn = sim.obstacle_phi_normal(ob, xc, r)
                return sim.contact_force(Delta + ph[:, None] * nn, nn, kc, mu)
            Jl = complex_step_jac(lam_of_x, xs)
            Rx = Rx - _blocks_to_sparse(np.arange(nv), np.arange(nv), Jl, (N, N))
        self.Rx = Rx.tocsr()

        # grasp stiffness gradients: d_i(c), c = g_i - x_a(i)
        c = sim.grasp_offsets(sc, x, g)
        self.c = c
        rho = np.linalg.norm(c, axis=1)
        gd = complex_step_jac(lambda cc: sim.grasp_stiffness_of_c(sc, cc, SMOOTH)[..., None], c)[:, 0, :]
        gd[rho == 0.0] = 0.0          # |c| is not differentiable at 0: take 0 there
        self.grad_d_c = gd            # d d_i / d c_i ; d/dg_i = +gd, d/dx_a = -gd

        nq = sc.nq
        # dR/dq (through P's grasp block d_i(q) Delta_a) : N x nq
        Rq = np.zeros((N, nq))
        # dF/dtheta, theta = (x, g, u) : N x (nq + 6)
        Ft = np.zeros((N, nq + 6))
        Ft[np.arange(N), np.arange(N)] = -sc.w
        for i in range(2):
            a = sc.grasp[i]
            ra = slice(3 * a, 3 * a + 3)
            gcols = slice(N + 3 * i, N + 3 * i + 3)
            ucols = slice(nq + 3 * i, nq + 3 * i + 3)
            xa_cols = slice(3 * a, 3 * a + 3)
            off = xs[a] - gstar[i]
            Ft[ra, gcols] += -d[i] * np.eye(3) + np.outer(off, gd[i])
            Ft[ra, xa_cols] += np.outer(off, -gd[i])
            Ft[ra, ucols] += -d[i] * np.eye(3)
            Rq[ra, gcols] += np.outer(Delta[a], gd[i])
            Rq[ra, xa_cols] += np.outer(Delta[a], -gd[i])
        self.Rq, self.Ft = Rq, Ft

    # -- products ------------------------------------------------------------------------
    def vjp(self, qbar_next):
        """(qbar, ubar) = the adjoint of (q, u) given the adjoint of q+ (eq. diff-sim: solve
        with K^T, VJP with dG/dq*, solve with (dF/dq*)^T, VJP with dF/dtheta)."""
        sc = self.sc
        N, nq = sc.n, sc.nq
        xbar_p = qbar_next[:N]
        gbar_p = qbar_next[N:]
        mu = sim.band_solve_cols(self.cb2, xbar_p)
        xbar_s = xbar_p - self.Rx.T @ mu
        nu = sim.band_solve_cols(self.cb1, xbar_s)
        tbar = -(self.Ft.T @ nu)
        tbar[:nq] -= self.Rq.T @ mu
        tbar[N:nq] += gbar_p
        tbar[nq:] += gbar_p
        return tbar[:nq], tbar[nq:]

    def jvp(self, dq, du):
        sc = self.sc
        N = sc.n
        th = np.concatenate([dq, du])
        dxs = -sim.band_solve_cols(self.cb1, self.Ft @ th)
        dD = -sim.band_solve_cols(self.cb2, self.Rx @ dxs + self.Rq @ dq)
        return np.concatenate([dxs + dD, dq[N:] + du])

    def jacobians(self):
        """A = dq+/dq [nq, nq] and B = dq+/du [nq, 6] by forward-mode tangents."""
        sc = self.sc
        nq = sc.nq
        N = sc.n
        th = np.eye(nq + 6)
        dxs = -sim.band_solve_cols(self.cb1, self.Ft @ th)
        dD = -sim.band_solve_cols(self.cb2, self.Rx @ dxs + self.Rq @ th[:nq])
        J = np.zeros((nq, nq + 6))
        J[:N] = dxs + dD
        J[N:, N:nq] = np.eye(6)
        J[N:, nq:] = np.eye(6)
        return J[:, :nq], J[:, nq:]


# ------------------------------------------------------------------------------------------
# planning loss: goal + obstacle penalty + control effort
# ------------------------------------------------------------------------------------------

def loss_and_seeds(sc: sim.Scene, traj, U):
    """L = w_goal sum_{j in goal} |x_j(H) - goal_j|^2
           + w_pen sum_{t=1..H} sum_{j, o not a plane} max(0, margin - phi_jo(x_t))^2
           + w_u sum_t |u_t|^2,
    and dL/dq_t (t = 0..H), dL/du_t.  (The paper's planning cost J is not printed.)"""
    ls = sc.p["loss"]
    H = U.shape[0]
    seeds = np.zeros_like(traj)
    L = 0.0
    goal_nodes = np.asarray(ls["goal_nodes"], dtype=np.int64)
    if len(goal_nodes):
        xH = traj[H, : sc.n].reshape(sc.nv, 3)
        e = xH[goal_nodes] - np.asarray(ls["goal_pos"])
        L += ls["w_goal"] * float(np.sum(e * e))
        sH = seeds[H, : sc.n].reshape(sc.nv, 3)
        np.add.at(sH, goal_nodes, 2.0 * ls["w_goal"] * e)
    r = sc.p["node_radius"]
    for t in range(1, H + 1):
        xt = traj[t, : sc.n].reshape(sc.nv, 3)
        st = seeds[t, : sc.n].reshape(sc.nv, 3)
        for ob in sc.obstacles:
            if ob["type"] == "plane":
                continue
            ph, nn = sim.obstacle_phi_normal(ob, xt, r)
            v = np.maximum(0.0, ls["pen_margin"] - ph)
            L += ls["w_pen"] * float(np.sum(v * v))
            st += (-2.0 * ls["w_pen"] * v)[:, None] * nn
    L += ls["w_u"] * float(np.sum(U * U))
    dU = 2.0 * ls["w_u"] * U
    return L, seeds, dU


def rollout_vjp(sc: sim.Scene, q0, U, grad_mode="surrogate", dL_dtraj=None, tol=sim.TOL_X):
    """Forward rollout + adjoint.  grad_mode 'surrogate': nonsmooth forward, smooth Jacobians
    along it; 'consistent': smooth forward and its exact gradient.  The smooth re-solve of each
    step starts its Newton iteration at the forward step's stage-1 solution.  With dL_dtraj given, those
    seeds replace the planning loss.  Returns dict(traj, L, dL_du, dL_dq0, status)."""
    fwd = HARD if grad_mode == "surrogate" else SMOOTH
    xs_fwd = []
    traj, status, fwd_counts = sim.rollout(sc, q0, U, fwd, tol, xs_out=xs_fwd)
    H = U.shape[0]
    if dL_dtraj is None:
        L, seeds, dU = loss_and_seeds(sc, traj, U)
    else:
        L, seeds, dU = 0.0, np.asarray(dL_dtraj, dtype=np.float64), np.zeros_like(U)
    qbar = seeds[H].copy()
    dL_du = np.zeros_like(U)
    smooth_counts = []
    for t in range(H - 1, -1, -1):
        # the smooth re-solve starts its Newton iteration at the forward step's stage-1 solution
        # and its interior point at the forward step's stage-2 displacement
        D_fwd = traj[t + 1][: sc.n].reshape(sc.nv, 3) - xs_fwd[t]
        jac = SmoothStepJacobian(sc, traj[t], U[t], tol, x_start=xs_fwd[t], Delta_start=D_fwd)
        status |= jac.status
        smooth_counts.append(jac.counts)
        if not jac.defined:          # no gradient through a step without a defined Jacobian
            L, dL_du[:], qbar = np.nan, np.nan, np.full_like(qbar, np.nan)
            break
        qb, ub = jac.vjp(qbar)
        dL_du[t] = ub + dU[t]
        qbar = qb + seeds[t]
    return dict(traj=traj, L=L, dL_du=dL_du, dL_dq0=qbar, status=status, fwd_counts=fwd_counts,
                smooth_counts=smooth_counts[::-1])


def linearize(sc: sim.Scene, Z, V, tol=sim.TOL_X):
    """A_t = dq_{t+1}/dq_t and B_t = dq_{t+1}/du_t of the smooth step at each nominal (z_t, v_t)
    (the linearisation A(z, v), B(z, v) consumed by the SLS tube synthesis of Sec. 4.2).  The
    stage-1 Newton iteration of step t starts at the nominal next state z_{t+1}, so the step is
    linearised at the root next to the nominal trajectory."""
    H = V.shape[0]
    A = np.zeros((H, sc.nq, sc.nq))
    Bm = np.zeros((H, sc.nq, 6))
    for t in range(H):
        jac = SmoothStepJacobian(sc, Z[t], V[t], tol, x_start=np.asarray(Z[t + 1])[: sc.n].reshape(sc.nv, 3))
        if jac.defined:
            A[t], Bm[t] = jac.jacobians()
        else:
            A[t], Bm[t] = np.nan, np.nan
    return A, Bm
