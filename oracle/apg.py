"""FP64 oracle of the analytic policy gradient (APG; arxiv 2606.14188, Sec. 4.3).

TEST INFRASTRUCTURE ONLY (see oracle/sim.py).

APG differentiates the closed-loop rollout of a policy through the simulator (eq. diff-sim) instead
of estimating the gradient from samples.  Readings (the paper prints neither the policy nor the
training objective):
  * the policy is one tanh hidden layer, u = pi_theta(q) = W2 tanh(W1 q + b1) + b2, with
    theta = (W1 [h][n_q], b1 [h], W2 [6][h], b2 [6]) packed into one vector in that order;
  * the rollout q_{t+1} = f(q_t, pi_theta(q_t)), t = 0..H-1, runs the nonsmooth step, and the
    objective is the planning loss of that closed-loop trajectory (grad.loss_and_seeds: goal,
    obstacle penalty, effort);
  * the gradient is the surrogate one of eq. diff-sim (the smooth step's Jacobians along the
    nonsmooth trajectory, each smooth re-solve started at the forward step's solution), with the
    policy's own derivatives in the chain:
        lambda_H = dL/dq_H;  for t = H-1..0:
        g_t = df/du^T lambda_{t+1} + dL/du_t,
        lambda_t = df/dq^T lambda_{t+1} + dL/dq_t + dpi/dq(q_t)^T g_t,
        dL/dtheta += dpi/dtheta(q_t)^T g_t.
"""
from __future__ import annotations

import numpy as np

from . import grad, sim


def n_theta(nq: int, h: int) -> int:
    return h * nq + h + 6 * h + 6


def unpack(theta, nq: int, h: int):
    theta = np.asarray(theta, dtype=np.float64)
    o = 0
    W1 = theta[o:o + h * nq].reshape(h, nq); o += h * nq
    b1 = theta[o:o + h]; o += h
    W2 = theta[o:o + 6 * h].reshape(6, h); o += 6 * h
    b2 = theta[o:o + 6]
    return W1, b1, W2, b2


def policy(theta, q, h: int):
    """u = W2 tanh(W1 q + b1) + b2 and the hidden activations."""
    W1, b1, W2, b2 = unpack(theta, q.size, h)
    a = np.tanh(W1 @ q + b1)
    return W2 @ a + b2, a


def policy_vjp(theta, q, h: int, g):
    """(dpi/dq^T g, dpi/dtheta^T g) for an output cotangent g [6]."""
    W1, b1, W2, b2 = unpack(theta, q.size, h)
    a = np.tanh(W1 @ q + b1)
    ga = (W2.T @ g) * (1.0 - a * a)
    dq = W1.T @ ga
    dth = np.concatenate([np.outer(ga, q).ravel(), ga, np.outer(g, a).ravel(), g])
    return dq, dth


def rollout(sc: sim.Scene, q0, theta, h: int, H: int, tol=sim.TOL_X):
    """The closed-loop nonsmooth rollout: traj [H+1][n_q], controls [H][6], stage-1 solutions, status."""
    q = np.asarray(q0, dtype=np.float64)
    traj, U, xs = [q], [], []
    status = 0
    for t in range(H):
        u, _ = policy(theta, q, h)
        info = {}
        q, st = sim.step(sc, q, u, sim.HARD, tol, info)
        status |= st
        traj.append(q)
        U.append(u)
        xs.append(info["xs"])
        if st:
            break
    return np.array(traj), np.array(U), xs, status


def rollout_grad(sc: sim.Scene, q0, theta, h: int, H: int, tol=sim.TOL_X):
    """L (the planning loss of the closed-loop trajectory) and dL/dtheta, dL/dq0."""
    traj, U, xs, status = rollout(sc, q0, theta, h, H, tol)
    if status:
        return dict(L=np.nan, dtheta=np.zeros(n_theta(sc.nq, h)), dq0=np.zeros(sc.nq), status=status,
                    traj=traj, U=U)
    L, seeds, dU = grad.loss_and_seeds(sc, traj, U)
    lam = seeds[H].copy()
    dth = np.zeros(n_theta(sc.nq, h))
    for t in range(H - 1, -1, -1):
        D_fwd = traj[t + 1][: sc.n].reshape(sc.nv, 3) - xs[t]
        jac = grad.SmoothStepJacobian(sc, traj[t], U[t], tol, x_start=xs[t], Delta_start=D_fwd)
        status |= jac.status
        if not jac.defined:
            return dict(L=np.nan, dtheta=np.zeros_like(dth), dq0=np.zeros(sc.nq), status=status | 1,
                        traj=traj, U=U)
        qb, ub = jac.vjp(lam)
        g = ub + dU[t]
        dq, dt = policy_vjp(theta, traj[t], h, g)
        lam = qb + seeds[t] + dq
        dth += dt
    return dict(L=L, dtheta=dth, dq0=lam, status=status, traj=traj, U=U)
