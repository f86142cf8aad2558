"""FP64 oracle: the gradient-based MPC plan solve that the served planner runs.

TEST INFRASTRUCTURE ONLY (see oracle/sim.py).

Sec. 4.2 ("MPC ... nominal trajectory generation") and the planning experiments of Sec. 5 optimise
the control sequence of a rollout by gradients of the simulator (the surrogate gradients of
Sec. 4.1).  The paper prints neither the optimiser nor its settings; the planner here is:

  candidates   u^(0) = clip(w), u^(r) = clip(w + sigma eps^(r)), r = 1..R-1, with w the warm
               start and eps^(r)[t][d] standard normals drawn from a counter-based generator
               keyed by (seed, r, t, d);
  iterations   it = 1..G: L^(r), g^(r) = loss and surrogate gradient of rollout r (one batched
               forward + adjoint); after evaluations 1..G-1, one Adam step (Kingma & Ba 2015:
               bias-corrected first and second moments) on every candidate whose rollout
               succeeded, then clip to [-u_max, u_max];
  result       the evaluated control sequence with the lowest loss over all G evaluations and all
               candidates (ties: earlier evaluation, then lower r), with that loss.  Rollouts
               flagged by the simulator take no part in the minimum and are not updated.

Counter-based normals: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel random numbers: as
easy as 1, 2, 3", SC 2011): a 4 x 32-bit counter and a 2 x 32-bit key pass through 10 rounds of
two 32 x 32 -> 64-bit multiplications, with the key bumped by two Weyl constants between rounds.
Element e = 6 t + d of candidate r uses counter (e >> 1, r, 0, 0) and key (seed low 32 bits,
seed high 32 bits); words x0, x1 of the output give u1 = (x0 + 1) 2^-32 in (0, 1] and
u2 = x1 2^-32, and Box-Muller gives the pair sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2), of which
element e takes the first (e even) or the second (e odd).
"""
from __future__ import annotations

import math

import numpy as np

from . import sim
from . import grad

MASK32 = 0xFFFFFFFF
PHILOX_M0, PHILOX_M1 = 0xD2511F53, 0xCD9E8D57
PHILOX_W0, PHILOX_W1 = 0x9E3779B9, 0xBB67AE85

ADAM_B1, ADAM_B2, ADAM_EPS = 0.9, 0.999, 1e-8


def philox4x32_10(ctr, key):
    """Philox4x32 with 10 rounds on Python integers; returns the four 32-bit output words."""
    c0, c1, c2, c3 = (int(x) & MASK32 for x in ctr)
    k0, k1 = (int(x) & MASK32 for x in key)
    for rnd in range(10):
        if rnd:
            k0 = (k0 + PHILOX_W0) & MASK32
            k1 = (k1 + PHILOX_W1) & MASK32
        p0 = PHILOX_M0 * c0
        p1 = PHILOX_M1 * c2
        hi0, lo0 = p0 >> 32, p0 & MASK32
        hi1, lo1 = p1 >> 32, p1 & MASK32
        c0, c1, c2, c3 = (hi1 ^ c1 ^ k0) & MASK32, lo1, (hi0 ^ c3 ^ k1) & MASK32, lo0
    return c0, c1, c2, c3


def candidate_normals(seed: int, r: int, H: int) -> np.ndarray:
    """eps^(r) [H][6] of the planner's candidate r."""
    key = (seed & MASK32, (seed >> 32) & MASK32)
    out = np.zeros(6 * H)
    for e in range(6 * H):
        x0, x1, _, _ = philox4x32_10((e >> 1, r, 0, 0), key)
        u1 = (x0 + 1.0) * 2.0 ** -32
        u2 = x1 * 2.0 ** -32
        rad = math.sqrt(-2.0 * math.log(u1))
        ang = 2.0 * math.pi * u2
        out[e] = rad * (math.cos(ang) if e % 2 == 0 else math.sin(ang))
    return out.reshape(H, 6)


def initial_candidates(warm, R: int, sigma: float, u_max: float, seed: int) -> np.ndarray:
    H = warm.shape[0]
    U = np.zeros((R, H, 6))
    for r in range(R):
        U[r] = warm if r == 0 else warm + sigma * candidate_normals(seed, r, H)
    return np.clip(U, -u_max, u_max)


def adam_step(u, g, m, v, it: int, lr: float, u_max: float):
    """One Adam step (evaluation count it >= 1) followed by the box clip; returns (u, m, v)."""
    m = ADAM_B1 * m + (1.0 - ADAM_B1) * g
    v = ADAM_B2 * v + (1.0 - ADAM_B2) * g * g
    mh = m / (1.0 - ADAM_B1 ** it)
    vh = v / (1.0 - ADAM_B2 ** it)
    u = np.clip(u - lr * mh / (np.sqrt(vh) + ADAM_EPS), -u_max, u_max)
    return u, m, v


def plan_solve(sc: sim.Scene, q0, warm, R: int, G: int, lr: float = 0.005, sigma: float = 0.02,
               u_max: float = 0.05, seed: int = 0, tol=sim.TOL_X):
    """The plan solve: returns dict(u, L, it, r, losses [G][R], status [G][R])."""
    warm = np.asarray(warm, dtype=np.float64)
    U = initial_candidates(warm, R, sigma, u_max, seed)
    M = np.zeros_like(U)
    V = np.zeros_like(U)
    best = dict(u=U[0].copy(), L=math.inf, it=-1, r=-1)
    losses = np.full((G, R), np.nan)
    stats = np.zeros((G, R), dtype=np.int64)
    for it in range(1, G + 1):
        grads = np.zeros_like(U)
        for r in range(R):
            out = grad.rollout_vjp(sc, q0, U[r], "surrogate", tol=tol)
            losses[it - 1, r] = out["L"]
            stats[it - 1, r] = out["status"]
            grads[r] = out["dL_du"]
            if out["status"] == 0 and out["L"] < best["L"]:
                best = dict(u=U[r].copy(), L=float(out["L"]), it=it, r=r)
        if it < G:
            for r in range(R):
                if stats[it - 1, r] == 0:
                    U[r], M[r], V[r] = adam_step(U[r], grads[r], M[r], V[r], it, lr, u_max)
    best["losses"] = losses
    best["status"] = stats
    return best
