"""FP64 CPU oracle of the contact-smoothed quasi-static rope/cloth simulator.

TEST INFRASTRUCTURE ONLY.  This package is imported by tests/, by __graft_entry__.smoke() and
by bench.py's cpu_baseline leg and reference arm -- nothing else.  It shares no code with the
CUDA path (no kernels, headers, helpers or constants); both are fed from the seeded generator
in paper_2606_14188_b300/scenes.py, which holds no simulator arithmetic.

What is computed, in the paper's order (Sec. 4.1, "Differentiable Deformable Object Simulator
with Contact Smoothing"):

* Eq. (dynamics): the implicit quasi-static step  M (q+ - q)/dt^2 + dE/dq(q+) = tau(u) + sum J^T lam.
  State q = [x_1..x_nv, g_1, g_2] (3-D node positions, then the two 3-D gripper positions).
* Eq. (dynamics-first-stage): stage 1.  q* is the root of
      F(q*) = M (q* - q)/dt^2 + dE/dq(q*) - tau(u) + sum_i J_i^T D_i (J_i (q* - q) + c_i(q)),
  found by Newton's method.  The grasp constraint c_i(q) = g_i - x_a(i) is linear, so the grasp
  term is a zero-rest-length spring of stiffness d_i(q) between g_i* and x*_a(i).
* Eq. (dynamics-second-stage): stage 2.  q+ = q* + Delta minimises 1/2 Delta^T P Delta subject to
  J_i(q*) Delta + [phi_i(q*), 0, 0] in the dual friction cone, P = dF/dq*(q*).
* "Contact Smoothing": D_i = D_max exp(-|c_i(q)|/kappa_h) (smooth) or D_max 1[|c_i| <= r_grasp]
  (nonsmooth), and the complementarity s^T lam = 0 relaxed to s^T lam = kappa_c.

Readings taken where the paper is silent (the same readings drive the CUDA path):

* E is a mass-spring energy sum_s k_s/2 (|x_b - x_a| - L_s)^2 (stretch + bend for a rope,
  structural + shear + bend for a cloth; the paper names stretching and bending only).
* M is lumped: node_mass per node.  The grippers are kinematic (the limit of an infinite gripper
  mass with actuation tau_g = m_g u/dt^2), so g+ = g* = g + u exactly and contact acts on nodes only.
* The relaxed complementarity is realised by the log barrier -kappa/2 log(s_n^2 - mu^2 |s_t|^2)
  of the dual cone {s_n >= mu |s_t|}.  Its stationarity gives lam = kappa (s_n, -mu^2 s_t)/(...),
  a point of the friction cone with s^T lam = kappa exactly.  The barrier depends on the tangent
  plane only through |s_t|^2 = |sigma|^2 - (n.sigma)^2 with sigma = Delta_j + phi n in world
  coordinates, so no tangent basis is needed.
* Stage 2 is solved by a primal-dual interior point with Nesterov-Todd scaling (Vandenberghe's
  cone QP method).  Its central path at kappa is exactly the smoothed model (s o z = kappa e,
  s^T lam = kappa); the nonsmooth SOCP is the end of the path, declared reached at kappa_hard.
  When every phi_i(q*) >= 0, Delta = 0 is the exact nonsmooth optimum and is returned as is.
* Newton directions use the exact Hessian when it is positive definite, else (rope) the Hessian
  with each spring's transverse factor (1 - L/l) clamped at 0 or (cloth) the exact Hessian plus
  a multiple of the identity; a backtracking Armijo search on the stage-1 potential Psi (whose
  gradient is F) globalises it.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import cholesky_banded, cho_solve_banded, LinAlgError

HARD, SMOOTH = "hard", "smooth"

# per-rollout status bits (sticky over a rollout)
ST_NEWTON = 1      # stage-1 Newton hit its iteration cap
ST_CONTACT = 2     # stage-2 interior point hit its iteration cap or found no interior
ST_NONFINITE = 4
ST_NOTPD = 8       # a stage-2 / adjoint system was not positive definite

# oracle tolerances: far tighter than any GPU tolerance, so the oracle's result is the exact
# root / optimum to FP64 accuracy
TOL_X = 1e-13
NEWTON_MAX = 100
NEWTON_MAX_CLOTH = 300  # a slack cloth's first steps from the flat state need up to ~200 iterations
IPM_MAX = 200
STALL_ALPHA = 1e-6     # stage-2 step length counted as a stall
STALL_MAX = 5          # consecutive stalls after which stage 2 reports no solution


class Scene:
    """Topology, parameters and obstacles of one rope or cloth."""

    def __init__(self, params: dict, rest_x: np.ndarray):
        p = params
        self.p = p
        self.kind = p["kind"]
        rest_x = np.asarray(rest_x, dtype=np.float64)
        self.nv = rest_x.shape[0]
        a, b, k = [], [], []
        if self.kind == "rope":
            n = self.nv
            for j in range(n - 1):
                a.append(j); b.append(j + 1); k.append(p["k_stretch"])
            for j in range(n - 2):
                a.append(j); b.append(j + 2); k.append(p["k_bend"])
        else:
            R, C = p["rows"], p["cols"]
            idx = lambda r, c: r * C + c
            for r in range(R):
                for c in range(C):
                    if c + 1 < C:
                        a.append(idx(r, c)); b.append(idx(r, c + 1)); k.append(p["k_stretch"])
                    if r + 1 < R:
                        a.append(idx(r, c)); b.append(idx(r + 1, c)); k.append(p["k_stretch"])
                    if r + 1 < R and c + 1 < C:
                        a.append(idx(r, c)); b.append(idx(r + 1, c + 1)); k.append(p["k_shear"])
                        a.append(idx(r, c + 1)); b.append(idx(r + 1, c)); k.append(p["k_shear"])
                    if c + 2 < C:
                        a.append(idx(r, c)); b.append(idx(r, c + 2)); k.append(p["k_bend"])
                    if r + 2 < R:
                        a.append(idx(r, c)); b.append(idx(r + 2, c)); k.append(p["k_bend"])
        self.a = np.array(a, dtype=np.int64)
        self.b = np.array(b, dtype=np.int64)
        assert np.all(self.b > self.a)
        self.k = np.array(k, dtype=np.float64)
        self.L = np.linalg.norm(rest_x[self.b] - rest_x[self.a], axis=1)
        self.m = float(p["node_mass"])
        self.dt = float(p["dt"])
        self.w = self.m / self.dt ** 2                     # M/dt^2 per node DoF
        self.grav = np.asarray(p["gravity"], dtype=np.float64)
        self.grasp = np.array(p["grasp_nodes"], dtype=np.int64)
        self.obstacles = list(p["obstacles"])
        self.n = 3 * self.nv
        self.nq = self.n + 6
        # half bandwidth (scalar) of every node-coupled matrix
        self.bw = 3 * int(np.max(self.b - self.a)) + 2 if len(self.a) else 2


# ------------------------------------------------------------------------------------------
# elastic energy (mass-spring), its gradient and Hessian
# ------------------------------------------------------------------------------------------

def spring_geometry(sc: Scene, X):
    d = X[sc.b] - X[sc.a]
    l = np.sqrt((d * d).sum(axis=1))
    return d, l


def elastic_energy(sc: Scene, X) -> float:
    _, l = spring_geometry(sc, X)
    return 0.5 * float(np.sum(sc.k * (l - sc.L) ** 2))


def elastic_gradient(sc: Scene, X) -> np.ndarray:
    d, l = spring_geometry(sc, X)
    f = (sc.k * (l - sc.L) / l)[:, None] * d        # dE/dx_b ; dE/dx_a = -f
    G = np.zeros_like(X)
    np.add.at(G, sc.b, f)
    np.add.at(G, sc.a, -f)
    return G


def spring_hessian_d(k, L, d, project=False):
    """d^2/dd^2 of k/2 (|d| - L)^2 = k [u u^T + (1 - L/l)(I - u u^T)], u = d/|d| (vectorised;
    works for complex d, which the derivative checks use)."""
    l = np.sqrt((d * d).sum(axis=-1))
    u = d / l[..., None]
    c = 1.0 - L / l
    if project:
        c = np.maximum(c, 0.0)
    I = np.eye(3)
    uu = u[..., :, None] * u[..., None, :]
    return k[..., None, None] * (uu + c[..., None, None] * (I - uu))


def spring_hessians(sc: Scene, X, project=False):
    d, _ = spring_geometry(sc, X)
    return spring_hessian_d(sc.k, sc.L, d, project)


# ------------------------------------------------------------------------------------------
# grasp stiffness (Sec. 4.1 "Contact Smoothing")
# ------------------------------------------------------------------------------------------

def grasp_offsets(sc: Scene, x, g):
    """c_i(q) = g_i - x_a(i) (the holonomic constraint of eq. holonomic-constraint)."""
    return g - x[sc.grasp]


def grasp_stiffness_of_c(sc: Scene, c, mode):
    """d_i = D_max exp(-|c_i|/kappa_h) (smooth) or D_max 1[|c_i| <= r_grasp] (nonsmooth).
    |c| is written sqrt(c.c) so the complex-step derivative checks pass through it."""
    rho = np.sqrt((c * c).sum(axis=-1))
    p = sc.p
    if mode == SMOOTH:
        return p["D_max"] * np.exp(-rho / p["kappa_h"])
    return np.where(np.real(rho) <= p["r_grasp"], p["D_max"], 0.0)


def grasp_stiffness(sc: Scene, x, g, mode):
    return grasp_stiffness_of_c(sc, grasp_offsets(sc, x, g), mode)


# ------------------------------------------------------------------------------------------
# stage 1: F, Psi differences, banded Hessian
# ------------------------------------------------------------------------------------------

def stage1_residual(sc: Scene, X, x, gstar, d):
    """F(q*; q, u) of eq. (dynamics-first-stage), node rows (the gripper rows are satisfied by
    g* = g + u exactly)."""
    F = sc.w * (X - x) + elastic_gradient(sc, X) - sc.m * sc.grav[None, :]
    for i in range(2):
        F[sc.grasp[i]] += d[i] * (X[sc.grasp[i]] - gstar[i])
    return F


def psi_difference(sc: Scene, X, D, x, gstar, d):
    """Psi(X + D) - Psi(X) for the stage-1 potential
         Psi(z) = 1/(2 dt^2) |z - x|_M^2 + E(z) - m grav . sum z_j + sum_i d_i/2 |g*_i - z_a(i)|^2,
    whose gradient is F.  Each term is written in terms of the step D itself (e.g. a spring
    length change is (D_b - D_a).(2 d_X + D_b - D_a)/(l_Y + l_X)), so that the difference stays
    accurate when the step is tiny."""
    val = 0.5 * sc.w * float(np.sum(D * (2.0 * (X - x) + D)))
    val -= sc.m * float(np.sum(D @ sc.grav))
    dX = X[sc.b] - X[sc.a]
    dD = D[sc.b] - D[sc.a]
    dY = dX + dD
    lX = np.sqrt((dX * dX).sum(1))
    lY = np.sqrt((dY * dY).sum(1))
    dl = (dD * (2.0 * dX + dD)).sum(1) / (lY + lX)
    val += 0.5 * float(np.sum(sc.k * dl * (lY + lX - 2.0 * sc.L)))
    for i in range(2):
        j = sc.grasp[i]
        val += 0.5 * d[i] * float(np.dot(D[j], D[j] - 2.0 * (gstar[i] - X[j])))
    return val


def band_zeros(sc: Scene):
    return np.zeros((sc.bw + 1, sc.n))


def band_add_node_blocks(sc: Scene, ab, nodes, blocks):
    """ab (lower band storage, ab[I-J, J] = A[I, J]) += block-diagonal 3x3 `blocks` at `nodes`."""
    for al in range(3):
        for be in range(al + 1):
            np.add.at(ab[al - be], 3 * nodes + be, blocks[:, al, be])


def band_add_springs(sc: Scene, ab, Hs):
    for al in range(3):
        for be in range(3):
            if al >= be:
                np.add.at(ab[al - be], 3 * sc.a + be, Hs[:, al, be])
                np.add.at(ab[al - be], 3 * sc.b + be, Hs[:, al, be])
            # off-diagonal block: rows of b, columns of a (b > a), value -Hs
            np.add.at(ab, (3 * (sc.b - sc.a) + al - be, 3 * sc.a + be), -Hs[:, al, be])


def stage1_hessian_band(sc: Scene, X, d, project=False):
    """dF/dq* = M/dt^2 + d^2E(q*) + sum_i d_i J_i^T J_i (node block), in lower band storage."""
    ab = band_zeros(sc)
    ab[0, :] += sc.w
    band_add_springs(sc, ab, spring_hessians(sc, X, project))
    gb = np.zeros((2, 3, 3))
    gb[:, [0, 1, 2], [0, 1, 2]] = np.asarray(d)[:, None]
    band_add_node_blocks(sc, ab, sc.grasp, gb)
    return ab


def stage1_hessian_vec(sc: Scene, X, d, v, project=False):
    """(dF/dq*) v without forming the matrix (the projected Hessian when `project`)."""
    Hs = spring_hessians(sc, X, project)
    dv = v[sc.b] - v[sc.a]
    f = np.einsum("sij,sj->si", Hs, dv)
    out = sc.w * v.copy()
    np.add.at(out, sc.b, f)
    np.add.at(out, sc.a, -f)
    for i in range(2):
        out[sc.grasp[i]] += d[i] * v[sc.grasp[i]]
    return out


def band_factor(ab):
    return cholesky_banded(ab, lower=True)


def band_solve(cb, rhs):
    """Solve with a banded Cholesky factor; rhs is node-shaped [nv, 3]."""
    return cho_solve_banded((cb, True), rhs.reshape(-1)).reshape(rhs.shape)


def band_solve_cols(cb, R):
    """Solve with a banded Cholesky factor for the columns of R [n, k]."""
    return cho_solve_banded((cb, True), R)


def shift_floor(sc: Scene):
    """Smallest nonzero diagonal shift of the cloth's stage-1 Newton: a quarter of the proximal
    stiffness m/dt^2 of one node."""
    return 0.25 * sc.w


def shifted_factor(sc: Scene, X, d, tau_prev):
    """Cholesky factor of dF/dq* + tau I with the smallest tau of the sequence 0 or tau_prev/2,
    then doubling (at least shift_floor) that is positive definite -- Cholesky with an added
    multiple of the identity (Nocedal & Wright, Numerical Optimization, 2nd ed., Alg. 3.3), its
    first trial taken from the previous iteration's shift.  Returns (factor, tau) or (None, tau)."""
    ab = stage1_hessian_band(sc, X, d)
    beta = shift_floor(sc)
    tau = 0.5 * tau_prev if 0.5 * tau_prev >= beta else 0.0
    for _ in range(64):
        a2 = ab.copy()
        a2[0] += tau
        try:
            return band_factor(a2), tau
        except LinAlgError:
            tau = max(2.0 * tau, beta)
    return None, tau


def stage1_solve(sc: Scene, x, gstar, d, tol=TOL_X, maxit=NEWTON_MAX, x_start=None):
    """Damped Newton for the root q* of F, started at q (Sec. 4.1, "solved using Newton's
    method") or at x_start when given.  Stops when the Newton step is below `tol` in every
    coordinate (the step is then taken).  Returns (q*, iterations, status).

    The direction: for a rope, the exact Hessian, or the projected one where the exact one is
    not positive definite.  For a cloth, the exact Hessian plus the shift of `shifted_factor` (a
    slack cloth has many wrinkle modes of nearly zero stiffness, along which the projected
    Hessian, which drops their negative curvature, gives only linear convergence).  Either way the
    iteration stops only on a step taken with the exact (unshifted, unprojected) Hessian, so the
    root is a local minimiser of Psi: a stable equilibrium, where the QP of stage 2 is convex and
    dF/dq* of the adjoint is positive definite."""
    X = x.copy() if x_start is None else np.array(x_start, dtype=np.float64)
    cloth = sc.kind == "cloth"
    tau = 0.0
    for it in range(maxit):
        F = stage1_residual(sc, X, x, gstar, d)
        if not np.all(np.isfinite(F)):
            return X, it, ST_NONFINITE
        if cloth:
            cb, tau = shifted_factor(sc, X, d, tau)
            if cb is None:
                return X, it + 1, ST_NONFINITE
        else:
            try:
                cb = band_factor(stage1_hessian_band(sc, X, d))
            except LinAlgError:
                cb = band_factor(stage1_hessian_band(sc, X, d, project=True))
                tau = -1.0          # marks a projected (not exact) direction
        p = -band_solve(cb, F)
        if np.max(np.abs(p)) <= tol and tau == 0.0:
            return X + p, it + 1, 0
        if not cloth:
            tau = 0.0
        slope = float(np.sum(F * p))
        alpha = 1.0
        for _ in range(60):
            if psi_difference(sc, X, alpha * p, x, gstar, d) <= 1e-4 * alpha * slope:
                break
            alpha *= 0.5
        X = X + alpha * p
    return X, maxit, ST_NEWTON


# ------------------------------------------------------------------------------------------
# contact geometry: signed distances and normals (Sec. 4.1, eq. contact-constraint)
# ------------------------------------------------------------------------------------------

def _sqrt_dot(v):
    return np.sqrt((v * v).sum(axis=-1))


def obstacle_phi_normal(ob: dict, X, radius):
    """phi = sdf(x) - node radius and n = grad sdf for one obstacle, vectorised over points.
    Branch decisions use real parts only, so the functions also accept complex X."""
    if ob["type"] == "plane":
        nrm = np.asarray(ob["normal"], dtype=np.float64)
        phi = X @ nrm - ob["offset"] - radius
        n = np.broadcast_to(nrm, X.shape) + 0.0 * X
        return phi, n
    if ob["type"] == "sphere":
        r = X - np.asarray(ob["center"])
        dist = _sqrt_dot(r)
        return dist - ob["radius"] - radius, r / dist[..., None]
    if ob["type"] == "box":
        rel = X - np.asarray(ob["center"])
        s = np.where(np.real(rel) >= 0, 1.0, -1.0)
        q = rel * s - np.asarray(ob["half"])           # per-axis distance outside the faces
        out_mask = np.real(q) > 0
        qpos = np.where(out_mask, q, 0.0)
        any_out = out_mask.any(axis=-1)
        dist_out = _sqrt_dot(qpos)
        safe = np.where(any_out, dist_out, 1.0)
        n_out = s * qpos / safe[..., None]
        kmax = np.argmax(np.real(q), axis=-1)
        q_in = np.take_along_axis(q, kmax[..., None], axis=-1)[..., 0]
        n_in = np.zeros_like(q)
        np.put_along_axis(n_in, kmax[..., None], 1.0, axis=-1)
        n_in = n_in * s
        phi = np.where(any_out, dist_out, q_in) - radius
        n = np.where(any_out[..., None], n_out, n_in)
        return phi, n
    raise ValueError(ob["type"])


def contact_geometry(sc: Scene, X):
    """phi[j, o], n[j, o, :] for every node j and obstacle o (all pairs enter stage 2)."""
    r = sc.p["node_radius"]
    if not sc.obstacles:
        return np.zeros((X.shape[0], 0)), np.zeros((X.shape[0], 0, 3))
    phis, ns = [], []
    for ob in sc.obstacles:
        ph, nn = obstacle_phi_normal(ob, X, r)
        phis.append(ph); ns.append(nn)
    return np.stack(phis, axis=1), np.stack(ns, axis=1)


# ------------------------------------------------------------------------------------------
# stage 2: the contact problem and its log-barrier (relaxed complementarity)
# ------------------------------------------------------------------------------------------

def cone_gap(sig, n, mu):
    """g = (1+mu^2)(n.sigma)^2 - mu^2|sigma|^2 = s_n^2 - mu^2 |s_t|^2 and s_n = n.sigma."""
    sn = (n * sig).sum(-1)
    g = (1.0 + mu * mu) * sn * sn - mu * mu * (sig * sig).sum(-1)
    return sn, g


def contact_force(sig, n, kappa, mu):
    """lam = -grad_sigma b(sigma), b = -kappa/2 log g: the contact force of a pair."""
    sn, g = cone_gap(sig, n, mu)
    a = (1.0 + mu * mu) * sn[..., None] * n - mu * mu * sig
    return kappa * a / g[..., None]


def contact_force_jacobian(sig, n, kappa, mu):
    """W = d^2 b / d sigma^2 = -d lam / d sigma (3x3 per pair)."""
    sn, g = cone_gap(sig, n, mu)
    a = (1.0 + mu * mu) * sn[..., None] * n - mu * mu * sig
    I = np.eye(3)
    nn = n[..., :, None] * n[..., None, :]
    aa = a[..., :, None] * a[..., None, :]
    return (kappa / g)[..., None, None] * (mu * mu * I - (1.0 + mu * mu) * nn) \
        + (2.0 * kappa / g ** 2)[..., None, None] * aa


def in_cone_interior(sig, n, mu):
    sn, g = cone_gap(sig, n, mu)
    return bool(np.all(sn > 0) and np.all(g > 0))


def tangent_frame(n):
    """Unit tangents t1, t2 completing the unit normal n to an orthonormal basis, by the
    branchless construction of Duff et al., "Building an Orthonormal Basis, Revisited" (JCGT
    2017).  The solution of stage 2 does not depend on the choice of tangent basis."""
    sgn = np.where(n[..., 2] >= 0.0, 1.0, -1.0)
    a = -1.0 / (sgn + n[..., 2])
    b = n[..., 0] * n[..., 1] * a
    t1 = np.stack([1.0 + sgn * n[..., 0] ** 2 * a, sgn * b, -sgn * n[..., 0]], axis=-1)
    t2 = np.stack([b, sgn + n[..., 1] ** 2 * a, -n[..., 1]], axis=-1)
    return t1, t2


def cone_frames(n, mu):
    """A = [n; mu t1; mu t2]: maps a world vector sigma to the scaled cone coordinates
    s = (s_n, mu s_t), for which the dual friction cone {s_n >= mu |s_t|} is the standard
    second-order cone Q = {s_0 >= |s_{1:2}|}.  The contact force is lam = A^T z, z in Q."""
    t1, t2 = tangent_frame(n)
    return np.stack([n, mu * t1, mu * t2], axis=-2)


J3 = np.diag([1.0, -1.0, -1.0])


def soc_det(x):
    return x[..., 0] ** 2 - (x[..., 1:] ** 2).sum(-1)


def soc_interior(x):
    return bool(np.all(x[..., 0] > 0.0) and np.all(soc_det(x) > 0.0))


def jordan(x, y):
    """Jordan product of the second-order cone: x o y = (x.y, x_0 y_1 + y_0 x_1)."""
    return np.concatenate([(x * y).sum(-1, keepdims=True),
                           x[..., :1] * y[..., 1:] + y[..., :1] * x[..., 1:]], axis=-1)


def jordan_solve(x, r):
    """v with x o v = r (x in the interior of Q)."""
    v0 = (x[..., 0] * r[..., 0] - (x[..., 1:] * r[..., 1:]).sum(-1)) / soc_det(x)
    v1 = (r[..., 1:] - x[..., 1:] * v0[..., None]) / x[..., :1]
    return np.concatenate([v0[..., None], v1], axis=-1)


def jordan_inverse(x):
    return np.concatenate([x[..., :1], -x[..., 1:]], axis=-1) / soc_det(x)[..., None]


def nt_scaling(s, z):
    """Nesterov-Todd scaling of a pair s, z in int Q (Vandenberghe, "The CVXOPT linear and
    quadratic cone program solvers", 2010, second-order cone case): the symmetric W with
    W z = W^{-1} s.  Returns W, W^{-1} and the scaled point lam = W z."""
    ds, dz = soc_det(s), soc_det(z)
    sb = s / np.sqrt(ds)[..., None]
    zb = z / np.sqrt(dz)[..., None]
    gam = np.sqrt(0.5 * (1.0 + (sb * zb).sum(-1)))
    wb = (sb + zb @ J3) / (2.0 * gam)[..., None]
    e = np.zeros_like(wb); e[..., 0] = 1.0
    v = (wb + e) / np.sqrt(2.0 * (wb[..., 0] + 1.0))[..., None]
    beta = (ds / dz) ** 0.25
    vv = v[..., :, None] * v[..., None, :]
    W = beta[..., None, None] * (2.0 * vv - J3)
    Jv = v @ J3
    Winv = (1.0 / beta)[..., None, None] * (2.0 * Jv[..., :, None] * Jv[..., None, :] - J3)
    lam = np.einsum("...ab,...b->...a", W, z)
    return W, Winv, lam


def max_step(x, dx):
    """Largest alpha with x + alpha dx in Q (np.inf if unbounded), per cone."""
    a = dx[..., 0] ** 2 - (dx[..., 1:] ** 2).sum(-1)
    b = 2.0 * (x[..., 0] * dx[..., 0] - (x[..., 1:] * dx[..., 1:]).sum(-1))
    c = soc_det(x)
    out = np.full(a.shape, np.inf)
    disc = b * b - 4.0 * a * c
    with np.errstate(divide="ignore", invalid="ignore"):
        sq = np.sqrt(np.maximum(disc, 0.0))
        r1 = np.where(a != 0.0, (-b - sq) / (2.0 * a), np.where(b < 0.0, -c / b, np.inf))
        r2 = np.where(a != 0.0, (-b + sq) / (2.0 * a), np.inf)
    for r in (r1, r2):
        ok = (disc >= 0.0) & (r > 0.0)
        out = np.where(ok, np.minimum(out, r), out)
    with np.errstate(divide="ignore", invalid="ignore"):
        t0 = np.where(dx[..., 0] < 0.0, -x[..., 0] / dx[..., 0], np.inf)
    return np.minimum(out, t0)


def stage2_ipm(sc: Scene, xs, d, phi, n, kappa, kappa_final, tol=TOL_X, maxit=IPM_MAX,
               Delta_start=None, extra=None):
    """Primal-dual interior point with Nesterov-Todd scaling (the cone QP method of Vandenberghe
    2010) for
        min 1/2 Delta^T P Delta  s.t.  s_i = A_i Delta_j + phi_i e1 in Q,
    with multipliers z_i in Q (contact forces lam_i = A_i^T z_i) and the centering condition
    s_i o z_i = kappa e, i.e. the relaxed complementarity s^T lam = kappa of the smoothed model.
    The target is kappa throughout when kappa_final is None (smooth model).  Otherwise each
    iteration is a Mehrotra predictor-corrector step, as in the cited method: the affine
    direction (target 0) with its largest feasible step alpha_a gives the centring
    sigma = (1 - alpha_a)^3 and the target max(kappa_final, sigma <s, z>/m), and the combined
    direction adds the second-order term (W^{-1} ds_a) o (W dz_a) to the complementarity
    right-hand side.  Once the target has reached kappa_final, plain Newton steps towards that
    central point follow (no predictor, no correction), and the solve ends there.  Each direction solves
    H2 dDelta = rhs with the banded SPD matrix H2 = P + sum_i E_j A_i^T W_i^{-2} A_i E_j^T (one
    factorisation per iteration); steps keep s, z strictly inside Q (fraction to the boundary
    0.99).  `extra` (the second-order variant's damping, oracle/second_order.py) adds a constant
    symmetric term to P: its band `extra.band`, its node diagonal blocks `extra.diag` and its
    product `extra.vec(V)`.  Returns (Delta, sigma_world, iterations, status)."""
    mu = sc.p["mu"]
    nv, no = phi.shape
    Delta = np.zeros((nv, 3))
    if no == 0:
        return Delta, np.zeros((nv, 0, 3)), 0, 0
    A = cone_frames(n, mu)
    P_ab = stage1_hessian_band(sc, xs, d)
    if extra is not None:
        P_ab = P_ab + extra.band
    e1 = np.zeros((nv, no, 3)); e1[..., 0] = 1.0
    # interior start: the per-node closed form along each penetrating normal, then s from it
    # where it lies well inside Q, else (max(phi, sigma0), 0, 0); z central for that s
    Pdiag = stage1_hessian_vec_diag(sc, xs, d)
    if extra is not None:
        Pdiag = Pdiag + extra.diag
    Pd = np.einsum("joa,jab,job->jo", n, Pdiag, n)
    push = 0.5 * (-phi + np.sqrt(phi * phi + 4.0 * kappa / Pd))
    Delta = np.einsum("jo,joa->ja", np.where(phi < 0.0, push, 0.0), n)
    if Delta_start is not None:         # warm start (the central point reached does not depend on it)
        Delta = np.asarray(Delta_start, dtype=np.float64).reshape(nv, 3).copy()
    s = np.einsum("joab,jb->joa", A, Delta) + phi[..., None] * e1
    ok = (s[..., 0] > 0.0) & (soc_det(s) > 0.25 * s[..., 0] ** 2)
    s = np.where(ok[..., None], s, np.maximum(phi, sc.p["sigma0"])[..., None] * e1)
    z = kappa * jordan_inverse(s)
    m = nv * no
    stalls = 0
    centring = False        # the target has reached kappa_final
    for it in range(maxit):
        lam_w = np.einsum("joab,joa->job", A, z)
        r_d = stage1_hessian_vec(sc, xs, d, Delta) - lam_w.sum(axis=1)
        if extra is not None:
            r_d = r_d + extra.vec(Delta)
        r_z = s - np.einsum("joab,jb->joa", A, Delta) - phi[..., None] * e1
        W, Winv, lam = nt_scaling(s, z)
        M = Winv @ Winv
        AMA = np.einsum("joba,jobc,jocd->joad", A, M, A)     # A^T M A
        ab = P_ab.copy()
        band_add_node_blocks(sc, ab, np.arange(nv), AMA.sum(axis=1))
        try:
            cb = band_factor(ab)
        except LinAlgError:
            # H2 = P + sum A^T M A is not positive definite, so neither is P: the stage-1 root is
            # not a minimiser of its potential and the QP of eq. (dynamics-second-stage) is not
            # convex; the step has no defined contact solution
            return Delta, None, it, ST_NOTPD

        def direction(d_s):
            # W^{-1} ds + W dz = d_s, ds = A dDelta - r_z, P dDelta - sum A^T dz = -r_d
            g = r_z + np.einsum("joab,job->joa", W, d_s)
            rhs = -r_d + np.einsum("joba,job->ja", A, np.einsum("joab,job->joa", M, g))
            dD = band_solve(cb, rhs)
            ADd = np.einsum("joab,jb->joa", A, dD)
            return dD, ADd - r_z, np.einsum("joab,job->joa", M, g - ADd)

        if kappa_final is None or centring:
            target = kappa if kappa_final is None else kappa_final
            corr = 0.0
        else:
            _, dsa, dza = direction(-lam)                   # affine direction: target 0
            alpha_a = min(1.0, float(min(max_step(s, dsa).min(), max_step(z, dza).min())))
            target = max(kappa_final, (1.0 - alpha_a) ** 3 * float((s * z).sum()) / m)
            corr = jordan(np.einsum("joab,job->joa", Winv, dsa), np.einsum("joab,job->joa", W, dza))
            centring = target == kappa_final
            if centring:
                corr = 0.0
        d_s = jordan_solve(lam, target * e1 - jordan(lam, lam) - corr)
        dD, dsv, dz = direction(d_s)
        if not (np.all(np.isfinite(dD)) and np.all(np.isfinite(dz))):
            return Delta, None, it, ST_NONFINITE
        alpha = min(1.0, 0.99 * float(min(max_step(s, dsv).min(), max_step(z, dz).min())))
        # a linearised cone set can be empty (a node driven between two obstacles whose friction
        # cones do not meet); steps then collapse: give up after STALL_MAX tiny steps
        stalls = stalls + 1 if alpha < STALL_ALPHA else 0
        if stalls >= STALL_MAX:
            return Delta, Delta[:, None, :] + phi[..., None] * n, it + 1, ST_CONTACT
        Delta = Delta + alpha * dD
        s = s + alpha * dsv
        z = z + alpha * dz
        if not (soc_interior(s) and soc_interior(z)):
            return Delta, Delta[:, None, :] + phi[..., None] * n, it + 1, ST_CONTACT
        if target == (kappa if kappa_final is None else kappa_final) and alpha == 1.0 \
                and np.max(np.abs(dD)) <= tol and np.max(np.abs(dsv)) <= tol:
            return Delta, Delta[:, None, :] + phi[..., None] * n, it + 1, 0
    return Delta, Delta[:, None, :] + phi[..., None] * n, maxit, ST_CONTACT


def stage1_hessian_vec_diag(sc: Scene, X, d):
    """The 3x3 diagonal blocks P_jj of dF/dq*."""
    Hs = spring_hessians(sc, X)
    D = np.zeros((sc.nv, 3, 3))
    D[:, [0, 1, 2], [0, 1, 2]] = sc.w
    np.add.at(D, sc.a, Hs)
    np.add.at(D, sc.b, Hs)
    for i in range(2):
        D[sc.grasp[i]] += d[i] * np.eye(3)
    return D


def stage2_smooth(sc: Scene, xs, d, tol=TOL_X, Delta_start=None):
    """Smoothed stage 2: the central point at kappa_c (relaxed complementarity s^T lam = kappa_c)."""
    phi, n = contact_geometry(sc, xs)
    Delta, sig, it, st = stage2_ipm(sc, xs, d, phi, n, sc.p["kappa_c"], None, tol, Delta_start=Delta_start)
    return Delta, sig, phi, n, it, st


def stage2_hard(sc: Scene, xs, d, tol=TOL_X, Delta_start=None):
    """The nonsmooth contact SOCP of eq. (dynamics-second-stage).  Delta = 0 when no pair
    penetrates; otherwise the primal-dual path is followed from kappa_c down to kappa_hard."""
    phi, n = contact_geometry(sc, xs)
    if np.all(phi >= 0.0):
        return np.zeros((sc.nv, 3)), None, phi, n, 0, 0
    Delta, sig, it, st = stage2_ipm(sc, xs, d, phi, n, sc.p["kappa_c"], sc.p["kappa_hard"], tol,
                                    Delta_start=Delta_start)
    return Delta, sig, phi, n, it, st


# ------------------------------------------------------------------------------------------
# one step and a rollout
# ------------------------------------------------------------------------------------------

def split_q(sc: Scene, q):
    q = np.asarray(q, dtype=np.float64)
    return q[: sc.n].reshape(sc.nv, 3), q[sc.n:].reshape(2, 3)


def join_q(x, g):
    return np.concatenate([x.ravel(), g.ravel()])


def step(sc: Scene, q, u, mode, tol=TOL_X, info=None, x_start=None, Delta_start=None):
    """(q, u) -> q+ : stage 1 then stage 2 (Sec. 4.1, "Simulation Solver").  x_start: optional
    start of the stage-1 Newton iteration (default: q with the grasped nodes moved with their
    grippers)."""
    x, g = split_q(sc, q)
    gstar = g + np.asarray(u, dtype=np.float64).reshape(2, 3)
    if x_start is None:
        # stage 1 starts at q with each grasped node moved with its gripper
        x_start = x.copy()
        for i in range(2):
            x_start[sc.grasp[i]] += gstar[i] - g[i]
    d = grasp_stiffness(sc, x, g, mode)
    cap = NEWTON_MAX_CLOTH if sc.kind == "cloth" else NEWTON_MAX
    xs, it1, st1 = stage1_solve(sc, x, gstar, d, tol, maxit=cap, x_start=x_start)
    if mode == HARD:
        Delta, sig, phi, n, it2, st2 = stage2_hard(sc, xs, d, tol, Delta_start)
    else:
        Delta, sig, phi, n, it2, st2 = stage2_smooth(sc, xs, d, tol, Delta_start)
    if info is not None:
        info.update(xs=xs, Delta=Delta, sig=sig, phi=phi, n=n, d=d, gstar=gstar,
                    newton_it=it1, ipm_it=it2, status=st1 | st2)
    return join_q(xs + Delta, gstar), st1 | st2


def rollout(sc: Scene, q0, U, mode, tol=TOL_X, xs_out=None):
    """q_0 .. q_H for controls U[H, 6].  Returns (traj[H+1, nq], status, newton/ipm counts);
    xs_out, if a list, receives each step's stage-1 solution q*.  Stage 2 of a step starts its
    interior point at the previous step's Delta when that step ran stage 2 (the point it
    converges to does not depend on the start)."""
    H = U.shape[0]
    traj = np.zeros((H + 1, sc.nq))
    traj[0] = q0
    status = 0
    counts = []
    D_prev = None
    for t in range(H):
        info = {}
        traj[t + 1], st = step(sc, traj[t], U[t], mode, tol, info, Delta_start=D_prev)
        D_prev = info["Delta"] if np.any(info["Delta"] != 0.0) else None
        status |= st
        counts.append((info["newton_it"], info["ipm_it"]))
        if xs_out is not None:
            xs_out.append(info["xs"])
    return traj, status, counts
