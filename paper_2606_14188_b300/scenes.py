"""Seeded synthetic scenes and control sequences.

This module draws random numbers and lays out initial geometry; it holds none of the
simulator's arithmetic (no springs, no energies, no contact model).  Both the CUDA path and
the FP64 CPU oracle are fed from the arrays it returns, so the two sides see bit-identical
inputs.

The scenes stand in for the paper's rope and cloth tasks (Lift/Drag Rope, Fold/Flatten Cloth,
Sec. 5 and Table 1): the paper's hardware data are not public, so each scene is a seeded
synthetic layout with the sizes and structure the workloads call for (a 0.8 m rope, App. B.1;
a 0.38 m square cloth, App. B.2; grasped ends/corners; a table plane and sphere/box obstacles).

Parameter values are not printed in the paper; the defaults below are the readings used by
both implementations (gravity 9.81 m/s^2 along -z, rope mass 0.1 kg, cloth mass 0.05 kg,
k_stretch 500 N/m, k_shear 250 N/m, k_bend 25 N/m, D_max 1e4 N/m, kappa_h 0.01 m,
kappa_c 1e-4 N m, mu 0.5, dt 0.01 s).
"""
from __future__ import annotations

import copy
import numpy as np

BASE_SEED = 260614188

HARD, SMOOTH = "hard", "smooth"
SURROGATE, CONSISTENT = "surrogate", "consistent"


def default_params(kind: str = "rope") -> dict:
    """Physical and solver parameters shared by the oracle and the CUDA path."""
    p = dict(
        kind=kind,
        n_nodes=0, rows=0, cols=0,
        grasp_nodes=(0, 0),
        dt=0.01,
        gravity=(0.0, 0.0, -9.81),
        node_mass=0.0,
        k_stretch=500.0, k_shear=250.0, k_bend=25.0,
        D_max=1.0e4,
        kappa_h=0.01,          # grasp smoothing length [m]
        kappa_c=1.0e-4,        # contact smoothing (relaxed complementarity) [N m]
        kappa_hard=1.0e-6,     # central-path weight at which the nonsmooth SOCP is declared solved
        kappa_decay=0.1,       # path-following decrease of the barrier weight per stage
        mu=0.5,
        r_grasp=0.01,
        node_radius=0.005,
        sigma0=1.0e-3,         # interior start of a penetrating contact slack [m]
        obstacles=[],
        fwd_mode=HARD,
        grad_mode=SURROGATE,
        newton_max=30, newton_tol=2.0e-7,
        ipm_max=60, ipm_tol=2.0e-7,
        checkpoint_every=1,
        loss=dict(goal_nodes=(), goal_pos=np.zeros((0, 3)), w_goal=1.0,
                  w_pen=100.0, pen_margin=0.02, w_u=0.01),
    )
    return p


def plane(normal=(0.0, 0.0, 1.0), offset=0.0) -> dict:
    n = np.asarray(normal, dtype=np.float64)
    return dict(type="plane", normal=tuple(n / np.linalg.norm(n)), offset=float(offset))


def sphere(center, radius) -> dict:
    return dict(type="sphere", center=tuple(float(c) for c in center), radius=float(radius))


def box(center, half) -> dict:
    return dict(type="box", center=tuple(float(c) for c in center),
                half=tuple(float(h) for h in half))


def _point_clear(points: np.ndarray, ob: dict, clearance: float) -> bool:
    """Scene-generation rejection test: is every point at least `clearance` from the shape."""
    if ob["type"] == "sphere":
        c = np.asarray(ob["center"])
        return bool(np.all(np.linalg.norm(points - c, axis=1) - ob["radius"] >= clearance))
    if ob["type"] == "box":
        c = np.asarray(ob["center"]); h = np.asarray(ob["half"])
        outside = np.maximum(np.abs(points - c) - h, 0.0)
        return bool(np.all(np.linalg.norm(outside, axis=1) >= clearance))
    return True


def rope_scene(n_nodes: int, n_spheres: int = 1, n_boxes: int = 0, seed: int = BASE_SEED,
               length: float = 0.8, height: float = 0.3, total_mass: float = 0.1,
               sphere_box=((0.2, 0.6), (-0.1, 0.1), (0.05, 0.25)),
               box_box=((0.0, 1.0), (-0.2, 0.2), (0.0, 0.3)),
               sphere_r=(0.05, 0.15), box_half=(0.03, 0.1)) -> dict:
    """A straight rope along +x at height `height`, both ends grasped, ground plane z = 0.

    Obstacles are drawn uniformly in the given boxes and redrawn while they touch the initial
    rope (clearance of one node radius plus 1 cm).
    """
    rng = np.random.default_rng(seed)
    p = default_params("rope")
    p["n_nodes"] = n_nodes
    p["node_mass"] = total_mass / n_nodes
    p["grasp_nodes"] = (0, n_nodes - 1)
    p["node_radius"] = 0.005
    xs = np.linspace(0.1, 0.1 + length, n_nodes)
    rest = np.stack([xs, np.zeros(n_nodes), np.full(n_nodes, height)], axis=1)
    obs = [plane((0, 0, 1), 0.0)]
    clear = p["node_radius"] + 0.01
    for _ in range(n_spheres):
        for _try in range(100000):
            c = [rng.uniform(*sphere_box[k]) for k in range(3)]
            r = rng.uniform(*sphere_r)
            ob = sphere(c, r)
            if _point_clear(rest, ob, clear):
                break
        else:
            raise ValueError("no obstacle placement clear of the rest shape")
        obs.append(ob)
    for _ in range(n_boxes):
        for _try in range(100000):
            c = [rng.uniform(*box_box[k]) for k in range(3)]
            h = [rng.uniform(*box_half) for _ in range(3)]
            ob = box(c, h)
            if _point_clear(rest, ob, clear):
                break
        else:
            raise ValueError("no obstacle placement clear of the rest shape")
        obs.append(ob)
    p["obstacles"] = obs
    goal_nodes = (0, n_nodes - 1)
    p["loss"] = dict(goal_nodes=goal_nodes,
                     goal_pos=rest[list(goal_nodes)] + np.array([0.0, 0.0, 0.1]),
                     w_goal=1.0, w_pen=100.0, pen_margin=0.02, w_u=0.01)
    q0 = np.concatenate([rest.ravel(), rest[0], rest[-1]])
    return dict(params=p, rest_x=rest, q0=q0)


def cloth_scene(rows: int, cols: int, n_spheres: int = 2, seed: int = BASE_SEED,
                side: float = 0.38, height: float = 0.05, total_mass: float = 0.05) -> dict:
    """A flat square cloth at height `height` over the table z = 0; corners (0,0) and
    (0,cols-1) grasped; spheres drawn below/beside the cloth and redrawn while they touch it.
    The loss folds row 0 onto row rows-1."""
    rng = np.random.default_rng(seed)
    p = default_params("cloth")
    p["rows"], p["cols"] = rows, cols
    n = rows * cols
    p["n_nodes"] = n
    p["node_mass"] = total_mass / n
    p["grasp_nodes"] = (0, cols - 1)
    p["node_radius"] = 0.002
    p["k_stretch"], p["k_shear"], p["k_bend"] = 500.0, 250.0, 25.0
    r_idx, c_idx = np.meshgrid(np.arange(rows), np.arange(cols), indexing="ij")
    rest = np.stack([r_idx.ravel() * side / max(rows - 1, 1), c_idx.ravel() * side / max(cols - 1, 1),
                     np.full(n, height)], axis=1)
    obs = [plane((0, 0, 1), 0.0)]
    clear = p["node_radius"] + 0.01
    for _ in range(n_spheres):
        for _try in range(100000):
            c = [rng.uniform(-0.1, side + 0.1), rng.uniform(-0.1, side + 0.1),
                 rng.uniform(-0.1, 0.0)]
            r = rng.uniform(0.05, 0.15)
            ob = sphere(c, r)
            if _point_clear(rest, ob, clear):
                break
        else:
            raise ValueError("no obstacle placement clear of the rest shape")
        obs.append(ob)
    p["obstacles"] = obs
    goal_nodes = tuple(range(cols))
    goal_pos = rest[(rows - 1) * cols + np.arange(cols)].copy()
    p["loss"] = dict(goal_nodes=goal_nodes, goal_pos=goal_pos, w_goal=1.0, w_pen=100.0,
                     pen_margin=0.02, w_u=0.01)
    q0 = np.concatenate([rest.ravel(), rest[0], rest[cols - 1]])
    return dict(params=p, rest_x=rest, q0=q0)


def controls_uniform(B: int, H: int, n_u: int = 6, lo: float = -0.05, hi: float = 0.05,
                     seed: int = BASE_SEED) -> np.ndarray:
    rng = np.random.default_rng(seed + 7919)
    return rng.uniform(lo, hi, size=(B, H, n_u))


def controls_normal(B: int, H: int, n_u: int = 6, sigma: float = 0.02,
                    seed: int = BASE_SEED) -> np.ndarray:
    rng = np.random.default_rng(seed + 7919)
    return rng.normal(0.0, sigma, size=(B, H, n_u))


def _gripper_clear(p: np.ndarray, obstacles, clearance: float) -> np.ndarray:
    """Scene-generation test: gripper positions p [..., 3] at least `clearance` from every
    sphere and box and above every plane (no simulator arithmetic)."""
    ok = np.ones(p.shape[:-1], dtype=bool)
    for ob in obstacles:
        if ob["type"] == "plane":
            ok &= p @ np.asarray(ob["normal"]) - ob["offset"] >= clearance
        elif ob["type"] == "sphere":
            ok &= np.linalg.norm(p - np.asarray(ob["center"]), axis=-1) - ob["radius"] >= clearance
        else:
            out = np.maximum(np.abs(p - np.asarray(ob["center"])) - np.asarray(ob["half"]), 0.0)
            ok &= np.linalg.norm(out, axis=-1) >= clearance
    return ok


def controls_normal_clear(scene: dict, B: int, H: int, sigma: float = 0.02,
                          clearance: float = 0.02, seed: int = BASE_SEED) -> np.ndarray:
    """Gripper displacements ~ N(0, sigma^2) per coordinate, redrawn (up to 20 times, else 0)
    whenever a gripper would come within `clearance` of an obstacle or the table: a planner's
    candidates move the grippers in free space, as the robots of the paper's tasks do."""
    rng = np.random.default_rng(seed + 7919)
    g = np.repeat(scene["q0"][None, -6:].reshape(1, 2, 3), B, axis=0)
    obs = scene["params"]["obstacles"]
    U = np.zeros((B, H, 2, 3))
    for t in range(H):
        u = rng.normal(0.0, sigma, size=(B, 2, 3))
        bad = ~_gripper_clear(g + u, obs, clearance)
        for _ in range(20):
            if not bad.any():
                break
            u[bad] = rng.normal(0.0, sigma, size=(int(bad.sum()), 3))
            bad = ~_gripper_clear(g + u, obs, clearance)
        u[bad] = 0.0
        U[:, t] = u
        g = g + u
    return U.reshape(B, H, 6)


def batch_q0(scene: dict, B: int) -> np.ndarray:
    return np.repeat(scene["q0"][None, :], B, axis=0)


# ------------------------------------------------------------------------------------------
# The five workloads.  Each returns a dict with the scene, batch size, horizon, controls and
# precision.  `small=True` shrinks the batch so the oracle can finish in seconds.
# ------------------------------------------------------------------------------------------

def workload(i: int, B: int | None = None, H: int | None = None, shard: int = 0) -> dict:
    """Workload i (1..4).  shard > 0 draws other controls for the same scene (the share of one
    rank of a multi-GPU run)."""
    seed = BASE_SEED + i
    if i == 1:    # one 20-node rope, FP64, horizon 10, one sphere, uniform controls
        sc = rope_scene(20, n_spheres=1, n_boxes=0, seed=seed)
        B = B or 1; H = H or 10
        U = controls_uniform(B, H, seed=seed + 1000003 * shard)
        real = 8
        ck = 1
    elif i == 2:  # 1024 rollouts x 64-node rope, FP32, horizon 50, 2 spheres + 2 boxes
        sc = rope_scene(64, n_spheres=2, n_boxes=2, seed=seed,
                        sphere_box=((0.0, 1.0), (-0.2, 0.2), (0.0, 0.3)))
        B = B or 1024; H = H or 50
        U = controls_normal_clear(sc, B, H, seed=seed + 1000003 * shard)
        real = 4
        ck = 7
    elif i == 3:  # 512 rollouts of a 32x32 cloth, FP32, horizon 30, table + 2 spheres
        sc = cloth_scene(32, 32, n_spheres=2, seed=seed)
        B = B or 512; H = H or 30
        U = controls_normal_clear(sc, B, H, seed=seed + 1000003 * shard)
        real = 4
        ck = 5
    elif i == 4:  # 256 nominal trajectories of a 40-node rope, horizon 20 (linearisation)
        sc = rope_scene(40, n_spheres=1, n_boxes=0, seed=seed)
        B = B or 256; H = H or 20
        U = controls_normal_clear(sc, B, H, seed=seed + 1000003 * shard)
        real = 4
        ck = 1
    else:
        raise ValueError(f"unknown workload {i}")
    sc = copy.deepcopy(sc)
    sc["params"]["checkpoint_every"] = ck
    if real == 4:
        # the nonsmooth contact problem is declared solved at the central point of kappa_hard,
        # whose contact slacks are O(kappa_hard / lam_n): at 1e-6 N m and the 1-2 N sliding
        # contacts of these scenes they are below what single precision resolves at the state's
        # metre scale, at 1e-5 (10 um of slack at 1 N, under the FP32 state tolerance) they are not
        sc["params"]["kappa_hard"] = 1.0e-5
    return dict(scene=sc, B=B, H=H, U=U, q0=batch_q0(sc, B), real_bytes=real, seed=seed)


# ------------------------------------------------------------------------------------------
# output-feedback SLS stage inputs (Sec. 4.2)
# ------------------------------------------------------------------------------------------

def sls_observation_model(B: int, H: int, nv: int, seed: int = BASE_SEED + 500,
                          sigma_w: float = 0.005, sigma_e: float = 0.01, sigma_0: float = 0.02,
                          jitter: float = 0.05) -> dict:
    """Seeded observation model and disturbance scalings about B nominal rope trajectories of H
    steps (state q = [x, g], n = 3 nv + 6), the inputs of the observer stage besides A_t:
      C  [B][H][3 nv][n]  the node positions (what the vision front end measures), each entry
                          perturbed by N(0, jitter^2) (a perception model linearised along the
                          trajectory differs from step to step);
      E  [B][H][n][n]     diagonal process-disturbance scaling: sigma_w per node coordinate,
                          sigma_w / 10 on the gripper coordinates, each times U[0.5, 1.5];
      F  [B][H][3 nv][3 nv]  diagonal observation-noise scaling sigma_e U[0.5, 1.5];
      Xi [B][n][n]        diagonal initial uncertainty sigma_0 U[0.5, 1.5]."""
    rng = np.random.default_rng(seed)
    n, p = 3 * nv + 6, 3 * nv
    C = np.zeros((B, H, p, n))
    C[:, :, np.arange(p), np.arange(p)] = 1.0
    C += jitter * rng.normal(size=C.shape)
    ew = np.full(n, sigma_w)
    ew[3 * nv:] = sigma_w / 10
    E = np.zeros((B, H, n, n))
    E[:, :, np.arange(n), np.arange(n)] = ew * rng.uniform(0.5, 1.5, size=(B, H, n))
    F = np.zeros((B, H, p, p))
    F[:, :, np.arange(p), np.arange(p)] = sigma_e * rng.uniform(0.5, 1.5, size=(B, H, p))
    Xi = np.zeros((B, n, n))
    Xi[:, np.arange(n), np.arange(n)] = sigma_0 * rng.uniform(0.5, 1.5, size=(B, n))
    return dict(C=C, E=E, F=F, Xi=Xi)


def sls_random_system(B: int, N: int, n: int, p: int, nw: int, ne: int, n0: int,
                      seed: int = BASE_SEED + 501, rho: float = 0.9) -> dict:
    """Seeded dense time-varying systems of any size (every matrix differs at every step):
    A_j = rho Q_j + 0.1 G_j / sqrt(n) (Q_j orthogonal, G_j Gaussian), C_j, E_j, F_j, Xi Gaussian
    with F_j = 0.3 [I 0] + 0.1 G so that F_j F_j^T is positive definite."""
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(B, N, n, n)))
    A = rho * Q + 0.1 * rng.normal(size=(B, N, n, n)) / np.sqrt(n)
    C = rng.normal(size=(B, N, p, n)) / np.sqrt(n)
    E = 0.3 * rng.normal(size=(B, N, n, nw)) / np.sqrt(nw)
    F = 0.3 * np.eye(p, ne)[None, None] + 0.1 * rng.normal(size=(B, N, p, ne)) / np.sqrt(ne)
    Xi = 0.5 * rng.normal(size=(B, n, n0)) / np.sqrt(n0)
    return dict(A=A, C=C, E=E, F=F, Xi=Xi)


def sls_feedback_gains(B: int, N: int, m: int, n: int, scale: float = 0.05,
                       seed: int = BASE_SEED + 502) -> np.ndarray:
    """Seeded state-feedback gains K_k [B][N+1][m][n] ~ N(0, (scale / sqrt(n))^2): the input from
    which the tests and the benchmark form the state-feedback responses Phibar."""
    rng = np.random.default_rng(seed)
    return scale * rng.normal(size=(B, N + 1, m, n)) / np.sqrt(n)
