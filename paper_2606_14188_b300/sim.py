"""Python handle over libcordsim (argument marshalling only; all work runs in the CUDA kernels).

Tensors are torch CUDA tensors (torch provides device memory and streams); the library reads and
writes them in place through their device pointers, on the current torch stream.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib as L

DEFAULT_TOL = {4: dict(newton_tol=1e-5, ipm_tol=1e-7, newton_max=100, ipm_max=80),
               8: dict(newton_tol=1e-12, ipm_tol=1e-12, newton_max=100, ipm_max=200)}


def make_params(scene: dict, real_bytes: int = 4, max_batch: int = 1, max_horizon: int = 1,
                **overrides) -> L.cs_params:
    """cs_params from a scene dict of paper_2606_14188_b300.scenes (plus overrides)."""
    p = dict(scene["params"])
    p.update(overrides)
    P = L.cs_params()
    P.kind = L.CS_ROPE if p["kind"] == "rope" else L.CS_CLOTH
    P.n_nodes = int(p["n_nodes"])
    P.rows, P.cols = int(p.get("rows", 0)), int(p.get("cols", 0))
    P.grasp_node[0], P.grasp_node[1] = (int(v) for v in p["grasp_nodes"])
    P.dt = p["dt"]
    for i in range(3):
        P.gravity[i] = p["gravity"][i]
    P.node_mass = p["node_mass"]
    P.k_stretch, P.k_shear, P.k_bend = p["k_stretch"], p["k_shear"], p["k_bend"]
    P.D_max, P.kappa_h, P.kappa_c = p["D_max"], p["kappa_h"], p["kappa_c"]
    P.kappa_hard, P.kappa_decay, P.mu = p["kappa_hard"], p["kappa_decay"], p["mu"]
    P.r_grasp, P.node_radius, P.sigma0 = p["r_grasp"], p["node_radius"], p["sigma0"]
    obs = p["obstacles"]
    if len(obs) > L.CS_MAX_OBSTACLES:
        raise ValueError("too many obstacles")
    P.n_obstacles = len(obs)
    for o, ob in enumerate(obs):
        if ob["type"] == "plane":
            P.obstacles[o].type = L.CS_PLANE
            vals = list(ob["normal"]) + [ob["offset"]]
        elif ob["type"] == "sphere":
            P.obstacles[o].type = L.CS_SPHERE
            vals = list(ob["center"]) + [ob["radius"]]
        elif ob["type"] == "box":
            P.obstacles[o].type = L.CS_BOX
            vals = list(ob["center"]) + list(ob["half"])
        else:
            raise ValueError(ob["type"])
        for i, v in enumerate(vals):
            P.obstacles[o].p[i] = float(v)
    P.fwd_mode = L.CS_HARD if p["fwd_mode"] == "hard" else L.CS_SMOOTH
    P.grad_mode = L.CS_SURROGATE if p["grad_mode"] == "surrogate" else L.CS_CONSISTENT
    P.second_order = int(bool(p.get("second_order", False)))
    P.damp_alpha, P.damp_beta = float(p.get("damp_alpha", 0.0)), float(p.get("damp_beta", 0.0))
    tol = DEFAULT_TOL[real_bytes]
    P.newton_max = int(overrides.get("newton_max", tol["newton_max"]))
    P.ipm_max = int(overrides.get("ipm_max", tol["ipm_max"]))
    P.newton_tol = float(overrides.get("newton_tol", tol["newton_tol"]))
    P.ipm_tol = float(overrides.get("ipm_tol", tol["ipm_tol"]))
    P.checkpoint_every = int(p.get("checkpoint_every", 1))
    P.real_bytes = real_bytes
    P.max_batch, P.max_horizon = int(max_batch), int(max_horizon)
    return P


def make_loss(scene: dict) -> L.cs_loss:
    ls = scene["params"]["loss"]
    out = L.cs_loss()
    nodes = list(ls["goal_nodes"])
    if len(nodes) > L.CS_MAX_GOAL:
        raise ValueError("too many goal nodes")
    out.n_goal = len(nodes)
    gp = np.asarray(ls["goal_pos"], dtype=np.float64).reshape(-1, 3)
    for g, j in enumerate(nodes):
        out.goal_nodes[g] = int(j)
        for i in range(3):
            out.goal_pos[g][i] = float(gp[g, i])
    out.w_goal, out.w_pen = ls["w_goal"], ls["w_pen"]
    out.pen_margin, out.w_u = ls["pen_margin"], ls["w_u"]
    return out


def _ptr(t):
    return C.c_void_p(t.data_ptr()) if t is not None else None


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class Sim:
    """One scene on the GPU: sim_create / sim_rollout / sim_rollout_vjp / sim_linearize.

    The adjoint's checkpoint interval is the scene's params["checkpoint_every"] (1 when absent:
    every step recorded, nothing recomputed; 0: the library picks the shortest interval whose
    workspace fits in a quarter of the free device memory).  The gradients do not depend on it."""

    def __init__(self, scene: dict, real_bytes: int = 4, max_batch: int = 1, max_horizon: int = 1,
                 **overrides):
        self.scene = scene
        self.real_bytes = real_bytes
        self.dtype = torch.float32 if real_bytes == 4 else torch.float64
        self.params = make_params(scene, real_bytes, max_batch, max_horizon, **overrides)
        self.loss = make_loss(scene)
        self.nv = int(self.params.n_nodes)
        # state [x, g] (quasi-static), [x, v, g] (inertial variant)
        self.nq = (6 if self.params.second_order else 3) * self.nv + 6
        rest = np.ascontiguousarray(scene["rest_x"], dtype=np.float64)
        h = C.c_void_p()
        L.check(L.lib().sim_create(C.byref(self.params),
                                   rest.ctypes.data_as(C.POINTER(C.c_double)), C.byref(h)),
                "sim_create")
        self._h = h

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            L.lib().sim_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    # -- argument checks ------------------------------------------------------------------
    def _t(self, x, shape, name):
        if not (isinstance(x, torch.Tensor) and x.is_cuda):
            raise ValueError(f"{name} must be a CUDA tensor")
        if x.dtype != self.dtype:
            raise ValueError(f"{name} must be {self.dtype}")
        if tuple(x.shape) != tuple(shape):
            raise ValueError(f"{name} has shape {tuple(x.shape)}, expected {tuple(shape)}")
        if not x.is_contiguous():
            raise ValueError(f"{name} must be contiguous")
        return x

    def _new(self, *shape):
        return torch.empty(*shape, dtype=self.dtype, device="cuda")

    # -- calls ----------------------------------------------------------------------------
    def rollout(self, q0, U, want_traj=True):
        B, H = U.shape[0], U.shape[1]
        self._t(q0, (B, self.nq), "q0")
        self._t(U, (B, H, 6), "U")
        traj = self._new(B, H + 1, self.nq) if want_traj else None
        qH = self._new(B, self.nq)
        status = torch.zeros(B, dtype=torch.int32, device="cuda")
        L.check(L.lib().sim_rollout(self._h, B, H, _ptr(q0), _ptr(U), _ptr(traj), _ptr(qH),
                                    _ptr(status), _stream()), "sim_rollout")
        return traj, qH, status

    def rollout_counters(self, q0, U):
        """rollout plus per-step solver counters [B, H, 3] = (Newton its, IPM its, status)."""
        B, H = U.shape[0], U.shape[1]
        self._t(q0, (B, self.nq), "q0")
        self._t(U, (B, H, 6), "U")
        traj = self._new(B, H + 1, self.nq)
        qH = self._new(B, self.nq)
        status = torch.zeros(B, dtype=torch.int32, device="cuda")
        counters = torch.zeros(B, H, 3, dtype=torch.int32, device="cuda")
        L.check(L.lib().sim_rollout_counters(self._h, B, H, _ptr(q0), _ptr(U), _ptr(traj),
                                             _ptr(qH), _ptr(status), _ptr(counters), _stream()),
                "sim_rollout_counters")
        return traj, qH, status, counters

    def rollout_vjp(self, q0, U, dL_dtraj=None, use_loss=True, want_dq0=True):
        B, H = U.shape[0], U.shape[1]
        self._t(q0, (B, self.nq), "q0")
        self._t(U, (B, H, 6), "U")
        if dL_dtraj is not None:
            self._t(dL_dtraj, (B, H + 1, self.nq), "dL_dtraj")
        Lv = self._new(B)
        dU = self._new(B, H, 6)
        dq0 = self._new(B, self.nq) if want_dq0 else None
        status = torch.zeros(B, dtype=torch.int32, device="cuda")
        loss = C.byref(self.loss) if use_loss else None
        L.check(L.lib().sim_rollout_vjp(self._h, B, H, _ptr(q0), _ptr(U), _ptr(dL_dtraj), loss,
                                        _ptr(Lv), _ptr(dU), _ptr(dq0), _ptr(status), _stream()),
                "sim_rollout_vjp")
        return Lv, dU, dq0, status

    def apg_grad(self, q0, theta, hidden: int, H: int):
        """Analytic policy gradient: the closed-loop rollout of the tanh policy theta (packed
        [W1 (hidden x n_q), b1, W2 (6 x hidden), b2]) from q0 [B][n_q] over H steps and the
        gradient of the scene's planning loss -> L [B], dL/dtheta [n_theta], dL/dq0 [B][n_q],
        status [B]."""
        B = q0.shape[0]
        nth = hidden * self.nq + 7 * hidden + 6
        self._t(q0, (B, self.nq), "q0")
        self._t(theta, (nth,), "theta")
        Lv = self._new(B)
        dth = self._new(nth)
        dq0 = self._new(B, self.nq)
        status = torch.zeros(B, dtype=torch.int32, device="cuda")
        lib = L.lib()
        wsb = lib.apg_workspace(self._h, B, H, hidden)
        ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device="cuda")
        L.check(lib.apg_rollout_grad(self._h, B, H, hidden, _ptr(q0), _ptr(theta), C.byref(self.loss),
                                     _ptr(Lv), _ptr(dth), _ptr(dq0), _ptr(status), _ptr(ws), wsb,
                                     _stream()), "apg_rollout_grad")
        return Lv, dth, dq0, status

    def linearize(self, Z, V):
        B, H = V.shape[0], V.shape[1]
        self._t(Z, (B, H + 1, self.nq), "z")
        self._t(V, (B, H, 6), "v")
        A = self._new(B, H, self.nq, self.nq)
        Bm = self._new(B, H, self.nq, 6)
        status = torch.zeros(B, dtype=torch.int32, device="cuda")
        L.check(L.lib().sim_linearize(self._h, B, H, _ptr(Z), _ptr(V), _ptr(A), _ptr(Bm),
                                      _ptr(status), _stream()), "sim_linearize")
        return A, Bm, status


class RolloutFn(torch.autograd.Function):
    """traj = rollout(q0, U) as a differentiable layer: forward = sim_rollout, backward =
    sim_rollout_vjp with the incoming dL/dtraj (surrogate or consistent gradient per the
    handle's grad_mode).  The forward model follows grad_mode too (nonsmooth for surrogate)."""

    @staticmethod
    def forward(ctx, q0, U, sim: Sim):
        ctx.sim = sim
        ctx.save_for_backward(q0, U)
        traj, _, status = sim.rollout(q0.contiguous(), U.contiguous())
        ctx.mark_non_differentiable(status)
        return traj, status

    @staticmethod
    def backward(ctx, g_traj, g_status):
        q0, U = ctx.saved_tensors
        sim = ctx.sim
        _, dU, dq0, _ = sim.rollout_vjp(q0.contiguous(), U.contiguous(),
                                        dL_dtraj=g_traj.contiguous(), use_loss=False)
        return dq0, dU, None
