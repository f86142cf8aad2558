"""Python handle over the plan-solve server of libcordsim (argument marshalling only: the
candidates, rollouts, adjoints, selection and Adam steps all run in the library's CUDA kernels on
the server's own stream, driven by its native scheduler thread)."""
from __future__ import annotations

import ctypes as C

import numpy as np

from . import _lib as L
from .sim import make_loss, make_params

CS_ERR_TIMEOUT, CS_ERR_PENDING, CS_ERR_CANCELLED = 5, 6, 8


class PlanServer:
    """mpc_create / mpc_submit / mpc_poll / mpc_cancel / mpc_destroy.

    batched=True: continuous batching (requests join and leave the running set between
    evaluations; a stable set replays a captured CUDA graph).  batched=False: one request at a
    time with one launch per kernel per evaluation (the per-request form)."""

    def __init__(self, real_bytes: int = 4, mem_budget_bytes: int = 0, max_slots: int = 64,
                 batched: bool = True, use_graphs: bool = True, autotune: bool = False,
                 tuner_cache: str | None = None):
        cfg = L.cs_mpc_config()
        cfg.mem_budget_bytes = int(mem_budget_bytes)
        cfg.max_slots = int(max_slots)
        cfg.real_bytes = int(real_bytes)
        cfg.batched = int(batched)
        cfg.use_graphs = int(use_graphs)
        cfg.autotune = int(autotune)
        cfg.tuner_cache = tuner_cache.encode() if tuner_cache else None
        self._h = C.c_void_p()
        L.check(L.lib().mpc_create(C.byref(cfg), C.byref(self._h)), "mpc_create")
        self.real_bytes = real_bytes
        self._horizon = {}

    def submit(self, scene: dict, q0, H: int, R: int, G: int, lr: float = 0.005,
               sigma: float = 0.02, u_max: float = 0.05, seed: int = 0, warm=None,
               session_id: int = 0, deadline_ms: int = 0, **param_overrides) -> int:
        req = L.cs_mpc_request()
        req.params = make_params(scene, real_bytes=self.real_bytes, **param_overrides)
        rest = np.ascontiguousarray(scene["rest_x"], dtype=np.float64).ravel()
        q0 = np.ascontiguousarray(q0, dtype=np.float64).ravel()
        req.rest_x = rest.ctypes.data_as(C.POINTER(C.c_double))
        req.q0 = q0.ctypes.data_as(C.POINTER(C.c_double))
        if warm is not None:
            warm = np.ascontiguousarray(warm, dtype=np.float64).reshape(H, 6)
            req.warm = warm.ctypes.data_as(C.POINTER(C.c_double))
        req.loss = make_loss(scene)
        req.H, req.R, req.G = int(H), int(R), int(G)
        req.lr, req.sigma, req.u_max = float(lr), float(sigma), float(u_max)
        req.seed, req.session_id = int(seed), int(session_id)
        req.deadline_ms = int(deadline_ms)
        t = C.c_uint64()
        L.check(L.lib().mpc_submit(self._h, C.byref(req), C.byref(t)), "mpc_submit")
        self._horizon[t.value] = int(H)
        return t.value

    def poll(self, ticket: int, timeout_ms: int = -1):
        """The result dict, or None while it is pending; raises for a cancelled, timed-out
        (deadline passed) or failed solve."""
        H = self._horizon[ticket]
        u = np.zeros((H, 6))
        res = L.cs_mpc_result()
        res.u = u.ctypes.data_as(C.POINTER(C.c_double))
        rc = L.lib().mpc_poll(self._h, C.c_uint64(ticket), int(timeout_ms), C.byref(res))
        if rc == CS_ERR_PENDING:
            return None
        L.check(rc, "mpc_poll")
        del self._horizon[ticket]
        return dict(u=u, L=res.L, status=res.status, best_iter=res.best_iter,
                    best_candidate=res.best_candidate, t_submit_ns=res.t_submit_ns,
                    t_start_ns=res.t_start_ns, t_done_ns=res.t_done_ns)

    def cancel(self, ticket: int):
        L.check(L.lib().mpc_cancel(self._h, C.c_uint64(ticket)), "mpc_cancel")

    def stats(self) -> dict:
        v = [C.c_int64() for _ in range(4)]
        L.check(L.lib().mpc_stats(self._h, *[C.byref(x) for x in v]), "mpc_stats")
        return dict(ticks=v[0].value, graph_launches=v[1].value, kernel_launches=v[2].value,
                    graphs_built=v[3].value)

    def close(self):
        if self._h:
            L.lib().mpc_destroy(self._h)
            self._h = C.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
