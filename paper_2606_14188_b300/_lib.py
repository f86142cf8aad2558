"""ctypes declarations of the C ABI in include/cordsim.h (argument marshalling only).

The shared library is built in-tree (paper_2606_14188_b300/libcordsim.so).  There is no other
implementation: if the library is missing, loading raises.
"""
from __future__ import annotations

import ctypes as C
import os

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "libcordsim.so")

CS_MAX_OBSTACLES = 8
CS_MAX_GOAL = 64
CS_ROPE, CS_CLOTH = 0, 1
CS_PLANE, CS_SPHERE, CS_BOX = 0, 1, 2
CS_HARD, CS_SMOOTH = 0, 1
CS_SURROGATE, CS_CONSISTENT = 0, 1

STATUS_NAMES = {0: "CS_OK", 1: "CS_ERR_INVALID_ARG", 2: "CS_ERR_OOM", 3: "CS_ERR_NOCONVERGE",
                4: "CS_ERR_NONFINITE", 5: "CS_ERR_TIMEOUT", 6: "CS_ERR_PENDING", 7: "CS_ERR_CUDA",
                8: "CS_ERR_CANCELLED", 9: "CS_ERR_UNSUPPORTED"}


class cs_obstacle(C.Structure):
    _fields_ = [("type", C.c_int), ("p", C.c_double * 6)]


class cs_params(C.Structure):
    _fields_ = [
        ("kind", C.c_int), ("n_nodes", C.c_int), ("rows", C.c_int), ("cols", C.c_int),
        ("grasp_node", C.c_int * 2),
        ("dt", C.c_double), ("gravity", C.c_double * 3), ("node_mass", C.c_double),
        ("k_stretch", C.c_double), ("k_shear", C.c_double), ("k_bend", C.c_double),
        ("D_max", C.c_double), ("kappa_h", C.c_double), ("kappa_c", C.c_double),
        ("kappa_hard", C.c_double), ("kappa_decay", C.c_double), ("mu", C.c_double),
        ("r_grasp", C.c_double), ("node_radius", C.c_double), ("sigma0", C.c_double),
        ("n_obstacles", C.c_int), ("obstacles", cs_obstacle * CS_MAX_OBSTACLES),
        ("fwd_mode", C.c_int), ("grad_mode", C.c_int),
        ("newton_max", C.c_int), ("ipm_max", C.c_int),
        ("newton_tol", C.c_double), ("ipm_tol", C.c_double),
        ("checkpoint_every", C.c_int), ("real_bytes", C.c_int),
        ("max_batch", C.c_int), ("max_horizon", C.c_int),
        ("second_order", C.c_int), ("damp_alpha", C.c_double), ("damp_beta", C.c_double),
    ]


class cs_loss(C.Structure):
    _fields_ = [("n_goal", C.c_int), ("goal_nodes", C.c_int * CS_MAX_GOAL),
                ("goal_pos", (C.c_double * 3) * CS_MAX_GOAL),
                ("w_goal", C.c_double), ("w_pen", C.c_double), ("pen_margin", C.c_double),
                ("w_u", C.c_double)]


class cs_mpc_config(C.Structure):
    _fields_ = [("mem_budget_bytes", C.c_size_t), ("max_slots", C.c_int), ("real_bytes", C.c_int),
                ("batched", C.c_int), ("use_graphs", C.c_int), ("autotune", C.c_int),
                ("tuner_cache", C.c_char_p)]


class cs_mpc_request(C.Structure):
    _fields_ = [("params", cs_params), ("rest_x", C.POINTER(C.c_double)),
                ("q0", C.POINTER(C.c_double)), ("warm", C.POINTER(C.c_double)), ("loss", cs_loss),
                ("H", C.c_int), ("R", C.c_int), ("G", C.c_int),
                ("lr", C.c_double), ("sigma", C.c_double), ("u_max", C.c_double),
                ("seed", C.c_uint64), ("session_id", C.c_uint64), ("deadline_ms", C.c_int)]


class cs_mpc_result(C.Structure):
    _fields_ = [("u", C.POINTER(C.c_double)), ("L", C.c_double), ("status", C.c_int32),
                ("best_iter", C.c_int32), ("best_candidate", C.c_int32),
                ("t_submit_ns", C.c_int64), ("t_start_ns", C.c_int64), ("t_done_ns", C.c_int64)]


# exported symbols and their signatures: (restype, argtypes)
SIGNATURES = {
    "sim_create": (C.c_int, [C.POINTER(cs_params), C.POINTER(C.c_double), C.POINTER(C.c_void_p)]),
    "sim_destroy": (C.c_int, [C.c_void_p]),
    "sim_rollout": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.c_void_p, C.c_void_p]),
    "sim_rollout_counters": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                       C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "sim_rollout_vjp": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.POINTER(cs_loss), C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p]),
    "sim_rollout_vjp_noalloc": (C.c_int, [C.POINTER(cs_params), C.POINTER(C.c_double), C.c_int,
                                          C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.POINTER(cs_loss), C.c_void_p, C.c_void_p, C.c_void_p,
                                          C.c_void_p, C.c_void_p]),
    "sim_linearize": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p]),
    "mpc_create": (C.c_int, [C.POINTER(cs_mpc_config), C.POINTER(C.c_void_p)]),
    "mpc_submit": (C.c_int, [C.c_void_p, C.POINTER(cs_mpc_request), C.POINTER(C.c_uint64)]),
    "mpc_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_int, C.POINTER(cs_mpc_result)]),
    "mpc_cancel": (C.c_int, [C.c_void_p, C.c_uint64]),
    "mpc_destroy": (C.c_int, [C.c_void_p]),
    "mpc_stats": (C.c_int, [C.c_void_p, C.POINTER(C.c_int64), C.POINTER(C.c_int64),
                            C.POINTER(C.c_int64), C.POINTER(C.c_int64)]),
    "sls_observer_workspace": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "sls_observer": (C.c_int, [C.c_int] * 8 + [C.c_void_p] * 10 + [C.c_void_p, C.c_size_t, C.c_void_p]),
    "sls_response": (C.c_int, [C.c_int] * 4 + [C.c_void_p, C.c_void_p, C.c_void_p]),
    "sls_closed_loop_workspace": (C.c_size_t, [C.c_int, C.c_int, C.c_int, C.c_int, C.c_int]),
    "sls_closed_loop": (C.c_int, [C.c_int] * 6 + [C.c_void_p] * 9 + [C.c_void_p, C.c_size_t, C.c_void_p]),
    "sls_tubes_workspace": (C.c_size_t, [C.c_int] * 9),
    "sls_tubes": (C.c_int, [C.c_int] * 9 + [C.c_void_p] * 12 + [C.c_void_p, C.c_size_t, C.c_void_p]),
    "sls_conformal_radius": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_double,
                                       C.c_int, C.c_void_p, C.c_void_p, C.c_void_p]),
    "apg_workspace": (C.c_size_t, [C.c_void_p, C.c_int, C.c_int, C.c_int]),
    "apg_rollout_grad": (C.c_int, [C.c_void_p, C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p,
                                   C.POINTER(cs_loss), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                   C.c_void_p, C.c_size_t, C.c_void_p]),
    "sls_kalman_scan_workspace": (C.c_size_t, [C.c_int] * 5),
    "sls_kalman_scan": (C.c_int, [C.c_int] * 8 + [C.c_void_p] * 7 + [C.c_void_p, C.c_size_t, C.c_void_p]),
    "cs_launch_count": (C.c_int64, []),
    "cs_last_error": (C.c_char_p, []),
}

_lib = None


def lib():
    """The loaded libcordsim.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError(f"{LIB_PATH} is missing: build it with "
                               "`python -m paper_2606_14188_b300.build` (no CPU fallback exists)")
        L = C.CDLL(LIB_PATH)
        for name, (res, args) in SIGNATURES.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


class CordsimError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = lib().cs_last_error().decode()
        super().__init__(f"{where}: {STATUS_NAMES.get(code, code)}: {msg}")
        self.code = code


def check(code: int, where: str):
    if code != 0:
        raise CordsimError(code, where)
