"""The C-ABI library loads and exports every entry point include/cordsim.h declares, and the
ctypes mirrors of its structs have the C layout (CPU only: no compute call is made)."""
import ctypes as C
import os
import re
import subprocess
import tempfile

import numpy as np
import pytest

from paper_2606_14188_b300 import _lib as L

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "cordsim.h")


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\**\s*([a-z_][a-z0-9_]*)\s*\(",
                       text, flags=re.M)
    return sorted(set(names))


def test_library_exports_every_declared_symbol():
    lib = L.lib()
    names = declared_functions()
    assert {"sim_create", "sim_destroy", "sim_rollout", "sim_rollout_vjp", "sim_linearize",
            "cs_last_error"} <= set(names)
    for n in names:
        assert hasattr(lib, n), n
        assert n in L.SIGNATURES, f"{n} has no ctypes signature"


def test_struct_layout_matches_c():
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "cordsim.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(cs_params), sizeof(cs_loss), sizeof(cs_obstacle),
             offsetof(cs_params, obstacles), offsetof(cs_params, max_horizon),
             offsetof(cs_loss, goal_pos), offsetof(cs_params, newton_tol), offsetof(cs_params, damp_beta));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in out]
    assert vals == [C.sizeof(L.cs_params), C.sizeof(L.cs_loss), C.sizeof(L.cs_obstacle),
                    L.cs_params.obstacles.offset, L.cs_params.max_horizon.offset,
                    L.cs_loss.goal_pos.offset, L.cs_params.newton_tol.offset, L.cs_params.damp_beta.offset]


def test_mpc_struct_layout_matches_c():
    src = r"""
    #include <stdio.h>
    #include <stddef.h>
    #include "cordsim.h"
    int main(void) {
      printf("%zu %zu %zu %zu %zu %zu %zu %zu %zu %zu\n", sizeof(cs_mpc_config), sizeof(cs_mpc_request),
             sizeof(cs_mpc_result), offsetof(cs_mpc_config, tuner_cache), offsetof(cs_mpc_request, loss),
             offsetof(cs_mpc_request, H), offsetof(cs_mpc_request, session_id),
             offsetof(cs_mpc_request, deadline_ms),
             offsetof(cs_mpc_result, best_candidate), offsetof(cs_mpc_result, t_done_ns));
      return 0;
    }
    """
    with tempfile.TemporaryDirectory() as d:
        c = os.path.join(d, "t.c")
        exe = os.path.join(d, "t")
        open(c, "w").write(src)
        subprocess.run(["gcc", "-I", os.path.join(ROOT, "include"), c, "-o", exe], check=True)
        out = subprocess.run([exe], capture_output=True, text=True, check=True).stdout.split()
    vals = [int(v) for v in out]
    assert vals == [C.sizeof(L.cs_mpc_config), C.sizeof(L.cs_mpc_request), C.sizeof(L.cs_mpc_result),
                    L.cs_mpc_config.tuner_cache.offset, L.cs_mpc_request.loss.offset,
                    L.cs_mpc_request.H.offset, L.cs_mpc_request.session_id.offset,
                    L.cs_mpc_request.deadline_ms.offset, L.cs_mpc_result.best_candidate.offset,
                    L.cs_mpc_result.t_done_ns.offset]


def test_argument_errors_without_gpu():
    """Argument errors are reported before any device work (null arguments, bad kinds)."""
    lib = L.lib()
    h = C.c_void_p()
    assert lib.sim_create(None, None, C.byref(h)) == 1
    assert b"null" in lib.cs_last_error()
    assert lib.sim_rollout(None, 1, 1, None, None, None, None, None, None) == 1
    assert lib.sim_destroy(None) == 0
    assert lib.mpc_create(None, C.byref(h)) == 1
    assert lib.mpc_submit(None, None, None) == 1
    assert lib.mpc_poll(None, 1, 0, None) == 1
    assert lib.mpc_cancel(None, 1) == 1
    assert lib.mpc_destroy(None) == 0


def test_cloth_argument_errors_without_gpu():
    """Malformed cloth grids and unknown kinds are rejected before any device call."""
    from paper_2606_14188_b300 import scenes
    from paper_2606_14188_b300.sim import make_params
    lib = L.lib()
    sc = scenes.cloth_scene(4, 5, n_spheres=1, seed=1)
    rest = np.ascontiguousarray(sc["rest_x"], dtype=np.float64)
    rp = rest.ctypes.data_as(C.POINTER(C.c_double))
    h = C.c_void_p()
    for bad in (dict(rows=4, cols=6), dict(rows=0, cols=5), dict(rows=20, cols=1), dict(kind="x")):
        P = make_params(sc)
        if "kind" in bad:
            P.kind = 7
        else:
            P.rows, P.cols = bad["rows"], bad["cols"]
        assert lib.sim_create(C.byref(P), rp, C.byref(h)) == 1, bad
        assert not h.value


def test_noalloc_argument_errors_without_gpu():
    """The allocation-free entry point checks its parameters and loss as sim_create and
    sim_rollout_vjp do, before any device call: a goal list longer than CS_MAX_GOAL, a goal node
    past the chain, both grippers on one node, an unknown obstacle type, a non-positive time step
    or node mass, zero iteration caps and barrier parameters out of order all fail with
    CS_ERR_INVALID_ARG (the device pointers below are never dereferenced)."""
    from paper_2606_14188_b300 import scenes
    from paper_2606_14188_b300.sim import make_params, make_loss
    lib = L.lib()
    w = scenes.workload(2, B=2)
    sc = w["scene"]
    rest = np.ascontiguousarray(sc["rest_x"], dtype=np.float64)
    rp = rest.ctypes.data_as(C.POINTER(C.c_double))
    fake = C.c_void_p(256)            # a device address, never touched by a failing call

    def call(P, loss):
        return lib.sim_rollout_vjp_noalloc(C.byref(P), rp, 2, 5, fake, fake, None,
                                           C.byref(loss) if loss is not None else None,
                                           fake, fake, fake, fake, None)

    loss = make_loss(sc)
    loss.n_goal = L.CS_MAX_GOAL + 1
    assert call(make_params(sc, 4, 2, 5), loss) == 1
    assert b"n_goal" in lib.cs_last_error()
    loss = make_loss(sc)
    loss.goal_nodes[0] = sc["params"]["n_nodes"]
    assert call(make_params(sc, 4, 2, 5), loss) == 1
    assert b"goal node" in lib.cs_last_error()

    def bad(**kw):
        P = make_params(sc, 4, 2, 5)
        for k, v in kw.items():
            if k == "grasp":
                P.grasp_node[0], P.grasp_node[1] = v
            elif k == "ob_type":
                P.obstacles[0].type = v
            else:
                setattr(P, k, v)
        return P

    for P in (bad(grasp=(3, 3)), bad(ob_type=9), bad(dt=0.0), bad(node_mass=-1.0),
              bad(newton_max=0), bad(ipm_max=0), bad(kappa_decay=1.0), bad(kappa_hard=1.0),
              bad(real_bytes=2), bad(n_nodes=129), bad(checkpoint_every=0)):
        assert call(P, make_loss(sc)) == 1, lib.cs_last_error()


def test_sls_argument_errors_without_gpu():
    """The SLS observer-stage calls check sizes, pointers and the workspace before any device call
    (the device pointers below are never dereferenced); an empty batch without a status array
    makes no device call at all."""
    lib = L.lib()
    f = C.c_void_p(256)
    ws = lib.sls_observer_workspace(2, 3, 10, 4, 4)
    assert ws > 0 and lib.sls_observer_workspace(2, 3, 0, 4, 4) == 0

    def obs(B=2, N=3, n=10, p=4, rb=4, ptr=f, wsb=ws):
        return lib.sls_observer(B, N, n, p, n, p, n, rb, ptr, ptr, ptr, ptr, ptr, ptr, ptr, ptr, ptr,
                                None, ptr, wsb, None)

    assert obs(n=0) == 1
    assert obs(N=0) == 1
    assert obs(B=-1) == 1
    assert obs(rb=2) == 1
    assert obs(p=400) == 1 and b"shared memory" in lib.cs_last_error()
    assert obs(ptr=None) == 1 and b"null" in lib.cs_last_error()
    assert obs(wsb=ws - 1) == 1 and b"workspace" in lib.cs_last_error()
    assert obs(B=0, ptr=None, wsb=0) == 0
    assert lib.sls_response(1, 3, 0, 4, f, f, None) == 1
    assert lib.sls_response(1, 3, 4, 4, None, f, None) == 1
    cw = lib.sls_closed_loop_workspace(2, 3, 10, 4, 8)
    assert cw > 0
    assert lib.sls_closed_loop(2, 3, 10, 0, 4, 8, *([f] * 9), f, cw, None) == 1
    assert lib.sls_closed_loop(2, 3, 10, 6, 4, 8, *([f] * 9), f, cw - 1, None) == 1
    assert lib.sls_closed_loop(0, 3, 10, 6, 4, 8, *([None] * 9), None, 0, None) == 0


def test_tube_and_conformal_argument_errors_without_gpu():
    """sls_tubes and sls_conformal_radius check sizes, pointers, the workspace and the miscoverage
    level before any device call (the pointers below are never dereferenced)."""
    lib = L.lib()
    f = C.c_void_p(256)
    ws = lib.sls_tubes_workspace(2, 3, 10, 2, 4, 10, 4, 5, 4)
    assert ws > 0 and lib.sls_tubes_workspace(2, 3, 10, 2, 4, 10, 4, -1, 4) == 0

    def tub(nc=5, cons=f, wsb=ws, m=2):
        return lib.sls_tubes(2, 3, 10, m, 4, 10, 4, nc, 4, f, f, f, f, f, f, cons, cons, cons, cons, f,
                             cons, f, wsb, None)

    assert tub(m=0) == 1
    assert tub(nc=-1) == 1
    assert tub(cons=None) == 1 and b"constraint" in lib.cs_last_error()
    assert tub(wsb=ws - 1) == 1 and b"workspace" in lib.cs_last_error()
    cr = lib.sls_conformal_radius
    assert cr(0, 3, 4, f, f, 0.1, 1, None, f, None) == 1
    assert cr(8193, 3, 4, f, f, 0.1, 1, None, f, None) == 1
    assert cr(10, 3, 4, f, f, 0.0, 1, None, f, None) == 1
    assert cr(10, 3, 4, f, f, 1.0, 1, None, f, None) == 1
    assert cr(10, 3, 4, f, f, 0.1, 0, None, f, None) == 1
    assert cr(10, 3, 4, f, f, 0.1, 1, None, None, None) == 1
    assert cr(10, 3, 2, f, f, 0.1, 1, None, f, None) == 1


def test_apg_argument_errors_without_gpu():
    """apg_rollout_grad rejects a NULL handle and NULL arguments before any device call."""
    lib = L.lib()
    f = C.c_void_p(256)
    assert lib.apg_workspace(None, 1, 1, 1) == 0
    assert lib.apg_rollout_grad(None, 1, 1, 8, f, f, None, None, f, None, None, f, 1 << 20, None) == 1
    assert b"null" in lib.cs_last_error()
