"""The allocation-free rollout adjoint (sim_rollout_vjp_noalloc) against sim_rollout_vjp.

sim_rollout_vjp_noalloc serves callers that cannot allocate device memory (a real-time control
loop that must not block on a driver allocation, or a process whose device memory is owned by
another allocator): it keeps its scratch in a fixed device array inside the library.  Calls in a
row, through the C ABI, must give the results of the handle-based entry point, whatever the
previous call left in the shared scratch.  This file is collected last so that a run stopping at
the first failure has already run every other test.
"""
import copy
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL = {4: (1e-4, 1e-3), 8: (1e-8, 1e-8)}     # (loss / states, gradients) relative


def _dtype(rb):
    return torch.float32 if rb == 4 else torch.float64


def _call_noalloc(lib, params, rest, q0, U, loss, stream, rb):
    B, H = U.shape[0], U.shape[1]
    dt = _dtype(rb)
    Lv = torch.empty(B, dtype=dt, device="cuda")
    dU = torch.empty(B, H, 6, dtype=dt, device="cuda")
    dq0 = torch.empty_like(q0)
    st = torch.zeros(B, dtype=torch.int32, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())
    code = lib.sim_rollout_vjp_noalloc(C.byref(params), rest.ctypes.data_as(C.POINTER(C.c_double)),
                                       B, H, p(q0), p(U), None, C.byref(loss), p(Lv), p(dU), p(dq0),
                                       p(st), stream)
    return code, Lv, dU, dq0, st


def _case(nodes, B, H, rb, seed):
    """A rope of `nodes` nodes shaped like the 64-node workload (2 spheres, 2 boxes, both ends
    held), B rollouts of H steps, checkpoint every 7 steps."""
    from paper_2606_14188_b300 import scenes
    if nodes == 64:
        w = scenes.workload(2, B=B, H=H)
        sc, U = w["scene"], w["U"]
    else:
        sc = scenes.rope_scene(nodes, n_spheres=2, n_boxes=2, seed=seed,
                               sphere_box=((0.0, 1.0), (-0.2, 0.2), (0.0, 0.3)))
        U = scenes.controls_normal_clear(sc, B, H, seed=seed + 1)
    sc = copy.deepcopy(sc)
    sc["params"]["checkpoint_every"] = 7
    dt = _dtype(rb)
    q0 = torch.tensor(scenes.batch_q0(sc, B), dtype=dt, device="cuda")
    Ut = torch.tensor(U, dtype=dt, device="cuda")
    return sc, q0, Ut


def _check_against_handle(lib, sc, q0, U, rb, stream, calls=1):
    from paper_2606_14188_b300.sim import Sim, make_params, make_loss
    B, H = U.shape[0], U.shape[1]
    ref = Sim(sc, real_bytes=rb, max_batch=B, max_horizon=H)
    Lr, dUr, dqr, str_ = ref.rollout_vjp(q0, U)
    params = make_params(sc, rb, B, H)
    loss = make_loss(sc)
    rest = np.ascontiguousarray(sc["rest_x"], dtype=np.float64)
    tol_s, tol_g = TOL[rb]
    for _ in range(calls):
        code, Lv, dU, dq0, st = _call_noalloc(lib, params, rest, q0, U, loss, stream, rb)
        torch.cuda.synchronize()
        assert code == 0, lib.cs_last_error()
        assert torch.equal(st, str_)
        ok = st == 0
        assert int(ok.sum()) > 0
        rel = (Lv[ok] - Lr[ok]).abs().max() / Lr[ok].abs().max()
        assert float(rel) <= tol_s
        g, gr = dU[ok].reshape(-1), dUr[ok].reshape(-1)
        assert float((g - gr).norm() / gr.norm()) <= tol_g
        assert float((dq0[ok] - dqr[ok]).norm() / dqr[ok].norm()) <= tol_g
        # failed rollouts: L is NaN and the gradients zero, on both sides
        assert bool(Lv[~ok].isnan().all()) and bool((dU[~ok] == 0).all())


@pytest.mark.parametrize("rb,nodes,B,H", [(4, 64, 96, 50), (8, 64, 12, 16), (4, 100, 32, 20),
                                          (8, 100, 6, 10)])
def test_noalloc_matches_handle_entry_point_twice(rb, nodes, B, H):
    """FP32 and FP64, one pair per lane (64 nodes) and two (100 nodes): two calls in a row."""
    from paper_2606_14188_b300 import _lib
    lib = _lib.lib()
    sc, q0, U = _case(nodes, B, H, rb, seed=2606 + nodes)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    _check_against_handle(lib, sc, q0, U, rb, stream, calls=2)


def test_noalloc_large_call_then_small_calls_of_other_shapes():
    """The benchmark's 1024 x 64-node x 50-step call fills most of the shared scratch; the calls
    after it (a 30-node rope of 8 rollouts x 9 steps, then a 100-node rope in FP64) must not see
    anything it left there."""
    from paper_2606_14188_b300 import _lib
    lib = _lib.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for nodes, B, H, rb in ((64, 1024, 50, 4), (30, 8, 9, 4), (100, 4, 11, 8), (30, 8, 9, 4)):
        sc, q0, U = _case(nodes, B, H, rb, seed=77 + nodes)
        _check_against_handle(lib, sc, q0, U, rb, stream)


def test_noalloc_rejects_oversized_batches():
    from paper_2606_14188_b300 import scenes, _lib
    from paper_2606_14188_b300.sim import make_params, make_loss
    lib = _lib.lib()
    w = scenes.workload(2, B=4)
    sc = w["scene"]
    Bbig, H = 100000, 50
    params = make_params(sc, 4, Bbig, H)
    loss = make_loss(sc)
    rest = np.ascontiguousarray(sc["rest_x"], dtype=np.float64)
    dummy = torch.zeros(8, dtype=torch.float32, device="cuda")
    p = C.c_void_p(dummy.data_ptr())
    code = lib.sim_rollout_vjp_noalloc(C.byref(params), rest.ctypes.data_as(C.POINTER(C.c_double)),
                                       Bbig, H, p, p, None, C.byref(loss), p, p, p, p, None)
    assert code == 1
    assert b"CS_NOALLOC_SCRATCH_BYTES" in lib.cs_last_error()


def test_noalloc_benchmark_batch_without_the_work_queue():
    """The benchmark's 1024 rollouts: the allocation-free call runs the adjoint without the work
    queue (it has no room for per-step records: one launch, each rollout's forward and backward in
    one CTA), the handle-based call through it; same flags, results within the FP32 tolerances
    (the two kernels inline the same device code in different contexts, so the compiler may round
    a contraction differently)."""
    from paper_2606_14188_b300 import scenes, _lib
    from paper_2606_14188_b300.sim import Sim, make_params, make_loss
    lib = _lib.lib()
    w = scenes.workload(2)
    sc = w["scene"]
    B, H = w["B"], w["H"]
    q0 = torch.tensor(w["q0"], dtype=torch.float32, device="cuda")
    U = torch.tensor(w["U"], dtype=torch.float32, device="cuda")
    Lr, dUr, dqr, str_ = Sim(sc, real_bytes=4, max_batch=B, max_horizon=H).rollout_vjp(q0, U)
    params = make_params(sc, 4, B, H)
    loss = make_loss(sc)
    rest = np.ascontiguousarray(sc["rest_x"], dtype=np.float64)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    code, Lv, dU, dq0, st = _call_noalloc(lib, params, rest, q0, U, loss, stream, 4)
    torch.cuda.synchronize()
    assert code == 0, lib.cs_last_error()
    assert torch.equal(st, str_)
    ok = st == 0
    tol_s, tol_g = TOL[4]
    assert float((Lv[ok] - Lr[ok]).abs().max() / Lr[ok].abs().max()) <= tol_s
    for a, b in ((dU[ok], dUr[ok]), (dq0[ok], dqr[ok])):
        assert float((a - b).norm() / b.norm()) <= tol_g
    assert bool(Lv[~ok].isnan().all()) and bool((dU[~ok] == 0).all())
