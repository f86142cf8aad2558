"""The allocation-free rollout adjoint (sim_rollout_vjp_noalloc) against sim_rollout_vjp.

sim_rollout_vjp_noalloc serves callers that cannot allocate device memory (a real-time control
loop that must not block on a driver allocation, or a process whose device memory is owned by
another allocator): it keeps its scratch in a fixed device array inside the library.  Two calls
in a row, through the C ABI, must give the results of the handle-based entry point.  This file is
collected last so that a run stopping at the first failure has already run every other test.
"""
import ctypes as C

import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu

TOL_STATE32, TOL_GRAD32 = 1e-4, 1e-3


def _call_noalloc(lib, params, rest, q0, U, loss, stream):
    B, H = U.shape[0], U.shape[1]
    Lv = torch.empty(B, dtype=torch.float32, device="cuda")
    dU = torch.empty(B, H, 6, dtype=torch.float32, device="cuda")
    dq0 = torch.empty_like(q0)
    st = torch.zeros(B, dtype=torch.int32, device="cuda")
    p = lambda t: C.c_void_p(t.data_ptr())
    code = lib.sim_rollout_vjp_noalloc(C.byref(params), rest.ctypes.data_as(C.POINTER(C.c_double)),
                                       B, H, p(q0), p(U), None, C.byref(loss), p(Lv), p(dU), p(dq0),
                                       p(st), stream)
    return code, Lv, dU, dq0, st


def test_noalloc_matches_handle_entry_point_twice():
    from paper_2606_14188_b300 import scenes, _lib
    from paper_2606_14188_b300.sim import Sim, make_params, make_loss
    lib = _lib.lib()
    w = scenes.workload(2, B=96)
    sc = w["scene"]
    B, H = w["B"], w["H"]
    q0 = torch.tensor(w["q0"], dtype=torch.float32, device="cuda")
    U = torch.tensor(w["U"], dtype=torch.float32, device="cuda")
    ref = Sim(sc, real_bytes=4, max_batch=B, max_horizon=H)
    Lr, dUr, dqr, str_ = ref.rollout_vjp(q0, U)
    params = make_params(sc, 4, B, H)
    loss = make_loss(sc)
    rest = np.ascontiguousarray(sc["rest_x"], dtype=np.float64)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):
        code, Lv, dU, dq0, st = _call_noalloc(lib, params, rest, q0, U, loss, stream)
        torch.cuda.synchronize()
        assert code == 0, lib.cs_last_error()
        assert torch.equal(st, str_)
        ok = (st == 0)
        rel = (Lv[ok] - Lr[ok]).abs().max() / Lr[ok].abs().max()
        assert float(rel) <= TOL_STATE32
        g, gr = dU[ok].reshape(-1), dUr[ok].reshape(-1)
        assert float((g - gr).norm() / gr.norm()) <= TOL_GRAD32
        assert float((dq0[ok] - dqr[ok]).norm() / dqr[ok].norm()) <= TOL_GRAD32


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


def test_noalloc_benchmark_batch_two_part_launch():
    """The benchmark's 1024 rollouts (more than the device holds at once: forward parts, cost
    order and backward parts, the order arrays inside the fixed scratch) equal the handle-based
    call, bit for bit."""
    from paper_2606_14188_b300 import scenes, _lib
    from paper_2606_14188_b300.sim import Sim, make_params, make_loss
    lib = _lib.lib()
    w = scenes.workload(2)
    sc = w["scene"]
    B, H = w["B"], w["H"]
    q0 = torch.tensor(w["q0"], dtype=torch.float32, device="cuda")
    U = torch.tensor(w["U"], dtype=torch.float32, device="cuda")
    ref = Sim(sc, real_bytes=4, max_batch=B, max_horizon=H).rollout_vjp(q0, U)
    params = make_params(sc, 4, B, H)
    loss = make_loss(sc)
    rest = np.ascontiguousarray(sc["rest_x"], dtype=np.float64)
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    code, Lv, dU, dq0, st = _call_noalloc(lib, params, rest, q0, U, loss, stream)
    torch.cuda.synchronize()
    assert code == 0, lib.cs_last_error()
    for a, b in zip((Lv, dU, dq0, st), ref):
        assert torch.equal(a.isnan(), b.isnan()) and torch.equal(a.nan_to_num(), b.nan_to_num())
