"""The analytic policy gradient on the GPU (apg_rollout_grad; paper Sec. 4.3) against its FP64
oracle, oracle/apg.py: the closed-loop rollout of a tanh policy on ropes with obstacles (the
planning loss's goal, penalty and effort), its loss, dL/dtheta and dL/dq0, in FP64 and FP32."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import apg, sim as osim  # noqa: E402
from paper_2606_14188_b300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu


def _t(x, rb):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float32 if rb == 4 else torch.float64,
                        device="cuda")


def _theta(nq, h, seed, scale):
    rng = np.random.default_rng(seed)
    return scale * rng.normal(size=apg.n_theta(nq, h)) / np.sqrt(nq)


@pytest.mark.parametrize("rb,tol_l,tol_g,cos,nv,h,H", [(8, 1e-8, 1e-7, 1 - 1e-12, 12, 8, 5),
                                                     (4, 1e-4, 1e-3, 0.999, 20, 16, 10)])
def test_apg_matches_the_oracle(rb, tol_l, tol_g, cos, nv, h, H):
    from paper_2606_14188_b300.sim import Sim
    sc = scenes.rope_scene(nv, n_spheres=2, n_boxes=1, seed=61 + nv,
                           sphere_box=((0.0, 1.0), (-0.2, 0.2), (0.0, 0.3)))
    osc = osim.Scene(sc["params"], sc["rest_x"])
    B = 3
    q0 = scenes.batch_q0(sc, B)
    th = _theta(osc.nq, h, nv, 0.05)
    s = Sim(sc, real_bytes=rb, max_batch=B, max_horizon=H)
    Lv, dth, dq0, st = s.apg_grad(_t(q0, rb), _t(th, rb), h, H)
    assert np.all(st.cpu().numpy() == 0)
    ref_dth = np.zeros_like(th)
    for b in range(B):
        r = apg.rollout_grad(osc, q0[b], th, h, H)
        assert r["status"] == 0
        assert abs(float(Lv[b]) - r["L"]) <= tol_l * abs(r["L"]), b
        g = dq0[b].cpu().numpy()
        assert np.linalg.norm(g - r["dq0"]) <= tol_g * np.linalg.norm(r["dq0"]), b
        ref_dth += r["dtheta"]
    g = dth.cpu().numpy()
    assert np.linalg.norm(g - ref_dth) <= tol_g * np.linalg.norm(ref_dth)
    assert g @ ref_dth >= cos * np.linalg.norm(g) * np.linalg.norm(ref_dth)


def test_apg_state_blind_policy_equals_the_open_loop_gradient_on_the_gpu():
    """W1 = 0 on the GPU: dL/db2 equals the sum over t of sim_rollout_vjp's dL/du_t for the
    constant controls, dL/dq0 its dL/dq0 (both calls on the GPU, FP64)."""
    from paper_2606_14188_b300.sim import Sim
    sc = scenes.rope_scene(16, n_spheres=1, n_boxes=1, seed=71,
                           sphere_box=((0.0, 1.0), (-0.2, 0.2), (0.0, 0.3)))
    osc = osim.Scene(sc["params"], sc["rest_x"])
    B, h, H = 2, 4, 6
    q0 = scenes.batch_q0(sc, B)
    th = _theta(osc.nq, h, 72, 0.5)
    th[:h * osc.nq] = 0.0
    s = Sim(sc, real_bytes=8, max_batch=B, max_horizon=H)
    Lv, dth, dq0, st = s.apg_grad(_t(q0, 8), _t(th, 8), h, H)
    u0 = apg.policy(th, q0[0], h)[0]
    U = np.repeat(np.repeat(u0[None], H, 0)[None], B, 0)
    L2, dU, dq2, st2 = s.rollout_vjp(_t(q0, 8), _t(U, 8))
    assert np.all(st.cpu().numpy() == 0) and np.all(st2.cpu().numpy() == 0)
    assert np.allclose(Lv.cpu().numpy(), L2.cpu().numpy(), rtol=1e-12)
    assert np.allclose(dth.cpu().numpy()[-6:], dU.cpu().numpy().sum(axis=(0, 1)), rtol=1e-10, atol=1e-14)
    assert np.allclose(dq0.cpu().numpy(), dq2.cpu().numpy(), rtol=1e-10, atol=1e-14)
