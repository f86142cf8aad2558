"""Pins of the analytic-policy-gradient oracle (oracle/apg.py, paper Sec. 4.3): the policy's
derivatives against central differences, the closed-loop gradient against central differences of
the closed-loop loss where the smooth and nonsmooth steps coincide, and against the open-loop
adjoint when the policy ignores the state."""
import numpy as np

from oracle import apg, grad, sim
from paper_2606_14188_b300 import scenes
from test_oracle_pins import rope


def _theta(nq, h, seed, scale=0.3):
    rng = np.random.default_rng(seed)
    th = scale * rng.normal(size=apg.n_theta(nq, h)) / np.sqrt(nq)
    return th


def test_policy_derivatives_match_central_differences():
    nq, h = 12, 5
    rng = np.random.default_rng(1)
    th, q, g = _theta(nq, h, 2, 1.0), rng.normal(size=nq), rng.normal(size=6)
    dq, dth = apg.policy_vjp(th, q, h, g)
    eps = 1e-6
    for k in range(nq):
        e = np.zeros(nq); e[k] = eps
        fd = (apg.policy(th, q + e, h)[0] - apg.policy(th, q - e, h)[0]) @ g / (2 * eps)
        assert abs(fd - dq[k]) < 1e-8
    for k in range(0, th.size, 7):
        e = np.zeros(th.size); e[k] = eps
        fd = (apg.policy(th + e, q, h)[0] - apg.policy(th - e, q, h)[0]) @ g / (2 * eps)
        assert abs(fd - dth[k]) < 1e-8


def _free_rope():
    """No obstacles and the grasp held with kappa_h large: the smooth and nonsmooth steps coincide,
    so the surrogate closed-loop gradient is the exact gradient of the closed-loop loss."""
    X0 = np.stack([np.linspace(0.0, 0.3, 6), np.zeros(6), np.full(6, 0.3)], axis=1)
    sc, q0 = rope(6, X0, m=0.1 / 6)
    sc.p["kappa_h"] = 1e6
    sc.p["loss"] = dict(goal_nodes=(2, 3), goal_pos=X0[[2, 3]] + [0.0, 0.0, 0.05], w_goal=1.0,
                        w_pen=100.0, pen_margin=0.02, w_u=0.01)
    return sc, q0


def test_closed_loop_gradient_matches_central_differences():
    sc, q0 = _free_rope()
    h, H = 4, 5
    th = _theta(sc.nq, h, 3, 0.05)
    r = apg.rollout_grad(sc, q0, th, h, H)
    assert r["status"] == 0
    for t in range(H + 1):
        c = sim.grasp_offsets(sc, *sim.split_q(sc, r["traj"][t]))
        assert np.max(np.linalg.norm(c, axis=1)) < 0.1 * sc.p["r_grasp"]

    def loss(thv):
        traj, U, _, st = apg.rollout(sc, q0, thv, h, H)
        assert st == 0
        return grad.loss_and_seeds(sc, traj, U)[0]

    eps = 1e-6
    rng = np.random.default_rng(4)
    for k in list(rng.choice(th.size, 12, replace=False)) + [th.size - 1, th.size - 6]:
        e = np.zeros(th.size); e[k] = eps
        fd = (loss(th + e) - loss(th - e)) / (2 * eps)
        assert abs(fd - r["dtheta"][k]) <= 1e-6 * max(1.0, abs(fd)), k


def test_state_blind_policy_gradient_is_the_open_loop_gradient():
    """W1 = 0: the controls are the constant W2 tanh(b1) + b2, so dL/db2 is the sum over t of the
    open-loop adjoint's dL/du_t, on a rope in contact (grad.rollout_vjp, pinned elsewhere)."""
    sc = sim.Scene(*(lambda s: (s["params"], s["rest_x"]))(scenes.rope_scene(
        10, n_spheres=1, seed=5, sphere_box=((0.0, 1.0), (-0.1, 0.1), (0.0, 0.3)))))
    q0 = scenes.batch_q0(scenes.rope_scene(10, n_spheres=1, seed=5,
                                           sphere_box=((0.0, 1.0), (-0.1, 0.1), (0.0, 0.3))), 1)[0]
    h, H = 3, 4
    th = _theta(sc.nq, h, 6, 0.5)
    th[:h * sc.nq] = 0.0
    r = apg.rollout_grad(sc, q0, th, h, H)
    u0, _ = apg.policy(th, q0, h)
    ref = grad.rollout_vjp(sc, q0, np.repeat(u0[None], H, 0), "surrogate")
    assert r["status"] == 0 and ref["status"] == 0
    assert abs(r["L"] - ref["L"]) <= 1e-12 * abs(ref["L"])
    assert np.allclose(r["dtheta"][-6:], ref["dL_du"].sum(0), rtol=1e-9, atol=1e-12)
    assert np.allclose(r["dq0"], ref["dL_dq0"], rtol=1e-9, atol=1e-12)
