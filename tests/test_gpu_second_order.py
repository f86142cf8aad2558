"""The inertial variant (state [x, v, g], implicit Euler inertia, axial Rayleigh damping) on the GPU
against its FP64 oracle, oracle/second_order.py: the rope rollout and the rollout gradient of the
20-node workload, and the linearisation A_t, B_t of the 40-node workload (a 240 + 6 dimensional
state)."""
import copy

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sim as osim, second_order as so  # noqa: E402
from paper_2606_14188_b300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

ALPHA, BETA = 0.5, 0.02


def _inertial(scene):
    sc = copy.deepcopy(scene)
    sc["params"].update(second_order=True, damp_alpha=ALPHA, damp_beta=BETA)
    return sc


def _sim(scene, rb, B, H):
    from paper_2606_14188_b300.sim import Sim
    return Sim(scene, real_bytes=rb, max_batch=B, max_horizon=H)


def _t(x, rb):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float32 if rb == 4 else torch.float64,
                        device="cuda")


def _start(osc, q0, seed):
    """[x, v, g] with a small seeded initial velocity of the free nodes."""
    q2 = so.lift(osc, q0)
    rng = np.random.default_rng(seed)
    v = rng.normal(0.0, 0.05, (osc.nv, 3))
    v[list(osc.grasp)] = 0.0
    q2[osc.n:2 * osc.n] = v.ravel()
    return q2


@pytest.mark.parametrize("rb,tol", [(8, 1e-8), (4, 1e-4)])
def test_inertial_rope20_rollout_matches_the_oracle(rb, tol):
    w = scenes.workload(1, B=4)
    sc = _inertial(w["scene"])
    osc = osim.Scene(sc["params"], sc["rest_x"])
    B, H = 4, w["H"]
    Q0 = np.stack([_start(osc, w["q0"][b], 11 + b) for b in range(B)])
    s = _sim(sc, rb, B, H)
    assert s.nq == 6 * osc.nv + 6
    traj, qH, st = s.rollout(_t(Q0, rb), _t(w["U"][:B], rb))
    traj = traj.cpu().numpy()
    for b in range(B):
        ref, ost = so.rollout2(osc, Q0[b], w["U"][b], osim.HARD)
        assert ost == 0 and int(st[b]) == 0
        n = osc.n
        xs = np.max(np.abs(traj[b][:, :n] - ref[:, :n])) / np.max(np.abs(ref[:, :n]))
        vs = np.max(np.abs(traj[b][:, n:2 * n] - ref[:, n:2 * n])) / np.max(np.abs(ref[:, n:2 * n]))
        assert xs <= tol, (b, xs)
        assert vs <= 10 * tol, (b, vs)          # v = (x+ - x)/dt: position rounding over dt
        np.testing.assert_allclose(traj[b][:, 2 * n:], ref[:, 2 * n:], rtol=0, atol=10 * tol)


def test_inertial_rope40_linearize_fp64_matches_the_oracle():
    w = scenes.workload(4)
    sc = _inertial(w["scene"])
    osc = osim.Scene(sc["params"], sc["rest_x"])
    B, H = 2, 3
    V = w["U"][:B, :H]
    Z = np.stack([so.rollout2(osc, _start(osc, w["q0"][b], 5 + b), V[b], osim.HARD)[0] for b in range(B)])
    s = _sim(sc, 8, B, H)
    A, Bm, st = s.linearize(_t(Z, 8), _t(V, 8))
    assert np.all(st.cpu().numpy() == 0)
    assert A.shape[-1] == 6 * osc.nv + 6
    for b in range(B):
        Ar, Br = so.linearize2(osc, Z[b], V[b])
        Ag, Bg = A[b].cpu().numpy(), Bm[b].cpu().numpy()
        assert np.max(np.abs(Ag - Ar)) <= 1e-8 * np.max(np.abs(Ar)), b
        assert np.max(np.abs(Bg - Br)) <= 1e-8 * np.max(np.abs(Br)), b


def test_inertial_rope40_linearize_full_size_fp32_sampled():
    """The 256 x 20 linearisation workload in the inertial layout, FP32, sampled (b, t) against the
    oracle's Jacobians at the nominal states."""
    w = scenes.workload(4)
    sc = _inertial(w["scene"])
    osc = osim.Scene(sc["params"], sc["rest_x"])
    B, H = w["B"], w["H"]
    V = w["U"]
    Z = np.zeros((B, H + 1, so.nq2(osc)))
    picks = [0, 127, 255]
    for b in range(B):
        if b in picks:
            Z[b] = so.rollout2(osc, _start(osc, w["q0"][b], 100 + b), V[b], osim.HARD)[0]
        else:
            Z[b] = Z[picks[0]]                 # the other trajectories only fill the launch
    s = _sim(sc, 4, B, H)
    A, Bm, st = s.linearize(_t(Z, 4), _t(V, 4))
    assert np.count_nonzero(st.cpu().numpy()) == 0
    for b in picks:
        for t in (0, 9, H - 1):
            jac = so.SmoothStepJacobian2(osc, Z[b, t], V[b, t], x_start=Z[b, t + 1][: osc.n].reshape(osc.nv, 3))
            Ar, Br = jac.jacobians()
            Ag, Bg = A[b, t].cpu().numpy(), Bm[b, t].cpu().numpy()
            assert np.linalg.norm(Ag - Ar) <= 1e-3 * np.linalg.norm(Ar), (b, t)
            assert np.linalg.norm(Bg - Br) <= 1e-3 * np.linalg.norm(Br), (b, t)


@pytest.mark.parametrize("rb,tol_s,tol_g,cos", [(8, 1e-8, 1e-7, 1 - 1e-12), (4, 1e-4, 1e-3, 0.999)])
def test_inertial_rope20_gradient_matches_the_oracle(rb, tol_s, tol_g, cos):
    """Forward + checkpointed adjoint of the planning loss in the inertial variant (surrogate:
    nonsmooth forward, smooth step Jacobians along it), checkpoint every 3 steps (ragged last
    segment), against the oracle's rollout adjoint; also dL/dq0 (positions, velocities, grippers)."""
    w = scenes.workload(1, B=3)
    sc = _inertial(w["scene"])
    sc["params"]["checkpoint_every"] = 3
    osc = osim.Scene(sc["params"], sc["rest_x"])
    B, H = 3, w["H"]
    Q0 = np.stack([_start(osc, w["q0"][b], 21 + b) for b in range(B)])
    s = _sim(sc, rb, B, H)
    Lv, dU, dq0, st = s.rollout_vjp(_t(Q0, rb), _t(w["U"][:B], rb))
    for b in range(B):
        ref = so.rollout_vjp2(osc, Q0[b], w["U"][b], "surrogate")
        assert ref["status"] == 0 and int(st[b]) == 0
        assert abs(float(Lv[b]) - ref["L"]) <= tol_s * abs(ref["L"])
        for g, r in ((dU[b].cpu().numpy().ravel(), ref["dL_du"].ravel()),
                     (dq0[b].cpu().numpy(), ref["dL_dq0"])):
            assert np.linalg.norm(g - r) <= tol_g * np.linalg.norm(r), b
            assert g @ r >= cos * np.linalg.norm(g) * np.linalg.norm(r), b


@pytest.mark.parametrize("nv", [3, 21, 100])
def test_inertial_odd_and_long_chains_fp64(nv):
    """The inertial rollout and gradient on a three-node chain, an odd chain (a padded pair) and a
    chain of two nodes per thread, with obstacles, in FP64 against the oracle."""
    sc = _inertial(scenes.rope_scene(nv, n_spheres=2, n_boxes=1, seed=41 + nv,
                                     sphere_box=((0.0, 1.0), (-0.2, 0.2), (0.0, 0.3))))
    sc["params"]["checkpoint_every"] = 2
    osc = osim.Scene(sc["params"], sc["rest_x"])
    H = 6
    U = scenes.controls_uniform(2, H, seed=nv + 3)
    Q0 = np.stack([_start(osc, scenes.batch_q0(sc, 2)[b], 7 + b) for b in range(2)])
    s = _sim(sc, 8, 2, H)
    traj, _, st = s.rollout(_t(Q0, 8), _t(U, 8))
    Lv, dU, dq0, st2 = s.rollout_vjp(_t(Q0, 8), _t(U, 8))
    for b in range(2):
        ref, ost = so.rollout2(osc, Q0[b], U[b], osim.HARD)
        assert ost == 0 and int(st[b]) == 0 and int(st2[b]) == 0
        assert np.max(np.abs(traj[b].cpu().numpy() - ref)) <= 1e-8 * np.max(np.abs(ref))
        g = so.rollout_vjp2(osc, Q0[b], U[b], "surrogate")
        assert abs(float(Lv[b]) - g["L"]) <= 1e-8 * abs(g["L"])
        for a, r in ((dU[b].cpu().numpy().ravel(), g["dL_du"].ravel()), (dq0[b].cpu().numpy(), g["dL_dq0"])):
            assert np.linalg.norm(a - r) <= 1e-7 * np.linalg.norm(r)


def test_inertial_checkpoint_interval_does_not_change_the_adjoint():
    """Records every step, every 4 steps (ragged last segment) and a single segment give the same
    inertial gradient bit for bit: the recompute repeats the forward's steps exactly."""
    w = scenes.workload(1, B=2)
    base = _inertial(w["scene"])
    osc = osim.Scene(base["params"], base["rest_x"])
    Q0 = np.stack([_start(osc, w["q0"][b], 31 + b) for b in range(2)])
    outs = []
    for k in (1, 4, w["H"]):
        sc = copy.deepcopy(base)
        sc["params"]["checkpoint_every"] = k
        s = _sim(sc, 8, 2, w["H"])
        outs.append([x.cpu().numpy() for x in s.rollout_vjp(_t(Q0, 8), _t(w["U"][:2], 8))])
    for o in outs[1:]:
        for a, b in zip(o, outs[0]):
            assert np.array_equal(a, b)
