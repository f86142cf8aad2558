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
