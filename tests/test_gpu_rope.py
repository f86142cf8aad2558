"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle on the same seeded inputs.

Tolerances: FP32 states within 1e-4 relative (max-abs error over a rollout / max |q|), FP32
gradients within 1e-3 relative (2-norm) with cosine >= 0.999; FP64 within 1e-8 relative.
A rollout whose stage 2 has no solution at some step (a node driven between obstacles whose
linearised friction cones do not meet) is flagged CS_ST_CONTACT by both sides; flags must agree,
values are compared on unflagged rollouts.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sim as osim, grad as ograd  # noqa: E402
from paper_2606_14188_b300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

TOL_STATE32, TOL_GRAD32, COS32 = 1e-4, 1e-3, 0.999
TOL64 = 1e-8


def _sim(scene, real_bytes, B, H, **kw):
    from paper_2606_14188_b300.sim import Sim
    return Sim(scene, real_bytes=real_bytes, max_batch=max(B, 1), max_horizon=H, **kw)


def _t(x, rb):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float32 if rb == 4 else torch.float64,
                        device="cuda")


def _oscene(scene):
    return osim.Scene(scene["params"], scene["rest_x"])


def rel_state(a, b):
    return np.max(np.abs(a - b)) / np.max(np.abs(b))


def check_grad(g, ref, tol, cos_min):
    g, ref = g.ravel(), ref.ravel()
    rel = np.linalg.norm(g - ref) / np.linalg.norm(ref)
    cos = g @ ref / (np.linalg.norm(g) * np.linalg.norm(ref))
    assert rel <= tol and cos >= cos_min, (rel, cos)


# ------------------------------------------------------------------------------------------
# one 20-node rope, FP64, horizon 10 (ground plane + one sphere)
# ------------------------------------------------------------------------------------------

def test_rope20_fp64_rollout_hard_and_smooth():
    w = scenes.workload(1)
    sc = w["scene"]
    osc = _oscene(sc)
    for mode in ("hard", "smooth"):
        s = _sim(sc, 8, 1, 10, fwd_mode=mode)
        traj, qH, st = s.rollout(_t(w["q0"], 8), _t(w["U"], 8))
        ref, ost, _ = osim.rollout(osc, w["q0"][0], w["U"][0], mode)
        assert int(st[0]) == 0 and ost == 0
        assert rel_state(traj[0].cpu().numpy(), ref) <= TOL64
        assert rel_state(qH[0].cpu().numpy(), ref[-1]) <= TOL64


@pytest.mark.parametrize("grad_mode", ["surrogate", "consistent"])
def test_rope20_fp64_vjp(grad_mode):
    w = scenes.workload(1)
    sc = w["scene"]
    s = _sim(sc, 8, 1, 10, grad_mode=grad_mode)
    Lv, dU, dq0, st = s.rollout_vjp(_t(w["q0"], 8), _t(w["U"], 8))
    ref = ograd.rollout_vjp(_oscene(sc), w["q0"][0], w["U"][0], grad_mode)
    assert int(st[0]) == 0
    assert abs(float(Lv[0]) - ref["L"]) <= TOL64 * abs(ref["L"])
    check_grad(dU[0].cpu().numpy(), ref["dL_du"], TOL64, 1 - 1e-12)
    check_grad(dq0[0].cpu().numpy(), ref["dL_dq0"], TOL64, 1 - 1e-12)


# ------------------------------------------------------------------------------------------
# batched 64-node rope, FP32, horizon 50, 2 spheres + 2 boxes, checkpoint every 7 steps
# ------------------------------------------------------------------------------------------

def _rope64(B):
    w = scenes.workload(2)
    return w, w["scene"], w["q0"][:B], w["U"][:B]


def test_rope64_fp32_rollout_vs_oracle():
    B = 6
    w, sc, q0, U = _rope64(B)
    s = _sim(sc, 4, B, 50)
    traj, qH, st = s.rollout(_t(q0, 4), _t(U, 4))
    traj = traj.cpu().numpy()
    osc = _oscene(sc)
    clean = 0
    for b in range(B):
        ref, ost, _ = osim.rollout(osc, q0[b], U[b], "hard")
        assert (ost != 0) == (int(st[b]) != 0), (b, ost, int(st[b]))
        if ost == 0:
            clean += 1
            assert rel_state(traj[b], ref) <= TOL_STATE32, b
    assert clean >= B // 2


def test_rope64_fp32_vjp_vs_oracle():
    B = 5
    w, sc, q0, U = _rope64(B)
    s = _sim(sc, 4, B, 50)
    Lv, dU, dq0, st = s.rollout_vjp(_t(q0, 4), _t(U, 4))
    osc = _oscene(sc)
    clean = 0
    for b in range(B):
        ref = ograd.rollout_vjp(osc, q0[b], U[b], "surrogate")
        assert (ref["status"] != 0) == (int(st[b]) != 0), (b, ref["status"], int(st[b]))
        if ref["status"] == 0:
            clean += 1
            assert abs(float(Lv[b]) - ref["L"]) <= TOL_STATE32 * abs(ref["L"])
            check_grad(dU[b].cpu().numpy(), ref["dL_du"], TOL_GRAD32, COS32)
    assert clean >= B // 2


def test_rope64_full_batch_flags_and_values_match_the_oracle():
    """The launch the benchmark times (1024 rollouts x 50 steps, FP32): on 256 of its rollouts
    (every fourth) the status flags equal the oracle's, rollout for rollout, and every rollout the
    oracle completes is within 1e-4 on its nonsmooth trajectory, within 1e-4 on L and within 1e-3
    with cosine >= 0.999 on dL/du.  A flagged rollout stops at its failing step: L NaN, gradient 0."""
    import multiprocessing as mp
    import os
    from tests import oracle_jobs
    w = scenes.workload(2)
    sc = w["scene"]
    B, H = w["B"], w["H"]
    s = _sim(sc, 4, B, H)
    q0, U = _t(w["q0"], 4), _t(w["U"], 4)
    traj, _, st_f = s.rollout(q0, U)
    Lv, dU, _, st = s.rollout_vjp(q0, U, want_dq0=False)
    traj, st_f, st = traj.cpu().numpy(), st_f.cpu().numpy(), st.cpu().numpy()
    Lv, dU = Lv.cpu().numpy(), dU.cpu().numpy()
    fl = st != 0
    assert np.all(np.isnan(Lv[fl])) and np.all(dU[fl] == 0)
    assert np.all(np.isfinite(Lv[~fl])) and np.all(np.isfinite(dU[~fl]))
    idx = list(range(0, B, 4))
    with oracle_jobs.pool(max(1, min(os.cpu_count() or 1, 32))) as pool:
        refs = pool.map(oracle_jobs.rope64_rollout, idx)
    clean = 0
    for r in refs:
        b = r["b"]
        assert (int(st[b]) != 0) == (r["status"] != 0), (b, int(st[b]), r["status"])
        assert (int(st_f[b]) != 0) == (r["status_fwd"] != 0), (b, int(st_f[b]), r["status_fwd"])
        if r["status"] == 0:
            clean += 1
            assert rel_state(traj[b], r["traj"]) <= TOL_STATE32, b
            assert abs(float(Lv[b]) - r["L"]) <= TOL_STATE32 * abs(r["L"]), b
            check_grad(dU[b], r["dL_du"], TOL_GRAD32, COS32)
    assert clean >= len(idx) * 9 // 10


def test_rope64_two_part_launch_equals_one_launch():
    """1024 rollouts are more than the device holds at once, so the call runs the forward parts,
    orders the rollouts by their measured cost and runs the backward parts costliest first; 128
    of them (fewer than the device holds) run as one launch.  Each rollout's outputs must be
    bit-identical."""
    w = scenes.workload(2)
    sc = w["scene"]
    B, H = w["B"], w["H"]
    idx = np.r_[0:64, B - 64:B]
    big = _sim(sc, 4, B, H).rollout_vjp(_t(w["q0"], 4), _t(w["U"], 4))
    small = _sim(sc, 4, len(idx), H).rollout_vjp(_t(w["q0"][idx], 4), _t(w["U"][idx], 4))
    for a, b in zip(big, small):
        a = a[torch.as_tensor(idx, device=a.device)]
        assert torch.equal(a.isnan(), b.isnan()) and torch.equal(a.nan_to_num(), b.nan_to_num())


def test_rope64_checkpoint_interval_does_not_change_the_adjoint():
    """The recomputed segment steps reproduce the forward's steps exactly, so the adjoint with a
    record at every step (k = 1, no recompute) and with the interval sim_create picks (k = 0)
    equals the one with k = 7, bit for bit."""
    import copy
    B = 8
    w, sc, q0, U = _rope64(B)
    sc1 = copy.deepcopy(sc)
    sc1["params"]["checkpoint_every"] = 1
    sc0 = copy.deepcopy(sc)
    sc0["params"]["checkpoint_every"] = 0          # picked by sim_create from the free memory
    a = _sim(sc, 4, B, 50).rollout_vjp(_t(q0, 4), _t(U, 4))
    b = _sim(sc1, 4, B, 50).rollout_vjp(_t(q0, 4), _t(U, 4))
    c = _sim(sc0, 4, B, 50).rollout_vjp(_t(q0, 4), _t(U, 4))
    assert sc["params"]["checkpoint_every"] == 7
    for x, y, z in zip(a, b, c):
        assert torch.equal(x.isnan(), y.isnan()) and torch.equal(x.nan_to_num(), y.nan_to_num())
        assert torch.equal(x.isnan(), z.isnan()) and torch.equal(x.nan_to_num(), z.nan_to_num())


def test_rope64_deterministic():
    B = 32
    w, sc, q0, U = _rope64(B)
    s = _sim(sc, 4, B, 50)
    a = s.rollout_vjp(_t(q0, 4), _t(U, 4))
    b = s.rollout_vjp(_t(q0, 4), _t(U, 4))
    for x, y in zip(a, b):
        assert torch.equal(x.isnan(), y.isnan()) and torch.equal(x.nan_to_num(), y.nan_to_num())


# ------------------------------------------------------------------------------------------
# linearisation, 40-node rope
# ------------------------------------------------------------------------------------------

def test_rope40_linearize_vs_oracle():
    w = scenes.workload(4)
    sc = w["scene"]
    B, H = 2, 3
    osc = _oscene(sc)
    Z = np.zeros((B, H + 1, osc.nq))
    V = w["U"][:B, :H]
    for b in range(B):
        Z[b], _, _ = osim.rollout(osc, w["q0"][b], V[b], "hard")
    s = _sim(sc, 4, B, H)
    A, Bm, st = s.linearize(_t(Z, 4), _t(V, 4))
    A, Bm = A.cpu().numpy(), Bm.cpu().numpy()
    assert np.all(st.cpu().numpy() == 0)
    for b in range(B):
        Ar, Br = ograd.linearize(osc, Z[b], V[b])
        for t in range(H):
            assert np.linalg.norm(A[b, t] - Ar[t]) <= 1e-3 * np.linalg.norm(Ar[t])
            assert np.linalg.norm(Bm[b, t] - Br[t]) <= 1e-3 * np.linalg.norm(Br[t])


def test_rope40_fp32_rollout_and_vjp_vs_oracle():
    """FP32 with a partly filled warp (20 node pairs on 32 lanes)."""
    w = scenes.workload(4)
    sc, H = w["scene"], w["H"]
    B = 4
    osc = _oscene(sc)
    s = _sim(sc, 4, B, H)
    q0, U = _t(w["q0"][:B], 4), _t(w["U"][:B], 4)
    traj, _, st = s.rollout(q0, U)
    Lv, dU, _, st2 = s.rollout_vjp(q0, U)
    assert np.all(st.cpu().numpy() == 0) and np.all(st2.cpu().numpy() == 0)
    for b in range(B):
        ref, ost, _ = osim.rollout(osc, w["q0"][b], w["U"][b], "hard")
        assert ost == 0
        assert rel_state(traj[b].cpu().numpy(), ref) <= TOL_STATE32, b
        g = ograd.rollout_vjp(osc, w["q0"][b], w["U"][b], "surrogate")
        assert abs(float(Lv[b]) - g["L"]) <= TOL_STATE32 * abs(g["L"])
        check_grad(dU[b].cpu().numpy(), g["dL_du"], TOL_GRAD32, COS32)


def test_rope40_linearize_full_size_sampled():
    """The launch the benchmark times (256 nominal trajectories x horizon 20, 40-node rope, the
    nominal states rolled out by the oracle), sampled: A_t, B_t at 12 (b, t) against the oracle."""
    w = scenes.workload(4)
    sc, B, H = w["scene"], w["B"], w["H"]
    osc = _oscene(sc)
    V = w["U"]
    Z = np.stack([osim.rollout(osc, w["q0"][b], V[b], "hard")[0] for b in range(B)])
    picks = [0, 85, 170, 255]
    s = _sim(sc, 4, B, H)
    A, Bm, st = s.linearize(_t(Z, 4), _t(V, 4))
    st = st.cpu().numpy()
    assert np.count_nonzero(st) == 0
    for b in picks:
        for t in (0, 7, H - 1):
            xs0 = Z[b, t + 1][: osc.n].reshape(osc.nv, 3)
            Ar, Br = ograd.SmoothStepJacobian(osc, Z[b, t], V[b, t], x_start=xs0).jacobians()
            Ag, Bg = A[b, t].cpu().numpy(), Bm[b, t].cpu().numpy()
            assert np.linalg.norm(Ag - Ar) <= 1e-3 * np.linalg.norm(Ar), (b, t)
            assert np.linalg.norm(Bg - Br) <= 1e-3 * np.linalg.norm(Br), (b, t)


def test_rope20_fp64_linearize_vs_oracle():
    w = scenes.workload(1)
    sc = w["scene"]
    osc = _oscene(sc)
    H = 10
    Z, _, _ = osim.rollout(osc, w["q0"][0], w["U"][0], "hard")
    s = _sim(sc, 8, 1, H)
    A, Bm, st = s.linearize(_t(Z[None], 8), _t(w["U"], 8))
    Ar, Br = ograd.linearize(osc, Z, w["U"][0])
    assert int(st[0]) == 0
    assert np.max(np.abs(A[0].cpu().numpy() - Ar)) <= TOL64 * np.max(np.abs(Ar))
    assert np.max(np.abs(Bm[0].cpu().numpy() - Br)) <= TOL64 * np.max(np.abs(Br))


@pytest.mark.parametrize("nv", [3, 21, 64, 100])
def test_linearize_odd_and_long_chains_fp64(nv):
    """A_t, B_t in FP64 against the oracle's forward-mode Jacobians: a three-node chain, an odd chain
    (a padded pair), one node per thread and two (several passes of the tangent directions), with
    the nominal lowered onto the obstacles so that some steps have active contacts."""
    sc = scenes.rope_scene(nv, n_spheres=2, n_boxes=1, seed=29 + nv,
                           sphere_box=((0.0, 1.0), (-0.2, 0.2), (0.0, 0.3)))
    H = 5
    U = scenes.controls_uniform(2, H, seed=nv + 1)
    U[..., 2] = -0.03                              # both grippers move down
    U[..., 5] = -0.03
    q0 = scenes.batch_q0(sc, 2)
    osc = _oscene(sc)
    Z = np.stack([osim.rollout(osc, q0[b], U[b], "hard")[0] for b in range(2)])
    s = _sim(sc, 8, 2, H)
    A, Bm, st = s.linearize(_t(Z, 8), _t(U, 8))
    assert np.all(st.cpu().numpy() == 0)
    for b in range(2):
        Ar, Br = ograd.linearize(osc, Z[b], U[b])
        Ag, Bg = A[b].cpu().numpy(), Bm[b].cpu().numpy()
        assert np.max(np.abs(Ag - Ar)) <= TOL64 * np.max(np.abs(Ar)), b
        assert np.max(np.abs(Bg - Br)) <= TOL64 * np.max(np.abs(Br)), b


# ------------------------------------------------------------------------------------------
# edge cases
# ------------------------------------------------------------------------------------------

@pytest.mark.parametrize("nv", [2, 3, 21, 33, 100])
def test_odd_and_small_chains_fp64(nv):
    """Chains whose pair count is not a power of two, odd chains (a padded dummy node), the
    two-node chain and a chain longer than one pair per lane."""
    sc = scenes.rope_scene(nv, n_spheres=1, n_boxes=1, seed=17 + nv)
    H = 4
    U = scenes.controls_uniform(2, H, seed=nv)
    q0 = scenes.batch_q0(sc, 2)
    s = _sim(sc, 8, 2, H)
    traj, _, st = s.rollout(_t(q0, 8), _t(U, 8))
    osc = _oscene(sc)
    for b in range(2):
        ref, ost, _ = osim.rollout(osc, q0[b], U[b], "hard")
        assert int(st[b]) == ost == 0
        assert rel_state(traj[b].cpu().numpy(), ref) <= TOL64
    Lv, dU, _, st = s.rollout_vjp(_t(q0, 8), _t(U, 8))
    ref = ograd.rollout_vjp(osc, q0[1], U[1], "surrogate")
    check_grad(dU[1].cpu().numpy(), ref["dL_du"], TOL64, 1 - 1e-12)


def test_ragged_checkpoint_segments_and_no_obstacles():
    sc = scenes.rope_scene(16, n_spheres=1, seed=5)
    H = 10
    U = scenes.controls_uniform(3, H, seed=3)
    q0 = scenes.batch_q0(sc, 3)
    osc = _oscene(sc)
    ref = ograd.rollout_vjp(osc, q0[2], U[2], "surrogate")
    for k in (1, 3, 4, 10, 13):
        sc["params"]["checkpoint_every"] = k
        s = _sim(sc, 8, 3, H)
        _, dU, dq0, st = s.rollout_vjp(_t(q0, 8), _t(U, 8))
        check_grad(dU[2].cpu().numpy(), ref["dL_du"], TOL64, 1 - 1e-12)
    sc2 = scenes.rope_scene(16, n_spheres=0, seed=5)
    sc2["params"]["obstacles"] = []
    s = _sim(sc2, 8, 3, H)
    _, dU, _, st = s.rollout_vjp(_t(q0, 8), _t(U, 8))
    ref = ograd.rollout_vjp(_oscene(sc2), q0[0], U[0], "surrogate")
    check_grad(dU[0].cpu().numpy(), ref["dL_du"], TOL64, 1 - 1e-12)


def test_dL_dtraj_seeds_and_autograd():
    """The autograd layer's backward equals sim_rollout_vjp with the same dL/dtraj seeds, which
    equals the oracle's adjoint with those seeds."""
    from paper_2606_14188_b300.sim import RolloutFn
    sc = scenes.rope_scene(12, n_spheres=1, seed=9)
    H = 6
    U = scenes.controls_uniform(2, H, seed=2)
    q0 = scenes.batch_q0(sc, 2)
    s = _sim(sc, 8, 2, H)
    rng = np.random.default_rng(0)
    Wt = rng.normal(size=(2, H + 1, s.nq))
    qt = _t(q0, 8).requires_grad_(True)
    Ut = _t(U, 8).requires_grad_(True)
    traj, _ = RolloutFn.apply(qt, Ut, s)
    (traj * _t(Wt, 8)).sum().backward()
    ref = ograd.rollout_vjp(_oscene(sc), q0[1], U[1], "surrogate", dL_dtraj=Wt[1])
    check_grad(Ut.grad[1].cpu().numpy(), ref["dL_du"], TOL64, 1 - 1e-12)
    check_grad(qt.grad[1].cpu().numpy(), ref["dL_dq0"], TOL64, 1 - 1e-12)


def test_argument_errors_and_empty_batch():
    from paper_2606_14188_b300._lib import CordsimError
    sc = scenes.rope_scene(8, seed=1)
    s = _sim(sc, 4, 4, 5)
    q0 = _t(scenes.batch_q0(sc, 5), 4)
    U = _t(np.zeros((5, 5, 6)), 4)
    with pytest.raises(CordsimError) as e:
        s.rollout(q0, U)                     # B = 5 > max_batch = 4
    assert e.value.code == 1
    with pytest.raises(CordsimError):
        s.rollout(_t(scenes.batch_q0(sc, 1), 4), _t(np.zeros((1, 6, 6)), 4))   # H > max_horizon
    traj, qH, st = s.rollout(_t(np.zeros((0, s.nq)), 4), _t(np.zeros((0, 5, 6)), 4))
    assert qH.shape == (0, s.nq)


@pytest.mark.parametrize("rb", [4, 8])
def test_saddle_root_flagged_like_the_oracle(rb):
    """A straight chain compressed past Euler buckling, symmetric about its axis: the only root
    stage 1 can reach is a saddle of the potential, which the iteration does not accept (it
    accepts only exact-Hessian steps, i.e. minimisers), so both sides flag the step's stage 1
    (CS_ST_NEWTON at the cap; the oracle's adjoint adds CS_ST_NOTPD for the undefined step
    Jacobian) and the GPU's L is NaN, its gradients 0."""
    p = scenes.default_params("rope")
    L0 = 0.4
    X0 = np.array([[0.0, 0.0, 1.0], [L0, 0.0, 1.0], [2 * L0, 0.0, 1.0]])
    p.update(n_nodes=3, node_mass=1e-3, k_stretch=500.0, k_bend=0.0, gravity=(0, 0, 0),
             obstacles=[], grasp_nodes=(0, 2), grad_mode="consistent", fwd_mode="smooth")
    sc = dict(params=p, rest_x=X0)
    q0 = np.concatenate([X0.ravel(), X0[0], X0[2]])[None]
    u = np.array([[[0.02, 0.0, 0.0, -0.02, 0.0, 0.0]]])
    ref = ograd.rollout_vjp(_oscene(sc), q0[0], u[0], "consistent")
    s = _sim(sc, rb, 1, 1)
    Lv, dU, _, st = s.rollout_vjp(_t(q0, rb), _t(u, rb))
    assert ref["status"] & osim.ST_NEWTON and int(st[0]) & osim.ST_NEWTON
    assert ref["status"] & osim.ST_NOTPD
    assert np.isnan(float(Lv[0])) and float(dU.abs().max()) == 0.0


def test_rope100_fp32_two_pairs_per_lane_vs_oracle():
    """FP32 with two node pairs per lane (100 nodes): rollout and adjoint against the oracle."""
    sc = scenes.rope_scene(100, n_spheres=1, n_boxes=1, seed=17,
                           sphere_box=((0.0, 1.0), (-0.2, 0.2), (0.0, 0.3)))
    sc["params"]["checkpoint_every"] = 3
    B, H = 3, 10
    U = scenes.controls_normal_clear(sc, B, H, seed=17)
    q0 = scenes.batch_q0(sc, B)
    osc = _oscene(sc)
    s = _sim(sc, 4, B, H)
    traj, _, st = s.rollout(_t(q0, 4), _t(U, 4))
    Lv, dU, _, st2 = s.rollout_vjp(_t(q0, 4), _t(U, 4))
    for b in range(B):
        ref, ost, _ = osim.rollout(osc, q0[b], U[b], "hard")
        g = ograd.rollout_vjp(osc, q0[b], U[b], "surrogate")
        assert (ost != 0) == (int(st[b]) != 0) and (g["status"] != 0) == (int(st2[b]) != 0)
        if ost == 0 and g["status"] == 0:
            assert rel_state(traj[b].cpu().numpy(), ref) <= TOL_STATE32, b
            assert abs(float(Lv[b]) - g["L"]) <= TOL_STATE32 * abs(g["L"])
            check_grad(dU[b].cpu().numpy(), g["dL_du"], TOL_GRAD32, COS32)


def test_rope64_fp64_two_part_launch_equals_one_launch():
    """FP64 (about two one-warp CTAs per SM): 320 rollouts take the two-part launch; rollouts
    from both ends equal the same rollouts run alone, bit for bit."""
    w = scenes.workload(2)
    sc = w["scene"]
    B, H = 320, 12
    idx = np.r_[0:4, B - 4:B]
    q0, U = w["q0"][:B], w["U"][:B, :H]
    big = _sim(sc, 8, B, H).rollout_vjp(_t(q0, 8), _t(U, 8))
    small = _sim(sc, 8, len(idx), H).rollout_vjp(_t(q0[idx], 8), _t(U[idx], 8))
    for a, b in zip(big, small):
        a = a[torch.as_tensor(idx, device=a.device)]
        assert torch.equal(a.isnan(), b.isnan()) and torch.equal(a.nan_to_num(), b.nan_to_num())
