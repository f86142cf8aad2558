"""The output-feedback SLS observer stage on the GPU (sls_observer, sls_response, sls_closed_loop;
paper Sec. 4.2) against its FP64 oracle, oracle/sls.py, element by element: dense random systems
whose sizes span several 64-wide tiles with ragged tails, the 40-node rope's own Jacobians (the
oracle's linearisation of the 256 x 20 workload, state 126, 120 observed node coordinates), and
the full 256-trajectory launch sampled; plus the affine constraints of eq. phi_equation, which
hold at any size.

FP32 tolerances (relative, max over a trajectory's entries against the largest entry): 1e-4 on
the covariances Pi (state-like), 1e-3 on the gains and the responses (derivative-like: each is a
product of up to N closed-loop matrices, or a solve with the innovation matrix, whose condition
number multiplies the rounding of the covariance it is formed from)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import grad as ograd, sim as osim, sls, tubes  # noqa: E402
from paper_2606_14188_b300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {8: dict(pi=1e-10, gain=1e-9, phi=1e-9), 4: dict(pi=1e-4, gain=1e-3, phi=1e-3)}


def _g():
    from paper_2606_14188_b300 import sls as gsls
    return gsls


def _t(x, rb):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float32 if rb == 4 else torch.float64,
                        device="cuda")


def _rel(g, r):
    return float(np.max(np.abs(g - r)) / max(np.max(np.abs(r)), 1e-300))


def _oracle(sys_b):
    A, C, E, F, Xi = (sys_b[k] for k in ("A", "C", "E", "F", "Xi"))
    Pi, L = sls.kalman_recursion(A, C, E, F, Xi)
    PX, PY = sls.observer_responses(A, C, L)
    return Pi, L, PX, PY


def _check_observer(gout, sysd, picks, rb, N):
    gsls = _g()
    Pi, Lg, PX, PY, st = gout
    assert np.all(st.cpu().numpy() == 0)
    tol = TOL[rb]
    PXd, PYd = gsls.unpack(PX, N).cpu().numpy(), gsls.unpack(PY, N).cpu().numpy()
    errs = []
    for i, b in enumerate(picks):
        ref = _oracle({k: v[b] for k, v in sysd.items()})
        e = (_rel(Pi[i].cpu().numpy(), ref[0]), _rel(Lg[i].cpu().numpy(), ref[1]),
             _rel(PXd[i], ref[2]), _rel(PYd[i], ref[3]))
        errs.append(e)
        assert e[0] <= tol["pi"], (b, e)
        assert e[1] <= tol["gain"], (b, e)
        assert e[2] <= tol["phi"] and e[3] <= tol["phi"], (b, e)
    return errs


@pytest.mark.parametrize("rb", [8, 4])
@pytest.mark.parametrize("B,N,n,p,nw,ne,n0", [(3, 5, 12, 8, 10, 6, 12), (2, 4, 70, 65, 33, 65, 70),
                                              (1, 1, 1, 1, 1, 1, 1), (2, 3, 130, 3, 130, 3, 5)])
def test_observer_matches_the_oracle_on_random_systems(rb, B, N, n, p, nw, ne, n0):
    sysd = scenes.sls_random_system(B, N, n, p, nw, ne, n0, seed=7 * n + p)
    out = _g().observer(*(_t(sysd[k], rb) for k in ("A", "C", "E", "F", "Xi")))
    _check_observer(out, sysd, range(B), rb, N)


def _rope_inputs(B_or, H, seed=11):
    """The oracle's Jacobians A_t of the 40-node rope workload along B_or hard nominal rollouts and
    the seeded observation model of the node positions."""
    w = scenes.workload(4)
    osc = osim.Scene(w["scene"]["params"], w["scene"]["rest_x"])
    A = np.zeros((B_or, H, osc.n + 6, osc.n + 6))
    Bm = np.zeros((B_or, H, osc.n + 6, 6))
    for b in range(B_or):
        Z = osim.rollout(osc, w["q0"][b], w["U"][b, :H], "hard")[0]
        A[b], Bm[b] = ograd.linearize(osc, Z, w["U"][b, :H])
    obs = scenes.sls_observation_model(B_or, H, osc.nv, seed=seed)
    return dict(A=A, **obs), Bm


@pytest.mark.parametrize("rb", [8, 4])
def test_observer_on_rope40_jacobians(rb):
    sysd, _ = _rope_inputs(2, 20)
    out = _g().observer(*(_t(sysd[k], rb) for k in ("A", "C", "E", "F", "Xi")))
    errs = _check_observer(out, sysd, range(2), rb, 20)
    print("rope40 observer errors (Pi, L, PhiX, PhiY):", errs)


def _feedback_responses(A, Bm, K):
    return sls.state_feedback_responses(A, Bm, K)


@pytest.mark.parametrize("rb", [8, 4])
def test_response_matches_the_state_feedback_responses(rb):
    B, N, n, m = 2, 6, 70, 6
    sysd = scenes.sls_random_system(B, N, n, 3, 3, 3, 3, seed=5)
    rng = np.random.default_rng(6)
    Bm = rng.normal(size=(B, N, n, m)) / np.sqrt(n)
    K = scenes.sls_feedback_gains(B, N, m, n, seed=7)
    Acl = np.einsum("bjik,bjkl->bjil", Bm, K[:, :N]) + sysd["A"]
    Phi = _g().unpack(_g().response(_t(Acl, rb)), N).cpu().numpy()
    for b in range(B):
        ref, _ = _feedback_responses(sysd["A"][b], Bm[b], K[b])
        assert _rel(Phi[b], ref) <= TOL[rb]["phi"]


def _closed_loop_case(sysd, Bm, K, rb, picks_oracle, N):
    gsls = _g()
    A = _t(sysd["A"], rb)
    Pi, Lg, PX, PY, st = gsls.observer(A, *(_t(sysd[k], rb) for k in ("C", "E", "F", "Xi")))
    n, m = sysd["A"].shape[2], Bm.shape[3]
    PBX = np.zeros((len(picks_oracle), (N + 1) * n, (N + 1) * n))
    PBU = np.zeros((len(picks_oracle), (N + 1) * m, (N + 1) * n))
    for i, b in enumerate(picks_oracle):
        PBX[i], PBU[i] = _feedback_responses(sysd["A"][b], Bm[b], K[b])
    PBXg = gsls.pack(_t(PBX, rb), N, n, n)
    PBUg = gsls.pack(_t(PBU, rb), N, m, n)
    return gsls.closed_loop(A, PBXg, PBUg, PX, PY), (PBX, PBU)


@pytest.mark.parametrize("rb", [8, 4])
def test_closed_loop_maps_match_the_oracle_and_satisfy_the_constraints(rb):
    B, N, n, p, m = 2, 5, 70, 65, 6
    sysd = scenes.sls_random_system(B, N, n, p, n, p, n, seed=13)
    rng = np.random.default_rng(14)
    Bm = rng.normal(size=(B, N, n, m)) / np.sqrt(n)
    K = scenes.sls_feedback_gains(B, N, m, n, scale=0.3, seed=15)
    (XW, UW, XE, UE), (PBX, PBU) = _closed_loop_case(sysd, Bm, K, rb, range(B), N)
    gsls = _g()
    got = [gsls.unpack(x, N).cpu().numpy() for x in (XW, UW, XE, UE)]
    I = np.eye((N + 1) * n)
    for b in range(B):
        Ab, Cb = sysd["A"][b], sysd["C"][b]
        Pi, L = sls.kalman_recursion(Ab, Cb, sysd["E"][b], sysd["F"][b], sysd["Xi"][b])
        PX, PY = sls.observer_responses(Ab, Cb, L)
        ref = sls.closed_loop_maps(Ab, PBX[b], PBU[b], PX, PY)
        for g, r in zip(got, ref):
            assert _rel(g[b], r) <= TOL[rb]["phi"], b
        # eq. phi_equation on the GPU's maps (residuals relative to the identity blocks)
        M = I - sls.downshift(Ab, n, n)
        ZB, ZC = sls.downshift(Bm[b], n, m), sls.downshift(Cb, p, n)
        Phi = np.block([[got[0][b], got[2][b]], [got[1][b], got[3][b]]])
        left = np.hstack([M, -ZB]) @ Phi
        right = Phi @ np.vstack([M, -ZC])
        tol = 1e-9 if rb == 8 else 1e-3
        assert np.max(np.abs(left - np.hstack([I, np.zeros(((N + 1) * n, (N + 1) * p))]))) <= tol
        assert np.max(np.abs(right - np.vstack([I, np.zeros(((N + 1) * m, (N + 1) * n))]))) <= tol


def test_full_size_observer_and_closed_loop_fp32_sampled():
    """The 256-trajectory x 20-step, 126-state launch the benchmark times (FP32): the rope's own
    Jacobians on three sampled trajectories (the others repeat trajectory 0 to fill the launch),
    the observer, the closed-loop maps and the reachable tubes of those three compared with the
    oracle."""
    B, H = 256, 20
    picks = [0, 127, 255]
    sys3, Bm3 = _rope_inputs(3, H, seed=21)
    full = {k: np.repeat(v[:1], B, axis=0) for k, v in sys3.items()}
    Bm = np.repeat(Bm3[:1], B, axis=0)
    for i, b in enumerate(picks):
        for k in full:
            full[k][b] = sys3[k][i]
        Bm[b] = Bm3[i]
    n, m, p = 126, 6, 120
    K = scenes.sls_feedback_gains(B, H, m, n, seed=22)
    gsls = _g()
    A = _t(full["A"], 4)
    out = gsls.observer(A, *(_t(full[k], 4) for k in ("C", "E", "F", "Xi")))
    assert int(torch.count_nonzero(out[4])) == 0
    sub = [o[picks] for o in out]
    _check_observer(sub, {k: v[picks] for k, v in full.items()}, range(3), 4, H)
    # state-feedback responses of every trajectory on the GPU (an input here), the three sampled
    # ones checked against the oracle's
    Acl = torch.einsum("bjik,bjkl->bjil", _t(Bm, 4), _t(K[:, :H], 4)) + A
    PBX = gsls.response(Acl.contiguous())
    Kt = _t(K, 4)
    T = gsls.n_blocks(H)
    kidx = torch.tensor([k for k in range(H + 1) for _ in range(k + 1)], device="cuda")
    PBU = torch.einsum("btmn,btnc->btmc", Kt[:, kidx], PBX).contiguous()
    XW, UW, XE, UE = gsls.closed_loop(A, PBX, PBU, out[2], out[3])
    tau, _ = gsls.tubes(XW, UW, XE, UE, _t(full["E"], 4), _t(full["F"], 4))
    for i, b in enumerate(picks):
        PBXr, PBUr = _feedback_responses(full["A"][b], Bm[b], K[b])
        assert _rel(gsls.unpack(PBX[b:b + 1], H)[0].cpu().numpy(), PBXr) <= 1e-3
        Pi, L = sls.kalman_recursion(*(full[k][b] for k in ("A", "C", "E", "F", "Xi")))
        PX, PY = sls.observer_responses(full["A"][b], full["C"][b], L)
        ref = sls.closed_loop_maps(full["A"][b], PBXr, PBUr, PX, PY)
        for g, r in zip((XW, UW, XE, UE), ref):
            assert _rel(gsls.unpack(g[b:b + 1], H)[0].cpu().numpy(), r) <= 1e-3, b
        tref = tubes.tube_widths(*ref, full["E"][b], full["F"][b], H)
        assert _rel(tau[b].cpu().numpy(), tref) <= 1e-3, b
    assert T == 231


def test_not_positive_definite_innovation_is_flagged():
    """F_j = 0 with C_j = 0 at one step makes the innovation matrix zero: that trajectory is
    flagged CS_ST_NOTPD and its gains from that step on are NaN; the other trajectory is
    unaffected."""
    B, N, n, p = 2, 4, 10, 4
    sysd = scenes.sls_random_system(B, N, n, p, n, p, n, seed=31)
    sysd["F"][1, 2] = 0.0
    sysd["C"][1, 2] = 0.0
    out = _g().observer(*(_t(sysd[k], 8) for k in ("A", "C", "E", "F", "Xi")))
    st = out[4].cpu().numpy()
    assert st[0] == 0 and st[1] & 8
    L = out[1].cpu().numpy()
    assert np.all(np.isnan(L[1, 2]))
    assert np.all(np.isfinite(L[1, :2]))
    ref = _oracle({k: v[0] for k, v in sysd.items()})
    assert _rel(L[0], ref[1]) <= 1e-9


def test_empty_batch_is_a_no_op():
    sysd = scenes.sls_random_system(1, 2, 4, 2, 4, 2, 4)
    out = _g().observer(*(_t(sysd[k][:0], 8) for k in ("A", "C", "E", "F", "Xi")))
    assert out[0].shape == (0, 3, 4, 4)


@pytest.mark.parametrize("rb,p", [(4, 221), (8, 155)])
def test_observer_at_the_largest_innovation_the_gain_solve_holds(rb, p):
    """p at the gain kernel's shared-memory limit (221 in FP32, 155 in FP64: one right-hand side
    per pass), a state larger than it, against the oracle."""
    B, N, n = 1, 2, p + 9
    sysd = scenes.sls_random_system(B, N, n, p, n, p, n, seed=p)
    out = _g().observer(*(_t(sysd[k], rb) for k in ("A", "C", "E", "F", "Xi")))
    _check_observer(out, sysd, range(B), rb, N)


def test_observer_and_tubes_in_the_inertial_state():
    """The 246-dimensional inertial rope state (positions and velocities of 40 nodes, grippers)
    with the 120 node positions observed, FP32, against the oracle; the tubes' process scaling
    spans three 128-wide column tiles (nw = 300)."""
    from oracle import tubes as otubes
    B, N, n, p, m, nw = 2, 4, 246, 120, 6, 300
    sysd = scenes.sls_random_system(B, N, n, p, nw, p, n, seed=81)
    gsls = _g()
    A = _t(sysd["A"], 4)
    out = gsls.observer(A, *(_t(sysd[k], 4) for k in ("C", "E", "F", "Xi")))
    _check_observer(out, sysd, range(B), 4, N)
    rng = np.random.default_rng(82)
    Bm = rng.normal(size=(B, N, n, m)) / np.sqrt(n)
    K = scenes.sls_feedback_gains(B, N, m, n, seed=83)
    PB = [sls.state_feedback_responses(sysd["A"][b], Bm[b], K[b]) for b in range(B)]
    maps = gsls.closed_loop(A, gsls.pack(_t(np.stack([q[0] for q in PB]), 4), N, n, n),
                            gsls.pack(_t(np.stack([q[1] for q in PB]), 4), N, m, n), out[2], out[3])
    tau, _ = gsls.tubes(*maps, _t(sysd["E"], 4), _t(sysd["F"], 4))
    for b in range(B):
        Pi, L = sls.kalman_recursion(*(sysd[k][b] for k in ("A", "C", "E", "F", "Xi")))
        PX, PY = sls.observer_responses(sysd["A"][b], sysd["C"][b], L)
        ref = sls.closed_loop_maps(sysd["A"][b], PB[b][0], PB[b][1], PX, PY)
        for g, r in zip(maps, ref):
            assert _rel(gsls.unpack(g[b:b + 1], N)[0].cpu().numpy(), r) <= 1e-3, b
        tref = otubes.tube_widths(*ref, sysd["E"][b], sysd["F"][b], N)
        assert _rel(tau[b].cpu().numpy(), tref) <= 1e-3, b


@pytest.mark.parametrize("rb", [8, 4])
@pytest.mark.parametrize("B,N,n,p", [(3, 5, 12, 8), (2, 9, 70, 65), (1, 1, 1, 1)])
def test_kalman_scan_matches_the_recursion(rb, B, N, n, p):
    """The covariances by the GPU's associative scan (eq. combination_rules) against the oracle's
    step-by-step recursion: several levels, a horizon that is not a power of two, 1 x 1."""
    sysd = scenes.sls_random_system(B, N, n, p, n, p, n, seed=3 * n + N)
    Pi, st = _g().kalman_scan(*(_t(sysd[k], rb) for k in ("A", "C", "E", "F", "Xi")))
    assert np.all(st.cpu().numpy() == 0)
    for b in range(B):
        ref, _ = sls.kalman_recursion(*(sysd[k][b] for k in ("A", "C", "E", "F", "Xi")))
        assert _rel(Pi[b].cpu().numpy(), ref) <= TOL[rb]["pi"], b


@pytest.mark.parametrize("rb", [8, 4])
def test_kalman_scan_on_rope40_jacobians(rb):
    sysd, _ = _rope_inputs(2, 20)
    Pi, st = _g().kalman_scan(*(_t(sysd[k], rb) for k in ("A", "C", "E", "F", "Xi")))
    assert np.all(st.cpu().numpy() == 0)
    for b in range(2):
        ref, _ = sls.kalman_recursion(*(sysd[k][b] for k in ("A", "C", "E", "F", "Xi")))
        e = _rel(Pi[b].cpu().numpy(), ref)
        print("rope40 scan Pi error", rb, e)
        assert e <= TOL[rb]["pi"], b


def test_kalman_scan_flags_a_singular_observation_noise():
    """F_j = 0 at one step of trajectory 1: its scan element needs (F_j F_j^T)^{-1}, the trajectory
    is flagged CS_ST_NOTPD; trajectory 0 is unaffected."""
    B, N, n, p = 2, 4, 10, 4
    sysd = scenes.sls_random_system(B, N, n, p, n, p, n, seed=33)
    sysd["F"][1, 2] = 0.0
    Pi, st = _g().kalman_scan(*(_t(sysd[k], 8) for k in ("A", "C", "E", "F", "Xi")))
    s = st.cpu().numpy()
    assert s[0] == 0 and s[1] & 8
    ref, _ = sls.kalman_recursion(*(sysd[k][0] for k in ("A", "C", "E", "F", "Xi")))
    assert _rel(Pi[0].cpu().numpy(), ref) <= 1e-10
