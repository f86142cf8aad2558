"""Reachable tubes, constraint margins and the conformal radius on the GPU (sls_tubes,
sls_conformal_radius; paper Sec. 4.2 eq. of_optimization_tightening1/2, Sec. 4.4) against
oracle/tubes.py on the oracle's closed-loop maps of the same inputs: random systems whose
disturbance scalings span two column tiles, FP64 and FP32; the radius at several miscoverage
levels, at one sample and at the largest calibration set, with a NaN score."""
import math

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle import sls, tubes  # noqa: E402
from paper_2606_14188_b300 import scenes  # noqa: E402

pytestmark = pytest.mark.gpu

TOL = {8: 1e-9, 4: 1e-3}


def _t(x, rb):
    return torch.tensor(np.ascontiguousarray(x), dtype=torch.float32 if rb == 4 else torch.float64,
                        device="cuda")


def _rel(g, r):
    return float(np.max(np.abs(g - r)) / max(np.max(np.abs(r)), 1e-300))


def _case(B, N, n, p, m, nw, ne, seed):
    sysd = scenes.sls_random_system(B, N, n, p, nw, ne, n, seed=seed)
    rng = np.random.default_rng(seed + 1)
    Bm = rng.normal(size=(B, N, n, m)) / np.sqrt(n)
    K = scenes.sls_feedback_gains(B, N, m, n, scale=0.3, seed=seed + 2)
    return sysd, Bm, K


def _oracle_maps(sysd, Bm, K, b):
    A, C = sysd["A"][b], sysd["C"][b]
    PBX, PBU = sls.state_feedback_responses(A, Bm[b], K[b])
    _, L = sls.kalman_recursion(A, C, sysd["E"][b], sysd["F"][b], sysd["Xi"][b])
    PX, PY = sls.observer_responses(A, C, L)
    return (PBX, PBU), sls.closed_loop_maps(A, PBX, PBU, PX, PY)


@pytest.mark.parametrize("rb", [8, 4])
@pytest.mark.parametrize("nw,ne,nc", [(130, 65, 12), (33, 70, 0)])
def test_tubes_and_margins_match_the_oracle(rb, nw, ne, nc):
    from paper_2606_14188_b300 import sls as gsls
    B, N, n, p, m = 2, 5, 70, 65, 6
    sysd, Bm, K = _case(B, N, n, p, m, nw, ne, seed=41 + nw)
    A = _t(sysd["A"], rb)
    out = gsls.observer(A, *(_t(sysd[k], rb) for k in ("C", "E", "F", "Xi")))
    assert int(torch.count_nonzero(out[4])) == 0
    PB = [_oracle_maps(sysd, Bm, K, b) for b in range(B)]
    PBX = gsls.pack(_t(np.stack([q[0][0] for q in PB]), rb), N, n, n)
    PBU = gsls.pack(_t(np.stack([q[0][1] for q in PB]), rb), N, m, n)
    maps = gsls.closed_loop(A, PBX, PBU, out[2], out[3])
    rng = np.random.default_rng(nw)
    Ccon = np.vstack([rng.normal(size=(nc - 4, n + m)), np.eye(n + m)[[0, 5, n, n + m - 1]]]) if nc else None
    bcon = rng.normal(size=nc) if nc else None
    z, v = rng.normal(size=(B, N + 1, n)), rng.normal(size=(B, N, m))
    args = (_t(Ccon, rb), _t(bcon, rb), _t(z, rb), _t(v, rb)) if nc else ()
    tau, margin = gsls.tubes(*maps, _t(sysd["E"], rb), _t(sysd["F"], rb), *args)
    if not nc:
        assert margin is None
    for b in range(B):
        XW, UW, XE, UE = PB[b][1]
        ref = tubes.tube_widths(XW, UW, XE, UE, sysd["E"][b], sysd["F"][b], N)
        assert _rel(tau[b].cpu().numpy(), ref) <= TOL[rb], b
        assert np.all(tau[b, 0].cpu().numpy() == 0)
        if nc:
            mref = tubes.constraint_margins(XW, UW, XE, UE, sysd["E"][b], sysd["F"][b], N, Ccon, bcon,
                                            z[b], v[b])
            assert _rel(margin[b].cpu().numpy(), mref) <= TOL[rb], b


@pytest.mark.parametrize("rb", [8, 4])
def test_conformal_radius_matches_the_oracle(rb):
    from paper_2606_14188_b300 import sls as gsls
    rng = np.random.default_rng(51)
    for ncal, dim in ((100, 126), (1, 3), (8192, 6), (1000, 246)):
        qn = rng.normal(size=(ncal, dim))
        fp = qn + 0.01 * rng.exponential(size=(ncal, 1)) * rng.normal(size=(ncal, dim))
        ref_s = tubes.conformal_scores(qn, fp)
        for delta, T in ((0.1, 1), (0.2, 20), (0.5, 2), (1e-4, 1)):
            radius, scores = gsls.conformal_radius(_t(qn, rb), _t(fp, rb), delta, T)
            s = scores.cpu().numpy()
            assert _rel(s, ref_s) <= (1e-12 if rb == 8 else 1e-5)
            ref = tubes.conformal_radius(ref_s, delta, T)
            got = float(radius.cpu().numpy()[0])
            if math.isinf(ref):
                assert math.isinf(got) and got > 0
            else:
                assert abs(got - ref) <= (1e-12 if rb == 8 else 1e-5) * ref, (ncal, delta, T)


def test_conformal_nan_score_sorts_last():
    from paper_2606_14188_b300 import sls as gsls
    qn = np.array([[1.0, 0.0], [0.0, 0.0], [np.nan, 0.0], [3.0, 0.0], [2.0, 0.0]])
    fp = np.zeros_like(qn)
    # scores 1, 0, NaN, 3, 2 -> sorted 0, 1, 2, 3, (NaN as +inf); k = ceil(6 * 0.5) = 3 -> 2
    radius, _ = gsls.conformal_radius(_t(qn, 8), _t(fp, 8), 0.5, 1)
    assert float(radius.cpu()[0]) == 2.0
    radius, _ = gsls.conformal_radius(_t(qn, 8), _t(fp, 8), 0.1, 1)   # k = 6 > 5: +inf
    assert math.isinf(float(radius.cpu()[0]))
