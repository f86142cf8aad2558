"""Pins of the oracle's plan solve (oracle/plan.py): the counter-based generator against its
published known answers, the normal transform against the normal distribution, the Adam step
against its closed forms, and the planner's selection and descent on a small rope."""
import math
import os

import numpy as np
import pytest
from scipy import stats

from oracle import plan, sim as osim
from paper_2606_14188_b300 import scenes

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def test_philox_known_answers():
    n = 0
    for line in open(os.path.join(GOLDEN, "philox4x32_10_kat.txt")):
        if line.startswith("#") or not line.strip():
            continue
        w = [int(x, 16) for x in line.split()]
        assert plan.philox4x32_10(w[:4], w[4:6]) == tuple(w[6:10])
        n += 1
    assert n == 3


def test_first_normals_come_from_the_zero_counter():
    # seed 0, candidate 0, elements 0 and 1: counter (0,0,0,0), key (0,0) -- the first known
    # answer -- through the Box-Muller pair
    x0, x1 = 0x6627E8D5, 0xE169C58D
    rad = math.sqrt(-2.0 * math.log((x0 + 1.0) / 2.0 ** 32))
    eps = plan.candidate_normals(0, 0, 1)
    assert eps[0, 0] == pytest.approx(rad * math.cos(2 * math.pi * x1 / 2.0 ** 32), abs=1e-15)
    assert eps[0, 1] == pytest.approx(rad * math.sin(2 * math.pi * x1 / 2.0 ** 32), abs=1e-15)


def test_normals_are_standard_normal():
    z = np.concatenate([plan.candidate_normals(12345, r, 200).ravel() for r in range(1, 9)])
    assert abs(z.mean()) < 0.05 and abs(z.var() - 1.0) < 0.05
    assert stats.kstest(z, "norm").pvalue > 1e-3
    # distinct candidates and seeds give different draws
    a, b = plan.candidate_normals(1, 1, 4), plan.candidate_normals(1, 2, 4)
    c = plan.candidate_normals(2, 1, 4)
    assert not np.allclose(a, b) and not np.allclose(a, c)


def test_adam_first_and_constant_gradient_steps():
    """Bias-corrected Adam moves each coordinate by lr g / (|g| + eps) on the first step, and on
    every step while the gradient stays constant (m_hat = g, v_hat = g^2 exactly)."""
    rng = np.random.default_rng(0)
    u = rng.uniform(-0.01, 0.01, (5, 6))
    g = rng.normal(size=(5, 6))
    m = np.zeros_like(u)
    v = np.zeros_like(u)
    lr = 1e-3
    for it in range(1, 6):
        u2, m, v = plan.adam_step(u, g, m, v, it, lr, u_max=1.0)
        np.testing.assert_allclose(u - u2, lr * g / (np.abs(g) + plan.ADAM_EPS), rtol=1e-12, atol=1e-18)
        u = u2
    # the box clip
    u3, _, _ = plan.adam_step(np.full((1, 6), 0.0499), -np.ones((1, 6)), np.zeros((1, 6)),
                              np.zeros((1, 6)), 1, 0.01, u_max=0.05)
    assert np.all(u3 == 0.05)


@pytest.fixture(scope="module")
def small_plan():
    sc = scenes.rope_scene(8, n_spheres=0)
    p = sc["params"]
    osc = osim.Scene(p, sc["rest_x"])
    H, R, G = 4, 3, 4
    warm = np.zeros((H, 6))
    out = plan.plan_solve(osc, sc["q0"], warm, R, G, lr=0.01, seed=7)
    return out, warm, R, G


def test_planner_selection(small_plan):
    out, warm, R, G = small_plan
    L, st = out["losses"], out["status"]
    ok = st == 0
    assert np.all(ok)
    # the result is the lowest evaluated loss; ties go to the earliest evaluation, lowest r
    flat = np.where(ok, L, np.inf).ravel()
    k = int(np.argmin(flat))
    assert out["L"] == flat[k] and (out["it"], out["r"]) == (k // R + 1, k % R)
    assert np.all(np.abs(out["u"]) <= 0.05)
    # candidate 0 of the first evaluation is the warm start itself
    assert L[0, 0] >= out["L"]


def test_planner_descends(small_plan):
    """With the goal 10 cm above both grasped ends, gradient steps must lower the loss below
    every initial candidate's (a wrong gradient sign would leave the best at evaluation 1)."""
    out, warm, R, G = small_plan
    assert out["it"] > 1
    assert out["L"] < 0.9 * np.min(out["losses"][0])
