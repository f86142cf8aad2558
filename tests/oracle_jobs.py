"""Oracle work items for the GPU parity tests, run in a spawned process pool (this module imports
the oracle and the scene generator only, so that child processes start quickly)."""
import numpy as np

from oracle import grad as ograd, sim as osim
from paper_2606_14188_b300 import scenes


def rope64_rollout(b):
    """Rollout b of the 1024 x 64-node x 50-step rope workload: the oracle's nonsmooth trajectory
    and status, and its loss, surrogate gradient and status."""
    w = scenes.workload(2)
    sc = osim.Scene(w["scene"]["params"], w["scene"]["rest_x"])
    traj, st_f, _ = osim.rollout(sc, w["q0"][b], w["U"][b], osim.HARD)
    r = ograd.rollout_vjp(sc, w["q0"][b], w["U"][b], "surrogate")
    return dict(b=b, traj=traj, status_fwd=int(st_f), L=float(r["L"]), dL_du=r["dL_du"], status=int(r["status"]))
