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


def cloth_chain(args):
    """The surrogate gradient of one cloth rollout chained through the oracle's smooth-step
    Jacobians at the GPU's own states: traj [H+1][n_q] (the GPU's nonsmooth forward), controls
    U [H][6].  Each step's smooth Newton starts at the GPU's next node positions (its stage-1
    solution plus the stage-2 displacement), which lands on the root next to the GPU's.
    Returns dL/du [H][6] and L."""
    scene, traj, U = args
    sc = osim.Scene(scene["params"], scene["rest_x"])
    H = U.shape[0]
    L, seeds, dU = ograd.loss_and_seeds(sc, traj, U)
    lam = seeds[H].copy()
    g = np.zeros_like(U)
    for t in range(H - 1, -1, -1):
        xn = np.asarray(traj[t + 1][: sc.n]).reshape(sc.nv, 3)
        jac = ograd.SmoothStepJacobian(sc, traj[t], U[t], x_start=xn)
        if not jac.defined:
            return dict(L=L, dL_du=None, status=int(jac.status))
        qb, ub = jac.vjp(lam)
        g[t] = ub + dU[t]
        lam = qb + seeds[t]
    return dict(L=L, dL_du=g, status=0)


def cloth_stage2(args):
    """Stage 2 of one nonsmooth cloth step from the GPU's state q (the oracle's stage-1 root next
    to the GPU's next node positions xn): returns the oracle's q+ and its status."""
    scene, q, u, xn = args
    sc = osim.Scene(scene["params"], scene["rest_x"])
    qp, st = osim.step(sc, q, u, osim.HARD, x_start=np.asarray(xn).reshape(sc.nv, 3))
    return dict(q_next=qp, status=int(st))


_BLAS_ENV = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


def pool(procs):
    """A spawned pool whose workers run the oracle on one BLAS thread each (a process per core):
    the thread count is read from the environment when a worker loads numpy."""
    import multiprocessing as mp
    import os
    saved = {k: os.environ.get(k) for k in _BLAS_ENV}
    os.environ.update({k: "1" for k in _BLAS_ENV})
    try:
        return mp.get_context("spawn").Pool(procs)
    finally:
        for k, v in saved.items():
            if v is None:
                os.environ.pop(k, None)
            else:
                os.environ[k] = v
