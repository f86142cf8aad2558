#!/usr/bin/env python
"""Benchmark of the hot path: forward rollout + checkpointed adjoint of the batched rope workload
(1024 rollouts x 64-node rope, horizon 50, FP32, 2 spheres + 2 boxes + ground, checkpoint every
7 steps, nonsmooth forward with surrogate gradients), metric node-steps/s.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line.  `value` is device-timed (CUDA events on the launching stream, inputs
resident in HBM, L2 flushed between timed steps outside the timed intervals); `e2e` times the
same call from pinned host buffers with the host<->device copies inside the timed region.  With
N > 1 (torchrun), every rank runs its own 1024 rollouts (weak scaling, no collective on the data
path) and the slowest rank's time is used.  `--impl reference` times the FP64 CPU oracle on a
bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import copy
import csv
import hashlib
import glob
import io
import json
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2606_14188_b300 import scenes, flops  # noqa: E402

METRIC = "sim+adjoint node-steps/s"
UNIT = "node-steps/s"
WORKLOAD = "rope64_b1024_h50"
BASE_SERVED_SEED = 260614188 + 5
CLOCK_FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")


# ------------------------------------------------------------------------------------------
# oracle work (CPU baseline, reference arm, iteration counts for the flop model)
# ------------------------------------------------------------------------------------------

_BLAS_ENV = ("OPENBLAS_NUM_THREADS", "OMP_NUM_THREADS", "MKL_NUM_THREADS")


def _pool(procs):
    """A spawned pool whose workers run the oracle's linear algebra on one thread each (a process
    per core; multithreaded BLAS in every process would oversubscribe the cores).  A worker reads
    the BLAS thread count from its environment when it loads numpy, so the variables are set
    while the workers start."""
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


def _leg(name, t0):
    print(f"bench: {name} {time.perf_counter() - t0:.1f} s", file=sys.stderr, flush=True)


def _oracle_vjp(args):
    b, tol = args
    from oracle import sim as osim, grad as ograd
    w = scenes.workload(2)
    sc = osim.Scene(w["scene"]["params"], w["scene"]["rest_x"])
    t0 = time.perf_counter()
    r = ograd.rollout_vjp(sc, w["q0"][b], w["U"][b], "surrogate", tol=tol) if tol else \
        ograd.rollout_vjp(sc, w["q0"][b], w["U"][b], "surrogate")
    dt = time.perf_counter() - t0
    fwd = np.array(r["fwd_counts"], dtype=float).mean(axis=0)
    sm = np.array(r["smooth_counts"], dtype=float).mean(axis=0)
    return dict(seconds=dt, fwd_newton=fwd[0], fwd_ipm=fwd[1], sm_newton=sm[0], sm_ipm=sm[1])


def oracle_sample(rollouts, tol, procs):
    t0 = time.perf_counter()
    with _pool(procs) as pool:
        res = pool.map(_oracle_vjp, [(b, tol) for b in rollouts])
    wall = time.perf_counter() - t0
    return res, wall


def counts_mean(res):
    return {k: float(np.mean([r[k] for r in res])) for k in ("fwd_newton", "fwd_ipm", "sm_newton", "sm_ipm")}


# ------------------------------------------------------------------------------------------
# helpers
# ------------------------------------------------------------------------------------------

# the source files each kernel is compiled from (its own, the shared headers, its launcher)
KERNEL_SOURCES = {
    "rope": ["common.cuh", "cr.cuh", "rope.cuh", "rope_cta.cuh", "rope_cta_body.cuh", "rope_lin.cuh",
             "rope_lin_body.cuh", "launch_rope.cuh", "rope_vjp_f32.cu", "rope_rollout_f32.cu",
             "rope_linearize_f32.cu"],
    # the cloth VJP kernel's device code and its own launcher (the packed serving kernel, built
    # from the same headers, has a launcher of its own in the same file)
    "cloth": ["common.cuh", "rope.cuh", "cloth_band.cuh", "cloth.cuh", ("launch_cloth.cuh", "launch_cloth_vjp")],
    # the observer stage's block-triangular product: its tile routine and the kernel
    "sls_tri": [("sls.cu", "row_of"), ("sls.cu", "col_of"), ("sls.cu", "tile_mma"), ("sls.cu", "tile_store"),
                ("sls.cu", "sls_tri_kernel")],
}


def _source_lines(entry):
    """a whole file, or (file, function): that function's definition, from the line naming it to
    the first closing brace in column 0"""
    name, fn = (entry, None) if isinstance(entry, str) else entry
    lines = open(os.path.join(ROOT, "paper_2606_14188_b300", "csrc", name)).read().splitlines()
    if fn is None:
        return lines
    start = next(i for i, l in enumerate(lines) if f" {fn}(" in l and not l.lstrip().startswith("//"))
    end = next(i for i in range(start, len(lines)) if lines[i] == "}")
    return lines[start:end + 1]


def kernel_source_hash(kernel: str):
    """hash of the kernel family's sources with // comments and blank lines removed (editing a
    comment does not invalidate a measured figure)"""
    h = hashlib.sha256()
    fam = "cloth" if kernel.startswith("cloth") else "sls_tri" if kernel.startswith("sls_tri") else "rope"
    for entry in KERNEL_SOURCES[fam]:
        for line in _source_lines(entry):
            code = line.split("//", 1)[0].rstrip()
            if code:
                h.update(code.encode() + b"\n")
    return h.hexdigest()[:16]


def load_traffic(kernel: str, workload: str = WORKLOAD):
    """dram bytes per launch from a committed ncu summary, if it was taken on this exact kernel
    source and workload; else None."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    if not os.path.exists(path):
        return None
    try:
        d = json.load(open(path))
        e = d.get(kernel)
        if e and e.get("source_hash") == kernel_source_hash(kernel) and e.get("workload") == workload:
            return float(e["dram_bytes_per_launch"])
    except Exception:
        return None
    return None


class ClockSampler:
    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={CLOCK_FIELDS}", "--format=csv",
                 "-lms", "200"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.out = ""
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.out, _ = self.proc.communicate(timeout=5)
            except Exception:
                self.proc.kill()
        return False

    def summary(self):
        if not getattr(self, "out", ""):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        rows = list(csv.reader(io.StringIO(self.out)))
        hdr = [h.strip() for h in rows[0]]
        sm, smax, reasons = [], [], set()
        for r in rows[1:]:
            if len(r) != len(hdr):
                continue
            d = dict(zip(hdr, [x.strip() for x in r]))
            try:
                sm.append(float(d["clocks.current.sm [MHz]"].split()[0]))
                smax.append(float(d["clocks.max.sm [MHz]"].split()[0]))
            except Exception:
                continue
            for k, v in d.items():
                if k.startswith("clocks_event_reasons.") and k != "clocks_event_reasons.active" \
                        and v.lower() == "active":
                    reasons.add(k.split(".", 1)[1])
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None, "reasons": sorted(reasons),
                "samples": len(sm)}


# ------------------------------------------------------------------------------------------
# arms
# ------------------------------------------------------------------------------------------

def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    w = scenes.workload(2)
    nv, H = w["scene"]["params"]["n_nodes"], w["H"]
    cores = os.cpu_count() or 1
    procs = max(1, min(cores, 16))
    per_step = 2 * procs                      # rollouts per step (two per process)
    with _pool(procs) as pool:                # one pool for the run: start-up is not timed
        for s in range(args.warmup):
            pool.map(_oracle_vjp, [(b, None) for b in range(s * per_step, (s + 1) * per_step)])
        t = 0.0
        for s in range(args.steps):
            b0 = ((args.warmup + s) * per_step) % 1024
            t0 = time.perf_counter()
            pool.map(_oracle_vjp, [((b0 + i) % 1024, None) for i in range(per_step)])
            t += time.perf_counter() - t0
    value = args.steps * per_step * nv * H / t
    line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=args.gpus, steps=args.steps,
                warmup=args.warmup, ms_per_step=1e3 * t / args.steps, higher_is_better=True,
                scaling="weak", vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=WORKLOAD, rollouts_per_step=per_step, nodes=nv, horizon=H),
                impl="reference",
                cpu_baseline=dict(value=value, unit=UNIT, cores=procs, kind="oracle",
                                  sample=f"{per_step} of the workload's rollouts per step (full "
                                         f"horizon, forward + adjoint) on {procs} processes"),
                e2e=dict(value=value, unit=UNIT, h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)


def time_device(fn, steps, flush, stream):
    """per-call seconds of fn() by CUDA events on the launching stream, L2 flushed between calls
    outside the timed intervals"""
    import torch
    fn()
    torch.cuda.synchronize()
    starts = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(steps)]
    for i in range(steps):
        flush.fill_(float(i))
        starts[i].record(stream)
        fn()
        ends[i].record(stream)
    torch.cuda.synchronize()
    return [a.elapsed_time(b) * 1e-3 for a, b in zip(starts, ends)]


def max_over_ranks(t, world):
    from paper_2606_14188_b300.shard import max_over_ranks as mor
    return mor(t, "cuda") if world > 1 else t


def measured_hbm_peak():
    try:
        return float(json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


def inertial_leg(args, flush, stream, world):
    """The inertial step variant (state [x, v, g], implicit Euler inertia, Rayleigh damping
    alpha = 0.5 /s, beta = 0.02 s): forward + adjoint on the headline's 1024 rollouts of the
    64-node rope (at rest at t = 0) and the linearisation of the 256 x 20 40-node workload in the
    246-dimensional state, FP32."""
    import copy
    import torch
    from paper_2606_14188_b300.sim import Sim
    out = {}
    w = scenes.workload(2, B=args.rollouts, H=args.rope_horizon)
    sc = copy.deepcopy(w["scene"])
    sc["params"].update(second_order=True, damp_alpha=0.5, damp_beta=0.02)
    B, H, nv = w["B"], w["H"], sc["params"]["n_nodes"]
    s = Sim(sc, real_bytes=4, max_batch=B, max_horizon=H)
    q = np.zeros((B, s.nq), dtype=np.float32)
    q[:, :3 * nv] = w["q0"][:, :3 * nv]
    q[:, 6 * nv:] = w["q0"][:, 3 * nv:]
    q0 = torch.tensor(q, device="cuda")
    U = torch.tensor(w["U"], dtype=torch.float32, device="cuda")
    res = []
    per = time_device(lambda: res.append(s.rollout_vjp(q0, U, want_dq0=False)), args.steps, flush, stream)
    t = max_over_ranks(sum(per), world) / args.steps
    st = res[-1][3].cpu().numpy()
    out["rollout_vjp"] = dict(workload=f"rope{nv}_b{B}_h{H}, inertial", ms_per_step=1e3 * t,
                              value=world * int(np.count_nonzero(st == 0)) * nv * H / t, unit=UNIT,
                              status_nonzero=int(np.count_nonzero(st)))
    del s, res
    w = scenes.workload(4)
    sc = copy.deepcopy(w["scene"])
    sc["params"].update(second_order=True, damp_alpha=0.5, damp_beta=0.02)
    B, H, nv = w["B"], w["H"], sc["params"]["n_nodes"]
    s = Sim(sc, real_bytes=4, max_batch=B, max_horizon=H)
    q = np.zeros((B, s.nq), dtype=np.float32)
    q[:, :3 * nv] = w["q0"][:, :3 * nv]
    q[:, 6 * nv:] = w["q0"][:, 3 * nv:]
    V = torch.tensor(w["U"], dtype=torch.float32, device="cuda")
    Z, _, _ = s.rollout(torch.tensor(q, device="cuda"), V)
    A, Bm, st = s.linearize(Z, V)
    per = time_device(lambda: s.linearize(Z, V), args.steps, flush, stream)
    t = max_over_ranks(sum(per), world) / args.steps
    out["linearize"] = dict(workload=f"rope{nv}_b{B}_h{H}, inertial (n_q = {s.nq})", ms_per_step=1e3 * t,
                            value=world * B * H / t, unit="step Jacobians/s",
                            status_nonzero=int(torch.count_nonzero(st).item()))
    return out


def linearize_leg(args, flush, stream, world):
    """sim_linearize on 256 nominal trajectories of a 40-node rope (horizon 20): every A_t, B_t of
    the smooth step written to HBM.  Bound: HBM writes of A and B."""
    import torch
    from paper_2606_14188_b300.sim import Sim
    w = scenes.workload(4)
    sc, B, H = w["scene"], w["B"], w["H"]
    nv = sc["params"]["n_nodes"]
    nq = 3 * nv + 6
    s = Sim(sc, real_bytes=4, max_batch=B, max_horizon=H)
    q0 = torch.tensor(w["q0"], dtype=torch.float32, device="cuda")
    V = torch.tensor(w["U"], dtype=torch.float32, device="cuda")
    Z, _, _ = s.rollout(q0, V)                   # nominal trajectories (not timed)
    for _ in range(max(1, args.warmup)):
        A, Bm, st = s.linearize(Z, V)
    per = time_device(lambda: s.linearize(Z, V), args.steps, flush, stream)
    t = max_over_ranks(sum(per), world)
    avg = t / args.steps
    out_bytes = B * H * (nq * nq + nq * 6) * 4
    in_bytes = B * (H + 1) * nq * 4 + B * H * 6 * 4
    peak, src = measured_hbm_peak()
    gbs = (out_bytes + in_bytes) / avg / 1e9
    return dict(workload=f"rope{nv}_b{B}_h{H}", value=world * B * H / avg, unit="step Jacobians/s",
                ms_per_step=1e3 * avg, bytes_per_launch=out_bytes + in_bytes,
                status_nonzero=int(torch.count_nonzero(st).item()),
                roofline=dict(bound="hbm", achieved=gbs, peak=peak, unit="GB/s", frac=gbs / peak,
                              traffic=load_traffic("rope_linearize_call", f"rope{nv}_b{B}_h{H}"),
                              peak_source=f"{src} HBM copy bandwidth"))


def sls_leg(args, flush, stream, world):
    """The output-feedback SLS observer stage about the linearisation workload's nominal
    trajectories (the 40-node rope, 256 x 20 steps, state 126, the 120 node coordinates observed,
    FP32): sls_observer (Kalman recursion and observer responses) and sls_closed_loop (the four
    closed-loop maps) on the A_t, B_t that sim_linearize writes, the state-feedback responses from
    seeded gains.  Bound: FP32 FMA (dense products of 120-126 wide blocks)."""
    import torch
    from paper_2606_14188_b300 import sls as gsls
    from paper_2606_14188_b300.sim import Sim
    w = scenes.workload(4)
    sc, H = w["scene"], w["H"]
    B = min(w["B"], args.sls_trajectories)
    nv = sc["params"]["n_nodes"]
    n, m, p = 3 * nv + 6, 6, 3 * nv
    s = Sim(sc, real_bytes=4, max_batch=B, max_horizon=H)
    V = torch.tensor(w["U"][:B], dtype=torch.float32, device="cuda")
    Z, _, _ = s.rollout(torch.tensor(w["q0"][:B], dtype=torch.float32, device="cuda"), V)
    A, Bm, st = s.linearize(Z, V)
    lin_flagged = int(torch.count_nonzero(st).item())
    del s
    obs = scenes.sls_observation_model(B, H, nv)
    f32 = dict(dtype=torch.float32, device="cuda")
    Cm, E, F, Xi = (torch.tensor(obs[k], **f32) for k in ("C", "E", "F", "Xi"))
    A = torch.nan_to_num(A).contiguous()          # a flagged linearisation step (NaN) stands as 0
    Kg = torch.tensor(scenes.sls_feedback_gains(B, H, m, n), **f32)
    PBX = gsls.response((A + torch.nan_to_num(Bm) @ Kg[:, :H]).contiguous())
    kidx = torch.tensor([k for k in range(H + 1) for _ in range(k + 1)], device="cuda")
    PBU = (Kg[:, kidx] @ PBX).contiguous()
    for _ in range(max(1, args.warmup)):
        out = gsls.observer(A, Cm, E, F, Xi)
    flagged = int(torch.count_nonzero(out[4]).item())
    PX, PY = out[2], out[3]
    del out
    for _ in range(max(1, args.warmup)):
        maps = gsls.closed_loop(A, PBX, PBU, PX, PY)
    del maps
    t_obs = max_over_ranks(sum(time_device(lambda: gsls.observer(A, Cm, E, F, Xi), args.steps, flush,
                                           stream)), world) / args.steps
    t_cl = max_over_ranks(sum(time_device(lambda: gsls.closed_loop(A, PBX, PBU, PX, PY), args.steps,
                                          flush, stream)), world) / args.steps
    # the covariances alone by the associative scan of the combination rules (logarithmic depth)
    for _ in range(max(1, args.warmup)):
        _, st_scan = gsls.kalman_scan(A, Cm, E, F, Xi)
    t_scan = max_over_ranks(sum(time_device(lambda: gsls.kalman_scan(A, Cm, E, F, Xi), args.steps, flush,
                                            stream)), world) / args.steps
    # one trajectory (a single plan's nominal): the horizon is the only parallel direction there
    one = [x[:1].contiguous() for x in (A, Cm, E, F, Xi)]
    for _ in range(max(1, args.warmup)):
        gsls.observer(*one)
        gsls.kalman_scan(*one)
    t_obs1 = max_over_ranks(sum(time_device(lambda: gsls.observer(*one), args.steps, flush, stream)),
                            world) / args.steps
    t_scan1 = max_over_ranks(sum(time_device(lambda: gsls.kalman_scan(*one), args.steps, flush, stream)),
                             world) / args.steps
    # reachable tubes and the tightened margins of the node heights (z_i >= 0: -z_i <= 0) on the
    # closed-loop maps, and the conformal radius of 1000 one-step transitions of the rope
    maps = gsls.closed_loop(A, PBX, PBU, PX, PY)
    Ccon = torch.zeros(nv, n + m, **f32)
    Ccon[torch.arange(nv), 3 * torch.arange(nv) + 2] = -1.0
    bcon = torch.zeros(nv, **f32)
    zc, vc = torch.nan_to_num(Z).contiguous(), V.contiguous()
    for _ in range(max(1, args.warmup)):
        tau, margin = gsls.tubes(*maps, E, F, Ccon, bcon, zc, vc)
    t_tub = max_over_ranks(sum(time_device(lambda: gsls.tubes(*maps, E, F, Ccon, bcon, zc, vc), args.steps,
                                           flush, stream)), world) / args.steps
    tube_max = float(tau[:, -1, :3 * nv].max())
    robust_rows = float((margin >= 0).float().mean())
    del maps
    ncal = 1000
    rng = np.random.default_rng(scenes.BASE_SEED + 503)
    pick = rng.integers(0, B, ncal), rng.integers(0, H, ncal)
    qcal = zc[torch.tensor(pick[0], device="cuda"), torch.tensor(pick[1], device="cuda")].contiguous()
    ucal = vc[torch.tensor(pick[0], device="cuda"), torch.tensor(pick[1], device="cuda")][:, None].contiguous()
    s1 = Sim(sc, real_bytes=4, max_batch=ncal, max_horizon=1)
    _, fpred, _ = s1.rollout(qcal, ucal)
    qnext = (fpred + torch.tensor(0.003 * rng.standard_normal(fpred.shape), **f32)).contiguous()
    radius, _ = gsls.conformal_radius(qnext, fpred.contiguous(), 0.1, H)
    t_cp = max_over_ranks(sum(time_device(lambda: gsls.conformal_radius(qnext, fpred, 0.1, H), args.steps,
                                          flush, stream)), world) / args.steps
    del s1
    sms = torch.cuda.get_device_properties(0).multi_processor_count
    peak = sms * 128 * 2 * 2032e6 / 1e12
    f_obs = flops.sls_observer_flops(H, n, p, n, p, n) * B
    f_cl = flops.sls_closed_loop_flops(H, n, m, p) * B

    def roof(f, t):
        a = f / t / 1e12
        return dict(bound="alu", achieved=a, peak=peak, unit="TFLOP/s", frac=a / peak, traffic=None,
                    flops_per_call=f, peak_source=f"FP32 FMA: {sms} SMs x 128 lanes x 2 x 2032 MHz")

    return dict(workload=f"rope{nv}_b{B}_h{H} observer stage (n {n}, p {p}, m {m})",
                observer=dict(ms_per_step=1e3 * t_obs, value=world * B / t_obs, unit="trajectories/s",
                              roofline=roof(f_obs, t_obs)),
                closed_loop=dict(ms_per_step=1e3 * t_cl, value=world * B / t_cl, unit="trajectories/s",
                                 roofline=roof(f_cl, t_cl),
                                 dominant_kernel=dict(
                                     kernel="sls_tri_kernel (the Phi^xw launch)",
                                     dram_bytes_per_launch=load_traffic("sls_tri_kernel", f"rope{nv}_b{B}_h{H}"))),
                kalman_scan=dict(ms_per_step=1e3 * t_scan, value=world * B / t_scan, unit="trajectories/s",
                                 status_nonzero=int(torch.count_nonzero(st_scan).item()),
                                 what="sls_kalman_scan: Pi_0..Pi_20 by the associative scan (5 levels); "
                                      "the observer call forms them step by step",
                                 one_trajectory=dict(scan_ms=1e3 * t_scan1, observer_ms=1e3 * t_obs1)),
                tubes=dict(ms_per_step=1e3 * t_tub, value=world * B / t_tub, unit="trajectories/s",
                           roofline=roof(flops.sls_tubes_flops(H, n, m, p, n, p, nv) * B, t_tub),
                           what=f"sls_tubes: row-wise tubes of [x; u] and the margins of {nv} node-height "
                                "constraints over the 20 steps",
                           final_tube_max_m=tube_max, margins_nonnegative_fraction=robust_rows),
                conformal=dict(ms_per_step=1e3 * t_cp, calibration_samples=ncal, delta=0.1, horizon=H,
                               radius_m=float(radius.cpu()[0]),
                               what="sls_conformal_radius over one-step transitions of the rope from "
                                    "states of the nominal trajectories (f from sim_rollout, next "
                                    "perceived states with 3 mm noise per coordinate)"),
                status_nonzero=flagged, linearize_status_nonzero=lin_flagged)


def apg_leg(args, flush, stream, world):
    """The analytic policy gradient on the headline's rollouts: a tanh policy of 64 hidden units
    in the loop of the 1024 x 64-node x 50-step rope rollouts, the planning loss and dL/dtheta
    through the simulator (apg_rollout_grad; every step one rollout step and one adjoint step)."""
    import torch
    from paper_2606_14188_b300.sim import Sim
    w = scenes.workload(2, B=args.rollouts, H=args.rope_horizon)
    sc, B, H = w["scene"], w["B"], w["H"]
    nv = sc["params"]["n_nodes"]
    hidden = 64
    s = Sim(sc, real_bytes=4, max_batch=B, max_horizon=H)
    nth = hidden * s.nq + 7 * hidden + 6
    rng = np.random.default_rng(scenes.BASE_SEED + 504)
    th = torch.tensor(0.05 * rng.standard_normal(nth) / np.sqrt(s.nq), dtype=torch.float32, device="cuda")
    q0 = torch.tensor(w["q0"], dtype=torch.float32, device="cuda")
    for _ in range(max(1, args.warmup)):
        Lv, dth, _, st = s.apg_grad(q0, th, hidden, H)
    t = max_over_ranks(sum(time_device(lambda: s.apg_grad(q0, th, hidden, H), args.steps, flush, stream)),
                       world) / args.steps
    done = int(torch.count_nonzero(st == 0).item())
    return dict(workload=f"rope{nv}_b{B}_h{H}, tanh policy of {hidden} hidden units", ms_per_step=1e3 * t,
                value=world * done * nv * H / t, unit=UNIT, status_nonzero=B - done,
                dtheta_finite=bool(torch.isfinite(dth).all().item()),
                what="apg_rollout_grad: closed-loop forward and surrogate adjoint with the policy's "
                     "derivatives in the chain, node-steps of the completed rollouts per second")


def _cloth_sample_job(steps):
    from oracle import grad as ograd, sim as osim
    w = scenes.workload(3, B=1, H=steps)
    sc = w["scene"]
    osc = osim.Scene(sc["params"], sc["rest_x"])
    t0 = time.perf_counter()
    ograd.rollout_vjp(osc, w["q0"][0], w["U"][0], "surrogate")
    return time.perf_counter() - t0, sc["params"]["n_nodes"]


def cloth_oracle_sample(steps=2):
    """The oracle's forward + adjoint of one rollout of the cloth workload over `steps` steps (CPU,
    one process on one thread): node-steps/s and the sample described."""
    with _pool(1) as pool:
        dt, nv = pool.apply(_cloth_sample_job, (steps,))
    return dict(value=nv * steps / dt, unit=UNIT, cores=1, kind="oracle",
                sample=f"1 rollout x {steps} steps of the 32x32 cloth, forward + adjoint, {dt:.1f} s")


def _cloth_oracle_counts(args):
    """The oracle's iterations on one step of the cloth workload from a state the GPU reached:
    its nonsmooth step from q (the defined stage-1 start) and the smooth re-solve of the backward
    (started at the GPU's next node positions, the root next to the GPU's)."""
    scene, q, u, xn = args
    from oracle import grad as ograd, sim as osim
    sc = osim.Scene(scene["params"], scene["rest_x"])
    info = {}
    osim.step(sc, q, u, osim.HARD, info=info)
    jac = ograd.SmoothStepJacobian(sc, q, u, x_start=np.asarray(xn).reshape(sc.nv, 3))
    return dict(fwd_newton=info["newton_it"], fwd_ipm=info["ipm_it"], sm_newton=jac.counts[0],
                sm_ipm=jac.counts[1])


def cloth_leg(args, flush, stream, world, cpu):
    """sim_rollout_vjp on the batched cloth workload: 512 rollouts of a 32 x 32 cloth, FP32, horizon
    30, table + 2 spheres, checkpoint every 5 (flags --cloth-rollouts / --cloth-horizon shrink it
    for profiling captures only).  The flop count uses the FP64 oracle's iterations per step on a
    sample of (rollout, step) states the GPU's forward reached (untimed)."""
    import torch
    from paper_2606_14188_b300.sim import Sim
    props = torch.cuda.get_device_properties(torch.cuda.current_device())
    B = args.cloth_rollouts or 512
    H = args.cloth_horizon
    w = scenes.workload(3, B=B, H=H)
    sc = w["scene"]
    p = sc["params"]
    R, C, nv = p["rows"], p["cols"], p["n_nodes"]
    k = p["checkpoint_every"]
    nobs = len(p["obstacles"])
    n = 3 * nv
    s = Sim(sc, real_bytes=4, max_batch=B, max_horizon=H, newton_max=300)
    q0 = torch.tensor(w["q0"], dtype=torch.float32, device="cuda")
    U = torch.tensor(w["U"], dtype=torch.float32, device="cuda")
    # untimed: the forward's trajectory and counters, and the oracle's iterations at sampled states
    traj, _, st_f, cnt = s.rollout_counters(q0, U)
    c = cnt.cpu().numpy().reshape(B, H, 3)
    gpu_counts = dict(fwd_newton=float(c[..., 0].mean()), fwd_ipm=float(c[..., 1].mean()))
    samp_b = [int(x) for x in np.linspace(0, B - 1, 4).round()]
    samp_t = sorted({int(x) for x in np.linspace(0, H - 1, 5).round()})
    jobs = []
    tr = traj.cpu().numpy().astype(np.float64)
    for b in samp_b:
        for t in samp_t:
            if not np.any(c[b, :t + 1, 2]):
                jobs.append((sc, tr[b, t], w["U"][b, t], tr[b, t + 1, :n]))
    del traj, tr
    counts = None
    if jobs and not args.no_cpu:
        with _pool(max(1, min(os.cpu_count() or 1, 16))) as pool:
            res = pool.map(_cloth_oracle_counts, jobs)
        counts = {key: float(np.mean([r[key] for r in res])) for key in res[0]}
    outs = []          # the timer's untimed first call is the warm-up; the last timed call's outputs
    per = time_device(lambda: outs.append(s.rollout_vjp(q0, U, want_dq0=False)), args.cloth_steps, flush, stream)
    t = max_over_ranks(sum(per), world)
    avg = t / args.cloth_steps
    _, dU, _, st = outs[-1]
    status = st.cpu().numpy()
    node_steps = B * nv * H
    clean_steps = int(np.count_nonzero(status == 0)) * nv * H
    pband = flops.cloth_band(C)
    spn = flops.cloth_springs_per_node(R, C)
    sm_mhz = 2032.0
    peak = props.multi_processor_count * 128 * 2 * sm_mhz * 1e6 / 1e12
    wl = f"cloth{R}x{C}_b{B}_h{H}"
    roof = None
    if counts is not None:
        f_ns = flops.cloth_rollout_vjp_flops_per_node_step(counts, pband, spn, nobs, k)
        # a flagged rollout stops at its failed step: only the clean rollouts' work is counted
        achieved = f_ns * clean_steps / avg / 1e12
        roof = dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s", frac=achieved / peak,
                    traffic=load_traffic("cloth_vjp_kernel", wl),
                    peak_source="FP32 FMA at the max SM clock", flops_per_node_step=f_ns,
                    band_half_width=pband,
                    oracle_iterations_per_step=counts,
                    oracle_sample=f"{len(jobs)} (rollout, step) states of the GPU's forward: rollouts "
                                  f"{samp_b}, steps {samp_t}")
    return dict(workload=wl, what="the batched cloth workload: 512 rollouts x 32x32 cloth x 30 steps, "
                                  "checkpoint every 5" if (B, H) == (512, 30) else "reduced cloth case",
                value=world * node_steps / avg, unit=UNIT, ms_per_step=1e3 * avg, rollouts=B, horizon=H,
                checkpoint_every=k, value_clean_rollouts_only=world * clean_steps / avg,
                status_flagged=int(np.count_nonzero(status)),
                status_newton_cap=int(np.count_nonzero(status & 1)),
                grads_finite=bool(torch.isfinite(dU).all().item()),
                gpu_iterations_per_step=gpu_counts, roofline=roof, cpu_baseline=cpu)


def served_stream(n, seed, cloth_frac=0.0):
    """The served workload: n plan solves with rope sizes U{16..128}, horizons U{20..60}, candidates
    log-uniform in {64, ..., 1024}, 10 evaluations each, Poisson arrival order (times set later).
    With cloth_frac > 0 that fraction of the requests are cloths of side U{8..16}, horizon
    U{10..20}, candidates log-uniform in {32, 64, 128}."""
    rng = np.random.default_rng(seed)
    crng = np.random.default_rng(seed + 17)
    reqs = []
    for i in range(n):
        if cloth_frac > 0 and crng.random() < cloth_frac:
            side = int(crng.integers(8, 17))
            H = int(crng.integers(10, 21))
            R = int(2 ** crng.integers(5, 8))
            sc = scenes.cloth_scene(side, side, n_spheres=2, seed=seed + 1 + i)
            sc["params"]["checkpoint_every"] = 0      # the server picks it by memory
            reqs.append(dict(scene=sc, q0=sc["q0"], H=H, R=R, G=10, seed=seed + 7919 * i, nv=side * side,
                             kw=dict(newton_max=300)))
            continue
        nv = int(rng.integers(16, 129))
        H = int(rng.integers(20, 61))
        R = int(2 ** rng.integers(6, 11))
        sc = scenes.rope_scene(nv, n_spheres=int(rng.integers(1, 3)), n_boxes=int(rng.integers(0, 2)),
                               seed=seed + 1 + i, sphere_box=((0.0, 1.0), (-0.2, 0.2), (0.0, 0.3)))
        sc["params"]["checkpoint_every"] = 0          # the server picks it by memory
        reqs.append(dict(scene=sc, q0=sc["q0"], H=H, R=R, G=10, seed=seed + 7919 * i, nv=nv))
    return reqs


def serve_stream(reqs, gaps, batched):
    """Submit reqs with the given inter-arrival gaps [s]; returns (results, makespan [s])."""
    from paper_2606_14188_b300.serve import PlanServer
    srv = PlanServer(real_bytes=4, mem_budget_bytes=8 << 30, batched=batched, use_graphs=True,
                     autotune=batched)
    try:
        t0 = time.perf_counter()
        due = t0
        tickets = []
        for r, g in zip(reqs, gaps):
            due += g
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                time.sleep(min(due - now, 0.002))
            tickets.append(srv.submit(r["scene"], r["q0"], r["H"], r["R"], r["G"], seed=r["seed"], **r.get("kw", {})))
        out = [srv.poll(t, -1) for t in tickets]
        makespan = (max(o["t_done_ns"] for o in out) - min(o["t_submit_ns"] for o in out)) * 1e-9
        stats = srv.stats()
    finally:
        srv.close()
    return out, makespan, stats


def served_leg(args):
    """Served MPC plan solves, batched (continuous batching, graph replay) against one request at a
    time (one launch per kernel per evaluation, no graphs), on the same stream: each server's
    capacity with the whole stream submitted at once, then the stream arriving as a Poisson process
    at 70 % and 95 % of the batched capacity (of the first repeat), served both ways.  With
    --served-repeats R every measurement is taken R times (arrival gaps drawn afresh each time) and
    reported as the median with its [min, max] spread."""
    n = args.served_requests
    reps = max(1, args.served_repeats)
    reqs = served_stream(n, BASE_SERVED_SEED, args.served_cloth_fraction)
    ncloth = sum(1 for r in reqs if "kw" in r)
    node_steps = sum(r["R"] * r["H"] * r["nv"] * r["G"] for r in reqs)
    what = f"{n} plan solves: {n - ncloth} ropes (nodes U{{16..128}}, horizon U{{20..60}}, candidates " \
           f"log-U{{64..1024}})"
    if ncloth:
        what += f", {ncloth} cloths (side U{{8..16}}, horizon U{{10..20}}, candidates log-U{{32..128}})"

    def lat(out, t):
        ms = np.array([(o["t_done_ns"] - o["t_submit_ns"]) * 1e-6 for o in out])
        return dict(p50_ms=float(np.percentile(ms, 50)), p99_ms=float(np.percentile(ms, 99)),
                    throughput_solves_per_s=n / t)

    same = True

    def check(x, y):
        nonlocal same
        for a2, b2 in zip(x, y):
            same = same and a2["L"] == b2["L"] and np.array_equal(a2["u"], b2["u"])

    runs = []
    rate0 = None
    for rep in range(reps):
        run = {}
        ob, tb, sb = serve_stream(reqs, [0.0] * n, True)
        op, tp, _ = serve_stream(reqs, [0.0] * n, False)
        check(ob, op)
        run["capacity"] = dict(batched=n / tb, per_request=n / tp)
        if rate0 is None:
            rate0 = n / tb
        rng = np.random.default_rng(BASE_SERVED_SEED + 1 + rep)
        for load in (0.7, 0.95):
            gaps = rng.exponential(1.0 / (load * rate0), n)
            gaps[0] = 0.0
            ob, tb, sb = serve_stream(reqs, gaps, True)
            op, tp, sp = serve_stream(reqs, gaps, False)
            check(ob, op)
            run[f"load_{int(load * 100)}"] = dict(batched=dict(**lat(ob, tb), ticks=sb["ticks"],
                                                               graph_launches=sb["graph_launches"]),
                                                  per_request=dict(**lat(op, tp), ticks=sp["ticks"]))
        runs.append(run)

    def summ(vals):
        v = np.array(vals, dtype=float)
        return dict(median=float(np.median(v)), spread=[float(v.min()), float(v.max())])

    res = dict(workload=what + ", 10 evaluations each, FP32, checkpoint interval picked by the server "
                                "(checkpoint_every = 0: the shortest whose records fit in an eighth of "
                                "its memory budget)",
               requests=n, repeats=reps, node_steps=node_steps,
               capacity_solves_per_s=summ([r["capacity"]["batched"] for r in runs]),
               capacity_per_request_solves_per_s=summ([r["capacity"]["per_request"] for r in runs]))
    res["capacity_node_steps_per_s"] = node_steps * res["capacity_solves_per_s"]["median"] / n
    for load in (70, 95):
        key = f"load_{load}"
        ent = dict(rate_solves_per_s=load / 100 * rate0)
        for mode in ("batched", "per_request"):
            ent[mode] = {m: summ([r[key][mode][m] for r in runs])
                         for m in ("p50_ms", "p99_ms", "throughput_solves_per_s")}
        ent["batched"]["graph_launches"] = int(np.median([r[key]["batched"]["graph_launches"] for r in runs]))
        res[key] = ent
    res["results_identical_batched_vs_per_request"] = bool(same)
    return res


def run_ours(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))

    # CPU work first (spawned pool, before any CUDA call): the oracle baseline and the oracle's
    # iteration counts at the GPU tolerance for the flop model
    cpu = None
    counts = None
    if rank == 0 and not args.no_cpu:
        cores = os.cpu_count() or 1
        procs = max(1, min(cores, 16))
        nroll = 16 * procs
        t_leg = time.perf_counter()
        res, wall = oracle_sample(list(range(nroll)), None, procs)
        _leg("rope CPU baseline", t_leg)
        w0 = scenes.workload(2)
        ns = nroll * w0["scene"]["params"]["n_nodes"] * w0["H"]
        per_core = float(np.mean([ns / nroll / r["seconds"] for r in res]))
        cpu = dict(value=ns / wall, unit=UNIT, cores=procs, kind="oracle",
                   sample=f"{nroll} of the 1024 rollouts (full horizon 50, forward + adjoint) on "
                          f"{procs} processes; {wall:.1f} s wall",
                   one_core_value=per_core)
        t_leg = time.perf_counter()
        cres, _ = oracle_sample([0, 341, 682, 1023], 1e-5, 4)
        counts = counts_mean(cres)
        _leg("rope oracle iteration counts", t_leg)
    t_leg = time.perf_counter()
    cloth_cpu = cloth_oracle_sample() if rank == 0 and not args.no_cpu and args.cloth_horizon > 0 else None
    _leg("cloth CPU baseline", t_leg)

    import torch
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    dev = torch.cuda.current_device()
    from paper_2606_14188_b300.sim import Sim
    from paper_2606_14188_b300 import _lib

    # every rank simulates its own share of world x 1024 rollouts (different controls per rank)
    w = scenes.workload(2, B=args.rollouts, H=args.rope_horizon, shard=rank)
    sc, B, H = w["scene"], w["B"], w["H"]
    nv = sc["params"]["n_nodes"]
    k = sc["params"]["checkpoint_every"]
    nobs = len(sc["params"]["obstacles"])
    s = Sim(sc, real_bytes=4, max_batch=B, max_horizon=H)
    q0 = torch.tensor(w["q0"], dtype=torch.float32, device="cuda")
    U = torch.tensor(w["U"], dtype=torch.float32, device="cuda")
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device="cuda")
    stream = torch.cuda.current_stream()

    t_leg = time.perf_counter()
    for _ in range(args.warmup):
        s.rollout_vjp(q0, U, want_dq0=False)
    torch.cuda.synchronize()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    starts = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    ends = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    _lib.lib().cs_launch_count()
    barrier()
    with ClockSampler(dev) as clk:
        for i in range(args.steps):
            flush.fill_(float(i))
            starts[i].record(stream)
            Lv, dU, _, st = s.rollout_vjp(q0, U, want_dq0=False)
            ends[i].record(stream)
        barrier()
    launches = int(_lib.lib().cs_launch_count())
    per = [a.elapsed_time(b) * 1e-3 for a, b in zip(starts, ends)]
    t = sum(per)
    t = max_over_ranks(t, world)
    status = st.cpu().numpy()

    # end to end through the public call from pinned host buffers
    q0_h = torch.tensor(w["q0"], dtype=torch.float32).pin_memory()
    U_h = torch.tensor(w["U"], dtype=torch.float32).pin_memory()
    L_h = torch.empty(B, dtype=torch.float32).pin_memory()
    dU_h = torch.empty(B, H, 6, dtype=torch.float32).pin_memory()
    q0_d = torch.empty_like(q0)
    U_d = torch.empty_like(U)
    barrier()
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for i in range(args.steps):
        q0_d.copy_(q0_h, non_blocking=True)
        U_d.copy_(U_h, non_blocking=True)
        Lv2, dU2, _, _ = s.rollout_vjp(q0_d, U_d, want_dq0=False)
        L_h.copy_(Lv2, non_blocking=True)
        dU_h.copy_(dU2, non_blocking=True)
    e1.record(stream)
    barrier()
    te = e0.elapsed_time(e1) * 1e-3
    te = max_over_ranks(te, world)

    _leg("rope forward + adjoint and end-to-end", t_leg)
    t_leg = time.perf_counter()
    # forward alone (the same rollouts, nonsmooth forward, trajectory written)
    t_fwd = max_over_ranks(sum(time_device(lambda: s.rollout(q0, U), args.steps, flush, stream)),
                           world)
    # the same adjoint with a record at every step (k = 1: 51 records of 588 numbers per rollout,
    # 123 MB for 1024 rollouts) instead of recomputing each segment from its checkpoint
    sc1 = copy.deepcopy(sc)
    sc1["params"]["checkpoint_every"] = 1
    s1 = Sim(sc1, real_bytes=4, max_batch=B, max_horizon=H)
    t_k1 = max_over_ranks(sum(time_device(lambda: s1.rollout_vjp(q0, U, want_dq0=False), args.steps,
                                          flush, stream)), world)
    del s1
    _leg("rope forward alone and every-step records", t_leg)
    # linearisation workload: 256 nominal trajectories of a 40-node rope, horizon 20
    t_leg = time.perf_counter()
    lin = linearize_leg(args, flush, stream, world)
    _leg("linearisation", t_leg)
    t_leg = time.perf_counter()
    sls_out = sls_leg(args, flush, stream, world) if args.sls_trajectories > 0 else None
    _leg("observer stage", t_leg)
    t_leg = time.perf_counter()
    inertial = inertial_leg(args, flush, stream, world)
    _leg("inertial variant", t_leg)
    t_leg = time.perf_counter()
    apg_out = apg_leg(args, flush, stream, world)
    _leg("policy gradient", t_leg)
    t_leg = time.perf_counter()
    served = served_leg(args) if args.served_requests > 0 else None
    _leg("served", t_leg)
    t_leg = time.perf_counter()
    cloth = cloth_leg(args, flush, stream, world, cloth_cpu) if args.cloth_horizon > 0 else None
    _leg("cloth", t_leg)

    if rank == 0:
        # only the node-steps of the rollouts that completed count (a flagged rollout stops at
        # its failing step); every rank's shard has the same make-up in expectation
        node_steps = int(np.count_nonzero(status == 0)) * nv * H
        value = world * args.steps * node_steps / t
        e2e_value = world * args.steps * node_steps / te
        avg_launch = t / args.steps
        clocks = clk.summary()
        sm_mhz = clocks["sm_max_mhz"] or 2032.0
        props = torch.cuda.get_device_properties(dev)
        sms = props.multi_processor_count
        peak = sms * 128 * 2 * sm_mhz * 1e6 / 1e12           # FP32 FMA peak [TFLOP/s]
        roof = None
        if counts is not None:
            f_ns = flops.rollout_vjp_flops_per_node_step(counts, nobs, k)
            achieved = f_ns * node_steps / avg_launch / 1e12
            roof = dict(bound="alu", achieved=achieved, peak=peak, unit="TFLOP/s",
                        frac=achieved / peak, traffic=load_traffic("rope_vjp_call"),
                        kernels="one sim_rollout_vjp call: rope_cta_vjp_queue_kernel (forward jobs, "
                                "(rollout, segment) jobs, per-rollout adjoint chains) and "
                                "rope_queue_finish_kernel; achieved = the completed rollouts' flops / "
                                "the call's event time",
                        peak_source=f"FP32 FMA: {sms} SMs x 128 lanes x 2 x {sm_mhz:.0f} MHz "
                                    "(recipe unit counts and the max SM clock)",
                        flops_per_node_step=f_ns, oracle_iterations_per_step=counts)
        line = dict(metric=METRIC, value=value, unit=UNIT, n_gpus=world, steps=args.steps,
                    warmup=args.warmup, ms_per_step=1e3 * t / args.steps, higher_is_better=True,
                    scaling="weak", vs_baseline=None, dtype="f32", data="synthetic",
                    config=dict(workload=WORKLOAD if (B, H) == (1024, 50) else f"rope64_b{B}_h{H}", rollouts=B,
                                nodes=nv, horizon=H,
                                checkpoint_every=k, obstacles=nobs, grad_mode="surrogate",
                                parallelism=f"rollouts sharded, dp{world}",
                                l2="256 MB write between timed steps, outside the timed intervals"),
                    roofline=roof, cpu_baseline=cpu,
                    e2e=dict(value=e2e_value, unit=UNIT,
                             h2d_bytes_per_step=int(q0.numel() * 4 + U.numel() * 4),
                             d2h_bytes_per_step=int(B * 4 + B * H * 6 * 4)),
                    forward=dict(value=world * args.steps * node_steps / t_fwd, unit=UNIT,
                                 ms_per_step=1e3 * t_fwd / args.steps,
                                 what="sim_rollout alone on the same rollouts"),
                    adjoint_every_step_recorded=dict(
                        value=world * args.steps * node_steps / t_k1, unit=UNIT,
                        ms_per_step=1e3 * t_k1 / args.steps,
                        what="sim_rollout_vjp on the same rollouts with checkpoint_every = 1 (every "
                             "step's record stored, no segment recompute); not the headline, whose "
                             "workload checkpoints every 7 steps"),
                    linearize=lin, sls_observer_stage=sls_out, inertial_variant=inertial, policy_gradient=apg_out, served=served, cloth=cloth,
                    gpu_launches=launches, clocks=clocks,
                    status_nonzero=int(np.count_nonzero(status)),
                    node_steps_counted=f"{int(np.count_nonzero(status == 0))} of {B} rollouts "
                                       f"(the flagged ones excluded) x {nv} nodes x {H} steps",
                    per_step_ms=[round(x * 1e3, 4) for x in per])
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU oracle baseline")
    ap.add_argument("--served-requests", type=int, default=48,
                    help="plan solves in the served stream (0: skip the served leg)")
    ap.add_argument("--rollouts", type=int, default=None,
                    help="rollouts per GPU (default 1024; smaller only for profiling captures)")
    ap.add_argument("--rope-horizon", type=int, default=None,
                    help="horizon of the rope legs (default 50; shorter only for profiling captures)")
    ap.add_argument("--cloth-horizon", type=int, default=30,
                    help="horizon of the cloth leg (default 30, the workload's; 0: skip the cloth leg)")
    ap.add_argument("--cloth-rollouts", type=int, default=None,
                    help="rollouts of the cloth leg (default 512, the workload's)")
    ap.add_argument("--cloth-steps", type=int, default=1, help="timed calls of the cloth leg")
    ap.add_argument("--sls-trajectories", type=int, default=256,
                    help="nominal trajectories of the observer-stage leg (default 256; 0: skip)")
    ap.add_argument("--served-repeats", type=int, default=1,
                    help="repeats of every served measurement (median and spread reported)")
    ap.add_argument("--served-cloth-fraction", type=float, default=0.0,
                    help="fraction of the served requests that are cloths (default 0: ropes only)")
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
