"""Output-feedback SLS observer stage, reachable tubes and conformal radius over libcordsim
(argument marshalling only; every step runs in the library's CUDA kernels, on the current torch
stream).

    Pi, L, PhiX, PhiY, status = observer(A, C, E, F, Xi)     # Kalman recursion + observer responses
    Pi, status = kalman_scan(A, C, E, F, Xi)                  # the same Pi by the associative scan
    Phi = response(Acl)                                       # closed-loop response of given Acl_j
    XW, UW, XE, UE = closed_loop(A, PhiBarX, PhiBarU, PhiX, PhiY)
    tau, margin = tubes(XW, UW, XE, UE, E, F, Ccon, bcon, z, v)  # reachable tubes, tightening
    radius, scores = conformal_radius(q_next, f_pred, delta, T) # conformal radius

Block lower-triangular operators over times 0..N are packed [B][T][r][c], block (k, j) at index
k (k + 1) / 2 + j, T = (N + 1)(N + 2) / 2; unpack() turns them into dense block matrices.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib as L


def n_blocks(N: int) -> int:
    return (N + 1) * (N + 2) // 2


def _rb(*ts):
    dt = ts[0].dtype
    if dt not in (torch.float32, torch.float64):
        raise TypeError("tensors must be float32 or float64")
    for t in ts:
        if t.dtype != dt:
            raise TypeError("all tensors must have one dtype")
        if not t.is_cuda:
            raise ValueError("tensors must be CUDA tensors (the library has no CPU path)")
        if not t.is_contiguous():
            raise ValueError("tensors must be contiguous")
    return 4 if dt == torch.float32 else 8


def _p(t):
    return C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def observer(A, Cm, E, F, Xi):
    """A [B][N][n][n], C [B][N][p][n], E [B][N][n][nw], F [B][N][p][ne], Xi [B][n][n0] ->
    Pi [B][N+1][n][n], L [B][N][p][n] (L[:, j] = L_{j+1}), PhiX [B][T][n][n], PhiY [B][T][n][p],
    status [B] (int32, CS_ST_NOTPD bits)."""
    rb = _rb(A, Cm, E, F, Xi)
    B, N, n = A.shape[0], A.shape[1], A.shape[2]
    p, nw, ne, n0 = Cm.shape[2], E.shape[3], F.shape[3], Xi.shape[2]
    if (A.shape != (B, N, n, n) or Cm.shape != (B, N, p, n) or E.shape[:3] != (B, N, n)
            or F.shape[:3] != (B, N, p) or Xi.shape[:2] != (B, n)):
        raise ValueError("inconsistent shapes")
    T = n_blocks(N)
    kw = dict(dtype=A.dtype, device=A.device)
    Pi = torch.empty(B, N + 1, n, n, **kw)
    Lg = torch.empty(B, N, p, n, **kw)
    PX = torch.empty(B, T, n, n, **kw)
    PY = torch.empty(B, T, n, p, **kw)
    status = torch.zeros(B, dtype=torch.int32, device=A.device)
    lib = L.lib()
    wsb = lib.sls_observer_workspace(B, N, n, p, rb)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=A.device)
    L.check(lib.sls_observer(B, N, n, p, nw, ne, n0, rb, _p(A), _p(Cm), _p(E), _p(F), _p(Xi), _p(Pi),
                             _p(Lg), _p(PX), _p(PY), _p(status), _p(ws), wsb, _stream()), "sls_observer")
    return Pi, Lg, PX, PY, status


def kalman_scan(A, Cm, E, F, Xi):
    """The covariances Pi [B][N+1][n][n] of observer() by the associative scan of the combination
    rules (logarithmic depth in N) -> (Pi, status)."""
    rb = _rb(A, Cm, E, F, Xi)
    B, N, n = A.shape[0], A.shape[1], A.shape[2]
    p, nw, ne, n0 = Cm.shape[2], E.shape[3], F.shape[3], Xi.shape[2]
    if (A.shape != (B, N, n, n) or Cm.shape != (B, N, p, n) or E.shape[:3] != (B, N, n)
            or F.shape[:3] != (B, N, p) or Xi.shape[:2] != (B, n)):
        raise ValueError("inconsistent shapes")
    Pi = torch.empty(B, N + 1, n, n, dtype=A.dtype, device=A.device)
    status = torch.zeros(B, dtype=torch.int32, device=A.device)
    lib = L.lib()
    wsb = lib.sls_kalman_scan_workspace(B, N, n, p, rb)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=A.device)
    L.check(lib.sls_kalman_scan(B, N, n, p, nw, ne, n0, rb, _p(A), _p(Cm), _p(E), _p(F), _p(Xi), _p(Pi),
                                _p(status), _p(ws), wsb, _stream()), "sls_kalman_scan")
    return Pi, status


def response(Acl):
    """Acl [B][N][n][n] -> Phi [B][T][n][n], Phi_{k,k} = I, Phi_{k,j} = Phi_{k,j+1} Acl_j."""
    rb = _rb(Acl)
    B, N, n = Acl.shape[0], Acl.shape[1], Acl.shape[2]
    Phi = torch.empty(B, n_blocks(N), n, n, dtype=Acl.dtype, device=Acl.device)
    L.check(L.lib().sls_response(B, N, n, rb, _p(Acl), _p(Phi), _stream()), "sls_response")
    return Phi


def closed_loop(A, PBX, PBU, PX, PY):
    """A [B][N][n][n], Phibar^x [B][T][n][n], Phibar^u [B][T][m][n], Phihat^x [B][T][n][n],
    Phihat^y [B][T][n][p] -> Phi^xw [B][T][n][n], Phi^uw [B][T][m][n], Phi^xe [B][T][n][p],
    Phi^ue [B][T][m][p]."""
    rb = _rb(A, PBX, PBU, PX, PY)
    B, N, n = A.shape[0], A.shape[1], A.shape[2]
    T, m, p = n_blocks(N), PBU.shape[2], PY.shape[3]
    if (PBX.shape != (B, T, n, n) or PBU.shape != (B, T, m, n) or PX.shape != (B, T, n, n)
            or PY.shape != (B, T, n, p)):
        raise ValueError("inconsistent shapes")
    kw = dict(dtype=A.dtype, device=A.device)
    XW, UW = torch.empty(B, T, n, n, **kw), torch.empty(B, T, m, n, **kw)
    XE, UE = torch.empty(B, T, n, p, **kw), torch.empty(B, T, m, p, **kw)
    lib = L.lib()
    wsb = lib.sls_closed_loop_workspace(B, N, n, p, rb)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=A.device)
    L.check(lib.sls_closed_loop(B, N, n, m, p, rb, _p(A), _p(PBX), _p(PBU), _p(PX), _p(PY), _p(XW),
                                _p(UW), _p(XE), _p(UE), _p(ws), wsb, _stream()), "sls_closed_loop")
    return XW, UW, XE, UE


def tubes(XW, UW, XE, UE, E, F, Ccon=None, bcon=None, z=None, v=None):
    """Closed-loop maps (as closed_loop returns them), E [B][N][n][nw], F [B][N][p][ne] ->
    tau [B][N+1][n+m] (row-wise tube widths) and, with constraints Ccon [nc][n+m], bcon [nc] and
    the nominal z [B][N+1][n], v [B][N][m], margin [B][N][nc] (else None)."""
    cons = Ccon is not None
    ts = (XW, UW, XE, UE, E, F) + ((Ccon, bcon, z, v) if cons else ())
    rb = _rb(*ts)
    B, T, n = XW.shape[0], XW.shape[1], XW.shape[2]
    N, m, p = E.shape[1], UW.shape[2], XE.shape[3]
    nw, ne = E.shape[3], F.shape[3]
    nc = Ccon.shape[0] if cons else 0
    if (T != n_blocks(N) or UW.shape != (B, T, m, n) or XE.shape != (B, T, n, p) or UE.shape != (B, T, m, p)
            or E.shape[:3] != (B, N, n) or F.shape[:3] != (B, N, p)):
        raise ValueError("inconsistent shapes")
    if cons and (Ccon.shape != (nc, n + m) or bcon.shape != (nc,) or z.shape != (B, N + 1, n)
                 or v.shape != (B, N, m)):
        raise ValueError("inconsistent constraint shapes")
    tau = torch.empty(B, N + 1, n + m, dtype=XW.dtype, device=XW.device)
    margin = torch.empty(B, N, nc, dtype=XW.dtype, device=XW.device) if cons else None
    lib = L.lib()
    wsb = lib.sls_tubes_workspace(B, N, n, m, p, nw, ne, nc, rb)
    ws = torch.empty(max(wsb, 1), dtype=torch.uint8, device=XW.device)
    nul = C.c_void_p(None)
    L.check(lib.sls_tubes(B, N, n, m, p, nw, ne, nc, rb, _p(XW), _p(UW), _p(XE), _p(UE), _p(E), _p(F),
                          *((_p(Ccon), _p(bcon), _p(z), _p(v)) if cons else (nul, nul, nul, nul)),
                          _p(tau), _p(margin) if cons else nul, _p(ws), wsb, _stream()), "sls_tubes")
    return tau, margin


def conformal_radius(q_next, f_pred, delta: float, T: int):
    """q_next, f_pred [n_cal][dim] -> radius (a one-element tensor on the device: the
    ceil((n_cal + 1)(1 - delta / T))-th smallest score, +inf past n_cal) and the scores [n_cal]."""
    rb = _rb(q_next, f_pred)
    if q_next.shape != f_pred.shape or q_next.dim() != 2:
        raise ValueError("q_next and f_pred must be [n_cal][dim] of one shape")
    ncal, dim = q_next.shape
    scores = torch.empty(ncal, dtype=q_next.dtype, device=q_next.device)
    radius = torch.empty(1, dtype=q_next.dtype, device=q_next.device)
    L.check(L.lib().sls_conformal_radius(ncal, dim, rb, _p(q_next), _p(f_pred), float(delta), int(T),
                                         _p(scores), _p(radius), _stream()), "sls_conformal_radius")
    return radius, scores


def unpack(blocks, N: int):
    """Packed [B][T][r][c] -> dense [B][(N+1) r][(N+1) c] block lower-triangular matrices."""
    B, T, r, c = blocks.shape
    if T != n_blocks(N):
        raise ValueError("block count does not match N")
    out = blocks.new_zeros(B, (N + 1) * r, (N + 1) * c)
    t = 0
    for k in range(N + 1):
        for j in range(k + 1):
            out[:, k * r:(k + 1) * r, j * c:(j + 1) * c] = blocks[:, t]
            t += 1
    return out


def pack(dense, N: int, r: int, c: int):
    """Dense [B][(N+1) r][(N+1) c] -> packed [B][T][r][c] (the blocks on and below the diagonal)."""
    B = dense.shape[0]
    out = dense.new_empty(B, n_blocks(N), r, c)
    t = 0
    for k in range(N + 1):
        for j in range(k + 1):
            out[:, t] = dense[:, k * r:(k + 1) * r, j * c:(j + 1) * c]
            t += 1
    return out.contiguous()
