"""Algorithmic floating-point work of the rope hot path (the roofline numerator).

The count is per node and per solver iteration of the algorithm (not of the implementation):
one stage-1 Newton iteration assembles the residual and Hessian, factors the node-coupled matrix
with a banded LDL^T of half bandwidth p = 8 (n (p^2 + 3p) flops for n unknowns) and solves with
it (n (4p + 1)), and evaluates the Armijo merit; one stage-2 barrier iteration adds the contact
terms of every (node, obstacle) pair to the same assembly, factorisation and solve; one adjoint
step is a smooth re-solve plus two solves and the VJP products.  Iteration counts come from the
FP64 oracle on the same inputs, so extra iterations of the GPU earn no credit.

Per-operation counts (flops, an FMA counted as 2) of the formulas the method evaluates:
  spring force + 3x3 Hessian block ......................... 40
  scatter of a spring block into the matrix (4 blocks) ..... 36
  residual / matvec of one spring ........................... 24
  contact pair: signed distance, normal, force and 3x3 W ... 60
  contact pair: barrier merit evaluation .................... 25
  spring third-derivative contraction ....................... 30
  contact pair adjoint product ............................. 70
  contact pair: predictor step, scaling, second-order term .. 90
A predictor-corrector barrier iteration of the nonsmooth stage 2 adds a second solve with the same
factorisation, a second residual and the per-pair predictor terms.
"""
from __future__ import annotations

P_BAND = 8                          # scalar half bandwidth of a rope's node-coupled matrix
FACT_PER_DOF = P_BAND * P_BAND + 3 * P_BAND    # banded LDL^T
SOLVE_PER_DOF = 4 * P_BAND + 1


def newton_iter_per_node(springs_per_node: float = 2.0) -> float:
    assembly = springs_per_node * (40 + 36) + 10
    linalg = 3 * (FACT_PER_DOF + SOLVE_PER_DOF)
    merit = 1.5 * (springs_per_node * 24 + 12)     # ~1.5 Armijo evaluations per iteration
    return assembly + linalg + merit


def barrier_iter_per_node(nobs: int, springs_per_node: float = 2.0) -> float:
    assembly = springs_per_node * (40 + 36 + 24) + 10 + nobs * 60
    linalg = 3 * (FACT_PER_DOF + SOLVE_PER_DOF)
    merit = 1.5 * (springs_per_node * 24 + nobs * 25)
    return assembly + linalg + merit


def pc_barrier_iter_per_node(nobs: int, springs_per_node: float = 2.0) -> float:
    """barrier iteration of the nonsmooth stage 2 (Mehrotra predictor-corrector)"""
    extra = 3 * SOLVE_PER_DOF + springs_per_node * 24 + nobs * 90
    return barrier_iter_per_node(nobs, springs_per_node) + extra


def adjoint_per_node(nobs: int, springs_per_node: float = 2.0) -> float:
    solves = 2 * 3 * SOLVE_PER_DOF
    refactor = 3 * FACT_PER_DOF + springs_per_node * (40 + 36)
    vjp = springs_per_node * 30 + nobs * 70 + 12
    return solves + refactor + vjp


def rollout_vjp_flops_per_node_step(counts: dict, nobs: int, k: int) -> float:
    """counts: mean per step of the oracle's iterations over the sampled rollouts:
      fwd_newton, fwd_ipm   (nonsmooth forward),
      sm_newton, sm_ipm     (smooth re-solve of the backward).
    The forward is run twice except at checkpoints (recompute of k-1 of every k steps)."""
    fwd = counts["fwd_newton"] * newton_iter_per_node() + counts["fwd_ipm"] * pc_barrier_iter_per_node(nobs)
    recompute = fwd * (k - 1) / k
    back = counts["sm_newton"] * newton_iter_per_node() + counts["sm_ipm"] * barrier_iter_per_node(nobs) \
        + adjoint_per_node(nobs)
    return fwd + recompute + back


# ---- cloth: the node-coupled matrices are banded with scalar half bandwidth p = 3 span + 2
#      (span = 2 C for C columns); a cloth node has about 5.7 springs (structural, shear, bend)

def cloth_band(cols: int) -> int:
    return 3 * 2 * cols + 2


def cloth_springs_per_node(rows: int, cols: int) -> float:
    n = rows * cols
    s = rows * (cols - 1) + (rows - 1) * cols + 2 * (rows - 1) * (cols - 1) + rows * max(cols - 2, 0) \
        + max(rows - 2, 0) * cols
    return s / n


def band_factor_per_node(p: int) -> float:
    return 3 * (p * p + 3 * p)


def band_solve_per_node(p: int) -> float:
    return 3 * (4 * p + 1)


def cloth_newton_iter_per_node(p: int, spn: float) -> float:
    return spn * (40 + 36) + 10 + band_factor_per_node(p) + band_solve_per_node(p) + 1.5 * (spn * 24 + 12)


def cloth_pc_barrier_iter_per_node(p: int, spn: float, nobs: int) -> float:
    return spn * (40 + 36 + 24) + 10 + nobs * (60 + 90) + band_factor_per_node(p) + \
        2 * band_solve_per_node(p) + 1.5 * (spn * 24 + nobs * 25)


def cloth_barrier_iter_per_node(p: int, spn: float, nobs: int) -> float:
    """barrier iteration of the smooth stage 2 (fixed target, one solve)"""
    return spn * (40 + 36 + 24) + 10 + nobs * 60 + band_factor_per_node(p) + band_solve_per_node(p) + \
        1.5 * (spn * 24 + nobs * 25)


def cloth_rollout_vjp_flops_per_node_step(counts: dict, p: int, spn: float, nobs: int, k: int) -> float:
    """counts: mean iterations per step: fwd_newton, fwd_ipm (nonsmooth forward) and, when given,
    sm_newton, sm_ipm (the smooth re-solve of the backward).  Forward, the recompute of k-1 of
    every k steps, and a backward step: the smooth re-solve (at its minimum, one Newton iteration,
    without its counts), the factorisation of the adjoint's dF/dq*, two solves and the VJP products
    (spring third derivatives, contact terms).  Shift retries of the stage-1 factorisation are not
    counted."""
    fwd = counts["fwd_newton"] * cloth_newton_iter_per_node(p, spn) + \
        counts["fwd_ipm"] * cloth_pc_barrier_iter_per_node(p, spn, nobs)
    if "sm_newton" in counts:
        resolve = counts["sm_newton"] * cloth_newton_iter_per_node(p, spn) + \
            counts["sm_ipm"] * cloth_barrier_iter_per_node(p, spn, nobs)
    else:
        resolve = cloth_newton_iter_per_node(p, spn)
    back = resolve + band_factor_per_node(p) + 2 * band_solve_per_node(p) + spn * 30 + nobs * 70 + 12
    return fwd + fwd * (k - 1) / k + back


# ------------------------------------------------------------------------------------------
# output-feedback SLS observer stage (Sec. 4.2): dense products of the formulas as written,
# 2 r c k flops for an (r x k)(k x c) product; a Cholesky factorisation of a p x p matrix p^3 / 3,
# its two triangular solves with c right-hand sides 2 p^2 c
# ------------------------------------------------------------------------------------------

def _mm(r, c, k):
    return 2.0 * r * c * k


def sls_observer_flops(N: int, n: int, p: int, nw: int, ne: int, n0: int) -> float:
    """One trajectory of sls_observer: eq. kalman_recursions step by step (Pi C^T, C Pi C^T,
    F F^T, A Pi C^T, A Pi A^T, E E^T, the gain solve, A Pi C^T L), the closed-loop matrices
    A + L^T C, the N (N + 1) / 2 products of eq. backward_propagations and Phihat^y = Phihat^x L^T."""
    per_step = (_mm(n, p, n) + _mm(p, p, n) + _mm(p, p, ne) + _mm(n, p, n) + 2 * _mm(n, n, n)
                + _mm(n, n, nw) + p ** 3 / 3.0 + 2.0 * p * p * n + _mm(n, n, p) + _mm(n, n, p))
    tri = N * (N + 1) / 2.0
    return _mm(n, n, n0) + N * per_step + tri * _mm(n, n, n) + tri * _mm(n, p, n)


def sls_closed_loop_flops(N: int, n: int, m: int, p: int) -> float:
    """One trajectory of sls_closed_loop: M Phihat^x and M Phihat^y (one block product per block
    below the diagonal), then the block lower-triangular products Phibar^x (M Phihat^x),
    Phibar^u (M Phihat^x), Phibar^x (M Phihat^y), Phibar^u (M Phihat^y), block (k, j) summing
    k - j + 1 block products."""
    tri = N * (N + 1) / 2.0
    s3 = sum((N + 1 - d) * (d + 1) for d in range(N + 1))
    return (tri * (_mm(n, n, n) + _mm(n, p, n))
            + s3 * (_mm(n, n, n) + _mm(m, n, n) + _mm(n, p, n) + _mm(m, p, n)))


def sls_tubes_flops(N: int, n: int, m: int, p: int, nw: int, ne: int, nc: int) -> float:
    """One trajectory of sls_tubes: the products Phi_{k,j} E_{j-1}, Phi_{k,j} F_{j-1} of the blocks
    below the diagonal with their row sums of squares; for nc constraints the rows
    C [Phi^x; Phi^u] of every block and their products with E, F."""
    tri = N * (N + 1) / 2.0
    T = (N + 1) * (N + 2) / 2.0
    tubes = tri * ((_mm(n, nw, n) + _mm(m, nw, n)) + (_mm(n, ne, p) + _mm(m, ne, p)) + 2.0 * (n + m) * (nw + ne))
    cons = T * (_mm(nc, n, n) + _mm(nc, n, m) + _mm(nc, p, n) + _mm(nc, p, m)) + \
        tri * (_mm(nc, nw, n) + _mm(nc, ne, p) + 2.0 * nc * (nw + ne))
    return tubes + (cons if nc > 0 else 0.0)
