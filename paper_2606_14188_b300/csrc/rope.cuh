// Rope (particle chain) kernels: one warp per rollout for the whole horizon.  Node pair
// p = lane + 32 k (nodes 2p, 2p+1) lives in registers of its lane (slot k < PPL); the springs to
// the neighbouring pairs read their nodes through warp shuffles; the pair-block matrices and the
// contact variables live in element-major shared memory (lane-contiguous, conflict free).
//
// One step (arxiv 2606.14188, Sec. 4.1, "Simulation Solver"):
//   stage 1  Newton for q* with F(q*) = M(q*-q)/dt^2 + dE(q*) - tau(u) + sum_i d_i (x*_a - g*_i) = 0
//            (eq. dynamics-first-stage; kinematic grippers g* = g + u; d_i the grasp stiffness,
//            D_max 1[|c_i| <= r_grasp] nonsmooth, D_max exp(-|c_i|/kappa_h) smooth);
//   stage 2  Delta = argmin 1/2 Delta^T P Delta over the dual friction cones (eq.
//            dynamics-second-stage) by a primal-dual interior point whose central path at kappa is
//            the relaxed complementarity s^T lam = kappa (Sec. 4.1 "Contact Smoothing"): fixed
//            kappa_c (smooth) or followed down to kappa_hard (nonsmooth; skipped when no pair
//            penetrates, where Delta = 0 is exact).
// Newton iterates are offsets dx from the step's start x0 (x* = x0 + dx), and the grasp offsets
// c_i = g_i - x_a(i) are carried from step to step as sums of small increments, so that stiff
// springs see no absolute-coordinate cancellation in FP32.
#pragma once
#include "common.cuh"
#include "cr.cuh"

namespace cs {

// ------------------------------------------------------------------------------------------
// shared-memory layout of one warp
// ------------------------------------------------------------------------------------------
template <typename R>
struct WS {
  int NP;                     // pair slots (32 PPL)
  R *T, *B, *V, *r;           // cyclic-reduction storage, row strides CR_LDT, CR_LDM, CR_LDM, CR_LDV
  R *s, *z, *phi, *nrm;       // contact pairs: [(o*2+h)*3+c][NP] for vectors, [(o*2+h)][NP]
  R *pm, *pg, *prz;           // per-pair Newton terms of the current iteration: M (6), g (3), r_z (3)
  R *misc;                    // [64]
  R *u, *ub;                  // controls and their adjoint [6 H]
  // linearisation only
  R *T2, *B2, *V2;            // second factorisation
  R *xs, *Dn;                 // x* - x0 and Delta of every node [6][NP]
};

enum {
  M_G = 0,      // g [6]   gripper positions at the step start
  M_U = 6,      // u [6]   control of the step
  M_C = 12,     // c [6]   c_i = g_i - x0_a(i), carried across steps
  M_D = 18,     // d [2]   grasp stiffness
  M_GD = 20,    // gd [6]  d d_i / d c_i (smooth)
  M_GB = 26,    // gbar [6] adjoint of the gripper positions
  M_UB = 32,    // ubar [6] adjoint of the control (one step)
};

__host__ __device__ inline size_t ws_size(int NP, int nobs, int H, bool lin) {
  size_t s = (size_t)NP * (CR_LDT + 2 * CR_LDM + CR_LDV) + (size_t)nobs * 2 * NP * 22 + 64;
  s = ((s + 3) & ~(size_t)3) + 12 * (size_t)H;
  if (lin) s += (size_t)NP * (CR_LDT + 2 * CR_LDM) + 2 * 6 * (size_t)NP;
  return s;
}

template <typename R>
__device__ __forceinline__ WS<R> ws_carve(R* base, int NP, int nobs, int H, bool lin) {
  WS<R> w;
  w.NP = NP;
  R* p = base;
  auto take = [&](size_t n) { R* q = p; p += n; return q; };
  w.T = take(CR_LDT * (size_t)NP); w.B = take(CR_LDM * (size_t)NP); w.V = take(CR_LDM * (size_t)NP);
  w.r = take(CR_LDV * (size_t)NP);
  w.s = take((size_t)nobs * 2 * 3 * NP); w.z = take((size_t)nobs * 2 * 3 * NP);
  w.phi = take((size_t)nobs * 2 * NP); w.nrm = take((size_t)nobs * 2 * 3 * NP);
  w.pm = take((size_t)nobs * 2 * 6 * NP); w.pg = take((size_t)nobs * 2 * 3 * NP);
  w.prz = take((size_t)nobs * 2 * 3 * NP);
  w.misc = take(64);
  p = base + (((size_t)(p - base) + 3) & ~(size_t)3);
  w.u = take(6 * (size_t)H); w.ub = take(6 * (size_t)H);
  if (lin) {
    w.T2 = take(CR_LDT * (size_t)NP); w.B2 = take(CR_LDM * (size_t)NP); w.V2 = take(CR_LDM * (size_t)NP);
    w.xs = take(6 * (size_t)NP); w.Dn = take(6 * (size_t)NP);
  } else {
    w.T2 = w.B2 = w.V2 = w.xs = w.Dn = nullptr;
  }
  return w;
}

// checkpoint record of a state: q [n_q] | c [6] | dx [3 nv] | Delta [3 nv] (grasp offsets, and
// the stage-1 offset and stage-2 displacement of the step that produced the state)
__host__ __device__ inline int rec_len(int nv) { return 3 * nv + 6 + 6 + 6 * nv; }
// the record of the CTA kernels (rope_cta.cuh): the same, then (inertial variant) the velocities
// [3 nv]
__host__ __device__ inline int rec_len_rc(int nv, int so) { return rec_len(nv) + (so ? 3 * nv : 0); }

// contact-pair element addresses
__device__ __forceinline__ int cv(int o, int h, int c, int p, int NP) { return ((o * 2 + h) * 3 + c) * NP + p; }
__device__ __forceinline__ int cs1(int o, int h, int p, int NP) { return (o * 2 + h) * NP + p; }
__device__ __forceinline__ int cm6(int o, int h, int c, int p, int NP) { return ((o * 2 + h) * 6 + c) * NP + p; }

// ------------------------------------------------------------------------------------------
// per-lane register state
// ------------------------------------------------------------------------------------------
template <typename R, int PPL>
struct Lane {
  R x0[PPL][6];               // own pair at the step start
  R xm[PPL][6], xp[PPL][6];   // neighbouring pairs (p - 1, p + 1) at the step start
  R dx[PPL][6];               // x* - x0
  R Dl[PPL][6];               // Delta (stage 2)
  R pv[PPL][6];               // step / work vector
  R F[PPL][6];                // residual
  R Ls[PPL][3];               // rest lengths (2p-1,2p), (2p,2p+1), (2p+1,2p+2)
  R Lb[PPL][4];               // rest lengths (2p-2,2p), (2p-1,2p+1), (2p,2p+2), (2p+1,2p+3)
};

// every register array of the lane starts at zero: slots past the chain (p >= npair) are never
// assembled but take part in warp reductions (max step, slope) and must contribute nothing
template <typename R, int PPL>
__device__ __forceinline__ void zero_lane(Lane<R, PPL>& L) {
#pragma unroll
  for (int k = 0; k < PPL; ++k)
#pragma unroll
    for (int e = 0; e < 6; ++e)
      L.x0[k][e] = L.xm[k][e] = L.xp[k][e] = L.dx[k][e] = L.Dl[k][e] = L.pv[k][e] = L.F[k][e] = R(0);
}

// value of the neighbouring pairs p - 1 and p + 1 of every slot
template <typename R, int PPL>
__device__ __forceinline__ void nbr(const R v[PPL][6], R vm[PPL][6], R vp[PPL][6], int lane) {
#pragma unroll
  for (int k = 0; k < PPL; ++k)
#pragma unroll
    for (int e = 0; e < 6; ++e) {
      const R up = __shfl_up_sync(FULL, v[k][e], 1);
      const R dn = __shfl_down_sync(FULL, v[k][e], 1);
      R wm = R(0), wp = R(0);
      if (k > 0) wm = __shfl_sync(FULL, v[k > 0 ? k - 1 : 0][e], 31);
      if (k + 1 < PPL) wp = __shfl_sync(FULL, v[k + 1 < PPL ? k + 1 : 0][e], 0);
      vm[k][e] = lane == 0 ? wm : up;
      vp[k][e] = lane == 31 ? wp : dn;
    }
}

template <typename R, int PPL>
__device__ __forceinline__ void zero6(R v[PPL][6]) {
#pragma unroll
  for (int k = 0; k < PPL; ++k)
#pragma unroll
    for (int e = 0; e < 6; ++e) v[k][e] = R(0);
}

// The seven springs touching pair p, sid 0..6:
//   (2p-1,2p) (2p,2p+1) (2p+1,2p+2) stretch;  (2p-2,2p) (2p-1,2p+1) (2p,2p+2) (2p+1,2p+3) bend.
// For node a and b of spring sid: where (0 previous pair, 1 own pair, 2 next pair) and h.
__host__ __device__ constexpr int spr_wa(int s) { return (s == 0 || s == 3 || s == 4) ? 0 : 1; }
__host__ __device__ constexpr int spr_ha(int s) { return (s == 0 || s == 2 || s == 4 || s == 6) ? 1 : 0; }
__host__ __device__ constexpr int spr_wb(int s) { return (s == 2 || s == 5 || s == 6) ? 2 : 1; }
__host__ __device__ constexpr int spr_hb(int s) { return (s == 1 || s == 4 || s == 6) ? 1 : 0; }

__host__ __device__ constexpr int spr_node(int p, int where, int h) { return 2 * p + 2 * (where - 1) + h; }

template <typename R, int PPL>
__device__ __forceinline__ R pick(const R own[PPL][6], const R m[PPL][6], const R n[PPL][6],
                                  int k, int where, int e) {
  return where == 0 ? m[k][e] : (where == 1 ? own[k][e] : n[k][e]);
}

template <typename R, int PPL>
__device__ __forceinline__ void spring_rest(const Lane<R, PPL>& L, int k, int sid, R& kk, R& Lr,
                                            const Scene<R>& S) {
  if (sid < 3) { kk = S.k1; Lr = L.Ls[k][sid]; } else { kk = S.k2; Lr = L.Lb[k][sid - 3]; }
}

template <typename R, int PPL>
__device__ __forceinline__ void load_rest(const Scene<R>& S, Lane<R, PPL>& L, int lane) {
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
    for (int i = 0; i < 3; ++i) {
      const int a = 2 * p - 1 + i;
      L.Ls[k][i] = (a >= 0 && a + 1 < S.nv) ? S.L1[a] : R(1);
    }
    for (int i = 0; i < 4; ++i) {
      const int a = 2 * p - 2 + i;
      L.Lb[k][i] = (a >= 0 && a + 2 < S.nv) ? S.L2[a] : R(1);
    }
  }
}

// ------------------------------------------------------------------------------------------
// stage-1 assembly: T (lower 6x6), coupling B to pair p - 1, residual F of pair p (slot k).
// dxm/dxp: neighbours' dx.  grasp offsets and stiffness from misc.
// ------------------------------------------------------------------------------------------
template <typename R, int PPL>
__device__ __forceinline__ void assemble1(const Scene<R>& S, const Lane<R, PPL>& L, const R dxm[PPL][6],
                          const R dxp[PPL][6], const R* misc, int k, int p, bool proj,
                          R T[36], R Bc[36], R F[6]) {
#pragma unroll
  for (int e = 0; e < 36; ++e) { T[e] = R(0); Bc[e] = R(0); }
  const R* d = misc + M_D;
  const R* c = misc + M_C;
  const R* u = misc + M_U;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = 2 * p + h;
    if (j >= S.nv) {
      for (int i = 0; i < 3; ++i) { T[(3 * h + i) * 7] = R(1); F[3 * h + i] = R(0); }
      continue;
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      T[(3 * h + i) * 7] = S.w;
      F[3 * h + i] = S.w * L.dx[k][3 * h + i] - S.m * S.grav[i];
    }
#pragma unroll
    for (int gi = 0; gi < 2; ++gi)
      if (S.grasp[gi] == j) {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          T[(3 * h + i) * 7] += d[gi];
          F[3 * h + i] += d[gi] * (L.dx[k][3 * h + i] - (c[3 * gi + i] + u[3 * gi + i]));
        }
      }
  }
#pragma unroll
  for (int sid = 0; sid < 7; ++sid) {
    const int wa = spr_wa(sid), ha = spr_ha(sid), wb = spr_wb(sid), hb = spr_hb(sid);
    const int a = spr_node(p, wa, ha), b = spr_node(p, wb, hb);
    if (a < 0 || b >= S.nv) continue;
    R kk, Lr;
    spring_rest(L, k, sid, kk, Lr, S);
    R dv[3], f[3], H[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      dv[i] = (pick<R, PPL>(L.x0, L.xm, L.xp, k, wb, 3 * hb + i) - pick<R, PPL>(L.x0, L.xm, L.xp, k, wa, 3 * ha + i)) +
              (pick<R, PPL>(L.dx, dxm, dxp, k, wb, 3 * hb + i) - pick<R, PPL>(L.dx, dxm, dxp, k, wa, 3 * ha + i));
    spring_eval(dv, kk, Lr, proj, f, H);
    if (wa == 1) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        F[3 * ha + i] -= f[i];
#pragma unroll
        for (int q = 0; q <= i; ++q) T[(3 * ha + i) * 6 + 3 * ha + q] += H[i * 3 + q];
      }
    }
    if (wb == 1) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        F[3 * hb + i] += f[i];
#pragma unroll
        for (int q = 0; q <= i; ++q) T[(3 * hb + i) * 6 + 3 * hb + q] += H[i * 3 + q];
      }
    }
    if (wa == 1 && wb == 1) {          // (2p, 2p+1): lower block row hb = 1, column ha = 0
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 3; ++q) T[(3 * hb + i) * 6 + 3 * ha + q] -= H[i * 3 + q];
    } else if (wb == 1 && wa == 0) {   // coupling with the previous pair
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 3; ++q) Bc[(3 * hb + i) * 6 + 3 * ha + q] -= H[i * 3 + q];
    }
  }
}

// y = P v for pair p (P = exact or projected stage-1 Hessian at x0 + dx)
template <typename R, int PPL>
__device__ __forceinline__ void hessvec(const Scene<R>& S, const Lane<R, PPL>& L, const R dxm[PPL][6],
                        const R dxp[PPL][6], const R v[PPL][6], const R vm[PPL][6],
                        const R vp[PPL][6], const R* misc, int k, int p, bool proj, R y[6]) {
  const R* d = misc + M_D;
#pragma unroll
  for (int h = 0; h < 2; ++h) {
    const int j = 2 * p + h;
#pragma unroll
    for (int i = 0; i < 3; ++i) y[3 * h + i] = j < S.nv ? S.w * v[k][3 * h + i] : R(0);
#pragma unroll
    for (int gi = 0; gi < 2; ++gi)
      if (S.grasp[gi] == j)
#pragma unroll
        for (int i = 0; i < 3; ++i) y[3 * h + i] += d[gi] * v[k][3 * h + i];
  }
#pragma unroll
  for (int sid = 0; sid < 7; ++sid) {
    const int wa = spr_wa(sid), ha = spr_ha(sid), wb = spr_wb(sid), hb = spr_hb(sid);
    const int a = spr_node(p, wa, ha), b = spr_node(p, wb, hb);
    if (a < 0 || b >= S.nv) continue;
    R kk, Lr;
    spring_rest(L, k, sid, kk, Lr, S);
    R dv[3], f[3], H[9], dd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dv[i] = (pick<R, PPL>(L.x0, L.xm, L.xp, k, wb, 3 * hb + i) - pick<R, PPL>(L.x0, L.xm, L.xp, k, wa, 3 * ha + i)) +
              (pick<R, PPL>(L.dx, dxm, dxp, k, wb, 3 * hb + i) - pick<R, PPL>(L.dx, dxm, dxp, k, wa, 3 * ha + i));
      dd[i] = pick<R, PPL>(v, vm, vp, k, wb, 3 * hb + i) - pick<R, PPL>(v, vm, vp, k, wa, 3 * ha + i);
    }
    spring_eval(dv, kk, Lr, proj, f, H);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const R hv = H[i * 3] * dd[0] + H[i * 3 + 1] * dd[1] + H[i * 3 + 2] * dd[2];
      if (wb == 1) y[3 * hb + i] += hv;
      if (wa == 1) y[3 * ha + i] -= hv;
    }
  }
}

template <typename R>
__device__ __forceinline__ void put_rows(WS<R>& w, int p, const R T[36], const R Bc[36]) {
  st_lower(w.T, p, T);
  st36(w.B, p, Bc);
}

// ------------------------------------------------------------------------------------------
// stage 1
// ------------------------------------------------------------------------------------------
template <typename R, int PPL>
__device__ __forceinline__ R psi_diff(const Scene<R>& S, const Lane<R, PPL>& L, const R dxp[PPL][6],
                      const R pvp[PPL][6], const R* misc, R alpha, int lane) {
  const R* d = misc + M_D;
  const R* c = misc + M_C;
  const R* u = misc + M_U;
  R val = R(0);
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * p + h;
      if (j >= S.nv) continue;
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const R D = alpha * L.pv[k][3 * h + i];
        val += R(0.5) * S.w * D * (R(2) * L.dx[k][3 * h + i] + D) - S.m * S.grav[i] * D;
      }
#pragma unroll
      for (int gi = 0; gi < 2; ++gi)
        if (S.grasp[gi] == j)
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            const R D = alpha * L.pv[k][3 * h + i];
            val += R(0.5) * d[gi] * D * (D - R(2) * ((c[3 * gi + i] + u[3 * gi + i]) - L.dx[k][3 * h + i]));
          }
    }
    // springs whose first node is in pair p: sid 1, 2, 5, 6
#pragma unroll
    for (int t = 0; t < 4; ++t) {
      const int sid = t < 2 ? 1 + t : 3 + t;
      const int wa = spr_wa(sid), ha = spr_ha(sid), wb = spr_wb(sid), hb = spr_hb(sid);
      const int a = spr_node(p, wa, ha), b = spr_node(p, wb, hb);
      if (a < 0 || b >= S.nv) continue;
      R kk, Lr;
      spring_rest(L, k, sid, kk, Lr, S);
      R dX[3], dD[3], dY[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const R xb = wb == 1 ? L.x0[k][3 * hb + i] : L.xp[k][3 * hb + i];
        const R db = wb == 1 ? L.dx[k][3 * hb + i] : dxp[k][3 * hb + i];
        const R pb = wb == 1 ? L.pv[k][3 * hb + i] : pvp[k][3 * hb + i];
        dX[i] = (xb - L.x0[k][3 * ha + i]) + (db - L.dx[k][3 * ha + i]);
        dD[i] = alpha * (pb - L.pv[k][3 * ha + i]);
        dY[i] = dX[i] + dD[i];
      }
      const R lX = sqrt(dot3(dX, dX)), lY = sqrt(dot3(dY, dY));
      const R dl = (dD[0] * (R(2) * dX[0] + dD[0]) + dD[1] * (R(2) * dX[1] + dD[1]) +
                    dD[2] * (R(2) * dX[2] + dD[2])) / (lY + lX);
      val += R(0.5) * kk * dl * (lY + lX - R(2) * Lr);
    }
  }
  return val;
}

// registers -> CR right-hand side (zero rows for nodes past the chain)
template <typename R, int PPL>
__device__ __forceinline__ void put_rhs(const Scene<R>& S, WS<R>& w, const R v[PPL][6], R sign, int lane) {
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
    if (p >= S.npair) continue;
#pragma unroll
    for (int e = 0; e < 6; ++e) w.r[cr_v(p, e)] = (2 * p + e / 3 < S.nv) ? sign * v[k][e] : R(0);
  }
}

template <typename R, int PPL>
__device__ __forceinline__ void get_rhs(const Scene<R>& S, const WS<R>& w, R v[PPL][6], int lane) {
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int e = 0; e < 6; ++e) v[k][e] = (p < S.npair && 2 * p + e / 3 < S.nv) ? w.r[cr_v(p, e)] : R(0);
  }
}

// assemble P = dF/dq* at x0 + dx into the CR arrays (optionally keeping the residual in L.F)
template <typename R, int PPL>
__device__ __forceinline__ void assemble_P(const Scene<R>& S, Lane<R, PPL>& L, WS<R>& w, const R dxm[PPL][6],
                           const R dxp[PPL][6], bool proj, bool keepF, int lane) {
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
    if (p >= S.npair) {
      if (keepF)
#pragma unroll
        for (int e = 0; e < 6; ++e) L.F[k][e] = R(0);
      continue;
    }
    R T[36], Bc[36], F[6];
    assemble1(S, L, dxm, dxp, w.misc, k, p, proj, T, Bc, F);
    put_rows(w, p, T, Bc);
    if (keepF)
#pragma unroll
      for (int e = 0; e < 6; ++e) L.F[k][e] = F[e];
  }
}

// Damped Newton for stage 1 from dx = 0.  On exit the factorisation of the Hessian at the last
// iterate is in (T, B, V).
template <typename R, int PPL>
__device__ __forceinline__ int stage1_newton(const Scene<R>& S, Lane<R, PPL>& L, WS<R>& w, int lane, int* iters,
                                             bool warm) {
  if (!warm) {
    // start at the step's initial state with each grasped node moved with its gripper
    zero6<R, PPL>(L.dx);
#pragma unroll
    for (int k = 0; k < PPL; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h)
#pragma unroll
        for (int gi = 0; gi < 2; ++gi)
          if (S.grasp[gi] == 2 * (lane + 32 * k) + h)
#pragma unroll
            for (int i = 0; i < 3; ++i) L.dx[k][3 * h + i] = w.misc[M_U + 3 * gi + i];
  }
  R dxm[PPL][6], dxp[PPL][6];
  for (int it = 0; it < S.newton_max; ++it) {
    nbr<R, PPL>(L.dx, dxm, dxp, lane);
    bool ok = false, exact = false;
    // exact Hessian; if it is not positive definite, the projected one (same call site)
    for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
      assemble_P(S, L, w, dxm, dxp, attempt == 1, attempt == 0, lane);
      if (attempt == 0) put_rhs<R, PPL>(S, w, L.F, R(-1), lane);
      __syncwarp();
      ok = cr_factor(w.T, w.B, w.V, S.npair, lane);
      exact = ok && attempt == 0;
    }
    if (!ok) { *iters = it + 1; return ST_NOTPD; }
    cr_solve(w.T, w.B, w.V, w.r, S.npair, lane);
    get_rhs<R, PPL>(S, w, L.pv, lane);
    R pm = R(0), sl = R(0);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < PPL; ++k)
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        const R pv = L.pv[k][e];
        bad = bad || !(fabs(pv) <= R(1e30));
        pm = fmax(pm, fabs(pv));
        sl += L.F[k][e] * pv;
      }
    pm = wmax(pm);
    sl = wsum(sl);
    if (__any_sync(FULL, bad)) { *iters = it + 1; return ST_NONFINITE; }
    // converged only on an exact-Hessian step: the root is a local minimiser of the potential
    if (pm <= S.ntol && exact) {
#pragma unroll
      for (int k = 0; k < PPL; ++k)
#pragma unroll
        for (int e = 0; e < 6; ++e) L.dx[k][e] += L.pv[k][e];
      *iters = it + 1;
      return 0;
    }
    R pvm[PPL][6], pvp[PPL][6];
    nbr<R, PPL>(L.pv, pvm, pvp, lane);
    R alpha = R(1);
    for (int ls = 0; ls < 40; ++ls) {
      const R dv = wsum(psi_diff(S, L, dxp, pvp, w.misc, alpha, lane));
      if (dv <= R(1e-4) * alpha * sl) break;
      alpha *= R(0.5);
    }
#pragma unroll
    for (int k = 0; k < PPL; ++k)
#pragma unroll
      for (int e = 0; e < 6; ++e) L.dx[k][e] += alpha * L.pv[k][e];
  }
  *iters = S.newton_max;
  return ST_NEWTON;
}

// ------------------------------------------------------------------------------------------
// stage 2
// ------------------------------------------------------------------------------------------

// phi, n of the lane's (node, obstacle) pairs at x* = x0 + dx; returns the warp's min phi
template <typename R, int PPL>
__device__ __forceinline__ R contact_geometry(const Scene<R>& S, const Lane<R, PPL>& L, WS<R>& w, int lane) {
  R pmin = R(1e30);
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (2 * p + h >= S.nv) continue;
      R X[3] = {L.x0[k][3 * h] + L.dx[k][3 * h], L.x0[k][3 * h + 1] + L.dx[k][3 * h + 1],
                L.x0[k][3 * h + 2] + L.dx[k][3 * h + 2]};
      for (int o = 0; o < S.nobs; ++o) {
        R ph, n[3];
        obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, (R*)nullptr);
        w.phi[cs1(o, h, p, w.NP)] = ph;
#pragma unroll
        for (int i = 0; i < 3; ++i) w.nrm[cv(o, h, i, p, w.NP)] = n[i];
        pmin = fmin(pmin, ph);
      }
    }
  }
  return -wmax(-pmin);
}

template <typename R>
__device__ __forceinline__ void pair_frame(const WS<R>& w, int o, int h, int p, R mu, R A[9]) {
  R n[3] = {w.nrm[cv(o, h, 0, p, w.NP)], w.nrm[cv(o, h, 1, p, w.NP)], w.nrm[cv(o, h, 2, p, w.NP)]};
  cone_frame(n, mu, A);
}

// per pair: A, M = W^-2, r_z = s - A D - phi e1, W d_s with d_s = lam^{-1} o (target e - lam o lam)
template <typename R>
__device__ __forceinline__ void pair_terms(const Scene<R>& S, const WS<R>& w, int o, int h, int p,
                                           const R D[3], R target, R A[9], R M[9], R rz[3],
                                           R Wds[3]) {
  pair_frame(w, o, h, p, S.mu, A);
  R s[3], z[3];
#pragma unroll
  for (int c = 0; c < 3; ++c) { s[c] = w.s[cv(o, h, c, p, w.NP)]; z[c] = w.z[cv(o, h, c, p, w.NP)]; }
  const R ph = w.phi[cs1(o, h, p, w.NP)];
#pragma unroll
  for (int a = 0; a < 3; ++a)
    rz[a] = s[a] - (A[a * 3] * D[0] + A[a * 3 + 1] * D[1] + A[a * 3 + 2] * D[2]) - (a == 0 ? ph : R(0));
  R W[9], Wi[9], lam[3];
  nt_scaling(s, z, W, Wi, lam);
  R rhs[3] = {target - (lam[0] * lam[0] + lam[1] * lam[1] + lam[2] * lam[2]), R(-2) * lam[0] * lam[1],
              R(-2) * lam[0] * lam[2]};
  R ds[3];
  jordan_solve(lam, rhs, ds);
#pragma unroll
  for (int a = 0; a < 3; ++a) Wds[a] = W[a * 3] * ds[0] + W[a * 3 + 1] * ds[1] + W[a * 3 + 2] * ds[2];
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      M[a * 3 + b] = Wi[a * 3] * Wi[b] + Wi[a * 3 + 1] * Wi[3 + b] + Wi[a * 3 + 2] * Wi[6 + b];
}

// step of one pair from dD (the node's Delta step) with the terms stored by the assembly:
// ds = A dD - r_z, dz = M (g - A dD), g = r_z + W d_s
template <typename R>
__device__ __forceinline__ void pair_step(const Scene<R>& S, const WS<R>& w, int o, int h, int p,
                                          const R dD[3], R dsv[3], R dz[3]) {
  R A[9];
  pair_frame(w, o, h, p, S.mu, A);
  const int NP = w.NP;
  R m6[6];
#pragma unroll
  for (int c = 0; c < 6; ++c) m6[c] = w.pm[cm6(o, h, c, p, NP)];
  const R M[9] = {m6[0], m6[1], m6[2], m6[1], m6[3], m6[4], m6[2], m6[4], m6[5]};
  R g[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R ADd = A[a * 3] * dD[0] + A[a * 3 + 1] * dD[1] + A[a * 3 + 2] * dD[2];
    dsv[a] = ADd - w.prz[cv(o, h, a, p, NP)];
    g[a] = w.pg[cv(o, h, a, p, NP)] - ADd;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) dz[a] = M[a * 3] * g[0] + M[a * 3 + 1] * g[1] + M[a * 3 + 2] * g[2];
}

// diagonal 3x3 block of P for node (k, h): w I + grasp + incident spring Hessians
template <typename R, int PPL>
__device__ __forceinline__ void diag_block(const Scene<R>& S, const Lane<R, PPL>& L, const R dxm[PPL][6],
                           const R dxp[PPL][6], const R* misc, int k, int p, int h, R D[9]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) D[i] = R(0);
  const int j = 2 * p + h;
  for (int i = 0; i < 3; ++i) D[i * 4] = S.w;
  for (int gi = 0; gi < 2; ++gi)
    if (S.grasp[gi] == j) for (int i = 0; i < 3; ++i) D[i * 4] += misc[M_D + gi];
#pragma unroll
  for (int sid = 0; sid < 7; ++sid) {
    const int wa = spr_wa(sid), ha = spr_ha(sid), wb = spr_wb(sid), hb = spr_hb(sid);
    const int a = spr_node(p, wa, ha), b = spr_node(p, wb, hb);
    if (a < 0 || b >= S.nv) continue;
    if (!((wa == 1 && ha == h) || (wb == 1 && hb == h))) continue;
    R kk, Lr;
    spring_rest(L, k, sid, kk, Lr, S);
    R dv[3], f[3], H[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      dv[i] = (pick<R, PPL>(L.x0, L.xm, L.xp, k, wb, 3 * hb + i) - pick<R, PPL>(L.x0, L.xm, L.xp, k, wa, 3 * ha + i)) +
              (pick<R, PPL>(L.dx, dxm, dxp, k, wb, 3 * hb + i) - pick<R, PPL>(L.dx, dxm, dxp, k, wa, 3 * ha + i));
    spring_eval(dv, kk, Lr, false, f, H);
#pragma unroll
    for (int i = 0; i < 9; ++i) D[i] += H[i];
  }
}

// Primal-dual interior point with Nesterov-Todd scaling (Vandenberghe, "The CVXOPT linear and
// quadratic cone program solvers", 2010) for
//   min 1/2 D^T P D  s.t.  s_i = A_i D_j + phi_i e1 in Q,  z_i in Q  (forces lam_i = A_i^T z_i),
// centering s_i o z_i = kappa e.  kfinal < 0: fixed target kappa (smooth model).  Else each
// iteration is a Mehrotra predictor-corrector step: the affine direction (target 0) and its step
// length alpha_a give the target max(kfinal, (1 - alpha_a)^3 <s,z>/m), and the combined direction
// adds the second-order term (W^-1 ds_a) o (W dz_a); once the target is kfinal, centring steps at
// kfinal end the solve.  On exit (T, B, V) hold the factorisation of the last H2 = P + sum A^T W^-2 A.
template <typename R, int PPL>
__device__ __forceinline__ int stage2_ipm(const Scene<R>& S, Lane<R, PPL>& L, WS<R>& w, R kappa, R kfinal,
                          int lane, int* iters, bool warm = false) {
  const int nobs = S.nobs;
  const R mm = R(S.nv * nobs);
  const int NP = w.NP;
  R dxm[PPL][6], dxp[PPL][6];
  nbr<R, PPL>(L.dx, dxm, dxp, lane);
  // interior start
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (2 * p + h >= S.nv) { for (int i = 0; i < 3; ++i) L.Dl[k][3 * h + i] = R(0); continue; }
      R D[9];
      diag_block(S, L, dxm, dxp, w.misc, k, p, h, D);
      R Dj[3] = {0, 0, 0};
      if (warm) {                    // given start (L.Dl); the central point does not depend on it
        for (int i = 0; i < 3; ++i) Dj[i] = L.Dl[k][3 * h + i];
      } else
      for (int o = 0; o < nobs; ++o) {
        const R ph = w.phi[cs1(o, h, p, NP)];
        if (ph < R(0)) {
          R n[3] = {w.nrm[cv(o, h, 0, p, NP)], w.nrm[cv(o, h, 1, p, NP)], w.nrm[cv(o, h, 2, p, NP)]};
          R a = R(0);
          for (int i = 0; i < 3; ++i) a += n[i] * (D[i * 3] * n[0] + D[i * 3 + 1] * n[1] + D[i * 3 + 2] * n[2]);
          const R push = R(0.5) * (-ph + sqrt(ph * ph + R(4) * kappa / a));
          for (int i = 0; i < 3; ++i) Dj[i] += push * n[i];
        }
      }
      for (int i = 0; i < 3; ++i) L.Dl[k][3 * h + i] = Dj[i];
      for (int o = 0; o < nobs; ++o) {
        R A[9];
        pair_frame(w, o, h, p, S.mu, A);
        const R ph = w.phi[cs1(o, h, p, NP)];
        R sv[3];
        for (int a = 0; a < 3; ++a)
          sv[a] = A[a * 3] * Dj[0] + A[a * 3 + 1] * Dj[1] + A[a * 3 + 2] * Dj[2] + (a == 0 ? ph : R(0));
        const bool ok = sv[0] > R(0) && soc_det(sv) > R(0.25) * sv[0] * sv[0];
        if (!ok) { sv[0] = ph > S.sig0 ? ph : S.sig0; sv[1] = sv[2] = R(0); }
        const R dt = soc_det(sv);
        for (int a = 0; a < 3; ++a) w.s[cv(o, h, a, p, NP)] = sv[a];
        w.z[cv(o, h, 0, p, NP)] = kappa * sv[0] / dt;
        w.z[cv(o, h, 1, p, NP)] = -kappa * sv[1] / dt;
        w.z[cv(o, h, 2, p, NP)] = -kappa * sv[2] / dt;
      }
    }
  }
  int stalls = 0;
  const bool proj = false;    // stage 2 uses the exact P
  bool centring = false;      // the target has reached kfinal: plain centring steps from now on
  R xmax = R(0);
#pragma unroll
  for (int k = 0; k < PPL; ++k)
#pragma unroll
    for (int e = 0; e < 6; ++e) xmax = fmax(xmax, fabs(L.x0[k][e] + L.dx[k][e]));
  const R ilim = R(128) * (sizeof(R) == 4 ? R(1.1920928955078125e-7) : R(2.220446049250313e-16)) * wmax(xmax);
  for (int it = 0; it < S.ipm_max; ++it) {
    // predictor-corrector iteration (towards kfinal, not yet centring): assemble with the affine
    // right-hand side (target 0); otherwise with the fixed target
    const bool pc = kfinal >= R(0) && !centring;
    R target = kfinal < R(0) ? kappa : kfinal;
    R Dlm[PPL][6], Dlp[PPL][6];
    nbr<R, PPL>(L.Dl, Dlm, Dlp, lane);
    // assemble H2 and the right-hand side -P D + sum A^T (z + M g), g = r_z + W d_s.  H2 not
    // positive definite means P is not either (the stage-1 root is not a minimiser of its
    // potential, and the QP of eq. dynamics-second-stage is not convex): no contact solution.
    {
#pragma unroll
      for (int k = 0; k < PPL; ++k) {
        const int p = lane + 32 * k;
        if (p >= S.npair) continue;
        R T[36], Bc[36], F[6], PD[6];
        assemble1(S, L, dxm, dxp, w.misc, k, p, proj, T, Bc, F);
        hessvec(S, L, dxm, dxp, L.Dl, Dlm, Dlp, w.misc, k, p, proj, PD);
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          R rhs[3] = {-PD[3 * h], -PD[3 * h + 1], -PD[3 * h + 2]};
          if (2 * p + h < S.nv) {
            const R D[3] = {L.Dl[k][3 * h], L.Dl[k][3 * h + 1], L.Dl[k][3 * h + 2]};
            for (int o = 0; o < nobs; ++o) {
              R A[9], M[9], rz[3], Wds[3];
              pair_terms(S, w, o, h, p, D, pc ? R(0) : target, A, M, rz, Wds);
              const R g0 = rz[0] + Wds[0], g1 = rz[1] + Wds[1], g2 = rz[2] + Wds[2];
              w.pm[cm6(o, h, 0, p, NP)] = M[0]; w.pm[cm6(o, h, 1, p, NP)] = M[1];
              w.pm[cm6(o, h, 2, p, NP)] = M[2]; w.pm[cm6(o, h, 3, p, NP)] = M[4];
              w.pm[cm6(o, h, 4, p, NP)] = M[5]; w.pm[cm6(o, h, 5, p, NP)] = M[8];
              w.pg[cv(o, h, 0, p, NP)] = g0; w.pg[cv(o, h, 1, p, NP)] = g1; w.pg[cv(o, h, 2, p, NP)] = g2;
              w.prz[cv(o, h, 0, p, NP)] = rz[0]; w.prz[cv(o, h, 1, p, NP)] = rz[1];
              w.prz[cv(o, h, 2, p, NP)] = rz[2];
              R zg[3];
#pragma unroll
              for (int a = 0; a < 3; ++a)
                zg[a] = w.z[cv(o, h, a, p, NP)] + M[a * 3] * g0 + M[a * 3 + 1] * g1 + M[a * 3 + 2] * g2;
              R MA[9];
#pragma unroll
              for (int a = 0; a < 3; ++a)
#pragma unroll
                for (int c = 0; c < 3; ++c)
                  MA[a * 3 + c] = M[a * 3] * A[c] + M[a * 3 + 1] * A[3 + c] + M[a * 3 + 2] * A[6 + c];
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                rhs[i] += A[i] * zg[0] + A[3 + i] * zg[1] + A[6 + i] * zg[2];
#pragma unroll
                for (int c = 0; c <= i; ++c)
                  T[(3 * h + i) * 6 + 3 * h + c] += A[i] * MA[c] + A[3 + i] * MA[3 + c] + A[6 + i] * MA[6 + c];
              }
            }
          } else {
            rhs[0] = rhs[1] = rhs[2] = R(0);
          }
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            w.r[cr_v(p, 3 * h + i)] = rhs[i];
            L.F[k][3 * h + i] = rhs[i];       // kept for the corrector's right-hand side
          }
        }
        put_rows(w, p, T, Bc);
      }
      __syncwarp();
      if (!cr_factor(w.T, w.B, w.V, S.npair, lane)) { *iters = it + 1; return ST_NOTPD; }
    }
    cr_solve(w.T, w.B, w.V, w.r, S.npair, lane);
    get_rhs<R, PPL>(S, w, L.pv, lane);            // dDelta (affine when pc)
    if (pc) {
      // affine step length and duality measure -> centring target
      R aa = R(1e30), gap = R(0);
#pragma unroll
      for (int k = 0; k < PPL; ++k) {
        const int p = lane + 32 * k;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          if (2 * p + h >= S.nv) continue;
          const R dD[3] = {L.pv[k][3 * h], L.pv[k][3 * h + 1], L.pv[k][3 * h + 2]};
          for (int o = 0; o < nobs; ++o) {
            R dsa[3], dza[3], sv[3], zv[3];
            pair_step(S, w, o, h, p, dD, dsa, dza);
            for (int a = 0; a < 3; ++a) {
              sv[a] = w.s[cv(o, h, a, p, NP)];
              zv[a] = w.z[cv(o, h, a, p, NP)];
              gap += sv[a] * zv[a];
            }
            aa = fmin(aa, fmin(soc_max_step(sv, dsa), soc_max_step(zv, dza)));
          }
        }
      }
      aa = fmin(R(1), -wmax(-aa));
      gap = wsum(gap);
      const R om = R(1) - aa;
      target = fmax(kfinal, om * om * om * gap / mm);
      centring = target == kfinal;
      // combined right-hand side: d_s = lam^-1 o (target e - lam o lam - (W^-1 ds_a) o (W dz_a)),
      // the second-order term dropped once the target is kfinal; same factorisation.  Only g
      // changes from the affine system: rhs = rhs_aff + sum A^T M (g - g_aff).
#pragma unroll
      for (int k = 0; k < PPL; ++k) {
        const int p = lane + 32 * k;
        if (p >= S.npair) continue;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          R rhs[3] = {L.F[k][3 * h], L.F[k][3 * h + 1], L.F[k][3 * h + 2]};
          if (2 * p + h < S.nv) {
            const R dD[3] = {L.pv[k][3 * h], L.pv[k][3 * h + 1], L.pv[k][3 * h + 2]};
            for (int o = 0; o < nobs; ++o) {
              R A[9], W[9], Wi[9], lam[3], sv[3], zv[3], ga[3], rz[3];
              pair_frame(w, o, h, p, S.mu, A);
              const R m6[6] = {w.pm[cm6(o, h, 0, p, NP)], w.pm[cm6(o, h, 1, p, NP)], w.pm[cm6(o, h, 2, p, NP)],
                               w.pm[cm6(o, h, 3, p, NP)], w.pm[cm6(o, h, 4, p, NP)], w.pm[cm6(o, h, 5, p, NP)]};
              const R M[9] = {m6[0], m6[1], m6[2], m6[1], m6[3], m6[4], m6[2], m6[4], m6[5]};
              for (int a = 0; a < 3; ++a) {
                sv[a] = w.s[cv(o, h, a, p, NP)];
                zv[a] = w.z[cv(o, h, a, p, NP)];
                ga[a] = w.pg[cv(o, h, a, p, NP)];
                rz[a] = w.prz[cv(o, h, a, p, NP)];
              }
              nt_scaling(sv, zv, W, Wi, lam);
              R c3[3] = {R(0), R(0), R(0)};
              if (!centring) {
                // affine directions ds_a = A dD - r_z, dz_a = M (g_aff - A dD)
                R ADd[3], dsa[3], gm[3], dza[3];
                for (int a = 0; a < 3; ++a) {
                  ADd[a] = A[a * 3] * dD[0] + A[a * 3 + 1] * dD[1] + A[a * 3 + 2] * dD[2];
                  dsa[a] = ADd[a] - rz[a];
                  gm[a] = ga[a] - ADd[a];
                }
                for (int a = 0; a < 3; ++a) dza[a] = M[a * 3] * gm[0] + M[a * 3 + 1] * gm[1] + M[a * 3 + 2] * gm[2];
                R a1[3], a2[3];
                for (int a = 0; a < 3; ++a) {
                  a1[a] = Wi[a * 3] * dsa[0] + Wi[a * 3 + 1] * dsa[1] + Wi[a * 3 + 2] * dsa[2];
                  a2[a] = W[a * 3] * dza[0] + W[a * 3 + 1] * dza[1] + W[a * 3 + 2] * dza[2];
                }
                c3[0] = a1[0] * a2[0] + a1[1] * a2[1] + a1[2] * a2[2];
                c3[1] = a1[0] * a2[1] + a2[0] * a1[1];
                c3[2] = a1[0] * a2[2] + a2[0] * a1[2];
              }
              const R r3[3] = {target - (lam[0] * lam[0] + lam[1] * lam[1] + lam[2] * lam[2]) - c3[0],
                               R(-2) * lam[0] * lam[1] - c3[1], R(-2) * lam[0] * lam[2] - c3[2]};
              R ds[3];
              jordan_solve(lam, r3, ds);
              R dg[3];
              for (int a = 0; a < 3; ++a) {
                const R g = rz[a] + W[a * 3] * ds[0] + W[a * 3 + 1] * ds[1] + W[a * 3 + 2] * ds[2];
                w.pg[cv(o, h, a, p, NP)] = g;
                dg[a] = g - ga[a];
              }
              R Mdg[3];
              for (int a = 0; a < 3; ++a) Mdg[a] = M[a * 3] * dg[0] + M[a * 3 + 1] * dg[1] + M[a * 3 + 2] * dg[2];
              for (int i = 0; i < 3; ++i) rhs[i] += A[i] * Mdg[0] + A[3 + i] * Mdg[1] + A[6 + i] * Mdg[2];
            }
          } else {
            rhs[0] = rhs[1] = rhs[2] = R(0);
          }
#pragma unroll
          for (int i = 0; i < 3; ++i) w.r[cr_v(p, 3 * h + i)] = rhs[i];
        }
      }
      __syncwarp();
      cr_solve(w.T, w.B, w.V, w.r, S.npair, lane);
      get_rhs<R, PPL>(S, w, L.pv, lane);          // dDelta (combined)
    }
    const bool final_target = kfinal < R(0) || target == kfinal;
    // step length to the cone boundaries
    R amin = R(1e30), dmax = R(0);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      const int p = lane + 32 * k;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (2 * p + h >= S.nv) continue;
        const R dD[3] = {L.pv[k][3 * h], L.pv[k][3 * h + 1], L.pv[k][3 * h + 2]};
        for (int i = 0; i < 3; ++i) {
          dmax = fmax(dmax, fabs(dD[i]));
          bad = bad || !(fabs(dD[i]) <= R(1e30));
        }
        for (int o = 0; o < nobs; ++o) {
          R dsv[3], dz[3], sv[3], zv[3];
          pair_step(S, w, o, h, p, dD, dsv, dz);
          for (int a = 0; a < 3; ++a) {
            dmax = fmax(dmax, fabs(dsv[a]));
            bad = bad || !(fabs(dz[a]) <= R(1e30)) || !(fabs(dsv[a]) <= R(1e30));
            sv[a] = w.s[cv(o, h, a, p, NP)];
            zv[a] = w.z[cv(o, h, a, p, NP)];
            w.prz[cv(o, h, a, p, NP)] = dsv[a];     // the directions, for the update below
            w.pg[cv(o, h, a, p, NP)] = dz[a];
          }
          amin = fmin(amin, soc_max_step(sv, dsv));
          amin = fmin(amin, soc_max_step(zv, dz));
        }
      }
    }
    dmax = wmax(dmax);
    amin = -wmax(-amin);
    if (__any_sync(FULL, bad)) { *iters = it + 1; return ST_NONFINITE; }
    const R alpha = fmin(R(1), R(0.99) * amin);
    stalls = alpha < R(1e-6) ? stalls + 1 : 0;
    if (stalls >= 5) { *iters = it + 1; return ST_CONTACT; }
    bool inside = true;
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      const int p = lane + 32 * k;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        if (2 * p + h >= S.nv) continue;
        for (int o = 0; o < nobs; ++o) {
          R sv[3], zv[3];
          for (int a = 0; a < 3; ++a) {
            sv[a] = w.s[cv(o, h, a, p, NP)] + alpha * w.prz[cv(o, h, a, p, NP)];
            zv[a] = w.z[cv(o, h, a, p, NP)] + alpha * w.pg[cv(o, h, a, p, NP)];
            w.s[cv(o, h, a, p, NP)] = sv[a];
            w.z[cv(o, h, a, p, NP)] = zv[a];
          }
          inside = inside && soc_inside(sv) && soc_inside(zv);
        }
      }
#pragma unroll
      for (int e = 0; e < 6; ++e) L.Dl[k][e] += alpha * L.pv[k][e];
    }
    if (!__all_sync(FULL, inside)) { *iters = it + 1; return ST_CONTACT; }
    // stop at the central point: a full step below the tolerance, or (nonsmooth solve) any step
    // below 128 ulps of the state's scale (the resolution of the real type's directions at
    // near-boundary sliding contacts)
    if (final_target && ((alpha == R(1) && dmax <= S.itol) || (kfinal >= R(0) && dmax <= ilim))) {
      *iters = it + 1;
      return 0;
    }
  }
  *iters = S.ipm_max;
  return ST_CONTACT;
}

// ------------------------------------------------------------------------------------------
// one step: inputs x0 (registers + neighbours), misc g, u, c; with warm, the stage-1 start dx; with
// warm2, the stage-2 start Dl.  Outputs dx, Dl, contact data,
// misc d, gd.  smooth = the smooth grasp and the smooth (kappa_c) contact solve.
// ------------------------------------------------------------------------------------------
template <typename R, int PPL>
__device__ __forceinline__ int sim_step(const Scene<R>& S, Lane<R, PPL>& L, WS<R>& w, int lane, bool smooth,
                        int* nit, int* iit, bool warm = false, bool warm2 = false) {
  R* d = w.misc + M_D;
  R* gd = w.misc + M_GD;
  const R* c = w.misc + M_C;
  if (lane < 2) {
    R cc[3] = {c[3 * lane], c[3 * lane + 1], c[3 * lane + 2]};
    const R rho = sqrt(dot3(cc, cc));
    R dd;
    if (smooth) {
      dd = S.Dmax * exp(-rho / S.kh);
      const R f = rho > R(0) ? -dd / (S.kh * rho) : R(0);
      for (int i = 0; i < 3; ++i) gd[3 * lane + i] = f * cc[i];
    } else {
      dd = rho <= S.rgrasp ? S.Dmax : R(0);
      for (int i = 0; i < 3; ++i) gd[3 * lane + i] = R(0);
    }
    d[lane] = dd;
  }
  __syncwarp();
  if (!warm2) zero6<R, PPL>(L.Dl);
  int st = stage1_newton(S, L, w, lane, nit, warm);
  *iit = 0;
  if (S.nobs == 0) { zero6<R, PPL>(L.Dl); return st; }
  const R pmin = contact_geometry(S, L, w, lane);
  __syncwarp();
  if (!smooth && pmin >= R(0)) { zero6<R, PPL>(L.Dl); return st; }   // Delta = 0 is optimal
  st |= stage2_ipm(S, L, w, S.kc, smooth ? R(-1) : S.khard, lane, iit, warm2);
  return st;
}

// x0 <- x0 + dx + Dl ; g <- g + u ; c <- c + u - (dx_a + Dl_a)
template <typename R, int PPL>
__device__ __forceinline__ void advance_state(const Scene<R>& S, Lane<R, PPL>& L, WS<R>& w, int lane) {
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int gi = 0; gi < 2; ++gi)
        if (S.grasp[gi] == 2 * p + h)
#pragma unroll
          for (int i = 0; i < 3; ++i)
            w.misc[M_C + 3 * gi + i] += w.misc[M_U + 3 * gi + i] - (L.dx[k][3 * h + i] + L.Dl[k][3 * h + i]);
#pragma unroll
    for (int e = 0; e < 6; ++e) L.x0[k][e] += L.dx[k][e] + L.Dl[k][e];
  }
  __syncwarp();
  if (lane < 6) w.misc[M_G + lane] += w.misc[M_U + lane];
  nbr<R, PPL>(L.x0, L.xm, L.xp, lane);
  __syncwarp();
}

// ------------------------------------------------------------------------------------------
// adjoint of one smooth step (eq. diff-sim with the total derivative).
//   in : xb = xbar+ (adjoint of x+), misc GB = gbar+, the smooth solution in the lane state and
//        the factorisation of H2 in (T, B, V)
//   out: xb = xbar (adjoint of x), misc GB = gbar, misc UB = ubar
// ------------------------------------------------------------------------------------------
template <typename R, int PPL>
__device__ __forceinline__ int adjoint_step(const Scene<R>& S, Lane<R, PPL>& L, WS<R>& w, R xb[PPL][6], int lane) {
  const R mu_f = S.mu;
  const R kappa = S.kc;
  const R* d = w.misc + M_D;
  const R* c = w.misc + M_C;
  const R* u = w.misc + M_U;
  const R* gd = w.misc + M_GD;
  // mu = H2^{-1} xbar+
  R mu[PPL][6];
  put_rhs<R, PPL>(S, w, xb, R(1), lane);
  __syncwarp();
  cr_solve(w.T, w.B, w.V, w.r, S.npair, lane);
  get_rhs<R, PPL>(S, w, mu, lane);
  R mum[PPL][6], mup[PPL][6], Dlm[PPL][6], Dlp[PPL][6], dxm[PPL][6], dxp[PPL][6];
  nbr<R, PPL>(mu, mum, mup, lane);
  nbr<R, PPL>(L.Dl, Dlm, Dlp, lane);
  nbr<R, PPL>(L.dx, dxm, dxp, lane);
  // xbar* = xbar+ - (dR/dx*)^T mu
  R xs[PPL][6];
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int e = 0; e < 6; ++e) xs[k][e] = xb[k][e];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (2 * p + h >= S.nv) continue;
      R X[3] = {L.x0[k][3 * h] + L.dx[k][3 * h], L.x0[k][3 * h + 1] + L.dx[k][3 * h + 1],
                L.x0[k][3 * h + 2] + L.dx[k][3 * h + 2]};
      const R mj[3] = {mu[k][3 * h], mu[k][3 * h + 1], mu[k][3 * h + 2]};
      for (int o = 0; o < S.nobs; ++o) {
        R ph, n[3], N[9];
        obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, N);
        R sg[3];
        for (int i = 0; i < 3; ++i) sg[i] = L.Dl[k][3 * h + i] + ph * n[i];
        R lam[3], W[9];
        cone_force_jac(sg, n, kappa, mu_f, lam, W);
        R Wm[3], Lm[3];
        for (int i = 0; i < 3; ++i) Wm[i] = W[i * 3] * mj[0] + W[i * 3 + 1] * mj[1] + W[i * 3 + 2] * mj[2];
        cone_force_dn_T(sg, n, kappa, mu_f, mj, Lm);
        const R nWm = dot3(n, Wm);
        for (int i = 0; i < 3; ++i) {
          const R NW = N[i * 3] * Wm[0] + N[i * 3 + 1] * Wm[1] + N[i * 3 + 2] * Wm[2];
          const R NL = N[i * 3] * Lm[0] + N[i * 3 + 1] * Lm[1] + N[i * 3 + 2] * Lm[2];
          // (dR/dx*)^T mu contact part = -G^T mu, G^T mu = -(n (n.W mu) + phi N W mu) + N dlam/dn^T mu
          xs[k][3 * h + i] += -(n[i] * nWm + ph * NW) + NL;
        }
      }
    }
#pragma unroll
    for (int sid = 0; sid < 7; ++sid) {
      const int wa = spr_wa(sid), ha = spr_ha(sid), wb = spr_wb(sid), hb = spr_hb(sid);
      const int a = spr_node(p, wa, ha), b = spr_node(p, wb, hb);
      if (a < 0 || b >= S.nv) continue;
      R kk, Lr;
      spring_rest(L, k, sid, kk, Lr, S);
      R dv[3], mt[3], dl[3], t3[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        dv[i] = (pick<R, PPL>(L.x0, L.xm, L.xp, k, wb, 3 * hb + i) - pick<R, PPL>(L.x0, L.xm, L.xp, k, wa, 3 * ha + i)) +
                (pick<R, PPL>(L.dx, dxm, dxp, k, wb, 3 * hb + i) - pick<R, PPL>(L.dx, dxm, dxp, k, wa, 3 * ha + i));
        mt[i] = pick<R, PPL>(mu, mum, mup, k, wb, 3 * hb + i) - pick<R, PPL>(mu, mum, mup, k, wa, 3 * ha + i);
        dl[i] = pick<R, PPL>(L.Dl, Dlm, Dlp, k, wb, 3 * hb + i) - pick<R, PPL>(L.Dl, Dlm, Dlp, k, wa, 3 * ha + i);
      }
      spring_d3(dv, kk, Lr, mt, dl, t3);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        if (wb == 1) xs[k][3 * hb + i] -= t3[i];
        if (wa == 1) xs[k][3 * ha + i] += t3[i];
      }
    }
  }
  // nu = H1^{-1} xbar*  (factorise dF/dq* at x*)
  __syncwarp();
  assemble_P(S, L, w, dxm, dxp, false, false, lane);
  put_rhs<R, PPL>(S, w, xs, R(1), lane);
  __syncwarp();
  // not positive definite: the stage-1 root is a saddle of the potential (a buckled, unstable
  // equilibrium); the step's Jacobian is reported as undefined
  if (!cr_factor(w.T, w.B, w.V, S.npair, lane)) return ST_NOTPD;
  cr_solve(w.T, w.B, w.V, w.r, S.npair, lane);
  R nu[PPL][6];
  get_rhs<R, PPL>(S, w, nu, lane);
  // xbar = w nu + grasp terms; gbar, ubar
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int e = 0; e < 6; ++e) xb[k][e] = S.w * nu[k][e];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int gi = 0; gi < 2; ++gi)
        if (S.grasp[gi] == 2 * p + h) {
          R gam = R(0);
#pragma unroll
          for (int i = 0; i < 3; ++i)
            gam += (L.dx[k][3 * h + i] - (c[3 * gi + i] + u[3 * gi + i])) * nu[k][3 * h + i] +
                   mu[k][3 * h + i] * L.Dl[k][3 * h + i];
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            xb[k][3 * h + i] += gam * gd[3 * gi + i];
            const R gbp = w.misc[M_GB + 3 * gi + i];
            const R dnu = d[gi] * nu[k][3 * h + i];
            w.misc[M_GB + 3 * gi + i] = gbp + dnu - gam * gd[3 * gi + i];
            w.misc[M_UB + 3 * gi + i] = gbp + dnu;
          }
        }
  }
  __syncwarp();
  return 0;
}

// penalty part of the planning loss at the state x0: value (lane share) and seeds added to sd
template <typename R, int PPL>
__device__ __forceinline__ R penalty(const Scene<R>& S, const Lane<R, PPL>& L, R sd[PPL][6], bool seeds, int lane) {
  R val = R(0);
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      if (2 * p + h >= S.nv) continue;
      R X[3] = {L.x0[k][3 * h], L.x0[k][3 * h + 1], L.x0[k][3 * h + 2]};
      for (int o = 0; o < S.nobs; ++o) {
        if (S.ob_type[o] == CS_PLANE) continue;
        R ph, n[3];
        obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, (R*)nullptr);
        const R v = S.pen_m - ph > R(0) ? S.pen_m - ph : R(0);
        val += S.w_pen * v * v;
        if (seeds) for (int i = 0; i < 3; ++i) sd[k][3 * h + i] += R(-2) * S.w_pen * v * n[i];
      }
    }
  }
  return val;
}

// ------------------------------------------------------------------------------------------
// state transfer: q = [x, g]; checkpoint records [nq + 6] also carry the grasp offsets c
// ------------------------------------------------------------------------------------------
template <typename R, int PPL>
__device__ __forceinline__ void load_nodes(const Scene<R>& S, Lane<R, PPL>& L, const R* q, int lane) {
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int e = 0; e < 6; ++e) L.x0[k][e] = (2 * p + e / 3 < S.nv) ? q[6 * p + e] : R(0);
  }
  nbr<R, PPL>(L.x0, L.xm, L.xp, lane);
}

template <typename R, int PPL>
__device__ __forceinline__ void load_q(const Scene<R>& S, Lane<R, PPL>& L, WS<R>& w, const R* q, int lane) {
  load_nodes(S, L, q, lane);
  if (lane < 6) {
    const R g = q[3 * S.nv + lane];
    w.misc[M_G + lane] = g;
    w.misc[M_C + lane] = g - q[3 * S.grasp[lane / 3] + lane % 3];
  }
  __syncwarp();
}

template <typename R, int PPL>
__device__ __forceinline__ void store_q(const Scene<R>& S, const Lane<R, PPL>& L, const WS<R>& w, R* q, int lane) {
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int e = 0; e < 6; ++e)
      if (2 * p + e / 3 < S.nv) q[6 * p + e] = L.x0[k][e];
  }
  if (lane < 6) q[3 * S.nv + lane] = w.misc[M_G + lane];
}

// record layout: q [nq] | c [6] | dx [3 nv] (the stage-1 offset x* - x of the step that
// produced q, used to start the smooth re-solve of the backward pass)
template <typename R, int PPL>
__device__ __forceinline__ void store_rec(const Scene<R>& S, const Lane<R, PPL>& L, const WS<R>& w, R* r, int lane) {
  store_q(S, L, w, r, lane);
  if (lane < 6) r[3 * S.nv + 6 + lane] = w.misc[M_C + lane];
  R* rd = r + 3 * S.nv + 12;
  R* rD = rd + 3 * S.nv;
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int e = 0; e < 6; ++e)
      if (2 * p + e / 3 < S.nv) { rd[6 * p + e] = L.dx[k][e]; rD[6 * p + e] = L.Dl[k][e]; }
  }
}

template <typename R, int PPL>
__device__ __forceinline__ void load_rec_dx(const Scene<R>& S, Lane<R, PPL>& L, const R* r, int lane) {
  const R* rd = r + 3 * S.nv + 12;
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int e = 0; e < 6; ++e) L.dx[k][e] = (2 * p + e / 3 < S.nv) ? rd[6 * p + e] : R(0);
  }
}

// the stage-2 displacement Delta of the step that produced the state of record r
template <typename R, int PPL>
__device__ __forceinline__ void load_rec_delta(const Scene<R>& S, Lane<R, PPL>& L, const R* r, int lane) {
  const R* rD = r + 6 * S.nv + 12;
#pragma unroll
  for (int k = 0; k < PPL; ++k) {
    const int p = lane + 32 * k;
#pragma unroll
    for (int e = 0; e < 6; ++e) L.Dl[k][e] = (2 * p + e / 3 < S.nv) ? rD[6 * p + e] : R(0);
  }
}

// true on every lane when some node has a nonzero Delta (the previous step ran stage 2)
template <typename R, int PPL>
__device__ __forceinline__ bool any_delta(const Lane<R, PPL>& L) {
  bool nz = false;
#pragma unroll
  for (int k = 0; k < PPL; ++k)
#pragma unroll
    for (int e = 0; e < 6; ++e) nz = nz || L.Dl[k][e] != R(0);
  return __any_sync(FULL, nz);
}

template <typename R, int PPL>
__device__ __forceinline__ void load_rec(const Scene<R>& S, Lane<R, PPL>& L, WS<R>& w, const R* r, int lane) {
  load_nodes(S, L, r, lane);
  if (lane < 6) {
    w.misc[M_G + lane] = r[3 * S.nv + lane];
    w.misc[M_C + lane] = r[3 * S.nv + 6 + lane];
  }
  __syncwarp();
}

template <typename R>
__device__ __forceinline__ void load_controls(R* dst, const R* src, int n, int lane) {
  if (sizeof(R) == 4 && (((uintptr_t)src) & 15) == 0 && (n & 3) == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int i = lane; i < n / 4; i += 32) d4[i] = s4[i];
  } else {
    for (int i = lane; i < n; i += 32) dst[i] = src[i];
  }
}

template <typename R>
__device__ __forceinline__ void store_controls(R* dst, const R* src, int n, int lane) {
  if (sizeof(R) == 4 && (((uintptr_t)dst) & 15) == 0 && (n & 3) == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int i = lane; i < n / 4; i += 32) d4[i] = s4[i];
  } else {
    for (int i = lane; i < n; i += 32) dst[i] = src[i];
  }
}

extern __shared__ __align__(16) unsigned char cs_smem[];

// ------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------
template <typename R, int PPL>
__global__ void __launch_bounds__(32) rope_rollout_kernel(Scene<R> S, int B, int H, const R* q0,
                                                         const R* U, R* traj, R* qH, int32_t* status,
                                                         int32_t* counters) {
  const int lane = threadIdx.x;
  const int nq = 3 * S.nv + 6;
  WS<R> w = ws_carve<R>(reinterpret_cast<R*>(cs_smem), 32 * PPL, S.nobs, H, false);
  Lane<R, PPL> L;
  zero_lane(L);
  load_rest(S, L, lane);
  const bool smooth = S.fwd_mode == CS_SMOOTH;
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    load_q(S, L, w, q0 + (size_t)b * nq, lane);
    zero6<R, PPL>(L.Dl);
    load_controls(w.u, U + (size_t)b * H * 6, 6 * H, lane);
    __syncwarp();
    if (traj) store_q(S, L, w, traj + (size_t)b * (H + 1) * nq, lane);
    int st = 0;
    for (int t = 0; t < H; ++t) {
      if (lane < 6) w.misc[M_U + lane] = w.u[6 * t + lane];
      __syncwarp();
      int ni, ii;
      // stage 2 starts from the previous step's Delta when that step ran stage 2
      const bool w2 = any_delta(L);
      const int s1 = sim_step(S, L, w, lane, smooth, &ni, &ii, false, w2);
      st |= s1;
      if (counters && lane == 0) {
        int32_t* c = counters + ((size_t)b * H + t) * 3;
        c[0] = ni; c[1] = ii; c[2] = s1;
      }
      advance_state(S, L, w, lane);
      if (traj) store_q(S, L, w, traj + ((size_t)b * (H + 1) + t + 1) * nq, lane);
    }
    if (qH) store_q(S, L, w, qH + (size_t)b * nq, lane);
    if (lane == 0 && status) status[b] = st;
    __syncwarp();
  }
}

// The parts of vjp_rollout a launch runs: both (one kernel), or the forward steps and the
// backward segments as two kernels with the rollouts of the second ordered by the cost the first
// measured (longest first).
enum { VJP_FWD = 1, VJP_BWD = 2, VJP_ALL = 3 };

// what the forward part hands to the backward part, per rollout, after its records: the adjoint
// seeds of q_H [6][32 PPL] (lane-major) and of the grippers [6]; with so (the inertial variant of
// the CTA kernels) room for the velocity seeds
__host__ __device__ constexpr int vjp_carry_elems(int PPL, int so = 0) { return (so ? 12 : 6) * 32 * PPL + 8; }

// elements of one rollout's adjoint workspace: checkpoint records, segment records, carry
__host__ __device__ inline size_t vjp_ws_elems(int nv, int H, int k, int so = 0) {
  const int nseg = (H + k - 1) / k;
  return ((size_t)(nseg + 1 + k) * rec_len_rc(nv, so) + 3) / 4 * 4 + vjp_carry_elems(2, so);
}

// the same for a cloth (one CTA per rollout): records, then a carry of the adjoint seeds of q_H
// [3 nv + 6]
__host__ __device__ inline size_t cloth_vjp_rec_elems(int nv, int H, int k) {
  const int nseg = (H + k - 1) / k;
  return ((size_t)(nseg + 1 + k) * rec_len(nv) + 3) / 4 * 4;
}
__host__ __device__ inline size_t cloth_vjp_ws_elems(int nv, int H, int k) {
  return cloth_vjp_rec_elems(nv, H, k) + ((size_t)3 * nv + 6 + 3) / 4 * 4;
}

// Forward rollout + checkpointed adjoint of one rollout by one warp.  Pointers are this
// rollout's: q0 [n_q], U [H][6], dLdtraj [H+1][n_q] (or null), Lout (or null), dLdu [H][6],
// dLdq0 [n_q] (or null), status (or null), ck: its workspace (records, then the carry).
// The steps run through one loop over a schedule -- the H forward steps, then for each segment
// (last to first) the recomputed steps and the backward steps -- so that the step and its
// adjoint are each inlined once.  PH = VJP_FWD stops after the forward steps: L and the carry are
// written, and *cost gets the forward's Newton and interior-point work (-1: the rollout failed and
// its outputs are final).  PH = VJP_BWD resumes from the carry at the last segment.
template <typename R, int PPL, int PH = VJP_ALL>
__device__ __forceinline__ void vjp_rollout(const Scene<R>& S, WS<R>& w, Lane<R, PPL>& L, int lane, int H,
                                            const R* q0, const R* U, const R* dLdtraj, R* Lout, R* dLdu,
                                            R* dLdq0, int32_t* status, R* ck, int32_t* cost = nullptr) {
  const int nq = 3 * S.nv + 6;
  const int rl = rec_len(S.nv);
  const int k = S.ckpt;
  const int nseg = (H + k - 1) / k;
  const bool fwd_smooth = S.grad_mode == CS_CONSISTENT;
  enum { FWD = 0, RECOMP = 1, BACK = 2 };
  R* seg = ck + (size_t)(nseg + 1) * rl;     // segment records [k][rl]
  R* carry = ck + (vjp_ws_elems(S.nv, H, k) - vjp_carry_elems(2));
  int st = 0;
  R Lacc = R(0);
  R xb[PPL][6];
  zero6<R, PPL>(xb);
  int work = 0;
  // schedule state
  int kind = FWD, t = 0, sgi = nseg - 1, t0 = 0, t1 = 0;
  // the first step of the segment sgi: its start state from the checkpoint, recomputed steps
  // (if it has more than one) then its backward steps
  auto begin_segment = [&]() {
    t0 = sgi * k;
    t1 = min(t0 + k, H);
    load_rec(S, L, w, ck + (size_t)sgi * rl, lane);
    load_rec_delta(S, L, ck + (size_t)sgi * rl, lane);
    store_rec(S, L, w, seg, lane);
    if (t1 - t0 > 1) { kind = RECOMP; t = t0; } else { kind = BACK; t = t0; }
  };
  if constexpr ((PH & VJP_FWD) != 0) {
    load_q(S, L, w, q0, lane);
    zero6<R, PPL>(L.Dl);
    load_controls(w.u, U, 6 * H, lane);
    __syncwarp();
    store_rec(S, L, w, ck, lane);
  } else {
    load_controls(w.u, U, 6 * H, lane);
#pragma unroll
    for (int kk = 0; kk < PPL; ++kk)
#pragma unroll
      for (int e = 0; e < 6; ++e) xb[kk][e] = carry[(kk * 6 + e) * 32 + lane];
    if (lane < 6) w.misc[M_GB + lane] = carry[6 * 32 * PPL + lane];
    __syncwarp();
    begin_segment();
  }
  while (true) {
    if (kind == BACK) {
      load_rec(S, L, w, seg + (size_t)(t - t0) * rl, lane);
      // start the smooth re-solve at the forward step's stage-1 solution and stage-2 displacement
      // (record of q_{t+1})
      const R* rn = t + 1 < t1 ? seg + (size_t)(t + 1 - t0) * rl : ck + (size_t)(sgi + 1) * rl;
      load_rec_dx(S, L, rn, lane);
      load_rec_delta(S, L, rn, lane);
    }
    if (lane < 6) w.misc[M_U + lane] = w.u[6 * t + lane];
    __syncwarp();
    int ni, ii;
    // stage-2 start: in the backward the forward step's Delta; forward and recompute start from
    // the previous step's Delta when it ran stage 2
    const bool w2 = kind == BACK || any_delta(L);
    st |= sim_step(S, L, w, lane, kind == BACK || fwd_smooth, &ni, &ii, kind == BACK, w2);
    if (st) break;                 // a failed step: the rollout's loss and gradient are undefined
    if (kind == FWD) work = min(work + 2 * ni + 5 * ii, 1 << 30);
    if (kind != BACK) {
      advance_state(S, L, w, lane);
      if (kind == FWD) {
        if ((t + 1) % k == 0 || t == H - 1) store_rec(S, L, w, ck + (size_t)((t + k) / k) * rl, lane);
        if (S.has_loss) Lacc += penalty(S, L, xb, false, lane);
      } else {
        store_rec(S, L, w, seg + (size_t)(t + 1 - t0) * rl, lane);
      }
    } else {
      st |= adjoint_step(S, L, w, xb, lane);
      if (st) break;
      if (lane < 6)
        w.ub[6 * t + lane] = w.misc[M_UB + lane] + (S.has_loss ? R(2) * S.w_u * w.u[6 * t + lane] : R(0));
    }
    // seeds dL/dq_t of the state the adjoint reaches next (q_H after the forward, q_t after a
    // backward step); x0 holds that state in both cases
    const bool seed_now = (kind == FWD && t == H - 1) || kind == BACK;
    if (seed_now) {
      if (kind == FWD) {
        if (lane < 6) w.misc[M_GB + lane] = R(0);
        __syncwarp();
        if (S.has_loss) {
#pragma unroll
          for (int kk = 0; kk < PPL; ++kk) {
            const int p = lane + 32 * kk;
            for (int gi = 0; gi < S.n_goal; ++gi) {
              const int j = S.goal[gi];
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                if (j != 2 * p + h) continue;
#pragma unroll
                for (int i = 0; i < 3; ++i) {
                  const R e = L.x0[kk][3 * h + i] - S.goal_pos[gi][i];
                  Lacc += S.w_goal * e * e;
                  xb[kk][3 * h + i] += R(2) * S.w_goal * e;
                }
              }
            }
          }
          for (int i = lane; i < 6 * H; i += 32) Lacc += S.w_u * w.u[i] * w.u[i];
        }
      }
      const int ts = kind == FWD ? H : t;        // index of the seeded state
      if (ts >= 1 && S.has_loss) penalty(S, L, xb, true, lane);
      if (dLdtraj) {
        const R* sd = dLdtraj + (size_t)ts * nq;
#pragma unroll
        for (int kk = 0; kk < PPL; ++kk) {
          const int p = lane + 32 * kk;
#pragma unroll
          for (int e = 0; e < 6; ++e)
            if (2 * p + e / 3 < S.nv) xb[kk][e] += sd[6 * p + e];
        }
        if (lane < 6) w.misc[M_GB + lane] += sd[3 * S.nv + lane];
      }
      __syncwarp();
    }
    // next schedule entry
    bool start_seg = false;
    if (kind == FWD) {
      if (++t == H) {
        if constexpr (PH == VJP_FWD) break;
        start_seg = true;
      }
    } else if (kind == RECOMP) {
      if (++t == t1 - 1) { kind = BACK; t = t1 - 1; }
    } else {
      if (--t < t0) { if (--sgi < 0) break; start_seg = true; }
    }
    if (start_seg) begin_segment();
  }
  __syncwarp();
  if constexpr (PH == VJP_FWD) {
    if (!st) {                     // hand the seeds over; L is final
#pragma unroll
      for (int kk = 0; kk < PPL; ++kk)
#pragma unroll
        for (int e = 0; e < 6; ++e) carry[(kk * 6 + e) * 32 + lane] = xb[kk][e];
      if (lane < 6) carry[6 * 32 * PPL + lane] = w.misc[M_GB + lane];
      Lacc = wsum(Lacc);
      if (lane == 0) {
        if (Lout) *Lout = Lacc;
        if (status) *status = 0;
        *cost = work;
      }
      __syncwarp();
      return;
    }
    if (lane == 0) *cost = -1;
  }
  if (st) {                        // failed rollout: L = NaN, gradients zero
    for (int i = lane; i < 6 * H; i += 32) w.ub[i] = R(0);
    zero6<R, PPL>(xb);
    if (lane < 6) w.misc[M_GB + lane] = R(0);
    Lacc = sizeof(R) == 4 ? R(nanf("")) : R(nan(""));
    __syncwarp();
  }
  store_controls(dLdu, w.ub, 6 * H, lane);
  if (dLdq0) {
#pragma unroll
    for (int kk = 0; kk < PPL; ++kk) {
      const int p = lane + 32 * kk;
#pragma unroll
      for (int e = 0; e < 6; ++e)
        if (2 * p + e / 3 < S.nv) dLdq0[6 * p + e] = xb[kk][e];
    }
    if (lane < 6) dLdq0[3 * S.nv + lane] = w.misc[M_GB + lane];
  }
  Lacc = wsum(Lacc);
  if (lane == 0) {
    // the backward part leaves the forward's L unless the rollout failed
    if (Lout && (PH != VJP_BWD || st)) *Lout = Lacc;
    if (status) *status = st;
  }
  __syncwarp();
}

// the rollouts i = blockIdx.x, blockIdx.x + gridDim.x, ... (through order[i] when given); the
// backward part skips a rollout whose forward failed (cost -1: its outputs are written)
template <typename R, int PPL, int PH>
__device__ __forceinline__ void vjp_rollouts(const Scene<R>& S, int B, int H, const R* q0, const R* U,
                                             const R* dLdtraj, R* Lout, R* dLdu, R* dLdq0, int32_t* status,
                                             R* ws, size_t ws_stride, int32_t* cost, const int32_t* order) {
  const int lane = threadIdx.x;
  const int nq = 3 * S.nv + 6;
  WS<R> w = ws_carve<R>(reinterpret_cast<R*>(cs_smem), 32 * PPL, S.nobs, H, false);
  Lane<R, PPL> L;
  zero_lane(L);
  load_rest(S, L, lane);
  for (int i = blockIdx.x; i < B; i += gridDim.x) {
    const int b = order ? order[i] : i;
    if (PH == VJP_BWD && cost[b] < 0) continue;
    vjp_rollout<R, PPL, PH>(S, w, L, lane, H, q0 + (size_t)b * nq, U + (size_t)b * H * 6,
                            dLdtraj ? dLdtraj + (size_t)b * (H + 1) * nq : nullptr, Lout ? Lout + b : nullptr,
                            dLdu + (size_t)b * H * 6, dLdq0 ? dLdq0 + (size_t)b * nq : nullptr,
                            status ? status + b : nullptr, ws + (size_t)b * ws_stride, cost ? cost + b : nullptr);
  }
}

// forward + adjoint in one launch
template <typename R, int PPL>
__global__ void __launch_bounds__(32) rope_vjp_kernel(Scene<R> S, int B, int H, const R* q0,
                                                     const R* U, const R* dLdtraj, R* Lout, R* dLdu,
                                                     R* dLdq0, int32_t* status, R* ws, size_t ws_stride) {
  vjp_rollouts<R, PPL, VJP_ALL>(S, B, H, q0, U, dLdtraj, Lout, dLdu, dLdq0, status, ws, ws_stride, nullptr,
                                nullptr);
}

// the forward part of every rollout: records, L, the carry and the cost of each
template <typename R, int PPL>
__global__ void __launch_bounds__(32) rope_vjp_fwd_kernel(Scene<R> S, int B, int H, const R* q0,
                                                         const R* U, const R* dLdtraj, R* Lout, R* dLdu,
                                                         R* dLdq0, int32_t* status, R* ws, size_t ws_stride,
                                                         int32_t* cost) {
  vjp_rollouts<R, PPL, VJP_FWD>(S, B, H, q0, U, dLdtraj, Lout, dLdu, dLdq0, status, ws, ws_stride, cost,
                                nullptr);
}

// the backward part, rollout order[i] in CTA i (the block scheduler starts CTAs in index order,
// so the costliest start first)
template <typename R, int PPL>
__global__ void __launch_bounds__(32) rope_vjp_bwd_kernel(Scene<R> S, int B, int H, const R* U,
                                                         const R* dLdtraj, R* Lout, R* dLdu, R* dLdq0,
                                                         int32_t* status, R* ws, size_t ws_stride,
                                                         int32_t* cost, const int32_t* order) {
  vjp_rollouts<R, PPL, VJP_BWD>(S, B, H, nullptr, U, dLdtraj, Lout, dLdu, dLdq0, status, ws, ws_stride, cost,
                                order);
}

// order[0..B) = the rollouts by decreasing cost, equal costs by increasing index (a bitonic sort
// of (cost, index) keys in shared memory by one CTA; B <= CS_ORDER_MAX)
constexpr int CS_ORDER_MAX = 4096;
constexpr int CS_ORDER_NT = 1024;

template <int NT>
__global__ void __launch_bounds__(NT) rope_order_kernel(const int32_t* cost, int B, int32_t* order) {
  __shared__ unsigned long long key[CS_ORDER_MAX];
  int n = 1;
  while (n < B) n <<= 1;
  for (int i = threadIdx.x; i < n; i += NT) {
    const long long c = i < B ? (long long)cost[i] : 0;
    // 0x7fffffff - cost in the high word: the costliest first; a failed rollout (-1) last but one
    // ahead of the padding
    key[i] = i < B ? ((unsigned long long)(0x7fffffffLL - c) << 32) | (unsigned)i : ~0ull;
  }
  for (int size = 2; size <= n; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      __syncthreads();
      for (int i = threadIdx.x; i < n; i += NT) {
        const int j = i ^ stride;
        if (j > i) {
          const unsigned long long a = key[i], b = key[j];
          if ((a > b) == ((i & size) == 0)) { key[i] = b; key[j] = a; }
        }
      }
    }
  __syncthreads();
  for (int i = threadIdx.x; i < B; i += NT) order[i] = (int32_t)(key[i] & 0xffffffffull);
}

// ------------------------------------------------------------------------------------------
// linearisation: one warp per (trajectory, step); tangents of the smooth step, 32 directions at
// a time (one per lane), each lane running its own solves on the two shared factorisations.
// ------------------------------------------------------------------------------------------
template <typename R, int PPL>
__global__ void __launch_bounds__(32) rope_linearize_kernel(Scene<R> S, int B, int H, const R* Z,
                                                           const R* Vc, R* A, R* Bm, int32_t* status) {
  const int lane = threadIdx.x;
  const int nv = S.nv, nq = 3 * nv + 6, N = S.npair;
  const int NP = 32 * PPL;
  WS<R> w = ws_carve<R>(reinterpret_cast<R*>(cs_smem), NP, S.nobs, 1, true);
  // per-lane tangent vectors in element-major pair layout, interleaved by lane
  // per-lane tangents, element a of pair row p at ((a * N + p) * 32 + lane), N = npair rows
  R* tv1 = w.Dn + 6 * (size_t)NP;
  R* tv2 = tv1 + (size_t)6 * N * 32;
  R* Kc = tv2 + (size_t)6 * N * 32;         // [nv nodes][9]
  R* Ks = Kc + (size_t)9 * nv;              // [nv nodes][2 springs][9]
  Lane<R, PPL> L;
  zero_lane(L);
  load_rest(S, L, lane);
  const int ndir = nq + 6;
  for (int job = blockIdx.x; job < B * H; job += gridDim.x) {
    const int b = job / H, t = job % H;
    const R* z = Z + ((size_t)b * (H + 1) + t) * nq;
    load_q(S, L, w, z, lane);
    if (lane < 6) w.misc[M_U + lane] = Vc[((size_t)b * H + t) * 6 + lane];
    // the stage-1 Newton iteration starts at the nominal next state z_{t+1}
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      const int p = lane + 32 * k;
#pragma unroll
      for (int e = 0; e < 6; ++e)
        L.dx[k][e] = (2 * p + e / 3 < nv) ? z[nq + 6 * p + e] - z[6 * p + e] : R(0);
    }
    __syncwarp();
    int ni, ii;
    int st = sim_step(S, L, w, lane, true, &ni, &ii, true);
    // keep H2's factorisation; factorise H1 at x* into the first slot
    for (int i = lane; i < CR_LDT * NP; i += 32) w.T2[i] = w.T[i];
    for (int i = lane; i < CR_LDM * NP; i += 32) { w.B2[i] = w.B[i]; w.V2[i] = w.V[i]; }
    R dxm[PPL][6], dxp[PPL][6];
    nbr<R, PPL>(L.dx, dxm, dxp, lane);
    assemble_P(S, L, w, dxm, dxp, false, false, lane);
#pragma unroll
    for (int k = 0; k < PPL; ++k) {
      const int p = lane + 32 * k;
#pragma unroll
      for (int e = 0; e < 6; ++e) {
        w.xs[e * NP + p] = L.dx[k][e];
        w.Dn[e * NP + p] = L.Dl[k][e];
      }
    }
    __syncwarp();
    if (!cr_factor(w.T, w.B, w.V, N, lane)) st |= ST_NOTPD;
    const R* d = w.misc + M_D;
    const R* c = w.misc + M_C;
    const R* u = w.misc + M_U;
    const R* gd = w.misc + M_GD;
    auto node_dx = [&](int j, int i) -> R { return w.xs[(3 * (j & 1) + i) * NP + (j >> 1)]; };
    auto node_D = [&](int j, int i) -> R { return w.Dn[(3 * (j & 1) + i) * NP + (j >> 1)]; };
    auto T1 = [&](int j, int i) -> R& { return tv1[((size_t)(3 * (j & 1) + i) * N + (j >> 1)) * 32 + lane]; };
    auto T2v = [&](int j, int i) -> R& { return tv2[((size_t)(3 * (j & 1) + i) * N + (j >> 1)) * 32 + lane]; };
    // dR/dx* (direction independent): per node the contact block Kc = sum_o [-W (n n^T + phi N)
    // + (d lam / d n) N] and per spring (j, j+o) the third-derivative block Ks with
    // t = Ks (v_b - v_a); each direction then needs only these 3x3 products
    for (int j = lane; j < nv; j += 32) {
      R X[3], Dj[3];
      for (int i = 0; i < 3; ++i) { X[i] = z[3 * j + i] + node_dx(j, i); Dj[i] = node_D(j, i); }
      R K[9];
      for (int i = 0; i < 9; ++i) K[i] = R(0);
      for (int o = 0; o < S.nobs; ++o) {
        R ph, n[3], Nm[9];
        obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, Nm);
        R sg[3];
        for (int i = 0; i < 3; ++i) sg[i] = Dj[i] + ph * n[i];
        R lam[3], W[9];
        cone_force_jac(sg, n, S.kc, S.mu, lam, W);
        // d lam / d n = c1 (n sg^T + sn I) - c2 a sg^T (as cone_force_dn)
        const R mu2 = S.mu * S.mu, sn = dot3(n, sg);
        const R g = (R(1) + mu2) * sn * sn - mu2 * dot3(sg, sg);
        const R c1 = S.kc * (R(1) + mu2) / g, c2 = R(2) * S.kc * (R(1) + mu2) * sn / (g * g);
        R Gn[9], Ds[9];
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            const R aa = (R(1) + mu2) * sn * n[a] - mu2 * sg[a];
            Gn[a * 3 + b] = c1 * (n[a] * sg[b] + (a == b ? sn : R(0))) - c2 * aa * sg[b];
            Ds[a * 3 + b] = n[a] * n[b] + ph * Nm[a * 3 + b];
          }
        for (int a = 0; a < 3; ++a)
          for (int b = 0; b < 3; ++b) {
            R t = R(0);
            for (int e = 0; e < 3; ++e) t += -W[a * 3 + e] * Ds[e * 3 + b] + Gn[a * 3 + e] * Nm[e * 3 + b];
            K[a * 3 + b] += t;
          }
      }
      for (int i = 0; i < 9; ++i) Kc[9 * j + i] = K[i];
      for (int o = 1; o <= 2; ++o) {
        const int b2 = j + o;
        R Sm[9];
        for (int i = 0; i < 9; ++i) Sm[i] = R(0);
        if (b2 < nv) {
          const R kk = o == 1 ? S.k1 : S.k2;
          const R Lr = o == 1 ? S.L1[j] : S.L2[j];
          R dv[3], dl[3];
          for (int i = 0; i < 3; ++i) {
            dv[i] = (z[3 * b2 + i] - z[3 * j + i]) + (node_dx(b2, i) - node_dx(j, i));
            dl[i] = node_D(b2, i) - Dj[i];
          }
          // spring_d3 as a matrix on mt: c (u dl^T + (u.dl) I + dl u^T - 3 (u.dl) u u^T)
          const R l = sqrt(dot3(dv, dv)), inv = R(1) / l;
          const R uu[3] = {dv[0] * inv, dv[1] * inv, dv[2] * inv};
          const R cc2 = kk * Lr * inv * inv, ud = dot3(uu, dl);
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
              Sm[a * 3 + b] = cc2 * (uu[a] * dl[b] + (a == b ? ud : R(0)) + dl[a] * uu[b] - R(3) * ud * uu[a] * uu[b]);
        }
        for (int i = 0; i < 9; ++i) Ks[(2 * j + o - 1) * 9 + i] = Sm[i];
      }
    }
    __syncwarp();
    for (int d0 = 0; d0 < ndir; d0 += 32) {
      const int dir = d0 + lane;
      const bool act = dir < ndir;
      int kind = 0, jn = 0, cc = 0, gi = 0;
      if (dir < 3 * nv) { kind = 0; jn = dir / 3; cc = dir % 3; }
      else if (dir < nq) { kind = 1; gi = (dir - 3 * nv) / 3; cc = (dir - 3 * nv) % 3; }
      else { kind = 2; gi = (dir - nq) / 3; cc = (dir - nq) % 3; if (gi > 1) gi = 1; }
      for (int r = 0; r < 6 * N; ++r) { tv1[(size_t)r * 32 + lane] = R(0); tv2[(size_t)r * 32 + lane] = R(0); }
      // rhs1 = -(dF/dtheta) e_dir ; dx* = H1^{-1} rhs1
      if (act) {
        if (kind == 0) {
          T1(jn, cc) += S.w;
          for (int g2 = 0; g2 < 2; ++g2)
            if (S.grasp[g2] == jn) {
              const R dd = -gd[3 * g2 + cc];
              for (int i = 0; i < 3; ++i) T1(jn, i) -= (node_dx(jn, i) - (c[3 * g2 + i] + u[3 * g2 + i])) * dd;
            }
        } else {
          const int a = S.grasp[gi];
          T1(a, cc) += d[gi];
          if (kind == 1)
            for (int i = 0; i < 3; ++i) T1(a, i) -= (node_dx(a, i) - (c[3 * gi + i] + u[3 * gi + i])) * gd[3 * gi + cc];
        }
      }
      cr_solve_serial(w.T, w.B, w.V, tv1 + lane, 32, N, N);
      // rhs2 = -(Rx dx* + Rq theta)
      for (int j = 0; j < nv; ++j) {
        const R v[3] = {T1(j, 0), T1(j, 1), T1(j, 2)};
        const R* K = Kc + 9 * j;
        for (int i = 0; i < 3; ++i) T2v(j, i) -= K[i * 3] * v[0] + K[i * 3 + 1] * v[1] + K[i * 3 + 2] * v[2];
        for (int o = 1; o <= 2; ++o) {
          const int b2 = j + o;
          if (b2 >= nv) continue;
          const R* Sm = Ks + (2 * j + o - 1) * 9;
          const R mt[3] = {T1(b2, 0) - v[0], T1(b2, 1) - v[1], T1(b2, 2) - v[2]};
          for (int i = 0; i < 3; ++i) {
            const R t3 = Sm[i * 3] * mt[0] + Sm[i * 3 + 1] * mt[1] + Sm[i * 3 + 2] * mt[2];
            T2v(b2, i) += t3;
            T2v(j, i) -= t3;
          }
        }
      }
      if (act && kind != 2) {
        for (int g2 = 0; g2 < 2; ++g2) {
          const int a = S.grasp[g2];
          R dd = R(0);
          if (kind == 1 && gi == g2) dd = gd[3 * g2 + cc];
          if (kind == 0 && jn == a) dd = -gd[3 * g2 + cc];
          for (int i = 0; i < 3; ++i) T2v(a, i) += node_D(a, i) * dd;
        }
      }
      for (int j = 0; j < nv; ++j)
        for (int i = 0; i < 3; ++i) T2v(j, i) = -T2v(j, i);
      cr_solve_serial(w.T2, w.B2, w.V2, tv2 + lane, 32, N, N);
      if (act) {
        R* out;
        size_t ld;
        int col;
        if (dir < nq) { out = A + ((size_t)b * H + t) * nq * nq; ld = nq; col = dir; }
        else { out = Bm + ((size_t)b * H + t) * nq * 6; ld = 6; col = dir - nq; }
        for (int j = 0; j < nv; ++j)
          for (int i = 0; i < 3; ++i) out[(size_t)(3 * j + i) * ld + col] = T1(j, i) + T2v(j, i);
        for (int r = 0; r < 6; ++r) {
          R v = R(0);
          if (kind >= 1 && r == 3 * gi + cc) v = R(1);
          out[(size_t)(3 * nv + r) * ld + col] = v;
        }
      }
    }
    st = __reduce_or_sync(FULL, st);
    if (lane == 0 && status) atomicOr(reinterpret_cast<int*>(status) + b, st);
    __syncwarp();
  }
}

}  // namespace cs
