// Rope (particle chain) kernels: one warp per rollout, the rollout's whole state in shared memory
// across the horizon, node pairs (2p, 2p+1) owned by lane p (mod 32).
//
// One step (arxiv 2606.14188, Sec. 4.1, "Simulation Solver"):
//   stage 1  Newton for q* with F(q*) = M(q*-q)/dt^2 + dE(q*) - tau(u) + sum_i d_i (x*_a - g*_i) = 0
//            (eq. dynamics-first-stage; kinematic grippers g* = g + u; d_i the grasp stiffness,
//            D_max 1[|c_i| <= r_grasp] nonsmooth, D_max exp(-|c_i|/kappa_h) smooth);
//   stage 2  Delta = argmin 1/2 Delta^T P Delta over the dual friction cones (eq.
//            dynamics-second-stage), by the log barrier of the relaxed complementarity
//            s^T lam = kappa (Sec. 4.1 "Contact Smoothing"): one barrier solve at kappa_c
//            (smooth) or a path-following sequence down to kappa_hard (nonsmooth, skipped when
//            no pair penetrates).
// Newton iterates are kept as offsets dx from the step's start state x0 (x* = x0 + dx) so the
// stiff grasp and spring forces are evaluated without absolute-coordinate cancellation.
#pragma once
#include "common.cuh"
#include "cr.cuh"

namespace cs {

// per-warp shared-memory views
template <typename R>
struct WM {
  R *x0, *dx, *p, *F, *Dl, *PD, *v1, *v2, *v3;  // node vectors [3 nv]
  R *sig, *zz, *phi, *nrm;                       // per (node, obstacle): s [3], z [3], phi, n [3]
  R *T, *B, *V, *r;                              // cyclic-reduction storage
  R *T2, *B2, *V2;                               // second factorisation (linearisation only)
  R *u, *ub;                                     // controls / their adjoint [6 H]
  R *misc;                                       // [64]
};

// misc layout
enum {
  M_G = 0,      // g [6]   gripper positions at the step start
  M_U = 6,      // u [6]   control of the step
  M_C = 12,     // c [6]   c_i = g_i - x0_a(i)
  M_D = 18,     // d [2]   grasp stiffness
  M_GD = 20,    // gd [6]  d d_i / d c_i (smooth)
  M_GB = 26,    // gbar [6] adjoint of the gripper positions
  M_TMP = 32
};

__host__ __device__ inline size_t wm_size(int nv, int npair, int nobs, int H, bool two_fact) {
  size_t s = 9 * 3 * (size_t)nv + (size_t)nv * nobs * 10 + (size_t)npair * (3 * 36 + 6) + 64;
  s = ((s + 3) & ~(size_t)3) + 12 * (size_t)H;
  if (two_fact) s += (size_t)npair * 3 * 36;
  return s;
}

template <typename R>
__device__ WM<R> wm_carve(R* base, int nv, int npair, int nobs, int H, bool two_fact) {
  WM<R> m;
  R* p = base;
  auto take = [&](size_t n) { R* q = p; p += n; return q; };
  m.x0 = take(3 * nv); m.dx = take(3 * nv); m.p = take(3 * nv); m.F = take(3 * nv);
  m.Dl = take(3 * nv); m.PD = take(3 * nv); m.v1 = take(3 * nv); m.v2 = take(3 * nv);
  m.v3 = take(3 * nv);
  m.sig = take((size_t)nv * nobs * 3); m.zz = take((size_t)nv * nobs * 3);
  m.phi = take((size_t)nv * nobs);
  m.nrm = take((size_t)nv * nobs * 3);
  m.T = take(npair * 36); m.B = take(npair * 36); m.V = take(npair * 36); m.r = take(npair * 6);
  m.misc = take(64);
  p = base + (((size_t)(p - base) + 3) & ~(size_t)3);   // 16-byte align the control rows
  m.u = take(6 * H); m.ub = take(6 * H);
  if (two_fact) { m.T2 = take(npair * 36); m.B2 = take(npair * 36); m.V2 = take(npair * 36); }
  else { m.T2 = m.B2 = m.V2 = nullptr; }
  return m;
}

// ------------------------------------------------------------------------------------------
// springs of the chain touching pair p: (a, b = a + o), o = 1 stretch, o = 2 bend
// ------------------------------------------------------------------------------------------
template <typename R, typename Fn>
__device__ __forceinline__ void springs_of_pair(const Scene<R>& S, int p, Fn fn) {
  for (int o = 1; o <= 2; ++o)
    for (int a = 2 * p - o; a <= 2 * p + 1; ++a) {
      const int b = a + o;
      if (a < 0 || b >= S.nv) continue;
      if ((a >> 1) != p && (b >> 1) != p) continue;
      fn(a, b, o);
    }
}

template <typename R>
__device__ __forceinline__ void spring_params(const Scene<R>& S, int a, int o, R& k, R& L) {
  if (o == 1) { k = S.k1; L = S.L1[a]; } else { k = S.k2; L = S.L2[a]; }
}

// d = (x0_b + dx_b) - (x0_a + dx_a), formed as (x0_b - x0_a) + (dx_b - dx_a)
template <typename R>
__device__ __forceinline__ void spring_vec(const WM<R>& m, int a, int b, R d[3]) {
  for (int i = 0; i < 3; ++i)
    d[i] = (m.x0[3 * b + i] - m.x0[3 * a + i]) + (m.dx[3 * b + i] - m.dx[3 * a + i]);
}

// Hessian P = dF/dq* of pair p into (T, Bk): w I + spring blocks + grasp d I; dummy node of an
// odd-length chain gets the identity.  Optionally also the residual F of the pair's nodes.
template <typename R>
__device__ void assemble_pair(const Scene<R>& S, const WM<R>& m, int p, R* T, R* Bk, bool proj,
                              bool want_F, R* Fout) {
  for (int i = 0; i < 36; ++i) { T[i] = R(0); Bk[i] = R(0); }
  const R* d = m.misc + M_D;
  const R* c = m.misc + M_C;
  const R* u = m.misc + M_U;
  R Fl[6] = {0, 0, 0, 0, 0, 0};
  for (int h = 0; h < 2; ++h) {
    const int j = 2 * p + h;
    if (j >= S.nv) {
      for (int i = 0; i < 3; ++i) T[(3 * h + i) * 6 + 3 * h + i] = R(1);
      continue;
    }
    for (int i = 0; i < 3; ++i) {
      T[(3 * h + i) * 6 + 3 * h + i] += S.w;
      Fl[3 * h + i] = S.w * m.dx[3 * j + i] - S.m * S.grav[i];
    }
    for (int gi = 0; gi < 2; ++gi)
      if (S.grasp[gi] == j) {
        for (int i = 0; i < 3; ++i) {
          T[(3 * h + i) * 6 + 3 * h + i] += d[gi];
          // x*_a - g*_i = dx_a - (c_i + u_i)
          Fl[3 * h + i] += d[gi] * (m.dx[3 * j + i] - (c[3 * gi + i] + u[3 * gi + i]));
        }
      }
  }
  springs_of_pair(S, p, [&](int a, int b, int o) {
    R k, L;
    spring_params(S, a, o, k, L);
    R dv[3], f[3], H[9];
    spring_vec(m, a, b, dv);
    spring_eval(dv, k, L, proj, f, H);
    const bool ina = (a >> 1) == p, inb = (b >> 1) == p;
    const int ha = a - 2 * p, hb = b - 2 * p;
    if (ina) {
      for (int i = 0; i < 3; ++i) {
        Fl[3 * ha + i] -= f[i];
        for (int q = 0; q < 3; ++q) T[(3 * ha + i) * 6 + 3 * ha + q] += H[i * 3 + q];
      }
    }
    if (inb) {
      for (int i = 0; i < 3; ++i) {
        Fl[3 * hb + i] += f[i];
        for (int q = 0; q < 3; ++q) T[(3 * hb + i) * 6 + 3 * hb + q] += H[i * 3 + q];
      }
    }
    if (ina && inb) {
      for (int i = 0; i < 3; ++i)
        for (int q = 0; q < 3; ++q) {
          T[(3 * hb + i) * 6 + 3 * ha + q] -= H[i * 3 + q];
          T[(3 * ha + i) * 6 + 3 * hb + q] -= H[i * 3 + q];
        }
    } else if (inb && (a >> 1) == p - 1) {
      const int hl = a - 2 * (p - 1);
      for (int i = 0; i < 3; ++i)
        for (int q = 0; q < 3; ++q) Bk[(3 * hb + i) * 6 + 3 * hl + q] -= H[i * 3 + q];
    }
  });
  if (want_F) for (int i = 0; i < 6; ++i) Fout[i] = Fl[i];
}

// y = P v for the nodes of pair p (P the exact stage-1 Hessian at x0 + dx)
template <typename R>
__device__ void hess_vec_pair(const Scene<R>& S, const WM<R>& m, int p, const R* v, R* y,
                              bool proj = false) {
  const R* d = m.misc + M_D;
  for (int h = 0; h < 2; ++h) {
    const int j = 2 * p + h;
    if (j >= S.nv) continue;
    for (int i = 0; i < 3; ++i) y[3 * j + i] = S.w * v[3 * j + i];
    for (int gi = 0; gi < 2; ++gi)
      if (S.grasp[gi] == j)
        for (int i = 0; i < 3; ++i) y[3 * j + i] += d[gi] * v[3 * j + i];
  }
  springs_of_pair(S, p, [&](int a, int b, int o) {
    R k, L;
    spring_params(S, a, o, k, L);
    R dv[3], f[3], H[9];
    spring_vec(m, a, b, dv);
    spring_eval(dv, k, L, proj, f, H);
    R dd[3] = {v[3 * b] - v[3 * a], v[3 * b + 1] - v[3 * a + 1], v[3 * b + 2] - v[3 * a + 2]};
    R hv[3];
    for (int i = 0; i < 3; ++i) hv[i] = H[i * 3] * dd[0] + H[i * 3 + 1] * dd[1] + H[i * 3 + 2] * dd[2];
    if ((b >> 1) == p) for (int i = 0; i < 3; ++i) y[3 * b + i] += hv[i];
    if ((a >> 1) == p) for (int i = 0; i < 3; ++i) y[3 * a + i] -= hv[i];
  });
}

// copy node vector <-> pair-ordered right-hand side (dummy node rows set to 0)
template <typename R>
__device__ __forceinline__ void to_rhs(const Scene<R>& S, const R* v, R* r, int lane, R sign) {
  for (int p = lane; p < S.npair; p += 32)
    for (int t = 0; t < 6; ++t) {
      const int j = 2 * p + t / 3;
      r[p * 6 + t] = j < S.nv ? sign * v[6 * p + t] : R(0);
    }
}

template <typename R>
__device__ __forceinline__ void from_rhs(const Scene<R>& S, const R* r, R* v, int lane) {
  for (int p = lane; p < S.npair; p += 32)
    for (int t = 0; t < 6; ++t) {
      const int j = 2 * p + t / 3;
      if (j < S.nv) v[6 * p + t] = r[p * 6 + t];
    }
}

// ------------------------------------------------------------------------------------------
// stage 1
// ------------------------------------------------------------------------------------------

// Psi(x0+dx+alpha p) - Psi(x0+dx), lane's share (nodes of its pairs; springs a -> a + o)
template <typename R>
__device__ R psi_diff_lane(const Scene<R>& S, const WM<R>& m, R alpha, int lane) {
  R val = R(0);
  const R* d = m.misc + M_D;
  const R* c = m.misc + M_C;
  const R* u = m.misc + M_U;
  for (int p = lane; p < S.npair; p += 32)
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * p + h;
      if (j >= S.nv) continue;
      for (int i = 0; i < 3; ++i) {
        const R D = alpha * m.p[3 * j + i];
        val += R(0.5) * S.w * D * (R(2) * m.dx[3 * j + i] + D) - S.m * S.grav[i] * D;
      }
      for (int gi = 0; gi < 2; ++gi)
        if (S.grasp[gi] == j)
          for (int i = 0; i < 3; ++i) {
            const R D = alpha * m.p[3 * j + i];
            // g* - X_a = (c + u) - dx_a
            val += R(0.5) * d[gi] * D * (D - R(2) * ((c[3 * gi + i] + u[3 * gi + i]) - m.dx[3 * j + i]));
          }
      for (int o = 1; o <= 2; ++o) {
        const int a = j, b = j + o;
        if (b >= S.nv) continue;
        R k, L;
        spring_params(S, a, o, k, L);
        R dX[3], dD[3], dY[3];
        spring_vec(m, a, b, dX);
        for (int i = 0; i < 3; ++i) {
          dD[i] = alpha * (m.p[3 * b + i] - m.p[3 * a + i]);
          dY[i] = dX[i] + dD[i];
        }
        const R lX = sqrt(dot3(dX, dX)), lY = sqrt(dot3(dY, dY));
        const R dl = (dD[0] * (R(2) * dX[0] + dD[0]) + dD[1] * (R(2) * dX[1] + dD[1]) +
                      dD[2] * (R(2) * dX[2] + dD[2])) / (lY + lX);
        val += R(0.5) * k * dl * (lY + lX - R(2) * L);
      }
    }
  return val;
}

// Damped Newton for stage 1; dx must be zero on entry (start at q).  Leaves the factorisation
// of the Hessian at the last iterate in (T, B, V).
template <typename R>
__device__ int stage1_newton(const Scene<R>& S, WM<R>& m, int lane, int* iters) {
  for (int it = 0; it < S.newton_max; ++it) {
    R Fl[6];
    for (int p = lane; p < S.npair; p += 32) {
      assemble_pair(S, m, p, m.T + p * 36, m.B + p * 36, false, true, Fl);
      for (int t = 0; t < 6; ++t) {
        const int j = 2 * p + t / 3;
        if (j < S.nv) m.F[6 * p + t] = Fl[t];
        m.r[p * 6 + t] = j < S.nv ? -Fl[t] : R(0);
      }
    }
    __syncwarp();
    bool ok = cr_factor(m.T, m.B, m.V, S.npair, lane);
    if (!ok) {
      for (int p = lane; p < S.npair; p += 32)
        assemble_pair(S, m, p, m.T + p * 36, m.B + p * 36, true, false, (R*)nullptr);
      __syncwarp();
      ok = cr_factor(m.T, m.B, m.V, S.npair, lane);
      if (!ok) { *iters = it + 1; return ST_NOTPD; }
    }
    cr_solve(m.T, m.B, m.V, m.r, S.npair, lane);
    R pm = R(0), sl = R(0);
    bool bad = false;
    for (int p = lane; p < S.npair; p += 32)
      for (int t = 0; t < 6; ++t) {
        const int j = 2 * p + t / 3;
        if (j >= S.nv) continue;
        const R pv = m.r[p * 6 + t];
        m.p[6 * p + t] = pv;
        bad = bad || !(fabs(pv) <= R(1e30));
        pm = fmax(pm, fabs(pv));
        sl += m.F[6 * p + t] * pv;
      }
    pm = wmax(pm);
    sl = wsum(sl);
    bad = __any_sync(FULL, bad);
    __syncwarp();
    if (bad) { *iters = it + 1; return ST_NONFINITE; }
    if (pm <= S.ntol) {
      for (int p = lane; p < S.npair; p += 32)
        for (int t = 0; t < 6; ++t)
          if (2 * p + t / 3 < S.nv) m.dx[6 * p + t] += m.p[6 * p + t];
      __syncwarp();
      *iters = it + 1;
      return 0;
    }
    R alpha = R(1);
    for (int ls = 0; ls < 40; ++ls) {
      const R dv = wsum(psi_diff_lane(S, m, alpha, lane));
      if (dv <= R(1e-4) * alpha * sl) break;
      alpha *= R(0.5);
    }
    for (int p = lane; p < S.npair; p += 32)
      for (int t = 0; t < 6; ++t)
        if (2 * p + t / 3 < S.nv) m.dx[6 * p + t] += alpha * m.p[6 * p + t];
    __syncwarp();
  }
  *iters = S.newton_max;
  return ST_NEWTON;
}

// ------------------------------------------------------------------------------------------
// stage 2
// ------------------------------------------------------------------------------------------

template <typename R>
__device__ __forceinline__ void node_pos(const WM<R>& m, int j, R X[3]) {
  for (int i = 0; i < 3; ++i) X[i] = m.x0[3 * j + i] + m.dx[3 * j + i];
}

// phi, n of every (node, obstacle) pair at x* = x0 + dx; returns min phi over the warp
template <typename R>
__device__ R contact_geometry(const Scene<R>& S, WM<R>& m, int lane) {
  R pmin = R(1e30);
  for (int p = lane; p < S.npair; p += 32)
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * p + h;
      if (j >= S.nv) continue;
      R X[3];
      node_pos(m, j, X);
      for (int o = 0; o < S.nobs; ++o) {
        R ph, n[3];
        obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, (R*)nullptr);
        const int q = j * S.nobs + o;
        m.phi[q] = ph;
        for (int i = 0; i < 3; ++i) m.nrm[3 * q + i] = n[i];
        pmin = fmin(pmin, ph);
      }
    }
  pmin = -wmax(-pmin);
  __syncwarp();
  return pmin;
}

// diagonal 3x3 block P_jj of the stage-1 Hessian at x*
template <typename R>
__device__ void diag_block(const Scene<R>& S, const WM<R>& m, int j, R D[9]) {
  const R* d = m.misc + M_D;
  for (int i = 0; i < 9; ++i) D[i] = R(0);
  for (int i = 0; i < 3; ++i) D[i * 4] = S.w;
  for (int gi = 0; gi < 2; ++gi)
    if (S.grasp[gi] == j) for (int i = 0; i < 3; ++i) D[i * 4] += d[gi];
  for (int o = 1; o <= 2; ++o)
    for (int a = j - o; a <= j; a += o) {
      const int b = a + o;
      if (a < 0 || b >= S.nv) continue;
      R k, L, dv[3], f[3], H[9];
      spring_params(S, a, o, k, L);
      spring_vec(m, a, b, dv);
      spring_eval(dv, k, L, false, f, H);
      for (int i = 0; i < 9; ++i) D[i] += H[i];
    }
}

// Stage 2: primal-dual interior point with Nesterov-Todd scaling (Vandenberghe, "The CVXOPT
// linear and quadratic cone program solvers", 2010) for
//     min 1/2 D^T P D   s.t.  s_i = A_i D_j + phi_i e1 in Q,   z_i in Q (forces lam_i = A_i^T z_i),
// with the centering s_i o z_i = kappa e (the relaxed complementarity of the smoothed model).
// kfinal < 0: fixed target kappa (smooth model); else the target falls each iteration to
// max(kfinal, min(kappa, 0.1 <s,z>/m)) and the solve ends at the central point of kfinal.
// On exit (T, B, V) hold the factorisation of the last Newton matrix H2 = P + sum A^T W^-2 A.
template <typename R>
__device__ __forceinline__ void pair_frame(const Scene<R>& S, const WM<R>& m, int q, R A[9]) {
  R n[3] = {m.nrm[3 * q], m.nrm[3 * q + 1], m.nrm[3 * q + 2]};
  cone_frame(n, S.mu, A);
}

// per pair: residual r_z = s - A D_j - phi e1, NT scaling, d_s = lam^{-1} o (target e - lam o lam)
template <typename R>
__device__ __forceinline__ void pair_newton_terms(const Scene<R>& S, const WM<R>& m, int j, int q,
                                                  R target, R A[9], R W[9], R M[9], R rz[3],
                                                  R Wds[3]) {
  pair_frame(S, m, q, A);
  const R* s = m.sig + 3 * q;
  const R* z = m.zz + 3 * q;
  for (int a = 0; a < 3; ++a)
    rz[a] = s[a] - (A[a * 3] * m.Dl[3 * j] + A[a * 3 + 1] * m.Dl[3 * j + 1] +
                    A[a * 3 + 2] * m.Dl[3 * j + 2]) - (a == 0 ? m.phi[q] : R(0));
  R Wi[9], lam[3];
  nt_scaling(s, z, W, Wi, lam);
  R ll[3] = {lam[0] * lam[0] + lam[1] * lam[1] + lam[2] * lam[2], R(2) * lam[0] * lam[1],
             R(2) * lam[0] * lam[2]};
  R rhs[3] = {target - ll[0], -ll[1], -ll[2]};
  R ds[3];
  jordan_solve(lam, rhs, ds);
  for (int a = 0; a < 3; ++a) Wds[a] = W[a * 3] * ds[0] + W[a * 3 + 1] * ds[1] + W[a * 3 + 2] * ds[2];
  for (int a = 0; a < 3; ++a)
    for (int b = 0; b < 3; ++b)
      M[a * 3 + b] = Wi[a * 3] * Wi[b] + Wi[a * 3 + 1] * Wi[3 + b] + Wi[a * 3 + 2] * Wi[6 + b];
}

// step of one pair from dDelta_j (in m.p): dz = M(-A dD + W d_s + r_z), ds = A dD - r_z
template <typename R>
__device__ __forceinline__ void pair_step(const Scene<R>& S, const WM<R>& m, int j, int q, R target,
                                          R dsv[3], R dz[3]) {
  R A[9], W[9], M[9], rz[3], Wds[3];
  pair_newton_terms(S, m, j, q, target, A, W, M, rz, Wds);
  R ADd[3], g[3];
  for (int a = 0; a < 3; ++a) {
    ADd[a] = A[a * 3] * m.p[3 * j] + A[a * 3 + 1] * m.p[3 * j + 1] + A[a * 3 + 2] * m.p[3 * j + 2];
    dsv[a] = ADd[a] - rz[a];
    g[a] = -ADd[a] + Wds[a] + rz[a];
  }
  for (int a = 0; a < 3; ++a) dz[a] = M[a * 3] * g[0] + M[a * 3 + 1] * g[1] + M[a * 3 + 2] * g[2];
}

template <typename R>
__device__ int stage2_ipm(const Scene<R>& S, WM<R>& m, R kappa, R kfinal, int lane, int* iters) {
  const int nobs = S.nobs;
  const R mm = R(S.nv * nobs);
  // interior start: per-node closed form along each penetrating normal, then s, z = kappa s^-1
  for (int p = lane; p < S.npair; p += 32)
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * p + h;
      if (j >= S.nv) continue;
      R D[9];
      diag_block(S, m, j, D);
      R Dj[3] = {0, 0, 0};
      for (int o = 0; o < nobs; ++o) {
        const int q = j * nobs + o;
        const R ph = m.phi[q];
        if (ph < R(0)) {
          const R* n = m.nrm + 3 * q;
          R a = R(0);
          for (int i = 0; i < 3; ++i)
            a += n[i] * (D[i * 3] * n[0] + D[i * 3 + 1] * n[1] + D[i * 3 + 2] * n[2]);
          const R push = R(0.5) * (-ph + sqrt(ph * ph + R(4) * kappa / a));
          for (int i = 0; i < 3; ++i) Dj[i] += push * n[i];
        }
      }
      for (int i = 0; i < 3; ++i) m.Dl[3 * j + i] = Dj[i];
      for (int o = 0; o < nobs; ++o) {
        const int q = j * nobs + o;
        R A[9];
        pair_frame(S, m, q, A);
        R sv[3];
        for (int a = 0; a < 3; ++a)
          sv[a] = A[a * 3] * Dj[0] + A[a * 3 + 1] * Dj[1] + A[a * 3 + 2] * Dj[2] + (a == 0 ? m.phi[q] : R(0));
        const bool ok = sv[0] > R(0) && soc_det(sv) > R(0.25) * sv[0] * sv[0];
        if (!ok) { sv[0] = m.phi[q] > S.sig0 ? m.phi[q] : S.sig0; sv[1] = sv[2] = R(0); }
        const R dt = soc_det(sv);
        for (int a = 0; a < 3; ++a) m.sig[3 * q + a] = sv[a];
        m.zz[3 * q] = kappa * sv[0] / dt;
        m.zz[3 * q + 1] = -kappa * sv[1] / dt;
        m.zz[3 * q + 2] = -kappa * sv[2] / dt;
      }
    }
  __syncwarp();
  int stalls = 0;
  bool proj = false;
  for (int it = 0; it < S.ipm_max; ++it) {
    R target = kappa;
    if (kfinal >= R(0)) {
      R gap = R(0);
      for (int p = lane; p < S.npair; p += 32)
        for (int h = 0; h < 2; ++h) {
          const int j = 2 * p + h;
          if (j >= S.nv) continue;
          for (int o = 0; o < nobs; ++o) gap += dot3(m.sig + 3 * (j * nobs + o), m.zz + 3 * (j * nobs + o));
        }
      gap = wsum(gap);
      target = fmax(kfinal, fmin(kappa, R(0.1) * gap / mm));
    }
    const bool final_target = kfinal < R(0) || target == kfinal;
    // assemble H2 and the right-hand side; if H2 is not positive definite with the exact P
    // (stage 1 ended where d^2E is indefinite), P becomes the projected spring Hessian for the
    // rest of this solve
    for (int attempt = 0; attempt < 2; ++attempt) {
    for (int p = lane; p < S.npair; p += 32) hess_vec_pair(S, m, p, m.Dl, m.v3, proj);
    __syncwarp();
    for (int p = lane; p < S.npair; p += 32) {
      R* T = m.T + p * 36;
      assemble_pair(S, m, p, T, m.B + p * 36, proj, false, (R*)nullptr);
      for (int h = 0; h < 2; ++h) {
        const int j = 2 * p + h;
        if (j >= S.nv) { for (int i = 0; i < 3; ++i) m.r[p * 6 + 3 * h + i] = R(0); continue; }
        R rhs[3] = {-m.v3[3 * j], -m.v3[3 * j + 1], -m.v3[3 * j + 2]};
        for (int o = 0; o < nobs; ++o) {
          const int q = j * nobs + o;
          R A[9], W[9], M[9], rz[3], Wds[3];
          pair_newton_terms(S, m, j, q, target, A, W, M, rz, Wds);
          const R* z = m.zz + 3 * q;
          R g[3], Mg[3];
          for (int a = 0; a < 3; ++a) g[a] = rz[a] + Wds[a];
          for (int a = 0; a < 3; ++a) Mg[a] = M[a * 3] * g[0] + M[a * 3 + 1] * g[1] + M[a * 3 + 2] * g[2];
          // MA = M A ; T += A^T M A ; rhs += A^T z (force) + A^T M g
          R MA[9];
          for (int a = 0; a < 3; ++a)
            for (int c = 0; c < 3; ++c)
              MA[a * 3 + c] = M[a * 3] * A[c] + M[a * 3 + 1] * A[3 + c] + M[a * 3 + 2] * A[6 + c];
          for (int i = 0; i < 3; ++i) {
            rhs[i] += A[i] * (z[0] + Mg[0]) + A[3 + i] * (z[1] + Mg[1]) + A[6 + i] * (z[2] + Mg[2]);
            for (int c = 0; c < 3; ++c)
              T[(3 * h + i) * 6 + 3 * h + c] += A[i] * MA[c] + A[3 + i] * MA[3 + c] + A[6 + i] * MA[6 + c];
          }
        }
        for (int i = 0; i < 3; ++i) m.r[p * 6 + 3 * h + i] = rhs[i];
      }
    }
    __syncwarp();
    if (cr_factor(m.T, m.B, m.V, S.npair, lane)) break;
    if (proj) { *iters = it + 1; return ST_NOTPD; }
    proj = true;
    }
    cr_solve(m.T, m.B, m.V, m.r, S.npair, lane);
    from_rhs(S, m.r, m.p, lane);          // p = dDelta
    __syncwarp();
    // step length to the cone boundaries, step sizes
    R amin = R(1e30), dmax = R(0);
    bool bad = false;
    for (int p = lane; p < S.npair; p += 32)
      for (int h = 0; h < 2; ++h) {
        const int j = 2 * p + h;
        if (j >= S.nv) continue;
        for (int i = 0; i < 3; ++i) {
          dmax = fmax(dmax, fabs(m.p[3 * j + i]));
          bad = bad || !(fabs(m.p[3 * j + i]) <= R(1e30));
        }
        for (int o = 0; o < nobs; ++o) {
          const int q = j * nobs + o;
          R dsv[3], dz[3];
          pair_step(S, m, j, q, target, dsv, dz);
          for (int a = 0; a < 3; ++a) {
            dmax = fmax(dmax, fabs(dsv[a]));
            bad = bad || !(fabs(dz[a]) <= R(1e30)) || !(fabs(dsv[a]) <= R(1e30));
          }
          amin = fmin(amin, soc_max_step(m.sig + 3 * q, dsv));
          amin = fmin(amin, soc_max_step(m.zz + 3 * q, dz));
        }
      }
    dmax = wmax(dmax);
    amin = -wmax(-amin);
    if (__any_sync(FULL, bad)) { *iters = it + 1; return ST_NONFINITE; }
    const R alpha = fmin(R(1), R(0.99) * amin);
    stalls = alpha < R(1e-6) ? stalls + 1 : 0;
    if (stalls >= 5) { *iters = it + 1; return ST_CONTACT; }
    // update s, z (they read Delta), then Delta
    bool inside = true;
    for (int p = lane; p < S.npair; p += 32)
      for (int h = 0; h < 2; ++h) {
        const int j = 2 * p + h;
        if (j >= S.nv) continue;
        for (int o = 0; o < nobs; ++o) {
          const int q = j * nobs + o;
          R dsv[3], dz[3];
          pair_step(S, m, j, q, target, dsv, dz);
          R* sq = m.sig + 3 * q;
          R* zq = m.zz + 3 * q;
          for (int a = 0; a < 3; ++a) { sq[a] += alpha * dsv[a]; zq[a] += alpha * dz[a]; }
          inside = inside && soc_inside(sq) && soc_inside(zq);
        }
        for (int i = 0; i < 3; ++i) m.Dl[3 * j + i] += alpha * m.p[3 * j + i];
      }
    __syncwarp();
    if (!__all_sync(FULL, inside)) { *iters = it + 1; return ST_CONTACT; }
    if (final_target && alpha == R(1) && dmax <= S.itol) { *iters = it + 1; return 0; }
  }
  *iters = S.ipm_max;
  return ST_CONTACT;
}

template <typename R>
__device__ void zero_nodes(const Scene<R>& S, R* v, int lane) {
  for (int i = lane; i < 3 * S.nv; i += 32) v[i] = R(0);
}

// ------------------------------------------------------------------------------------------
// one step.  Inputs: x0 (nodes), misc g, u.  Outputs: dx (x* - x0), Dl (Delta), sig, phi, nrm,
// misc d, c, gd.  smooth = use the smooth grasp and the single smooth barrier solve.
// ------------------------------------------------------------------------------------------
template <typename R>
__device__ int sim_step(const Scene<R>& S, WM<R>& m, int lane, bool smooth, int* nit, int* iit) {
  R* c = m.misc + M_C;
  R* d = m.misc + M_D;
  R* gd = m.misc + M_GD;
  if (lane < 2) {
    // c_i = g_i - x0_a(i), maintained by the caller (see advance_state) so that it keeps its
    // relative precision when it is small next to the absolute coordinates
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
  zero_nodes(S, m.dx, lane);
  zero_nodes(S, m.Dl, lane);
  __syncwarp();
  int st = stage1_newton(S, m, lane, nit);
  *iit = 0;
  if (S.nobs == 0) return st;
  const R pmin = contact_geometry(S, m, lane);
  if (!smooth && pmin >= R(0)) return st;
  st |= stage2_ipm(S, m, S.kc, smooth ? R(-1) : S.khard, lane, iit);
  return st;
}

// x0 <- x0 + dx + Dl ; g <- g + u ; c <- c + u - (dx_a + Dl_a) (formed from the small
// increments, not from the absolute coordinates)
template <typename R>
__device__ void advance_state(const Scene<R>& S, WM<R>& m, int lane) {
  if (lane < 6) {
    const int a = S.grasp[lane / 3], i = lane % 3;
    m.misc[M_C + lane] += m.misc[M_U + lane] - (m.dx[3 * a + i] + m.Dl[3 * a + i]);
  }
  __syncwarp();
  for (int i = lane; i < 3 * S.nv; i += 32) m.x0[i] += m.dx[i] + m.Dl[i];
  if (lane < 6) m.misc[M_G + lane] += m.misc[M_U + lane];
  __syncwarp();
}

// ------------------------------------------------------------------------------------------
// adjoint of one smooth step (eq. diff-sim with the total derivative).
//   in : v1 = xbar+ (adjoint of x+), misc GB = gbar+, the smooth solution of the step and the
//        factorisation of H2 in (T, B, V)
//   out: v1 = xbar (adjoint of x), misc GB = gbar, ub6 = ubar (6)
// ------------------------------------------------------------------------------------------
template <typename R>
__device__ void adjoint_step(const Scene<R>& S, WM<R>& m, int lane, R* ub6) {
  const R mu = S.mu;
  const R kappa = S.kc;
  const R* d = m.misc + M_D;
  const R* c = m.misc + M_C;
  const R* u = m.misc + M_U;
  const R* gd = m.misc + M_GD;
  // mu = H2^{-1} xbar+  -> v2
  to_rhs(S, m.v1, m.r, lane, R(1));
  __syncwarp();
  cr_solve(m.T, m.B, m.V, m.r, S.npair, lane);
  from_rhs(S, m.r, m.v2, lane);
  __syncwarp();
  // xbar* = xbar+ - (dR/dx*)^T mu  -> p
  for (int p = lane; p < S.npair; p += 32) {
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * p + h;
      if (j >= S.nv) continue;
      R acc[3] = {0, 0, 0};
      R X[3];
      node_pos(m, j, X);
      const R* mj = m.v2 + 3 * j;
      for (int o = 0; o < S.nobs; ++o) {
        const int q = j * S.nobs + o;
        R ph, n[3], N[9];
        obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, N);
        R sg[3];     // world slack of the converged (primal-feasible) point
        for (int i = 0; i < 3; ++i) sg[i] = m.Dl[3 * j + i] + ph * n[i];
        R lam[3], W[9];
        cone_force_jac(sg, n, kappa, mu, lam, W);
        R Wm[3];
        for (int i = 0; i < 3; ++i) Wm[i] = W[i * 3] * mj[0] + W[i * 3 + 1] * mj[1] + W[i * 3 + 2] * mj[2];
        R Lm[3];
        cone_force_dn_T(sg, n, kappa, mu, mj, Lm);
        // G^T mu = -(n (n.W mu) + phi N W mu) + N (dlam/dn)^T mu ; dR/dx* contact = -G
        const R nWm = dot3(n, Wm);
        for (int i = 0; i < 3; ++i) {
          R NW = N[i * 3] * Wm[0] + N[i * 3 + 1] * Wm[1] + N[i * 3 + 2] * Wm[2];
          R NL = N[i * 3] * Lm[0] + N[i * 3 + 1] * Lm[1] + N[i * 3 + 2] * Lm[2];
          const R GTm = -(n[i] * nWm + ph * NW) + NL;
          acc[i] -= GTm;      // (dR/dx*)^T mu contact part = -G^T mu
        }
      }
      for (int i = 0; i < 3; ++i) m.p[3 * j + i] = m.v1[3 * j + i] - acc[i];
    }
    springs_of_pair(S, p, [&](int a, int b, int o) {
      R k, L, dv[3];
      spring_params(S, a, o, k, L);
      spring_vec(m, a, b, dv);
      R mt[3], dl[3], t3[3];
      for (int i = 0; i < 3; ++i) {
        mt[i] = m.v2[3 * b + i] - m.v2[3 * a + i];
        dl[i] = m.Dl[3 * b + i] - m.Dl[3 * a + i];
      }
      spring_d3(dv, k, L, mt, dl, t3);
      if ((b >> 1) == p) for (int i = 0; i < 3; ++i) m.p[3 * b + i] -= t3[i];
      if ((a >> 1) == p) for (int i = 0; i < 3; ++i) m.p[3 * a + i] += t3[i];
    });
  }
  __syncwarp();
  // nu = H1^{-1} xbar*  (factorise dF/dq* at x*)  -> v3
  for (int p = lane; p < S.npair; p += 32)
    assemble_pair(S, m, p, m.T + p * 36, m.B + p * 36, false, false, (R*)nullptr);
  to_rhs(S, m.p, m.r, lane, R(1));
  __syncwarp();
  cr_factor(m.T, m.B, m.V, S.npair, lane);
  cr_solve(m.T, m.B, m.V, m.r, S.npair, lane);
  from_rhs(S, m.r, m.v3, lane);
  __syncwarp();
  // grasp coefficients gamma_i = (x*_a - g*_i).nu_a + mu_a.Delta_a
  R gam[2];
  for (int gi = 0; gi < 2; ++gi) {
    const int a = S.grasp[gi];
    R s = R(0);
    for (int i = 0; i < 3; ++i)
      s += (m.dx[3 * a + i] - (c[3 * gi + i] + u[3 * gi + i])) * m.v3[3 * a + i] +
           m.v2[3 * a + i] * m.Dl[3 * a + i];
    gam[gi] = s;
  }
  __syncwarp();
  // xbar = w nu (+ grasp terms at a(i))
  for (int i = lane; i < 3 * S.nv; i += 32) m.v1[i] = S.w * m.v3[i];
  __syncwarp();
  if (lane == 0) {
    for (int gi = 0; gi < 2; ++gi) {
      const int a = S.grasp[gi];
      for (int i = 0; i < 3; ++i) {
        m.v1[3 * a + i] += gam[gi] * gd[3 * gi + i];
        const R gbp = m.misc[M_GB + 3 * gi + i];
        const R dnu = d[gi] * m.v3[3 * a + i];
        m.misc[M_GB + 3 * gi + i] = gbp + dnu - gam[gi] * gd[3 * gi + i];
        ub6[3 * gi + i] = gbp + dnu;
      }
    }
  }
  __syncwarp();
}

// penalty part of the planning loss at the current state x0: value (lane share) and seeds
// added to `seed` (node vector) when non-null
template <typename R>
__device__ R penalty_lane(const Scene<R>& S, const WM<R>& m, R* seed, int lane) {
  R val = R(0);
  for (int p = lane; p < S.npair; p += 32)
    for (int h = 0; h < 2; ++h) {
      const int j = 2 * p + h;
      if (j >= S.nv) continue;
      R X[3] = {m.x0[3 * j], m.x0[3 * j + 1], m.x0[3 * j + 2]};
      for (int o = 0; o < S.nobs; ++o) {
        if (S.ob_type[o] == CS_PLANE) continue;
        R ph, n[3];
        obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, (R*)nullptr);
        const R v = S.pen_m - ph > R(0) ? S.pen_m - ph : R(0);
        val += S.w_pen * v * v;
        if (seed) for (int i = 0; i < 3; ++i) seed[3 * j + i] += R(-2) * S.w_pen * v * n[i];
      }
    }
  return val;
}

// ------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------
// state q = [x, g] from global memory; the grasp offsets c = g - x_a are formed from it
template <typename R>
__device__ __forceinline__ void load_q(const Scene<R>& S, WM<R>& m, const R* q, int lane) {
  for (int i = lane; i < 3 * S.nv; i += 32) m.x0[i] = q[i];
  if (lane < 6) {
    const R g = q[3 * S.nv + lane];
    m.misc[M_G + lane] = g;
    m.misc[M_C + lane] = g - q[3 * S.grasp[lane / 3] + lane % 3];
  }
  __syncwarp();
}

template <typename R>
__device__ __forceinline__ void store_q(const Scene<R>& S, const WM<R>& m, R* q, int lane) {
  for (int i = lane; i < 3 * S.nv; i += 32) q[i] = m.x0[i];
  if (lane < 6) q[3 * S.nv + lane] = m.misc[M_G + lane];
}

// checkpoint record [nq + 6]: the state and the tracked grasp offsets
template <typename R>
__device__ __forceinline__ void store_rec(const Scene<R>& S, const WM<R>& m, R* r, int lane) {
  store_q(S, m, r, lane);
  if (lane < 6) r[3 * S.nv + 6 + lane] = m.misc[M_C + lane];
}

template <typename R>
__device__ __forceinline__ void load_rec(const Scene<R>& S, WM<R>& m, const R* r, int lane) {
  for (int i = lane; i < 3 * S.nv; i += 32) m.x0[i] = r[i];
  if (lane < 6) {
    m.misc[M_G + lane] = r[3 * S.nv + lane];
    m.misc[M_C + lane] = r[3 * S.nv + 6 + lane];
  }
  __syncwarp();
}

template <typename R>
__device__ __forceinline__ void load_controls(R* dst, const R* src, int n, int lane) {
  // 16-byte vector loads when aligned (FP32 rows of 6 H floats: H even keeps rows aligned)
  if (sizeof(R) == 4 && (((uintptr_t)src) & 15) == 0 && (n & 3) == 0) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (int i = lane; i < n / 4; i += 32) d4[i] = s4[i];
  } else {
    for (int i = lane; i < n; i += 32) dst[i] = src[i];
  }
}

extern __shared__ __align__(16) unsigned char cs_smem[];

template <typename R>
__global__ void __launch_bounds__(32) rope_rollout_kernel(Scene<R> S, int B, int H, const R* q0,
                                                         const R* U, R* traj, R* qH, int32_t* status,
                                                         int32_t* counters) {
  const int lane = threadIdx.x;
  const int nq = 3 * S.nv + 6;
  WM<R> m = wm_carve<R>(reinterpret_cast<R*>(cs_smem), S.nv, S.npair, S.nobs, H, false);
  const bool smooth = S.fwd_mode == CS_SMOOTH;
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    load_q(S, m, q0 + (size_t)b * nq, lane);
    load_controls(m.u, U + (size_t)b * H * 6, 6 * H, lane);
    __syncwarp();
    if (traj) store_q(S, m, traj + (size_t)b * (H + 1) * nq, lane);
    int st = 0;
    for (int t = 0; t < H; ++t) {
      if (lane < 6) m.misc[M_U + lane] = m.u[6 * t + lane];
      __syncwarp();
      int ni, ii;
      const int s1 = sim_step(S, m, lane, smooth, &ni, &ii);
      st |= s1;
      if (counters && lane == 0) {
        int32_t* c = counters + ((size_t)b * H + t) * 3;
        c[0] = ni; c[1] = ii; c[2] = s1;
      }
      advance_state(S, m, lane);
      if (traj) store_q(S, m, traj + ((size_t)b * (H + 1) + t + 1) * nq, lane);
    }
    if (qH) store_q(S, m, qH + (size_t)b * nq, lane);
    if (lane == 0 && status) status[b] = st;
    __syncwarp();
  }
}

// forward + checkpointed adjoint.  ws: per-rollout workspace [ (nck + k) * nq ]
template <typename R>
__global__ void __launch_bounds__(32) rope_vjp_kernel(Scene<R> S, int B, int H, const R* q0,
                                                     const R* U, const R* dLdtraj, R* Lout, R* dLdu,
                                                     R* dLdq0, int32_t* status, R* ws, size_t ws_stride) {
  const int lane = threadIdx.x;
  const int nq = 3 * S.nv + 6;
  const int k = S.ckpt;
  const int nseg = (H + k - 1) / k;
  WM<R> m = wm_carve<R>(reinterpret_cast<R*>(cs_smem), S.nv, S.npair, S.nobs, H, false);
  const bool fwd_smooth = S.grad_mode == CS_CONSISTENT;
  const int rl = nq + 6;                       // checkpoint record length
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    R* ck = ws + (size_t)b * ws_stride;        // checkpoints [nseg + 1][rl]
    R* seg = ck + (size_t)(nseg + 1) * rl;     // segment states [k][rl]
    load_q(S, m, q0 + (size_t)b * nq, lane);
    load_controls(m.u, U + (size_t)b * H * 6, 6 * H, lane);
    __syncwarp();
    store_rec(S, m, ck, lane);
    int st = 0;
    R Lacc = R(0);
    for (int t = 0; t < H; ++t) {
      if (lane < 6) m.misc[M_U + lane] = m.u[6 * t + lane];
      __syncwarp();
      int ni, ii;
      st |= sim_step(S, m, lane, fwd_smooth, &ni, &ii);
      advance_state(S, m, lane);
      if ((t + 1) % k == 0) store_rec(S, m, ck + (size_t)((t + 1) / k) * rl, lane);
      if (S.has_loss) Lacc += penalty_lane(S, m, (R*)nullptr, lane);
    }
    // seeds at q_H: goal + penalty + dL/dtraj[H]
    for (int i = lane; i < 3 * S.nv; i += 32) m.v1[i] = R(0);
    if (lane < 6) m.misc[M_GB + lane] = R(0);
    __syncwarp();
    if (S.has_loss) {
      penalty_lane(S, m, m.v1, lane);
      __syncwarp();
      if (lane == 0) {
        for (int gi = 0; gi < S.n_goal; ++gi) {
          const int j = S.goal[gi];
          for (int i = 0; i < 3; ++i) {
            const R e = m.x0[3 * j + i] - S.goal_pos[gi][i];
            Lacc += S.w_goal * e * e;
            m.v1[3 * j + i] += R(2) * S.w_goal * e;
          }
        }
      }
      for (int i = lane; i < 6 * H; i += 32) Lacc += S.w_u * m.u[i] * m.u[i];
    }
    if (dLdtraj) {
      const R* sd = dLdtraj + ((size_t)b * (H + 1) + H) * nq;
      __syncwarp();
      for (int i = lane; i < 3 * S.nv; i += 32) m.v1[i] += sd[i];
      if (lane < 6) m.misc[M_GB + lane] += sd[3 * S.nv + lane];
    }
    __syncwarp();
    // backward over segments
    for (int sgi = nseg - 1; sgi >= 0; --sgi) {
      const int t0 = sgi * k;
      const int t1 = min(t0 + k, H);
      // recompute states t0 .. t1-1 into seg (keep v1 / gbar: sim_step does not touch them)
      R gb_save = lane < 6 ? m.misc[M_GB + lane] : R(0);
      load_rec(S, m, ck + (size_t)sgi * rl, lane);
      store_rec(S, m, seg, lane);
      for (int t = t0; t < t1 - 1; ++t) {
        if (lane < 6) m.misc[M_U + lane] = m.u[6 * t + lane];
        __syncwarp();
        int ni, ii;
        st |= sim_step(S, m, lane, fwd_smooth, &ni, &ii);
        advance_state(S, m, lane);
        store_rec(S, m, seg + (size_t)(t + 1 - t0) * rl, lane);
      }
      __syncwarp();
      for (int t = t1 - 1; t >= t0; --t) {
        load_rec(S, m, seg + (size_t)(t - t0) * rl, lane);
        if (lane < 6) { m.misc[M_U + lane] = m.u[6 * t + lane]; m.misc[M_GB + lane] = gb_save; }
        __syncwarp();
        int ni, ii;
        st |= sim_step(S, m, lane, true, &ni, &ii);     // smooth step at the forward state
        R ub6[6];
        adjoint_step(S, m, lane, ub6);
        if (lane == 0)
          for (int i = 0; i < 6; ++i)
            m.ub[6 * t + i] = ub6[i] + (S.has_loss ? R(2) * S.w_u * m.u[6 * t + i] : R(0));
        // seeds at q_t
        if (t >= 1 && S.has_loss) penalty_lane(S, m, m.v1, lane);
        __syncwarp();
        if (dLdtraj) {
          const R* sd = dLdtraj + ((size_t)b * (H + 1) + t) * nq;
          for (int i = lane; i < 3 * S.nv; i += 32) m.v1[i] += sd[i];
          if (lane < 6) m.misc[M_GB + lane] += sd[3 * S.nv + lane];
        }
        __syncwarp();
        gb_save = lane < 6 ? m.misc[M_GB + lane] : R(0);
      }
    }
    __syncwarp();
    for (int i = lane; i < 6 * H; i += 32) dLdu[(size_t)b * H * 6 + i] = m.ub[i];
    if (dLdq0) {
      for (int i = lane; i < 3 * S.nv; i += 32) dLdq0[(size_t)b * nq + i] = m.v1[i];
      if (lane < 6) dLdq0[(size_t)b * nq + 3 * S.nv + lane] = m.misc[M_GB + lane];
    }
    Lacc = wsum(Lacc);
    if (lane == 0) {
      if (Lout) Lout[b] = Lacc;
      if (status) status[b] = st;
    }
    __syncwarp();
  }
}

// ------------------------------------------------------------------------------------------
// linearisation: one warp per (trajectory, step); tangents of the smooth step, 32 directions
// at a time (one per lane), each lane running its own solves on the shared factorisations.
// ------------------------------------------------------------------------------------------
template <typename R>
__global__ void __launch_bounds__(32) rope_linearize_kernel(Scene<R> S, int B, int H, const R* Z,
                                                           const R* Vc, R* A, R* Bm, int32_t* status) {
  const int lane = threadIdx.x;
  const int nv = S.nv, nq = 3 * nv + 6, N = S.npair;
  WM<R> m = wm_carve<R>(reinterpret_cast<R*>(cs_smem), nv, N, S.nobs, 1, true);
  // per-lane tangent vectors, interleaved by lane: [ (6 N) ][32]
  R* tv1 = m.T2 + (size_t)N * 3 * 36;       // placed after the carve (host sizes the region)
  R* tv2 = tv1 + (size_t)6 * N * 32;
  const int ndir = nq + 6;
  for (int job = blockIdx.x; job < B * H; job += gridDim.x) {
    const int b = job / H, t = job % H;
    load_q(S, m, Z + ((size_t)b * (H + 1) + t) * nq, lane);
    if (lane < 6) m.misc[M_U + lane] = Vc[((size_t)b * H + t) * 6 + lane];
    __syncwarp();
    int ni, ii;
    int st = sim_step(S, m, lane, true, &ni, &ii);
    // H2 factor is in (T,B,V) after a barrier solve; with no obstacles it is the stage-1 one.
    // Copy it to the second slot, then factorise H1 at x* into the first.
    for (int i = lane; i < N * 36; i += 32) { m.T2[i] = m.T[i]; m.B2[i] = m.B[i]; m.V2[i] = m.V[i]; }
    for (int p = lane; p < N; p += 32)
      assemble_pair(S, m, p, m.T + p * 36, m.B + p * 36, false, false, (R*)nullptr);
    __syncwarp();
    if (!cr_factor(m.T, m.B, m.V, N, lane)) st |= ST_NOTPD;
    const R* d = m.misc + M_D;
    const R* c = m.misc + M_C;
    const R* u = m.misc + M_U;
    const R* gd = m.misc + M_GD;
    for (int d0 = 0; d0 < ndir; d0 += 32) {
      const int dir = d0 + lane;
      const bool act = dir < ndir;
      // classify the direction: x (node jn, comp cc), g_i comp cc, or u_i comp cc
      int kind = 0, jn = 0, cc = 0, gi = 0;
      if (dir < 3 * nv) { kind = 0; jn = dir / 3; cc = dir % 3; }
      else if (dir < nq) { kind = 1; gi = (dir - 3 * nv) / 3; cc = (dir - 3 * nv) % 3; }
      else { kind = 2; gi = (dir - nq) / 3; cc = (dir - nq) % 3; }
      // rhs1 = -(dF/dtheta) e_dir   (then dx* = H1^{-1} rhs1)
      for (int r = 0; r < 6 * N; ++r) tv1[r * 32 + lane] = R(0);
      if (act) {
        if (kind == 0) {
          tv1[(3 * jn + cc) * 32 + lane] += S.w;
          for (int g2 = 0; g2 < 2; ++g2)
            if (S.grasp[g2] == jn) {
              const R dd = -gd[3 * g2 + cc];     // d d / d x_a = -gd
              for (int i = 0; i < 3; ++i)
                tv1[(3 * jn + i) * 32 + lane] -= (m.dx[3 * jn + i] - (c[3 * g2 + i] + u[3 * g2 + i])) * dd;
            }
        } else {
          const int a = S.grasp[gi];
          tv1[(3 * a + cc) * 32 + lane] += d[gi];
          if (kind == 1)
            for (int i = 0; i < 3; ++i)
              tv1[(3 * a + i) * 32 + lane] -= (m.dx[3 * a + i] - (c[3 * gi + i] + u[3 * gi + i])) * gd[3 * gi + cc];
        }
      }
      // dummy node rows stay 0
      cr_solve_serial(m.T, m.B, m.V, tv1 + lane, 32, N);       // tv1 = dx*
      // rhs2 = -(Rx dx* + Rq theta)
      for (int r = 0; r < 6 * N; ++r) tv2[r * 32 + lane] = R(0);
      for (int j = 0; j < nv; ++j) {
        R X[3];
        node_pos(m, j, X);
        R v[3] = {tv1[(3 * j) * 32 + lane], tv1[(3 * j + 1) * 32 + lane], tv1[(3 * j + 2) * 32 + lane]};
        R acc[3] = {0, 0, 0};
        for (int o = 0; o < S.nobs; ++o) {
          const int q = j * S.nobs + o;
          R ph, n[3], Nm[9];
          obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, Nm);
          R sg[3];
          for (int i = 0; i < 3; ++i) sg[i] = m.Dl[3 * j + i] + ph * n[i];
          R lam[3], W[9];
          cone_force_jac(sg, n, S.kc, S.mu, lam, W);
          // G v = -W (n (n.v) + phi N v) + dlam/dn N v ; Rx contact = -G
          R Nv[3], dsg[3], Wd[3], Ld[3];
          for (int i = 0; i < 3; ++i) Nv[i] = Nm[i * 3] * v[0] + Nm[i * 3 + 1] * v[1] + Nm[i * 3 + 2] * v[2];
          const R nv_ = dot3(n, v);
          for (int i = 0; i < 3; ++i) dsg[i] = n[i] * nv_ + ph * Nv[i];
          for (int i = 0; i < 3; ++i) Wd[i] = W[i * 3] * dsg[0] + W[i * 3 + 1] * dsg[1] + W[i * 3 + 2] * dsg[2];
          cone_force_dn(sg, n, S.kc, S.mu, Nv, Ld);
          for (int i = 0; i < 3; ++i) acc[i] -= (-Wd[i] + Ld[i]);
        }
        for (int i = 0; i < 3; ++i) tv2[(3 * j + i) * 32 + lane] += acc[i];
        for (int o = 1; o <= 2; ++o) {
          const int a = j, b2 = j + o;
          if (b2 >= nv) continue;
          R k, L, dv[3], mt[3], dl[3], t3[3];
          spring_params(S, a, o, k, L);
          spring_vec(m, a, b2, dv);
          for (int i = 0; i < 3; ++i) {
            mt[i] = tv1[(3 * b2 + i) * 32 + lane] - tv1[(3 * a + i) * 32 + lane];
            dl[i] = m.Dl[3 * b2 + i] - m.Dl[3 * a + i];
          }
          spring_d3(dv, k, L, mt, dl, t3);
          for (int i = 0; i < 3; ++i) {
            tv2[(3 * b2 + i) * 32 + lane] += t3[i];
            tv2[(3 * a + i) * 32 + lane] -= t3[i];
          }
        }
      }
      if (act && kind != 2) {
        // Rq theta: node a(i) gets Delta_a (dd_i . theta)
        for (int g2 = 0; g2 < 2; ++g2) {
          const int a = S.grasp[g2];
          R dd = R(0);
          if (kind == 1 && gi == g2) dd = gd[3 * g2 + cc];
          if (kind == 0 && jn == a) dd = -gd[3 * g2 + cc];
          for (int i = 0; i < 3; ++i) tv2[(3 * a + i) * 32 + lane] += m.Dl[3 * a + i] * dd;
        }
      }
      for (int r = 0; r < 3 * nv; ++r) tv2[r * 32 + lane] = -tv2[r * 32 + lane];
      cr_solve_serial(m.T2, m.B2, m.V2, tv2 + lane, 32, N);     // tv2 = dDelta
      // column dir of [A | B]: rows 0..3nv-1 = dx* + dDelta, gripper rows = identity part
      if (act) {
        R* out;
        size_t ld;
        int col;
        if (dir < nq) { out = A + ((size_t)b * H + t) * nq * nq; ld = nq; col = dir; }
        else { out = Bm + ((size_t)b * H + t) * nq * 6; ld = 6; col = dir - nq; }
        for (int r = 0; r < 3 * nv; ++r)
          out[(size_t)r * ld + col] = tv1[r * 32 + lane] + tv2[r * 32 + lane];
        for (int r = 0; r < 6; ++r) {
          R v = R(0);
          if (kind == 1 && r == 3 * gi + cc) v = R(1);
          if (kind == 2 && r == 3 * gi + cc) v = R(1);
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
