// Device side of the cloth path: one CTA (CL_NT threads) per rollout, node-parallel loops over
// the grid, the stage-1 and stage-2 Newton systems factored by the CTA's banded Cholesky
// (cloth_band.cuh).  The method is the rope path's, step for step (Sec. 4.1): the quasi-static
// two-stage step, the primal-dual interior point for the contact cone problem (Mehrotra
// predictor-corrector towards kappa_hard, fixed target kappa_c when smooth), the smooth re-solve
// and the implicit-function adjoint of each step, checkpoints every k steps with recomputation.
//
// Stage-1 globalisation of a cloth: the exact Hessian dF/dq* plus tau I, tau = 0 or half the
// previous iteration's tau, doubled from a floor of w/4 (w = m/dt^2) while the factorisation fails
// (Cholesky with an added multiple of the identity, Nocedal & Wright, Alg. 3.3); the iteration
// stops only on an unshifted step, so the root is a local minimiser of the stage-1 potential.
//
// Node state lives in a per-CTA workspace in global memory (L2-resident); shared memory holds the
// band window, the right-hand side and the step scalars.
#pragma once
#include "cloth_band.cuh"
#include "rope.cuh"

namespace cs {

template <typename R>
struct ClothWS {
  R *x0, *dx, *Dl, *pv, *F, *xb, *mu, *rA;    // [N] node vectors (x0, dx in shared memory)
  R *Dg;                                      // [nv][6] diagonal blocks of the matrix to factor
  R *s, *z, *nrm, *pg, *prz;                  // [nobs nv][3] contact pairs
  R *phi;                                     // [nobs nv]
  R *pm;                                      // [nobs nv][6]
  R *Lg;                                      // [N][LDB] band factor
  R *Wg;                                      // band window, when it is in global memory
};

// layout of one workspace slot (elements, each array padded to a multiple of 4): see cloth_ws_elems
template <typename R>
__device__ __forceinline__ ClothWS<R> cloth_carve(R* base, const ClothDims& D, int nobs) {
  ClothWS<R> w;
  const size_t N = (size_t)D.N, np = (size_t)nobs * D.nv;
  R* p = base;
  auto take = [&](size_t n) { R* q = p; p += (n + 3) & ~(size_t)3; return q; };
  // the state x0 and the stage-1 offset dx live in shared memory, after the step scalars
  w.x0 = reinterpret_cast<R*>(cs_smem) + cloth_smem_elems(D) - 2 * (size_t)D.N;
  w.dx = w.x0 + D.N;
  w.Dl = take(N); w.pv = take(N);
  w.F = take(N); w.xb = take(N); w.mu = take(N); w.rA = take(N);
  w.Dg = take(6 * (size_t)D.nv);
  w.s = take(3 * np); w.z = take(3 * np); w.nrm = take(3 * np); w.pg = take(3 * np); w.prz = take(3 * np);
  w.phi = take(np);
  w.pm = take(6 * np);
  w.Lg = take(N * D.LDB);
  w.Wg = D.win_global ? take(cloth_gwin_elems(D)) : nullptr;
  return w;
}

// shared-memory regions after the band window / staging area and the panel buffer
template <typename R>
struct ClothSm {
  R* sm;      // window
  R* vb;      // [N] right-hand side / solution
  R* red;     // [64] reductions ([63] = factorisation flag)
  R* misc;    // [64] step scalars (layout M_*)
};

template <typename R>
__device__ __forceinline__ ClothSm<R> cloth_sm(const ClothDims& D) {
  ClothSm<R> c;
  c.sm = reinterpret_cast<R*>(cs_smem);
  c.vb = c.sm + cloth_vb_off(D);
  c.red = c.vb + D.N + CL_KB;
  c.misc = c.red + 64;
  return c;
}

// the factorisation with the band window where this cloth keeps it
template <typename R>
__device__ __forceinline__ bool cl_factor_w(const Scene<R>& S, const ClothDims& D, const BandSrc<R>& M,
                                            const ClothWS<R>& w, R* sm) {
  return D.win_global ? cl_factor<R, true>(S, D, M, w.Lg, sm, w.Wg) : cl_factor<R, false>(S, D, M, w.Lg, sm, w.Wg);
}

template <typename R>
__device__ __forceinline__ void cl_X(const ClothWS<R>& w, int v, R X[3]) {
#pragma unroll
  for (int i = 0; i < 3; ++i) X[i] = w.x0[3 * v + i] + w.dx[3 * v + i];
}

// spring t of node v at x0 + dx: difference d = x_b - x_a (a the lower node), stiffness, rest
// length; returns false when the slot has no spring
template <typename R>
__device__ __forceinline__ bool cl_spring_at(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w,
                                             int v, int t, int& u, R d[3], R& k, R& L) {
  int fam;
  const int s = cl_incident(D, v, t, u, fam);
  if (s < 0) return false;
  const int a = (t & 1) ? u : v, b = (t & 1) ? v : u;
#pragma unroll
  for (int i = 0; i < 3; ++i) d[i] = (w.x0[3 * b + i] - w.x0[3 * a + i]) + (w.dx[3 * b + i] - w.dx[3 * a + i]);
  k = cl_stiff(S, fam);
  L = S.L1[s];
  return true;
}

// diagonal 3x3 block of P at node v (w I + grasp + incident spring Hessians) and, optionally,
// the row (P y)_v of the product with a node vector y
template <typename R>
__device__ __forceinline__ void cl_node_P(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w,
                                          const R* misc, int v, bool proj, R Dv[9], const R* y, R Py[3]) {
#pragma unroll
  for (int i = 0; i < 9; ++i) Dv[i] = R(0);
  R dg = S.w;
  for (int gi = 0; gi < 2; ++gi)
    if (S.grasp[gi] == v) dg += misc[M_D + gi];
  for (int i = 0; i < 3; ++i) Dv[i * 4] = dg;
  if (y)
    for (int i = 0; i < 3; ++i) Py[i] = dg * y[3 * v + i];
  for (int t = 0; t < 12; ++t) {
    int u;
    R d[3], k, L;
    if (!cl_spring_at(S, D, w, v, t, u, d, k, L)) continue;
    R f[3], H[9];
    spring_eval(d, k, L, proj, f, H);
#pragma unroll
    for (int i = 0; i < 9; ++i) Dv[i] += H[i];
    if (y) {
      R dy[3];
      for (int i = 0; i < 3; ++i) dy[i] = y[3 * v + i] - y[3 * u + i];
      for (int i = 0; i < 3; ++i) Py[i] += H[i * 3] * dy[0] + H[i * 3 + 1] * dy[1] + H[i * 3 + 2] * dy[2];
    }
  }
}

// residual F(x0 + dx) of stage 1 into w.F
template <typename R>
__device__ __forceinline__ void cl_residual(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w,
                                            const R* misc) {
  for (int v = threadIdx.x; v < D.nv; v += CL_NT) {
    R F[3];
    for (int i = 0; i < 3; ++i) F[i] = S.w * w.dx[3 * v + i] - S.m * S.grav[i];
    for (int t = 0; t < 12; ++t) {
      int u;
      R d[3], k, L;
      if (!cl_spring_at(S, D, w, v, t, u, d, k, L)) continue;
      const R l = sqrt(dot3(d, d));
      const R fm = k * (l - L) / l;
      const R sg = (t & 1) ? R(1) : R(-1);     // force on b is +fm d, on a is -fm d
      for (int i = 0; i < 3; ++i) F[i] += sg * fm * d[i];
    }
    for (int gi = 0; gi < 2; ++gi)
      if (S.grasp[gi] == v)
        for (int i = 0; i < 3; ++i)
          F[i] += misc[M_D + gi] * (w.dx[3 * v + i] - (misc[M_C + 3 * gi + i] + misc[M_U + 3 * gi + i]));
    for (int i = 0; i < 3; ++i) w.F[3 * v + i] = F[i];
  }
}

// this thread's share of Psi(x* + alpha p) - Psi(x*), p = w.pv (stage-1 potential; every term in
// terms of the step itself, so that the difference stays accurate for small steps)
template <typename R>
__device__ __forceinline__ R cl_psi(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w, const R* misc,
                                    R alpha) {
  R val = R(0);
  for (int v = threadIdx.x; v < D.nv; v += CL_NT) {
    for (int i = 0; i < 3; ++i) {
      const R Dv = alpha * w.pv[3 * v + i];
      val += R(0.5) * S.w * Dv * (R(2) * w.dx[3 * v + i] + Dv) - S.m * S.grav[i] * Dv;
    }
    for (int gi = 0; gi < 2; ++gi)
      if (S.grasp[gi] == v)
        for (int i = 0; i < 3; ++i) {
          const R Dv = alpha * w.pv[3 * v + i];
          val += R(0.5) * misc[M_D + gi] * Dv *
                 (Dv - R(2) * ((misc[M_C + 3 * gi + i] + misc[M_U + 3 * gi + i]) - w.dx[3 * v + i]));
        }
  }
  for (int s = threadIdx.x; s < D.nspr; s += CL_NT) {
    int a, b, fam;
    cl_spring(D, s, a, b, fam);
    R dX[3], dD[3], dY[3];
    for (int i = 0; i < 3; ++i) {
      dX[i] = (w.x0[3 * b + i] - w.x0[3 * a + i]) + (w.dx[3 * b + i] - w.dx[3 * a + i]);
      dD[i] = alpha * (w.pv[3 * b + i] - w.pv[3 * a + i]);
      dY[i] = dX[i] + dD[i];
    }
    const R lX = sqrt(dot3(dX, dX)), lY = sqrt(dot3(dY, dY));
    const R dl = (dD[0] * (R(2) * dX[0] + dD[0]) + dD[1] * (R(2) * dX[1] + dD[1]) +
                  dD[2] * (R(2) * dX[2] + dD[2])) / (lY + lX);
    val += R(0.5) * cl_stiff(S, fam) * dl * (lY + lX - R(2) * S.L1[s]);
  }
  return val;
}

// Dg = diagonal blocks of P (+ shift on the diagonal) for every node
template <typename R>
__device__ __forceinline__ void cl_diag(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w,
                                        const R* misc, bool proj, R shift) {
  for (int v = threadIdx.x; v < D.nv; v += CL_NT) {
    R Dv[9], Py[3];
    cl_node_P(S, D, w, misc, v, proj, Dv, (const R*)nullptr, Py);
    for (int i = 0; i < 3; ++i) Dv[i * 4] += shift;
#pragma unroll
    for (int b = 0; b < 3; ++b)
#pragma unroll
      for (int a = b; a < 3; ++a) w.Dg[6 * v + sym3(a, b)] = Dv[a * 3 + b];
  }
}

// ---- stage 1: damped Newton on F with the shifted exact Hessian
template <typename R>
__device__ int cl_stage1(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w, const ClothSm<R>& c,
                         int* iters, bool warm) {
  const int N = D.N;
  if (!warm) {
    // start at the step's initial state with each grasped node moved with its gripper
    for (int i = threadIdx.x; i < N; i += CL_NT) {
      const int v = i / 3;
      R val = R(0);
      for (int gi = 0; gi < 2; ++gi)
        if (S.grasp[gi] == v) val = c.misc[M_U + 3 * gi + i % 3];
      w.dx[i] = val;
    }
  }
  __syncthreads();
  const R beta = R(0.25) * S.w;
  R tau = R(0);
  for (int it = 0; it < S.newton_max; ++it) {
    cl_residual(S, D, w, c.misc);
    __syncthreads();
    R t = R(0.5) * tau >= beta ? R(0.5) * tau : R(0);
    bool ok = false;
    for (int attempt = 0; attempt < 64; ++attempt) {
      cl_diag(S, D, w, c.misc, false, t);
      for (int i = threadIdx.x; i < N; i += CL_NT) c.vb[i] = -w.F[i];
      __syncthreads();
      ok = cl_factor_w(S, D, BandSrc<R>{w.x0, w.dx, w.Dg, false}, w, c.sm);
      if (ok) break;
      t = fmax(R(2) * t, beta);
    }
    if (!ok) { *iters = it + 1; return ST_NONFINITE; }
    tau = t;
    cl_back(D, w.Lg, c.sm);
    R pmx = R(0), sl = R(0);
    bool bad = false;
    for (int i = threadIdx.x; i < N; i += CL_NT) {
      const R p = c.vb[i];
      bad = bad || !(fabs(p) <= R(1e30));
      pmx = fmax(pmx, fabs(p));
      sl += w.F[i] * p;
      w.pv[i] = p;
    }
    bad = __syncthreads_or(bad);
    pmx = cl_max(pmx, c.red);
    sl = cl_sum(sl, c.red);
    if (bad) { *iters = it + 1; return ST_NONFINITE; }
    if (pmx <= S.ntol && tau == R(0)) {
      for (int i = threadIdx.x; i < N; i += CL_NT) w.dx[i] += w.pv[i];
      __syncthreads();
      *iters = it + 1;
      return 0;
    }
    R alpha = R(1);
    for (int ls = 0; ls < 40; ++ls) {
      const R dv = cl_sum(cl_psi(S, D, w, c.misc, alpha), c.red);
      if (dv <= R(1e-4) * alpha * sl) break;
      alpha *= R(0.5);
    }
    for (int i = threadIdx.x; i < N; i += CL_NT) w.dx[i] += alpha * w.pv[i];
    __syncthreads();
  }
  *iters = S.newton_max;
  return ST_NEWTON;
}

// ---- stage 2
// phi, n of every (node, obstacle) pair at x* = x0 + dx; returns min phi
template <typename R>
__device__ __forceinline__ R cl_contact_geometry(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w,
                                                 R* red) {
  R pmin = R(1e30);
  for (int v = threadIdx.x; v < D.nv; v += CL_NT) {
    R X[3];
    cl_X(w, v, X);
    for (int o = 0; o < S.nobs; ++o) {
      R ph, n[3];
      obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, (R*)nullptr);
      const int po = o * D.nv + v;
      w.phi[po] = ph;
      for (int i = 0; i < 3; ++i) w.nrm[3 * po + i] = n[i];
      pmin = fmin(pmin, ph);
    }
  }
  return -cl_max(-pmin, red);
}

template <typename R>
__device__ __forceinline__ void cl_frame(const Scene<R>& S, const ClothWS<R>& w, int po, R A[9]) {
  const R n[3] = {w.nrm[3 * po], w.nrm[3 * po + 1], w.nrm[3 * po + 2]};
  cone_frame(n, S.mu, A);
}

// Primal-dual interior point with Nesterov-Todd scaling for
//   min 1/2 D^T P D  s.t.  s_i = A_i D_j + phi_i e1 in Q,  z_i in Q  (forces lam_i = A_i^T z_i),
// centering s_i o z_i = kappa e.  kfinal < 0: fixed target kappa (smooth model); else Mehrotra
// predictor-corrector iterations until the target reaches kfinal, then centring steps at kfinal.
template <typename R>
__device__ int cl_stage2(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w, const ClothSm<R>& c,
                         R kappa, R kfinal, int* iters, bool warm) {
  const int nobs = S.nobs, nv = D.nv, N = D.N;
  const R mm = R(nv * nobs);
  // interior start
  for (int v = threadIdx.x; v < nv; v += CL_NT) {
    R Dv[9], Py[3];
    cl_node_P(S, D, w, c.misc, v, false, Dv, (const R*)nullptr, Py);
    R Dj[3] = {R(0), R(0), R(0)};
    if (warm) {
      for (int i = 0; i < 3; ++i) Dj[i] = w.Dl[3 * v + i];
    } else {
      for (int o = 0; o < nobs; ++o) {
        const int po = o * nv + v;
        const R ph = w.phi[po];
        if (ph < R(0)) {
          const R n[3] = {w.nrm[3 * po], w.nrm[3 * po + 1], w.nrm[3 * po + 2]};
          R a = R(0);
          for (int i = 0; i < 3; ++i) a += n[i] * (Dv[i * 3] * n[0] + Dv[i * 3 + 1] * n[1] + Dv[i * 3 + 2] * n[2]);
          const R push = R(0.5) * (-ph + sqrt(ph * ph + R(4) * kappa / a));
          for (int i = 0; i < 3; ++i) Dj[i] += push * n[i];
        }
      }
    }
    for (int i = 0; i < 3; ++i) w.Dl[3 * v + i] = Dj[i];
    for (int o = 0; o < nobs; ++o) {
      const int po = o * nv + v;
      R A[9];
      cl_frame(S, w, po, A);
      const R ph = w.phi[po];
      R sv[3];
      for (int a = 0; a < 3; ++a)
        sv[a] = A[a * 3] * Dj[0] + A[a * 3 + 1] * Dj[1] + A[a * 3 + 2] * Dj[2] + (a == 0 ? ph : R(0));
      const bool ok = sv[0] > R(0) && soc_det(sv) > R(0.25) * sv[0] * sv[0];
      if (!ok) { sv[0] = ph > S.sig0 ? ph : S.sig0; sv[1] = sv[2] = R(0); }
      const R dt = soc_det(sv);
      for (int a = 0; a < 3; ++a) w.s[3 * po + a] = sv[a];
      w.z[3 * po] = kappa * sv[0] / dt;
      w.z[3 * po + 1] = -kappa * sv[1] / dt;
      w.z[3 * po + 2] = -kappa * sv[2] / dt;
    }
  }
  __syncthreads();
  int stalls = 0;
  const bool proj = false;    // stage 2 uses the exact P
  bool centring = false;
  for (int it = 0; it < S.ipm_max; ++it) {
    const bool pc = kfinal >= R(0) && !centring;
    R target = kfinal < R(0) ? kappa : kfinal;
    // assemble H2 = P + sum A^T M A and -P D + sum A^T (z + M g), g = r_z + W d_s (affine when pc)
    {
      for (int v = threadIdx.x; v < nv; v += CL_NT) {
        R Dv[9], PD[3];
        cl_node_P(S, D, w, c.misc, v, proj, Dv, w.Dl, PD);
        R rhs[3] = {-PD[0], -PD[1], -PD[2]};
        const R Dn[3] = {w.Dl[3 * v], w.Dl[3 * v + 1], w.Dl[3 * v + 2]};
        for (int o = 0; o < nobs; ++o) {
          const int po = o * nv + v;
          R A[9], sv[3], zv[3];
          cl_frame(S, w, po, A);
          for (int a = 0; a < 3; ++a) { sv[a] = w.s[3 * po + a]; zv[a] = w.z[3 * po + a]; }
          const R ph = w.phi[po];
          R rz[3];
          for (int a = 0; a < 3; ++a)
            rz[a] = sv[a] - (A[a * 3] * Dn[0] + A[a * 3 + 1] * Dn[1] + A[a * 3 + 2] * Dn[2]) - (a == 0 ? ph : R(0));
          R W[9], Wi[9], lam[3];
          nt_scaling(sv, zv, W, Wi, lam);
          const R tg = pc ? R(0) : target;
          R r3[3] = {tg - (lam[0] * lam[0] + lam[1] * lam[1] + lam[2] * lam[2]), R(-2) * lam[0] * lam[1],
                     R(-2) * lam[0] * lam[2]};
          R ds[3];
          jordan_solve(lam, r3, ds);
          R M[9];
          for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b)
              M[a * 3 + b] = Wi[a * 3] * Wi[b] + Wi[a * 3 + 1] * Wi[3 + b] + Wi[a * 3 + 2] * Wi[6 + b];
          R g[3];
          for (int a = 0; a < 3; ++a) g[a] = rz[a] + W[a * 3] * ds[0] + W[a * 3 + 1] * ds[1] + W[a * 3 + 2] * ds[2];
          w.pm[6 * po] = M[0]; w.pm[6 * po + 1] = M[1]; w.pm[6 * po + 2] = M[2];
          w.pm[6 * po + 3] = M[4]; w.pm[6 * po + 4] = M[5]; w.pm[6 * po + 5] = M[8];
          for (int a = 0; a < 3; ++a) { w.pg[3 * po + a] = g[a]; w.prz[3 * po + a] = rz[a]; }
          R zg[3];
          for (int a = 0; a < 3; ++a) zg[a] = zv[a] + M[a * 3] * g[0] + M[a * 3 + 1] * g[1] + M[a * 3 + 2] * g[2];
          R MA[9];
          for (int a = 0; a < 3; ++a)
            for (int q = 0; q < 3; ++q)
              MA[a * 3 + q] = M[a * 3] * A[q] + M[a * 3 + 1] * A[3 + q] + M[a * 3 + 2] * A[6 + q];
          for (int i = 0; i < 3; ++i) {
            rhs[i] += A[i] * zg[0] + A[3 + i] * zg[1] + A[6 + i] * zg[2];
            for (int q = 0; q < 3; ++q) Dv[i * 3 + q] += A[i] * MA[q] + A[3 + i] * MA[3 + q] + A[6 + i] * MA[6 + q];
          }
        }
        for (int b = 0; b < 3; ++b)
          for (int a = b; a < 3; ++a) w.Dg[6 * v + sym3(a, b)] = Dv[a * 3 + b];
        for (int i = 0; i < 3; ++i) { c.vb[3 * v + i] = rhs[i]; w.rA[3 * v + i] = rhs[i]; }
      }
      __syncthreads();
      // H2 not positive definite means P is not either (the stage-1 root is not a minimiser of
      // its potential, and the QP of eq. dynamics-second-stage is not convex): no contact solution
      if (!cl_factor_w(S, D, BandSrc<R>{w.x0, w.dx, w.Dg, proj}, w, c.sm)) { *iters = it + 1; return ST_NOTPD; }
    }
    cl_back(D, w.Lg, c.sm);
    for (int i = threadIdx.x; i < N; i += CL_NT) w.pv[i] = c.vb[i];
    __syncthreads();
    if (pc) {
      // affine step length and duality measure -> centring target
      R aa = R(1e30), gap = R(0);
      for (int v = threadIdx.x; v < nv; v += CL_NT) {
        const R dD[3] = {w.pv[3 * v], w.pv[3 * v + 1], w.pv[3 * v + 2]};
        for (int o = 0; o < nobs; ++o) {
          const int po = o * nv + v;
          R A[9], sv[3], zv[3], dsa[3], dza[3], gm[3];
          cl_frame(S, w, po, A);
          const R M[9] = {w.pm[6 * po], w.pm[6 * po + 1], w.pm[6 * po + 2], w.pm[6 * po + 1], w.pm[6 * po + 3],
                          w.pm[6 * po + 4], w.pm[6 * po + 2], w.pm[6 * po + 4], w.pm[6 * po + 5]};
          for (int a = 0; a < 3; ++a) {
            const R ADd = A[a * 3] * dD[0] + A[a * 3 + 1] * dD[1] + A[a * 3 + 2] * dD[2];
            dsa[a] = ADd - w.prz[3 * po + a];
            gm[a] = w.pg[3 * po + a] - ADd;
            sv[a] = w.s[3 * po + a];
            zv[a] = w.z[3 * po + a];
            gap += sv[a] * zv[a];
          }
          for (int a = 0; a < 3; ++a) dza[a] = M[a * 3] * gm[0] + M[a * 3 + 1] * gm[1] + M[a * 3 + 2] * gm[2];
          aa = fmin(aa, fmin(soc_max_step(sv, dsa), soc_max_step(zv, dza)));
        }
      }
      aa = fmin(R(1), -cl_max(-aa, c.red));
      gap = cl_sum(gap, c.red);
      const R om = R(1) - aa;
      target = fmax(kfinal, om * om * om * gap / mm);
      centring = target == kfinal;
      // combined right-hand side: rhs_aff + sum A^T M (g - g_aff), g from
      // d_s = lam^-1 o (target e - lam o lam - (W^-1 ds_a) o (W dz_a)) (second-order term dropped
      // once the target is kfinal)
      for (int v = threadIdx.x; v < nv; v += CL_NT) {
        R rhs[3] = {w.rA[3 * v], w.rA[3 * v + 1], w.rA[3 * v + 2]};
        const R dD[3] = {w.pv[3 * v], w.pv[3 * v + 1], w.pv[3 * v + 2]};
        for (int o = 0; o < nobs; ++o) {
          const int po = o * nv + v;
          R A[9], W[9], Wi[9], lam[3], sv[3], zv[3], ga[3], rz[3];
          cl_frame(S, w, po, A);
          const R M[9] = {w.pm[6 * po], w.pm[6 * po + 1], w.pm[6 * po + 2], w.pm[6 * po + 1], w.pm[6 * po + 3],
                          w.pm[6 * po + 4], w.pm[6 * po + 2], w.pm[6 * po + 4], w.pm[6 * po + 5]};
          for (int a = 0; a < 3; ++a) {
            sv[a] = w.s[3 * po + a];
            zv[a] = w.z[3 * po + a];
            ga[a] = w.pg[3 * po + a];
            rz[a] = w.prz[3 * po + a];
          }
          nt_scaling(sv, zv, W, Wi, lam);
          R c3[3] = {R(0), R(0), R(0)};
          if (!centring) {
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
            w.pg[3 * po + a] = g;
            dg[a] = g - ga[a];
          }
          R Mdg[3];
          for (int a = 0; a < 3; ++a) Mdg[a] = M[a * 3] * dg[0] + M[a * 3 + 1] * dg[1] + M[a * 3 + 2] * dg[2];
          for (int i = 0; i < 3; ++i) rhs[i] += A[i] * Mdg[0] + A[3 + i] * Mdg[1] + A[6 + i] * Mdg[2];
        }
        for (int i = 0; i < 3; ++i) c.vb[3 * v + i] = rhs[i];
      }
      __syncthreads();
      cl_fwd(D, w.Lg, c.sm);
      cl_back(D, w.Lg, c.sm);
      for (int i = threadIdx.x; i < N; i += CL_NT) w.pv[i] = c.vb[i];
      __syncthreads();
    }
    const bool final_target = kfinal < R(0) || target == kfinal;
    // step length to the cone boundaries; the directions are kept for the update
    R amin = R(1e30), dmax = R(0);
    bool bad = false;
    for (int v = threadIdx.x; v < nv; v += CL_NT) {
      const R dD[3] = {w.pv[3 * v], w.pv[3 * v + 1], w.pv[3 * v + 2]};
      for (int i = 0; i < 3; ++i) {
        dmax = fmax(dmax, fabs(dD[i]));
        bad = bad || !(fabs(dD[i]) <= R(1e30));
      }
      for (int o = 0; o < nobs; ++o) {
        const int po = o * nv + v;
        R A[9], sv[3], zv[3], dsv[3], dz[3], gm[3];
        cl_frame(S, w, po, A);
        const R M[9] = {w.pm[6 * po], w.pm[6 * po + 1], w.pm[6 * po + 2], w.pm[6 * po + 1], w.pm[6 * po + 3],
                        w.pm[6 * po + 4], w.pm[6 * po + 2], w.pm[6 * po + 4], w.pm[6 * po + 5]};
        for (int a = 0; a < 3; ++a) {
          const R ADd = A[a * 3] * dD[0] + A[a * 3 + 1] * dD[1] + A[a * 3 + 2] * dD[2];
          dsv[a] = ADd - w.prz[3 * po + a];
          gm[a] = w.pg[3 * po + a] - ADd;
        }
        for (int a = 0; a < 3; ++a) dz[a] = M[a * 3] * gm[0] + M[a * 3 + 1] * gm[1] + M[a * 3 + 2] * gm[2];
        for (int a = 0; a < 3; ++a) {
          dmax = fmax(dmax, fabs(dsv[a]));
          bad = bad || !(fabs(dz[a]) <= R(1e30)) || !(fabs(dsv[a]) <= R(1e30));
          sv[a] = w.s[3 * po + a];
          zv[a] = w.z[3 * po + a];
          w.prz[3 * po + a] = dsv[a];
          w.pg[3 * po + a] = dz[a];
        }
        amin = fmin(amin, soc_max_step(sv, dsv));
        amin = fmin(amin, soc_max_step(zv, dz));
      }
    }
    bad = __syncthreads_or(bad);
    dmax = cl_max(dmax, c.red);
    amin = -cl_max(-amin, c.red);
    if (bad) { *iters = it + 1; return ST_NONFINITE; }
    const R alpha = fmin(R(1), R(0.99) * amin);
    stalls = alpha < R(1e-6) ? stalls + 1 : 0;
    if (stalls >= 5) { *iters = it + 1; return ST_CONTACT; }
    bool inside = true;
    for (int v = threadIdx.x; v < nv; v += CL_NT) {
      for (int o = 0; o < nobs; ++o) {
        const int po = o * nv + v;
        R sv[3], zv[3];
        for (int a = 0; a < 3; ++a) {
          sv[a] = w.s[3 * po + a] + alpha * w.prz[3 * po + a];
          zv[a] = w.z[3 * po + a] + alpha * w.pg[3 * po + a];
          w.s[3 * po + a] = sv[a];
          w.z[3 * po + a] = zv[a];
        }
        inside = inside && soc_inside(sv) && soc_inside(zv);
      }
      for (int i = 0; i < 3; ++i) w.Dl[3 * v + i] += alpha * w.pv[3 * v + i];
    }
    inside = __syncthreads_and(inside);
    if (!inside) { *iters = it + 1; return ST_CONTACT; }
    if (final_target && alpha == R(1) && dmax <= S.itol) { *iters = it + 1; return 0; }
  }
  *iters = S.ipm_max;
  return ST_CONTACT;
}

// ---- one step.  In: x0, misc g, c, u (and dx with warm, Dl with warm2).  Out: dx, Dl, the
//      contact geometry at x*, misc d, gd.  smooth: the smooth grasp and the kappa_c contact solve.
template <typename R>
__device__ int cl_step(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w, const ClothSm<R>& c,
                       bool smooth, int* nit, int* iit, bool warm, bool warm2) {
  R* misc = c.misc;
  if (threadIdx.x < 2) {
    const int l = threadIdx.x;
    const R cc[3] = {misc[M_C + 3 * l], misc[M_C + 3 * l + 1], misc[M_C + 3 * l + 2]};
    const R rho = sqrt(dot3(cc, cc));
    R dd;
    if (smooth) {
      dd = S.Dmax * exp(-rho / S.kh);
      const R f = rho > R(0) ? -dd / (S.kh * rho) : R(0);
      for (int i = 0; i < 3; ++i) misc[M_GD + 3 * l + i] = f * cc[i];
    } else {
      dd = rho <= S.rgrasp ? S.Dmax : R(0);
      for (int i = 0; i < 3; ++i) misc[M_GD + 3 * l + i] = R(0);
    }
    misc[M_D + l] = dd;
  }
  if (!warm2)
    for (int i = threadIdx.x; i < D.N; i += CL_NT) w.Dl[i] = R(0);
  __syncthreads();
  int st = cl_stage1(S, D, w, c, nit, warm);
  *iit = 0;
  bool zeroD = S.nobs == 0;
  if (!zeroD) {
    const R pmin = cl_contact_geometry(S, D, w, c.red);
    zeroD = !smooth && pmin >= R(0);          // Delta = 0 is the nonsmooth optimum
    if (!zeroD) st |= cl_stage2(S, D, w, c, S.kc, smooth ? R(-1) : S.khard, iit, warm2);
  }
  if (zeroD) {
    for (int i = threadIdx.x; i < D.N; i += CL_NT) w.Dl[i] = R(0);
    __syncthreads();
  }
  return st;
}

// x0 <- x0 + dx + Dl ; g <- g + u ; c <- c + u - (dx_a + Dl_a)
template <typename R>
__device__ __forceinline__ void cl_advance(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w, R* misc) {
  if (threadIdx.x < 6) {
    const int gi = threadIdx.x / 3, i = threadIdx.x % 3, a = S.grasp[gi];
    misc[M_C + threadIdx.x] += misc[M_U + threadIdx.x] - (w.dx[3 * a + i] + w.Dl[3 * a + i]);
    misc[M_G + threadIdx.x] += misc[M_U + threadIdx.x];
  }
  __syncthreads();
  for (int i = threadIdx.x; i < D.N; i += CL_NT) w.x0[i] += w.dx[i] + w.Dl[i];
  __syncthreads();
}

// ---- state transfer: q = [x, g]; records q [n_q] | c [6] | dx [3 nv] | Delta [3 nv]
template <typename R>
__device__ __forceinline__ void cl_load_q(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w, R* misc,
                                          const R* q) {
  for (int i = threadIdx.x; i < D.N; i += CL_NT) w.x0[i] = q[i];
  if (threadIdx.x < 6) {
    const R g = q[D.N + threadIdx.x];
    misc[M_G + threadIdx.x] = g;
    misc[M_C + threadIdx.x] = g - q[3 * S.grasp[threadIdx.x / 3] + threadIdx.x % 3];
  }
  __syncthreads();
}

template <typename R>
__device__ __forceinline__ void cl_store_q(const ClothDims& D, const ClothWS<R>& w, const R* misc, R* q) {
  for (int i = threadIdx.x; i < D.N; i += CL_NT) q[i] = w.x0[i];
  if (threadIdx.x < 6) q[D.N + threadIdx.x] = misc[M_G + threadIdx.x];
}

template <typename R>
__device__ __forceinline__ void cl_store_rec(const ClothDims& D, const ClothWS<R>& w, const R* misc, R* r) {
  cl_store_q(D, w, misc, r);
  if (threadIdx.x < 6) r[D.N + 6 + threadIdx.x] = misc[M_C + threadIdx.x];
  R* rd = r + D.N + 12;
  R* rD = rd + D.N;
  for (int i = threadIdx.x; i < D.N; i += CL_NT) { rd[i] = w.dx[i]; rD[i] = w.Dl[i]; }
}

template <typename R>
__device__ __forceinline__ void cl_load_rec(const ClothDims& D, const ClothWS<R>& w, R* misc, const R* r) {
  for (int i = threadIdx.x; i < D.N; i += CL_NT) w.x0[i] = r[i];
  if (threadIdx.x < 6) {
    misc[M_G + threadIdx.x] = r[D.N + threadIdx.x];
    misc[M_C + threadIdx.x] = r[D.N + 6 + threadIdx.x];
  }
  __syncthreads();
}

template <typename R>
__device__ __forceinline__ void cl_load_rec_dx(const ClothDims& D, const ClothWS<R>& w, const R* r) {
  for (int i = threadIdx.x; i < D.N; i += CL_NT) w.dx[i] = r[D.N + 12 + i];
}

template <typename R>
__device__ __forceinline__ void cl_load_rec_delta(const ClothDims& D, const ClothWS<R>& w, const R* r) {
  for (int i = threadIdx.x; i < D.N; i += CL_NT) w.Dl[i] = r[2 * D.N + 12 + i];
}

// some node has a nonzero Delta (the previous step ran stage 2)
template <typename R>
__device__ __forceinline__ bool cl_any_delta(const ClothDims& D, const ClothWS<R>& w) {
  bool nz = false;
  for (int i = threadIdx.x; i < D.N; i += CL_NT) nz = nz || w.Dl[i] != R(0);
  return __syncthreads_or(nz);
}

// penalty part of the planning loss at the state x0: this thread's share of the value; with
// seeds, its gradient is added to w.xb
template <typename R>
__device__ __forceinline__ R cl_penalty(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w, bool seeds) {
  R val = R(0);
  for (int v = threadIdx.x; v < D.nv; v += CL_NT) {
    const R X[3] = {w.x0[3 * v], w.x0[3 * v + 1], w.x0[3 * v + 2]};
    for (int o = 0; o < S.nobs; ++o) {
      if (S.ob_type[o] == CS_PLANE) continue;
      R ph, n[3];
      obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, (R*)nullptr);
      const R e = S.pen_m - ph > R(0) ? S.pen_m - ph : R(0);
      val += S.w_pen * e * e;
      if (seeds)
        for (int i = 0; i < 3; ++i) w.xb[3 * v + i] += R(-2) * S.w_pen * e * n[i];
    }
  }
  return val;
}

// ---- adjoint of one smooth step (eq. diff-sim with the total derivative).
//      in : w.xb = xbar+, misc GB = gbar+, the smooth solution (x0, dx, Dl, contact geometry)
//      out: w.xb = xbar, misc GB = gbar, misc UB = ubar
template <typename R>
__device__ int cl_adjoint(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w, const ClothSm<R>& c) {
  const int nv = D.nv, N = D.N;
  R* misc = c.misc;
  // mu = H2^{-1} xbar+, H2 = P + sum W(sigma), sigma = Delta + phi n
  for (int v = threadIdx.x; v < nv; v += CL_NT) {
    R Dv[9], Py[3];
    cl_node_P(S, D, w, misc, v, false, Dv, (const R*)nullptr, Py);
    for (int o = 0; o < S.nobs; ++o) {
      const int po = o * nv + v;
      const R n[3] = {w.nrm[3 * po], w.nrm[3 * po + 1], w.nrm[3 * po + 2]};
      R sg[3], lam[3], W[9];
      for (int i = 0; i < 3; ++i) sg[i] = w.Dl[3 * v + i] + w.phi[po] * n[i];
      cone_force_jac(sg, n, S.kc, S.mu, lam, W);
      for (int i = 0; i < 9; ++i) Dv[i] += W[i];
    }
    for (int b = 0; b < 3; ++b)
      for (int a = b; a < 3; ++a) w.Dg[6 * v + sym3(a, b)] = Dv[a * 3 + b];
    for (int i = 0; i < 3; ++i) c.vb[3 * v + i] = w.xb[3 * v + i];
  }
  __syncthreads();
  if (!cl_factor_w(S, D, BandSrc<R>{w.x0, w.dx, w.Dg, false}, w, c.sm)) return ST_NOTPD;
  cl_back(D, w.Lg, c.sm);
  for (int i = threadIdx.x; i < N; i += CL_NT) w.mu[i] = c.vb[i];
  __syncthreads();
  // xbar* = xbar+ - (dR/dx*)^T mu: contact part and spring third-derivative part
  for (int v = threadIdx.x; v < nv; v += CL_NT) {
    R xs[3] = {w.xb[3 * v], w.xb[3 * v + 1], w.xb[3 * v + 2]};
    R X[3];
    cl_X(w, v, X);
    const R mj[3] = {w.mu[3 * v], w.mu[3 * v + 1], w.mu[3 * v + 2]};
    for (int o = 0; o < S.nobs; ++o) {
      R ph, n[3], Nn[9];
      obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, Nn);
      R sg[3];
      for (int i = 0; i < 3; ++i) sg[i] = w.Dl[3 * v + i] + ph * n[i];
      R lam[3], W[9];
      cone_force_jac(sg, n, S.kc, S.mu, lam, W);
      R Wm[3], Lm[3];
      for (int i = 0; i < 3; ++i) Wm[i] = W[i * 3] * mj[0] + W[i * 3 + 1] * mj[1] + W[i * 3 + 2] * mj[2];
      cone_force_dn_T(sg, n, S.kc, S.mu, mj, Lm);
      const R nWm = dot3(n, Wm);
      for (int i = 0; i < 3; ++i) {
        const R NW = Nn[i * 3] * Wm[0] + Nn[i * 3 + 1] * Wm[1] + Nn[i * 3 + 2] * Wm[2];
        const R NL = Nn[i * 3] * Lm[0] + Nn[i * 3 + 1] * Lm[1] + Nn[i * 3 + 2] * Lm[2];
        xs[i] += -(n[i] * nWm + ph * NW) + NL;
      }
    }
    for (int t = 0; t < 12; ++t) {
      int u;
      R d[3], k, L;
      if (!cl_spring_at(S, D, w, v, t, u, d, k, L)) continue;
      const int a = (t & 1) ? u : v, b = (t & 1) ? v : u;
      R mt[3], dl[3], t3[3];
      for (int i = 0; i < 3; ++i) {
        mt[i] = w.mu[3 * b + i] - w.mu[3 * a + i];
        dl[i] = w.Dl[3 * b + i] - w.Dl[3 * a + i];
      }
      spring_d3(d, k, L, mt, dl, t3);
      const R sg = (t & 1) ? R(-1) : R(1);     // - on node b, + on node a
      for (int i = 0; i < 3; ++i) xs[i] += sg * t3[i];
    }
    for (int i = 0; i < 3; ++i) c.vb[3 * v + i] = xs[i];
  }
  // nu = (dF/dq*)^{-1} xbar*; not positive definite: the root is a saddle of the potential and
  // the step's Jacobian is undefined
  cl_diag(S, D, w, misc, false, R(0));
  __syncthreads();
  if (!cl_factor_w(S, D, BandSrc<R>{w.x0, w.dx, w.Dg, false}, w, c.sm)) return ST_NOTPD;
  cl_back(D, w.Lg, c.sm);
  for (int i = threadIdx.x; i < N; i += CL_NT) w.xb[i] = S.w * c.vb[i];
  __syncthreads();
  if (threadIdx.x < 2) {
    const int gi = threadIdx.x, a = S.grasp[gi];
    R gam = R(0);
    for (int i = 0; i < 3; ++i)
      gam += (w.dx[3 * a + i] - (misc[M_C + 3 * gi + i] + misc[M_U + 3 * gi + i])) * c.vb[3 * a + i] +
             w.mu[3 * a + i] * w.Dl[3 * a + i];
    for (int i = 0; i < 3; ++i) {
      w.xb[3 * a + i] += gam * misc[M_GD + 3 * gi + i];
      const R gbp = misc[M_GB + 3 * gi + i];
      const R dnu = misc[M_D + gi] * c.vb[3 * a + i];
      misc[M_GB + 3 * gi + i] = gbp + dnu - gam * misc[M_GD + 3 * gi + i];
      misc[M_UB + 3 * gi + i] = gbp + dnu;
    }
  }
  __syncthreads();
  return 0;
}

// ---- kernels: one CTA per rollout at a time (grid <= workspace slots)

// the rollout a CTA takes after rollout b: with more rollouts than CTAs, the next unstarted one,
// claimed from a counter zeroed before the launch (the first wave is b = blockIdx.x), so that a
// CTA whose rollouts were cheap takes more of them; without a counter, b + gridDim.x.  Every
// thread gets the same value.
__device__ __forceinline__ int cl_next_rollout(int b, int B, int* claim) {
  __shared__ int next;
  if (!claim) return b + (int)gridDim.x;
  if (B <= (int)gridDim.x) return B;
  __syncthreads();
  if (threadIdx.x == 0) next = (int)gridDim.x + atomicAdd(claim, 1);
  __syncthreads();
  return next;
}

template <typename R>
__global__ void __launch_bounds__(CL_NT) cloth_rollout_kernel(Scene<R> S, ClothDims D, int B, int H, const R* q0,
                                                             const R* U, R* traj, R* qH, int32_t* status,
                                                             int32_t* counters, R* slots, size_t slot_stride,
                                                             int* claim) {
  const ClothSm<R> c = cloth_sm<R>(D);
  const ClothWS<R> w = cloth_carve<R>(slots + blockIdx.x * slot_stride, D, S.nobs);
  const int nq = D.N + 6;
  const bool smooth = S.fwd_mode == CS_SMOOTH;
  for (int b = blockIdx.x; b < B; b = cl_next_rollout(b, B, claim)) {
    cl_load_q(S, D, w, c.misc, q0 + (size_t)b * nq);
    for (int i = threadIdx.x; i < D.N; i += CL_NT) w.Dl[i] = R(0);
    __syncthreads();
    if (traj) cl_store_q(D, w, c.misc, traj + (size_t)b * (H + 1) * nq);
    int st = 0;
    for (int t = 0; t < H; ++t) {
      if (threadIdx.x < 6) c.misc[M_U + threadIdx.x] = U[((size_t)b * H + t) * 6 + threadIdx.x];
      __syncthreads();
      int ni, ii;
      const bool w2 = cl_any_delta(D, w);
      const int s1 = cl_step(S, D, w, c, smooth, &ni, &ii, false, w2);
      st |= s1;
      if (counters && threadIdx.x == 0) {
        int32_t* cn = counters + ((size_t)b * H + t) * 3;
        cn[0] = ni; cn[1] = ii; cn[2] = s1;
      }
      cl_advance(S, D, w, c.misc);
      if (traj) cl_store_q(D, w, c.misc, traj + ((size_t)b * (H + 1) + t + 1) * nq);
    }
    if (qH) cl_store_q(D, w, c.misc, qH + (size_t)b * nq);
    if (threadIdx.x == 0 && status) status[b] = st;
    __syncthreads();
  }
}

// Forward rollout + checkpointed adjoint of one cloth rollout by one CTA (the schedule of
// vjp_rollout for ropes).  PH = VJP_FWD stops after the forward steps: L and the carry are
// written and *cost gets the forward's work (2 x Newton + 5 x interior-point iterations; -1: the
// rollout failed and its outputs are final); PH = VJP_BWD resumes from the carry at the last
// segment.
template <typename R, int PH = VJP_ALL>
__device__ void cl_vjp_rollout(const Scene<R>& S, const ClothDims& D, const ClothWS<R>& w, const ClothSm<R>& c,
                               int H, const R* q0, const R* U, const R* dLdtraj, R* Lout, R* dLdu, R* dLdq0,
                               int32_t* status, R* ck, int32_t* cost = nullptr) {
  const int N = D.N, nq = N + 6;
  const int rl = rec_len(D.nv);
  const int k = S.ckpt;
  const int nseg = (H + k - 1) / k;
  const bool fwd_smooth = S.grad_mode == CS_CONSISTENT;
  R* misc = c.misc;
  enum { FWD = 0, RECOMP = 1, BACK = 2 };
  R* seg = ck + (size_t)(nseg + 1) * rl;
  R* carry = ck + cloth_vjp_rec_elems(D.nv, H, k);
  int st = 0;
  R Lacc = R(0);
  int work = 0;
  int kind = FWD, t = 0, sgi = nseg - 1, t0 = 0, t1 = 0;
  auto begin_segment = [&]() {
    t0 = sgi * k;
    t1 = min(t0 + k, H);
    cl_load_rec(D, w, misc, ck + (size_t)sgi * rl);
    cl_load_rec_delta(D, w, ck + (size_t)sgi * rl);
    __syncthreads();
    cl_store_rec(D, w, misc, seg);
    if (t1 - t0 > 1) { kind = RECOMP; t = t0; } else { kind = BACK; t = t0; }
  };
  if constexpr ((PH & VJP_FWD) != 0) {
    cl_load_q(S, D, w, misc, q0);
    for (int i = threadIdx.x; i < N; i += CL_NT) { w.Dl[i] = R(0); w.dx[i] = R(0); w.xb[i] = R(0); }
    __syncthreads();
    cl_store_rec(D, w, misc, ck);
  } else {
    for (int i = threadIdx.x; i < N; i += CL_NT) { w.dx[i] = R(0); w.xb[i] = carry[i]; }
    if (threadIdx.x < 6) misc[M_GB + threadIdx.x] = carry[N + threadIdx.x];
    __syncthreads();
    begin_segment();
    __syncthreads();
  }
  while (true) {
    if (kind == BACK) {
      cl_load_rec(D, w, misc, seg + (size_t)(t - t0) * rl);
      // the smooth re-solve starts at the forward step's stage-1 solution and stage-2
      // displacement (record of q_{t+1})
      const R* rn = t + 1 < t1 ? seg + (size_t)(t + 1 - t0) * rl : ck + (size_t)(sgi + 1) * rl;
      cl_load_rec_dx(D, w, rn);
      cl_load_rec_delta(D, w, rn);
    }
    if (threadIdx.x < 6) misc[M_U + threadIdx.x] = U[6 * t + threadIdx.x];
    __syncthreads();
    int ni, ii;
    const bool w2 = kind == BACK || cl_any_delta(D, w);
    st |= cl_step(S, D, w, c, kind == BACK || fwd_smooth, &ni, &ii, kind == BACK, w2);
    if (st) break;                 // a failed step: the rollout's loss and gradient are undefined
    if (kind == FWD) work = min(work + 2 * ni + 5 * ii, 1 << 30);
    if (kind != BACK) {
      cl_advance(S, D, w, misc);
      if (kind == FWD) {
        if ((t + 1) % k == 0 || t == H - 1) cl_store_rec(D, w, misc, ck + (size_t)((t + k) / k) * rl);
        if (S.has_loss) Lacc += cl_penalty(S, D, w, false);
      } else {
        cl_store_rec(D, w, misc, seg + (size_t)(t + 1 - t0) * rl);
      }
    } else {
      st |= cl_adjoint(S, D, w, c);
      if (st) break;
      if (threadIdx.x < 6)
        dLdu[6 * t + threadIdx.x] =
            misc[M_UB + threadIdx.x] + (S.has_loss ? R(2) * S.w_u * U[6 * t + threadIdx.x] : R(0));
    }
    // seeds dL/dq_t of the state the adjoint reaches next (q_H after the forward, q_t after a
    // backward step); x0 holds that state in both cases
    const bool seed_now = (kind == FWD && t == H - 1) || kind == BACK;
    if (seed_now) {
      if (kind == FWD) {
        if (threadIdx.x < 6) misc[M_GB + threadIdx.x] = R(0);
        if (S.has_loss) {
          if (threadIdx.x == 0)
            for (int gi = 0; gi < S.n_goal; ++gi) {
              const int j = S.goal[gi];
              for (int i = 0; i < 3; ++i) {
                const R e = w.x0[3 * j + i] - S.goal_pos[gi][i];
                Lacc += S.w_goal * e * e;
                w.xb[3 * j + i] += R(2) * S.w_goal * e;
              }
            }
          for (int i = threadIdx.x; i < 6 * H; i += CL_NT) Lacc += S.w_u * U[i] * U[i];
        }
        __syncthreads();
      }
      const int ts = kind == FWD ? H : t;
      if (ts >= 1 && S.has_loss) cl_penalty(S, D, w, true);
      if (dLdtraj) {
        const R* sd = dLdtraj + (size_t)ts * nq;
        for (int i = threadIdx.x; i < N; i += CL_NT) w.xb[i] += sd[i];
        if (threadIdx.x < 6) misc[M_GB + threadIdx.x] += sd[N + threadIdx.x];
      }
      __syncthreads();
    }
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
    __syncthreads();
  }
  __syncthreads();
  Lacc = cl_sum(Lacc, c.red);
  if constexpr (PH == VJP_FWD) {
    if (!st) {                     // hand the seeds over; L is final
      for (int i = threadIdx.x; i < N; i += CL_NT) carry[i] = w.xb[i];
      if (threadIdx.x < 6) carry[N + threadIdx.x] = misc[M_GB + threadIdx.x];
      if (threadIdx.x == 0) {
        if (Lout) *Lout = Lacc;
        if (status) *status = 0;
        *cost = work;
      }
      __syncthreads();
      return;
    }
    if (threadIdx.x == 0) *cost = -1;
  }
  if (st) {                        // failed rollout: L = NaN, gradients zero
    for (int i = threadIdx.x; i < 6 * H; i += CL_NT) dLdu[i] = R(0);
    for (int i = threadIdx.x; i < N; i += CL_NT) w.xb[i] = R(0);
    if (threadIdx.x < 6) misc[M_GB + threadIdx.x] = R(0);
    Lacc = sizeof(R) == 4 ? R(nanf("")) : R(nan(""));
    __syncthreads();
  }
  if (dLdq0) {
    for (int i = threadIdx.x; i < N; i += CL_NT) dLdq0[i] = w.xb[i];
    if (threadIdx.x < 6) dLdq0[N + threadIdx.x] = misc[M_GB + threadIdx.x];
  }
  if (threadIdx.x == 0) {
    // the backward part leaves the forward's L unless the rollout failed
    if (Lout && (PH != VJP_BWD || st)) *Lout = Lacc;
    if (status) *status = st;
  }
  __syncthreads();
}

// the rollouts of one CTA (order[i] when given): the first wave by blockIdx.x, then handed out
// by the counter; the backward part skips a rollout whose forward failed (cost -1)
template <typename R, int PH>
__device__ __forceinline__ void cl_vjp_rollouts(const Scene<R>& S, const ClothDims& D, int B, int H, const R* q0,
                                                const R* U, const R* dLdtraj, R* Lout, R* dLdu, R* dLdq0,
                                                int32_t* status, R* slots, size_t slot_stride, R* ck,
                                                size_t ck_stride, int* claim, int32_t* cost,
                                                const int32_t* order) {
  const ClothSm<R> c = cloth_sm<R>(D);
  const ClothWS<R> w = cloth_carve<R>(slots + blockIdx.x * slot_stride, D, S.nobs);
  const int nq = D.N + 6;
  for (int i = blockIdx.x; i < B; i = cl_next_rollout(i, B, claim)) {
    const int b = order ? order[i] : i;
    if (PH == VJP_BWD && cost[b] < 0) continue;
    cl_vjp_rollout<R, PH>(S, D, w, c, H, q0 + (size_t)b * nq, U + (size_t)b * H * 6,
                          dLdtraj ? dLdtraj + (size_t)b * (H + 1) * nq : nullptr, Lout ? Lout + b : nullptr,
                          dLdu + (size_t)b * H * 6, dLdq0 ? dLdq0 + (size_t)b * nq : nullptr,
                          status ? status + b : nullptr, ck + (size_t)b * ck_stride, cost ? cost + b : nullptr);
  }
}

template <typename R>
__global__ void __launch_bounds__(CL_NT) cloth_vjp_kernel(Scene<R> S, ClothDims D, int B, int H, const R* q0,
                                                         const R* U, const R* dLdtraj, R* Lout, R* dLdu, R* dLdq0,
                                                         int32_t* status, R* slots, size_t slot_stride, R* ck,
                                                         size_t ck_stride, int* claim) {
  cl_vjp_rollouts<R, VJP_ALL>(S, D, B, H, q0, U, dLdtraj, Lout, dLdu, dLdq0, status, slots, slot_stride, ck,
                              ck_stride, claim, nullptr, nullptr);
}

// the forward parts of a two-part launch (more rollouts than CTAs): records, L, the carry and the
// cost of each rollout
template <typename R>
__global__ void __launch_bounds__(CL_NT) cloth_vjp_fwd_kernel(Scene<R> S, ClothDims D, int B, int H, const R* q0,
                                                             const R* U, const R* dLdtraj, R* Lout, R* dLdu,
                                                             R* dLdq0, int32_t* status, R* slots, size_t slot_stride,
                                                             R* ck, size_t ck_stride, int* claim, int32_t* cost) {
  cl_vjp_rollouts<R, VJP_FWD>(S, D, B, H, q0, U, dLdtraj, Lout, dLdu, dLdq0, status, slots, slot_stride, ck,
                              ck_stride, claim, cost, nullptr);
}

// the backward parts, rollout order[i] as the i-th one handed out (costliest first)
template <typename R>
__global__ void __launch_bounds__(CL_NT) cloth_vjp_bwd_kernel(Scene<R> S, ClothDims D, int B, int H, const R* U,
                                                             const R* dLdtraj, R* Lout, R* dLdu, R* dLdq0,
                                                             int32_t* status, R* slots, size_t slot_stride, R* ck,
                                                             size_t ck_stride, int* claim, int32_t* cost,
                                                             const int32_t* order) {
  cl_vjp_rollouts<R, VJP_BWD>(S, D, B, H, nullptr, U, dLdtraj, Lout, dLdu, dLdq0, status, slots, slot_stride, ck,
                              ck_stride, claim, cost, order);
}

}  // namespace cs
