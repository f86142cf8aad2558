// Shared device-side definitions of the CUDA path: the scene as the kernels see it, warp
// reductions and small dense 3x3 / 6x6 kernels.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "cordsim.h"

namespace cs {

constexpr unsigned FULL = 0xffffffffu;
constexpr int MAX_OBS = CS_MAX_OBSTACLES;
constexpr int MAX_GOAL = CS_MAX_GOAL;

// status bits (same meaning as CS_ST_* in cordsim.h)
constexpr int ST_NEWTON = CS_ST_NEWTON;
constexpr int ST_CONTACT = CS_ST_CONTACT;
constexpr int ST_NONFINITE = CS_ST_NONFINITE;
constexpr int ST_NOTPD = CS_ST_NOTPD;

// The scene in the kernels' real type, passed by value as a kernel parameter.
template <typename R>
struct Scene {
  int nv, npair, nobs, grasp[2];
  int kind, rows, cols;
  int fwd_mode, grad_mode, newton_max, ipm_max, ckpt;
  R w;              // node_mass / dt^2
  R m;              // node mass
  R grav[3];
  R Dmax, kh, kc, khard, kdecay, mu, rgrasp, rad, sig0, ntol, itol;
  R k1, k2, k3;     // rope: stretch (j,j+1), bend (j,j+2); cloth: stretch, shear, bend
  int so, nq;       // inertial variant (state [x, v, g]); state length
  R dt, cm, cb;     // time step; damp_alpha m / dt; damp_beta / dt
  int ob_type[MAX_OBS];
  R ob[MAX_OBS][6];
  const R* L1;      // rest lengths (rope: stretch [nv-1], bend [nv-2])
  const R* L2;
  // planning loss
  int has_loss, n_goal;
  int goal[MAX_GOAL];
  R goal_pos[MAX_GOAL][3];
  R w_goal, w_pen, pen_m, w_u;
};

template <typename R>
__device__ __forceinline__ R wsum(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(FULL, v, o);
  return v;
}

template <typename R>
__device__ __forceinline__ R wmax(R v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    R t = __shfl_xor_sync(FULL, v, o);
    v = t > v ? t : v;
  }
  return v;
}

// reciprocal square root (hardware approximation, within 2 ulp in single precision)
__device__ __forceinline__ float rsq(float x) { return rsqrtf(x); }
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }

template <typename R>
__device__ __forceinline__ R dot3(const R* a, const R* b) {
  return a[0] * b[0] + a[1] * b[1] + a[2] * b[2];
}

// ---- one obstacle: signed distance phi (minus node radius), normal n = grad phi, and the
//      normal's derivative N = dn/dx (symmetric 3x3; zero for planes, box faces and the inside)
template <typename R>
__device__ __forceinline__ void obstacle_eval(int type, const R* P, const R X[3], R rad, R& phi,
                                              R n[3], R* N /* 9 or nullptr */) {
  if (type == CS_PLANE) {
    phi = P[0] * X[0] + P[1] * X[1] + P[2] * X[2] - P[3] - rad;
    n[0] = P[0]; n[1] = P[1]; n[2] = P[2];
    if (N) for (int i = 0; i < 9; ++i) N[i] = R(0);
    return;
  }
  if (type == CS_SPHERE) {
    R r[3] = {X[0] - P[0], X[1] - P[1], X[2] - P[2]};
    R dist = sqrt(dot3(r, r));
    R inv = R(1) / dist;
    n[0] = r[0] * inv; n[1] = r[1] * inv; n[2] = r[2] * inv;
    phi = dist - P[3] - rad;
    if (N)
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k) N[i * 3 + k] = ((i == k ? R(1) : R(0)) - n[i] * n[k]) * inv;
    return;
  }
  // axis-aligned box
  R s[3], q[3];
  bool any = false;
  for (int i = 0; i < 3; ++i) {
    R rel = X[i] - P[i];
    s[i] = rel >= R(0) ? R(1) : R(-1);
    q[i] = rel * s[i] - P[3 + i];
    any = any || (q[i] > R(0));
  }
  if (any) {
    R qp[3];
    for (int i = 0; i < 3; ++i) qp[i] = q[i] > R(0) ? q[i] : R(0);
    R dist = sqrt(dot3(qp, qp));
    R inv = R(1) / dist;
    for (int i = 0; i < 3; ++i) n[i] = s[i] * qp[i] * inv;
    phi = dist - rad;
    if (N)
      for (int i = 0; i < 3; ++i)
        for (int k = 0; k < 3; ++k)
          N[i * 3 + k] = ((i == k && q[i] > R(0)) ? R(1) : R(0)) * inv - n[i] * n[k] * inv;
  } else {
    int km = 0;
    for (int i = 1; i < 3; ++i)
      if (q[i] > q[km]) km = i;
    phi = q[km] - rad;
    n[0] = n[1] = n[2] = R(0);
    n[km] = s[km];
    if (N) for (int i = 0; i < 9; ++i) N[i] = R(0);
  }
}

// ---- barrier of the dual friction cone {s_n >= mu |s_t|} in world coordinates:
//      sigma = slack vector, s_n = n.sigma, g = (1+mu^2) s_n^2 - mu^2 |sigma|^2,
//      b = -kappa/2 log g, lam = -grad b, W = hess b.
template <typename R>
__device__ __forceinline__ bool cone_inside(const R sg[3], const R n[3], R mu) {
  R sn = dot3(n, sg);
  R g = (R(1) + mu * mu) * sn * sn - mu * mu * dot3(sg, sg);
  return sn > R(0) && g > R(0);
}

template <typename R>
__device__ __forceinline__ void cone_force(const R sg[3], const R n[3], R kappa, R mu, R lam[3]) {
  R sn = dot3(n, sg);
  R g = (R(1) + mu * mu) * sn * sn - mu * mu * dot3(sg, sg);
  R c = kappa / g;
  for (int i = 0; i < 3; ++i) lam[i] = c * ((R(1) + mu * mu) * sn * n[i] - mu * mu * sg[i]);
}

template <typename R>
__device__ __forceinline__ void cone_force_jac(const R sg[3], const R n[3], R kappa, R mu,
                                               R lam[3], R W[9]) {
  R sn = dot3(n, sg);
  R g = (R(1) + mu * mu) * sn * sn - mu * mu * dot3(sg, sg);
  R a[3];
  for (int i = 0; i < 3; ++i) a[i] = (R(1) + mu * mu) * sn * n[i] - mu * mu * sg[i];
  R c1 = kappa / g, c2 = R(2) * kappa / (g * g);
  for (int i = 0; i < 3; ++i) {
    lam[i] = c1 * a[i];
    for (int k = 0; k < 3; ++k)
      W[i * 3 + k] = c1 * ((i == k ? mu * mu : R(0)) - (R(1) + mu * mu) * n[i] * n[k]) +
                     c2 * a[i] * a[k];
  }
}

// transpose-product of d lam / d n with a vector m:  (d lam/d n)^T m
template <typename R>
__device__ __forceinline__ void cone_force_dn_T(const R sg[3], const R n[3], R kappa, R mu,
                                                const R m[3], R out[3]) {
  R sn = dot3(n, sg);
  R g = (R(1) + mu * mu) * sn * sn - mu * mu * dot3(sg, sg);
  R a[3];
  for (int i = 0; i < 3; ++i) a[i] = (R(1) + mu * mu) * sn * n[i] - mu * mu * sg[i];
  R c1 = kappa * (R(1) + mu * mu) / g;
  R c2 = R(2) * kappa * (R(1) + mu * mu) * sn / (g * g);
  R nm = dot3(n, m), am = dot3(a, m);
  // d lam/dn = c1 (n sg^T + sn I) - c2 a sg^T
  for (int i = 0; i < 3; ++i) out[i] = c1 * (sg[i] * nm + sn * m[i]) - c2 * sg[i] * am;
}

// product of d lam / d n with a vector v: (d lam/d n) v
template <typename R>
__device__ __forceinline__ void cone_force_dn(const R sg[3], const R n[3], R kappa, R mu,
                                              const R v[3], R out[3]) {
  R sn = dot3(n, sg);
  R g = (R(1) + mu * mu) * sn * sn - mu * mu * dot3(sg, sg);
  R a[3];
  for (int i = 0; i < 3; ++i) a[i] = (R(1) + mu * mu) * sn * n[i] - mu * mu * sg[i];
  R c1 = kappa * (R(1) + mu * mu) / g;
  R c2 = R(2) * kappa * (R(1) + mu * mu) * sn / (g * g);
  R sv = dot3(sg, v);
  for (int i = 0; i < 3; ++i) out[i] = c1 * (n[i] * sv + sn * v[i]) - c2 * a[i] * sv;
}

// ---- second-order cone machinery of the stage-2 interior point.
//      The dual friction cone {s_n >= mu |s_t|} becomes the standard cone Q = {x0 >= |x_{1:2}|}
//      in the scaled coordinates s = A sigma, A = [n; mu t1; mu t2]; contact force lam = A^T z.

// unit tangents completing n (Duff et al., "Building an Orthonormal Basis, Revisited", JCGT 2017)
template <typename R>
__device__ __forceinline__ void tangent_frame(const R n[3], R t1[3], R t2[3]) {
  const R sg = n[2] >= R(0) ? R(1) : R(-1);
  const R a = R(-1) / (sg + n[2]);
  const R b = n[0] * n[1] * a;
  t1[0] = R(1) + sg * n[0] * n[0] * a; t1[1] = sg * b; t1[2] = -sg * n[0];
  t2[0] = b; t2[1] = sg + n[1] * n[1] * a; t2[2] = -n[1];
}

template <typename R>
__device__ __forceinline__ void cone_frame(const R n[3], R mu, R A[9]) {
  R t1[3], t2[3];
  tangent_frame(n, t1, t2);
  for (int i = 0; i < 3; ++i) { A[i] = n[i]; A[3 + i] = mu * t1[i]; A[6 + i] = mu * t2[i]; }
}

template <typename R>
__device__ __forceinline__ R soc_det(const R x[3]) { return x[0] * x[0] - x[1] * x[1] - x[2] * x[2]; }

template <typename R>
__device__ __forceinline__ bool soc_inside(const R x[3]) { return x[0] > R(0) && soc_det(x) > R(0); }

// v with x o v = r (Jordan product x o v = (x.v, x0 v1 + v0 x1))
template <typename R>
__device__ __forceinline__ void jordan_solve(const R x[3], const R r[3], R v[3]) {
  const R v0 = (x[0] * r[0] - x[1] * r[1] - x[2] * r[2]) / soc_det(x);
  v[0] = v0;
  v[1] = (r[1] - x[1] * v0) / x[0];
  v[2] = (r[2] - x[2] * v0) / x[0];
}

// Nesterov-Todd scaling of s, z in int Q: symmetric W with W z = W^{-1} s (Vandenberghe 2010)
template <typename R>
__device__ __forceinline__ void nt_scaling(const R s[3], const R z[3], R W[9], R Wi[9], R lam[3]) {
  const R ds = soc_det(s), dz = soc_det(z);
  const R rs = R(1) / sqrt(ds), rz = R(1) / sqrt(dz);
  R sb[3] = {s[0] * rs, s[1] * rs, s[2] * rs};
  R zb[3] = {z[0] * rz, z[1] * rz, z[2] * rz};
  const R gam = sqrt(R(0.5) * (R(1) + sb[0] * zb[0] + sb[1] * zb[1] + sb[2] * zb[2]));
  const R ig = R(1) / (R(2) * gam);
  R wb[3] = {(sb[0] + zb[0]) * ig, (sb[1] - zb[1]) * ig, (sb[2] - zb[2]) * ig};
  const R iv = R(1) / sqrt(R(2) * (wb[0] + R(1)));
  R v[3] = {(wb[0] + R(1)) * iv, wb[1] * iv, wb[2] * iv};
  const R beta = sqrt(sqrt(ds / dz));
  R Jv[3] = {v[0], -v[1], -v[2]};
  for (int i = 0; i < 3; ++i)
    for (int k = 0; k < 3; ++k) {
      const R J = i == k ? (i == 0 ? R(1) : R(-1)) : R(0);
      W[i * 3 + k] = beta * (R(2) * v[i] * v[k] - J);
      Wi[i * 3 + k] = (R(2) * Jv[i] * Jv[k] - J) / beta;
    }
  for (int i = 0; i < 3; ++i) lam[i] = W[i * 3] * z[0] + W[i * 3 + 1] * z[1] + W[i * 3 + 2] * z[2];
}

// largest alpha with x + alpha dx in Q (1e30 when unbounded), x in int Q.  Computed in the frame
// where x is the cone's centre: with g = sqrt(det x) and xh = x / g, the hyperbolic rotation that
// takes xh to e = (1, 0, 0) takes dx / g to y with y0 = (xh0 dx0 - xh1.dx1) / g and
// y1 = dx1 / g - (y0 + dx0 / g) / (xh0 + 1) xh1; the step to the boundary is 1 / (|y1| - y0) when
// that is positive (an eigenvalue y0 - |y1| of y reaches -1).  Well conditioned near the boundary,
// unlike the roots of the quadratic det(x + alpha dx) = 0.
template <typename R>
__device__ __forceinline__ R soc_max_step(const R x[3], const R dx[3]) {
  const R ig = rsq(soc_det(x));
  const R xh[3] = {x[0] * ig, x[1] * ig, x[2] * ig};
  const R y0 = (xh[0] * dx[0] - xh[1] * dx[1] - xh[2] * dx[2]) * ig;
  const R f = (y0 + dx[0] * ig) / (xh[0] + R(1));
  const R y1 = dx[1] * ig - f * xh[1], y2 = dx[2] * ig - f * xh[2];
  const R t = sqrt(y1 * y1 + y2 * y2) - y0;
  return t > R(0) ? R(1) / t : R(1e30);
}

// ---- spring k/2 (|d| - L)^2 with d = x_b - x_a: force on b (f = dE/dx_b), and the Hessian
//      block H = k [u u^T + c (I - u u^T)], c = 1 - L/l (clamped at 0 when `proj`).
template <typename R>
__device__ __forceinline__ void spring_eval(const R d[3], R k, R L, bool proj, R f[3], R H[9]) {
  R l = sqrt(dot3(d, d));
  R inv = R(1) / l;
  R u[3] = {d[0] * inv, d[1] * inv, d[2] * inv};
  R c = R(1) - L * inv;
  R fm = k * (l - L);
  for (int i = 0; i < 3; ++i) f[i] = fm * u[i];
  if (proj && c < R(0)) c = R(0);
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j)
      H[i * 3 + j] = k * ((R(1) - c) * u[i] * u[j] + (i == j ? c : R(0)));
}

// Third-derivative contraction of the spring energy: grad_d [ mt^T H(d) dl ] with mt, dl the
// differences (b - a) of two node vectors:
//   (k L / l^2) [ (mt.dl) u + (u.dl) mt + (u.mt) dl - 3 (u.mt)(u.dl) u ].
// It is symmetric in (mt, dl); the result acts with + on node b and - on node a.
template <typename R>
__device__ __forceinline__ void spring_d3(const R d[3], R k, R L, const R mt[3], const R dl[3],
                                          R out[3]) {
  R l = sqrt(dot3(d, d));
  R inv = R(1) / l;
  R u[3] = {d[0] * inv, d[1] * inv, d[2] * inv};
  R c = k * L * inv * inv;
  R md = dot3(mt, dl), ud = dot3(u, dl), um = dot3(u, mt);
  for (int i = 0; i < 3; ++i)
    out[i] = c * (md * u[i] + ud * mt[i] + um * dl[i] - R(3) * um * ud * u[i]);
}

// ---- 6x6 dense kernels (row-major, lower Cholesky with reciprocal diagonal) -----------------
template <typename R>
__device__ __forceinline__ bool chol6(R* T) {
  bool ok = true;
#pragma unroll
  for (int j = 0; j < 6; ++j) {
    R s = T[j * 6 + j];
#pragma unroll
    for (int k = 0; k < j; ++k) s -= T[j * 6 + k] * T[j * 6 + k];
    ok = ok && (s > R(0));
    R iv = rsq(s > R(0) ? s : R(1));
    T[j * 6 + j] = iv;
#pragma unroll
    for (int i = j + 1; i < 6; ++i) {
      R t = T[i * 6 + j];
#pragma unroll
      for (int k = 0; k < j; ++k) t -= T[i * 6 + k] * T[j * 6 + k];
      T[i * 6 + j] = t * iv;
    }
  }
  return ok;
}

// y <- L^{-1} y, y with element stride `st`
template <typename R>
__device__ __forceinline__ void lsolve6(const R* L, R* y, int st) {
  R v[6];
#pragma unroll
  for (int i = 0; i < 6; ++i) {
    R t = y[i * st];
#pragma unroll
    for (int k = 0; k < i; ++k) t -= L[i * 6 + k] * v[k];
    v[i] = t * L[i * 6 + i];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i * st] = v[i];
}

// y <- L^{-T} y
template <typename R>
__device__ __forceinline__ void ltsolve6(const R* L, R* y, int st) {
  R v[6];
#pragma unroll
  for (int i = 5; i >= 0; --i) {
    R t = y[i * st];
#pragma unroll
    for (int k = i + 1; k < 6; ++k) t -= L[k * 6 + i] * v[k];
    v[i] = t * L[i * 6 + i];
  }
#pragma unroll
  for (int i = 0; i < 6; ++i) y[i * st] = v[i];
}

}  // namespace cs
