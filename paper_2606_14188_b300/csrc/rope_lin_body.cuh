// The body of rope_lin.cuh, included once per step variant: namespace RC_NS, and RC_SO_ON(S)
// true only in the inertial variant's copy (false at compile time in the quasi-static copy,
// which then holds none of the inertial code).  No include guard: rope_lin.cuh includes it twice.
namespace cs {
namespace RC_NS {

template <typename R>
__device__ __forceinline__ bool block_chol_pairs(R* T, R* B, int N);

// ------------------------------------------------------------------------------------------
// the smooth step of each job and its record
// ------------------------------------------------------------------------------------------
template <typename R, int NPT>
__global__ void __launch_bounds__(NT, (ctas_per_sm<R, NPT>())) rope_cta_lin_step_kernel(
    Scene<R> S, int B, int H, const R* Z, const R* Vc, R* fac, size_t fac_stride, int32_t* status) {
  const int nq = S.nq;
  Sm<R> w = sm_carve<R>(reinterpret_cast<R*>(rc_smem), NPT, S.nobs);
  Red rb;
  Nd<R, NPT> N;
  zero_nd(N);
  load_rest(S, N);
  const size_t fb = fac_block(NPT), fs = fac_step_elems(NPT, S.nv);
  const int tid = threadIdx.x;
  for (long long job = blockIdx.x; job < (long long)B * H; job += gridDim.x) {
    const int b = (int)(job / H), t = (int)(job % H);
    const R* z = Z + ((size_t)b * (H + 1) + t) * nq;
    R* rec = fac + (size_t)b * fac_stride + (size_t)t * fs;
    load_q(S, N, w, z);
    if (tid < 6) w.misc[M_U + tid] = Vc[(size_t)job * 6 + tid];
    // stage 1 starts at the nominal next state
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      const int j = node_of(k);
#pragma unroll
      for (int i = 0; i < 3; ++i) N.dx[k][i] = j < S.nv ? z[nq + 3 * j + i] - z[3 * j + i] : R(0);
    }
    int ni, ii;
    int st = sim_step(S, N, w, rb, true, &ni, &ii, true, false);
    if (!st) {
      __syncthreads();
      assemble_h2(S, N, w);                           // H2 = P + sum A^T W^-2 A at the solution
      __syncthreads();
      if (!block_chol_pairs(w.T, w.B, S.npair)) st = ST_NOTPD;
      copy_block(rec, w.T, fb);
      __syncthreads();
      assemble_P(S, N, w, false, false);              // H1 = dF/dq* at x*
      __syncthreads();
      if (!block_chol_pairs(w.T, w.B, S.npair)) st = ST_NOTPD;
      copy_block(rec + fb, w.T, fb);
    }
    R* rn = rec + 2 * fb;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      const int j = node_of(k);
      if (j < S.nv)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          rn[3 * j + i] = N.x0[k][i];
          rn[3 * S.nv + 3 * j + i] = N.dx[k][i];
          rn[6 * S.nv + 3 * j + i] = N.Dl[k][i];
        }
    }
    if (tid < 32) rn[9 * S.nv + tid] = w.misc[tid];
    if (tid == 0) {
      rn[9 * S.nv + 32] = R(st);
      if (st && status) atomicOr(reinterpret_cast<int*>(status) + b, st);
    }
    __syncthreads();
  }
}

// ------------------------------------------------------------------------------------------
// the tangents
// ------------------------------------------------------------------------------------------
// Block Cholesky H = L L^T of a block-tridiagonal matrix in node pairs: per pair row p the
// diagonal factor L_p (6 x 6 lower, reciprocal diagonal) and the coupling M_p = L_{p,p-1}
// (6 x 6).  block_chol_pairs factors in place in the pair storage (L_p over the lower triangle of
// H_pp in T, M_p over H_{p,p-1} in B); every thread of a 64-thread CTA calls it and gets whether H
// is positive definite.
template <typename R>
__device__ __forceinline__ bool block_chol_pairs(R* T, R* B, int N) {
  const int tid = threadIdx.x;
  bool ok = true;
  for (int p = 0; p < N; ++p) {
    // M_p = H_{p,p-1} L_{p-1}^-T, row i by thread i
    if (p > 0 && tid < 6) {
      R L[36], y[6];
      ld_low(T, p - 1, L);
#pragma unroll
      for (int c = 0; c < 6; ++c) y[c] = B[cr_m(p, tid * 6 + c)];
      lsolve6(L, y, 1);
#pragma unroll
      for (int c = 0; c < 6; ++c) B[cr_m(p, tid * 6 + c)] = y[c];
    }
    __syncthreads();
    // H_pp - M_p M_p^T, packed entry e by thread e
    if (p > 0 && tid < 21) {
      const int a = (tid >= 1) + (tid >= 3) + (tid >= 6) + (tid >= 10) + (tid >= 15);
      const int b2 = tid - a * (a + 1) / 2;
      R v = T[rt(p, a, b2)];
#pragma unroll
      for (int q = 0; q < 6; ++q) v -= B[cr_m(p, a * 6 + q)] * B[cr_m(p, b2 * 6 + q)];
      T[rt(p, a, b2)] = v;
    }
    __syncthreads();
    if (tid == 0) {
      R L[36];
      ld_low(T, p, L);
      ok = chol6(L) && ok;
#pragma unroll
      for (int i = 0; i < 6; ++i)
#pragma unroll
        for (int q = 0; q <= i; ++q) T[rt(p, i, q)] = L[i * 6 + q];
    }
    __syncthreads();
  }
  return __syncthreads_and(ok);
}

// shared memory of rope_lin_tangent_kernel (elements of R): the factor of H1 [72 N] (then the dR/dx*
// blocks: Kc [9 nv], Ks [2 springs][6 (symmetric)] x nv, 21 nv <= 72 N), the factor of H2 [72 N],
// the step's scalars [32], the grasped nodes' dx and Delta [12], then the direction columns,
// element e of the column of thread c at [e * dpr + c] (e = 6 p + a for element a of pair p).  A
// factor holds [L_p (36, zeros above) | M_p (36)] at 72 p.
__host__ __device__ inline size_t lin_fixed_elems(int npair, int nv) {
  (void)nv;
  return 144 * (size_t)npair + 32 + 12;
}
__host__ __device__ inline size_t lin_smem_elems(int npair, int nv, int dpr) {
  return (lin_fixed_elems(npair, nv) + 3) / 4 * 4 + 6 * (size_t)npair * dpr;
}

// four consecutive elements by vector loads (one float4, or two double2); p 16-byte aligned
template <typename R>
__device__ __forceinline__ void ld_vec(const R* p, R* v) {
  if (sizeof(R) == 4) {
    const float4 q = *reinterpret_cast<const float4*>(p);
    v[0] = q.x; v[1] = q.y; v[2] = q.z; v[3] = q.w;
  } else {
    const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
}
template <typename R>
__device__ __forceinline__ void ld36(const R* p, R* v) {
#pragma unroll
  for (int i = 0; i < 9; ++i) ld_vec(p + 4 * i, v + 4 * i);
}

// a record's factor block (T, B of the pair storage, rows 0..N-1) into the layout above
template <typename R>
__device__ __forceinline__ void unpack_factor(const R* h, int NP, int N, R* F) {
  const R* hT = h;
  const R* hB = h + (size_t)LDT * NP;
  for (int i = threadIdx.x; i < 72 * N; i += blockDim.x) {
    const int p = i / 72, e = i % 72;
    R v;
    if (e < 36) {
      const int a = e / 6, b2 = e % 6;
      v = b2 <= a ? hT[rt(p, a, b2)] : R(0);
    } else {
      v = p > 0 ? hB[cr_m(p, e - 36)] : R(0);
    }
    F[i] = v;
  }
}

// x <- H^-1 x for one column (element (p, a) at r[(6 p + a) ld]) with a factor F of the layout above:
// L y = x forward, then L^T x = y backward, one pair row at a time with its neighbour's values in
// registers
template <typename R>
__device__ __forceinline__ void block_solve_col(const R* F, R* r, int ld, int N) {
  auto X = [&](int p, int a) -> R& { return r[(6 * p + a) * ld]; };
  R prev[6] = {0, 0, 0, 0, 0, 0};
  for (int p = 0; p < N; ++p) {
    R y[6], L[36];
#pragma unroll
    for (int a = 0; a < 6; ++a) y[a] = X(p, a);
    if (p > 0) {
      R M[36];
      ld36(F + 72 * p + 36, M);
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int q = 0; q < 6; ++q) y[a] -= M[a * 6 + q] * prev[q];
    }
    ld36(F + 72 * p, L);
    lsolve6(L, y, 1);
#pragma unroll
    for (int a = 0; a < 6; ++a) { X(p, a) = y[a]; prev[a] = y[a]; }
  }
  for (int p = N - 1; p >= 0; --p) {
    R y[6], L[36];
#pragma unroll
    for (int a = 0; a < 6; ++a) y[a] = X(p, a);
    if (p < N - 1) {
      R M[36];
      ld36(F + 72 * (p + 1) + 36, M);
#pragma unroll
      for (int q = 0; q < 6; ++q)
#pragma unroll
        for (int a = 0; a < 6; ++a) y[q] -= M[a * 6 + q] * prev[a];
    }
    ld36(F + 72 * p, L);
    ltsolve6(L, y, 1);
#pragma unroll
    for (int a = 0; a < 6; ++a) { X(p, a) = y[a]; prev[a] = y[a]; }
  }
}

// Inertial variant, direction e of node jn's coordinate cc.  With rhs1: adds (D/dt) e - G e to
// the column, G = d/dx [(D/dt) y] at y = x* - x; else (rhs2) adds -G e at y = Delta.  For the
// spring (jn, jo), u the unit vector from jn to jo at the step start, c = (damp_beta/dt) k and
// yd = y_jo - y_jn, the damping force on jo is f = c u (u.yd) (on jn -f) and
// df/d(x_jo - x_jn) = (c/l) [(u.yd)(I - u u^T) + u (yd - u (u.yd))^T].  yofs: y in the record
// (3 nv: dx, 6 nv: Delta).
template <typename R, typename Col>
__device__ __forceinline__ void damp_tangent(const Scene<R>& S, const R* rn, int jn, int cc, int yofs, Col E,
                                             bool with_D) {
  const int nv = S.nv;
  if (with_D) E(jn, cc) += S.cm;
#pragma unroll
  for (int si = 0; si < 4; ++si) {
    const int o = si == 0 ? -2 : (si == 1 ? -1 : (si == 2 ? 1 : 2));
    const int jo = jn + o;
    if (jo < 0 || jo >= nv) continue;
    const int a = o < 0 ? jo : jn;
    (void)a;
    R ua[3], yd[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      ua[i] = rn[3 * jo + i] - rn[3 * jn + i];
      yd[i] = rn[yofs + 3 * jo + i] - rn[yofs + 3 * jn + i];
    }
    const R l = sqrt(dot3(ua, ua)), il = R(1) / l;
#pragma unroll
    for (int i = 0; i < 3; ++i) ua[i] *= il;
    const R cs = S.cb * ((si == 1 || si == 2) ? S.k1 : S.k2);
    const R uy = dot3(ua, yd);
    // G e at jo (e = e_cc at jn, d/dx_jn of (x_jo - x_jn) = -I): -J e; at jn: +J e
    R Je[3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
      Je[i] = cs * il * (uy * ((i == cc ? R(1) : R(0)) - ua[i] * ua[cc]) + ua[i] * (yd[cc] - ua[cc] * uy));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      E(jn, i) -= Je[i];
      E(jo, i) += Je[i];
      if (with_D) {
        const R t = cs * ua[i] * ua[cc];
        E(jn, i) += t;
        E(jo, i) -= t;
      }
    }
  }
}

// dR/dx* blocks of a job from its record's node state: per node Kc = sum_o [-W (n n^T + phi N) +
// (d lam / d n) N], per spring (j, j+o) the third-derivative block Ks with t = Ks (v_b - v_a)
template <typename R>
__device__ __forceinline__ void dR_blocks(const Scene<R>& S, const R* rn, R* Kc, R* Ks) {
  const int nv = S.nv;
  for (int j = threadIdx.x; j < nv; j += blockDim.x) {
    R X[3], Dj[3];
    #pragma unroll
    for (int i = 0; i < 3; ++i) {
      X[i] = rn[3 * j + i] + rn[3 * nv + 3 * j + i];
      Dj[i] = rn[6 * nv + 3 * j + i];
    }
    R K[9];
    #pragma unroll
    for (int i = 0; i < 9; ++i) K[i] = R(0);
    for (int o = 0; o < S.nobs; ++o) {
      R ph, n[3], Nm[9];
      obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, Nm);
      R sg[3];
      #pragma unroll
      for (int i = 0; i < 3; ++i) sg[i] = Dj[i] + ph * n[i];
      R lam[3], W[9];
      cone_force_jac(sg, n, S.kc, S.mu, lam, W);
      // d lam / d n = c1 (n sg^T + sn I) - c2 a sg^T (as cone_force_dn)
      const R mu2 = S.mu * S.mu, sn = dot3(n, sg);
      const R g = (R(1) + mu2) * sn * sn - mu2 * dot3(sg, sg);
      const R c1 = S.kc * (R(1) + mu2) / g, c2 = R(2) * S.kc * (R(1) + mu2) * sn / (g * g);
      R Gn[9], Ds[9];
      #pragma unroll
      for (int a = 0; a < 3; ++a)
        #pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
          const R aa = (R(1) + mu2) * sn * n[a] - mu2 * sg[a];
          Gn[a * 3 + bb] = c1 * (n[a] * sg[bb] + (a == bb ? sn : R(0))) - c2 * aa * sg[bb];
          Ds[a * 3 + bb] = n[a] * n[bb] + ph * Nm[a * 3 + bb];
        }
      #pragma unroll
      for (int a = 0; a < 3; ++a)
        #pragma unroll
        for (int bb = 0; bb < 3; ++bb) {
          R tt = R(0);
          #pragma unroll
          for (int e = 0; e < 3; ++e) tt += -W[a * 3 + e] * Ds[e * 3 + bb] + Gn[a * 3 + e] * Nm[e * 3 + bb];
          K[a * 3 + bb] += tt;
        }
    }
    #pragma unroll
    for (int i = 0; i < 9; ++i) Kc[9 * j + i] = K[i];
    for (int o = 1; o <= 2; ++o) {
      const int b2 = j + o;
      R Sy[6] = {0, 0, 0, 0, 0, 0};
      if (b2 < nv) {
        const R kk = o == 1 ? S.k1 : S.k2;
        const R Lr = o == 1 ? S.L1[j] : S.L2[j];
        R dv[3], dl[3];
        #pragma unroll
        for (int i = 0; i < 3; ++i) {
          dv[i] = (rn[3 * b2 + i] + rn[3 * nv + 3 * b2 + i]) - X[i];
          dl[i] = rn[6 * nv + 3 * b2 + i] - Dj[i];
        }
        // spring_d3 as a matrix on mt: c (u dl^T + (u.dl) I + dl u^T - 3 (u.dl) u u^T), symmetric
        const R l = sqrt(dot3(dv, dv)), inv = R(1) / l;
        const R uu[3] = {dv[0] * inv, dv[1] * inv, dv[2] * inv};
        const R cc2 = kk * Lr * inv * inv, ud = dot3(uu, dl);
        int e = 0;
        #pragma unroll
        for (int a = 0; a < 3; ++a)
          #pragma unroll
          for (int bb = a; bb < 3; ++bb, ++e)
            Sy[e] = cc2 * (uu[a] * dl[bb] + (a == bb ? ud : R(0)) + dl[a] * uu[bb] - R(3) * ud * uu[a] * uu[bb]);
      }
      #pragma unroll
      for (int e = 0; e < 6; ++e) Ks[(2 * j + o - 1) * 6 + e] = Sy[e];
    }
  }
}

// one CTA of 32 ceil(dpr / 32) threads per job; dpr directions per pass (every direction of the
// step in one pass when shared memory allows)
template <typename R>
__global__ void __launch_bounds__(160, 3) rope_lin_tangent_kernel(Scene<R> S, int B, int H, int NP,
                                                                 const R* fac, size_t fac_stride, int dpr,
                                                                 R* A, R* Bm) {
  const int nv = S.nv, nq = S.nq, N = S.npair, ndir = nq + 6;
  const size_t fb = (size_t)(LDT + 2 * CR_LDM) * NP;
  const size_t fs = (2 * fb + 9 * (size_t)nv + 32 + 1 + 3) / 4 * 4;
  R* sm = reinterpret_cast<R*>(rc_smem);
  R* F1 = sm;                                        // the factor of H1, then the dR/dx* blocks
  R* Kc = sm;                                        // [nv][9]
  R* Ks = Kc + 9 * (size_t)nv;                       // [nv][2][6]
  R* F2 = sm + 72 * (size_t)N;                       // the factor of H2
  R* gm = F2 + 72 * (size_t)N;                       // step scalars (misc slots 0..31)
  R* ga = gm + 32;                                   // grasped nodes: dx [2][3], Delta [2][3]
  R* tv = sm + (lin_fixed_elems(N, nv) + 3) / 4 * 4;
  const int tid = threadIdx.x;
  const R* d = gm + M_D;
  const R* c = gm + M_C;
  const R* u = gm + M_U;
  const R* gd = gm + M_GD;
  const R nanv = sizeof(R) == 4 ? R(nanf("")) : R(nan(""));
  for (long long job = blockIdx.x; job < (long long)B * H; job += gridDim.x) {
    const int b = (int)(job / H), t = (int)(job % H);
    const R* rec = fac + (size_t)b * fac_stride + (size_t)t * fs;
    const R* rn = rec + 2 * fb;
    R* outA = A + (size_t)job * nq * nq;
    R* outB = Bm + (size_t)job * nq * 6;
    if (rn[9 * nv + 32] != R(0)) {
      // the smooth step failed (its status is set): the step's Jacobians are undefined
      for (int i = tid; i < nq * nq; i += blockDim.x) outA[i] = nanv;
      for (int i = tid; i < nq * 6; i += blockDim.x) outB[i] = nanv;
      continue;
    }
    if (tid < 32) gm[tid] = rn[9 * nv + tid];
    if (tid < 12) {
      const int gi = tid / 6, e = tid % 6, a = S.grasp[gi];
      ga[tid] = e < 3 ? rn[3 * nv + 3 * a + e] : rn[6 * nv + 3 * a + e - 3];
    }
    unpack_factor(rec, NP, N, F2);
    const int rounds = (ndir + dpr - 1) / dpr;
    for (int rd = 0; rd < rounds; ++rd) {
      unpack_factor(rec + fb, NP, N, F1);
      __syncthreads();
      const int dir = rd * dpr + tid;
      const bool act = tid < dpr && dir < ndir;
      // kind 0: node position, 3: node velocity (inertial variant), 1: gripper, 2: control
      int kind = 0, jn = 0, cc = 0, gi = 0;
      if (dir < 3 * nv) { kind = 0; jn = dir / 3; cc = dir % 3; }
      else if (dir < nq - 6) { kind = 3; jn = (dir - 3 * nv) / 3; cc = (dir - 3 * nv) % 3; }
      else if (dir < nq) { kind = 1; gi = (dir - (nq - 6)) / 3; cc = (dir - (nq - 6)) % 3; }
      else { kind = 2; gi = (dir - nq) / 3; cc = (dir - nq) % 3; if (gi > 1) gi = 1; }
      R* col = tv + (tid < dpr ? tid : 0);
      auto E = [&](int j, int i) -> R& { return col[(size_t)(3 * j + i) * dpr]; };
      // controls are the columns of B, every other direction a column of A
      R* out = kind == 2 ? outB : outA;
      const int ld = kind == 2 ? 6 : nq;
      const int oc = kind == 2 ? dir - nq : dir;
      if (act) {
        for (int e = 0; e < 6 * N; ++e) col[(size_t)e * dpr] = R(0);
        // rhs1 = -(dF/dtheta)
        if (kind == 0) {
          E(jn, cc) += S.w;
          for (int g2 = 0; g2 < 2; ++g2)
            if (S.grasp[g2] == jn) {
              const R dd = -gd[3 * g2 + cc];
              for (int i = 0; i < 3; ++i) E(jn, i) -= (ga[6 * g2 + i] - (c[3 * g2 + i] + u[3 * g2 + i])) * dd;
            }
          if (RC_SO_ON(S)) damp_tangent(S, rn, jn, cc, 3 * nv, E, true);   // (D/dt) e - d/dx[(D/dt)(x* - x)] e
        } else if (kind == 3) {
          E(jn, cc) += S.w * S.dt;                                  // -dF/dv = M/dt
        } else {
          const int a = S.grasp[gi];
          E(a, cc) += d[gi];
          if (kind == 1)
            for (int i = 0; i < 3; ++i) E(a, i) -= (ga[6 * gi + i] - (c[3 * gi + i] + u[3 * gi + i])) * gd[3 * gi + cc];
        }
        block_solve_col(F1, col, dpr, N);             // dx*
        for (int j = 0; j < nv; ++j)
          for (int i = 0; i < 3; ++i) out[(size_t)(3 * j + i) * ld + oc] = E(j, i);
        for (int r = 0; r < 6; ++r)
          out[(size_t)(nq - 6 + r) * ld + oc] = ((kind == 1 || kind == 2) && r == 3 * gi + cc) ? R(1) : R(0);
      }
      __syncthreads();                                // F1 read by every direction
      dR_blocks(S, rn, Kc, Ks);
      __syncthreads();
      if (act) {
        // rhs2 = -(dR/dx* dx* + dR/dtheta), in place: node j needs dx* of j-2 .. j+2, the two
        // below it kept in registers once overwritten
        R p2[3] = {0, 0, 0}, p1[3] = {0, 0, 0}, c0[3], c1[3], c2[3];
        for (int i = 0; i < 3; ++i) {
          c0[i] = E(0, i);
          c1[i] = nv > 1 ? E(1, i) : R(0);
          c2[i] = nv > 2 ? E(2, i) : R(0);
        }
        for (int j = 0; j < nv; ++j) {
          const R* K = Kc + 9 * j;
          R rr[3];
          for (int i = 0; i < 3; ++i) rr[i] = K[i * 3] * c0[0] + K[i * 3 + 1] * c0[1] + K[i * 3 + 2] * c0[2];
#pragma unroll
          for (int o = 1; o <= 2; ++o) {
            // spring (j, j+o): +Ks (v_{j+o} - v_j) on node j
            if (j + o < nv) {
              const R* Sy = Ks + (2 * j + o - 1) * 6;
              const R mt[3] = {(o == 1 ? c1[0] : c2[0]) - c0[0], (o == 1 ? c1[1] : c2[1]) - c0[1],
                               (o == 1 ? c1[2] : c2[2]) - c0[2]};
              rr[0] += Sy[0] * mt[0] + Sy[1] * mt[1] + Sy[2] * mt[2];
              rr[1] += Sy[1] * mt[0] + Sy[3] * mt[1] + Sy[4] * mt[2];
              rr[2] += Sy[2] * mt[0] + Sy[4] * mt[1] + Sy[5] * mt[2];
            }
            // spring (j-o, j): -Ks (v_j - v_{j-o}) on node j
            if (j - o >= 0) {
              const R* Sy = Ks + (2 * (j - o) + o - 1) * 6;
              const R mt[3] = {c0[0] - (o == 1 ? p1[0] : p2[0]), c0[1] - (o == 1 ? p1[1] : p2[1]),
                               c0[2] - (o == 1 ? p1[2] : p2[2])};
              rr[0] -= Sy[0] * mt[0] + Sy[1] * mt[1] + Sy[2] * mt[2];
              rr[1] -= Sy[1] * mt[0] + Sy[3] * mt[1] + Sy[4] * mt[2];
              rr[2] -= Sy[2] * mt[0] + Sy[4] * mt[1] + Sy[5] * mt[2];
            }
          }
          for (int g2 = 0; g2 < 2; ++g2)
            if (S.grasp[g2] == j) {
              R dd = R(0);
              if (kind == 1 && gi == g2) dd = gd[3 * g2 + cc];
              if (kind == 0 && jn == j) dd = -gd[3 * g2 + cc];
              for (int i = 0; i < 3; ++i) rr[i] -= ga[6 * g2 + 3 + i] * dd;
            }
          for (int i = 0; i < 3; ++i) {
            E(j, i) = rr[i];
            p2[i] = p1[i];
            p1[i] = c0[i];
            c0[i] = c1[i];
            c1[i] = c2[i];
            c2[i] = j + 3 < nv ? E(j + 3, i) : R(0);
          }
        }
        // inertial variant: P's damping depends on the step start, -d/dx[(D/dt) Delta] e
        if (RC_SO_ON(S) && kind == 0) damp_tangent(S, rn, jn, cc, 6 * nv, E, false);
        block_solve_col(F2, col, dpr, N);             // dDelta
        // dq+/dtheta = dx* (written above) + dDelta, read back a pair of nodes at a time; the
        // inertial variant's velocity rows (dx+/dtheta - dx/dtheta)/dt
        for (int j0 = 0; j0 < nv; j0 += 2) {
          const int nn = j0 + 1 < nv ? 6 : 3;
          R o6[6];
#pragma unroll
          for (int e = 0; e < 6; ++e)
            if (e < nn) o6[e] = out[(size_t)(3 * j0 + e) * ld + oc];
#pragma unroll
          for (int e = 0; e < 6; ++e)
            if (e < nn) {
              const R xp = o6[e] + col[(size_t)(3 * j0 + e) * dpr];
              out[(size_t)(3 * j0 + e) * ld + oc] = xp;
              if (RC_SO_ON(S)) {
                const R ex = (kind == 0 && 3 * j0 + e == 3 * jn + cc) ? R(1) : R(0);
                out[(size_t)(3 * nv + 3 * j0 + e) * ld + oc] = (xp - ex) / S.dt;
              }
            }
        }
      }
      __syncthreads();                                // F1 / Kc, Ks free for the next pass
    }
  }
}

}  // namespace RC_NS
}  // namespace cs
