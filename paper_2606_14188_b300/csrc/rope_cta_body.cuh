// The body of rope_cta.cuh, included once per step variant: namespace RC_NS, and RC_SO_ON(S)
// true only in the inertial variant's copy (false at compile time in the quasi-static copy,
// which then holds none of the inertial code).  No include guard: rope_cta.cuh includes it twice.
namespace cs {
namespace RC_NS {

constexpr int NT = 64;   // threads per rollout
constexpr int LDT = 21;  // row stride of a packed lower triangle (odd: a thread per row touches 32 banks)

__device__ __forceinline__ int rt(int p, int i, int j) { return p * LDT + i * (i + 1) / 2 + j; }

template <typename R>
__device__ __forceinline__ void ld_low(const R* T, int row, R* a) {
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int k = 0; k <= i; ++k) a[i * 6 + k] = T[rt(row, i, k)];
}

__host__ __device__ constexpr int pow2ceil(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

// ------------------------------------------------------------------------------------------
// shared memory of one CTA (elements of the real type)
// ------------------------------------------------------------------------------------------
template <typename R>
struct Sm {
  int NVP;                      // node slots: 64 NPT
  R *T, *B, *V, *r;             // block cyclic reduction: rows of stride LDT, CR_LDM, CR_LDM, CR_LDV
  R *x0, *dx, *v1;              // node exchange: element c of node j at [c * NVP + j]
  R *s, *z, *g;                 // contact pairs (obstacle o, node j): element c at [(o * 3 + c) * NVP + j]
  R *wp;                        // Nesterov-Todd scaling of a pair: (v1, v2, beta) at [(o * 3 + c) * NVP + j]
  R *misc;                      // [64]: grippers, controls, grasp offsets and stiffness (M_* slots)
  R *red;                       // [4]: block reductions (two buffers of one value per warp)
};

// The signed distances and normals of the contact pairs are recomputed from x* where needed (they
// are fixed during a stage-2 solve), a pair's scaling W = beta (2 v v^T - J) is kept as (v1, v2,
// beta) (v0 = sqrt(1 + v1^2 + v2^2) on the unit hyperboloid), and the controls are read from global
// memory: a 64-node rope with 5 obstacles takes 31 KB, 7 CTAs per SM.
__host__ __device__ inline size_t sm_elems(int NPT, int nobs) {
  const size_t NVP = 64 * (size_t)NPT, N = 32 * (size_t)NPT;
  return N * (LDT + 2 * CR_LDM + CR_LDV) + 3 * 3 * NVP + (size_t)nobs * 12 * NVP + 64 + 4;
}

template <typename R>
__device__ __forceinline__ Sm<R> sm_carve(R* base, int NPT, int nobs) {
  Sm<R> w;
  const size_t NVP = 64 * (size_t)NPT, N = 32 * (size_t)NPT;
  w.NVP = (int)NVP;
  R* p = base;
  auto take = [&](size_t n) { R* q = p; p += n; return q; };
  w.T = take(LDT * N); w.B = take(CR_LDM * N); w.V = take(CR_LDM * N); w.r = take(CR_LDV * N);
  w.x0 = take(3 * NVP); w.dx = take(3 * NVP); w.v1 = take(3 * NVP);
  w.s = take((size_t)nobs * 3 * NVP); w.z = take((size_t)nobs * 3 * NVP);
  w.g = take((size_t)nobs * 3 * NVP); w.wp = take((size_t)nobs * 3 * NVP);
  w.misc = take(64);
  w.red = take(4);
  return w;
}

__device__ __forceinline__ int pv_(int o, int c, int j, int NVP) { return (o * 3 + c) * NVP + j; }

// ------------------------------------------------------------------------------------------
// block reductions (every thread calls them; the result is the same on every thread)
// ------------------------------------------------------------------------------------------
struct Red {
  int buf = 0;
};

template <typename R>
__device__ __forceinline__ R bsum(R v, R* red, Red& rb) {
  v = wsum(v);
  if ((threadIdx.x & 31) == 0) red[rb.buf * 2 + (threadIdx.x >> 5)] = v;
  __syncthreads();
  const R t = red[rb.buf * 2] + red[rb.buf * 2 + 1];
  rb.buf ^= 1;
  return t;
}

template <typename R>
__device__ __forceinline__ R bmax(R v, R* red, Red& rb) {
  v = wmax(v);
  if ((threadIdx.x & 31) == 0) red[rb.buf * 2 + (threadIdx.x >> 5)] = v;
  __syncthreads();
  const R a = red[rb.buf * 2], b = red[rb.buf * 2 + 1];
  rb.buf ^= 1;
  return a > b ? a : b;
}

template <typename R>
__device__ __forceinline__ R bmin(R v, R* red, Red& rb) { return -bmax(-v, red, rb); }

// ------------------------------------------------------------------------------------------
// block cyclic reduction of a symmetric positive definite block-tridiagonal matrix (6x6 blocks of
// node pairs), the storage of cr.cuh: T lower triangle (replaced by its Cholesky factor with
// reciprocal diagonal), B coupling with the row s below at level s, V work block, r right-hand side.
// Level s eliminates the rows k = s (mod 2s); a group of G threads works on each row (G = 64 over
// the number of rows of the level, at most a warp), then the survivors absorb their eliminated
// neighbours' Schur complements, each entry of a survivor's blocks computed by one thread of its
// group.  A Cholesky factorisation in the odd-even order: it fails exactly when the matrix is not
// positive definite.
// ------------------------------------------------------------------------------------------
template <typename R>
__device__ __noinline__ bool crb_factor(R* T, R* B, R* V, int N) {
  const int tid = threadIdx.x;
  bool ok = true;
  for (int s = 1; s < N; s <<= 1) {
    const int cnt = (N - s + 2 * s - 1) / (2 * s);
    int G = NT / pow2ceil(cnt);
    G = G > 32 ? 32 : G;
    {
      const int idx = tid / G, g = tid & (G - 1);
      const bool act = idx < cnt;
      const unsigned m = __ballot_sync(FULL, act);
      if (act) {
        const int k = s + 2 * s * idx;
        R L[36];
        ld_low(T, k, L);
        __syncwarp(m);                        // the group has read T_k before it is overwritten
        ok = chol6(L) && ok;
        int e = 0;
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int b = 0; b <= a; ++b, ++e)
            if ((e & (G - 1)) == g) T[rt(k, a, b)] = L[a * 6 + b];
        // column c of U_k = L_k^-1 B_k (c < 6) or of V_k = L_k^-1 B_{k+s}^T (c >= 6): the same
        // instructions on every lane, the operands chosen by address
        const int ncol = k + s < N ? 12 : 6;
        for (int c = g; c < ncol; c += G) {
          const bool uc = c < 6;
          const R* src = uc ? B + cr_m(k, c) : B + cr_m(k + s, (c - 6) * 6);
          R* dst = uc ? B + cr_m(k, c) : V + cr_m(k, c - 6);
          const int sst = uc ? 6 : 1;
          R y[6];
#pragma unroll
          for (int i = 0; i < 6; ++i) y[i] = src[i * sst];
          lsolve6(L, y, 1);
#pragma unroll
          for (int i = 0; i < 6; ++i) dst[i * 6] = y[i];
        }
      }
    }
    __syncthreads();
    const int cnt2 = (N + 2 * s - 1) / (2 * s);
    int G2 = NT / pow2ceil(cnt2);
    G2 = G2 > 32 ? 32 : G2;
    {
      const int idx = tid / G2, g = tid & (G2 - 1);
      if (idx < cnt2) {
        const int i = 2 * s * idx;
        const bool hr = i + s < N, hl = i - s >= 0;
        // T_i -= U_{i+s}^T U_{i+s} + V_{i-s}^T V_{i-s} (21 entries) and B_i = -V_{i-s}^T U_{i-s}
        // (36): entry e by the thread with e = g (mod G2), its row and column computed, so that the
        // lanes of a warp run the same instructions on different entries
        const R* Ur = B + cr_m(hr ? i + s : i, 0);
        const R* Vl = V + cr_m(hl ? i - s : i, 0);
        const R* Ul = B + cr_m(hl ? i - s : i, 0);
        for (int e = g; e < 21; e += G2) {
          const int a = (e >= 1) + (e >= 3) + (e >= 6) + (e >= 10) + (e >= 15);
          const int b = e - a * (a + 1) / 2;
          R t = T[rt(i, a, b)];
          if (hr) {
#pragma unroll
            for (int q = 0; q < 6; ++q) t -= Ur[q * 6 + a] * Ur[q * 6 + b];
          }
          if (hl) {
#pragma unroll
            for (int q = 0; q < 6; ++q) t -= Vl[q * 6 + a] * Vl[q * 6 + b];
          }
          T[rt(i, a, b)] = t;
        }
        if (hl) {
          for (int e = g; e < 36; e += G2) {
            const int a = e / 6, b = e - 6 * (e / 6);
            R t = R(0);
#pragma unroll
            for (int q = 0; q < 6; ++q) t += Vl[q * 6 + a] * Ul[q * 6 + b];
            B[cr_m(i, e)] = -t;
          }
        }
      }
    }
    __syncthreads();
  }
  if (tid == 0) {
    R L[36];
    ld_low(T, 0, L);
    ok = chol6(L) && ok;
#pragma unroll
    for (int i = 0; i < 6; ++i)
#pragma unroll
      for (int q = 0; q <= i; ++q) T[rt(0, i, q)] = L[i * 6 + q];
  }
  return __syncthreads_and(ok);
}

// Solve with the factorisation of crb_factor; thread t handles block row t (N <= 64): one barrier
// per level (the rows eliminated at level 2s are the survivors of level s, each updated by its own
// thread).
template <typename R>
__device__ __noinline__ void crb_solve(const R* T, const R* B, const R* V, R* r, int N) {
  const int t = threadIdx.x;
  const bool row = t < N;
  int top = 1;
  while (top < N) top <<= 1;
  for (int s = 1; s < N; s <<= 1) {
    if (row && (t & (2 * s - 1)) == s) {
      R L[36], y[6];
      ld_low(T, t, L);
#pragma unroll
      for (int a = 0; a < 6; ++a) y[a] = r[cr_v(t, a)];
      lsolve6(L, y, 1);
#pragma unroll
      for (int a = 0; a < 6; ++a) r[cr_v(t, a)] = y[a];
    }
    __syncthreads();
    if (row && (t & (2 * s - 1)) == 0) {
      R acc[6] = {0, 0, 0, 0, 0, 0};
      if (t + s < N) {
        R w[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) w[q] = r[cr_v(t + s, q)];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int q = 0; q < 6; ++q) acc[a] += B[cr_m(t + s, q * 6 + a)] * w[q];
      }
      if (t - s >= 0) {
        R w[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) w[q] = r[cr_v(t - s, q)];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int q = 0; q < 6; ++q) acc[a] += V[cr_m(t - s, q * 6 + a)] * w[q];
      }
#pragma unroll
      for (int a = 0; a < 6; ++a) r[cr_v(t, a)] -= acc[a];
    }
  }
  if (t == 0) {
    R L[36], y[6];
    ld_low(T, 0, L);
#pragma unroll
    for (int a = 0; a < 6; ++a) y[a] = r[cr_v(0, a)];
    lsolve6(L, y, 1);
    ltsolve6(L, y, 1);
#pragma unroll
    for (int a = 0; a < 6; ++a) r[cr_v(0, a)] = y[a];
  }
  __syncthreads();
  for (int s = top >> 1; s >= 1; s >>= 1) {
    if (row && (t & (2 * s - 1)) == s) {
      R y[6], xl[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) { y[a] = r[cr_v(t, a)]; xl[a] = r[cr_v(t - s, a)]; }
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int q = 0; q < 6; ++q) y[a] -= B[cr_m(t, a * 6 + q)] * xl[q];
      if (t + s < N) {
        R xr[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) xr[a] = r[cr_v(t + s, a)];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int q = 0; q < 6; ++q) y[a] -= V[cr_m(t, a * 6 + q)] * xr[q];
      }
      R L[36];
      ld_low(T, t, L);
      ltsolve6(L, y, 1);
#pragma unroll
      for (int a = 0; a < 6; ++a) r[cr_v(t, a)] = y[a];
    }
    __syncthreads();
  }
}


// ------------------------------------------------------------------------------------------
// per-thread state of its nodes j = threadIdx.x + 64 k
// ------------------------------------------------------------------------------------------
template <typename R, int NPT>
struct Nd {
  R x0[NPT][3];               // node at the step start
  R dx[NPT][3];               // x* - x0
  R Dl[NPT][3];               // Delta (stage 2)
  R pv[NPT][3];               // step / work vector
  R F[NPT][3];                // residual
  R Ls[NPT][4];               // rest lengths of the springs to j-2, j-1, j+1, j+2 (1 where absent)
  R v[NPT][3];                // velocity at the step start (inertial variant)
};

__device__ __forceinline__ int node_of(int k) { return threadIdx.x + NT * k; }

// the springs of node j: to j + off(si), si = 0..3 (bend, stretch, stretch, bend)
__host__ __device__ constexpr int spr_off(int si) { return si == 0 ? -2 : (si == 1 ? -1 : (si == 2 ? 1 : 2)); }

template <typename R, int NPT>
__device__ __forceinline__ void zero3(R v[NPT][3]) {
#pragma unroll
  for (int k = 0; k < NPT; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) v[k][c] = R(0);
}

template <typename R, int NPT>
__device__ __forceinline__ void zero_nd(Nd<R, NPT>& N) {
  zero3<R, NPT>(N.x0); zero3<R, NPT>(N.dx); zero3<R, NPT>(N.Dl); zero3<R, NPT>(N.pv); zero3<R, NPT>(N.F);
  zero3<R, NPT>(N.v);
}

template <typename R, int NPT>
__device__ __forceinline__ void load_rest(const Scene<R>& S, Nd<R, NPT>& N) {
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
#pragma unroll
    for (int si = 0; si < 4; ++si) {
      const int o = spr_off(si), jo = j + o;
      const int a = o < 0 ? jo : j;
      const bool ok = j < S.nv && jo >= 0 && jo < S.nv;
      N.Ls[k][si] = ok ? (si == 1 || si == 2 ? S.L1[a] : S.L2[a]) : R(1);
    }
  }
}

// write a node vector to the exchange array dst (element c of node j at [c * NVP + j])
template <typename R, int NPT>
__device__ __forceinline__ void publish(R* dst, const R v[NPT][3], int NVP) {
#pragma unroll
  for (int k = 0; k < NPT; ++k)
#pragma unroll
    for (int c = 0; c < 3; ++c) dst[c * NVP + node_of(k)] = v[k][c];
}

// the spring vector e = x_jo - x_j at x0 + dx (offsets subtracted first: no absolute-coordinate
// cancellation in single precision)
template <typename R, int NPT>
__device__ __forceinline__ void spring_vec(const Nd<R, NPT>& N, const Sm<R>& w, int k, int jo, R e[3]) {
#pragma unroll
  for (int c = 0; c < 3; ++c)
    e[c] = (w.x0[c * w.NVP + jo] - N.x0[k][c]) + (w.dx[c * w.NVP + jo] - N.dx[k][c]);
}

// Inertial variant: the Rayleigh damping term of the spring (j, jo) is c u u^T with u the unit
// spring vector at the step start x0 and c = (damp_beta / dt) k; returns c and sets u.
template <typename R, int NPT>
__device__ __forceinline__ R damp_axis(const Scene<R>& S, const Nd<R, NPT>& N, const Sm<R>& w, int k, int si, R u[3]) {
  const int jo = node_of(k) + spr_off(si);
#pragma unroll
  for (int c = 0; c < 3; ++c) u[c] = w.x0[c * w.NVP + jo] - N.x0[k][c];
  const R il = R(1) / sqrt(dot3(u, u));
#pragma unroll
  for (int c = 0; c < 3; ++c) u[c] *= il;
  return S.cb * ((si == 1 || si == 2) ? S.k1 : S.k2);
}

// Inertial variant, adjoint: for the damping term of the spring (j, jo) with unit vector u (at the
// step start, from j to jo), length l and c = damp_axis's coefficient, the force on jo,
// f = c u (u.y) with y = y_jo - y_j, has df/d(x_jo - x_j) = J = (c/l) [(u.y)(I - u u^T) + u (y - u (u.y))^T];
// returns J^T z = (c/l) [(u.y) z + (u.z) y - 2 (u.y)(u.z) u] (symmetric in y, z).
template <typename R>
__device__ __forceinline__ void damp_jt(R c, R il, const R u[3], const R y[3], const R z[3], R out[3]) {
  const R uy = dot3(u, y), uz = dot3(u, z);
#pragma unroll
  for (int i = 0; i < 3; ++i) out[i] = c * il * (uy * z[i] + uz * y[i] - R(2) * uy * uz * u[i]);
}

// Stage-1 rows of node j (slot k) at x0 + dx: the diagonal 3x3 block D of P = dF/dq*, its couplings
// C1 (with j-1) and C2 (with j-2), and the residual F (eq. dynamics-first-stage).  A spring's force
// on j is -k (l - L) e/l and its Hessian block H(e) = k [u u^T + c (I - u u^T)] enters D with + and
// the coupling with -.
template <typename R, int NPT>
__device__ __forceinline__ void node_rows(const Scene<R>& S, const Nd<R, NPT>& N, const Sm<R>& w, int k,
                                          bool proj, R D[9], R C1[9], R C2[9], R F[3]) {
  const int j = node_of(k);
  const R* d = w.misc + M_D;
  const R* c = w.misc + M_C;
  const R* u = w.misc + M_U;
#pragma unroll
  for (int i = 0; i < 9; ++i) { D[i] = R(0); C1[i] = R(0); C2[i] = R(0); }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    D[i * 4] = S.w;
    F[i] = S.w * N.dx[k][i] - S.m * S.grav[i];
  }
#pragma unroll
  for (int gi = 0; gi < 2; ++gi)
    if (S.grasp[gi] == j) {
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        D[i * 4] += d[gi];
        F[i] += d[gi] * (N.dx[k][i] - (c[3 * gi + i] + u[3 * gi + i]));
      }
    }
#pragma unroll
  for (int si = 0; si < 4; ++si) {
    const int jo = j + spr_off(si);
    if (jo < 0 || jo >= S.nv) continue;
    R e[3], f[3], H[9];
    spring_vec(N, w, k, jo, e);
    spring_eval(e, (si == 1 || si == 2) ? S.k1 : S.k2, N.Ls[k][si], proj, f, H);
    if (RC_SO_ON(S)) {
      // damping: F += c u u^T (dx_j - dx_jo), the block c u u^T with + and the coupling with -
      R ua[3];
      const R cs = damp_axis(S, N, w, k, si, ua);
      R dd = R(0);
#pragma unroll
      for (int i = 0; i < 3; ++i) dd += ua[i] * (N.dx[k][i] - w.dx[i * w.NVP + jo]);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        f[i] -= cs * dd * ua[i];
#pragma unroll
        for (int q = 0; q < 3; ++q) H[i * 3 + q] += cs * ua[i] * ua[q];
      }
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) F[i] -= f[i];
#pragma unroll
    for (int i = 0; i < 9; ++i) D[i] += H[i];
    if (si == 1) {
#pragma unroll
      for (int i = 0; i < 9; ++i) C1[i] = -H[i];
    } else if (si == 0) {
#pragma unroll
      for (int i = 0; i < 9; ++i) C2[i] = -H[i];
    }
  }
  if (RC_SO_ON(S)) {
    // inertia about x0 + dt v and the mass-proportional damping: F += -w dt v + cm dx, D += cm I
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      F[i] += S.cm * N.dx[k][i] - S.w * S.dt * N.v[k][i];
      D[i * 4] += S.cm;
    }
  }
}

// node j's three rows of block row p = j/2 (rows 3h..3h+2, h = j & 1) in the reduction storage:
// T (lower triangle) holds the diagonal block and, for h = 1, the coupling with node 2p; B holds the
// couplings with the nodes of pair p - 1 (node 2p-2 in columns 0..2, 2p-1 in columns 3..5).
template <typename R>
__device__ __forceinline__ void put_node_rows(const Sm<R>& w, int j, const R D[9], const R C1[9], const R C2[9]) {
  const int p = j >> 1, h = j & 1;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int row = 3 * h + i;
    if (h == 0) {
#pragma unroll
      for (int q = 0; q <= i; ++q) w.T[rt(p, row, q)] = D[i * 3 + q];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        w.B[cr_m(p, row * 6 + q)] = C2[i * 3 + q];
        w.B[cr_m(p, row * 6 + 3 + q)] = C1[i * 3 + q];
      }
    } else {
#pragma unroll
      for (int q = 0; q < 3; ++q) w.T[rt(p, row, q)] = C1[i * 3 + q];
#pragma unroll
      for (int q = 0; q <= i; ++q) w.T[rt(p, row, 3 + q)] = D[i * 3 + q];
#pragma unroll
      for (int q = 0; q < 3; ++q) {
        w.B[cr_m(p, row * 6 + q)] = R(0);
        w.B[cr_m(p, row * 6 + 3 + q)] = C2[i * 3 + q];
      }
    }
  }
}

// rows of a node past the chain (the odd node of the last pair of an odd chain): identity
template <typename R>
__device__ __forceinline__ void put_pad_rows(const Sm<R>& w, int j) {
  R D[9] = {1, 0, 0, 0, 1, 0, 0, 0, 1}, Z[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  put_node_rows(w, j, D, Z, Z);
}

// assemble P = dF/dq* at x0 + dx (exact, or with the transverse factors clamped when proj); with
// keepF, the residual goes to N.F.  Needs x0 and dx published.
template <typename R, int NPT>
__device__ __forceinline__ void assemble_P(const Scene<R>& S, Nd<R, NPT>& N, const Sm<R>& w, bool proj, bool keepF) {
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
    if (j < S.nv) {
      R D[9], C1[9], C2[9], F[3];
      node_rows(S, N, w, k, proj, D, C1, C2, F);
      put_node_rows(w, j, D, C1, C2);
      if (keepF)
#pragma unroll
        for (int i = 0; i < 3; ++i) N.F[k][i] = F[i];
    } else {
      if (j < 2 * S.npair) put_pad_rows(w, j);
      if (keepF)
#pragma unroll
        for (int i = 0; i < 3; ++i) N.F[k][i] = R(0);
    }
  }
}

// y = P v for node j (slot k); v of the neighbours from the exchange array vx
template <typename R, int NPT>
__device__ __forceinline__ void hessvec(const Scene<R>& S, const Nd<R, NPT>& N, const Sm<R>& w, int k,
                                        bool proj, const R v[NPT][3], const R* vx, R y[3]) {
  const int j = node_of(k);
  const R* d = w.misc + M_D;
  R dg = S.w;
#pragma unroll
  for (int gi = 0; gi < 2; ++gi)
    if (S.grasp[gi] == j) dg += d[gi];
#pragma unroll
  for (int i = 0; i < 3; ++i) y[i] = dg * v[k][i];
#pragma unroll
  for (int si = 0; si < 4; ++si) {
    const int jo = j + spr_off(si);
    if (jo < 0 || jo >= S.nv) continue;
    R e[3], f[3], H[9], dd[3];
    spring_vec(N, w, k, jo, e);
    spring_eval(e, (si == 1 || si == 2) ? S.k1 : S.k2, N.Ls[k][si], proj, f, H);
#pragma unroll
    for (int i = 0; i < 3; ++i) dd[i] = v[k][i] - vx[i * w.NVP + jo];
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] += H[i * 3] * dd[0] + H[i * 3 + 1] * dd[1] + H[i * 3 + 2] * dd[2];
    if (RC_SO_ON(S)) {
      R ua[3];
      const R cs = damp_axis(S, N, w, k, si, ua) * dot3(ua, dd);
#pragma unroll
      for (int i = 0; i < 3; ++i) y[i] += cs * ua[i];
    }
  }
  if (RC_SO_ON(S))
#pragma unroll
    for (int i = 0; i < 3; ++i) y[i] += S.cm * v[k][i];
}

// this thread's share of Psi(x* + alpha pv) - Psi(x*) (stage-1 potential, gradient F), in difference
// form; springs counted at their first node.  Needs pv published to w.v1.
template <typename R, int NPT>
__device__ __forceinline__ R psi_diff(const Scene<R>& S, const Nd<R, NPT>& N, const Sm<R>& w, R alpha) {
  const R* d = w.misc + M_D;
  const R* c = w.misc + M_C;
  const R* u = w.misc + M_U;
  R val = R(0);
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
    if (j >= S.nv) continue;
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      const R D = alpha * N.pv[k][i];
      val += R(0.5) * S.w * D * (R(2) * N.dx[k][i] + D) - S.m * S.grav[i] * D;
      if (RC_SO_ON(S)) val += D * (S.cm * (N.dx[k][i] + R(0.5) * D) - S.w * S.dt * N.v[k][i]);
    }
#pragma unroll
    for (int gi = 0; gi < 2; ++gi)
      if (S.grasp[gi] == j)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          const R D = alpha * N.pv[k][i];
          val += R(0.5) * d[gi] * D * (D - R(2) * ((c[3 * gi + i] + u[3 * gi + i]) - N.dx[k][i]));
        }
#pragma unroll
    for (int si = 2; si < 4; ++si) {
      const int jo = j + spr_off(si);
      if (jo >= S.nv) continue;
      R dX[3], dD[3], dY[3];
      spring_vec(N, w, k, jo, dX);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        dD[i] = alpha * (w.v1[i * w.NVP + jo] - N.pv[k][i]);
        dY[i] = dX[i] + dD[i];
      }
      const R lX = sqrt(dot3(dX, dX)), lY = sqrt(dot3(dY, dY));
      const R dl = (dD[0] * (R(2) * dX[0] + dD[0]) + dD[1] * (R(2) * dX[1] + dD[1]) +
                    dD[2] * (R(2) * dX[2] + dD[2])) / (lY + lX);
      val += R(0.5) * (si == 2 ? S.k1 : S.k2) * dl * (lY + lX - R(2) * N.Ls[k][si]);
      if (RC_SO_ON(S)) {
        // damping potential (y_jo - y_j)^T c u u^T (y_jo - y_j)/2 of the displacement y = dx
        R ua[3], yd[3];
        const R cs = damp_axis(S, N, w, k, si, ua);
#pragma unroll
        for (int i = 0; i < 3; ++i) yd[i] = w.dx[i * w.NVP + jo] - N.dx[k][i] + R(0.5) * dD[i];
        val += cs * dot3(ua, dD) * dot3(ua, yd);
      }
    }
  }
  return val;
}

// node vectors <-> right-hand side of the reduction (zero rows past the chain)
template <typename R, int NPT>
__device__ __forceinline__ void put_rhs(const Scene<R>& S, const Sm<R>& w, const R v[NPT][3], R sign) {
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
    if (j >= 2 * S.npair) continue;
#pragma unroll
    for (int i = 0; i < 3; ++i) w.r[cr_v(j >> 1, 3 * (j & 1) + i)] = j < S.nv ? sign * v[k][i] : R(0);
  }
}

template <typename R, int NPT>
__device__ __forceinline__ void get_rhs(const Scene<R>& S, const Sm<R>& w, R v[NPT][3]) {
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
#pragma unroll
    for (int i = 0; i < 3; ++i) v[k][i] = j < S.nv ? w.r[cr_v(j >> 1, 3 * (j & 1) + i)] : R(0);
  }
}

// Damped Newton for stage 1.  Without warm, from dx = 0 with each grasped node moved with its
// gripper (the start that keeps the grasp offsets of q).  On exit the factorisation of the Hessian
// at the last iterate is in (T, B, V).  Entry: x0 published and synchronised.
template <typename R, int NPT>
__device__ __forceinline__ int stage1_newton(const Scene<R>& S, Nd<R, NPT>& N, const Sm<R>& w, Red& rb,
                                             int* iters, bool warm) {
  if (!warm) {
    // the inertial variant starts at the predictor x0 + dt v
#pragma unroll
    for (int k = 0; k < NPT; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) N.dx[k][i] = RC_SO_ON(S) ? S.dt * N.v[k][i] : R(0);
#pragma unroll
    for (int k = 0; k < NPT; ++k)
#pragma unroll
      for (int gi = 0; gi < 2; ++gi)
        if (S.grasp[gi] == node_of(k))
#pragma unroll
          for (int i = 0; i < 3; ++i) N.dx[k][i] = w.misc[M_U + 3 * gi + i];
  }
  for (int it = 0; it < S.newton_max; ++it) {
    publish<R, NPT>(w.dx, N.dx, w.NVP);
    __syncthreads();
    bool ok = false, exact = false;
    // exact Hessian; if it is not positive definite, the projected one (same call site)
    for (int attempt = 0; attempt < 2 && !ok; ++attempt) {
      assemble_P(S, N, w, attempt == 1, attempt == 0);
      if (attempt == 0) put_rhs<R, NPT>(S, w, N.F, R(-1));
      __syncthreads();
      ok = crb_factor(w.T, w.B, w.V, S.npair);
      exact = ok && attempt == 0;
    }
    if (!ok) { *iters = it + 1; return ST_NOTPD; }
    crb_solve(w.T, w.B, w.V, w.r, S.npair);
    get_rhs<R, NPT>(S, w, N.pv);
    R pm = R(0), sl = R(0);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < NPT; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        const R pv = N.pv[k][i];
        bad = bad || !(fabs(pv) <= R(1e30));
        pm = fmax(pm, fabs(pv));
        sl += N.F[k][i] * pv;
      }
    if (__syncthreads_or(bad)) { *iters = it + 1; return ST_NONFINITE; }
    pm = bmax(pm, w.red, rb);
    sl = bsum(sl, w.red, rb);
    // converged only on an exact-Hessian step: the root is a local minimiser of the potential
    if (pm <= S.ntol && exact) {
#pragma unroll
      for (int k = 0; k < NPT; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) N.dx[k][i] += N.pv[k][i];
      *iters = it + 1;
      return 0;
    }
    publish<R, NPT>(w.v1, N.pv, w.NVP);
    __syncthreads();
    R alpha = R(1);
    for (int ls = 0; ls < 40; ++ls) {
      const R dv = bsum(psi_diff(S, N, w, alpha), w.red, rb);
      if (dv <= R(1e-4) * alpha * sl) break;
      alpha *= R(0.5);
    }
#pragma unroll
    for (int k = 0; k < NPT; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) N.dx[k][i] += alpha * N.pv[k][i];
  }
  *iters = S.newton_max;
  return ST_NEWTON;
}


// ------------------------------------------------------------------------------------------
// stage 2
// ------------------------------------------------------------------------------------------

// phi and n of pair (node of slot k, obstacle o) at x* = x0 + dx
template <typename R, int NPT>
__device__ __forceinline__ void pair_geom(const Scene<R>& S, const Nd<R, NPT>& N, int k, int o, R& ph, R n[3]) {
  const R X[3] = {N.x0[k][0] + N.dx[k][0], N.x0[k][1] + N.dx[k][1], N.x0[k][2] + N.dx[k][2]};
  obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, (R*)nullptr);
}

// the rollout's smallest signed distance at x* = x0 + dx
template <typename R, int NPT>
__device__ __forceinline__ R min_phi(const Scene<R>& S, const Nd<R, NPT>& N, const Sm<R>& w, Red& rb) {
  R pmin = R(1e30);
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    if (node_of(k) >= S.nv) continue;
    for (int o = 0; o < S.nobs; ++o) {
      R ph, n[3];
      pair_geom(S, N, k, o, ph, n);
      pmin = fmin(pmin, ph);
    }
  }
  return bmin(pmin, w.red, rb);
}

template <typename R>
__device__ __forceinline__ void pair_sz(const Sm<R>& w, int o, int j, R sv[3], R zv[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a) { sv[a] = w.s[pv_(o, a, j, w.NVP)]; zv[a] = w.z[pv_(o, a, j, w.NVP)]; }
}

// M = W^-2 of a pair from its stored scaling (v1, v2, beta): with u = J v = (v0, -v1, -v2),
// W^-1 = (2 u u^T - J) / beta, so M = (4 (u.u) u u^T - 2 (u v^T + v u^T) + I) / beta^2
template <typename R>
__device__ __forceinline__ void pair_M(const Sm<R>& w, int o, int j, R M[9]) {
  const R v1 = w.wp[pv_(o, 0, j, w.NVP)], v2 = w.wp[pv_(o, 1, j, w.NVP)], be = w.wp[pv_(o, 2, j, w.NVP)];
  const R v0 = sqrt(R(1) + v1 * v1 + v2 * v2);
  const R v[3] = {v0, v1, v2}, u[3] = {v0, -v1, -v2};
  const R uu = v0 * v0 + v1 * v1 + v2 * v2;
  const R ib2 = R(1) / (be * be);
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b)
      M[a * 3 + b] = (R(4) * uu * u[a] * u[b] - R(2) * (u[a] * v[b] + v[a] * u[b]) + (a == b ? R(1) : R(0))) * ib2;
}

// the scaling W, W^-1 and lam = W z of a pair (Vandenberghe 2010, second-order cone), and its
// compact form (v1, v2, beta) for pair_M
template <typename R>
__device__ __forceinline__ void nt_scaling_v(const R s[3], const R z[3], R W[9], R Wi[9], R lam[3], R wp[3]) {
  const R ds = soc_det(s), dz = soc_det(z);
  const R rs = R(1) / sqrt(ds), rz = R(1) / sqrt(dz);
  const R sb[3] = {s[0] * rs, s[1] * rs, s[2] * rs};
  const R zb[3] = {z[0] * rz, z[1] * rz, z[2] * rz};
  const R gam = sqrt(R(0.5) * (R(1) + sb[0] * zb[0] + sb[1] * zb[1] + sb[2] * zb[2]));
  const R ig = R(1) / (R(2) * gam);
  const R wb[3] = {(sb[0] + zb[0]) * ig, (sb[1] - zb[1]) * ig, (sb[2] - zb[2]) * ig};
  const R iv = R(1) / sqrt(R(2) * (wb[0] + R(1)));
  const R v[3] = {(wb[0] + R(1)) * iv, wb[1] * iv, wb[2] * iv};
  const R beta = sqrt(sqrt(ds / dz));
  const R Jv[3] = {v[0], -v[1], -v[2]};
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const R J = i == k ? (i == 0 ? R(1) : R(-1)) : R(0);
      W[i * 3 + k] = beta * (R(2) * v[i] * v[k] - J);
      Wi[i * 3 + k] = (R(2) * Jv[i] * Jv[k] - J) / beta;
    }
#pragma unroll
  for (int i = 0; i < 3; ++i) lam[i] = W[i * 3] * z[0] + W[i * 3 + 1] * z[1] + W[i * 3 + 2] * z[2];
  wp[0] = v[1]; wp[1] = v[2]; wp[2] = beta;
}

// residual of the slack r_z = s - A D - phi e1
template <typename R>
__device__ __forceinline__ void pair_rz(const R A[9], const R sv[3], const R D[3], R ph, R rz[3]) {
#pragma unroll
  for (int a = 0; a < 3; ++a)
    rz[a] = sv[a] - (A[a * 3] * D[0] + A[a * 3 + 1] * D[1] + A[a * 3 + 2] * D[2]) - (a == 0 ? ph : R(0));
}

// step of one pair from the node's Delta step dD: ds = A dD - r_z, dz = M (g - A dD)
template <typename R>
__device__ __forceinline__ void pair_step(const R A[9], const R M[9], const R rz[3], const R g[3],
                                          const R dD[3], R dsv[3], R dz[3]) {
  R gm[3];
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    const R ADd = A[a * 3] * dD[0] + A[a * 3 + 1] * dD[1] + A[a * 3 + 2] * dD[2];
    dsv[a] = ADd - rz[a];
    gm[a] = g[a] - ADd;
  }
#pragma unroll
  for (int a = 0; a < 3; ++a) dz[a] = M[a * 3] * gm[0] + M[a * 3 + 1] * gm[1] + M[a * 3 + 2] * gm[2];
}

// ds, dz of pair (slot k, obstacle o) for the node step dD, from the stored s, M and g
template <typename R, int NPT>
__device__ __forceinline__ void pair_dir(const Scene<R>& S, const Nd<R, NPT>& N, const Sm<R>& w, int k, int o,
                                         const R dD[3], R sv[3], R zv[3], R dsv[3], R dz[3]) {
  const int j = node_of(k);
  R ph, n[3], A[9], M[9], g[3], rz[3];
  pair_geom(S, N, k, o, ph, n);
  cone_frame(n, S.mu, A);
  pair_sz(w, o, j, sv, zv);
  pair_M(w, o, j, M);
#pragma unroll
  for (int a = 0; a < 3; ++a) g[a] = w.g[pv_(o, a, j, w.NVP)];
  const R D[3] = {N.Dl[k][0], N.Dl[k][1], N.Dl[k][2]};
  pair_rz(A, sv, D, ph, rz);
  pair_step(A, M, rz, g, dD, dsv, dz);
}

// diagonal 3x3 block of P for node j: w I + grasp + incident spring Hessians (exact)
template <typename R, int NPT>
__device__ __forceinline__ void diag_block(const Scene<R>& S, const Nd<R, NPT>& N, const Sm<R>& w, int k, R D[9]) {
  const int j = node_of(k);
#pragma unroll
  for (int i = 0; i < 9; ++i) D[i] = R(0);
#pragma unroll
  for (int i = 0; i < 3; ++i) D[i * 4] = S.w;
#pragma unroll
  for (int gi = 0; gi < 2; ++gi)
    if (S.grasp[gi] == j)
#pragma unroll
      for (int i = 0; i < 3; ++i) D[i * 4] += w.misc[M_D + gi];
#pragma unroll
  for (int si = 0; si < 4; ++si) {
    const int jo = j + spr_off(si);
    if (jo < 0 || jo >= S.nv) continue;
    R e[3], f[3], H[9];
    spring_vec(N, w, k, jo, e);
    spring_eval(e, (si == 1 || si == 2) ? S.k1 : S.k2, N.Ls[k][si], false, f, H);
#pragma unroll
    for (int i = 0; i < 9; ++i) D[i] += H[i];
    if (RC_SO_ON(S)) {
      R ua[3];
      const R cs = damp_axis(S, N, w, k, si, ua);
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int q = 0; q < 3; ++q) D[i * 3 + q] += cs * ua[i] * ua[q];
    }
  }
  if (RC_SO_ON(S))
#pragma unroll
    for (int i = 0; i < 3; ++i) D[i * 4] += S.cm;
}

// Primal-dual interior point with Nesterov-Todd scaling (Vandenberghe, "The CVXOPT linear and
// quadratic cone program solvers", 2010) for
//   min 1/2 D^T P D  s.t.  s_i = A_i D_j + phi_i e1 in Q,  z_i in Q  (forces lam_i = A_i^T z_i),
// centering s_i o z_i = kappa e.  kfinal < 0: fixed target kappa (smooth model).  Else each
// iteration is a Mehrotra predictor-corrector step: the affine direction (target 0) and its step
// length alpha_a give the target max(kfinal, (1 - alpha_a)^3 <s,z>/m), and the combined direction
// adds the second-order term (W^-1 ds_a) o (W dz_a); once the target is kfinal, centring steps at
// kfinal end the solve.  P is the exact dF/dq*: H2 = P + sum A^T W^-2 A not positive definite means
// P is not either and the QP of eq. dynamics-second-stage is not convex (CS_ST_NOTPD).  On exit
// (T, B, V) hold the factorisation of the last H2.  Entry: x0, dx published and synchronised; with
// warm, N.Dl the start.
template <typename R, int NPT>
__device__ __forceinline__ int stage2_ipm(const Scene<R>& S, Nd<R, NPT>& N, const Sm<R>& w, Red& rb, R kappa,
                                          R kfinal, int* iters, bool warm, R frac) {
  const int nobs = S.nobs;
  const int NVP = w.NVP;
  const R mm = R(S.nv * nobs);
  // interior start
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
    if (j >= S.nv) { for (int i = 0; i < 3; ++i) N.Dl[k][i] = R(0); continue; }
    R Dj[3] = {R(0), R(0), R(0)};
    if (warm) {                      // given start; the central point does not depend on it
      for (int i = 0; i < 3; ++i) Dj[i] = N.Dl[k][i];
    } else {
      R D[9];
      diag_block(S, N, w, k, D);
      for (int o = 0; o < nobs; ++o) {
        R ph, n[3];
        pair_geom(S, N, k, o, ph, n);
        if (ph < R(0)) {
          R a = R(0);
          for (int i = 0; i < 3; ++i) a += n[i] * (D[i * 3] * n[0] + D[i * 3 + 1] * n[1] + D[i * 3 + 2] * n[2]);
          const R push = R(0.5) * (-ph + sqrt(ph * ph + R(4) * kappa / a));
          for (int i = 0; i < 3; ++i) Dj[i] += push * n[i];
        }
      }
    }
    for (int i = 0; i < 3; ++i) N.Dl[k][i] = Dj[i];
    for (int o = 0; o < nobs; ++o) {
      R ph, n[3], A[9];
      pair_geom(S, N, k, o, ph, n);
      cone_frame(n, S.mu, A);
      R sv[3];
      for (int a = 0; a < 3; ++a)
        sv[a] = A[a * 3] * Dj[0] + A[a * 3 + 1] * Dj[1] + A[a * 3 + 2] * Dj[2] + (a == 0 ? ph : R(0));
      const bool ok = sv[0] > R(0) && soc_det(sv) > R(0.25) * sv[0] * sv[0];
      if (!ok) { sv[0] = ph > S.sig0 ? ph : S.sig0; sv[1] = sv[2] = R(0); }
      const R dt = soc_det(sv);
      for (int a = 0; a < 3; ++a) w.s[pv_(o, a, j, NVP)] = sv[a];
      w.z[pv_(o, 0, j, NVP)] = kappa * sv[0] / dt;
      w.z[pv_(o, 1, j, NVP)] = -kappa * sv[1] / dt;
      w.z[pv_(o, 2, j, NVP)] = -kappa * sv[2] / dt;
    }
  }
  int stalls = 0;
  bool centring = false;      // the target has reached kfinal: plain centring steps from now on
  R xmax = R(0);
#pragma unroll
  for (int k = 0; k < NPT; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) xmax = fmax(xmax, fabs(N.x0[k][i] + N.dx[k][i]));
  const R ilim = R(128) * (sizeof(R) == 4 ? R(1.1920928955078125e-7) : R(2.220446049250313e-16)) *
                 bmax(xmax, w.red, rb);
  for (int it = 0; it < S.ipm_max; ++it) {
    const bool pc = kfinal >= R(0) && !centring;
    R target = kfinal < R(0) ? kappa : kfinal;
    R rhsA[NPT][3];           // right-hand side of this iteration's first system (the corrector's base)
    publish<R, NPT>(w.v1, N.Dl, NVP);
    __syncthreads();
    // assemble H2 and the right-hand side -P D + sum A^T (z + M g), g = r_z + W d_s (the affine
    // right-hand side, target 0, when pc)
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      const int j = node_of(k);
      for (int i = 0; i < 3; ++i) rhsA[k][i] = R(0);
      if (j >= S.nv) {
        if (j < 2 * S.npair) {
          put_pad_rows(w, j);
          for (int i = 0; i < 3; ++i) w.r[cr_v(j >> 1, 3 * (j & 1) + i)] = R(0);
        }
        continue;
      }
      R D[9], C1[9], C2[9], F[3], PD[3];
      node_rows(S, N, w, k, false, D, C1, C2, F);
      hessvec(S, N, w, k, false, N.Dl, w.v1, PD);
      R rhs[3] = {-PD[0], -PD[1], -PD[2]};
      const R Dn[3] = {N.Dl[k][0], N.Dl[k][1], N.Dl[k][2]};
      for (int o = 0; o < nobs; ++o) {
        R ph, n[3], A[9], sv[3], zv[3], rz[3], W[9], Wi[9], lam[3], M[9];
        pair_geom(S, N, k, o, ph, n);
        cone_frame(n, S.mu, A);
        pair_sz(w, o, j, sv, zv);
        pair_rz(A, sv, Dn, ph, rz);
        R wpv[3];
        nt_scaling_v(sv, zv, W, Wi, lam, wpv);
        const R tg = pc ? R(0) : target;
        const R r3[3] = {tg - (lam[0] * lam[0] + lam[1] * lam[1] + lam[2] * lam[2]), R(-2) * lam[0] * lam[1],
                         R(-2) * lam[0] * lam[2]};
        R ds[3];
        jordan_solve(lam, r3, ds);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
          for (int b = 0; b < 3; ++b)
            M[a * 3 + b] = Wi[a * 3] * Wi[b] + Wi[a * 3 + 1] * Wi[3 + b] + Wi[a * 3 + 2] * Wi[6 + b];
#pragma unroll
        for (int a = 0; a < 3; ++a) w.wp[pv_(o, a, j, NVP)] = wpv[a];
        R g[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) {
          g[a] = rz[a] + W[a * 3] * ds[0] + W[a * 3 + 1] * ds[1] + W[a * 3 + 2] * ds[2];
          w.g[pv_(o, a, j, NVP)] = g[a];
        }
        R zg[3];
#pragma unroll
        for (int a = 0; a < 3; ++a) zg[a] = zv[a] + M[a * 3] * g[0] + M[a * 3 + 1] * g[1] + M[a * 3 + 2] * g[2];
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
          for (int c = 0; c <= i; ++c) D[i * 3 + c] += A[i] * MA[c] + A[3 + i] * MA[3 + c] + A[6 + i] * MA[6 + c];
        }
      }
      put_node_rows(w, j, D, C1, C2);     // takes the lower triangle of D
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        w.r[cr_v(j >> 1, 3 * (j & 1) + i)] = rhs[i];
        rhsA[k][i] = rhs[i];
      }
    }
    __syncthreads();
    if (!crb_factor(w.T, w.B, w.V, S.npair)) { *iters = it + 1; return ST_NOTPD; }
    crb_solve(w.T, w.B, w.V, w.r, S.npair);
    get_rhs<R, NPT>(S, w, N.pv);            // dDelta (affine when pc)
    if (pc) {
      // affine step length and duality measure -> centring target
      R aa = R(1e30), gap = R(0);
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        if (node_of(k) >= S.nv) continue;
        const R dD[3] = {N.pv[k][0], N.pv[k][1], N.pv[k][2]};
        for (int o = 0; o < nobs; ++o) {
          R sv[3], zv[3], dsa[3], dza[3];
          pair_dir(S, N, w, k, o, dD, sv, zv, dsa, dza);
          for (int a = 0; a < 3; ++a) gap += sv[a] * zv[a];
          aa = fmin(aa, fmin(soc_max_step(sv, dsa), soc_max_step(zv, dza)));
        }
      }
      aa = fmin(R(1), bmin(aa, w.red, rb));
      gap = bsum(gap, w.red, rb);
      const R om = R(1) - aa;
      target = fmax(kfinal, om * om * om * gap / mm);
      centring = target == kfinal;
      // combined right-hand side: d_s = lam^-1 o (target e - lam o lam - (W^-1 ds_a) o (W dz_a)),
      // the second-order term dropped once the target is kfinal; same factorisation.  Only g
      // changes from the affine system: rhs = rhs_aff + sum A^T M (g - g_aff).
#pragma unroll
      for (int k = 0; k < NPT; ++k) {
        const int j = node_of(k);
        if (j >= 2 * S.npair) continue;
        R rhs[3] = {rhsA[k][0], rhsA[k][1], rhsA[k][2]};
        if (j < S.nv) {
          const R dD[3] = {N.pv[k][0], N.pv[k][1], N.pv[k][2]};
          const R Dn[3] = {N.Dl[k][0], N.Dl[k][1], N.Dl[k][2]};
          for (int o = 0; o < nobs; ++o) {
            R ph, n[3], A[9], W[9], Wi[9], lam[3], sv[3], zv[3], ga[3], rz[3], M[9];
            pair_geom(S, N, k, o, ph, n);
            cone_frame(n, S.mu, A);
            pair_sz(w, o, j, sv, zv);
            pair_rz(A, sv, Dn, ph, rz);
            nt_scaling(sv, zv, W, Wi, lam);
            pair_M(w, o, j, M);
            for (int a = 0; a < 3; ++a) ga[a] = w.g[pv_(o, a, j, NVP)];
            R c3[3] = {R(0), R(0), R(0)};
            if (!centring) {
              // affine directions ds_a = A dD - r_z, dz_a = M (g_aff - A dD)
              R dsa[3], dza[3];
              pair_step(A, M, rz, ga, dD, dsa, dza);
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
              w.g[pv_(o, a, j, NVP)] = g;
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
        for (int i = 0; i < 3; ++i) w.r[cr_v(j >> 1, 3 * (j & 1) + i)] = rhs[i];
      }
      __syncthreads();
      crb_solve(w.T, w.B, w.V, w.r, S.npair);
      get_rhs<R, NPT>(S, w, N.pv);          // dDelta (combined)
    }
    const bool final_target = kfinal < R(0) || target == kfinal;
    // step length to the cone boundaries
    R amin = R(1e30), dmax = R(0);
    bool bad = false;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      if (node_of(k) >= S.nv) continue;
      const R dD[3] = {N.pv[k][0], N.pv[k][1], N.pv[k][2]};
      for (int i = 0; i < 3; ++i) {
        dmax = fmax(dmax, fabs(dD[i]));
        bad = bad || !(fabs(dD[i]) <= R(1e30));
      }
      for (int o = 0; o < nobs; ++o) {
        const int j = node_of(k);
        R sv[3], zv[3], dsv[3], dz[3];
        pair_dir(S, N, w, k, o, dD, sv, zv, dsv, dz);
        for (int a = 0; a < 3; ++a) {
          dmax = fmax(dmax, fabs(dsv[a]));
          bad = bad || !(fabs(dz[a]) <= R(1e30)) || !(fabs(dsv[a]) <= R(1e30));
        }
        amin = fmin(amin, fmin(soc_max_step(sv, dsv), soc_max_step(zv, dz)));
        // g and the scaling are not needed after this: they keep the directions for the update
        for (int a = 0; a < 3; ++a) { w.g[pv_(o, a, j, NVP)] = dsv[a]; w.wp[pv_(o, a, j, NVP)] = dz[a]; }
      }
    }
    if (__syncthreads_or(bad)) { *iters = it + 1; return ST_NONFINITE; }
    dmax = bmax(dmax, w.red, rb);
    amin = bmin(amin, w.red, rb);
    const R alpha = fmin(R(1), frac * amin);
    stalls = alpha < R(1e-6) ? stalls + 1 : 0;
    if (stalls >= 5) { *iters = it + 1; return ST_CONTACT; }
    // update with the directions kept by the step-length pass
    bool inside = true;
#pragma unroll
    for (int k = 0; k < NPT; ++k) {
      const int j = node_of(k);
      if (j >= S.nv) continue;
      for (int o = 0; o < nobs; ++o) {
        R sv[3], zv[3];
        pair_sz(w, o, j, sv, zv);
        for (int a = 0; a < 3; ++a) {
          sv[a] += alpha * w.g[pv_(o, a, j, NVP)];
          zv[a] += alpha * w.wp[pv_(o, a, j, NVP)];
          w.s[pv_(o, a, j, NVP)] = sv[a];
          w.z[pv_(o, a, j, NVP)] = zv[a];
        }
        inside = inside && soc_inside(sv) && soc_inside(zv);
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) N.Dl[k][i] += alpha * N.pv[k][i];
    }
    if (!__syncthreads_and(inside)) { *iters = it + 1; return ST_CONTACT; }
    // stop at the central point: a full step below the tolerance, or (nonsmooth solve) any step
    // below 128 ulps of the state's scale, the resolution the real type's directions reach at the
    // near-boundary sliding contacts of the nonsmooth end of the path
    if (final_target && ((alpha == R(1) && dmax <= S.itol) || (kfinal >= R(0) && dmax <= ilim))) {
      *iters = it + 1;
      return 0;
    }
  }
  *iters = S.ipm_max;
  return ST_CONTACT;
}

// H2 = P + sum A^T W^-2 A assembled at the final iterate of a smooth stage 2 (the scaling from the
// stored s, z; with no obstacle H2 = P) into (T, B, V), unfactorised: the interior point leaves the
// factorisation of its last Newton matrix, taken one step before the solution, where a pressed
// contact's W^-2 (of order z/s) still differs by that step relative to s.  Entry: x0, dx published.
template <typename R, int NPT>
__device__ __forceinline__ void assemble_h2(const Scene<R>& S, const Nd<R, NPT>& N, const Sm<R>& w) {
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
    if (j >= S.nv) {
      if (j < 2 * S.npair) put_pad_rows(w, j);
      continue;
    }
    R D[9], C1[9], C2[9], F[3];
    node_rows(S, N, w, k, false, D, C1, C2, F);
    for (int o = 0; o < S.nobs; ++o) {
      R ph, n[3], A[9], sv[3], zv[3], W[9], Wi[9], lam[3], wpv[3], M[9];
      pair_geom(S, N, k, o, ph, n);
      cone_frame(n, S.mu, A);
      pair_sz(w, o, j, sv, zv);
      nt_scaling_v(sv, zv, W, Wi, lam, wpv);
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b)
          M[a * 3 + b] = Wi[a * 3] * Wi[b] + Wi[a * 3 + 1] * Wi[3 + b] + Wi[a * 3 + 2] * Wi[6 + b];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int c = 0; c <= i; ++c) {
          R t = R(0);
#pragma unroll
          for (int a = 0; a < 3; ++a)
            t += A[a * 3 + i] * (M[a * 3] * A[c] + M[a * 3 + 1] * A[3 + c] + M[a * 3 + 2] * A[6 + c]);
          D[i * 3 + c] += t;
        }
    }
    put_node_rows(w, j, D, C1, C2);     // takes the lower triangle of D
  }
}

// ------------------------------------------------------------------------------------------
// one step: x0 (registers, published), misc g, u, c; with warm the stage-1 start dx, with warm2 the
// stage-2 start Dl.  Outputs dx, Dl (dx published on exit), misc d, gd.  smooth = the smooth grasp
// and the smooth (kappa_c) contact solve.
// ------------------------------------------------------------------------------------------
template <typename R, int NPT>
__device__ __forceinline__ int sim_step(const Scene<R>& S, Nd<R, NPT>& N, const Sm<R>& w, Red& rb, bool smooth,
                                        int* nit, int* iit, bool warm, bool warm2) {
  R* d = w.misc + M_D;
  R* gd = w.misc + M_GD;
  const R* c = w.misc + M_C;
  if (threadIdx.x < 2) {
    const int gi = threadIdx.x;
    const R cc[3] = {c[3 * gi], c[3 * gi + 1], c[3 * gi + 2]};
    const R rho = sqrt(dot3(cc, cc));
    R dd;
    if (smooth) {
      dd = S.Dmax * exp(-rho / S.kh);
      const R f = rho > R(0) ? -dd / (S.kh * rho) : R(0);
      for (int i = 0; i < 3; ++i) gd[3 * gi + i] = f * cc[i];
    } else {
      dd = rho <= S.rgrasp ? S.Dmax : R(0);
      for (int i = 0; i < 3; ++i) gd[3 * gi + i] = R(0);
    }
    d[gi] = dd;
  }
  __syncthreads();
  if (!warm2) zero3<R, NPT>(N.Dl);
  int st = stage1_newton(S, N, w, rb, nit, warm);
  publish<R, NPT>(w.dx, N.dx, w.NVP);
  __syncthreads();
  *iit = 0;
  if (S.nobs == 0) { zero3<R, NPT>(N.Dl); return st; }
  const R pmin = min_phi(S, N, w, rb);
  if (!smooth && pmin >= R(0)) { zero3<R, NPT>(N.Dl); return st; }   // Delta = 0 is optimal
  // The interior point takes steps of 0.99 of the distance to the cone boundaries; if it fails it
  // is run again on paths that stay further inside the cones (single precision loses the
  // near-boundary iterates of hard sliding contacts): 0.9 from the same start, 0.9 and then 0.75
  // from the per-node closed-form start.  The central point reached does not depend on the path.
  R D0[NPT][3];
#pragma unroll
  for (int k = 0; k < NPT; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) D0[k][i] = N.Dl[k][i];
  int st2 = 0, it2 = 0;
  for (int attempt = 0; attempt < 4; ++attempt) {
    if (attempt) {
#pragma unroll
      for (int k = 0; k < NPT; ++k)
#pragma unroll
        for (int i = 0; i < 3; ++i) N.Dl[k][i] = D0[k][i];
    }
    int ii = 0;
    st2 = stage2_ipm(S, N, w, rb, S.kc, smooth ? R(-1) : S.khard, &ii, warm2 && attempt < 2,
                     attempt == 0 ? R(0.99) : (attempt < 3 ? R(0.9) : R(0.75)));
    it2 += ii;
    if (!(st2 & ST_CONTACT)) break;
  }
  *iit = it2;
  return st | st2;
}

// x0 <- x0 + dx + Dl ; g <- g + u ; c <- c + u - (dx_a + Dl_a); x0 published on exit
template <typename R, int NPT>
__device__ __forceinline__ void advance_state(const Scene<R>& S, Nd<R, NPT>& N, const Sm<R>& w) {
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
#pragma unroll
    for (int gi = 0; gi < 2; ++gi)
      if (S.grasp[gi] == j)
#pragma unroll
        for (int i = 0; i < 3; ++i)
          w.misc[M_C + 3 * gi + i] += w.misc[M_U + 3 * gi + i] - (N.dx[k][i] + N.Dl[k][i]);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      N.x0[k][i] += N.dx[k][i] + N.Dl[k][i];
      if (RC_SO_ON(S)) N.v[k][i] = (N.dx[k][i] + N.Dl[k][i]) / S.dt;
    }
  }
  if (threadIdx.x < 6) w.misc[M_G + threadIdx.x] += w.misc[M_U + threadIdx.x];
  publish<R, NPT>(w.x0, N.x0, w.NVP);
  __syncthreads();
}

// ------------------------------------------------------------------------------------------
// adjoint of one smooth step (eq. diff-sim with the total derivative).
//   in : xb = xbar+ (adjoint of x+), misc GB = gbar+, the smooth solution in the node state and
//        the factorisation of H2 in (T, B, V); x0 and dx published
//   out: xb = xbar (adjoint of x), misc GB = gbar, misc UB = ubar
// ------------------------------------------------------------------------------------------
// the first half of the adjoint of one smooth step (eq. diff-sim with the total derivative):
//   in : xb = xbar+, the smooth solution in the node state, x0 and dx published, the factorisation of
//        H2 in (T, B, V)
//   out: mu = H2^-1 xbar+, xs = xbar* = xbar+ - (dR/dx*)^T mu
template <typename R, int NPT>
__device__ __forceinline__ void adjoint_xs(const Scene<R>& S, const Nd<R, NPT>& N, const Sm<R>& w,
                                           const R xb[NPT][3], R mu[NPT][3], R xs[NPT][3], R tR[NPT][3]) {
  const R kappa = S.kc;
  const R* d = w.misc + M_D;
  const R* c = w.misc + M_C;
  const R* u = w.misc + M_U;
  const R* gd = w.misc + M_GD;
  const int NVP = w.NVP;
  // mu = H2^{-1} xbar+
  put_rhs<R, NPT>(S, w, xb, R(1));
  __syncthreads();
  crb_solve(w.T, w.B, w.V, w.r, S.npair);
  get_rhs<R, NPT>(S, w, mu);
  __syncthreads();                             // every thread has its mu before r is reused
  publish<R, NPT>(w.v1, mu, NVP);
  put_rhs<R, NPT>(S, w, N.Dl, R(1));           // Delta of the neighbours, through r (free until nu)
  __syncthreads();
  // xbar* = xbar+ - (dR/dx*)^T mu
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
#pragma unroll
    for (int i = 0; i < 3; ++i) xs[k][i] = xb[k][i];
    if (j >= S.nv) continue;
    const R X[3] = {N.x0[k][0] + N.dx[k][0], N.x0[k][1] + N.dx[k][1], N.x0[k][2] + N.dx[k][2]};
    const R mj[3] = {mu[k][0], mu[k][1], mu[k][2]};
    for (int o = 0; o < S.nobs; ++o) {
      R ph, n[3], Nm[9];
      obstacle_eval(S.ob_type[o], S.ob[o], X, S.rad, ph, n, Nm);
      R sg[3];
      for (int i = 0; i < 3; ++i) sg[i] = N.Dl[k][i] + ph * n[i];
      R lam[3], W[9];
      cone_force_jac(sg, n, kappa, S.mu, lam, W);
      R Wm[3], Lm[3];
      for (int i = 0; i < 3; ++i) Wm[i] = W[i * 3] * mj[0] + W[i * 3 + 1] * mj[1] + W[i * 3 + 2] * mj[2];
      cone_force_dn_T(sg, n, kappa, S.mu, mj, Lm);
      const R nWm = dot3(n, Wm);
      for (int i = 0; i < 3; ++i) {
        const R NW = Nm[i * 3] * Wm[0] + Nm[i * 3 + 1] * Wm[1] + Nm[i * 3 + 2] * Wm[2];
        const R NL = Nm[i * 3] * Lm[0] + Nm[i * 3 + 1] * Lm[1] + Nm[i * 3 + 2] * Lm[2];
        // contact part of (dR/dx*)^T mu = -G^T mu, G^T mu = -(n (n.W mu) + phi N W mu) + N dlam/dn^T mu
        xs[k][i] += -(n[i] * nWm + ph * NW) + NL;
      }
    }
#pragma unroll
    for (int si = 0; si < 4; ++si) {
      const int jo = j + spr_off(si);
      if (jo < 0 || jo >= S.nv) continue;
      R e[3], mt[3], dl[3], t3[3];
      spring_vec(N, w, k, jo, e);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        mt[i] = w.v1[i * NVP + jo] - mu[k][i];
        dl[i] = w.r[cr_v(jo >> 1, 3 * (jo & 1) + i)] - N.Dl[k][i];
      }
      // third-derivative contraction of the spring energy (odd in the spring vector: the same
      // expression at either end of the spring)
      spring_d3(e, (si == 1 || si == 2) ? S.k1 : S.k2, N.Ls[k][si], mt, dl, t3);
#pragma unroll
      for (int i = 0; i < 3; ++i) xs[k][i] += t3[i];
    }
  }
  // inertial variant: tR = -(d/dx [(D/dt) Delta])^T mu, the damping's dependence on the step start
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
#pragma unroll
    for (int i = 0; i < 3; ++i) tR[k][i] = R(0);
    if (!RC_SO_ON(S) || j >= S.nv) continue;
#pragma unroll
    for (int si = 0; si < 4; ++si) {
      const int jo = j + spr_off(si);
      if (jo < 0 || jo >= S.nv) continue;
      R ua[3], y[3], z[3], t3[3];
#pragma unroll
      for (int i = 0; i < 3; ++i) ua[i] = w.x0[i * w.NVP + jo] - N.x0[k][i];
      const R il = R(1) / sqrt(dot3(ua, ua));
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        ua[i] *= il;
        y[i] = w.r[cr_v(jo >> 1, 3 * (jo & 1) + i)] - N.Dl[k][i];
        z[i] = w.v1[i * w.NVP + jo] - mu[k][i];
      }
      damp_jt(S.cb * ((si == 1 || si == 2) ? S.k1 : S.k2), il, ua, y, z, t3);
#pragma unroll
      for (int i = 0; i < 3; ++i) tR[k][i] += t3[i];
    }
  }
  __syncthreads();                             // the neighbours' Delta are read before r is overwritten
}

// the second half of the adjoint of one smooth step: nu = H1^-1 xbar*, then xbar, gbar, ubar
template <typename R, int NPT>
__device__ __forceinline__ void adjoint_nu(const Scene<R>& S, const Nd<R, NPT>& N, const Sm<R>& w,
                                           const R mu[NPT][3], const R xs[NPT][3], R xb[NPT][3],
                                           const R tR[NPT][3], R vb[NPT][3]) {
  const R* d = w.misc + M_D;
  const R* c = w.misc + M_C;
  const R* u = w.misc + M_U;
  const R* gd = w.misc + M_GD;
  // nu = H1^{-1} xbar*, the factorisation of H1 = dF/dq* at x* in (T, B, V)
  put_rhs<R, NPT>(S, w, xs, R(1));
  __syncthreads();
  crb_solve(w.T, w.B, w.V, w.r, S.npair);
  R nu[NPT][3];
  get_rhs<R, NPT>(S, w, nu);
  // xbar = w nu + grasp terms; gbar, ubar
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
#pragma unroll
    for (int i = 0; i < 3; ++i) xb[k][i] = S.w * nu[k][i];
#pragma unroll
    for (int gi = 0; gi < 2; ++gi)
      if (S.grasp[gi] == j) {
        R gam = R(0);
#pragma unroll
        for (int i = 0; i < 3; ++i)
          gam += (N.dx[k][i] - (c[3 * gi + i] + u[3 * gi + i])) * nu[k][i] + mu[k][i] * N.Dl[k][i];
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          xb[k][i] += gam * gd[3 * gi + i];
          const R gbp = w.misc[M_GB + 3 * gi + i];
          const R dnu = d[gi] * nu[k][i];
          w.misc[M_GB + 3 * gi + i] = gbp + dnu - gam * gd[3 * gi + i];
          w.misc[M_UB + 3 * gi + i] = gbp + dnu;
        }
      }
    if (RC_SO_ON(S) && j < S.nv) {
      // inertial variant: xbar += (D/dt) nu - (d/dx [(D/dt)(x* - x)])^T nu + tR - vbar+/dt, and
      // vbar = (M/dt) nu (nu of the neighbours from the solve's vector)
#pragma unroll
      for (int i = 0; i < 3; ++i) xb[k][i] += S.cm * nu[k][i] + tR[k][i] - vb[k][i] / S.dt;
#pragma unroll
      for (int si = 0; si < 4; ++si) {
        const int jo = j + spr_off(si);
        if (jo < 0 || jo >= S.nv) continue;
        R ua[3], y[3], z[3], t3[3];
#pragma unroll
        for (int i = 0; i < 3; ++i) ua[i] = w.x0[i * w.NVP + jo] - N.x0[k][i];
        const R il = R(1) / sqrt(dot3(ua, ua));
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          ua[i] *= il;
          y[i] = w.dx[i * w.NVP + jo] - N.dx[k][i];
          z[i] = w.r[cr_v(jo >> 1, 3 * (jo & 1) + i)] - nu[k][i];
        }
        const R cs = S.cb * ((si == 1 || si == 2) ? S.k1 : S.k2);
        damp_jt(cs, il, ua, y, z, t3);
        const R uz = cs * dot3(ua, z);
#pragma unroll
        for (int i = 0; i < 3; ++i) xb[k][i] += t3[i] - uz * ua[i];
      }
#pragma unroll
      for (int i = 0; i < 3; ++i) vb[k][i] = S.w * S.dt * nu[k][i];
    }
  }
  __syncthreads();
}


// adjoint of one smooth step at its solution: H2 and H1 are assembled and factorised here; not
// positive definite means the stage-1 root is a saddle of the potential (a buckled, unstable
// equilibrium) and the step's Jacobian is reported as undefined
template <typename R, int NPT>
__device__ __forceinline__ int adjoint_step(const Scene<R>& S, Nd<R, NPT>& N, const Sm<R>& w, R xb[NPT][3],
                                            R vb[NPT][3]) {
  R mu[NPT][3], xs[NPT][3], tR[NPT][3];
  __syncthreads();
  assemble_h2(S, N, w);
  __syncthreads();
  if (!crb_factor(w.T, w.B, w.V, S.npair)) return ST_NOTPD;
  if (RC_SO_ON(S))                                    // v+ = (x+ - x)/dt: xbar+ takes vbar+/dt
#pragma unroll
    for (int k = 0; k < NPT; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) xb[k][i] += vb[k][i] / S.dt;
  adjoint_xs(S, N, w, xb, mu, xs, tR);
  assemble_P(S, N, w, false, false);
  __syncthreads();
  if (!crb_factor(w.T, w.B, w.V, S.npair)) return ST_NOTPD;
  adjoint_nu(S, N, w, mu, xs, xb, tR, vb);
  return 0;
}

// the same with both factorisations stored: H2 in (T, B, V), H1 at h1 (global)
template <typename R, int NPT>
__device__ __forceinline__ int adjoint_step_stored(const Scene<R>& S, Nd<R, NPT>& N, const Sm<R>& w, R xb[NPT][3],
                                                   R vb[NPT][3], const R* h1);

// penalty part of the planning loss at the state x0: this thread's share of the value, and the
// seeds added to sd
template <typename R, int NPT>
__device__ __forceinline__ R penalty(const Scene<R>& S, const Nd<R, NPT>& N, R sd[NPT][3], bool seeds) {
  R val = R(0);
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    if (node_of(k) >= S.nv) continue;
    for (int o = 0; o < S.nobs; ++o) {
      if (S.ob_type[o] == CS_PLANE) continue;
      R ph, n[3];
      obstacle_eval(S.ob_type[o], S.ob[o], N.x0[k], S.rad, ph, n, (R*)nullptr);
      const R v = S.pen_m - ph > R(0) ? S.pen_m - ph : R(0);
      val += S.w_pen * v * v;
      if (seeds)
        for (int i = 0; i < 3; ++i) sd[k][i] += R(-2) * S.w_pen * v * n[i];
    }
  }
  return val;
}

// ------------------------------------------------------------------------------------------
// state transfer: q = [x, g]; a checkpoint record (the layout of rope.cuh) is q [n_q] | c [6] |
// dx [3 nv] | Delta [3 nv]
// ------------------------------------------------------------------------------------------
template <typename R, int NPT>
__device__ __forceinline__ void load_q(const Scene<R>& S, Nd<R, NPT>& N, const Sm<R>& w, const R* q) {
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      N.x0[k][i] = j < S.nv ? q[3 * j + i] : R(0);
      N.v[k][i] = (RC_SO_ON(S) && j < S.nv) ? q[3 * S.nv + 3 * j + i] : R(0);
    }
  }
  const int t = threadIdx.x;
  if (t < 6) {
    const R g = q[S.nq - 6 + t];
    w.misc[M_G + t] = g;
    w.misc[M_C + t] = g - q[3 * S.grasp[t / 3] + t % 3];
  }
  publish<R, NPT>(w.x0, N.x0, w.NVP);
  __syncthreads();
}

template <typename R, int NPT>
__device__ __forceinline__ void store_q(const Scene<R>& S, const Nd<R, NPT>& N, const Sm<R>& w, R* q) {
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
    if (j < S.nv)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        q[3 * j + i] = N.x0[k][i];
        if (RC_SO_ON(S)) q[3 * S.nv + 3 * j + i] = N.v[k][i];
      }
  }
  if (threadIdx.x < 6) q[S.nq - 6 + threadIdx.x] = w.misc[M_G + threadIdx.x];
}

template <typename R, int NPT>
__device__ __forceinline__ void store_rec(const Scene<R>& S, const Nd<R, NPT>& N, const Sm<R>& w, R* r) {
  if (threadIdx.x < 6) {
    r[3 * S.nv + threadIdx.x] = w.misc[M_G + threadIdx.x];
    r[3 * S.nv + 6 + threadIdx.x] = w.misc[M_C + threadIdx.x];
  }
  R* rd = r + 3 * S.nv + 12;
  R* rD = rd + 3 * S.nv;
  R* rv = rD + 3 * S.nv;
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
    if (j < S.nv)
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        r[3 * j + i] = N.x0[k][i];
        rd[3 * j + i] = N.dx[k][i];
        rD[3 * j + i] = N.Dl[k][i];
        if (RC_SO_ON(S)) rv[3 * j + i] = N.v[k][i];
      }
  }
}

template <typename R, int NPT>
__device__ __forceinline__ void load_rec_dx(const Scene<R>& S, Nd<R, NPT>& N, const R* r) {
  const R* rd = r + 3 * S.nv + 12;
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
#pragma unroll
    for (int i = 0; i < 3; ++i) N.dx[k][i] = j < S.nv ? rd[3 * j + i] : R(0);
  }
}

// the stage-2 displacement Delta of the step that produced the state of record r
template <typename R, int NPT>
__device__ __forceinline__ void load_rec_delta(const Scene<R>& S, Nd<R, NPT>& N, const R* r) {
  const R* rD = r + 6 * S.nv + 12;
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
#pragma unroll
    for (int i = 0; i < 3; ++i) N.Dl[k][i] = j < S.nv ? rD[3 * j + i] : R(0);
  }
}

template <typename R, int NPT>
__device__ __forceinline__ void load_rec(const Scene<R>& S, Nd<R, NPT>& N, const Sm<R>& w, const R* r) {
#pragma unroll
  for (int k = 0; k < NPT; ++k) {
    const int j = node_of(k);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      N.x0[k][i] = j < S.nv ? r[3 * j + i] : R(0);
      N.v[k][i] = (RC_SO_ON(S) && j < S.nv) ? r[9 * S.nv + 12 + 3 * j + i] : R(0);
    }
  }
  if (threadIdx.x < 6) {
    w.misc[M_G + threadIdx.x] = r[3 * S.nv + threadIdx.x];
    w.misc[M_C + threadIdx.x] = r[3 * S.nv + 6 + threadIdx.x];
  }
  publish<R, NPT>(w.x0, N.x0, w.NVP);
  __syncthreads();
}

// true on every thread when some node has a nonzero Delta (the previous step ran stage 2)
template <typename R, int NPT>
__device__ __forceinline__ bool any_delta(const Nd<R, NPT>& N) {
  bool nz = false;
#pragma unroll
  for (int k = 0; k < NPT; ++k)
#pragma unroll
    for (int i = 0; i < 3; ++i) nz = nz || N.Dl[k][i] != R(0);
  return __syncthreads_or(nz);
}

extern __shared__ __align__(16) unsigned char rc_smem[];

// ------------------------------------------------------------------------------------------
// kernels
// ------------------------------------------------------------------------------------------
// CTAs per SM the register budget is sized for: FP32 64-node ropes fit 7 (31 KB of shared memory);
// FP64 and 128-node scenes are held to fewer by shared memory, so they keep more registers
template <typename R, int NPT>
__host__ __device__ constexpr int ctas_per_sm() { return sizeof(R) == 4 && NPT == 1 ? 7 : (NPT == 1 ? 3 : 2); }

template <typename R, int NPT>
__global__ void __launch_bounds__(NT, (ctas_per_sm<R, NPT>())) rope_cta_rollout_kernel(
    Scene<R> S, int B, int H, const R* q0, const R* U, R* traj, R* qH, int32_t* status, int32_t* counters) {
  const int nq = S.nq;
  Sm<R> w = sm_carve<R>(reinterpret_cast<R*>(rc_smem), NPT, S.nobs);
  Red rb;
  Nd<R, NPT> N;
  zero_nd(N);
  load_rest(S, N);
  const bool smooth = S.fwd_mode == CS_SMOOTH;
  for (int b = blockIdx.x; b < B; b += gridDim.x) {
    load_q(S, N, w, q0 + (size_t)b * nq);
    zero3<R, NPT>(N.Dl);
    if (traj) store_q(S, N, w, traj + (size_t)b * (H + 1) * nq);
    int st = 0;
    const R* Ub = U + (size_t)b * H * 6;
    for (int t = 0; t < H; ++t) {
      if (threadIdx.x < 6) w.misc[M_U + threadIdx.x] = Ub[6 * t + threadIdx.x];
      // stage 2 starts from the previous step's Delta when that step ran stage 2
      const bool w2 = any_delta(N);          // also publishes the controls (a barrier)
      int ni, ii;
      const int s1 = sim_step(S, N, w, rb, smooth, &ni, &ii, false, w2);
      st |= s1;
      if (counters && threadIdx.x == 0) {
        int32_t* c = counters + ((size_t)b * H + t) * 3;
        c[0] = ni; c[1] = ii; c[2] = s1;
      }
      advance_state(S, N, w);
      if (traj) store_q(S, N, w, traj + ((size_t)b * (H + 1) + t + 1) * nq);
    }
    if (qH) store_q(S, N, w, qH + (size_t)b * nq);
    if (threadIdx.x == 0 && status) status[b] = st;
    __syncthreads();
  }
}

// what the forward part hands to the backward part, per rollout, after its records: the adjoint
// seeds of q_H (node j at [3 j + c], the grippers at [3 nv + c], the inertial variant's velocities
// at [3 nv + 6 + 3 j + c]); fits in the carry room of vjp_ws_elems (6 x 64 + 8 >= 3 x 128 + 6,
// 12 x 64 + 8 >= 6 x 128 + 6)
template <typename R, int NPT, int PH>
__device__ __forceinline__ void vjp_rollout(const Scene<R>& S, const Sm<R>& w, Nd<R, NPT>& N, Red& rb, int H,
                                            const R* q0, const R* U, const R* dLdtraj, R* Lout, R* dLdu,
                                            R* dLdq0, int32_t* status, R* ck, int32_t* cost) {
  const int nq = S.nq;
  const int rl = rec_len_rc(S.nv, RC_SO_ON(S));
  const int k = S.ckpt;
  const int nseg = (H + k - 1) / k;
  const bool fwd_smooth = S.grad_mode == CS_CONSISTENT;
  const int tid = threadIdx.x;
  enum { FWD = 0, RECOMP = 1, BACK = 2 };
  R* seg = ck + (size_t)(nseg + 1) * rl;     // segment records [k][rl]
  R* carry = ck + (vjp_ws_elems(S.nv, H, k, RC_SO_ON(S)) - vjp_carry_elems(2, RC_SO_ON(S)));
  int st = 0;
  R Lacc = R(0);
  R xb[NPT][3], vb[NPT][3];        // adjoints of the positions and (inertial variant) velocities
  zero3<R, NPT>(xb);
  zero3<R, NPT>(vb);
  int work = 0;
  int kind = FWD, t = 0, sgi = nseg - 1, t0 = 0, t1 = 0;
  // the first step of segment sgi: its start state from the checkpoint, recomputed steps (if it
  // has more than one) then its backward steps
  auto begin_segment = [&]() {
    t0 = sgi * k;
    t1 = min(t0 + k, H);
    load_rec(S, N, w, ck + (size_t)sgi * rl);
    load_rec_delta(S, N, ck + (size_t)sgi * rl);
    store_rec(S, N, w, seg);
    if (t1 - t0 > 1) { kind = RECOMP; t = t0; } else { kind = BACK; t = t0; }
  };
  if constexpr ((PH & VJP_FWD) != 0) {
    load_q(S, N, w, q0);
    zero3<R, NPT>(N.Dl);
    store_rec(S, N, w, ck);
  } else {
#pragma unroll
    for (int kk = 0; kk < NPT; ++kk) {
      const int j = node_of(kk);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        xb[kk][i] = j < S.nv ? carry[3 * j + i] : R(0);
        vb[kk][i] = (RC_SO_ON(S) && j < S.nv) ? carry[3 * S.nv + 6 + 3 * j + i] : R(0);
      }
    }
    if (tid < 6) w.misc[M_GB + tid] = carry[3 * S.nv + tid];
    begin_segment();
  }
  while (true) {
    if (kind == BACK) {
      load_rec(S, N, w, seg + (size_t)(t - t0) * rl);
      // start the smooth re-solve at the forward step's stage-1 solution and stage-2 displacement
      // (record of q_{t+1})
      const R* rn = t + 1 < t1 ? seg + (size_t)(t + 1 - t0) * rl : ck + (size_t)(sgi + 1) * rl;
      load_rec_dx(S, N, rn);
      load_rec_delta(S, N, rn);
    }
    if (tid < 6) w.misc[M_U + tid] = U[6 * t + tid];
    // stage-2 start: in the backward the forward step's Delta; forward and recompute start from
    // the previous step's Delta when it ran stage 2 (any_delta is also the barrier after the
    // controls)
    const bool w2 = any_delta(N) || kind == BACK;
    int ni, ii;
    st |= sim_step(S, N, w, rb, kind == BACK || fwd_smooth, &ni, &ii, kind == BACK, w2);
    if (st) break;                 // a failed step: the rollout's loss and gradient are undefined
    if (kind == FWD) work = min(work + 2 * ni + 5 * ii, 1 << 30);
    if (kind != BACK) {
      advance_state(S, N, w);
      if (kind == FWD) {
        if ((t + 1) % k == 0 || t == H - 1) store_rec(S, N, w, ck + (size_t)((t + k) / k) * rl);
        if (S.has_loss) Lacc += penalty(S, N, xb, false);
      } else {
        store_rec(S, N, w, seg + (size_t)(t + 1 - t0) * rl);
      }
    } else {
      st |= adjoint_step(S, N, w, xb, vb);
      if (st) break;
      if (tid < 6)
        dLdu[6 * t + tid] = w.misc[M_UB + tid] + (S.has_loss ? R(2) * S.w_u * U[6 * t + tid] : R(0));
    }
    // seeds dL/dq_t of the state the adjoint reaches next (q_H after the forward, q_t after a
    // backward step); x0 holds that state in both cases
    const bool seed_now = (kind == FWD && t == H - 1) || kind == BACK;
    if (seed_now) {
      if (kind == FWD) {
        if (tid < 6) w.misc[M_GB + tid] = R(0);
        if (S.has_loss) {
#pragma unroll
          for (int kk = 0; kk < NPT; ++kk) {
            const int j = node_of(kk);
            for (int gi = 0; gi < S.n_goal; ++gi) {
              if (S.goal[gi] != j) continue;
#pragma unroll
              for (int i = 0; i < 3; ++i) {
                const R e = N.x0[kk][i] - S.goal_pos[gi][i];
                Lacc += S.w_goal * e * e;
                xb[kk][i] += R(2) * S.w_goal * e;
              }
            }
          }
          for (int i = tid; i < 6 * H; i += NT) Lacc += S.w_u * U[i] * U[i];
        }
        __syncthreads();
      }
      const int ts = kind == FWD ? H : t;        // index of the seeded state
      if (ts >= 1 && S.has_loss) penalty(S, N, xb, true);
      if (dLdtraj) {
        const R* sd = dLdtraj + (size_t)ts * nq;
#pragma unroll
        for (int kk = 0; kk < NPT; ++kk) {
          const int j = node_of(kk);
          if (j < S.nv)
#pragma unroll
            for (int i = 0; i < 3; ++i) {
              xb[kk][i] += sd[3 * j + i];
              if (RC_SO_ON(S)) vb[kk][i] += sd[3 * S.nv + 3 * j + i];
            }
        }
        if (tid < 6) w.misc[M_GB + tid] += sd[nq - 6 + tid];
      }
      __syncthreads();
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
  __syncthreads();
  if constexpr (PH == VJP_FWD) {
    if (!st) {                     // hand the seeds over; L is final
#pragma unroll
      for (int kk = 0; kk < NPT; ++kk) {
        const int j = node_of(kk);
        if (j < S.nv)
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            carry[3 * j + i] = xb[kk][i];
            if (RC_SO_ON(S)) carry[3 * S.nv + 6 + 3 * j + i] = vb[kk][i];
          }
      }
      if (tid < 6) carry[3 * S.nv + tid] = w.misc[M_GB + tid];
      Lacc = bsum(Lacc, w.red, rb);
      if (tid == 0) {
        if (Lout) *Lout = Lacc;
        if (status) *status = 0;
        *cost = work;
      }
      __syncthreads();
      return;
    }
    if (tid == 0) *cost = -1;
  }
  if (st) {                        // failed rollout: L = NaN, gradients zero
    for (int i = tid; i < 6 * H; i += NT) dLdu[i] = R(0);
    zero3<R, NPT>(xb);
    zero3<R, NPT>(vb);
    if (tid < 6) w.misc[M_GB + tid] = R(0);
    Lacc = sizeof(R) == 4 ? R(nanf("")) : R(nan(""));
    __syncthreads();
  }
  if (dLdq0) {
#pragma unroll
    for (int kk = 0; kk < NPT; ++kk) {
      const int j = node_of(kk);
      if (j < S.nv)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          dLdq0[3 * j + i] = xb[kk][i];
          if (RC_SO_ON(S)) dLdq0[3 * S.nv + 3 * j + i] = vb[kk][i];
        }
    }
    if (tid < 6) dLdq0[nq - 6 + tid] = w.misc[M_GB + tid];
  }
  Lacc = bsum(Lacc, w.red, rb);
  if (tid == 0) {
    // the backward part leaves the forward's L unless the rollout failed
    if (Lout && (PH != VJP_BWD || st)) *Lout = Lacc;
    if (status) *status = st;
  }
  __syncthreads();
}

// the rollouts i = blockIdx.x, blockIdx.x + gridDim.x, ... (through order[i] when given); the
// backward part skips a rollout whose forward failed (cost -1: its outputs are written)
template <typename R, int NPT, int PH>
__device__ __forceinline__ void vjp_rollouts(const Scene<R>& S, int B, int H, const R* q0, const R* U,
                                             const R* dLdtraj, R* Lout, R* dLdu, R* dLdq0, int32_t* status,
                                             R* ws, size_t ws_stride, int32_t* cost, const int32_t* order) {
  const int nq = S.nq;
  Sm<R> w = sm_carve<R>(reinterpret_cast<R*>(rc_smem), NPT, S.nobs);
  Red rb;
  Nd<R, NPT> N;
  zero_nd(N);
  load_rest(S, N);
  for (int i = blockIdx.x; i < B; i += gridDim.x) {
    const int b = order ? order[i] : i;
    if (PH == VJP_BWD && cost[b] < 0) continue;
    RC_NS::vjp_rollout<R, NPT, PH>(S, w, N, rb, H, q0 ? q0 + (size_t)b * nq : nullptr, U + (size_t)b * H * 6,
                            dLdtraj ? dLdtraj + (size_t)b * (H + 1) * nq : nullptr, Lout ? Lout + b : nullptr,
                            dLdu + (size_t)b * H * 6, dLdq0 ? dLdq0 + (size_t)b * nq : nullptr,
                            status ? status + b : nullptr, ws + (size_t)b * ws_stride, cost ? cost + b : nullptr);
  }
}

// forward + adjoint in one launch
template <typename R, int NPT>
__global__ void __launch_bounds__(NT, (ctas_per_sm<R, NPT>())) rope_cta_vjp_kernel(
    Scene<R> S, int B, int H, const R* q0, const R* U, const R* dLdtraj, R* Lout, R* dLdu, R* dLdq0,
    int32_t* status, R* ws, size_t ws_stride) {
  RC_NS::vjp_rollouts<R, NPT, VJP_ALL>(S, B, H, q0, U, dLdtraj, Lout, dLdu, dLdq0, status, ws, ws_stride, nullptr,
                                nullptr);
}

// the forward part of every rollout: records, L, the carry and the cost of each
template <typename R, int NPT>
__global__ void __launch_bounds__(NT, (ctas_per_sm<R, NPT>())) rope_cta_vjp_fwd_kernel(
    Scene<R> S, int B, int H, const R* q0, const R* U, const R* dLdtraj, R* Lout, R* dLdu, R* dLdq0,
    int32_t* status, R* ws, size_t ws_stride, int32_t* cost) {
  RC_NS::vjp_rollouts<R, NPT, VJP_FWD>(S, B, H, q0, U, dLdtraj, Lout, dLdu, dLdq0, status, ws, ws_stride, cost,
                                nullptr);
}

// the backward part, rollout order[i] in CTA i (the block scheduler starts CTAs in index order,
// so the costliest start first)
template <typename R, int NPT>
__global__ void __launch_bounds__(NT, (ctas_per_sm<R, NPT>())) rope_cta_vjp_bwd_kernel(
    Scene<R> S, int B, int H, const R* U, const R* dLdtraj, R* Lout, R* dLdu, R* dLdq0, int32_t* status,
    R* ws, size_t ws_stride, int32_t* cost, const int32_t* order) {
  RC_NS::vjp_rollouts<R, NPT, VJP_BWD>(S, B, H, nullptr, U, dLdtraj, Lout, dLdu, dLdq0, status, ws, ws_stride, cost,
                                order);
}


// ------------------------------------------------------------------------------------------
// Work-queue adjoint.  The backward's expensive part -- recomputing each segment from its
// checkpoint, the smooth re-solve of every step and the two factorisations of its adjoint -- does
// not depend on the adjoint seeds, so it runs as independent (rollout, segment) jobs that any CTA
// takes as soon as that rollout's forward has finished; each job stores, per step, the
// factorisations of H2 and H1 and the smooth solution.  The rollout's adjoint chain (two solves
// with stored factors and the VJP products per step, last step to first) runs in the CTA that
// finishes its last segment.  One persistent launch: CTAs take the forward jobs first, then
// segment jobs in the order the forwards publish them; a CTA waits only for a forward that a
// running CTA has already taken (bounded wait; on expiry the rollout gets CS_ST_TIMEOUT).
// ------------------------------------------------------------------------------------------

// per-step record of the queue path: [H2 factor T|B|V][H1 factor T|B|V][x0 3nv][dx 3nv][Delta 3nv]
// [misc 32][status], padded to 4 elements
__host__ __device__ inline size_t fac_block(int NPT) { return (size_t)(LDT + 2 * CR_LDM) * 32 * NPT; }
__host__ __device__ inline size_t fac_step_elems(int NPT, int nv) {
  return (2 * fac_block(NPT) + 9 * (size_t)nv + 32 + 1 + 3) / 4 * 4;
}

// queue state (int32, zeroed before the launch): [0] next forward job, [1] next queue slot taken,
// [2] queue slots filled, [3] spare, then slot entries [nslot], slot ready flags [nslot], segments
// done per rollout [B]
__host__ __device__ inline size_t queue_ints(int B, int nseg) { return 4 + 2 * (size_t)B * nseg + (size_t)B; }

constexpr long long QUEUE_WAIT_MAX = 1ll << 21;   // polls of 1 us: about 2 s

template <typename R>
__device__ __forceinline__ void copy_block(R* dst, const R* src, size_t n) {
  // n is a multiple of 4 and both pointers 16-byte aligned
  if (sizeof(R) == 4) {
    const float4* s4 = reinterpret_cast<const float4*>(src);
    float4* d4 = reinterpret_cast<float4*>(dst);
    for (size_t i = threadIdx.x; i < n / 4; i += NT) d4[i] = s4[i];
  } else {
    const double2* s2 = reinterpret_cast<const double2*>(src);
    double2* d2 = reinterpret_cast<double2*>(dst);
    for (size_t i = threadIdx.x; i < n / 2; i += NT) d2[i] = s2[i];
  }
}

template <typename R, int NPT>
__device__ __forceinline__ int adjoint_step_stored(const Scene<R>& S, Nd<R, NPT>& N, const Sm<R>& w, R xb[NPT][3],
                                                   R vb[NPT][3], const R* h1) {
  R mu[NPT][3], xs[NPT][3], tR[NPT][3];
  if (RC_SO_ON(S))
#pragma unroll
    for (int k = 0; k < NPT; ++k)
#pragma unroll
      for (int i = 0; i < 3; ++i) xb[k][i] += vb[k][i] / S.dt;
  adjoint_xs(S, N, w, xb, mu, xs, tR);
  copy_block(w.T, h1, fac_block(NPT));
  adjoint_nu(S, N, w, mu, xs, xb, tR, vb);
  return 0;
}

// one (rollout, segment) job: the hard steps of the segment from its checkpoint and, at each of
// their start states, the smooth step with the factorisations of its adjoint, stored per step
template <typename R, int NPT>
__device__ __forceinline__ void seg_job(const Scene<R>& S, const Sm<R>& w, Nd<R, NPT>& N, Red& rb, int H,
                                        const R* U, const R* ck, R* fac, int sgi) {
  const int rl = rec_len_rc(S.nv, RC_SO_ON(S));
  const int k = S.ckpt;
  const int t0 = sgi * k, t1 = min(t0 + k, H);
  const size_t fb = fac_block(NPT), fs = fac_step_elems(NPT, S.nv);
  const int tid = threadIdx.x;
  load_rec(S, N, w, ck + (size_t)sgi * rl);
  load_rec_delta(S, N, ck + (size_t)sgi * rl);
  for (int t = t0; t < t1; ++t) {
    R* rec = fac + (size_t)t * fs;
    if (tid < 6) w.misc[M_U + tid] = U[6 * t + tid];
    // the hard step, as the forward took it (same start, same interior-point start)
    const bool w2 = any_delta(N);
    int ni, ii;
    int st = sim_step(S, N, w, rb, false, &ni, &ii, false, w2);
    const int hard_st = st;
    R dxh[NPT][3], Dlh[NPT][3];
#pragma unroll
    for (int kk = 0; kk < NPT; ++kk)
#pragma unroll
      for (int i = 0; i < 3; ++i) { dxh[kk][i] = N.dx[kk][i]; Dlh[kk][i] = N.Dl[kk][i]; }
    // the smooth step from the same state, started at the hard step's solution
    if (!st) st = sim_step(S, N, w, rb, true, &ni, &ii, true, true);
    if (!st) {
      __syncthreads();
      assemble_h2(S, N, w);                           // H2 = P + sum A^T W^-2 A at the solution
      __syncthreads();
      if (!crb_factor(w.T, w.B, w.V, S.npair)) st = ST_NOTPD;
      copy_block(rec, w.T, fb);
      __syncthreads();
      assemble_P(S, N, w, false, false);              // H1 = dF/dq* at the smooth x*
      __syncthreads();
      if (!crb_factor(w.T, w.B, w.V, S.npair)) st = ST_NOTPD;
      copy_block(rec + fb, w.T, fb);
    }
    R* rn = rec + 2 * fb;
#pragma unroll
    for (int kk = 0; kk < NPT; ++kk) {
      const int j = node_of(kk);
      if (j < S.nv)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          rn[3 * j + i] = N.x0[kk][i];
          rn[3 * S.nv + 3 * j + i] = N.dx[kk][i];
          rn[6 * S.nv + 3 * j + i] = N.Dl[kk][i];
        }
    }
    if (tid < 32) rn[9 * S.nv + tid] = w.misc[tid];
    if (tid == 0) rn[9 * S.nv + 32] = R(st);
    // advance with the hard step (a failed smooth step only marks its record: the chain stops at
    // the latest failed step and reads every later record)
#pragma unroll
    for (int kk = 0; kk < NPT; ++kk)
#pragma unroll
      for (int i = 0; i < 3; ++i) { N.dx[kk][i] = dxh[kk][i]; N.Dl[kk][i] = Dlh[kk][i]; }
    __syncthreads();
    advance_state(S, N, w);
    if (hard_st) {
      // the recomputed hard step failed (the forward did not: it does not happen); the
      // remaining records of the segment are marked failed too
      for (int t2 = t + 1; t2 < t1; ++t2)
        if (tid == 0) fac[(size_t)t2 * fs + 2 * fb + 9 * S.nv + 32] = R(hard_st);
      break;
    }
  }
  __syncthreads();
}

// the adjoint chain of one rollout from its stored per-step records: steps H-1 .. 0 (eq. diff-sim
// with the total derivative, as adjoint_step)
template <typename R, int NPT>
__device__ __forceinline__ void chain_job(const Scene<R>& S, const Sm<R>& w, Nd<R, NPT>& N, Red& rb, int H,
                                          const R* U, const R* dLdtraj, R* Lout, R* dLdu, R* dLdq0,
                                          int32_t* status, const R* ck, const R* fac) {
  const int nq = S.nq;
  const int k = S.ckpt;
  const int tid = threadIdx.x;
  const size_t fb = fac_block(NPT), fs = fac_step_elems(NPT, S.nv);
  const R* carry = ck + (vjp_ws_elems(S.nv, H, k, RC_SO_ON(S)) - vjp_carry_elems(2, RC_SO_ON(S)));
  R xb[NPT][3], vb[NPT][3];
#pragma unroll
  for (int kk = 0; kk < NPT; ++kk) {
    const int j = node_of(kk);
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      xb[kk][i] = j < S.nv ? carry[3 * j + i] : R(0);
      vb[kk][i] = (RC_SO_ON(S) && j < S.nv) ? carry[3 * S.nv + 6 + 3 * j + i] : R(0);
    }
  }
  if (tid < 6) w.misc[M_GB + tid] = carry[3 * S.nv + tid];
  int st = 0;
  for (int t = H - 1; t >= 0; --t) {
    const R* rec = fac + (size_t)t * fs;
    const R* rn = rec + 2 * fb;
    st |= (int)rn[9 * S.nv + 32];
    if (st) break;
#pragma unroll
    for (int kk = 0; kk < NPT; ++kk) {
      const int j = node_of(kk);
#pragma unroll
      for (int i = 0; i < 3; ++i) {
        N.x0[kk][i] = j < S.nv ? rn[3 * j + i] : R(0);
        N.dx[kk][i] = j < S.nv ? rn[3 * S.nv + 3 * j + i] : R(0);
        N.Dl[kk][i] = j < S.nv ? rn[6 * S.nv + 3 * j + i] : R(0);
      }
    }
    if (tid < 32 && tid != M_GB && !(tid > M_GB && tid < M_GB + 6)) w.misc[tid] = rn[9 * S.nv + tid];
    publish<R, NPT>(w.x0, N.x0, w.NVP);
    publish<R, NPT>(w.dx, N.dx, w.NVP);
    copy_block(w.T, rec, fb);
    __syncthreads();
    st |= adjoint_step_stored(S, N, w, xb, vb, rec + fb);
    if (st) break;
    if (tid < 6)
      dLdu[6 * t + tid] = w.misc[M_UB + tid] + (S.has_loss ? R(2) * S.w_u * U[6 * t + tid] : R(0));
    // seeds dL/dq_t of q_t (x0)
    if (t >= 1 && S.has_loss) penalty(S, N, xb, true);
    if (dLdtraj) {
      const R* sd = dLdtraj + (size_t)t * nq;
#pragma unroll
      for (int kk = 0; kk < NPT; ++kk) {
        const int j = node_of(kk);
        if (j < S.nv)
#pragma unroll
          for (int i = 0; i < 3; ++i) {
            xb[kk][i] += sd[3 * j + i];
            if (RC_SO_ON(S)) vb[kk][i] += sd[3 * S.nv + 3 * j + i];
          }
      }
      if (tid < 6) w.misc[M_GB + tid] += sd[nq - 6 + tid];
    }
    __syncthreads();
  }
  if (st) {                        // failed rollout: L = NaN, gradients zero
    for (int i = tid; i < 6 * H; i += NT) dLdu[i] = R(0);
    zero3<R, NPT>(xb);
    zero3<R, NPT>(vb);
    if (tid < 6) w.misc[M_GB + tid] = R(0);
    __syncthreads();
  }
  if (dLdq0) {
#pragma unroll
    for (int kk = 0; kk < NPT; ++kk) {
      const int j = node_of(kk);
      if (j < S.nv)
#pragma unroll
        for (int i = 0; i < 3; ++i) {
          dLdq0[3 * j + i] = xb[kk][i];
          if (RC_SO_ON(S)) dLdq0[3 * S.nv + 3 * j + i] = vb[kk][i];
        }
    }
    if (tid < 6) dLdq0[nq - 6 + tid] = w.misc[M_GB + tid];
  }
  if (tid == 0 && st) {
    if (Lout) *Lout = sizeof(R) == 4 ? R(nanf("")) : R(nan(""));
    if (status) *status = st;
  }
  __syncthreads();
}

template <typename R, int NPT>
__global__ void __launch_bounds__(NT, (ctas_per_sm<R, NPT>())) rope_cta_vjp_queue_kernel(
    Scene<R> S, int B, int H, const R* q0, const R* U, const R* dLdtraj, R* Lout, R* dLdu, R* dLdq0,
    int32_t* status, R* ws, size_t ws_stride, R* fac, size_t fac_stride, int* q) {
  const int nq = S.nq;
  const int nseg = (H + S.ckpt - 1) / S.ckpt;
  const int nslot = B * nseg;
  int* slot = q + 4;
  int* ready = slot + nslot;
  int* done = ready + nslot;
  Sm<R> w = sm_carve<R>(reinterpret_cast<R*>(rc_smem), NPT, S.nobs);
  __shared__ int job[2];
  Red rb;
  Nd<R, NPT> N;
  zero_nd(N);
  load_rest(S, N);
  const int tid = threadIdx.x;
  // the record and copy geometry every access below relies on: 16-byte aligned blocks of a
  // multiple of 4 elements, H records per rollout within its stride (q[3] bit 2 otherwise)
  {
    const size_t fb = fac_block(NPT), fs = fac_step_elems(NPT, S.nv);
    const bool geom = ((uintptr_t)fac & 15) == 0 && ((uintptr_t)w.T & 15) == 0 && fb % 4 == 0 && fs % 4 == 0 &&
                      fac_stride % 4 == 0 && (size_t)H * fs <= fac_stride && 2 * fb + 9 * (size_t)S.nv + 33 <= fs;
    if (!geom) {
      if (tid == 0 && blockIdx.x == 0) atomicOr(&q[3], 2);
      return;
    }
  }
  while (true) {
    // take a job: a forward while any is left, else the next queue slot
    if (tid == 0) {
      int kind = 0, val = -1;
      if (*(volatile int*)&q[0] < B) {
        const int b = atomicAdd(&q[0], 1);
        if (b < B) { kind = 1; val = b; }
      }
      if (kind == 0) {
        const int p = atomicAdd(&q[1], 1);
        if (p < nslot) {
          long long n = 0;
          while (*(volatile int*)&ready[p] == 0 && n < QUEUE_WAIT_MAX) { __nanosleep(1000); ++n; }
          __threadfence();
          if (n >= QUEUE_WAIT_MAX) { kind = 3; val = p; } else { kind = 2; val = *(volatile int*)&slot[p]; }
        }
      }
      job[0] = kind;
      job[1] = val;
    }
    __syncthreads();
    const int kind = job[0], val = job[1];
    __syncthreads();
    if (kind == 0) break;
    if (kind == 3) {                 // the wait ran out: nothing is known about this slot's rollout
      if (tid == 0) atomicOr(&q[3], 1);
      break;
    }
    if (kind == 1) {
      const int b = val;
      R* ck = ws + (size_t)b * ws_stride;
      int32_t cost = 0;
      RC_NS::vjp_rollout<R, NPT, VJP_FWD>(S, w, N, rb, H, q0 + (size_t)b * nq, U + (size_t)b * H * 6,
                                       dLdtraj ? dLdtraj + (size_t)b * (H + 1) * nq : nullptr,
                                       Lout ? Lout + b : nullptr, dLdu + (size_t)b * H * 6,
                                       dLdq0 ? dLdq0 + (size_t)b * nq : nullptr, status ? status + b : nullptr,
                                       ck, &cost);
      // publish the segment jobs (negative: the forward failed and its outputs are final)
      __syncthreads();
      if (tid == 0) {
        __threadfence();
        const int p0 = atomicAdd(&q[2], nseg);
        if (p0 + nseg > nslot) { atomicOr(&q[3], 8); continue; }   // cannot happen: B x nseg slots
        for (int sg = 0; sg < nseg; ++sg) slot[p0 + sg] = cost < 0 ? -1 : b * nseg + sg;
        __threadfence();
        for (int sg = 0; sg < nseg; ++sg) atomicExch(&ready[p0 + sg], 1);
      }
      continue;
    }
    if (val < 0) continue;           // a failed forward's placeholder
    const int b = val / nseg, sg = val % nseg;
    if (b >= B) {                    // cannot happen: entries are written as b nseg + sg
      if (tid == 0) atomicOr(&q[3], 8);
      continue;
    }
    const R* Ub = U + (size_t)b * H * 6;
    R* ck = ws + (size_t)b * ws_stride;
    R* fb = fac + (size_t)b * fac_stride;
    seg_job<R, NPT>(S, w, N, rb, H, Ub, ck, fb, sg);
    if (tid == 0) {
      __threadfence();
      const int old = atomicAdd(&done[b], 1);
      __threadfence();
      job[0] = old == nseg - 1;
    }
    __syncthreads();
    const bool last = job[0];
    __syncthreads();
    if (last)
      chain_job<R, NPT>(S, w, N, rb, H, Ub, dLdtraj ? dLdtraj + (size_t)b * (H + 1) * nq : nullptr,
                        Lout ? Lout + b : nullptr, dLdu + (size_t)b * H * 6,
                        dLdq0 ? dLdq0 + (size_t)b * nq : nullptr, status ? status + b : nullptr, ck, fb);
  }
}


// after a queue launch: a rollout whose segments did not all finish (a wait ran out, q[3] set)
// gets CS_ST_TIMEOUT, L = NaN and zero gradients
template <typename R>
__global__ void rope_queue_finish_kernel(int B, int H, int nseg, const int* q, R* Lout, R* dLdu,
                                         int32_t* status) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B || q[3] == 0) return;
  const int* done = q + 4 + 2 * (size_t)B * nseg;
  if (done[b] >= nseg || (status && status[b] != 0)) return;
  if (status) status[b] |= CS_ST_TIMEOUT;
  if (Lout) Lout[b] = sizeof(R) == 4 ? R(nanf("")) : R(nan(""));
  for (int i = 0; i < 6 * H; ++i) dLdu[(size_t)b * H * 6 + i] = R(0);
}

}  // namespace RC_NS
}  // namespace cs
