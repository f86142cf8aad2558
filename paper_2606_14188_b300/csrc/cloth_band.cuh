// Cloth topology and the CTA-wide banded Cholesky of the cloth path.
//
// A cloth of R x C nodes (node (r, c) = r C + c, row-major) has six spring families: structural
// along rows (r, c)-(r, c+1) and columns (r, c)-(r+1, c), shear along both diagonals of every cell,
// and bend at distance two along rows and columns.  Every node-coupled matrix of the method
// (dF/dq*, the stage-2 Newton matrix H2 = P + sum A^T M A) is symmetric and banded with scalar half
// bandwidth bw = 3 span + 2, span = the largest node-index difference of a spring (2 C).
//
// Factorisation: one CTA, right-looking and blocked by panels of CL_KB columns over a window of
// the band held in shared memory: column c in slot c mod WC, its row i at offset i - (c & ~3), so
// that every 4-row segment starting at a multiple of 4 is 16-byte aligned.  Columns are assembled straight into the window as they enter it
// (spring Hessian blocks computed there, diagonal blocks from a node array), the panel is factored
// by one warp while the rank-CL_KB update of the trailing triangle is shared by all threads, and the
// finished panel is written to global memory (column-major band, stride LDB) for the backward
// solve.  The forward substitution of one right-hand side is fused into the panel step.
#pragma once
#include "common.cuh"

namespace cs {

constexpr int CL_NT = 512;              // threads per CTA
constexpr int CL_NW = CL_NT / 32;
constexpr int CL_KB = 12;               // panel width (four nodes)

struct ClothDims {
  int R, C, nv, N;       // grid, nodes, unknowns (3 nv)
  int bw;                // scalar half bandwidth
  int LDW, WC;           // window: column stride (multiple of 4), columns held (multiple of 3)
  int LDB;               // global factor column stride (multiple of 4, > bw + 1)
  int PL;                // panel buffer row length
  int nspr;              // springs
  int off[7];            // first spring of each family (off[6] = nspr)
  int win_global;        // the band window lives in the CTA's global workspace slot (too wide
                         // for shared memory) instead of shared memory
};

__host__ __device__ inline int cl_rup(int x, int m) { return (x + m - 1) / m * m; }

__host__ __device__ inline ClothDims cloth_dims(int R, int C) {
  ClothDims d;
  d.R = R; d.C = C; d.nv = R * C; d.N = 3 * d.nv;
  int span = 0;
  if (C >= 2) span = 1;
  if (C >= 3) span = 2;
  if (R >= 2 && C > span) span = C;
  if (R >= 2 && C >= 2 && C + 1 > span) span = C + 1;
  if (R >= 3 && 2 * C > span) span = 2 * C;
  d.bw = 3 * span + 2;
  d.LDW = cl_rup(d.bw + 5, 4);          // padding (c & 3) in front, at least one spare entry behind
  d.WC = cl_rup(d.bw + CL_KB, 3);
  d.LDB = cl_rup(d.bw + 2, 4);          // at least one spare entry behind the band
  d.PL = cl_rup(d.bw + CL_KB + 3, 4);
  const int nh = R * (C - 1), nvt = (R - 1) * C, nd = (R - 1) * (C - 1);
  const int nbh = C >= 3 ? R * (C - 2) : 0, nbv = R >= 3 ? (R - 2) * C : 0;
  d.off[0] = 0;
  d.off[1] = d.off[0] + (C >= 2 ? nh : 0);
  d.off[2] = d.off[1] + (R >= 2 ? nvt : 0);
  d.off[3] = d.off[2] + (R >= 2 && C >= 2 ? nd : 0);
  d.off[4] = d.off[3] + (R >= 2 && C >= 2 ? nd : 0);
  d.off[5] = d.off[4] + nbh;
  d.off[6] = d.off[5] + nbv;
  d.nspr = d.off[6];
  d.win_global = 0;
  return d;
}

// shared memory of one CTA (elements of the real type): window (or the two staging panels of a
// solve), panel buffer, solve barriers, right-hand side, panel partial sums, reductions, step
// scalars, state and stage-1 offset
__host__ __device__ inline size_t cloth_win_elems(const ClothDims& d) {
  const size_t win = d.win_global ? 0 : (size_t)d.WC * d.LDW;
  const size_t stg = (size_t)2 * CL_KB * d.LDB;
  return ((win > stg ? win : stg) + 3) & ~(size_t)3;       // keeps the panel buffer 16-byte aligned
}

// the band window in global memory, when it is there
__host__ __device__ inline size_t cloth_gwin_elems(const ClothDims& d) {
  return d.win_global ? (((size_t)d.WC * d.LDW + 3) & ~(size_t)3) : 0;
}

// after the panel buffer: the solves' two mbarriers and a failure flag (32 bytes or more,
// 16-byte aligned), then the right-hand side
__host__ __device__ inline size_t cloth_mbar_off(const ClothDims& d) {
  return cloth_win_elems(d) + (size_t)CL_KB * d.PL;
}
__host__ __device__ inline size_t cloth_vb_off(const ClothDims& d) { return cloth_mbar_off(d) + 8; }

__host__ __device__ inline size_t cloth_smem_elems(const ClothDims& d) {
  return cloth_vb_off(d) + (size_t)d.N + CL_KB + 64 + 64 + 2 * (size_t)d.N;
}

// place the band window (shared memory when it fits, else the global workspace slot); false when
// even the rest does not fit in shared memory
inline bool cloth_fit(ClothDims& d, size_t real_bytes, size_t smem_optin) {
  const size_t avail = smem_optin - 256;   // the kernels' static shared variables come on top
  d.win_global = 0;
  if (cloth_smem_elems(d) * real_bytes <= avail) return true;
  d.win_global = 1;
  return cloth_smem_elems(d) * real_bytes <= avail;
}

// four consecutive elements (16-byte aligned for float)
template <typename R>
__device__ __forceinline__ void ld4(const R* p, R o[4]) { o[0] = p[0]; o[1] = p[1]; o[2] = p[2]; o[3] = p[3]; }
template <>
__device__ __forceinline__ void ld4<float>(const float* p, float o[4]) {
  const float4 v = *reinterpret_cast<const float4*>(p);
  o[0] = v.x; o[1] = v.y; o[2] = v.z; o[3] = v.w;
}
template <typename R>
__device__ __forceinline__ void st4(R* p, const R v[4]) { p[0] = v[0]; p[1] = v[1]; p[2] = v[2]; p[3] = v[3]; }
template <>
__device__ __forceinline__ void st4<float>(float* p, const float v[4]) {
  *reinterpret_cast<float4*>(p) = make_float4(v[0], v[1], v[2], v[3]);
}

// elements of one CTA's workspace slot in global memory: six node vectors [N], the diagonal
// blocks [nv][6], the contact pairs (s, z, n, g, r_z [3], phi [1], M [6] per pair), the band
// factor [N][LDB] and, for a cloth too wide for shared memory, the band window; each array padded
// to a multiple of 4 elements
__host__ __device__ inline size_t cloth_ws_elems(const ClothDims& D, int nobs) {
  const size_t N = (size_t)D.N, np = (size_t)nobs * D.nv;
  auto r4 = [](size_t x) { return (x + 3) & ~(size_t)3; };
  return 6 * r4(N) + r4(6 * (size_t)D.nv) + 5 * r4(3 * np) + r4(np) + r4(6 * np) + r4(N * D.LDB) +
         cloth_gwin_elems(D);
}

// spring s -> nodes a < b and family (0, 1 structural; 2, 3 shear; 4, 5 bend)
__device__ __forceinline__ void cl_spring(const ClothDims& D, int s, int& a, int& b, int& fam) {
  fam = 0;
  while (s >= D.off[fam + 1]) ++fam;
  const int i = s - D.off[fam], C = D.C;
  int r, c;
  switch (fam) {
    case 0: r = i / (C - 1); c = i - r * (C - 1); a = r * C + c; b = a + 1; break;
    case 1: r = i / C; c = i - r * C; a = r * C + c; b = a + C; break;
    case 2: r = i / (C - 1); c = i - r * (C - 1); a = r * C + c; b = a + C + 1; break;
    case 3: r = i / (C - 1); c = i - r * (C - 1); a = r * C + c + 1; b = (r + 1) * C + c; break;
    case 4: r = i / (C - 2); c = i - r * (C - 2); a = r * C + c; b = a + 2; break;
    default: r = i / C; c = i - r * C; a = r * C + c; b = a + 2 * C; break;
  }
}

template <typename R>
__device__ __forceinline__ R cl_stiff(const Scene<R>& S, int fam) {
  return fam < 2 ? S.k1 : (fam < 4 ? S.k3 : S.k2);
}

// incident spring t (0..11) of node v = (r, c): returns its index (or -1) and the other node u;
// even t: v is the lower node (d = x_u - x_v), odd t: v is the upper node (d = x_v - x_u)
__device__ __forceinline__ int cl_incident(const ClothDims& D, int v, int t, int& u, int& fam) {
  const int C = D.C, Rr = D.R;
  const int r = v / C, c = v - r * C;
  fam = t >> 1;
  switch (t) {
    case 0: if (c + 1 < C) { u = v + 1; return D.off[0] + r * (C - 1) + c; } break;
    case 1: if (c >= 1) { u = v - 1; return D.off[0] + r * (C - 1) + c - 1; } break;
    case 2: if (r + 1 < Rr) { u = v + C; return D.off[1] + r * C + c; } break;
    case 3: if (r >= 1) { u = v - C; return D.off[1] + (r - 1) * C + c; } break;
    case 4: if (r + 1 < Rr && c + 1 < C) { u = v + C + 1; return D.off[2] + r * (C - 1) + c; } break;
    case 5: if (r >= 1 && c >= 1) { u = v - C - 1; return D.off[2] + (r - 1) * (C - 1) + c - 1; } break;
    case 6: if (r + 1 < Rr && c >= 1) { u = v + C - 1; return D.off[3] + r * (C - 1) + c - 1; } break;
    case 7: if (r >= 1 && c + 1 < C) { u = v - C + 1; return D.off[3] + (r - 1) * (C - 1) + c; } break;
    case 8: if (c + 2 < C) { u = v + 2; return D.off[4] + r * (C - 2) + c; } break;
    case 9: if (c >= 2) { u = v - 2; return D.off[4] + r * (C - 2) + c - 2; } break;
    case 10: if (r + 2 < Rr) { u = v + 2 * C; return D.off[5] + r * C + c; } break;
    default: if (r >= 2) { u = v - 2 * C; return D.off[5] + (r - 2) * C + c; } break;
  }
  return -1;
}

// ---- CTA reductions (every thread gets the same value, summed in the same order)
template <typename R>
__device__ __forceinline__ R cl_sum(R v, R* red) {
  v = wsum(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  R t = R(0);
#pragma unroll
  for (int i = 0; i < CL_NW; ++i) t += red[i];
  __syncthreads();
  return t;
}

template <typename R>
__device__ __forceinline__ R cl_max(R v, R* red) {
  v = wmax(v);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  R t = red[0];
#pragma unroll
  for (int i = 1; i < CL_NW; ++i) t = red[i] > t ? red[i] : t;
  __syncthreads();
  return t;
}

// symmetric 3x3 block as 6 numbers: (0,0) (1,0) (1,1) (2,0) (2,1) (2,2)
__device__ __forceinline__ int sym3(int a, int b) { return a >= b ? a * (a + 1) / 2 + b : b * (b + 1) / 2 + a; }

// The matrix being factored: diagonal 3x3 blocks Dg[v] (already holding everything node-local)
// and, for every spring (v, u > v), the off-diagonal block -H_s at the positions x0 + dx.
template <typename R>
struct BandSrc {
  const R* x0;
  const R* dx;
  const R* Dg;       // [nv][6]
  bool proj;         // projected spring Hessians (transverse factor clamped at 0)
};

// spring Hessian block of spring s between v (lower) and u at the positions x0 + dx
template <typename R>
__device__ __forceinline__ void cl_spring_hess(const Scene<R>& S, const R* x0, const R* dx, int v, int u,
                                               int s, int fam, bool proj, R f[3], R H[9]) {
  R d[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) d[i] = (x0[3 * u + i] - x0[3 * v + i]) + (dx[3 * u + i] - dx[3 * v + i]);
  spring_eval(d, cl_stiff(S, fam), S.L1[s], proj, f, H);
}

// assemble the columns of nodes [v0, v1) into their window slots; slot0 = (3 v0) mod WC
template <typename R>
__device__ __forceinline__ void cl_load_cols(const Scene<R>& S, const ClothDims& D, const BandSrc<R>& M,
                                             R* Wn, int v0, int v1, int slot0) {
  const int ncol = 3 * (v1 - v0);
  for (int cl = 0; cl < ncol; ++cl) {
    int sl = slot0 + cl;
    while (sl >= D.WC) sl -= D.WC;
    R* col = Wn + sl * D.LDW;
    for (int r = threadIdx.x; r < D.LDW; r += CL_NT) col[r] = R(0);
  }
  __syncthreads();
  for (int task = threadIdx.x; task < 7 * (v1 - v0); task += CL_NT) {
    const int vl = task / 7, t = task - 7 * vl, v = v0 + vl;
    int sl[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      sl[b] = slot0 + 3 * vl + b;
      while (sl[b] >= D.WC) sl[b] -= D.WC;
    }
    if (t == 0) {
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = b; a < 3; ++a) Wn[sl[b] * D.LDW + (a - b) + ((3 * v + b) & 3)] = M.Dg[6 * v + sym3(a, b)];
    } else {
      int u, fam;
      const int s = cl_incident(D, v, 2 * (t - 1), u, fam);
      if (s < 0) continue;
      R f[3], H[9];
      cl_spring_hess(S, M.x0, M.dx, v, u, s, fam, M.proj, f, H);
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          Wn[sl[b] * D.LDW + (3 * (u - v) + a - b) + ((3 * v + b) & 3)] = -H[a * 3 + b];
    }
  }
  __syncthreads();
}

// the same, by one warp (the others update the trailing triangle meanwhile)
template <typename R>
__device__ __forceinline__ void cl_load_cols_warp(const Scene<R>& S, const ClothDims& D, const BandSrc<R>& M,
                                                  R* Wn, int v0, int v1, int slot0) {
  const int lane = threadIdx.x & 31;
  const int ncol = 3 * (v1 - v0);
  for (int cl = 0; cl < ncol; ++cl) {
    int sl = slot0 + cl;
    while (sl >= D.WC) sl -= D.WC;
    R* col = Wn + sl * D.LDW;
    for (int r = lane; r < D.LDW; r += 32) col[r] = R(0);
  }
  __syncwarp();
  for (int task = lane; task < 7 * (v1 - v0); task += 32) {
    const int vl = task / 7, t = task - 7 * vl, v = v0 + vl;
    int sl[3];
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      sl[b] = slot0 + 3 * vl + b;
      while (sl[b] >= D.WC) sl[b] -= D.WC;
    }
    if (t == 0) {
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = b; a < 3; ++a) Wn[sl[b] * D.LDW + (a - b) + ((3 * v + b) & 3)] = M.Dg[6 * v + sym3(a, b)];
    } else {
      int u, fam;
      const int s = cl_incident(D, v, 2 * (t - 1), u, fam);
      if (s < 0) continue;
      R f[3], H[9];
      cl_spring_hess(S, M.x0, M.dx, v, u, s, fam, M.proj, f, H);
#pragma unroll
      for (int b = 0; b < 3; ++b)
#pragma unroll
        for (int a = 0; a < 3; ++a)
          Wn[sl[b] * D.LDW + (3 * (u - v) + a - b) + ((3 * v + b) & 3)] = -H[a * 3 + b];
    }
  }
  __syncwarp();
}

// Cholesky factorisation L L^T of the band matrix M into Lg [N][LDB] (column c: rows c .. c+bw),
// with the forward substitution L y = vb fused (vb in shared memory becomes y).  Returns false,
// uniformly over the CTA, when a pivot is not positive (the matrix is not positive definite).
// GW: the band window is Wg in global memory (a cloth too wide for shared memory), else it is the
// start of shared memory.  Inlined at every call: as a called function under the 128-register
// budget of a 512-thread CTA it spilled registers with no stack frame of its own (ptxas -v), and
// with the window in global memory its results were nondeterministic.
template <typename R, bool GW>
__device__ __forceinline__ bool cl_factor(const Scene<R>& S, const ClothDims& D, const BandSrc<R>& M, R* Lg, R* sm,
                                       R* Wg) {
  R* Wn = GW ? Wg : sm;                    // the band window: global workspace or shared memory
  R* Pb = sm + cloth_win_elems(D);
  R* vb = sm + cloth_vb_off(D);
  R* ild = vb + D.N;                       // reciprocal pivots of the current panel [CL_KB]
  R* flag = vb + D.N + CL_KB + 63;         // last slot of the reduction area: failure flag
  const int N = D.N, bw = D.bw, WC = D.WC, LDW = D.LDW;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) flag[0] = R(0);
  cl_load_cols(S, D, M, Wn, 0, min(WC, N) / 3, 0);
  int slot0 = 0;                           // window slot of column j
  for (int j = 0; j < N; j += CL_KB) {
    const int jn = min(j + CL_KB, N), kbp = jn - j;
    int cb[CL_KB];                         // window offsets of the panel's columns
    {
      int sl = slot0;
#pragma unroll
      for (int cc = 0; cc < CL_KB; ++cc) {
        cb[cc] = sl * LDW + (cc & 3);        // row i of column j + cc at cb[cc] + (i - j - cc)
        if (++sl == WC) sl = 0;
      }
    }
    // (a) diagonal block [j, jn): lane l holds row j + l in registers; right-looking with
    //     shuffles, the forward substitution of the block rows alongside
    if (warp == 0) {
      R row[CL_KB];
      const int l = lane;
#pragma unroll
      for (int cc = 0; cc < CL_KB; ++cc)
        row[cc] = (cc < kbp && l < kbp && cc <= l && l - cc <= bw) ? Wn[cb[cc] + (l - cc)] : R(0);
      R yv = l < kbp ? vb[j + l] : R(0);
      bool bad = false;
#pragma unroll
      for (int cc = 0; cc < CL_KB; ++cc) {
        if (cc >= kbp) break;
        const R piv = __shfl_sync(FULL, row[cc], cc);
        bad = bad || !(piv > R(0)) || !(piv < R(1e300));
        const R il = rsq(piv), lp = piv * il;   // one reciprocal square root per pivot
        const R ycc = __shfl_sync(FULL, yv, cc) * il;
        // branch-free: lane cc takes the pivot, the lanes below scale their entry
        const R rs = row[cc] * il;
        row[cc] = l == cc ? lp : (l > cc ? rs : row[cc]);
        yv = l == cc ? ycc : (l > cc ? yv - rs * ycc : yv);
        const R rc = l > cc ? rs : R(0);
#pragma unroll
        for (int c2 = cc + 1; c2 < CL_KB; ++c2) {
          const R lc2 = __shfl_sync(FULL, rs, c2);
          row[c2] -= (l >= c2 ? rc : R(0)) * lc2;
        }
        if (l == 0) ild[cc] = il;
      }
      if (l < kbp) {
#pragma unroll
        for (int cc = 0; cc < CL_KB; ++cc)
          if (cc <= l && l - cc <= bw) {
            Wn[cb[cc] + (l - cc)] = row[cc];
            Lg[(size_t)(j + cc) * D.LDB + (l - cc)] = row[cc];
          }
        vb[j + l] = yv;
      }
      if (bad && l == 0) flag[0] = R(1);
    }
    __syncthreads();
    if (flag[0] != R(0)) return false;
    // (b) rows below the block: L21 = A21 L11^-T, one row per thread, and the fused forward
    //     substitution vb_i -= L21_i . y_panel; the rows also go to the panel buffer
    const int imax = min(j + kbp - 1 + bw, N - 1);
    for (int i = jn + threadIdx.x; i <= imax; i += CL_NT) {
      // branch-free: entries outside the band are read at a clamped address and replaced by 0;
      // their results (exactly 0) are stored to each column's spare last entry (window: LDW - 1,
      // factor: LDB - 1), which nothing reads
      R a[CL_KB];
      bool in[CL_KB];
#pragma unroll
      for (int cc = 0; cc < CL_KB; ++cc) {
        const int off = i - j - cc;
        in[cc] = cc < kbp && off <= bw;
        const R v = Wn[cb[cc] + min(max(off, 0), bw)];
        a[cc] = in[cc] ? v : R(0);
      }
      R acc = R(0);
#pragma unroll
      for (int cc = 0; cc < CL_KB; ++cc) {
        if (cc >= kbp) break;
        R sv = a[cc];
#pragma unroll
        for (int cp = 0; cp < cc; ++cp)           // L11[cc][cp]: column j + cp, offset cc - cp
          if (cc - cp <= bw) sv -= a[cp] * Wn[cb[cp] + (cc - cp)];
        sv *= ild[cc];
        a[cc] = sv;
        acc += sv * vb[j + cc];
      }
      vb[i] -= acc;
#pragma unroll
      for (int cc = 0; cc < CL_KB; ++cc) {
        if (cc >= kbp) break;
        const int off = i - j - cc;
        Wn[in[cc] ? cb[cc] + off : cb[cc] - (cc & 3) + LDW - 1] = a[cc];
        Lg[(size_t)(j + cc) * D.LDB + (in[cc] ? off : D.LDB - 1)] = a[cc];
        Pb[cc * D.PL + CL_KB + (i - jn)] = a[cc];
      }
    }
    // panel buffer: row i >= jn of column j + cc at [cc][CL_KB + i - jn]; everything outside
    // [jn, imax] is zero (band tail, tile padding, unused columns of a short last panel)
    for (int cc = 0; cc < CL_KB; ++cc)
      for (int ii = threadIdx.x; ii < D.PL; ii += CL_NT)
        if (cc >= kbp || ii < CL_KB || jn + ii - CL_KB > imax) Pb[cc * D.PL + ii] = R(0);
    __syncthreads();                         // the panel is final (and in Lg): its slots are free
    // the last warp assembles the columns entering the window into the panel's slots while the
    // others apply the rank-kbp update to the trailing triangle [jn, jn + T)
    const int c0 = j + WC, c1 = min(j + WC + kbp, N);
    if (warp == CL_NW - 1) {
      if (c0 < c1) cl_load_cols_warp(S, D, M, Wn, c0 / 3, c1 / 3, slot0);
    } else {
      const int T = min(bw, N - jn);
      const int nt = (T + 3) >> 2, ntiles = nt * (nt + 1) / 2;
      const int tslot = slot0 + kbp;           // window slot of column jn (before wrapping)
      for (int id = threadIdx.x; id < ntiles; id += CL_NT - 32) {
        int a = (int)((sqrtf(8.0f * (float)id + 1.0f) - 1.0f) * 0.5f);
        while (a * (a + 1) / 2 > id) --a;
        while ((a + 1) * (a + 2) / 2 <= id) ++a;
        const int b = id - a * (a + 1) / 2;
        R acc[4][4];
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = R(0);
        const R* pr = Pb + CL_KB + 4 * a;
        const R* pc = Pb + CL_KB + 4 * b;
        for (int cc = 0; cc < kbp; ++cc) {
          R ra[4], cbv[4];
          ld4(pr + cc * D.PL, ra);
          ld4(pc + cc * D.PL, cbv);
#pragma unroll
          for (int x = 0; x < 4; ++x)
#pragma unroll
            for (int y = 0; y < 4; ++y) acc[x][y] += ra[x] * cbv[y];
        }
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          const int kk = 4 * b + y;
          if (kk >= T) continue;                // (such a slot may be refilled meanwhile)
          int sl = tslot + kk;
          while (sl >= WC) sl -= WC;
          // rows jn + 4a .. jn + 4a + 3 of column jn + kk: offset 4 (a - b), aligned; rows past the
          // triangle get zero updates, rows above the diagonal land in the column's padding
          R* dst = Wn + sl * LDW + 4 * (a - b);
          R d4[4];
          ld4(dst, d4);
#pragma unroll
          for (int x = 0; x < 4; ++x) d4[x] -= acc[x][y];
          st4(dst, d4);
        }
      }
    }
    __syncthreads();
    slot0 += CL_KB;
    if (slot0 >= WC) slot0 -= WC;
  }
  return true;
}

// The two substitutions stream the factor from global memory panel by panel.  A panel (kbp
// columns of LDB elements) is contiguous in Lg, so it reaches shared memory as ONE bulk copy of the
// TMA engine (cp.async.bulk, global -> shared), completed on an mbarrier; two buffers alternate so
// that the copy of the next panel overlaps the work on the current one.  Alignment: Lg, the panel
// start j LDB (j a multiple of CL_KB, LDB a multiple of 4) and both buffers sit on 16-byte
// boundaries, and kbp LDB sizeof(R) is a multiple of 16 bytes.
//
// Every wait is bounded.  A thread whose wait runs out records it and carries on (the loop's
// indices do not depend on the data, so nothing goes out of bounds); after the loop the CTA waits
// once more, bounded, for copies still in flight and sets the solution to NaN, so that the step
// fails as non-finite instead of hanging.
constexpr unsigned CL_WAIT_LIMIT = 1u << 22;

struct ClBar {
  unsigned long long b[2];   // one mbarrier per staging buffer
  int fail;                  // a wait ran out
};
static_assert(sizeof(ClBar) <= 8 * sizeof(float), "barrier slot of the cloth shared-memory layout");

__device__ __forceinline__ unsigned cl_saddr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

template <typename R>
__device__ __forceinline__ ClBar* cl_bar(const ClothDims& D, R* sm) {
  return reinterpret_cast<ClBar*>(sm + cloth_mbar_off(D));
}

// both barriers expect one arrival per phase; every thread orders its earlier generic accesses of
// the factor (written in global memory by the factorisation) and of the staging buffers (the
// window, before) before the copies of the async proxy.  The caller synchronises afterwards.
__device__ __forceinline__ void cl_bar_init(ClBar* B) {
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cl_saddr(&B->b[0])) : "memory");
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(cl_saddr(&B->b[1])) : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    B->fail = 0;
  }
  asm volatile("fence.proxy.async;" ::: "memory");
}

// thread 0: copy panel [j, j + kbp) of the factor into buf, completing on barrier bar
template <typename R>
__device__ __forceinline__ void cl_bulk(const ClothDims& D, const R* Lg, int j, int kbp, R* buf,
                                        unsigned long long* bar) {
  const unsigned bytes = (unsigned)((size_t)kbp * D.LDB * sizeof(R));
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(cl_saddr(bar)), "r"(bytes)
               : "memory");
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
               ::"r"(cl_saddr(buf)), "l"(Lg + (size_t)j * D.LDB), "r"(bytes), "r"(cl_saddr(bar))
               : "memory");
}

// poll the barrier until the phase of the given parity has completed, at most CL_WAIT_LIMIT times
__device__ __forceinline__ bool cl_bar_wait(unsigned long long* bar, unsigned parity) {
  const unsigned a = cl_saddr(bar);
  for (unsigned it = 0; it < CL_WAIT_LIMIT; ++it) {
    unsigned done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(done)
        : "r"(a), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}

__device__ __forceinline__ bool cl_bar_failed(ClBar* B) { return *reinterpret_cast<volatile int*>(&B->fail) != 0; }

// wait for buffer b's copy (phase parity in bit b of ph, flipped afterwards); a wait that runs out
// is recorded in B->fail, and once one has, no thread waits again
__device__ __forceinline__ void cl_bar_take(ClBar* B, int b, unsigned& ph) {
  if (!cl_bar_failed(B) && !cl_bar_wait(&B->b[b], (ph >> b) & 1u)) B->fail = 1;
  ph ^= 1u << b;
}

// after the loop (all threads past a barrier): on a recorded failure wait once more, bounded, for
// the last phase taken on each buffer (the copy that may still be in flight) and poison the
// solution; then release the barriers
template <typename R>
__device__ __forceinline__ void cl_bar_finish(ClBar* B, R* vb, int N, unsigned ph) {
  if (B->fail) {
    cl_bar_wait(&B->b[0], (ph & 1u) ^ 1u);
    cl_bar_wait(&B->b[1], ((ph >> 1) & 1u) ^ 1u);
    const R q = sizeof(R) == 4 ? R(nanf("")) : R(nan(""));
    for (int i = threadIdx.x; i < N; i += CL_NT) vb[i] = q;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(cl_saddr(&B->b[0])) : "memory");
    asm volatile("mbarrier.inval.shared::cta.b64 [%0];" ::"r"(cl_saddr(&B->b[1])) : "memory");
  }
}

// backward substitution L^T x = vb in place (vb in shared memory), panels from the last
template <typename R>
__device__ __noinline__ void cl_back(const ClothDims& D, const R* Lg, R* sm) {
  R* vb = sm + cloth_vb_off(D);
  R* tc = vb + D.N;
  ClBar* B = cl_bar(D, sm);
  const int N = D.N, bw = D.bw, LDB = D.LDB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int jlast = ((N - 1) / CL_KB) * CL_KB;
  cl_bar_init(B);
  __syncthreads();
  if (threadIdx.x == 0) cl_bulk(D, Lg, jlast, N - jlast, sm, &B->b[0]);
  unsigned ph = 0;
  int buf = 0;
  for (int j = jlast; j >= 0; j -= CL_KB) {
    const int jn = min(j + CL_KB, N), kbp = jn - j;
    const R* Lb = sm + (size_t)buf * CL_KB * LDB;
    cl_bar_take(B, buf, ph);
    // the other buffer was last read before the previous iteration's closing barrier
    if (j > 0 && threadIdx.x == 0 && !cl_bar_failed(B))
      cl_bulk(D, Lg, j - CL_KB, CL_KB, sm + (size_t)(buf ^ 1) * CL_KB * LDB, &B->b[buf ^ 1]);
    for (int cc = warp; cc < kbp; cc += CL_NW) {
      const int c = j + cc;
      const R* col = Lb + cc * LDB;
      const int imax = min(c + bw, N - 1);
      R acc = R(0);
      for (int i = jn + lane; i <= imax; i += 32) acc += col[i - c] * vb[i];
      acc = wsum(acc);
      if (lane == 0) tc[cc] = acc;
    }
    __syncthreads();
    if (warp == 0) {
      // lane l holds y_{j+l} - (contributions of the rows below the panel); from the last column
      // up, x_c is broadcast and the lanes above it subtract L[c][l] x_c
      const int l = lane;
      R yl = l < kbp ? vb[j + l] - tc[l] : R(0);
      for (int cc = kbp - 1; cc >= 0; --cc) {
        const R xc = __shfl_sync(FULL, yl, cc) / Lb[cc * LDB];
        if (l == cc) yl = xc;
        else if (l < cc && cc - l <= bw) yl -= Lb[l * LDB + (cc - l)] * xc;
      }
      if (l < kbp) vb[j + l] = yl;
    }
    __syncthreads();
    buf ^= 1;
  }
  cl_bar_finish(B, vb, N, ph);
}

// forward substitution L y = vb in place
template <typename R>
__device__ __noinline__ void cl_fwd(const ClothDims& D, const R* Lg, R* sm) {
  R* vb = sm + cloth_vb_off(D);
  ClBar* B = cl_bar(D, sm);
  const int N = D.N, bw = D.bw, LDB = D.LDB;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  cl_bar_init(B);
  __syncthreads();
  if (threadIdx.x == 0) cl_bulk(D, Lg, 0, min(CL_KB, N), sm, &B->b[0]);
  unsigned ph = 0;
  int buf = 0;
  for (int j = 0; j < N; j += CL_KB) {
    const int jn = min(j + CL_KB, N), kbp = jn - j;
    const R* Lb = sm + (size_t)buf * CL_KB * LDB;
    cl_bar_take(B, buf, ph);
    if (jn < N && threadIdx.x == 0 && !cl_bar_failed(B))
      cl_bulk(D, Lg, jn, min(CL_KB, N - jn), sm + (size_t)(buf ^ 1) * CL_KB * LDB, &B->b[buf ^ 1]);
    if (warp == 0) {
      for (int c = j; c < jn; ++c) {
        const R* col = Lb + (c - j) * LDB;
        const R y = vb[c] / col[0];
        __syncwarp();
        if (lane == 0) vb[c] = y;
        const int i = c + 1 + lane;
        if (i < jn && i - c <= bw) vb[i] -= col[i - c] * y;
        __syncwarp();
      }
    }
    __syncthreads();
    // rows below the panel
    const int imax = min(jn - 1 + bw, N - 1);
    for (int i = jn + threadIdx.x; i <= imax; i += CL_NT) {
      R acc = R(0);
      for (int cc = 0; cc < kbp; ++cc) {
        const int c = j + cc;
        if (i - c <= bw) acc += Lb[cc * LDB + (i - c)] * vb[c];
      }
      vb[i] -= acc;
    }
    __syncthreads();
    buf ^= 1;
  }
  cl_bar_finish(B, vb, N, ph);
}

}  // namespace cs
