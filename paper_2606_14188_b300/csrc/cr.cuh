// Block cyclic reduction for symmetric positive definite block-tridiagonal systems with 6x6
// blocks, run by one warp over a matrix held in shared memory.
//
// A rope's node-coupled matrices (dF/dq*, the stage-2 Newton matrix) couple node j with j+1
// (stretch) and j+2 (bend): block-pentadiagonal in 3x3 node blocks, i.e. block-tridiagonal in
// 6x6 blocks of node pairs (2p, 2p+1).  Per row p of the block system:
//   T  6x6 diagonal block (lower triangle; replaced by its Cholesky factor, reciprocal diagonal)
//   B  6x6 coupling of row p with row p - s at the current reduction level
//   V  6x6 work block
//   r  6-vector right-hand side / solution
// Storage: entry e = 6 i + j of row p's B or V block at X[p * CR_LDM + e], the lower triangle
// of T packed row by row at T[p * CR_LDT + i (i + 1) / 2 + j], entry a of the vector at
// r[p * CR_LDV + a].  All strides are odd, so a warp with one lane per row touches 32 distinct
// banks.  The factorisation and the solve are called (not inlined) from every solver phase so
// that one copy of their code serves the whole kernel.
// Odd-even reduction: at level s the rows k = s (mod 2s) are eliminated in parallel and each
// survivor absorbs its two eliminated neighbours' Schur complements.  This is a Cholesky
// factorisation in the odd-even ordering, so it fails (returns false) exactly when the matrix is
// not positive definite; depth log2(N) instead of N.
#pragma once
#include "common.cuh"

namespace cs {

constexpr int CR_LDM = 37;   // row stride of a 6x6 block
constexpr int CR_LDT = 21 + 2;  // row stride of a packed lower triangle (21 entries; odd)
constexpr int CR_LDV = 7;    // row stride of a 6-vector

__device__ __forceinline__ int cr_m(int p, int e) { return p * CR_LDM + e; }
__device__ __forceinline__ int cr_t(int p, int i, int j) { return p * CR_LDT + i * (i + 1) / 2 + j; }
__device__ __forceinline__ int cr_v(int p, int a) { return p * CR_LDV + a; }

template <typename R>
__device__ __forceinline__ void ld36(const R* X, int row, R* a) {
#pragma unroll
  for (int e = 0; e < 36; ++e) a[e] = X[cr_m(row, e)];
}

template <typename R>
__device__ __forceinline__ void st36(R* X, int row, const R* a) {
#pragma unroll
  for (int e = 0; e < 36; ++e) X[cr_m(row, e)] = a[e];
}

// lower triangle of a diagonal block: packed in shared memory, row-major 6x6 in registers
template <typename R>
__device__ __forceinline__ void ld_lower(const R* T, int row, R* a) {
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int k = 0; k <= i; ++k) a[i * 6 + k] = T[cr_t(row, i, k)];
}

template <typename R>
__device__ __forceinline__ void st_lower(R* T, int row, const R* a) {
#pragma unroll
  for (int i = 0; i < 6; ++i)
#pragma unroll
    for (int k = 0; k <= i; ++k) T[cr_t(row, i, k)] = a[i * 6 + k];
}

// Factorise in place; lane i handles rows i, i + 32, ... of each reduction level.
template <typename R>
__device__ __noinline__ bool cr_factor(R* T, R* B, R* V, int N, int lane) {
  bool ok = true;
  for (int s = 1; s < N; s <<= 1) {
    const int cnt = (N - s + 2 * s - 1) / (2 * s);
    for (int idx = lane; idx < cnt; idx += 32) {
      const int k = s + 2 * s * idx;
      R L[36], U[36];
      ld_lower(T, k, L);
      ok = chol6(L) && ok;
      st_lower(T, k, L);
      ld36(B, k, U);                     // U_k = L_k^{-1} B_k (B_k couples k to k - s)
#pragma unroll
      for (int c = 0; c < 6; ++c) lsolve6(L, U + c, 6);
      st36(B, k, U);
      if (k + s < N) {                   // V_k = L_k^{-1} B_{k+s}^T
        R W[36];
#pragma unroll
        for (int c = 0; c < 6; ++c)
#pragma unroll
          for (int i = 0; i < 6; ++i) W[i * 6 + c] = B[cr_m(k + s, c * 6 + i)];
#pragma unroll
        for (int c = 0; c < 6; ++c) lsolve6(L, W + c, 6);
        st36(V, k, W);
      }
    }
    __syncwarp();
    const int cnt2 = (N + 2 * s - 1) / (2 * s);
    for (int idx = lane; idx < cnt2; idx += 32) {
      const int i = 2 * s * idx;
      R Ti[36];
      ld_lower(T, i, Ti);
      if (i + s < N) {                   // T_i -= U_{i+s}^T U_{i+s}
        R U[36];
        ld36(B, i + s, U);
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int b = 0; b <= a; ++b) {
            R t = R(0);
#pragma unroll
            for (int r = 0; r < 6; ++r) t += U[r * 6 + a] * U[r * 6 + b];
            Ti[a * 6 + b] -= t;
          }
      }
      if (i - s >= 0) {                  // T_i -= V^T V ; B_i = -V^T U   (k = i - s)
        R Vl[36], Ul[36], Bi[36];
        ld36(V, i - s, Vl);
        ld36(B, i - s, Ul);
#pragma unroll
        for (int a = 0; a < 6; ++a) {
#pragma unroll
          for (int b = 0; b <= a; ++b) {
            R t = R(0);
#pragma unroll
            for (int r = 0; r < 6; ++r) t += Vl[r * 6 + a] * Vl[r * 6 + b];
            Ti[a * 6 + b] -= t;
          }
#pragma unroll
          for (int b = 0; b < 6; ++b) {
            R t = R(0);
#pragma unroll
            for (int r = 0; r < 6; ++r) t += Vl[r * 6 + a] * Ul[r * 6 + b];
            Bi[a * 6 + b] = -t;
          }
        }
        st36(B, i, Bi);
      }
      st_lower(T, i, Ti);
    }
    __syncwarp();
  }
  if (lane == 0) {
    R L[36];
    ld_lower(T, 0, L);
    ok = chol6(L) && ok;
    st_lower(T, 0, L);
  }
  __syncwarp();
  return __all_sync(FULL, ok);
}

// Solve with the factorisation left by cr_factor; r is overwritten by the solution.
template <typename R>
__device__ __noinline__ void cr_solve(const R* T, const R* B, const R* V, R* r, int N, int lane) {
  int top = 1;
  while (top < N) top <<= 1;
  for (int s = 1; s < N; s <<= 1) {
    const int cnt = (N - s + 2 * s - 1) / (2 * s);
    for (int idx = lane; idx < cnt; idx += 32) {
      const int k = s + 2 * s * idx;
      R L[36], y[6];
      ld_lower(T, k, L);
#pragma unroll
      for (int a = 0; a < 6; ++a) y[a] = r[cr_v(k, a)];
      lsolve6(L, y, 1);
#pragma unroll
      for (int a = 0; a < 6; ++a) r[cr_v(k, a)] = y[a];
    }
    __syncwarp();
    const int cnt2 = (N + 2 * s - 1) / (2 * s);
    for (int idx = lane; idx < cnt2; idx += 32) {
      const int i = 2 * s * idx;
      R acc[6] = {0, 0, 0, 0, 0, 0};
      if (i + s < N) {
        R w[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) w[q] = r[cr_v(i + s, q)];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int q = 0; q < 6; ++q) acc[a] += B[cr_m(i + s, q * 6 + a)] * w[q];
      }
      if (i - s >= 0) {
        R w[6];
#pragma unroll
        for (int q = 0; q < 6; ++q) w[q] = r[cr_v(i - s, q)];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int q = 0; q < 6; ++q) acc[a] += V[cr_m(i - s, q * 6 + a)] * w[q];
      }
#pragma unroll
      for (int a = 0; a < 6; ++a) r[cr_v(i, a)] -= acc[a];
    }
    __syncwarp();
  }
  if (lane == 0) {
    R L[36], y[6];
    ld_lower(T, 0, L);
#pragma unroll
    for (int a = 0; a < 6; ++a) y[a] = r[cr_v(0, a)];
    lsolve6(L, y, 1);
    ltsolve6(L, y, 1);
#pragma unroll
    for (int a = 0; a < 6; ++a) r[cr_v(0, a)] = y[a];
  }
  __syncwarp();
  for (int s = top >> 1; s >= 1; s >>= 1) {
    const int cnt = (N - s + 2 * s - 1) / (2 * s);
    for (int idx = lane; idx < cnt; idx += 32) {
      const int k = s + 2 * s * idx;
      R y[6], xl[6];
#pragma unroll
      for (int a = 0; a < 6; ++a) { y[a] = r[cr_v(k, a)]; xl[a] = r[cr_v(k - s, a)]; }
#pragma unroll
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int q = 0; q < 6; ++q) y[a] -= B[cr_m(k, a * 6 + q)] * xl[q];
      if (k + s < N) {
        R xr[6];
#pragma unroll
        for (int a = 0; a < 6; ++a) xr[a] = r[cr_v(k + s, a)];
#pragma unroll
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int q = 0; q < 6; ++q) y[a] -= V[cr_m(k, a * 6 + q)] * xr[q];
      }
      R L[36];
      ld_lower(T, k, L);
      ltsolve6(L, y, 1);
#pragma unroll
      for (int a = 0; a < 6; ++a) r[cr_v(k, a)] = y[a];
    }
    __syncwarp();
  }
}

// The same solve run by a single thread on its own right-hand side, stored at
// rr[(a * NP + row) * st] (element a of row `row`); many right-hand sides at once, one per lane.
template <typename R>
__device__ __noinline__ void cr_solve_serial(const R* T, const R* B, const R* V, R* rr, int st, int N, int NP) {
  auto at = [&](int a, int row) -> R& { return rr[((size_t)a * NP + row) * st]; };
  int top = 1;
  while (top < N) top <<= 1;
  for (int s = 1; s < N; s <<= 1) {
    for (int k = s; k < N; k += 2 * s) {
      R L[36], y[6];
      ld_lower(T, k, L);
      for (int a = 0; a < 6; ++a) y[a] = at(a, k);
      lsolve6(L, y, 1);
      for (int a = 0; a < 6; ++a) at(a, k) = y[a];
    }
    for (int i = 0; i < N; i += 2 * s) {
      R acc[6] = {0, 0, 0, 0, 0, 0};
      if (i + s < N)
        for (int a = 0; a < 6; ++a)
          for (int q = 0; q < 6; ++q) acc[a] += B[cr_m(i + s, q * 6 + a)] * at(q, i + s);
      if (i - s >= 0)
        for (int a = 0; a < 6; ++a)
          for (int q = 0; q < 6; ++q) acc[a] += V[cr_m(i - s, q * 6 + a)] * at(q, i - s);
      for (int a = 0; a < 6; ++a) at(a, i) -= acc[a];
    }
  }
  {
    R L[36], y[6];
    ld_lower(T, 0, L);
    for (int a = 0; a < 6; ++a) y[a] = at(a, 0);
    lsolve6(L, y, 1);
    ltsolve6(L, y, 1);
    for (int a = 0; a < 6; ++a) at(a, 0) = y[a];
  }
  for (int s = top >> 1; s >= 1; s >>= 1) {
    for (int k = s; k < N; k += 2 * s) {
      R y[6];
      for (int a = 0; a < 6; ++a) y[a] = at(a, k);
      for (int a = 0; a < 6; ++a)
        for (int q = 0; q < 6; ++q) y[a] -= B[cr_m(k, a * 6 + q)] * at(q, k - s);
      if (k + s < N)
        for (int a = 0; a < 6; ++a)
          for (int q = 0; q < 6; ++q) y[a] -= V[cr_m(k, a * 6 + q)] * at(q, k + s);
      R L[36];
      ld_lower(T, k, L);
      ltsolve6(L, y, 1);
      for (int a = 0; a < 6; ++a) at(a, k) = y[a];
    }
  }
}

}  // namespace cs
