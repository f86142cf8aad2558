// Block cyclic reduction for symmetric positive definite block-tridiagonal systems with 6x6
// blocks, run by one warp over a matrix held in shared memory.
//
// A rope's node-coupled matrices (dF/dq*, the stage-2 Newton matrix) couple node j with j+1
// (stretch) and j+2 (bend): block-pentadiagonal in 3x3 node blocks, i.e. block-tridiagonal in
// 6x6 blocks of node pairs (2p, 2p+1).  Storage per pair row p:
//   T[p]  6x6 diagonal block (lower triangle used; overwritten by its Cholesky factor with the
//         reciprocal on the diagonal),
//   B[p]  6x6 coupling block (row p, column p-s) at the current reduction level,
//   V[p]  6x6 work block,
//   r[p]  6-vector right-hand side / solution.
// Odd-even reduction: at level s the rows k = s (mod 2s) are eliminated in parallel; each
// survivor absorbs its two eliminated neighbours' Schur complements.  This is a Cholesky
// factorisation in the odd-even ordering, so it fails (returns false) exactly when the matrix
// is not positive definite.  Depth is log2(npair) instead of npair.
#pragma once
#include "common.cuh"

namespace cs {

template <typename R>
__device__ bool cr_factor(R* T, R* B, R* V, int N, int lane) {
  bool ok = true;
  for (int s = 1; s < N; s <<= 1) {
    const int cnt = (N - s + 2 * s - 1) / (2 * s);
    for (int idx = lane; idx < cnt; idx += 32) {
      const int k = s + 2 * s * idx;
      R* L = T + k * 36;
      ok = chol6(L) && ok;
      R* U = B + k * 36;                       // U_k = L_k^{-1} B_k   (B_k couples k to k-s)
#pragma unroll 1
      for (int c = 0; c < 6; ++c) lsolve6(L, U + c, 6);
      if (k + s < N) {                         // V_k = L_k^{-1} B_{k+s}^T
        const R* Bn = B + (k + s) * 36;
        R* Vk = V + k * 36;
        for (int c = 0; c < 6; ++c)
          for (int i = 0; i < 6; ++i) Vk[i * 6 + c] = Bn[c * 6 + i];
#pragma unroll 1
        for (int c = 0; c < 6; ++c) lsolve6(L, Vk + c, 6);
      }
    }
    __syncwarp();
    const int cnt2 = (N + 2 * s - 1) / (2 * s);
    for (int idx = lane; idx < cnt2; idx += 32) {
      const int i = 2 * s * idx;
      R* Ti = T + i * 36;
      if (i + s < N) {                         // T_i -= U_{i+s}^T U_{i+s}
        const R* U = B + (i + s) * 36;
        for (int a = 0; a < 6; ++a)
          for (int b = 0; b <= a; ++b) {
            R t = R(0);
#pragma unroll
            for (int r = 0; r < 6; ++r) t += U[r * 6 + a] * U[r * 6 + b];
            Ti[a * 6 + b] -= t;
          }
      }
      if (i - s >= 0) {                        // T_i -= V^T V ; B_i = -V^T U   (k = i - s)
        const R* Vl = V + (i - s) * 36;
        const R* Ul = B + (i - s) * 36;
        R* Bi = B + i * 36;
        for (int a = 0; a < 6; ++a) {
          for (int b = 0; b <= a; ++b) {
            R t = R(0);
#pragma unroll
            for (int r = 0; r < 6; ++r) t += Vl[r * 6 + a] * Vl[r * 6 + b];
            Ti[a * 6 + b] -= t;
          }
          for (int b = 0; b < 6; ++b) {
            R t = R(0);
#pragma unroll
            for (int r = 0; r < 6; ++r) t += Vl[r * 6 + a] * Ul[r * 6 + b];
            Bi[a * 6 + b] = -t;
          }
        }
      }
    }
    __syncwarp();
  }
  if (lane == 0) ok = chol6(T) && ok;
  __syncwarp();
  return __all_sync(FULL, ok);
}

// Solve with the factorisation left by cr_factor; r [N][6] is overwritten by the solution.
template <typename R>
__device__ void cr_solve(const R* T, const R* B, const R* V, R* r, int N, int lane) {
  int top = 1;
  while (top < N) top <<= 1;
  for (int s = 1; s < N; s <<= 1) {
    const int cnt = (N - s + 2 * s - 1) / (2 * s);
    for (int idx = lane; idx < cnt; idx += 32) {
      const int k = s + 2 * s * idx;
      lsolve6(T + k * 36, r + k * 6, 1);
    }
    __syncwarp();
    const int cnt2 = (N + 2 * s - 1) / (2 * s);
    for (int idx = lane; idx < cnt2; idx += 32) {
      const int i = 2 * s * idx;
      R* ri = r + i * 6;
      R acc[6] = {0, 0, 0, 0, 0, 0};
      if (i + s < N) {
        const R* U = B + (i + s) * 36;
        const R* w = r + (i + s) * 6;
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int q = 0; q < 6; ++q) acc[a] += U[q * 6 + a] * w[q];
      }
      if (i - s >= 0) {
        const R* Vl = V + (i - s) * 36;
        const R* w = r + (i - s) * 6;
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int q = 0; q < 6; ++q) acc[a] += Vl[q * 6 + a] * w[q];
      }
      for (int a = 0; a < 6; ++a) ri[a] -= acc[a];
    }
    __syncwarp();
  }
  if (lane == 0) {
    lsolve6(T, r, 1);
    ltsolve6(T, r, 1);
  }
  __syncwarp();
  for (int s = top >> 1; s >= 1; s >>= 1) {
    const int cnt = (N - s + 2 * s - 1) / (2 * s);
    for (int idx = lane; idx < cnt; idx += 32) {
      const int k = s + 2 * s * idx;
      R y[6];
      for (int a = 0; a < 6; ++a) y[a] = r[k * 6 + a];
      const R* U = B + k * 36;
      const R* xl = r + (k - s) * 6;
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int q = 0; q < 6; ++q) y[a] -= U[a * 6 + q] * xl[q];
      if (k + s < N) {
        const R* Vk = V + k * 36;
        const R* xr = r + (k + s) * 6;
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int q = 0; q < 6; ++q) y[a] -= Vk[a * 6 + q] * xr[q];
      }
      ltsolve6(T + k * 36, y, 1);
      for (int a = 0; a < 6; ++a) r[k * 6 + a] = y[a];
    }
    __syncwarp();
  }
}

// The same solve run by a single thread on its own right-hand side, stored with element stride
// `st` (r[(p*6 + a) * st]); used to solve many right-hand sides at once, one per lane.
template <typename R>
__device__ void cr_solve_serial(const R* T, const R* B, const R* V, R* r, int st, int N) {
  int top = 1;
  while (top < N) top <<= 1;
  for (int s = 1; s < N; s <<= 1) {
    for (int k = s; k < N; k += 2 * s) lsolve6(T + k * 36, r + k * 6 * st, st);
    for (int i = 0; i < N; i += 2 * s) {
      R acc[6] = {0, 0, 0, 0, 0, 0};
      if (i + s < N) {
        const R* U = B + (i + s) * 36;
        const R* w = r + (i + s) * 6 * st;
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int q = 0; q < 6; ++q) acc[a] += U[q * 6 + a] * w[q * st];
      }
      if (i - s >= 0) {
        const R* Vl = V + (i - s) * 36;
        const R* w = r + (i - s) * 6 * st;
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int q = 0; q < 6; ++q) acc[a] += Vl[q * 6 + a] * w[q * st];
      }
      for (int a = 0; a < 6; ++a) r[(i * 6 + a) * st] -= acc[a];
    }
  }
  lsolve6(T, r, st);
  ltsolve6(T, r, st);
  for (int s = top >> 1; s >= 1; s >>= 1) {
    for (int k = s; k < N; k += 2 * s) {
      R y[6];
      for (int a = 0; a < 6; ++a) y[a] = r[(k * 6 + a) * st];
      const R* U = B + k * 36;
      for (int a = 0; a < 6; ++a)
#pragma unroll
        for (int q = 0; q < 6; ++q) y[a] -= U[a * 6 + q] * r[((k - s) * 6 + q) * st];
      if (k + s < N) {
        const R* Vk = V + k * 36;
        for (int a = 0; a < 6; ++a)
#pragma unroll
          for (int q = 0; q < 6; ++q) y[a] -= Vk[a * 6 + q] * r[((k + s) * 6 + q) * st];
      }
      ltsolve6(T + k * 36, y, 1);
      for (int a = 0; a < 6; ++a) r[(k * 6 + a) * st] = y[a];
    }
  }
}

}  // namespace cs
