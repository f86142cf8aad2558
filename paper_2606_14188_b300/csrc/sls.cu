// Output-feedback SLS observer stage (arxiv 2606.14188, Sec. 4.2): the Kalman recursion
// (eq. kalman_recursions), the observer's closed-loop responses (eq. backward_propagations) and the
// assembly of the closed-loop maps Phi^xw, Phi^uw, Phi^xe, Phi^ue, batched over nominal
// trajectories.
//
// Every stage is a batch of dense products of small matrices (n, p ~ 100-250), computed by one
// tile routine on 256-thread CTAs: in FP32 a 128 x 128 output tile, 8 x 8 outputs per thread
// (two 4 x 4 quads 64 apart, so that a quarter warp's vector reads of a panel row are contiguous);
// in FP64 64 x 64, 4 x 4 per thread; for products with few rows (the m = 6 control rows)
// 16 x 128, 1 x 8 per thread.  The operand panels are staged through shared memory 16 deep, the
// next panel's global loads issued before the current panel's products.  The trajectories, the blocks of a block-triangular
// operator and the output tiles are the grid; the horizon is the sequential direction:
//   Kalman   per step j, five batched products and one gain solve (a CTA per trajectory:
//            Cholesky factor of the innovation matrix in shared memory, a thread per gain column);
//   Phihat^x the products Abar_{k-1} ... Abar_j of every block by doubling, the associative scan of
//            the paper's propagation: distance 1 from Abar, then each level the blocks of distance
//            (2^(m-1), 2^m] as Phi_{k,j+h} Phi_{j+h,j}, all trajectories at once: ceil(log2 N) + 1
//            launches;
//   assembly block lower-triangular products sum_i X_{k,i} Y_{i,j}, a CTA per output block tile
//            (blocks of at most 8 rows: split over the warps along K instead).
// The paper forms the horizon direction by associative scans to reach logarithmic depth for one
// trajectory; with hundreds of trajectories in one call the batch already fills the GPU, and the
// step-by-step recursion does several times fewer flops than a scan over the same elements.
//
// Packed block storage: block (k, j), 0 <= j <= k <= N, of a block lower-triangular operator over
// times 0..N at index k (k + 1) / 2 + j of T = (N + 1)(N + 2) / 2 blocks, each row-major.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <string>

#include "cordsim.h"

cs_status cs_fail(cs_status s, const std::string& msg);
cs_status cs_cuda_fail(cudaError_t e, const char* where);
void cs_count_launch();

namespace {

constexpr int TK = 16, NTH = 256, PADS = 4;
constexpr size_t kGainSmemBudget = 200 * 1024;   // shared memory of the gain kernel

// tile geometries: BM x BN outputs per CTA, RM x RN per thread (16 x 16 threads)
struct GBig { static constexpr int BM = 128, BN = 128, RM = 8, RN = 8; };
struct GMid { static constexpr int BM = 64, BN = 64, RM = 4, RN = 4; };
struct GShort { static constexpr int BM = 16, BN = 128, RM = 1, RN = 8; };

template <typename R, class G>
struct Tile {
  R a[TK][G::BM + PADS];   // op(A) panel, k-major
  R b[TK][G::BN + PADS];   // op(B) panel, k-major
};

// the tile row of this thread's r-th output row (quads of 4 rows, BM / (RM / 4) apart), likewise
// for columns
template <class G>
__device__ __forceinline__ int row_of(int ty, int r) {
  if constexpr (G::RM >= 4) return (r >> 2) * (G::BM / (G::RM / 4)) + 4 * ty + (r & 3);
  else return ty * G::RM + r;
}
template <class G>
__device__ __forceinline__ int col_of(int tx, int c) {
  if constexpr (G::RN >= 4) return (c >> 2) * (G::BN / (G::RN / 4)) + 4 * tx + (c & 3);
  else return tx * G::RN + c;
}

__device__ __forceinline__ void ld4(const float* p, float* v) {
  const float4 t = *reinterpret_cast<const float4*>(p);
  v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void ld4(const double* p, double* v) {
  const double2 a = *reinterpret_cast<const double2*>(p), b = *reinterpret_cast<const double2*>(p + 2);
  v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
}

// acc += alpha op(A)[r0.., 0..K) op(B)[0..K, c0..] for this thread's outputs.  op(X)(i, k) =
// X[i ld + k] (t = 0) or X[k ld + i] (t = 1); entries outside M x K and K x N read as zero.
template <typename R, class G>
__device__ __forceinline__ void tile_mma(R (&acc)[G::RM][G::RN], const R* __restrict__ ap, int lda,
                                         int ta, R alpha, const R* __restrict__ bp, int ldb, int tb,
                                         int M, int N, int K, int r0, int c0, Tile<R, G>& sm) {
  constexpr int LA = G::BM * TK / NTH, LB = TK * G::BN / NTH;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  R ra[LA], rb[LB];
  auto fetch = [&](int k0) {
#pragma unroll
    for (int s = 0; s < LA; ++s) {
      const int e = tid + s * NTH;
      int i, k;
      if (ta) { i = e % G::BM; k = e / G::BM; } else { k = e % TK; i = e / TK; }
      const int gi = r0 + i, gk = k0 + k;
      ra[s] = (gi < M && gk < K) ? alpha * (ta ? ap[(size_t)gk * lda + gi] : ap[(size_t)gi * lda + gk])
                                 : R(0);
    }
#pragma unroll
    for (int s = 0; s < LB; ++s) {
      const int e = tid + s * NTH;
      int k, j;
      if (tb) { k = e % TK; j = e / TK; } else { j = e % G::BN; k = e / G::BN; }
      const int gk = k0 + k, gj = c0 + j;
      rb[s] = (gk < K && gj < N) ? (tb ? bp[(size_t)gj * ldb + gk] : bp[(size_t)gk * ldb + gj]) : R(0);
    }
  };
  fetch(0);
  for (int k0 = 0; k0 < K; k0 += TK) {
#pragma unroll
    for (int s = 0; s < LA; ++s) {
      const int e = tid + s * NTH;
      if (ta) sm.a[e / G::BM][e % G::BM] = ra[s]; else sm.a[e % TK][e / TK] = ra[s];
    }
#pragma unroll
    for (int s = 0; s < LB; ++s) {
      const int e = tid + s * NTH;
      if (tb) sm.b[e % TK][e / TK] = rb[s]; else sm.b[e / G::BN][e % G::BN] = rb[s];
    }
    __syncthreads();
    if (k0 + TK < K) fetch(k0 + TK);
#pragma unroll
    for (int kk = 0; kk < TK; ++kk) {
      R av[G::RM], bv[G::RN];
      if constexpr (G::RM >= 4) {
#pragma unroll
        for (int q = 0; q < G::RM / 4; ++q) ld4(&sm.a[kk][row_of<G>(ty, 4 * q)], av + 4 * q);
      } else {
#pragma unroll
        for (int r = 0; r < G::RM; ++r) av[r] = sm.a[kk][row_of<G>(ty, r)];
      }
#pragma unroll
      for (int q = 0; q < G::RN / 4; ++q) ld4(&sm.b[kk][col_of<G>(tx, 4 * q)], bv + 4 * q);
#pragma unroll
      for (int r = 0; r < G::RM; ++r)
#pragma unroll
        for (int c = 0; c < G::RN; ++c) acc[r][c] = fma(av[r], bv[c], acc[r][c]);
    }
    __syncthreads();
  }
}

// out = acc (+ d1) (+ d2) on the tile, within M x N (all three row-major with their own ld)
template <typename R, class G>
__device__ __forceinline__ void tile_store(const R (&acc)[G::RM][G::RN], R* __restrict__ out, int ldo,
                                           const R* d1, int ld1, const R* d2, int ld2, int M, int N,
                                           int r0, int c0) {
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < G::RM; ++u) {
    const int i = r0 + row_of<G>(ty, u);
    if (i >= M) continue;
#pragma unroll
    for (int v = 0; v < G::RN; ++v) {
      const int j = c0 + col_of<G>(tx, v);
      if (j >= N) continue;
      R x = acc[u][v];
      if (d1) x += d1[(size_t)i * ld1 + j];
      if (d2) x += d2[(size_t)i * ld2 + j];
      out[(size_t)i * ldo + j] = x;
    }
  }
}

__device__ __forceinline__ void unpack_block(long long t, int& k, int& j) {
  int kk = (int)((sqrt(8.0 * (double)t + 1.0) - 1.0) * 0.5);
  while ((long long)kk * (kk + 1) / 2 > t) --kk;
  while ((long long)(kk + 1) * (kk + 2) / 2 <= t) ++kk;
  k = kk;
  j = (int)(t - (long long)kk * (kk + 1) / 2);
}

__host__ __device__ __forceinline__ long long tri_index(int k, int j) { return (long long)k * (k + 1) / 2 + j; }

// ---------------------------------------------------------------------------------------------
// batched C = sum_q alpha_q op(A_q) op(B_q) (+ D), batch item z = blockIdx.z + zoff
// ---------------------------------------------------------------------------------------------

template <typename R>
struct Prod {
  const R* a;
  long long sa;
  int lda, ta;
  R alpha;
  const R* b;
  long long sb;
  int ldb, tb;
  int K;
};

template <typename R>
struct Gemm {
  int M, N, np;
  Prod<R> pr[3];
  const R* d;
  long long sd;
  int ldd;
  R* c;
  long long sc;
  int ldc;
  long long zoff;
};

template <typename R, class G>
__global__ void __launch_bounds__(NTH, 2) sls_gemm_kernel(Gemm<R> g) {
  __shared__ __align__(16) Tile<R, G> sm;
  const long long z = blockIdx.z + g.zoff;
  const int r0 = blockIdx.y * G::BM, c0 = blockIdx.x * G::BN;
  R acc[G::RM][G::RN] = {};
  for (int q = 0; q < g.np; ++q) {
    const Prod<R> P = g.pr[q];
    tile_mma<R, G>(acc, P.a + z * P.sa, P.lda, P.ta, P.alpha, P.b + z * P.sb, P.ldb, P.tb, g.M, g.N, P.K,
             r0, c0, sm);
  }
  tile_store<R, G>(acc, g.c + z * g.sc, g.ldc, g.d ? g.d + z * g.sd : nullptr, g.ldd, (const R*)nullptr,
             0, g.M, g.N, r0, c0);
}

// ---------------------------------------------------------------------------------------------
// Kalman gain of one step for every trajectory (a CTA each):
//   L = -S^{-1} W^T,  S = F F^T + C Pi C^T  (p x p, SPD),  W = A Pi C^T  (n x p)
// S is factorised S = G G^T in shared memory, right-looking, one barrier per column: phase c
// subtracts column c's outer product (scaled by 1/S_cc) from the trailing block and scales column
// c - 1 into G; then four threads solve G G^T x = w for each column of W^T.  Up to 64 columns
// per pass keep a 120-wide innovation matrix and its right-hand sides within 93 KB (FP32), two
// CTAs per SM.
// ---------------------------------------------------------------------------------------------

template <typename R>
__global__ void __launch_bounds__(NTH) sls_gain_kernel(int p, int n, int cw, const R* __restrict__ S,
                                                       const R* __restrict__ W, R* __restrict__ L,
                                                       long long sL, int32_t* status) {
  extern __shared__ __align__(16) unsigned char sls_smem[];
  R* s = reinterpret_cast<R*>(sls_smem);   // p x p, row stride p
  R* dg = s + (size_t)p * p;               // p pivots S_cc
  R* x = dg + p;                           // p x cw right-hand sides, row stride cw + 8
  __shared__ int bad;
  const int b = blockIdx.x, tid = threadIdx.x;
  const R* Sb = S + (size_t)b * p * p;
  for (int e = tid; e < p * p; e += NTH) s[e] = Sb[e];
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int c = 0; c < p; ++c) {
    R d = s[(size_t)c * p + c];
    if (!(d > R(0))) {        // not positive definite (or NaN): continue on 1 and flag
      if (tid == 0) bad = 1;
      d = R(1);
    }
    if (tid == 0) dg[c] = d;
    const R rd = R(1) / d;
    // trailing update of the lower triangle: rows c+1+(tid/16)+16r, columns c+1+(tid%16)+16q <= row
    for (int i = c + 1 + (tid >> 4); i < p; i += 16) {
      const R lic = s[(size_t)i * p + c] * rd;
      for (int j = c + 1 + (tid & 15); j <= i; j += 16) s[(size_t)i * p + j] -= lic * s[(size_t)j * p + c];
    }
    if (c > 0) {
      const R rs = R(1) / sqrt(dg[c - 1]);
      for (int i = c + tid; i < p; i += NTH) s[(size_t)i * p + c - 1] *= rs;
    }
    __syncthreads();
  }
  for (int c = tid; c < p; c += NTH) s[(size_t)c * p + c] = sqrt(dg[c]);
  __syncthreads();

  // the right-hand sides, cw columns per pass, four threads per column: thread part q sums the
  // terms k = q mod 4 of each row's dot product and the four partial sums meet by shuffles; every
  // x_k is written and read by the one thread with q = k mod 4 (row stride cw + 8: the four parts
  // and eight columns of a warp fall in distinct banks)
  const int xs = cw + 8;
  const R* Wb = W + (size_t)b * n * p;
  R* Lb = L + (size_t)b * sL;
  const R nan = R(NAN);
  const int col = tid >> 2, part = tid & 3;
  for (int c0 = 0; c0 < n; c0 += cw) {
    const int cn = min(cw, n - c0);
    for (int e = tid; e < p * cn; e += NTH) {
      const int i = e / cn, t = e % cn;
      x[(size_t)i * xs + t] = Wb[(size_t)(c0 + t) * p + i];
    }
    __syncthreads();
    const bool act = col < cn;
    R* xc = x + col;
    for (int i = 0; i < p; ++i) {            // G y = w
      const R* gi = s + (size_t)i * p;
      R a = R(0);
      if (act)
        for (int k = part; k < i; k += 4) a -= gi[k] * xc[(size_t)k * xs];
      a += __shfl_xor_sync(0xffffffffu, a, 1);
      a += __shfl_xor_sync(0xffffffffu, a, 2);
      if (act && part == (i & 3)) xc[(size_t)i * xs] = (xc[(size_t)i * xs] + a) / gi[i];
    }
    for (int i = p - 1; i >= 0; --i) {       // G^T z = y
      R a = R(0);
      if (act)
        for (int k = i + 1 + ((part - i - 1) & 3); k < p; k += 4) a -= s[(size_t)k * p + i] * xc[(size_t)k * xs];
      a += __shfl_xor_sync(0xffffffffu, a, 1);
      a += __shfl_xor_sync(0xffffffffu, a, 2);
      if (act && part == (i & 3)) xc[(size_t)i * xs] = (xc[(size_t)i * xs] + a) / s[(size_t)i * p + i];
    }
    __syncthreads();
    for (int e = tid; e < p * cn; e += NTH) {
      const int i = e / cn, t = e % cn;
      Lb[(size_t)i * n + c0 + t] = bad ? nan : -x[(size_t)i * xs + t];
    }
    __syncthreads();
  }
  if (tid == 0 && bad && status) atomicOr(status + b, CS_ST_NOTPD);
}

// ---------------------------------------------------------------------------------------------
// Block-triangular operators (packed storage; item z = blockIdx.z + zoff over (trajectory, block))
// ---------------------------------------------------------------------------------------------

// identity diagonal blocks Phi_{k,k} = I of every trajectory
template <typename R>
__global__ void sls_identity_kernel(long long nb, int N, int n, R* Phi) {
  const long long T = (long long)(N + 1) * (N + 2) / 2;
  const long long total = nb * (N + 1) * n * n;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < total;
       e += (long long)gridDim.x * blockDim.x) {
    const long long blk = e / ((long long)n * n);
    const int r = (int)(e % ((long long)n * n));
    const long long b = blk / (N + 1);
    const int k = (int)(blk % (N + 1));
    Phi[(b * T + tri_index(k, k)) * n * n + r] = (r / n == r % n) ? R(1) : R(0);
  }
}

// one doubling level of the closed-loop products (the associative scan of eq.
// backward_propagations, combination Phi_{k,i} Phi_{i,j}): every block (k, j) at distance
// k - j in [lo, hi] of every trajectory, Phi_{k,j} = Phi_{k,j+h} Phi_{j+h,j} (both at smaller
// distances, formed by earlier levels), or for h = 0 (distance 1) Phi_{k,k-1} = Phi_{k,k} Acl_{k-1}
template <typename R, class G>
__global__ void __launch_bounds__(NTH, 2) sls_level_kernel(int N, int n, int lo, int hi, int h,
                                                        const R* __restrict__ Acl, R* Phi, long long zoff) {
  __shared__ __align__(16) Tile<R, G> sm;
  const long long z = blockIdx.z + zoff;
  long long per = 0;
  for (int dd = lo; dd <= hi; ++dd) per += N - dd + 1;
  const long long b = z / per;
  long long o = z % per;
  int d = lo;
  while (o >= N - d + 1) { o -= N - d + 1; ++d; }
  const int k = d + (int)o, j = k - d;
  const long long T = (long long)(N + 1) * (N + 2) / 2, nn = (long long)n * n;
  R* base = Phi + b * T * nn;
  const R* X = base + tri_index(k, j + (h > 0 ? h : 1)) * nn;
  const R* Y = h > 0 ? base + tri_index(j + h, j) * nn : Acl + (b * N + j) * nn;
  const int r0 = blockIdx.y * G::BM, c0 = blockIdx.x * G::BN;
  R acc[G::RM][G::RN] = {};
  tile_mma<R, G>(acc, X, n, 0, R(1), Y, n, 0, n, n, n, r0, c0, sm);
  tile_store<R, G>(acc, base + tri_index(k, j) * nn, n, (const R*)nullptr, 0, (const R*)nullptr, 0, n, n, r0,
                   c0);
}

// Phihat^y_{k,j} = Phihat^x_{k,j} L_j^T (L_j = Lg[j - 1], p x n), zero for j = 0
template <typename R, class G>
__global__ void __launch_bounds__(NTH, 2) sls_phiy_kernel(int N, int n, int p, const R* __restrict__ PX,
                                                       const R* __restrict__ Lg, R* PY, long long zoff) {
  __shared__ __align__(16) Tile<R, G> sm;
  const long long z = blockIdx.z + zoff;
  const long long T = (long long)(N + 1) * (N + 2) / 2;
  const long long b = z / T, t = z % T;
  int k, j;
  unpack_block(t, k, j);
  const int r0 = blockIdx.y * G::BM, c0 = blockIdx.x * G::BN;
  R acc[G::RM][G::RN] = {};
  if (j > 0)
    tile_mma<R, G>(acc, PX + (b * T + t) * n * n, n, 0, R(1), Lg + (b * N + j - 1) * p * n, n, 1, n, p, n, r0,
             c0, sm);
  tile_store<R, G>(acc, PY + (b * T + t) * n * p, p, (const R*)nullptr, 0, (const R*)nullptr, 0, n, p, r0, c0);
}

// (M X)_{k,j} = X_{k,j} - A_{k-1} X_{k-1,j} (j < k), X_{k,k} (j = k); M = I - Z A, X blocks n x c
template <typename R, class G>
__global__ void __launch_bounds__(NTH, 2) sls_shift_kernel(int N, int n, int c, const R* __restrict__ A,
                                                        const R* __restrict__ X, R* out, long long zoff) {
  __shared__ __align__(16) Tile<R, G> sm;
  const long long z = blockIdx.z + zoff;
  const long long T = (long long)(N + 1) * (N + 2) / 2;
  const long long b = z / T, t = z % T;
  int k, j;
  unpack_block(t, k, j);
  const int r0 = blockIdx.y * G::BM, c0 = blockIdx.x * G::BN;
  R acc[G::RM][G::RN] = {};
  if (j < k)
    tile_mma<R, G>(acc, A + (b * N + k - 1) * n * n, n, 0, R(-1), X + (b * T + tri_index(k - 1, j)) * n * c, c,
             0, n, c, n, r0, c0, sm);
  tile_store<R, G>(acc, out + (b * T + t) * n * c, c, X + (b * T + t) * n * c, c, (const R*)nullptr, 0, n, c,
             r0, c0);
}

// out_{k,j} = alpha sum_{i=j..k} X_{k,i} Y_{i,j} (+ d1_{k,j}) (+ d2_{k,j});
// X blocks r x n, Y blocks n x c, out / d1 / d2 blocks r x c
template <typename R, class G>
__global__ void __launch_bounds__(NTH, 2) sls_tri_kernel(int N, int r, int n, int c, R alpha,
                                                      const R* __restrict__ X, const R* __restrict__ Y,
                                                      const R* d1, const R* d2, R* out, long long zoff) {
  __shared__ __align__(16) Tile<R, G> sm;
  const long long z = blockIdx.z + zoff;
  const long long T = (long long)(N + 1) * (N + 2) / 2;
  const long long b = z / T, t = z % T;
  int k, j;
  unpack_block(t, k, j);
  const int r0 = blockIdx.y * G::BM, c0 = blockIdx.x * G::BN;
  R acc[G::RM][G::RN] = {};
  for (int i = j; i <= k; ++i)
    tile_mma<R, G>(acc, X + (b * T + tri_index(k, i)) * r * n, n, 0, alpha, Y + (b * T + tri_index(i, j)) * n * c,
             c, 0, r, c, n, r0, c0, sm);
  const long long o = (b * T + t) * r * c;
  tile_store<R, G>(acc, out + o, c, d1 ? d1 + o : nullptr, c, d2 ? d2 + o : nullptr, c, r, c, r0, c0);
}

// the same for blocks of r <= 8 rows (the control rows): each warp takes every eighth k of every
// product (split K), each lane VPL adjacent columns of Y's rows; a product's X block is staged in
// shared memory 128 columns at a time, transposed and padded to 8 rows (two vector reads per k);
// the eight warps' partial tiles are summed in shared memory at the end
constexpr int kThinRows = 8, kThinK = 128;

template <typename R>
__global__ void __launch_bounds__(NTH) sls_tri_thin_kernel(int N, int r, int n, int c, R alpha,
                                                           const R* __restrict__ X,
                                                           const R* __restrict__ Y, const R* d1,
                                                           const R* d2, R* out, long long zoff) {
  constexpr int VPL = sizeof(R) == 4 ? 4 : 2, CW = 32 * VPL, NW = NTH / 32;
  __shared__ R part[NW][kThinRows][CW];
  __shared__ __align__(16) R xs[kThinK][kThinRows];
  const long long z = blockIdx.z + zoff;
  const long long T = (long long)(N + 1) * (N + 2) / 2;
  const long long b = z / T, t = z % T;
  int k, j;
  unpack_block(t, k, j);
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cl = blockIdx.x * CW + lane * VPL;
  bool cv[VPL];
#pragma unroll
  for (int v = 0; v < VPL; ++v) cv[v] = cl + v < c;
  R acc[kThinRows][VPL] = {};
  for (int i = j; i <= k; ++i) {
    const R* Xb = X + (b * T + tri_index(k, i)) * r * n;
    const R* Yb = Y + (b * T + tri_index(i, j)) * n * c;
    for (int kc = 0; kc < n; kc += kThinK) {
      const int kn = min(kThinK, n - kc);
      __syncthreads();                         // the previous panel's readers are done
      for (int e = threadIdx.x; e < kThinRows * kThinK; e += NTH) {
        const int rr = e / kThinK, kk = e % kThinK;
        xs[kk][rr] = (rr < r && kk < kn) ? alpha * Xb[(size_t)rr * n + kc + kk] : R(0);
      }
      __syncthreads();
      const R* yrow = Yb + (size_t)(kc + warp) * c + cl;
      for (int kk = warp; kk < kn; kk += NW, yrow += (size_t)NW * c) {
        R yv[VPL], xv[kThinRows];
#pragma unroll
        for (int v = 0; v < VPL; ++v) yv[v] = cv[v] ? yrow[v] : R(0);
        ld4(&xs[kk][0], xv);
        ld4(&xs[kk][4], xv + 4);
#pragma unroll
        for (int rr = 0; rr < kThinRows; ++rr)
#pragma unroll
          for (int v = 0; v < VPL; ++v) acc[rr][v] = fma(xv[rr], yv[v], acc[rr][v]);
      }
    }
  }
#pragma unroll
  for (int rr = 0; rr < kThinRows; ++rr)
#pragma unroll
    for (int v = 0; v < VPL; ++v) part[warp][rr][lane * VPL + v] = acc[rr][v];
  __syncthreads();
  for (int e = threadIdx.x; e < kThinRows * CW; e += NTH) {
    const int rr = e / CW, cc = e % CW, gc = blockIdx.x * CW + cc;
    if (rr >= r || gc >= c) continue;
    R sum = R(0);
#pragma unroll
    for (int w = 0; w < NW; ++w) sum += part[w][rr][cc];
    const long long o = (b * T + t) * r * c + (long long)rr * c + gc;
    if (d1) sum += d1[o];
    if (d2) sum += d2[o];
    out[o] = sum;
  }
}

// ---------------------------------------------------------------------------------------------
// The Kalman covariances by the associative scan of eq. combination_rules (eq. initialization)
// ---------------------------------------------------------------------------------------------

// elements of every trajectory: XA[b][0] = XD[b][0] = 0, XA[b][j+1] = A_j^T; Ct[b][j] = C_j^T
// (n x p)
template <typename R>
__global__ void sls_scan_build_kernel(long long B, int N, int n, int p, const R* __restrict__ A,
                                      const R* __restrict__ Cm, R* XA, R* XD, R* Ct) {
  const long long nn = (long long)n * n, np_ = (long long)n * p;
  const long long tot_a = B * (N + 1) * nn, tot_c = B * N * np_;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot_a + tot_c;
       e += (long long)gridDim.x * blockDim.x) {
    if (e < tot_a) {
      const long long bi = e / nn;
      const int r = (int)((e % nn) / n), c = (int)(e % n);
      const long long b = bi / (N + 1);
      const int i = (int)(bi % (N + 1));
      XA[e] = i == 0 ? R(0) : A[(b * N + i - 1) * nn + (long long)c * n + r];
      if (i == 0) XD[e] = R(0);
    } else {
      const long long f = e - tot_a;             // Ct[b][j][r][c] = C[b][j][c][r]
      const long long bj = f / np_;
      const int r = (int)((f % np_) / p), c = (int)(f % p);
      Ct[f] = Cm[bj * np_ + (long long)c * n + r];
    }
  }
}

// (I + M_z) [X1 | X2] = [B1 | B2] for z = blockIdx.x + zoff (n x n blocks, stride n^2): LU with
// partial pivoting in shared memory (four barriers per column; ties to the lower row), then the
// right-hand sides cw columns at a time, four threads per column as in the gain solve; a zero
// pivot writes NaN and flags CS_ST_NOTPD on the trajectory (z + d) / N1
template <typename R>
__global__ void __launch_bounds__(NTH) sls_lu_solve_kernel(int n, int cw, const R* __restrict__ M,
                                                           const R* __restrict__ B1, const R* __restrict__ B2,
                                                           R* X1, R* X2, int32_t* status, int N1, int d,
                                                           long long zoff) {
  extern __shared__ __align__(16) unsigned char sls_smem[];
  R* a = reinterpret_cast<R*>(sls_smem);      // n x n, row stride n
  R* x = a + (size_t)n * n;                   // n x cw, row stride cw + 8
  int* perm = reinterpret_cast<int*>(x + (size_t)n * (cw + 8));
  __shared__ R wbest[NTH / 32];
  __shared__ int wbi[NTH / 32], piv, bad;
  const long long z = blockIdx.x + zoff;
  const long long nn = (long long)n * n;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const R* Mz = M + z * nn;
  for (int e = tid; e < n * n; e += NTH) a[e] = Mz[e] + ((e / n == e % n) ? R(1) : R(0));
  if (tid == 0) bad = 0;
  for (int i = tid; i < n; i += NTH) perm[i] = i;
  __syncthreads();
  for (int c = 0; c < n; ++c) {
    R best = R(-1);
    int bi = c;
    for (int i = c + tid; i < n; i += NTH) {
      const R v = fabs(a[(size_t)i * n + c]);
      if (v > best) { best = v; bi = i; }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      const R ov = __shfl_down_sync(0xffffffffu, best, o);
      const int oi = __shfl_down_sync(0xffffffffu, bi, o);
      if (ov > best || (ov == best && oi < bi)) { best = ov; bi = oi; }
    }
    if (lane == 0) { wbest[warp] = best; wbi[warp] = bi; }
    __syncthreads();
    if (tid == 0) {
      R b0 = wbest[0];
      int i0 = wbi[0];
      for (int w = 1; w < NTH / 32; ++w)
        if (wbest[w] > b0 || (wbest[w] == b0 && wbi[w] < i0)) { b0 = wbest[w]; i0 = wbi[w]; }
      piv = i0;
      if (!(b0 > R(0))) bad = 1;
      const int t = perm[c]; perm[c] = perm[i0]; perm[i0] = t;
    }
    __syncthreads();
    const int pr = piv;
    if (pr != c)
      for (int j = tid; j < n; j += NTH) {
        const R t = a[(size_t)c * n + j];
        a[(size_t)c * n + j] = a[(size_t)pr * n + j];
        a[(size_t)pr * n + j] = t;
      }
    __syncthreads();
    R dcc = a[(size_t)c * n + c];
    if (!(fabs(dcc) > R(0))) dcc = R(1);
    const R rd = R(1) / dcc;
    for (int i = c + 1 + tid; i < n; i += NTH) a[(size_t)i * n + c] *= rd;
    __syncthreads();
    for (int i = c + 1 + (tid >> 4); i < n; i += 16) {
      const R lic = a[(size_t)i * n + c];
      for (int j = c + 1 + (tid & 15); j < n; j += 16) a[(size_t)i * n + j] -= lic * a[(size_t)c * n + j];
    }
    __syncthreads();
  }
  const int xs = cw + 8, col = tid >> 2, part = tid & 3;
  const R nan = R(NAN);
  for (int c0 = 0; c0 < 2 * n; c0 += cw) {
    const int cn = min(cw, 2 * n - c0);
    for (int e = tid; e < n * cn; e += NTH) {
      const int i = e / cn, t = e % cn, cc = c0 + t;
      const R* src = cc < n ? B1 + z * nn + cc : B2 + z * nn + (cc - n);
      x[(size_t)i * xs + t] = src[(size_t)perm[i] * n];
    }
    __syncthreads();
    const bool act = col < cn;
    R* xc = x + col;
    for (int i = 0; i < n; ++i) {             // unit lower L y = P b
      const R* ai = a + (size_t)i * n;
      R s = R(0);
      if (act)
        for (int k = part; k < i; k += 4) s -= ai[k] * xc[(size_t)k * xs];
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (act && part == (i & 3)) xc[(size_t)i * xs] += s;
    }
    for (int i = n - 1; i >= 0; --i) {        // U x = y
      const R* ai = a + (size_t)i * n;
      R s = R(0);
      if (act)
        for (int k = i + 1 + ((part - i - 1) & 3); k < n; k += 4) s -= ai[k] * xc[(size_t)k * xs];
      s += __shfl_xor_sync(0xffffffffu, s, 1);
      s += __shfl_xor_sync(0xffffffffu, s, 2);
      if (act && part == (i & 3)) xc[(size_t)i * xs] = (xc[(size_t)i * xs] + s) / ai[i];
    }
    __syncthreads();
    for (int e = tid; e < n * cn; e += NTH) {
      const int i = e / cn, t = e % cn, cc = c0 + t;
      R* dst = cc < n ? X1 + z * nn + cc : X2 + z * nn + (cc - n);
      dst[(size_t)i * n] = bad ? nan : x[(size_t)i * xs + t];
    }
    __syncthreads();
  }
  // pairs across two trajectories (local index below d) are discarded by the caller: no flag
  if (tid == 0 && bad && status && (z + d) % N1 >= d) atomicOr(status + (z + d) / N1, CS_ST_NOTPD);
}

// XD[b][j+1] = Dt[b][j], XP[b][j+1] = Pt[b][j]: the step elements, formed for all (b, j) at once,
// into the scan's layout (the prior first)
template <typename R>
__global__ void sls_scan_place_kernel(long long B, int N, int n, const R* Dt, const R* Pt, R* XD, R* XP) {
  const long long nn = (long long)n * n, per = (long long)N * nn;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < B * per;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / per, o = (b * (N + 1) + 1) * nn + e % per;
    XD[o] = Dt[e];
    XP[o] = Pt[e];
  }
}

// status[b] |= the flags of trajectory b's N step solves
__global__ void sls_flag_rows_kernel(int B, int N, const int32_t* fl, int32_t* status) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) {
    int32_t f = 0;
    for (int j = 0; j < N; ++j) f |= fl[(size_t)b * N + j];
    status[b] |= f;
  }
}

// Y[b][i] = X[b][i] for i < d (the elements a level leaves as they are), three arrays
template <typename R>
__global__ void sls_scan_keep_kernel(long long B, int N, int n, int d, const R* XA, const R* XD,
                                     const R* XP, R* YA, R* YD, R* YP) {
  const long long nn = (long long)n * n, per = (long long)d * nn;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < B * per;
       e += (long long)gridDim.x * blockDim.x) {
    const long long o = (e / per) * (N + 1) * nn + e % per;
    YA[o] = XA[o];
    YD[o] = XD[o];
    YP[o] = XP[o];
  }
}

// ---------------------------------------------------------------------------------------------
// Reachable tubes and constraint tightening (Sec. 4.2 eq. of_optimization_tightening1/2) and the
// conformal radius (Sec. 4.4)
// ---------------------------------------------------------------------------------------------

// row sums of squares of X_{k,j} S_{j-1} for blocks j >= 1 (X blocks r x kd packed, S [B][N][kd][c]):
// ssq[b][t][column tile][row], one tile product per CTA, the 16 threads of a row group summing
// their squares by shuffles
template <typename R, class G>
__global__ void __launch_bounds__(NTH, 2) sls_rownorm_kernel(int N, int r, int kd, int c,
                                                             const R* __restrict__ X,
                                                             const R* __restrict__ S, R* ssq,
                                                             int nct, long long zoff) {
  __shared__ __align__(16) Tile<R, G> sm;
  const long long z = blockIdx.z + zoff;
  const long long T = (long long)(N + 1) * (N + 2) / 2;
  const long long b = z / T, t = z % T;
  int k, j;
  unpack_block(t, k, j);
  const int r0 = blockIdx.y * G::BM, c0 = blockIdx.x * G::BN;
  R acc[G::RM][G::RN] = {};
  if (j > 0)
    tile_mma<R, G>(acc, X + (b * T + t) * r * kd, kd, 0, R(1), S + (b * N + j - 1) * kd * c, c, 0, r, c, kd,
                   r0, c0, sm);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int u = 0; u < G::RM; ++u) {
    R q = R(0);
#pragma unroll
    for (int v = 0; v < G::RN; ++v) q = fma(acc[u][v], acc[u][v], q);
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) q += __shfl_xor_sync(0xffffffffu, q, o);
    const int i = r0 + row_of<G>(ty, u);
    if (tx == 0 && i < r) ssq[((b * T + t) * nct + blockIdx.x) * r + i] = q;
  }
}

// the row-wise 2-norm of block (k, j): sqrt of its column tiles' sums of squares
template <typename R>
__device__ __forceinline__ R block_row_norm(const R* ssq, long long bt, int nct, int r, int i) {
  R q = R(0);
  for (int ct = 0; ct < nct; ++ct) q += ssq[(bt * nct + ct) * r + i];
  return sqrt(q);
}

// tau[b][k][i] = sum_{j=1..k} |row i of Phi^w_{k,j} E_{j-1}| + |row i of Phi^e_{k,j} F_{j-1}|,
// rows i < n from the x blocks, n <= i < n + m from the u blocks
template <typename R>
__global__ void sls_tube_sum_kernel(long long B, int N, int n, int m, int nxw, int nuw, int nxe, int nue,
                                    const R* sxw, const R* suw, const R* sxe, const R* sue, R* tau) {
  const long long T = (long long)(N + 1) * (N + 2) / 2, per = (long long)(N + 1) * (n + m);
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < B * per;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / per;
    const int k = (int)(e % per) / (n + m), i = (int)(e % per) % (n + m);
    R acc = R(0);
    for (int j = 1; j <= k; ++j) {
      const long long bt = b * T + tri_index(k, j);
      acc += i < n ? block_row_norm(sxw, bt, nxw, n, i) + block_row_norm(sxe, bt, nxe, n, i)
                   : block_row_norm(suw, bt, nuw, m, i - n) + block_row_norm(sue, bt, nue, m, i - n);
    }
    tau[e] = acc;
  }
}

// margin[b][k][i] = -b_i - c_i^T [z_k; v_k] - sum_{j=1..k} (|c_i^T Phi^w_{k,j} E_{j-1}| +
// |c_i^T Phi^e_{k,j} F_{j-1}|), k = 0..N-1; the c_i^T Phi products are the rows of the G blocks
template <typename R>
__global__ void sls_margin_kernel(long long B, int N, int n, int m, int nc, int ncw, int nce,
                                  const R* sgw, const R* sge, const R* Ccon, const R* bcon,
                                  const R* zn, const R* vn, R* margin) {
  const long long T = (long long)(N + 1) * (N + 2) / 2, per = (long long)N * nc;
  for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < B * per;
       e += (long long)gridDim.x * blockDim.x) {
    const long long b = e / per;
    const int k = (int)(e % per) / nc, i = (int)(e % per) % nc;
    const R* ci = Ccon + (size_t)i * (n + m);
    const R* zk = zn + (b * (N + 1) + k) * n;
    const R* vk = vn + (b * N + k) * m;
    R lin = R(0);
    for (int q = 0; q < n; ++q) lin = fma(ci[q], zk[q], lin);
    for (int q = 0; q < m; ++q) lin = fma(ci[n + q], vk[q], lin);
    R acc = R(0);
    for (int j = 1; j <= k; ++j) {
      const long long bt = b * T + tri_index(k, j);
      acc += block_row_norm(sgw, bt, ncw, nc, i) + block_row_norm(sge, bt, nce, nc, i);
    }
    margin[e] = -bcon[i] - lin - acc;
  }
}

// conformal radius: scores s_i = |q_next_i - f_pred_i|_2 (NaN read as +inf), sorted in shared
// memory by a bitonic network over np (a power of two) entries padded with +inf, then the
// kth-smallest (1-based, kth >= 1; past ncal: +inf)
template <typename R>
__global__ void __launch_bounds__(1024) sls_conformal_kernel(int ncal, int dim, int np, int kth,
                                                             const R* __restrict__ qn,
                                                             const R* __restrict__ fp, R* scores,
                                                             R* radius) {
  extern __shared__ __align__(16) unsigned char sls_smem[];
  R* sc = reinterpret_cast<R*>(sls_smem);
  const R inf = R(INFINITY);
  for (int i = threadIdx.x; i < np; i += blockDim.x) {
    R v = inf;
    if (i < ncal) {
      R q = R(0);
      for (int d = 0; d < dim; ++d) {
        const R x = qn[(size_t)i * dim + d] - fp[(size_t)i * dim + d];
        q = fma(x, x, q);
      }
      v = sqrt(q);
      if (scores) scores[i] = v;
      if (!(v == v)) v = inf;
    }
    sc[i] = v;
  }
  __syncthreads();
  for (int size = 2; size <= np; size <<= 1)
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < np; i += blockDim.x) {
        const int q = i ^ stride;
        if (q > i) {
          const R a = sc[i], c = sc[q];
          if ((a > c) == ((i & size) == 0)) {
            sc[i] = c;
            sc[q] = a;
          }
        }
      }
      __syncthreads();
    }
  if (threadIdx.x == 0) radius[0] = kth <= ncal ? sc[kth - 1] : inf;
}

// ---------------------------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------------------------

constexpr long long kMaxZ = 65535;

inline cs_status launched(const char* what) {
  cs_count_launch();
  cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CS_OK : cs_cuda_fail(e, what);
}

inline size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

template <class G>
inline dim3 tiles(int M, int N, long long z) {
  return dim3((unsigned)((N + G::BN - 1) / G::BN), (unsigned)((M + G::BM - 1) / G::BM), (unsigned)z);
}

// f(geometry) with the tile geometry for products of M rows in real type R
template <typename R, typename F>
cs_status with_geom(int M, F&& f) {
  if (M <= 16) return f(GShort{});
  if constexpr (sizeof(R) == 4) return f(GBig{});
  else return f(GMid{});
}

template <typename R, class G>
cs_status gemm_with(Gemm<R> g, long long batch, cudaStream_t st) {
  for (long long z0 = 0; z0 < batch; z0 += kMaxZ) {
    g.zoff = z0;
    sls_gemm_kernel<R, G><<<tiles<G>(g.M, g.N, std::min(kMaxZ, batch - z0)), NTH, 0, st>>>(g);
    cs_status r = launched("sls_gemm_kernel");
    if (r) return r;
  }
  return CS_OK;
}

template <typename R>
cs_status gemm(Gemm<R> g, long long batch, cudaStream_t st) {
  return with_geom<R>(g.M, [&](auto geo) -> cs_status { return gemm_with<R, decltype(geo)>(g, batch, st); });
}

template <typename R>
Prod<R> prod(const R* a, long long sa, int lda, int ta, const R* b, long long sb, int ldb, int tb, int K,
             R alpha = R(1)) {
  Prod<R> P;
  P.a = a; P.sa = sa; P.lda = lda; P.ta = ta; P.alpha = alpha;
  P.b = b; P.sb = sb; P.ldb = ldb; P.tb = tb; P.K = K;
  return P;
}

template <typename R>
Gemm<R> gemm_desc(int M, int N, R* c, long long sc, int ldc) {
  Gemm<R> g{};
  g.M = M; g.N = N; g.np = 0; g.c = c; g.sc = sc; g.ldc = ldc; g.d = nullptr; g.sd = 0; g.ldd = 0;
  return g;
}

// gain kernel: right-hand-side columns per pass that fit the shared-memory budget
inline int gain_cols(int n, int p, size_t rb) {
  const long long room = (long long)(kGainSmemBudget / rb) - (long long)p * p - p;
  long long cw = room > 0 ? room / p - 8 : 0;
  cw = std::min<long long>(std::min<long long>(cw, NTH / 4), n);
  return (int)std::max<long long>(cw, 0);
}

inline size_t gain_smem(int p, int cw, size_t rb) {
  return ((size_t)p * p + p + (size_t)p * (cw + 8)) * rb;
}

struct ObsWs {
  size_t t1, s, w, t2, abar, total;
};

inline ObsWs observer_ws(long long B, int N, int n, int p, size_t rb) {
  ObsWs o;
  size_t off = 0;
  o.t1 = off; off = align256(off + (size_t)B * n * p * rb);
  o.s = off; off = align256(off + (size_t)B * p * p * rb);
  o.w = off; off = align256(off + (size_t)B * n * p * rb);
  o.t2 = off; off = align256(off + (size_t)B * n * n * rb);
  o.abar = off; off = align256(off + (size_t)B * N * n * n * rb);
  o.total = off;
  return o;
}

template <typename R>
cs_status response_levels(int B, int N, int n, const R* Acl, R* Phi, cudaStream_t st) {
  {
    const long long total = (long long)B * (N + 1) * n * n;
    const int grid = (int)std::min<long long>((total + 255) / 256, 148LL * 16);
    sls_identity_kernel<R><<<grid, 256, 0, st>>>(B, N, n, Phi);
    cs_status r = launched("sls_identity_kernel");
    if (r) return r;
  }
  // doubling levels: distance 1 from Acl, then distances (2^(m-1), 2^m] from two earlier blocks:
  // ceil(log2 N) + 1 launches
  return with_geom<R>(n, [&](auto geo) -> cs_status {
    using G = decltype(geo);
    for (int lo = 1, hi = 1, h = 0; lo <= N; h = hi, lo = hi + 1, hi = std::min(2 * hi, N)) {
      long long items = 0;
      for (int d = lo; d <= hi; ++d) items += (long long)B * (N - d + 1);
      for (long long z0 = 0; z0 < items; z0 += kMaxZ) {
        sls_level_kernel<R, G><<<tiles<G>(n, n, std::min(kMaxZ, items - z0)), NTH, 0, st>>>(N, n, lo, hi, h,
                                                                                          Acl, Phi, z0);
        cs_status r = launched("sls_level_kernel");
        if (r) return r;
      }
    }
    return CS_OK;
  });
}

template <typename R>
cs_status observer(int B, int N, int n, int p, int nw, int ne, int n0, const R* A, const R* Cm,
                   const R* E, const R* F, const R* Xi, R* Pi, R* L, R* PX, R* PY, int32_t* status,
                   unsigned char* ws, cudaStream_t st) {
  const ObsWs o = observer_ws(B, N, n, p, sizeof(R));
  R* T1 = reinterpret_cast<R*>(ws + o.t1);
  R* S = reinterpret_cast<R*>(ws + o.s);
  R* W = reinterpret_cast<R*>(ws + o.w);
  R* T2 = reinterpret_cast<R*>(ws + o.t2);
  R* Abar = reinterpret_cast<R*>(ws + o.abar);
  const long long nn = (long long)n * n, np_ = (long long)n * p, sPi = (N + 1) * nn;
  cs_status r;
  if (status) {
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t) * (size_t)B, st);
    if (e != cudaSuccess) return cs_cuda_fail(e, "cudaMemsetAsync");
  }
  if (B == 0) return CS_OK;
  {  // Pi_0 = Xi Xi^T
    Gemm<R> g = gemm_desc<R>(n, n, Pi, sPi, n);
    g.pr[g.np++] = prod<R>(Xi, (long long)n * n0, n0, 0, Xi, (long long)n * n0, n0, 1, n0);
    if ((r = gemm(g, B, st))) return r;
  }
  const int cw = gain_cols(n, p, sizeof(R));
  const size_t gsm = gain_smem(p, cw, sizeof(R));
  {
    cudaError_t e = cudaFuncSetAttribute(sls_gain_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)gsm);
    if (e != cudaSuccess) return cs_cuda_fail(e, "cudaFuncSetAttribute");
  }
  for (int j = 0; j < N; ++j) {
    const R* Pj = Pi + j * nn;
    const R* Aj = A + j * nn;
    const R* Cj = Cm + (long long)j * p * n;
    const R* Ej = E + (long long)j * n * nw;
    const R* Fj = F + (long long)j * p * ne;
    const long long sA = N * nn, sC = (long long)N * p * n, sE = (long long)N * n * nw,
                    sF = (long long)N * p * ne;
    R* Lj = L + (long long)j * p * n;
    {  // T1 = Pi_j C_j^T (n x p)
      Gemm<R> g = gemm_desc<R>(n, p, T1, np_, p);
      g.pr[g.np++] = prod<R>(Pj, sPi, n, 0, Cj, sC, n, 1, n);
      if ((r = gemm(g, B, st))) return r;
    }
    {  // S = C_j T1 + F_j F_j^T (p x p)
      Gemm<R> g = gemm_desc<R>(p, p, S, (long long)p * p, p);
      g.pr[g.np++] = prod<R>(Cj, sC, n, 0, T1, np_, p, 0, n);
      g.pr[g.np++] = prod<R>(Fj, sF, ne, 0, Fj, sF, ne, 1, ne);
      if ((r = gemm(g, B, st))) return r;
    }
    {  // W = A_j T1 = A_j Pi_j C_j^T (n x p)
      Gemm<R> g = gemm_desc<R>(n, p, W, np_, p);
      g.pr[g.np++] = prod<R>(Aj, sA, n, 0, T1, np_, p, 0, n);
      if ((r = gemm(g, B, st))) return r;
    }
    {  // T2 = A_j Pi_j (n x n)
      Gemm<R> g = gemm_desc<R>(n, n, T2, nn, n);
      g.pr[g.np++] = prod<R>(Aj, sA, n, 0, Pj, sPi, n, 0, n);
      if ((r = gemm(g, B, st))) return r;
    }
    // L_{j+1} = -S^{-1} W^T (p x n)
    sls_gain_kernel<R><<<B, NTH, gsm, st>>>(p, n, cw, S, W, Lj, (long long)N * p * n, status);
    if ((r = launched("sls_gain_kernel"))) return r;
    {  // Pi_{j+1} = T2 A_j^T + E_j E_j^T + W L_{j+1}
      Gemm<R> g = gemm_desc<R>(n, n, Pi + (j + 1) * nn, sPi, n);
      g.pr[g.np++] = prod<R>(T2, nn, n, 0, Aj, sA, n, 1, n);
      g.pr[g.np++] = prod<R>(Ej, sE, nw, 0, Ej, sE, nw, 1, nw);
      g.pr[g.np++] = prod<R>(W, np_, p, 0, Lj, (long long)N * p * n, n, 0, p);
      if ((r = gemm(g, B, st))) return r;
    }
  }
  {  // Abar_j = A_j + L_{j+1}^T C_j for every (trajectory, step)
    Gemm<R> g = gemm_desc<R>(n, n, Abar, nn, n);
    g.pr[g.np++] = prod<R>(L, (long long)p * n, n, 1, Cm, (long long)p * n, n, 0, p);
    g.d = A; g.sd = nn; g.ldd = n;
    if ((r = gemm(g, (long long)B * N, st))) return r;
  }
  if ((r = response_levels<R>(B, N, n, Abar, PX, st))) return r;
  const long long T = (long long)(N + 1) * (N + 2) / 2, items = (long long)B * T;
  return with_geom<R>(n, [&](auto geo) -> cs_status {
    using G = decltype(geo);
    for (long long z0 = 0; z0 < items; z0 += kMaxZ) {
      sls_phiy_kernel<R, G><<<tiles<G>(n, p, std::min(kMaxZ, items - z0)), NTH, 0, st>>>(N, n, p, PX, L, PY,
                                                                                         z0);
      cs_status q = launched("sls_phiy_kernel");
      if (q) return q;
    }
    return CS_OK;
  });
}

template <typename R>
cs_status closed_loop(int B, int N, int n, int m, int p, const R* A, const R* PBX, const R* PBU,
                      const R* PX, const R* PY, R* XW, R* UW, R* XE, R* UE, unsigned char* ws,
                      cudaStream_t st) {
  const long long T = (long long)(N + 1) * (N + 2) / 2, items = (long long)B * T;
  R* MX = reinterpret_cast<R*>(ws);
  R* MY = reinterpret_cast<R*>(ws + align256((size_t)B * T * n * n * sizeof(R)));
  cs_status r;
  // (M Phihat^x) and (M Phihat^y)
  r = with_geom<R>(n, [&](auto geo) -> cs_status {
    using G = decltype(geo);
    for (long long z0 = 0; z0 < items; z0 += kMaxZ) {
      const long long zc = std::min(kMaxZ, items - z0);
      sls_shift_kernel<R, G><<<tiles<G>(n, n, zc), NTH, 0, st>>>(N, n, n, A, PX, MX, z0);
      cs_status q = launched("sls_shift_kernel");
      if (q) return q;
      sls_shift_kernel<R, G><<<tiles<G>(n, p, zc), NTH, 0, st>>>(N, n, p, A, PY, MY, z0);
      if ((q = launched("sls_shift_kernel"))) return q;
    }
    return CS_OK;
  });
  if (r) return r;
  // out = -(X (M Y)) + d1 + d2 over the blocks, X blocks rows x n
  auto tri = [&](int rows, int c, const R* X, const R* Y, const R* d1, const R* d2, R* out) {
    if (rows <= kThinRows) {
      constexpr int CW = sizeof(R) == 4 ? 128 : 64;
      for (long long z0 = 0; z0 < items; z0 += kMaxZ) {
        const dim3 grid((unsigned)((c + CW - 1) / CW), 1, (unsigned)std::min(kMaxZ, items - z0));
        sls_tri_thin_kernel<R><<<grid, NTH, 0, st>>>(N, rows, n, c, R(-1), X, Y, d1, d2, out, z0);
        cs_status q = launched("sls_tri_thin_kernel");
        if (q) return q;
      }
      return CS_OK;
    }
    return with_geom<R>(rows, [&](auto geo) -> cs_status {
      using G = decltype(geo);
      for (long long z0 = 0; z0 < items; z0 += kMaxZ) {
        const long long zc = std::min(kMaxZ, items - z0);
        sls_tri_kernel<R, G><<<tiles<G>(rows, c, zc), NTH, 0, st>>>(N, rows, n, c, R(-1), X, Y, d1, d2, out,
                                                                    z0);
        cs_status q = launched("sls_tri_kernel");
        if (q) return q;
      }
      return CS_OK;
    });
  };
  if ((r = tri(n, n, PBX, MX, PBX, PX, XW))) return r;         // Phi^xw
  if ((r = tri(m, n, PBU, MX, PBU, nullptr, UW))) return r;    // Phi^uw
  if ((r = tri(n, p, PBX, MY, PY, nullptr, XE))) return r;     // Phi^xe
  return tri(m, p, PBU, MY, nullptr, nullptr, UE);             // Phi^ue
}

// tile width (columns) of the row-norm products with `rows` rows
template <typename R>
inline int geom_bn(int rows) {
  return rows <= 16 ? GShort::BN : (sizeof(R) == 4 ? GBig::BN : GMid::BN);
}

struct TubeWs {
  int nxw, nuw, nxe, nue, ngw, nge;       // column tiles of each product
  size_t sxw, suw, sxe, sue, gw, ge, sgw, sge, total;
};

template <typename R>
TubeWs tube_ws(long long B, int N, int n, int m, int p, int nw, int ne, int nc) {
  const size_t T = (size_t)(N + 1) * (N + 2) / 2, rb = sizeof(R);
  TubeWs w;
  w.nxw = (nw + geom_bn<R>(n) - 1) / geom_bn<R>(n);
  w.nuw = (nw + geom_bn<R>(m) - 1) / geom_bn<R>(m);
  w.nxe = (ne + geom_bn<R>(n) - 1) / geom_bn<R>(n);
  w.nue = (ne + geom_bn<R>(m) - 1) / geom_bn<R>(m);
  w.ngw = nc > 0 ? (nw + geom_bn<R>(nc) - 1) / geom_bn<R>(nc) : 0;
  w.nge = nc > 0 ? (ne + geom_bn<R>(nc) - 1) / geom_bn<R>(nc) : 0;
  size_t off = 0;
  auto take = [&](size_t elems) { const size_t o = off; off = align256(off + elems * rb); return o; };
  w.sxw = take(B * T * w.nxw * n);
  w.suw = take(B * T * w.nuw * m);
  w.sxe = take(B * T * w.nxe * n);
  w.sue = take(B * T * w.nue * m);
  w.gw = take(B * T * (size_t)nc * n);
  w.ge = take(B * T * (size_t)nc * p);
  w.sgw = take(B * T * w.ngw * nc);
  w.sge = take(B * T * w.nge * nc);
  w.total = off;
  return w;
}

template <typename R>
cs_status rownorms(int B, int N, int r, int kd, int c, const R* X, const R* S, R* ssq, int nct,
                   cudaStream_t st) {
  const long long items = (long long)B * (N + 1) * (N + 2) / 2;
  return with_geom<R>(r, [&](auto geo) -> cs_status {
    using G = decltype(geo);
    for (long long z0 = 0; z0 < items; z0 += kMaxZ) {
      sls_rownorm_kernel<R, G><<<tiles<G>(r, c, std::min(kMaxZ, items - z0)), NTH, 0, st>>>(N, r, kd, c, X, S,
                                                                                          ssq, nct, z0);
      cs_status q = launched("sls_rownorm_kernel");
      if (q) return q;
    }
    return CS_OK;
  });
}

template <typename R>
cs_status tubes(int B, int N, int n, int m, int p, int nw, int ne, int nc, const R* XW, const R* UW,
                const R* XE, const R* UE, const R* E, const R* F, const R* Ccon, const R* bcon,
                const R* zn, const R* vn, R* tau, R* margin, unsigned char* ws, cudaStream_t st) {
  const TubeWs w = tube_ws<R>(B, N, n, m, p, nw, ne, nc);
  auto at = [&](size_t o) { return reinterpret_cast<R*>(ws + o); };
  cs_status r;
  if ((r = rownorms<R>(B, N, n, n, nw, XW, E, at(w.sxw), w.nxw, st))) return r;
  if ((r = rownorms<R>(B, N, m, n, nw, UW, E, at(w.suw), w.nuw, st))) return r;
  if ((r = rownorms<R>(B, N, n, p, ne, XE, F, at(w.sxe), w.nxe, st))) return r;
  if ((r = rownorms<R>(B, N, m, p, ne, UE, F, at(w.sue), w.nue, st))) return r;
  const long long T = (long long)(N + 1) * (N + 2) / 2;
  {
    const long long tot = (long long)B * (N + 1) * (n + m);
    const int grid = (int)std::min<long long>((tot + 255) / 256, 148LL * 16);
    sls_tube_sum_kernel<R><<<grid, 256, 0, st>>>(B, N, n, m, w.nxw, w.nuw, w.nxe, w.nue, at(w.sxw), at(w.suw),
                                                 at(w.sxe), at(w.sue), tau);
    if ((r = launched("sls_tube_sum_kernel"))) return r;
  }
  if (nc == 0) return CS_OK;
  // G^w = C_x Phi^xw + C_u Phi^uw (nc x n), G^e = C_x Phi^xe + C_u Phi^ue (nc x p), every block
  {
    Gemm<R> g = gemm_desc<R>(nc, n, at(w.gw), (long long)nc * n, n);
    g.pr[g.np++] = prod<R>(Ccon, 0, n + m, 0, XW, (long long)n * n, n, 0, n);
    g.pr[g.np++] = prod<R>(Ccon + n, 0, n + m, 0, UW, (long long)m * n, n, 0, m);
    if ((r = gemm(g, B * T, st))) return r;
  }
  {
    Gemm<R> g = gemm_desc<R>(nc, p, at(w.ge), (long long)nc * p, p);
    g.pr[g.np++] = prod<R>(Ccon, 0, n + m, 0, XE, (long long)n * p, p, 0, n);
    g.pr[g.np++] = prod<R>(Ccon + n, 0, n + m, 0, UE, (long long)m * p, p, 0, m);
    if ((r = gemm(g, B * T, st))) return r;
  }
  if ((r = rownorms<R>(B, N, nc, n, nw, at(w.gw), E, at(w.sgw), w.ngw, st))) return r;
  if ((r = rownorms<R>(B, N, nc, p, ne, at(w.ge), F, at(w.sge), w.nge, st))) return r;
  const long long tot = (long long)B * N * nc;
  const int grid = (int)std::min<long long>((tot + 255) / 256, 148LL * 16);
  sls_margin_kernel<R><<<grid, 256, 0, st>>>(B, N, n, m, nc, w.ngw, w.nge, at(w.sgw), at(w.sge), Ccon, bcon,
                                             zn, vn, margin);
  return launched("sls_margin_kernel");
}

struct ScanWs {
  size_t xa, xd, xp, ya, yd, yp, m, r2, sa, sd, t, ct, rm, lp, fl, total;
};

template <typename R>
ScanWs scan_ws(long long B, int N, int n, int p) {
  ScanWs w;
  size_t off = 0;
  auto take = [&](size_t elems) { const size_t o = off; off = align256(off + elems * sizeof(R)); return o; };
  const size_t E = (size_t)B * (N + 1) * n * n;
  w.xa = take(E); w.xd = take(E); w.xp = take(E);
  w.ya = take(E); w.yd = take(E); w.yp = take(E);
  w.m = take(E); w.r2 = take(E); w.sa = take(E); w.sd = take(E); w.t = take(E);
  w.ct = take((size_t)N * B * n * p);
  w.rm = take((size_t)N * B * p * p);
  w.lp = take((size_t)N * B * p * n);
  w.fl = take((size_t)N * B);                       // int32 flags of the (trajectory, step) solves
  w.total = off;
  return w;
}

// LU solve: right-hand-side columns per pass within the shared-memory budget
inline int lu_cols(int n, size_t rb) {
  const long long room = (long long)(kGainSmemBudget / rb) - (long long)n * n - n;
  long long cw = room > 0 ? room / n - 8 : 0;
  cw = std::min<long long>(std::min<long long>(cw, NTH / 4), 2LL * n);
  return (int)std::max<long long>(cw, 0);
}

inline size_t lu_smem(int n, int cw, size_t rb) {
  return ((size_t)n * n + (size_t)n * (cw + 8)) * rb + (size_t)n * sizeof(int);
}

template <typename R>
cs_status kalman_scan(int B, int N, int n, int p, int nw, int ne, int n0, const R* A, const R* Cm, const R* E,
                      const R* F, const R* Xi, R* Pi, int32_t* status, unsigned char* ws, cudaStream_t st) {
  const ScanWs w = scan_ws<R>(B, N, n, p);
  auto at = [&](size_t o) { return reinterpret_cast<R*>(ws + o); };
  R *XA = at(w.xa), *XD = at(w.xd), *XP = at(w.xp), *YA = at(w.ya), *YD = at(w.yd), *YP = at(w.yp);
  const long long nn = (long long)n * n, sE = (long long)(N + 1) * nn;
  cs_status r;
  if (status) {
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t) * (size_t)B, st);
    if (e != cudaSuccess) return cs_cuda_fail(e, "cudaMemsetAsync");
  }
  if (B == 0) return CS_OK;
  const int gcw = gain_cols(n, p, sizeof(R)), lcw = lu_cols(n, sizeof(R));
  const size_t gsm = gain_smem(p, gcw, sizeof(R)), lsm = lu_smem(n, lcw, sizeof(R));
  cudaError_t e = cudaFuncSetAttribute(sls_gain_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gsm);
  if (e != cudaSuccess) return cs_cuda_fail(e, "cudaFuncSetAttribute");
  e = cudaFuncSetAttribute(sls_lu_solve_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)lsm);
  if (e != cudaSuccess) return cs_cuda_fail(e, "cudaFuncSetAttribute");
  // elements: the prior (0, 0, Xi Xi^T), step j (A_j^T, C_j^T (F_j F_j^T)^{-1} C_j, E_j E_j^T)
  sls_scan_build_kernel<R><<<148 * 8, 256, 0, st>>>(B, N, n, p, A, Cm, XA, XD, at(w.ct));
  if ((r = launched("sls_scan_build_kernel"))) return r;
  {
    Gemm<R> g = gemm_desc<R>(n, n, XP, sE, n);
    g.pr[g.np++] = prod<R>(Xi, (long long)n * n0, n0, 0, Xi, (long long)n * n0, n0, 1, n0);
    if ((r = gemm(g, B, st))) return r;
  }
  // the step elements of all (trajectory, step) at once, then placed after each prior: E E^T into
  // the M slots, F F^T, the gain solve Lp = -(F F^T)^{-1} C, Dtil = C^T (F F^T)^{-1} C = -C^T Lp into
  // the R2 slots
  const long long BN = (long long)B * N;
  {
    Gemm<R> g = gemm_desc<R>(n, n, at(w.m), nn, n);
    g.pr[g.np++] = prod<R>(E, (long long)n * nw, nw, 0, E, (long long)n * nw, nw, 1, nw);
    if ((r = gemm(g, BN, st))) return r;
  }
  {
    Gemm<R> g = gemm_desc<R>(p, p, at(w.rm), (long long)p * p, p);
    g.pr[g.np++] = prod<R>(F, (long long)p * ne, ne, 0, F, (long long)p * ne, ne, 1, ne);
    if ((r = gemm(g, BN, st))) return r;
  }
  int32_t* fl = reinterpret_cast<int32_t*>(ws + w.fl);
  if ((e = cudaMemsetAsync(fl, 0, sizeof(int32_t) * (size_t)BN, st)) != cudaSuccess)
    return cs_cuda_fail(e, "cudaMemsetAsync");
  for (long long z0 = 0; z0 < BN; z0 += kMaxZ) {
    const long long zc = std::min(kMaxZ, BN - z0);
    sls_gain_kernel<R><<<(unsigned)zc, NTH, gsm, st>>>(p, n, gcw, at(w.rm) + z0 * p * p, at(w.ct) + z0 * n * p,
                                                       at(w.lp) + z0 * p * n, (long long)p * n, fl + z0);
    if ((r = launched("sls_gain_kernel"))) return r;
  }
  if (status) {
    sls_flag_rows_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, N, fl, status);
    if ((r = launched("sls_flag_rows_kernel"))) return r;
  }
  {
    Gemm<R> g = gemm_desc<R>(n, n, at(w.r2), nn, n);
    g.pr[g.np++] = prod<R>(Cm, (long long)p * n, n, 1, at(w.lp), (long long)p * n, n, 0, p, R(-1));
    if ((r = gemm(g, BN, st))) return r;
  }
  sls_scan_place_kernel<R><<<148 * 8, 256, 0, st>>>(B, N, n, at(w.r2), at(w.m), XD, XP);
  if ((r = launched("sls_scan_place_kernel"))) return r;
  // levels: x_i <- x_i (x) x_{i-d} for i >= d (the later step on the left), d = 1, 2, 4, ...
  for (int d = 1; d <= N; d <<= 1) {
    const long long Z = (long long)B * (N + 1) - d, off = (long long)d * nn;
    {  // M = D1 P2
      Gemm<R> g = gemm_desc<R>(n, n, at(w.m), nn, n);
      g.pr[g.np++] = prod<R>(XD + off, nn, n, 0, XP, nn, n, 0, n);
      if ((r = gemm(g, Z, st))) return r;
    }
    {  // R2 = D1 A2^T
      Gemm<R> g = gemm_desc<R>(n, n, at(w.r2), nn, n);
      g.pr[g.np++] = prod<R>(XD + off, nn, n, 0, XA, nn, n, 1, n);
      if ((r = gemm(g, Z, st))) return r;
    }
    for (long long z0 = 0; z0 < Z; z0 += kMaxZ) {  // [Xa | Xd] = (I + D1 P2)^{-1} [A1 | D1 A2^T]
      sls_lu_solve_kernel<R><<<(unsigned)std::min(kMaxZ, Z - z0), NTH, lsm, st>>>(
          n, lcw, at(w.m), XA + off, at(w.r2), at(w.sa), at(w.sd), status, N + 1, d, z0);
      if ((r = launched("sls_lu_solve_kernel"))) return r;
    }
    {  // T = P2 Xa
      Gemm<R> g = gemm_desc<R>(n, n, at(w.t), nn, n);
      g.pr[g.np++] = prod<R>(XP, nn, n, 0, at(w.sa), nn, n, 0, n);
      if ((r = gemm(g, Z, st))) return r;
    }
    {  // Ptil = A1^T T + P1
      Gemm<R> g = gemm_desc<R>(n, n, YP + off, nn, n);
      g.pr[g.np++] = prod<R>(XA + off, nn, n, 1, at(w.t), nn, n, 0, n);
      g.d = XP + off; g.sd = nn; g.ldd = n;
      if ((r = gemm(g, Z, st))) return r;
    }
    {  // Atil = A2 Xa
      Gemm<R> g = gemm_desc<R>(n, n, YA + off, nn, n);
      g.pr[g.np++] = prod<R>(XA, nn, n, 0, at(w.sa), nn, n, 0, n);
      if ((r = gemm(g, Z, st))) return r;
    }
    {  // Dtil = A2 Xd + D2
      Gemm<R> g = gemm_desc<R>(n, n, YD + off, nn, n);
      g.pr[g.np++] = prod<R>(XA, nn, n, 0, at(w.sd), nn, n, 0, n);
      g.d = XD; g.sd = nn; g.ldd = n;
      if ((r = gemm(g, Z, st))) return r;
    }
    sls_scan_keep_kernel<R><<<148 * 8, 256, 0, st>>>(B, N, n, d, XA, XD, XP, YA, YD, YP);
    if ((r = launched("sls_scan_keep_kernel"))) return r;
    std::swap(XA, YA);
    std::swap(XD, YD);
    std::swap(XP, YP);
  }
  e = cudaMemcpyAsync(Pi, XP, sizeof(R) * (size_t)B * sE, cudaMemcpyDeviceToDevice, st);
  return e == cudaSuccess ? CS_OK : cs_cuda_fail(e, "cudaMemcpyAsync");
}

constexpr int kConformalMax = 8192;   // calibration samples one shared-memory sort holds (64 KB in FP64)

cs_status check_sizes(int B, int N, int n, int real_bytes) {
  if (B < 0) return cs_fail(CS_ERR_INVALID_ARG, "B must be >= 0");
  if (N < 1 || n < 1) return cs_fail(CS_ERR_INVALID_ARG, "N and n must be >= 1");
  if (real_bytes != 4 && real_bytes != 8) return cs_fail(CS_ERR_INVALID_ARG, "real_bytes must be 4 or 8");
  if (N > 4096 || n > 4096) return cs_fail(CS_ERR_INVALID_ARG, "N and n must be <= 4096");
  return CS_OK;
}

}  // namespace

extern "C" {

size_t sls_observer_workspace(int B, int N, int n, int p, int real_bytes) {
  if (B < 0 || N < 1 || n < 1 || p < 1 || (real_bytes != 4 && real_bytes != 8)) return 0;
  return observer_ws(B, N, n, p, (size_t)real_bytes).total;
}

cs_status sls_observer(int B, int N, int n, int p, int nw, int ne, int n0, int real_bytes, const void* A,
                       const void* C, const void* E, const void* F, const void* Xi, void* Pi, void* L,
                       void* PhiX, void* PhiY, int32_t* status, void* workspace, size_t workspace_bytes,
                       void* stream) {
  cs_status r = check_sizes(B, N, n, real_bytes);
  if (r) return r;
  if (p < 1 || nw < 1 || ne < 1 || n0 < 1 || p > 4096 || nw > 4096 || ne > 4096 || n0 > 4096)
    return cs_fail(CS_ERR_INVALID_ARG, "p, nw, ne and n0 must be in [1, 4096]");
  if (gain_cols(n, p, (size_t)real_bytes) < 1)
    return cs_fail(CS_ERR_INVALID_ARG, "p too large for the gain kernel's shared memory");
  if (B > 0 && (!A || !C || !E || !F || !Xi || !Pi || !L || !PhiX || !PhiY || !workspace))
    return cs_fail(CS_ERR_INVALID_ARG, "null pointer");
  if (workspace_bytes < sls_observer_workspace(B, N, n, p, real_bytes))
    return cs_fail(CS_ERR_INVALID_ARG, "workspace smaller than sls_observer_workspace()");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* ws = (unsigned char*)workspace;
  if (real_bytes == 4)
    return observer<float>(B, N, n, p, nw, ne, n0, (const float*)A, (const float*)C, (const float*)E,
                           (const float*)F, (const float*)Xi, (float*)Pi, (float*)L, (float*)PhiX,
                           (float*)PhiY, status, ws, st);
  return observer<double>(B, N, n, p, nw, ne, n0, (const double*)A, (const double*)C, (const double*)E,
                          (const double*)F, (const double*)Xi, (double*)Pi, (double*)L, (double*)PhiX,
                          (double*)PhiY, status, ws, st);
}

cs_status sls_response(int B, int N, int n, int real_bytes, const void* Acl, void* Phi, void* stream) {
  cs_status r = check_sizes(B, N, n, real_bytes);
  if (r) return r;
  if (B > 0 && (!Acl || !Phi)) return cs_fail(CS_ERR_INVALID_ARG, "null pointer");
  if (B == 0) return CS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  if (real_bytes == 4) return response_levels<float>(B, N, n, (const float*)Acl, (float*)Phi, st);
  return response_levels<double>(B, N, n, (const double*)Acl, (double*)Phi, st);
}

size_t sls_closed_loop_workspace(int B, int N, int n, int p, int real_bytes) {
  if (B < 0 || N < 1 || n < 1 || p < 1 || (real_bytes != 4 && real_bytes != 8)) return 0;
  const size_t T = (size_t)(N + 1) * (N + 2) / 2;
  return align256((size_t)B * T * n * n * real_bytes) + align256((size_t)B * T * n * p * real_bytes);
}

cs_status sls_closed_loop(int B, int N, int n, int m, int p, int real_bytes, const void* A,
                          const void* PhiBarX, const void* PhiBarU, const void* PhiX, const void* PhiY,
                          void* PhiXW, void* PhiUW, void* PhiXE, void* PhiUE, void* workspace,
                          size_t workspace_bytes, void* stream) {
  cs_status r = check_sizes(B, N, n, real_bytes);
  if (r) return r;
  if (m < 1 || p < 1 || m > 4096 || p > 4096) return cs_fail(CS_ERR_INVALID_ARG, "m and p must be in [1, 4096]");
  if (B > 0 && (!A || !PhiBarX || !PhiBarU || !PhiX || !PhiY || !PhiXW || !PhiUW || !PhiXE || !PhiUE ||
                !workspace))
    return cs_fail(CS_ERR_INVALID_ARG, "null pointer");
  if (workspace_bytes < sls_closed_loop_workspace(B, N, n, p, real_bytes))
    return cs_fail(CS_ERR_INVALID_ARG, "workspace smaller than sls_closed_loop_workspace()");
  if (B == 0) return CS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* ws = (unsigned char*)workspace;
  if (real_bytes == 4)
    return closed_loop<float>(B, N, n, m, p, (const float*)A, (const float*)PhiBarX, (const float*)PhiBarU,
                              (const float*)PhiX, (const float*)PhiY, (float*)PhiXW, (float*)PhiUW,
                              (float*)PhiXE, (float*)PhiUE, ws, st);
  return closed_loop<double>(B, N, n, m, p, (const double*)A, (const double*)PhiBarX,
                             (const double*)PhiBarU, (const double*)PhiX, (const double*)PhiY,
                             (double*)PhiXW, (double*)PhiUW, (double*)PhiXE, (double*)PhiUE, ws, st);
}

size_t sls_tubes_workspace(int B, int N, int n, int m, int p, int nw, int ne, int nc, int real_bytes) {
  if (B < 0 || N < 1 || n < 1 || m < 1 || p < 1 || nw < 1 || ne < 1 || nc < 0 ||
      (real_bytes != 4 && real_bytes != 8))
    return 0;
  return real_bytes == 4 ? tube_ws<float>(B, N, n, m, p, nw, ne, nc).total
                         : tube_ws<double>(B, N, n, m, p, nw, ne, nc).total;
}

cs_status sls_tubes(int B, int N, int n, int m, int p, int nw, int ne, int nc, int real_bytes,
                    const void* PhiXW, const void* PhiUW, const void* PhiXE, const void* PhiUE,
                    const void* E, const void* F, const void* Ccon, const void* bcon, const void* z,
                    const void* v, void* tau, void* margin, void* workspace, size_t workspace_bytes,
                    void* stream) {
  cs_status r = check_sizes(B, N, n, real_bytes);
  if (r) return r;
  if (m < 1 || p < 1 || nw < 1 || ne < 1 || nc < 0 || m > 4096 || p > 4096 || nw > 4096 || ne > 4096 ||
      nc > 4096)
    return cs_fail(CS_ERR_INVALID_ARG, "m, p, nw, ne must be in [1, 4096] and nc in [0, 4096]");
  if (B > 0 && (!PhiXW || !PhiUW || !PhiXE || !PhiUE || !E || !F || !tau || !workspace))
    return cs_fail(CS_ERR_INVALID_ARG, "null pointer");
  if (B > 0 && nc > 0 && (!Ccon || !bcon || !z || !v || !margin))
    return cs_fail(CS_ERR_INVALID_ARG, "null constraint pointer with nc > 0");
  if (workspace_bytes < sls_tubes_workspace(B, N, n, m, p, nw, ne, nc, real_bytes))
    return cs_fail(CS_ERR_INVALID_ARG, "workspace smaller than sls_tubes_workspace()");
  if (B == 0) return CS_OK;
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* ws = (unsigned char*)workspace;
  if (real_bytes == 4)
    return tubes<float>(B, N, n, m, p, nw, ne, nc, (const float*)PhiXW, (const float*)PhiUW,
                        (const float*)PhiXE, (const float*)PhiUE, (const float*)E, (const float*)F,
                        (const float*)Ccon, (const float*)bcon, (const float*)z, (const float*)v,
                        (float*)tau, (float*)margin, ws, st);
  return tubes<double>(B, N, n, m, p, nw, ne, nc, (const double*)PhiXW, (const double*)PhiUW,
                       (const double*)PhiXE, (const double*)PhiUE, (const double*)E, (const double*)F,
                       (const double*)Ccon, (const double*)bcon, (const double*)z, (const double*)v,
                       (double*)tau, (double*)margin, ws, st);
}

cs_status sls_conformal_radius(int n_cal, int dim, int real_bytes, const void* q_next, const void* f_pred,
                               double delta, int T, void* scores, void* radius, void* stream) {
  if (n_cal < 1 || n_cal > kConformalMax || dim < 1 || dim > (1 << 20))
    return cs_fail(CS_ERR_INVALID_ARG, "n_cal must be in [1, 8192] and dim in [1, 2^20]");
  if (real_bytes != 4 && real_bytes != 8) return cs_fail(CS_ERR_INVALID_ARG, "real_bytes must be 4 or 8");
  if (!(delta > 0.0 && delta < 1.0) || T < 1)
    return cs_fail(CS_ERR_INVALID_ARG, "delta must be in (0, 1) and T >= 1");
  if (!q_next || !f_pred || !radius) return cs_fail(CS_ERR_INVALID_ARG, "null pointer");
  long long kth = (long long)std::ceil((n_cal + 1.0) * (1.0 - delta / T));
  kth = std::max<long long>(kth, 1);
  const int k = (int)std::min<long long>(kth, (long long)n_cal + 1);
  int np = 1;
  while (np < n_cal) np <<= 1;
  const size_t smem = (size_t)np * real_bytes;
  cudaStream_t st = (cudaStream_t)stream;
  if (real_bytes == 4) {
    cudaError_t e = cudaFuncSetAttribute(sls_conformal_kernel<float>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cs_cuda_fail(e, "cudaFuncSetAttribute");
    sls_conformal_kernel<float><<<1, 1024, smem, st>>>(n_cal, dim, np, k, (const float*)q_next,
                                                       (const float*)f_pred, (float*)scores, (float*)radius);
  } else {
    cudaError_t e = cudaFuncSetAttribute(sls_conformal_kernel<double>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return cs_cuda_fail(e, "cudaFuncSetAttribute");
    sls_conformal_kernel<double><<<1, 1024, smem, st>>>(n_cal, dim, np, k, (const double*)q_next,
                                                        (const double*)f_pred, (double*)scores, (double*)radius);
  }
  return launched("sls_conformal_kernel");
}

size_t sls_kalman_scan_workspace(int B, int N, int n, int p, int real_bytes) {
  if (B < 0 || N < 1 || n < 1 || p < 1 || (real_bytes != 4 && real_bytes != 8)) return 0;
  return real_bytes == 4 ? scan_ws<float>(B, N, n, p).total : scan_ws<double>(B, N, n, p).total;
}

cs_status sls_kalman_scan(int B, int N, int n, int p, int nw, int ne, int n0, int real_bytes, const void* A,
                          const void* C, const void* E, const void* F, const void* Xi, void* Pi, int32_t* status,
                          void* workspace, size_t workspace_bytes, void* stream) {
  cs_status r = check_sizes(B, N, n, real_bytes);
  if (r) return r;
  if (p < 1 || nw < 1 || ne < 1 || n0 < 1 || p > 4096 || nw > 4096 || ne > 4096 || n0 > 4096)
    return cs_fail(CS_ERR_INVALID_ARG, "p, nw, ne and n0 must be in [1, 4096]");
  if (gain_cols(n, p, (size_t)real_bytes) < 1)
    return cs_fail(CS_ERR_INVALID_ARG, "p too large for the gain kernel's shared memory");
  if (lu_cols(n, (size_t)real_bytes) < 1)
    return cs_fail(CS_ERR_INVALID_ARG, "n too large for the scan's shared-memory LU");
  if (B > 0 && (!A || !C || !E || !F || !Xi || !Pi || !workspace))
    return cs_fail(CS_ERR_INVALID_ARG, "null pointer");
  if (workspace_bytes < sls_kalman_scan_workspace(B, N, n, p, real_bytes))
    return cs_fail(CS_ERR_INVALID_ARG, "workspace smaller than sls_kalman_scan_workspace()");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* ws = (unsigned char*)workspace;
  if (real_bytes == 4)
    return kalman_scan<float>(B, N, n, p, nw, ne, n0, (const float*)A, (const float*)C, (const float*)E,
                              (const float*)F, (const float*)Xi, (float*)Pi, status, ws, st);
  return kalman_scan<double>(B, N, n, p, nw, ne, n0, (const double*)A, (const double*)C, (const double*)E,
                             (const double*)F, (const double*)Xi, (double*)Pi, status, ws, st);
}

}  // extern "C"
