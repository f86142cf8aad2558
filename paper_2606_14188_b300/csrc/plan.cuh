// Device side of the served plan solve: a packed forward + adjoint launch over the candidate
// rollouts of many requests at once, and the per-request optimiser kernels (candidate
// initialisation from counter-based normals, best-candidate selection, Adam step).
//
// Planner (the paper optimises nominal control sequences by gradients of the simulator, Sec. 4.2
// and Sec. 5, without printing the optimiser): R candidates u^(0) = clip(w), u^(r) = clip(w +
// sigma eps^(r)); G evaluations, each a batched rollout + adjoint of every candidate; after
// evaluations 1..G-1 a bias-corrected Adam step (Kingma & Ba 2015) and the box clip on every
// candidate whose rollout succeeded; result = the evaluated candidate with the lowest loss over
// all evaluations (ties: earlier evaluation, then lower r).
#pragma once
#include "rope.cuh"

namespace cs {

// optimiser state of one request (device memory)
struct PlanState {
  double best_L;   // lowest evaluated loss so far (+inf before the first evaluation)
  int it;          // number of the next evaluation (1-based)
  int it_cur;      // evaluation the optimiser step of this tick belongs to
  int best_it, best_r;
  int flags;       // OR of the candidates' status bits at the last evaluation
  int n_ok;        // candidates that succeeded at the last evaluation
};

// one request as the kernels see it (an array of these lives in device memory; 16-byte aligned so
// that the array's stride, sizeof(PlanJob), is also the host table's stride)
template <typename R>
struct alignas(16) PlanJob {
  Scene<R> S;            // scene and planning loss; S.L1/S.L2 point at the request's rest lengths
  const R* q0;           // [n_q]
  const R* warm;         // [warm_H][6] or null (zeros)
  R* U;                  // [Rc][H][6] candidates
  R* M;                  // [Rc][H][6] Adam first moments
  R* V;                  // [Rc][H][6] Adam second moments
  R* dU;                 // [Rc][H][6] gradients of the last evaluation
  R* L;                  // [Rc] losses of the last evaluation
  int32_t* status;       // [Rc]
  R* ws;                 // [Rc][ws_stride] checkpoint records
  R* best_u;             // [H][6]
  PlanState* st;
  size_t ws_stride;
  unsigned long long seed;
  int H, Rc, G, warm_H, warm_shift;
  int cloth_wg;          // cloth: its band window lives in global memory (too wide for shared)
  R lr, sigma, u_max;
};

template <typename R>
__host__ __device__ constexpr size_t plan_scene_bytes() {
  return (sizeof(Scene<R>) + 15) & ~(size_t)15;
}

// ---- Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC 2011): 10 rounds of two 32x32->64-bit
//      multiplications on a 4-word counter, the 2-word key bumped by Weyl constants between rounds
__device__ __forceinline__ uint4 philox4x32_10(uint4 c, uint2 k) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const unsigned lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const unsigned lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k.x, lo1, hi0 ^ c.w ^ k.y, lo0);
  }
  return c;
}

__device__ __forceinline__ void sin_cos_pi(float x, float* s, float* c) { sincospif(x, s, c); }
__device__ __forceinline__ void sin_cos_pi(double x, double* s, double* c) { sincospi(x, s, c); }

// standard normal eps^(r)[e], e = 6 t + d: counter (e >> 1, r, 0, 0), key = the seed's two
// 32-bit halves; Box-Muller on the first two output words, first (even e) or second (odd e)
template <typename R>
__device__ __forceinline__ R philox_normal(unsigned long long seed, int r, int e) {
  const uint4 x = philox4x32_10(make_uint4((unsigned)(e >> 1), (unsigned)r, 0u, 0u),
                                make_uint2((unsigned)(seed & 0xFFFFFFFFull), (unsigned)(seed >> 32)));
  const R two32inv = R(1) / R(4294967296.0);
  const R u1 = (R(x.x) + R(1)) * two32inv;
  const R u2 = R(x.y) * two32inv;
  const R rad = sqrt(R(-2) * log(u1));
  R sn, cs;
  sin_cos_pi(R(2) * u2, &sn, &cs);
  return rad * ((e & 1) ? sn : cs);
}

// ---- packed forward + adjoint: item g of [0, total) is candidate g - first[j] of job j
//      (first[] ascending, first[0] = 0); W = blockDim.x / 32 warps per CTA, one item per warp
//      at a time; each warp copies its job's scene into its own shared-memory slice.
template <typename R, int PPL>
__global__ void __launch_bounds__(128) rope_vjp_packed_kernel(const PlanJob<R>* jobs, const int* first,
                                                              int njobs, int total, size_t warp_smem) {
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, W = blockDim.x >> 5;
  unsigned char* mine = cs_smem + (size_t)wid * warp_smem;
  Scene<R>* Ssm = reinterpret_cast<Scene<R>*>(mine);
  R* wsb = reinterpret_cast<R*>(mine + plan_scene_bytes<R>());
  for (int g = blockIdx.x * W + wid; g < total; g += gridDim.x * W) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (first[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const PlanJob<R>* J = jobs + lo;
    const int r = g - first[lo];
    const int* src = reinterpret_cast<const int*>(&J->S);
    int* dst = reinterpret_cast<int*>(Ssm);
    for (int i = lane; i < (int)(sizeof(Scene<R>) / sizeof(int)); i += 32) dst[i] = src[i];
    __syncwarp();
    const Scene<R>& S = *Ssm;
    const int H = J->H;
    WS<R> w = ws_carve<R>(wsb, 32 * PPL, S.nobs, H, false);
    Lane<R, PPL> L;
    zero_lane(L);
    load_rest(S, L, lane);
    vjp_rollout<R, PPL>(S, w, L, lane, H, J->q0, J->U + (size_t)r * H * 6, nullptr, J->L + r,
                        J->dU + (size_t)r * H * 6, nullptr, J->status + r, J->ws + (size_t)r * J->ws_stride);
    __syncwarp();
  }
}

// ---- candidates of newly admitted jobs j0 .. j0 + gridDim.y - 1
template <typename R>
__global__ void plan_init_kernel(const PlanJob<R>* jobs, int j0) {
  const PlanJob<R>& J = jobs[j0 + blockIdx.y];
  const int per = J.H * 6;
  const int n = J.Rc * per;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    const int r = e / per, te = e - r * per, t = te / 6, d = te - 6 * t;
    R base = R(0);
    if (J.warm) {
      const int ts = min(t + J.warm_shift, J.warm_H - 1);
      base = J.warm[ts * 6 + d];
    }
    const R u = base + (r > 0 ? J.sigma * philox_normal<R>(J.seed, r, te) : R(0));
    J.U[e] = fmin(fmax(u, -J.u_max), J.u_max);
    J.M[e] = R(0);
    J.V[e] = R(0);
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    PlanState* ps = J.st;
    ps->best_L = __longlong_as_double(0x7FF0000000000000ll);   // +inf
    ps->it = 1;
    ps->it_cur = 0;
    ps->best_it = -1;
    ps->best_r = -1;
    ps->flags = 0;
    ps->n_ok = 0;
  }
}

// ---- after an evaluation: best candidate of this evaluation (lowest loss among the rollouts that
//      succeeded, lowest r on ties) against the best so far; one CTA per job
template <typename R>
__global__ void __launch_bounds__(256) plan_select_kernel(const PlanJob<R>* jobs) {
  const PlanJob<R>& J = jobs[blockIdx.x];
  PlanState* ps = J.st;
  double bv = __longlong_as_double(0x7FF0000000000000ll);
  int br = 0x7FFFFFFF, fl = 0, nok = 0;
  for (int r = threadIdx.x; r < J.Rc; r += blockDim.x) {
    const int32_t s = J.status[r];
    fl |= s;
    if (s == 0) {
      ++nok;
      const double v = (double)J.L[r];
      if (v < bv || (v == bv && r < br)) { bv = v; br = r; }
    }
  }
  // warp, then block reduction of (bv, br), flags, counts
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    const double v2 = __shfl_xor_sync(FULL, bv, o);
    const int r2 = __shfl_xor_sync(FULL, br, o);
    if (v2 < bv || (v2 == bv && r2 < br)) { bv = v2; br = r2; }
    fl |= __shfl_xor_sync(FULL, fl, o);
    nok += __shfl_xor_sync(FULL, nok, o);
  }
  __shared__ double sv[8];
  __shared__ int sr[8], sf[8], sn[8];
  __shared__ int improved, sel;
  const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (lane == 0) { sv[wid] = bv; sr[wid] = br; sf[wid] = fl; sn[wid] = nok; }
  __syncthreads();
  if (threadIdx.x == 0) {
    const int nw = blockDim.x >> 5;
    for (int i = 1; i < nw; ++i) {
      if (sv[i] < bv || (sv[i] == bv && sr[i] < br)) { bv = sv[i]; br = sr[i]; }
      fl |= sf[i];
      nok += sn[i];
    }
    const int it = ps->it;
    improved = 0;
    if (nok > 0 && bv < ps->best_L) {
      ps->best_L = bv;
      ps->best_it = it;
      ps->best_r = br;
      improved = 1;
    }
    ps->flags = fl;
    ps->n_ok = nok;
    ps->it_cur = it;
    ps->it = it + 1;
    sel = br;
  }
  __syncthreads();
  if (improved) {
    const int per = J.H * 6;
    for (int e = threadIdx.x; e < per; e += blockDim.x) J.best_u[e] = J.U[(size_t)sel * per + e];
  }
}

// ---- Adam step (bias-corrected, evaluation count it_cur) and box clip of every candidate whose
//      rollout succeeded; nothing after the last evaluation.  grid.y = job
template <typename R>
__global__ void plan_adam_kernel(const PlanJob<R>* jobs) {
  const PlanJob<R>& J = jobs[blockIdx.y];
  const int it = J.st->it_cur;
  if (it >= J.G) return;
  const R b1 = R(0.9), b2 = R(0.999), eps = R(1e-8);
  const R c1 = R(1) - pow(b1, R(it)), c2 = R(1) - pow(b2, R(it));
  const int per = J.H * 6;
  const int n = J.Rc * per;
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) {
    if (J.status[e / per] != 0) continue;
    const R g = J.dU[e];
    const R m = b1 * J.M[e] + (R(1) - b1) * g;
    const R v = b2 * J.V[e] + (R(1) - b2) * g * g;
    J.M[e] = m;
    J.V[e] = v;
    const R u = J.U[e] - J.lr * (m / c1) / (sqrt(v / c2) + eps);
    J.U[e] = fmin(fmax(u, -J.u_max), J.u_max);
  }
}

}  // namespace cs
