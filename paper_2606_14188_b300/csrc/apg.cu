// Analytic policy gradient (arxiv 2606.14188, Sec. 4.3): a policy u = pi_theta(q) in the loop of
// the batched rollout and its gradient dL/dtheta through the simulator (eq. diff-sim).
//
// The policy is one tanh hidden layer shared by the rollouts, u = W2 tanh(W1 q + b1) + b2,
// theta = (W1 [h][n_q], b1 [h], W2 [6][h], b2 [6]).  The call runs
//   forward  for t = 0..H-1: apg_policy_fwd_kernel (u_t and the hidden activations of every
//            rollout, one CTA each), then one step of the nonsmooth model for all rollouts
//            (sim_rollout with H = 1);
//   backward for t = H-1..0: the step's adjoint for all rollouts (sim_rollout_vjp with H = 1,
//            seeded with lambda_{t+1} on q_{t+1}; its loss is the planning loss's terms of
//            q_{t+1}: the obstacle penalty, the goal at the last step), then
//            apg_policy_bwd_kernel: g = dL/du_t + 2 w_u u_t, lambda_t = dL/dq_t + dpi/dq^T g,
//            each rollout's dL/dtheta += dpi/dtheta^T g;
//   reduce   apg_reduce_kernel: dL/dtheta summed over the rollouts that completed (fixed order),
//            L per rollout (NaN for a flagged one).
// The step kernels are the rollout and adjoint kernels of the open-loop calls; the per-step
// adjoint recomputes its step from the stored state (every step a checkpoint).
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

#include "cordsim.h"
#include "internal.h"

namespace {

constexpr int kApgThreads = 128;
constexpr int kApgMaxHidden = 1024;

template <typename R>
__device__ __forceinline__ const R* apg_w2(const R* th, int nq, int h) { return th + (size_t)h * nq + h; }

// u_t = W2 tanh(W1 q_t + b1) + b2 for rollout blockIdx.x; effort[b] += w_u |u_t|^2
template <typename R>
__global__ void __launch_bounds__(kApgThreads) apg_policy_fwd_kernel(int nq, int h, const R* __restrict__ th,
                                                                     const R* __restrict__ q, R* __restrict__ u,
                                                                     R* __restrict__ hid, R w_u,
                                                                     R* __restrict__ effort) {
  extern __shared__ __align__(16) unsigned char apg_smem[];
  R* qs = reinterpret_cast<R*>(apg_smem);   // n_q
  R* as = qs + nq;                          // h
  R* us = as + h;                           // 6
  const int b = blockIdx.x;
  for (int k = threadIdx.x; k < nq; k += blockDim.x) qs[k] = q[(size_t)b * nq + k];
  __syncthreads();
  const R* b1 = th + (size_t)h * nq;
  for (int i = threadIdx.x; i < h; i += blockDim.x) {
    const R* w = th + (size_t)i * nq;
    R a = b1[i];
    for (int k = 0; k < nq; ++k) a = fma(w[k], qs[k], a);
    a = tanh(a);
    as[i] = a;
    hid[(size_t)b * h + i] = a;
  }
  __syncthreads();
  const R* W2 = apg_w2(th, nq, h);
  if (threadIdx.x < 6) {
    const int o = threadIdx.x;
    R v = W2[6 * h + o];
    for (int i = 0; i < h; ++i) v = fma(W2[(size_t)o * h + i], as[i], v);
    u[(size_t)b * 6 + o] = v;
    us[o] = v;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    R e = R(0);
    for (int o = 0; o < 6; ++o) e = fma(us[o], us[o], e);
    effort[b] += w_u * e;
  }
}

// g = dL/du_t + 2 w_u u_t; lambda_t = dL/dq_t + W1^T ((W2^T g) .* (1 - a^2)) written as the next
// seed; rollout b's dL/dtheta accumulated; Lsum[b] += the step's loss terms
template <typename R>
__global__ void __launch_bounds__(kApgThreads) apg_policy_bwd_kernel(
    int nq, int h, const R* __restrict__ th, const R* __restrict__ q, const R* __restrict__ hid,
    const R* __restrict__ u, const R* __restrict__ dLdu, const R* __restrict__ dLdq, const R* __restrict__ Lt,
    R w_u, R* __restrict__ seed_next, R* __restrict__ dth, R* __restrict__ Lsum) {
  extern __shared__ __align__(16) unsigned char apg_smem[];
  R* qs = reinterpret_cast<R*>(apg_smem);   // n_q
  R* ga = qs + nq;                          // h
  R* as = ga + h;                           // h
  R* gs = as + h;                           // 6
  const int b = blockIdx.x;
  const size_t nth = (size_t)h * nq + 7 * (size_t)h + 6;
  for (int k = threadIdx.x; k < nq; k += blockDim.x) qs[k] = q[(size_t)b * nq + k];
  for (int i = threadIdx.x; i < h; i += blockDim.x) as[i] = hid[(size_t)b * h + i];
  if (threadIdx.x < 6) gs[threadIdx.x] = dLdu[(size_t)b * 6 + threadIdx.x] + R(2) * w_u * u[(size_t)b * 6 + threadIdx.x];
  if (threadIdx.x == 0) Lsum[b] += Lt[b];
  __syncthreads();
  const R* W2 = apg_w2(th, nq, h);
  for (int i = threadIdx.x; i < h; i += blockDim.x) {
    R s = R(0);
    for (int o = 0; o < 6; ++o) s = fma(W2[(size_t)o * h + i], gs[o], s);
    ga[i] = s * (R(1) - as[i] * as[i]);
  }
  __syncthreads();
  for (int k = threadIdx.x; k < nq; k += blockDim.x) {
    R s = dLdq[(size_t)b * nq + k];
    for (int i = 0; i < h; ++i) s = fma(th[(size_t)i * nq + k], ga[i], s);
    seed_next[(size_t)b * 2 * nq + nq + k] = s;          // the next (earlier) step's seed on q_t
  }
  R* d = dth + (size_t)b * nth;
  for (size_t e = threadIdx.x; e < (size_t)h * nq; e += blockDim.x) d[e] += ga[e / nq] * qs[e % nq];
  R* db1 = d + (size_t)h * nq;
  for (int i = threadIdx.x; i < h; i += blockDim.x) db1[i] += ga[i];
  R* dW2 = db1 + h;
  for (int e = threadIdx.x; e < 6 * h; e += blockDim.x) dW2[e] += gs[e / h] * as[e % h];
  if (threadIdx.x < 6) dW2[6 * h + threadIdx.x] += gs[threadIdx.x];
}

// dtheta = sum over the completed rollouts of their dL/dtheta (in rollout order); L[b], dq0[b]
template <typename R>
__global__ void apg_reduce_kernel(int B, int nq, size_t nth, const R* __restrict__ dthb,
                                  const int32_t* __restrict__ st, R* __restrict__ dtheta) {
  for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x; e < nth; e += (size_t)gridDim.x * blockDim.x) {
    R s = R(0);
    for (int b = 0; b < B; ++b)
      if (st[b] == 0) s += dthb[(size_t)b * nth + e];
    dtheta[e] = s;
  }
}

template <typename R>
__global__ void apg_finish_kernel(int B, int nq, const int32_t* __restrict__ st, const R* __restrict__ Lsum,
                                  const R* __restrict__ effort, const R* __restrict__ seeds, R* L, R* dq0) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < B * (nq + 1); e += gridDim.x * blockDim.x) {
    const int b = e / (nq + 1), k = e % (nq + 1);
    if (k == nq) {
      if (L) L[b] = st[b] ? R(NAN) : Lsum[b] + effort[b];
    } else if (dq0) {
      dq0[(size_t)b * nq + k] = st[b] ? R(0) : seeds[(size_t)b * 2 * nq + nq + k];
    }
  }
}

__global__ void apg_or_kernel(int B, const int32_t* __restrict__ src, int32_t* __restrict__ dst) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < B; b += gridDim.x * blockDim.x) dst[b] |= src[b];
}

struct ApgWs {
  size_t q, u, hid, seeds, dldu, dldq, lt, lsum, effort, dth, st_step, st_acc, total;
};

inline size_t al256(size_t x) { return (x + 255) & ~(size_t)255; }

ApgWs apg_ws(long long B, int H, int nq, int h, size_t rb) {
  ApgWs w;
  size_t off = 0;
  auto take = [&](size_t bytes) { const size_t o = off; off = al256(off + bytes); return o; };
  const size_t nth = (size_t)h * nq + 7 * (size_t)h + 6;
  w.q = take((size_t)(H + 1) * B * nq * rb);
  w.u = take((size_t)H * B * 6 * rb);
  w.hid = take((size_t)H * B * h * rb);
  w.seeds = take((size_t)B * 2 * nq * rb);
  w.dldu = take((size_t)B * 6 * rb);
  w.dldq = take((size_t)B * nq * rb);
  w.lt = take((size_t)B * rb);
  w.lsum = take((size_t)B * rb);
  w.effort = take((size_t)B * rb);
  w.dth = take((size_t)B * nth * rb);
  w.st_step = take((size_t)B * sizeof(int32_t));
  w.st_acc = take((size_t)B * sizeof(int32_t));
  w.total = off;
  return w;
}

template <typename R>
cs_status run(cs_sim* s, int B, int H, int h, const R* q0, const R* th, const cs_loss* loss, R* L, R* dtheta,
              R* dq0, int32_t* status, unsigned char* ws, cudaStream_t st) {
  const int nq = s->nq;
  const ApgWs w = apg_ws(B, H, nq, h, sizeof(R));
  auto at = [&](size_t o) { return reinterpret_cast<R*>(ws + o); };
  R* Q = at(w.q);
  R* U = at(w.u);
  R* HID = at(w.hid);
  R* seeds = at(w.seeds);
  int32_t* st_step = reinterpret_cast<int32_t*>(ws + w.st_step);
  int32_t* st_acc = reinterpret_cast<int32_t*>(ws + w.st_acc);
  const size_t nth = (size_t)h * nq + 7 * (size_t)h + 6;
  const R w_u = (R)loss->w_u;
  cudaError_t e;
  if ((e = cudaMemcpyAsync(Q, q0, sizeof(R) * (size_t)B * nq, cudaMemcpyDeviceToDevice, st)) != cudaSuccess)
    return cs_cuda_fail(e, "cudaMemcpyAsync");
  if ((e = cudaMemsetAsync(ws + w.seeds, 0, w.st_acc + sizeof(int32_t) * (size_t)B - w.seeds, st)) != cudaSuccess)
    return cs_cuda_fail(e, "cudaMemsetAsync");
  const size_t smf = sizeof(R) * ((size_t)nq + h + 6), smb = sizeof(R) * ((size_t)nq + 2 * h + 6);
  cs_status r;
  for (int t = 0; t < H; ++t) {
    R* qt = Q + (size_t)t * B * nq;
    R* ut = U + (size_t)t * B * 6;
    apg_policy_fwd_kernel<R><<<B, kApgThreads, smf, st>>>(nq, h, th, qt, ut, HID + (size_t)t * B * h, w_u,
                                                          at(w.effort));
    if ((r = csi::check_launch("apg_policy_fwd_kernel"))) return r;
    if ((r = sim_rollout(s, B, 1, qt, ut, nullptr, qt + (size_t)B * nq, st_step, st))) return r;
    apg_or_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, st_step, st_acc);
    if ((r = csi::check_launch("apg_or_kernel"))) return r;
  }
  for (int t = H - 1; t >= 0; --t) {
    cs_loss lt = *loss;
    lt.w_u = 0.0;                                   // the effort is the policy kernels' term
    if (t != H - 1) lt.w_goal = 0.0;                // the goal is on q_H alone
    const R* qt = Q + (size_t)t * B * nq;
    const R* ut = U + (size_t)t * B * 6;
    if ((r = sim_rollout_vjp(s, B, 1, qt, ut, seeds, &lt, at(w.lt), at(w.dldu), at(w.dldq), st_step, st)))
      return r;
    apg_or_kernel<<<(B + 255) / 256, 256, 0, st>>>(B, st_step, st_acc);
    if ((r = csi::check_launch("apg_or_kernel"))) return r;
    apg_policy_bwd_kernel<R><<<B, kApgThreads, smb, st>>>(nq, h, th, qt, HID + (size_t)t * B * h, ut,
                                                          at(w.dldu), at(w.dldq), at(w.lt), w_u, seeds,
                                                          at(w.dth), at(w.lsum));
    if ((r = csi::check_launch("apg_policy_bwd_kernel"))) return r;
  }
  apg_reduce_kernel<R><<<(int)std::min<size_t>((nth + 255) / 256, 1184), 256, 0, st>>>(B, nq, nth, at(w.dth),
                                                                                       st_acc, dtheta);
  if ((r = csi::check_launch("apg_reduce_kernel"))) return r;
  apg_finish_kernel<R><<<(B * (nq + 1) + 255) / 256, 256, 0, st>>>(B, nq, st_acc, at(w.lsum), at(w.effort),
                                                                   seeds, L, dq0);
  if ((r = csi::check_launch("apg_finish_kernel"))) return r;
  if (status && (e = cudaMemcpyAsync(status, st_acc, sizeof(int32_t) * (size_t)B, cudaMemcpyDeviceToDevice, st)) !=
                    cudaSuccess)
    return cs_cuda_fail(e, "cudaMemcpyAsync");
  return CS_OK;
}

}  // namespace

extern "C" {

size_t apg_workspace(const cs_sim* s, int B, int H, int hidden) {
  if (!s || B < 0 || H < 1 || hidden < 1) return 0;
  return apg_ws(B, H, s->nq, hidden, (size_t)s->real_bytes).total;
}

cs_status apg_rollout_grad(cs_sim* s, int B, int H, int hidden, const void* q0, const void* theta,
                           const cs_loss* loss, void* L, void* dtheta, void* dq0, int32_t* status,
                           void* workspace, size_t workspace_bytes, void* stream) {
  if (!s) return cs_fail(CS_ERR_INVALID_ARG, "null handle");
  if (B < 1 || B > s->P.max_batch) return cs_fail(CS_ERR_INVALID_ARG, "B must be in [1, max_batch]");
  if (H < 1) return cs_fail(CS_ERR_INVALID_ARG, "H must be >= 1");
  if (hidden < 1 || hidden > kApgMaxHidden) return cs_fail(CS_ERR_INVALID_ARG, "hidden must be in [1, 1024]");
  if (!q0 || !theta || !loss || !dtheta || !workspace) return cs_fail(CS_ERR_INVALID_ARG, "null pointer");
  cs_status r = cs_validate_loss(loss, s->nv);
  if (r) return r;
  if (workspace_bytes < apg_workspace(s, B, H, hidden))
    return cs_fail(CS_ERR_INVALID_ARG, "workspace smaller than apg_workspace()");
  cudaStream_t st = (cudaStream_t)stream;
  unsigned char* ws = (unsigned char*)workspace;
  if (s->real_bytes == 4)
    return run<float>(s, B, H, hidden, (const float*)q0, (const float*)theta, loss, (float*)L, (float*)dtheta,
                      (float*)dq0, status, ws, st);
  return run<double>(s, B, H, hidden, (const double*)q0, (const double*)theta, loss, (double*)L,
                     (double*)dtheta, (double*)dq0, status, ws, st);
}

}  // extern "C"
