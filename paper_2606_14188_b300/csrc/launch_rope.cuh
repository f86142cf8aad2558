// Kernel launchers for the rope kernels (instantiated per real type in rope_*.cu).  Rollouts and
// adjoints run one 64-thread CTA per rollout (rope_cta.cuh; nodes per thread NPT = 1 up to 64
// nodes, 2 up to 128); the linearisation runs a CTA per (trajectory, step) in two launches
// (rope_lin.cuh) with the handle's per-step records, else one warp per (trajectory, step)
// (rope.cuh; pairs per lane PPL = 1 up to 64 nodes, 2 up to 128).
#pragma once
#include <algorithm>
#include "internal.h"
#include "rope.cuh"
#include "rope_cta.cuh"
#include "rope_lin.cuh"

namespace csi {

template <typename Kern>
inline cs_status launch_prep(Kern k, size_t smem, const cs_sim* s) {
  if (smem > s->smem_optin) return cs_fail(CS_ERR_INVALID_ARG, "scene too large for shared memory");
  return prep_kernel(k, smem);
}

template <typename R, int NPT>
cs_status rollout_cta(cs_sim* s, int B, int H, const void* q0, const void* u, void* traj,
                      void* qH, int32_t* status, int32_t* counters, cudaStream_t st) {
  cs::Scene<R> S = make_scene<R>(s, nullptr);
  const size_t smem = cs::rc::sm_elems(NPT, s->P.n_obstacles) * sizeof(R);
  const bool so = s->P.second_order != 0;    // the inertial variant's copy of the kernels
  auto kr = so ? cs::rci::rope_cta_rollout_kernel<R, NPT> : cs::rc::rope_cta_rollout_kernel<R, NPT>;
  cs_status r = launch_prep(kr, smem, s);
  if (r) return r;
  kr<<<B, cs::rc::NT, smem, st>>>(S, B, H, (const R*)q0, (const R*)u,
                                                                       (R*)traj, (R*)qH, status, counters);
  return check_launch("rope_cta_rollout_kernel");
}

template <typename R>
cs_status launch_rollout(cs_sim* s, int B, int H, const void* q0, const void* u, void* traj,
                         void* qH, int32_t* status, int32_t* counters, cudaStream_t st) {
  return s->nv <= 64 ? rollout_cta<R, 1>(s, B, H, q0, u, traj, qH, status, counters, st)
                     : rollout_cta<R, 2>(s, B, H, q0, u, traj, qH, status, counters, st);
}

template <typename R, int NPT>
cs_status vjp_cta(cs_sim* s, int B, int H, const void* q0, const void* u, const void* dLdtraj,
                  const cs_loss* loss, void* L, void* dLdu, void* dLdq0, int32_t* status,
                  cudaStream_t st) {
  cs::Scene<R> S = make_scene<R>(s, loss);
  const size_t smem = cs::rc::sm_elems(NPT, s->P.n_obstacles) * sizeof(R);
  const bool so = s->P.second_order != 0;    // the inertial variant's copy of the kernels
  auto k_all = so ? cs::rci::rope_cta_vjp_kernel<R, NPT> : cs::rc::rope_cta_vjp_kernel<R, NPT>;
  auto k_fwd = so ? cs::rci::rope_cta_vjp_fwd_kernel<R, NPT> : cs::rc::rope_cta_vjp_fwd_kernel<R, NPT>;
  auto k_bwd = so ? cs::rci::rope_cta_vjp_bwd_kernel<R, NPT> : cs::rc::rope_cta_vjp_bwd_kernel<R, NPT>;
  cs_status r = launch_prep(k_all, smem, s);
  if (r) return r;
  const int NT = cs::rc::NT;
  if (s->d_fac && s->d_queue) {
    // work queue: forward jobs, then (rollout, segment) jobs, each rollout's adjoint chain in the
    // CTA that finishes its last segment; a persistent grid of the CTAs the device holds at once
    auto kq = so ? cs::rci::rope_cta_vjp_queue_kernel<R, NPT> : cs::rc::rope_cta_vjp_queue_kernel<R, NPT>;
    if ((r = launch_prep(kq, smem, s))) return r;
    const int nseg = (H + s->P.checkpoint_every - 1) / s->P.checkpoint_every;
    int per_sm = 0;
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kq, NT, smem);
    if (per_sm < 1) return cs_fail(CS_ERR_INVALID_ARG, "scene too large for shared memory");
    const long long jobs = (long long)B * (1 + nseg);
    const int grid = (int)std::min<long long>((long long)per_sm * s->sms, jobs);
    cudaError_t e = cudaMemsetAsync(s->d_queue, 0, cs::rc::queue_ints(B, nseg) * sizeof(int), st);
    if (e != cudaSuccess) return cs_cuda_fail(e, "cudaMemsetAsync");
    int* q = static_cast<int*>(s->d_queue);
    kq<<<grid, NT, smem, st>>>(S, B, H, (const R*)q0, (const R*)u, (const R*)dLdtraj, (R*)L, (R*)dLdu, (R*)dLdq0,
                              status, (R*)s->d_ws, s->ws_stride, (R*)s->d_fac, s->fac_stride, q);
    if ((r = check_launch("rope_cta_vjp_queue_kernel"))) return r;
    cs::rc::rope_queue_finish_kernel<R><<<(B + 127) / 128, 128, 0, st>>>(B, H, nseg, q, (R*)L, (R*)dLdu, status);
    return check_launch("rope_queue_finish_kernel");
  }
  // More rollouts than the device holds at once: the late starters decide when the launch ends,
  // so the forward parts run first (each measuring its cost), then the backward parts, costliest
  // first, leaving the cheap ones to start late.
  int per_sm = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_all, NT, smem);
  if ((long long)per_sm * s->sms < B && B <= cs::CS_ORDER_MAX) {
    if ((r = launch_prep(k_fwd, smem, s))) return r;
    if ((r = launch_prep(k_bwd, smem, s))) return r;
    int32_t* cost = reinterpret_cast<int32_t*>(static_cast<char*>(s->d_ws) +
                                               vjp_ord_offset(s->ws_stride, s->P.max_batch, s->real_bytes));
    int32_t* order = cost + B;
    k_fwd<<<B, NT, smem, st>>>(S, B, H, (const R*)q0, (const R*)u,
                                                                 (const R*)dLdtraj, (R*)L, (R*)dLdu, (R*)dLdq0,
                                                                 status, (R*)s->d_ws, s->ws_stride, cost);
    if ((r = check_launch("rope_cta_vjp_fwd_kernel"))) return r;
    cs::rope_order_kernel<cs::CS_ORDER_NT><<<1, cs::CS_ORDER_NT, 0, st>>>(cost, B, order);
    if ((r = check_launch("rope_order_kernel"))) return r;
    k_bwd<<<B, NT, smem, st>>>(S, B, H, (const R*)u, (const R*)dLdtraj, (R*)L,
                                                                 (R*)dLdu, (R*)dLdq0, status, (R*)s->d_ws,
                                                                 s->ws_stride, cost, order);
    return check_launch("rope_cta_vjp_bwd_kernel");
  }
  k_all<<<B, NT, smem, st>>>(S, B, H, (const R*)q0, (const R*)u,
                                                           (const R*)dLdtraj, (R*)L, (R*)dLdu, (R*)dLdq0,
                                                           status, (R*)s->d_ws, s->ws_stride);
  return check_launch("rope_cta_vjp_kernel");
}

template <typename R>
cs_status launch_vjp(cs_sim* s, int B, int H, const void* q0, const void* u, const void* dLdtraj,
                     const cs_loss* loss, void* L, void* dLdu, void* dLdq0, int32_t* status,
                     cudaStream_t st) {
  return s->nv <= 64 ? vjp_cta<R, 1>(s, B, H, q0, u, dLdtraj, loss, L, dLdu, dLdq0, status, st)
                     : vjp_cta<R, 2>(s, B, H, q0, u, dLdtraj, loss, L, dLdu, dLdq0, status, st);
}

// The linearisation in two launches (rope_lin.cuh) when the handle holds per-step records: the
// smooth step of every (trajectory, step) job with its record, then every tangent direction of a
// job in one pass of a CTA.
template <typename R, int NPT>
cs_status linearize_cta(cs_sim* s, int B, int H, const void* z, const void* v, void* A, void* Bm,
                        int32_t* status, cudaStream_t st) {
  cs::Scene<R> S = make_scene<R>(s, nullptr);
  const size_t smem1 = cs::rc::sm_elems(NPT, s->P.n_obstacles) * sizeof(R);
  const bool so = s->P.second_order != 0;    // the inertial variant's copy of the kernels
  auto k1 = so ? cs::rci::rope_cta_lin_step_kernel<R, NPT> : cs::rc::rope_cta_lin_step_kernel<R, NPT>;
  auto k2 = so ? cs::rci::rope_lin_tangent_kernel<R> : cs::rc::rope_lin_tangent_kernel<R>;
  cs_status r = launch_prep(k1, smem1, s);
  if (r) return r;
  const int nv = s->nv, N = s->npair, ndir = s->nq + 6;
  const size_t rb = sizeof(R);
  const size_t fixed = (cs::rc::lin_fixed_elems(N, nv) + 3) / 4 * 4 * rb, per = 6 * (size_t)N * rb;
  // directions per pass: what fits three CTAs on an SM, else two
  size_t budget = 76000;
  long long dpr = fixed < budget ? (long long)((budget - fixed) / per) : 0;
  if (dpr < 32) {
    budget = std::min<size_t>(s->smem_optin, 2 * budget);
    dpr = fixed < budget ? (long long)((budget - fixed) / per) : 0;
  }
  dpr = std::min<long long>(std::min<long long>(dpr, ndir), 160);
  if (dpr < 1) return cs_fail(CS_ERR_INVALID_ARG, "scene too large for shared memory");
  const int threads = (int)((dpr + 31) / 32 * 32);
  const size_t smem2 = cs::rc::lin_smem_elems(N, nv, (int)dpr) * rb;
  if ((r = launch_prep(k2, smem2, s))) return r;
  if (status) {
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t) * (size_t)B, st);
    if (e != cudaSuccess) return cs_cuda_fail(e, "cudaMemsetAsync");
  }
  const long long jobs = (long long)B * H;
  int per1 = 0, per2 = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per1, k1, cs::rc::NT, smem1);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per2, k2, threads, smem2);
  if (per1 < 1 || per2 < 1) return cs_fail(CS_ERR_INVALID_ARG, "scene too large for shared memory");
  const int g1 = (int)std::min<long long>((long long)per1 * s->sms, jobs);
  const int g2 = (int)std::min<long long>((long long)per2 * s->sms, jobs);
  k1<<<g1, cs::rc::NT, smem1, st>>>(S, B, H, (const R*)z, (const R*)v, (R*)s->d_fac, s->fac_stride, status);
  if ((r = check_launch("rope_cta_lin_step_kernel"))) return r;
  k2<<<g2, threads, smem2, st>>>(S, B, H, 32 * NPT, (const R*)s->d_fac, s->fac_stride, (int)dpr, (R*)A, (R*)Bm);
  return check_launch("rope_lin_tangent_kernel");
}

template <typename R, int PPL>
cs_status linearize_ppl(cs_sim* s, int B, int H, const void* z, const void* v, void* A, void* Bm,
                        int32_t* status, cudaStream_t st) {
  cs::Scene<R> S = make_scene<R>(s, nullptr);
  const size_t smem = smem_bytes(s, H, true);
  cs_status r = launch_prep(cs::rope_linearize_kernel<R, PPL>, smem, s);
  if (r) return r;
  if (status) {
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t) * (size_t)B, st);
    if (e != cudaSuccess) return cs_cuda_fail(e, "cudaMemsetAsync");
  }
  const long long jobs = (long long)B * H;
  const int grid = (int)(jobs < 65535LL * 32 ? jobs : 65535LL * 32);
  cs::rope_linearize_kernel<R, PPL><<<grid, 32, smem, st>>>(S, B, H, (const R*)z, (const R*)v,
                                                             (R*)A, (R*)Bm, status);
  return check_launch("rope_linearize_kernel");
}

template <typename R>
cs_status launch_linearize(cs_sim* s, int B, int H, const void* z, const void* v, void* A,
                           void* Bm, int32_t* status, cudaStream_t st) {
  if (s->d_fac)
    return s->nv <= 64 ? linearize_cta<R, 1>(s, B, H, z, v, A, Bm, status, st)
                       : linearize_cta<R, 2>(s, B, H, z, v, A, Bm, status, st);
  if (s->P.second_order)
    return cs_fail(CS_ERR_UNSUPPORTED, "the inertial linearisation needs the handle's per-step records");
  return s->npair <= 32 ? linearize_ppl<R, 1>(s, B, H, z, v, A, Bm, status, st)
                        : linearize_ppl<R, 2>(s, B, H, z, v, A, Bm, status, st);
}

}  // namespace csi
