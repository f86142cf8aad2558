// Kernel launchers of the cloth path (instantiated per real type in cloth_*.cu).  One CTA per
// rollout at a time over a grid of at most s->nslots CTAs, each with its own workspace slot.
#pragma once
#include "cloth_plan.cuh"
#include "internal.h"

namespace csi {

inline size_t cloth_smem_bytes(const cs_sim* s) { return cs::cloth_smem_elems(s->cd) * (size_t)s->real_bytes; }

// a launch with more rollouts than CTAs hands out the rest through a counter: zero both first
inline cs_status zero_claim(cs_sim* s, int B, int grid, cudaStream_t st) {
  if (B <= grid) return CS_OK;
  const cudaError_t e = cudaMemsetAsync(s->d_claim, 0, 2 * sizeof(int), st);
  return e == cudaSuccess ? CS_OK : cs_cuda_fail(e, "cudaMemsetAsync");
}

template <typename R>
cs_status launch_cloth_rollout(cs_sim* s, int B, int H, const void* q0, const void* u, void* traj, void* qH,
                               int32_t* status, int32_t* counters, cudaStream_t st) {
  cs::Scene<R> S = make_scene<R>(s, nullptr);
  const size_t smem = cloth_smem_bytes(s);
  cs_status r = prep_kernel(cs::cloth_rollout_kernel<R>, smem);
  if (r) return r;
  const int grid = B < s->nslots ? B : s->nslots;
  if ((r = zero_claim(s, B, grid, st))) return r;
  cs::cloth_rollout_kernel<R><<<grid, cs::CL_NT, smem, st>>>(S, s->cd, B, H, (const R*)q0, (const R*)u, (R*)traj,
                                                            (R*)qH, status, counters, (R*)s->d_slots,
                                                            s->slot_stride, (int*)s->d_claim);
  return check_launch("cloth_rollout_kernel");
}

template <typename R>
cs_status launch_cloth_vjp(cs_sim* s, int B, int H, const void* q0, const void* u, const void* dLdtraj,
                           const cs_loss* loss, void* L, void* dLdu, void* dLdq0, int32_t* status,
                           cudaStream_t st) {
  cs::Scene<R> S = make_scene<R>(s, loss);
  const size_t smem = cloth_smem_bytes(s);
  cs_status r = prep_kernel(cs::cloth_vjp_kernel<R>, smem);
  if (r) return r;
  const int grid = B < s->nslots ? B : s->nslots;
  if ((r = zero_claim(s, B, grid, st))) return r;
  // more rollouts than CTAs: the forward parts first (each measuring its Newton and interior-point
  // work), then the backward parts handed out costliest first, so that the late ones are cheap
  if (B > grid && B <= cs::CS_ORDER_MAX) {
    if ((r = prep_kernel(cs::cloth_vjp_fwd_kernel<R>, smem))) return r;
    if ((r = prep_kernel(cs::cloth_vjp_bwd_kernel<R>, smem))) return r;
    int32_t* cost = reinterpret_cast<int32_t*>(static_cast<char*>(s->d_ws) +
                                               vjp_ord_offset(s->ws_stride, s->P.max_batch, s->real_bytes));
    int32_t* order = cost + B;
    int* claim = static_cast<int*>(s->d_claim);
    cs::cloth_vjp_fwd_kernel<R><<<grid, cs::CL_NT, smem, st>>>(S, s->cd, B, H, (const R*)q0, (const R*)u,
                                                              (const R*)dLdtraj, (R*)L, (R*)dLdu, (R*)dLdq0, status,
                                                              (R*)s->d_slots, s->slot_stride, (R*)s->d_ws,
                                                              s->ws_stride, claim, cost);
    if ((r = check_launch("cloth_vjp_fwd_kernel"))) return r;
    cs::rope_order_kernel<cs::CS_ORDER_NT><<<1, cs::CS_ORDER_NT, 0, st>>>(cost, B, order);
    if ((r = check_launch("rope_order_kernel"))) return r;
    cs::cloth_vjp_bwd_kernel<R><<<grid, cs::CL_NT, smem, st>>>(S, s->cd, B, H, (const R*)u, (const R*)dLdtraj,
                                                              (R*)L, (R*)dLdu, (R*)dLdq0, status, (R*)s->d_slots,
                                                              s->slot_stride, (R*)s->d_ws, s->ws_stride, claim + 1,
                                                              cost, order);
    return check_launch("cloth_vjp_bwd_kernel");
  }
  cs::cloth_vjp_kernel<R><<<grid, cs::CL_NT, smem, st>>>(S, s->cd, B, H, (const R*)q0, (const R*)u,
                                                        (const R*)dLdtraj, (R*)L, (R*)dLdu, (R*)dLdq0, status,
                                                        (R*)s->d_slots, s->slot_stride, (R*)s->d_ws,
                                                        s->ws_stride, (int*)s->d_claim);
  return check_launch("cloth_vjp_kernel");
}

// plan solves: every candidate of the njobs cloth jobs (device job table `jobs`, candidate offsets
// `first`), over at most nslots CTAs of smem bytes (scene copy at scene_off)
template <typename R>
cs_status launch_cloth_packed(const void* jobs, const int* first, int njobs, int total, void* slots,
                              size_t slot_stride, int nslots, size_t smem, size_t scene_off, cudaStream_t st) {
  const int grid = total < nslots ? total : nslots;
  cs::cloth_vjp_packed_kernel<R><<<grid, cs::CL_NT, smem, st>>>(static_cast<const cs::PlanJob<R>*>(jobs), first,
                                                               njobs, total, static_cast<R*>(slots), slot_stride,
                                                               scene_off);
  return check_launch("cloth_vjp_packed_kernel");
}

// raise the packed kernel's shared-memory limit (not a stream operation: before a capture) and
// report its resident CTAs per SM
template <typename R>
cs_status cloth_packed_prepare(size_t smem, int* ctas_per_sm) {
  cs_status r = prep_kernel(cs::cloth_vjp_packed_kernel<R>, smem);
  if (r) return r;
  int a = 0;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, cs::cloth_vjp_packed_kernel<R>, cs::CL_NT, smem);
  *ctas_per_sm = a > 0 ? a : 1;
  return CS_OK;
}

// resident CTAs per SM of the cloth kernels at their shared-memory size (at least 1)
template <typename R>
int cloth_ctas_per_sm(const cs_sim* s) {
  const size_t smem = cloth_smem_bytes(s);
  int a = 0, b = 0;
  if (prep_kernel(cs::cloth_rollout_kernel<R>, smem) || prep_kernel(cs::cloth_vjp_kernel<R>, smem)) return 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&a, cs::cloth_rollout_kernel<R>, cs::CL_NT, smem);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, cs::cloth_vjp_kernel<R>, cs::CL_NT, smem);
  const int m = a > b ? a : b;
  return m > 0 ? m : 1;
}

}  // namespace csi
