// Kernel launchers for the rope kernels (instantiated per real type in rope_*.cu).
#pragma once
#include "internal.h"
#include "rope.cuh"

namespace csi {

template <typename R>
cs_status launch_rollout(cs_sim* s, int B, int H, const void* q0, const void* u, void* traj,
                         void* qH, int32_t* status, int32_t* counters, cudaStream_t st) {
  cs::Scene<R> S = make_scene<R>(s, nullptr);
  const size_t smem = smem_bytes(s, H, false);
  if (smem > s->smem_optin) return cs_fail(CS_ERR_INVALID_ARG, "horizon too long for shared memory");
  cs_status r = prep_kernel(cs::rope_rollout_kernel<R>, smem);
  if (r) return r;
  cs::rope_rollout_kernel<R><<<B, 32, smem, st>>>(S, B, H, (const R*)q0, (const R*)u, (R*)traj,
                                                   (R*)qH, status, counters);
  return check_launch("rope_rollout_kernel");
}

template <typename R>
cs_status launch_vjp(cs_sim* s, int B, int H, const void* q0, const void* u, const void* dLdtraj,
                     const cs_loss* loss, void* L, void* dLdu, void* dLdq0, int32_t* status,
                     cudaStream_t st) {
  cs::Scene<R> S = make_scene<R>(s, loss);
  const size_t smem = smem_bytes(s, H, false);
  if (smem > s->smem_optin) return cs_fail(CS_ERR_INVALID_ARG, "horizon too long for shared memory");
  cs_status r = prep_kernel(cs::rope_vjp_kernel<R>, smem);
  if (r) return r;
  cs::rope_vjp_kernel<R><<<B, 32, smem, st>>>(S, B, H, (const R*)q0, (const R*)u,
                                               (const R*)dLdtraj, (R*)L, (R*)dLdu, (R*)dLdq0,
                                               status, (R*)s->d_ws, s->ws_stride);
  return check_launch("rope_vjp_kernel");
}

template <typename R>
cs_status launch_linearize(cs_sim* s, int B, int H, const void* z, const void* v, void* A,
                           void* Bm, int32_t* status, cudaStream_t st) {
  cs::Scene<R> S = make_scene<R>(s, nullptr);
  const size_t smem = smem_bytes(s, H, true);
  if (smem > s->smem_optin) return cs_fail(CS_ERR_INVALID_ARG, "scene too large for shared memory");
  cs_status r = prep_kernel(cs::rope_linearize_kernel<R>, smem);
  if (r) return r;
  if (status) {
    cudaError_t e = cudaMemsetAsync(status, 0, sizeof(int32_t) * (size_t)B, st);
    if (e != cudaSuccess) return cs_cuda_fail(e, "cudaMemsetAsync");
  }
  const long long jobs = (long long)B * H;
  const int grid = (int)(jobs < 65535LL * 32 ? jobs : 65535LL * 32);
  cs::rope_linearize_kernel<R><<<grid, 32, smem, st>>>(S, B, H, (const R*)z, (const R*)v, (R*)A,
                                                        (R*)Bm, status);
  return check_launch("rope_linearize_kernel");
}



}  // namespace csi
