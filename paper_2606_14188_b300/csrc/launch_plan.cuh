// Host launchers of the plan-solve kernels (instantiated per real type in plan_*.cu) and the
// real-type independent description of one request that the server fills.
#pragma once
#include "internal.h"
#include "plan.cuh"

namespace csi {

// one request's device buffers and settings, independent of the real type
struct PlanSpec {
  cs_params P;
  cs_loss loss;
  const void *L1, *L2, *q0, *warm;
  void *U, *M, *V, *dU, *L, *ws, *best_u;
  int32_t* status;
  cs::PlanState* st;
  size_t ws_stride;
  unsigned long long seed;
  int H, Rc, G, warm_H, warm_shift;
  int cloth_wg;
  double lr, sigma, u_max;
};

template <typename R>
inline size_t plan_job_bytes() {
  static_assert(sizeof(cs::PlanJob<R>) % 16 == 0, "the job table's stride must be sizeof(PlanJob)");
  return sizeof(cs::PlanJob<R>);
}

template <typename R>
inline void plan_fill_job(void* out, const PlanSpec& p) {
  cs::PlanJob<R> J;
  std::memset(&J, 0, sizeof(J));
  J.S = make_scene_from<R>(p.P, p.L1, p.L2, &p.loss);
  J.q0 = static_cast<const R*>(p.q0);
  J.warm = static_cast<const R*>(p.warm);
  J.U = static_cast<R*>(p.U);
  J.M = static_cast<R*>(p.M);
  J.V = static_cast<R*>(p.V);
  J.dU = static_cast<R*>(p.dU);
  J.L = static_cast<R*>(p.L);
  J.status = p.status;
  J.ws = static_cast<R*>(p.ws);
  J.best_u = static_cast<R*>(p.best_u);
  J.st = p.st;
  J.ws_stride = p.ws_stride;
  J.seed = p.seed;
  J.H = p.H;
  J.Rc = p.Rc;
  J.G = p.G;
  J.warm_H = p.warm_H;
  J.warm_shift = p.warm_shift;
  J.cloth_wg = p.cloth_wg;
  J.lr = (R)p.lr;
  J.sigma = (R)p.sigma;
  J.u_max = (R)p.u_max;
  std::memcpy(out, &J, sizeof(J));
}

// shared memory of one warp of the packed launch
template <typename R>
inline size_t plan_warp_smem(int ppl, int nobs_max, int H_max) {
  const size_t b = cs::plan_scene_bytes<R>() + cs::ws_size(32 * ppl, nobs_max, H_max, false) * sizeof(R);
  return (b + 15) & ~(size_t)15;
}

// raise the packed kernel's dynamic shared-memory limit (not a stream operation: call it before
// a stream capture)
template <typename R>
cs_status plan_prepare(int ppl, size_t smem) {
  return ppl == 1 ? prep_kernel(cs::rope_vjp_packed_kernel<R, 1>, smem)
                  : prep_kernel(cs::rope_vjp_packed_kernel<R, 2>, smem);
}

template <typename R>
cs_status launch_plan_vjp(const void* jobs, const int* first, int njobs, int total, int ppl, int warps,
                          size_t warp_smem, int grid, cudaStream_t st) {
  const size_t smem = warp_smem * (size_t)warps;
  if (ppl == 1)
    cs::rope_vjp_packed_kernel<R, 1><<<grid, 32 * warps, smem, st>>>(
        static_cast<const cs::PlanJob<R>*>(jobs), first, njobs, total, warp_smem);
  else
    cs::rope_vjp_packed_kernel<R, 2><<<grid, 32 * warps, smem, st>>>(
        static_cast<const cs::PlanJob<R>*>(jobs), first, njobs, total, warp_smem);
  return check_launch("rope_vjp_packed_kernel");
}

inline int plan_elem_grid(int max_elems) {
  const int g = (max_elems + 255) / 256;
  return g < 1 ? 1 : (g > 512 ? 512 : g);
}

template <typename R>
cs_status launch_plan_init(const void* jobs, int j0, int n, int max_elems, cudaStream_t st) {
  cs::plan_init_kernel<R><<<dim3(plan_elem_grid(max_elems), n), 256, 0, st>>>(
      static_cast<const cs::PlanJob<R>*>(jobs), j0);
  return check_launch("plan_init_kernel");
}

template <typename R>
cs_status launch_plan_select(const void* jobs, int njobs, cudaStream_t st) {
  cs::plan_select_kernel<R><<<njobs, 256, 0, st>>>(static_cast<const cs::PlanJob<R>*>(jobs));
  return check_launch("plan_select_kernel");
}

template <typename R>
cs_status launch_plan_adam(const void* jobs, int njobs, int max_elems, cudaStream_t st) {
  cs::plan_adam_kernel<R><<<dim3(plan_elem_grid(max_elems), njobs), 256, 0, st>>>(
      static_cast<const cs::PlanJob<R>*>(jobs));
  return check_launch("plan_adam_kernel");
}

#ifndef CS_PLAN_INSTANTIATE
// the kernels are compiled once, in plan_f32.cu / plan_f64.cu
#define CS_PLAN_EXTERN(R)                                                                           \
  extern template cs_status plan_prepare<R>(int, size_t);                                           \
  extern template cs_status launch_plan_vjp<R>(const void*, const int*, int, int, int, int, size_t, int, \
                                               cudaStream_t);                                       \
  extern template cs_status launch_plan_init<R>(const void*, int, int, int, cudaStream_t);          \
  extern template cs_status launch_plan_select<R>(const void*, int, cudaStream_t);                  \
  extern template cs_status launch_plan_adam<R>(const void*, int, int, cudaStream_t);
CS_PLAN_EXTERN(float)
CS_PLAN_EXTERN(double)
#undef CS_PLAN_EXTERN
#endif

}  // namespace csi
