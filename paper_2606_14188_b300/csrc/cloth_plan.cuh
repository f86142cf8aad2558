// Served plan solves of a cloth: the forward + adjoint of every candidate of one request, one CTA
// per candidate at a time (the cloth path's kernel body), candidates and results in the request's
// PlanJob.  The scene comes by value (kernel parameter space); the CTA workspace slots are the
// server's pool.
#pragma once
#include "cloth.cuh"
#include "plan.cuh"

namespace cs {

template <typename R>
__global__ void __launch_bounds__(CL_NT) cloth_vjp_plan_kernel(Scene<R> S, ClothDims D, const PlanJob<R>* job,
                                                              R* slots, size_t slot_stride) {
  const ClothSm<R> c = cloth_sm<R>(D);
  const ClothWS<R> w = cloth_carve<R>(slots + blockIdx.x * slot_stride, D, S.nobs);
  const PlanJob<R>& J = *job;
  const int H = J.H;
  for (int r = blockIdx.x; r < J.Rc; r += gridDim.x)
    cl_vjp_rollout<R>(S, D, w, c, H, J.q0, J.U + (size_t)r * H * 6, nullptr, J.L + r, J.dU + (size_t)r * H * 6,
                      nullptr, J.status + r, J.ws + (size_t)r * J.ws_stride);
}

}  // namespace cs
