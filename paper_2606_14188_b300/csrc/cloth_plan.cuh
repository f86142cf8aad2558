// Served plan solves of cloths: one packed launch over the candidates of every running cloth
// request, one CTA per candidate at a time (the cloth path's kernel body), candidates and results in
// each request's PlanJob; the CTA workspace slots are the server's pool.
#pragma once
#include "cloth.cuh"
#include "plan.cuh"

namespace cs {

// item g of [0, total) is candidate g - first[j] of cloth job j (first[] ascending, first[0] = 0);
// one CTA per item at a time, on its own workspace slot; the item's scene is copied to shared
// memory at scene_off (past the widest job's layout) and its band geometry recomputed from it
template <typename R>
__global__ void __launch_bounds__(CL_NT) cloth_vjp_packed_kernel(const PlanJob<R>* jobs, const int* first, int njobs,
                                                                int total, R* slots, size_t slot_stride,
                                                                size_t scene_off) {
  Scene<R>* Ssm = reinterpret_cast<Scene<R>*>(cs_smem + scene_off);
  for (int g = blockIdx.x; g < total; g += gridDim.x) {
    int lo = 0, hi = njobs - 1;
    while (lo < hi) {
      const int mid = (lo + hi + 1) >> 1;
      if (first[mid] <= g) lo = mid; else hi = mid - 1;
    }
    const PlanJob<R>* J = jobs + lo;
    const int r = g - first[lo];
    __syncthreads();                       // the previous item is done with the scene copy
    const int* src = reinterpret_cast<const int*>(&J->S);
    int* dst = reinterpret_cast<int*>(Ssm);
    for (int i = threadIdx.x; i < (int)(sizeof(Scene<R>) / sizeof(int)); i += CL_NT) dst[i] = src[i];
    __syncthreads();
    const Scene<R>& S = *Ssm;
    ClothDims D = cloth_dims(S.rows, S.cols);
    D.win_global = J->cloth_wg;
    const ClothSm<R> c = cloth_sm<R>(D);
    const ClothWS<R> w = cloth_carve<R>(slots + blockIdx.x * slot_stride, D, S.nobs);
    const int H = J->H;
    cl_vjp_rollout<R>(S, D, w, c, H, J->q0, J->U + (size_t)r * H * 6, nullptr, J->L + r,
                      J->dU + (size_t)r * H * 6, nullptr, J->status + r, J->ws + (size_t)r * J->ws_stride);
  }
}

}  // namespace cs
