// Plan-solve kernels, float instantiation.
#define CS_PLAN_INSTANTIATE
#include "launch_plan.cuh"

namespace csi {
template cs_status plan_prepare<float>(int, size_t);
template cs_status launch_plan_vjp<float>(const void*, const int*, int, int, int, int, size_t, int, cudaStream_t);
template cs_status launch_plan_init<float>(const void*, int, int, int, cudaStream_t);
template cs_status launch_plan_select<float>(const void*, int, cudaStream_t);
template cs_status launch_plan_adam<float>(const void*, int, int, cudaStream_t);
}  // namespace csi
