// Plan-solve kernels, double instantiation.
#define CS_PLAN_INSTANTIATE
#include "launch_plan.cuh"

namespace csi {
template cs_status plan_prepare<double>(int, size_t);
template cs_status launch_plan_vjp<double>(const void*, const int*, int, int, int, int, size_t, int, cudaStream_t);
template cs_status launch_plan_init<double>(const void*, int, int, int, cudaStream_t);
template cs_status launch_plan_select<double>(const void*, int, cudaStream_t);
template cs_status launch_plan_adam<double>(const void*, int, int, cudaStream_t);
}  // namespace csi
