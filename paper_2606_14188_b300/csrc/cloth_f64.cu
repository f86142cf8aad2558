// cloth kernels, double instantiation.
#include "launch_cloth.cuh"

namespace csi {
template cs_status launch_cloth_rollout<double>(cs_sim*, int, int, const void*, const void*, void*, void*, int32_t*, int32_t*, cudaStream_t);
template cs_status launch_cloth_vjp<double>(cs_sim*, int, int, const void*, const void*, const void*, const cs_loss*, void*, void*, void*, int32_t*, cudaStream_t);
template int cloth_ctas_per_sm<double>(const cs_sim*);
template cs_status launch_cloth_packed<double>(const void*, const int*, int, int, void*, size_t, int, size_t, size_t, cudaStream_t);
template cs_status cloth_packed_prepare<double>(size_t, int*);
}  // namespace csi
