// cloth kernels, float instantiation.
#include "launch_cloth.cuh"

namespace csi {
template cs_status launch_cloth_rollout<float>(cs_sim*, int, int, const void*, const void*, void*, void*, int32_t*, int32_t*, cudaStream_t);
template cs_status launch_cloth_vjp<float>(cs_sim*, int, int, const void*, const void*, const void*, const cs_loss*, void*, void*, void*, int32_t*, cudaStream_t);
template int cloth_ctas_per_sm<float>(const cs_sim*);
template cs_status launch_cloth_packed<float>(const void*, const int*, int, int, void*, size_t, int, size_t, size_t, cudaStream_t);
template cs_status cloth_packed_prepare<float>(size_t, int*);
}  // namespace csi
