// rollout kernel, double instantiation.
#include "launch_rope.cuh"

namespace csi {
template cs_status launch_rollout<double>(cs_sim*, int, int, const void*, const void*, void*, void*, int32_t*, int32_t*, cudaStream_t);
}  // namespace csi
