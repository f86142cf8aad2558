// vjp kernel, float instantiation.
#include "launch_rope.cuh"

namespace csi {
template cs_status launch_vjp<float>(cs_sim*, int, int, const void*, const void*, const void*, const cs_loss*, void*, void*, void*, int32_t*, cudaStream_t);
}  // namespace csi
