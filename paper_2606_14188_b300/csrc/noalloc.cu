// sim_rollout_vjp_noalloc: the rollout adjoint without any device allocation.
//
// Some callers cannot allocate device memory: a real-time control loop that must not block on a
// driver allocation (cudaMalloc can take milliseconds and synchronise the device), or a process
// whose device memory is already owned by another allocator (a framework's caching allocator
// holding all free memory).  This entry point serves them: it needs no handle (sim_create
// allocates) and keeps its scratch -- the spring rest lengths and the adjoint's checkpoint
// records -- in one file-scope device array of fixed size, which every GPU that loads the
// library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>

#include "cordsim.h"
#include "internal.h"

namespace {

// scratch layout: [L1 rest lengths | L2 rest lengths | adjoint workspace (checkpoint records and
// carry per rollout, then the cost and order arrays)], 256-byte aligned parts
constexpr size_t kRestBytes = 256 * sizeof(double);   // room for 128 nodes of either real type
static __device__ __align__(256) unsigned char g_noalloc_scratch[CS_NOALLOC_SCRATCH_BYTES];

constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};
std::mutex g_scratch_mu;

// device address of the scratch array on the current device (looked up once per device)
cs_status scratch_address(void** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cs_cuda_fail(e, "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return cs_fail(CS_ERR_INVALID_ARG, "device index too large");
  std::lock_guard<std::mutex> lock(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return cs_cuda_fail(e, "cudaGetSymbolAddress");
    g_scratch_addr[dev] = p;
  }
  *out = g_scratch_addr[dev];
  return CS_OK;
}

// the rest lengths travel in the kernel's argument (by value): no host buffer has to outlive the
// call and no host-to-device copy is issued
template <typename R>
struct RestLengths {
  R L1[128];   // stretch (j, j+1)
  R L2[128];   // bend (j, j+2)
};

template <typename R>
__global__ void noalloc_rest_kernel(RestLengths<R> a, R* dst1, R* dst2) {
  for (int i = threadIdx.x; i < 128; i += blockDim.x) {
    dst1[i] = a.L1[i];
    dst2[i] = a.L2[i];
  }
}

template <typename R>
cs_status upload_rest(const double* rest_x, int nv, R* dst1, R* dst2, cudaStream_t st) {
  RestLengths<R> a;
  for (int i = 0; i < 128; ++i) a.L1[i] = a.L2[i] = R(0);
  auto dist = [&](int i, int j) {
    const double d0 = rest_x[3 * j] - rest_x[3 * i], d1 = rest_x[3 * j + 1] - rest_x[3 * i + 1],
                 d2 = rest_x[3 * j + 2] - rest_x[3 * i + 2];
    return std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  };
  for (int j = 0; j + 1 < nv; ++j) a.L1[j] = (R)dist(j, j + 1);
  for (int j = 0; j + 2 < nv; ++j) a.L2[j] = (R)dist(j, j + 2);
  noalloc_rest_kernel<R><<<1, 128, 0, st>>>(a, dst1, dst2);
  return csi::check_launch("noalloc_rest_kernel");
}

}  // namespace

extern "C" cs_status sim_rollout_vjp_noalloc(const cs_params* P, const double* rest_x, int B, int H,
                                             const void* q0, const void* u, const void* dL_dtraj,
                                             const cs_loss* loss, void* L, void* dL_du, void* dL_dq0,
                                             int32_t* status, void* stream) {
  if (!P || !rest_x) return cs_fail(CS_ERR_INVALID_ARG, "null params or rest_x");
  cs_status r = cs_validate_params(P);
  if (r) return r;
  if (P->kind != CS_ROPE) return cs_fail(CS_ERR_UNSUPPORTED, "only kind = CS_ROPE is built");
  if (P->second_order) return cs_fail(CS_ERR_UNSUPPORTED, "built for the quasi-static step");
  const int nv = P->n_nodes;
  if (P->checkpoint_every < 1) return cs_fail(CS_ERR_INVALID_ARG, "checkpoint_every must be >= 1");
  if (B < 0 || H < 1) return cs_fail(CS_ERR_INVALID_ARG, "B must be >= 0 and H >= 1");
  if (!dL_dtraj && !loss) return cs_fail(CS_ERR_INVALID_ARG, "give dL_dtraj or a loss");
  if (loss && (r = cs_validate_loss(loss, nv))) return r;
  if (B == 0) return CS_OK;
  if (!q0 || !u || !dL_du) return cs_fail(CS_ERR_INVALID_ARG, "q0, u and dL_du are required");

  // the handle lives on the stack and points into the scratch array
  cs_sim s;
  s.P = *P;
  s.P.max_batch = B;
  s.P.max_horizon = H;
  s.nv = nv;
  s.npair = (nv + 1) / 2;
  s.nq = 3 * nv + 6;
  s.real_bytes = P->real_bytes;
  const int k = P->checkpoint_every;
  s.ws_stride = cs::vjp_ws_elems(nv, H, k);
  const size_t need = 2 * kRestBytes + csi::vjp_ws_bytes(s.ws_stride, B, (size_t)s.real_bytes);
  if (need > CS_NOALLOC_SCRATCH_BYTES)
    return cs_fail(CS_ERR_INVALID_ARG,
                   "B x horizon exceed the allocation-free scratch (CS_NOALLOC_SCRATCH_BYTES)");
  void* base = nullptr;
  if ((r = scratch_address(&base))) return r;
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  s.sms = v;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  s.smem_optin = (size_t)v;
  unsigned char* b8 = static_cast<unsigned char*>(base);
  s.d_L1 = b8;
  s.d_L2 = b8 + kRestBytes;
  s.d_ws = b8 + 2 * kRestBytes;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  // every element the kernel reads is written earlier in the same call: nothing needs zeroing
  if (s.real_bytes == 4) {
    r = upload_rest<float>(rest_x, nv, (float*)s.d_L1, (float*)s.d_L2, st);
    if (!r) r = csi::launch_vjp<float>(&s, B, H, q0, u, dL_dtraj, loss, L, dL_du, dL_dq0, status, st);
  } else {
    r = upload_rest<double>(rest_x, nv, (double*)s.d_L1, (double*)s.d_L2, st);
    if (!r) r = csi::launch_vjp<double>(&s, B, H, q0, u, dL_dtraj, loss, L, dL_du, dL_dq0, status, st);
  }
  return r;
}
