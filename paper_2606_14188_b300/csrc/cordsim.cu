// C-ABI host side of libcordsim: argument checking, workspace, scene upload, kernel launches.
// Every entry point is declared (with its contract) in include/cordsim.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "cordsim.h"
#include "common.cuh"
#include "internal.h"

namespace {

thread_local std::string g_err;
thread_local int64_t g_launches = 0;

}  // namespace

cs_status cs_fail(cs_status s, const std::string& msg) {
  g_err = msg;
  return s;
}

cs_status cs_cuda_fail(cudaError_t e, const char* where) {
  g_err = std::string(where) + ": " + cudaGetErrorString(e);
  return CS_ERR_CUDA;
}

void cs_count_launch() { ++g_launches; }

using namespace csi;

static cs_status check_common(cs_sim* s, int B, int H) {
  if (!s) return cs_fail(CS_ERR_INVALID_ARG, "null handle");
  if (B < 0 || H < 1) return cs_fail(CS_ERR_INVALID_ARG, "B must be >= 0 and H >= 1");
  if (B > s->P.max_batch) return cs_fail(CS_ERR_INVALID_ARG, "B exceeds max_batch");
  if (H > s->P.max_horizon) return cs_fail(CS_ERR_INVALID_ARG, "H exceeds max_horizon");
  return CS_OK;
}


cs_status cs_validate_params(const cs_params* P) {
  if (!P) return cs_fail(CS_ERR_INVALID_ARG, "null params");
  if (P->kind != CS_ROPE && P->kind != CS_CLOTH) return cs_fail(CS_ERR_INVALID_ARG, "unknown kind");
  const bool cloth = P->kind == CS_CLOTH;
  const int nv = P->n_nodes;
  if (!cloth && (nv < 2 || nv > 128)) return cs_fail(CS_ERR_INVALID_ARG, "rope n_nodes must be in [2, 128]");
  if (cloth && (P->rows < 1 || P->cols < 2 || P->rows > 256 || P->cols > 256 || nv != P->rows * P->cols))
    return cs_fail(CS_ERR_INVALID_ARG, "cloth needs rows >= 1, cols >= 2 and n_nodes = rows * cols");
  for (int i = 0; i < 2; ++i)
    if (P->grasp_node[i] < 0 || P->grasp_node[i] >= nv)
      return cs_fail(CS_ERR_INVALID_ARG, "grasp_node out of range");
  if (P->grasp_node[0] == P->grasp_node[1])
    return cs_fail(CS_ERR_INVALID_ARG, "the two grippers must hold different nodes");
  if (P->real_bytes != 4 && P->real_bytes != 8)
    return cs_fail(CS_ERR_INVALID_ARG, "real_bytes must be 4 or 8");
  if (P->n_obstacles < 0 || P->n_obstacles > CS_MAX_OBSTACLES)
    return cs_fail(CS_ERR_INVALID_ARG, "n_obstacles out of range");
  for (int o = 0; o < P->n_obstacles; ++o) {
    const int t = P->obstacles[o].type;
    if (t != CS_PLANE && t != CS_SPHERE && t != CS_BOX)
      return cs_fail(CS_ERR_INVALID_ARG, "unknown obstacle type");
  }
  if (!(P->dt > 0) || !(P->node_mass > 0)) return cs_fail(CS_ERR_INVALID_ARG, "dt and node_mass must be > 0");
  if (P->newton_max < 1 || P->ipm_max < 1) return cs_fail(CS_ERR_INVALID_ARG, "iteration caps must be >= 1");
  if (!(P->kappa_decay > 0 && P->kappa_decay < 1)) return cs_fail(CS_ERR_INVALID_ARG, "kappa_decay must be in (0,1)");
  if (!(P->kappa_c > 0) || !(P->kappa_hard > 0) || P->kappa_hard > P->kappa_c)
    return cs_fail(CS_ERR_INVALID_ARG, "need 0 < kappa_hard <= kappa_c");
  if (P->second_order && cloth) return cs_fail(CS_ERR_UNSUPPORTED, "the inertial variant is built for ropes only");
  if (P->second_order && !(P->damp_alpha >= 0 && P->damp_beta >= 0 && P->damp_alpha < 1e30 && P->damp_beta < 1e30))
    return cs_fail(CS_ERR_INVALID_ARG, "damp_alpha and damp_beta must be finite and >= 0");
  return CS_OK;
}

cs_status cs_validate_loss(const cs_loss* loss, int nv) {
  if (!loss) return CS_OK;
  if (loss->n_goal < 0 || loss->n_goal > CS_MAX_GOAL) return cs_fail(CS_ERR_INVALID_ARG, "n_goal out of range");
  for (int g = 0; g < loss->n_goal; ++g)
    if (loss->goal_nodes[g] < 0 || loss->goal_nodes[g] >= nv)
      return cs_fail(CS_ERR_INVALID_ARG, "goal node out of range");
  return CS_OK;
}

extern "C" {

cs_status sim_create(const cs_params* P, const double* rest_x, cs_sim** out) {
  if (!P || !rest_x || !out) return cs_fail(CS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  cs_status vr = cs_validate_params(P);
  if (vr) return vr;
  const bool cloth = P->kind == CS_CLOTH;
  const int nv = P->n_nodes;
  if (P->checkpoint_every < 0) return cs_fail(CS_ERR_INVALID_ARG, "checkpoint_every must be >= 0");
  if (P->max_batch < 1 || P->max_horizon < 1) return cs_fail(CS_ERR_INVALID_ARG, "max_batch/max_horizon must be >= 1");

  cs_sim* s = new cs_sim();
  s->P = *P;
  s->nv = nv;
  s->npair = (nv + 1) / 2;
  s->nq = (P->second_order ? 6 : 3) * nv + 6;
  s->real_bytes = P->real_bytes;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) { delete s; return cs_cuda_fail(e, "cudaGetDevice"); }
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev);
  s->sms = v;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  s->smem_optin = (size_t)v;
  auto dist = [&](int a, int b) {
    double d0 = rest_x[3 * b] - rest_x[3 * a], d1 = rest_x[3 * b + 1] - rest_x[3 * a + 1],
           d2 = rest_x[3 * b + 2] - rest_x[3 * a + 2];
    return std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  };
  // rest lengths in the kernels' real type (cloth: every spring, family by family)
  std::vector<double> L1, L2(1, 0.0);
  if (cloth) {
    s->cd = cs::cloth_dims(P->rows, P->cols);
    if (!cs::cloth_fit(s->cd, (size_t)P->real_bytes, s->smem_optin)) {
      delete s;
      return cs_fail(CS_ERR_INVALID_ARG, "cloth too large for one CTA's shared memory");
    }
    cloth_rest_lengths(P->rows, P->cols, rest_x, L1);
    if ((int)L1.size() != s->cd.nspr) {
      delete s;
      return cs_fail(CS_ERR_INVALID_ARG, "cloth spring count mismatch");
    }
  } else {
    if (smem_bytes(s, 1, false) > s->smem_optin) {
      delete s;
      return cs_fail(CS_ERR_INVALID_ARG, "scene too large for one warp's shared memory");
    }
    L1.assign(nv - 1, 0.0);
    L2.assign(nv > 2 ? nv - 2 : 1, 0.0);
    for (int j = 0; j + 1 < nv; ++j) L1[j] = dist(j, j + 1);
    for (int j = 0; j + 2 < nv; ++j) L2[j] = dist(j, j + 2);
  }
  const size_t rb = (size_t)s->real_bytes;
  auto upload = [&](const std::vector<double>& h, void** d) -> cudaError_t {
    cudaError_t er = cudaMalloc(d, h.size() * rb);
    if (er != cudaSuccess) return er;
    if (rb == 8) return cudaMemcpy(*d, h.data(), h.size() * 8, cudaMemcpyHostToDevice);
    std::vector<float> f(h.begin(), h.end());
    return cudaMemcpy(*d, f.data(), f.size() * 4, cudaMemcpyHostToDevice);
  };
  if ((e = upload(L1, &s->d_L1)) != cudaSuccess || (e = upload(L2, &s->d_L2)) != cudaSuccess) {
    sim_destroy(s);
    return e == cudaErrorMemoryAllocation ? cs_fail(CS_ERR_OOM, "rest lengths") : cs_cuda_fail(e, "upload");
  }
  auto ws_elems = [&](int kk) {
    return cloth ? cs::cloth_vjp_ws_elems(nv, P->max_horizon, kk) : cs::vjp_ws_elems(nv, P->max_horizon, kk, P->second_order ? 1 : 0);
  };
  if (s->P.checkpoint_every == 0) {
    // automatic: the smallest interval whose adjoint workspace fits in a quarter of the free
    // device memory, at most about sqrt(max_horizon) (the adjoint is the same for every
    // interval; a shorter one recomputes fewer steps)
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    const int kmax = std::max(1, (int)std::lround(std::sqrt((double)P->max_horizon)));
    int kk = 1;
    while (kk < kmax && vjp_ws_bytes(ws_elems(kk), P->max_batch, rb) > free_b / 4) ++kk;
    s->P.checkpoint_every = kk;
  }
  const int k = s->P.checkpoint_every;
  // checkpoint records (state, grasp offsets, stage-1 offset and stage-2 displacement of the
  // producing step) and the carry of the two-part launch
  s->ws_stride = ws_elems(k);
  e = cudaMalloc(&s->d_ws, vjp_ws_bytes(s->ws_stride, P->max_batch, rb));
  if (e != cudaSuccess) {
    sim_destroy(s);
    return e == cudaErrorMemoryAllocation ? cs_fail(CS_ERR_OOM, "adjoint workspace") : cs_cuda_fail(e, "cudaMalloc");
  }
  if (!cloth) {
    // the work-queue adjoint's per-step records; without room for them the adjoint runs as the
    // one-launch or two-part form instead (same results)
    const int NPT = nv <= 64 ? 1 : 2;
    const int nseg = (P->max_horizon + k - 1) / k;
    s->fac_stride = (size_t)P->max_horizon * cs::rc::fac_step_elems(NPT, nv);
    const size_t fac_bytes = s->fac_stride * (size_t)P->max_batch * rb;
    size_t free_b = 0, total_b = 0;
    cudaMemGetInfo(&free_b, &total_b);
    if (fac_bytes <= free_b / 2) {
      if (cudaMalloc(&s->d_fac, fac_bytes) != cudaSuccess ||
          cudaMalloc(&s->d_queue, cs::rc::queue_ints(P->max_batch, nseg) * sizeof(int)) != cudaSuccess) {
        cudaGetLastError();          // clear the allocation failure: the handle works without the queue
        if (s->d_fac) cudaFree(s->d_fac);
        s->d_fac = s->d_queue = nullptr;
      }
    }
  }
  if (cloth) {
    // one workspace slot per CTA the device holds at once (the kernels' grid never exceeds it)
    const int per_sm = rb == 4 ? cloth_ctas_per_sm<float>(s) : cloth_ctas_per_sm<double>(s);
    const int resident = per_sm * s->sms;
    s->nslots = P->max_batch < resident ? P->max_batch : resident;
    s->slot_stride = cs::cloth_ws_elems(s->cd, P->n_obstacles);
    e = cudaMalloc(&s->d_slots, s->slot_stride * (size_t)s->nslots * rb);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_claim, 2 * sizeof(int));
    if (e != cudaSuccess) {
      sim_destroy(s);
      return e == cudaErrorMemoryAllocation ? cs_fail(CS_ERR_OOM, "cloth workspace") : cs_cuda_fail(e, "cudaMalloc");
    }
  }
  *out = s;
  g_err.clear();
  return CS_OK;
}

cs_status sim_destroy(cs_sim* s) {
  if (!s) return CS_OK;
  cudaDeviceSynchronize();
  if (s->d_L1) cudaFree(s->d_L1);
  if (s->d_L2) cudaFree(s->d_L2);
  if (s->d_ws) cudaFree(s->d_ws);
  if (s->d_slots) cudaFree(s->d_slots);
  if (s->d_claim) cudaFree(s->d_claim);
  if (s->d_fac) cudaFree(s->d_fac);
  if (s->d_queue) cudaFree(s->d_queue);
  delete s;
  return CS_OK;
}

cs_status sim_rollout(cs_sim* s, int B, int H, const void* q0, const void* u, void* traj, void* qH,
                      int32_t* status, void* stream) {
  return sim_rollout_counters(s, B, H, q0, u, traj, qH, status, nullptr, stream);
}

cs_status sim_rollout_counters(cs_sim* s, int B, int H, const void* q0, const void* u, void* traj,
                               void* qH, int32_t* status, int32_t* counters, void* stream) {
  cs_status r = check_common(s, B, H);
  if (r) return r;
  if (B == 0) return CS_OK;
  if (!q0 || !u) return cs_fail(CS_ERR_INVALID_ARG, "q0 and u are required");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (s->P.kind == CS_CLOTH)
    return s->real_bytes == 4 ? launch_cloth_rollout<float>(s, B, H, q0, u, traj, qH, status, counters, st)
                              : launch_cloth_rollout<double>(s, B, H, q0, u, traj, qH, status, counters, st);
  return s->real_bytes == 4 ? launch_rollout<float>(s, B, H, q0, u, traj, qH, status, counters, st)
                            : launch_rollout<double>(s, B, H, q0, u, traj, qH, status, counters, st);
}

cs_status sim_rollout_vjp(cs_sim* s, int B, int H, const void* q0, const void* u,
                          const void* dL_dtraj, const cs_loss* loss, void* L, void* dL_du,
                          void* dL_dq0, int32_t* status, void* stream) {
  cs_status r = check_common(s, B, H);
  if (r) return r;
  if (!dL_dtraj && !loss) return cs_fail(CS_ERR_INVALID_ARG, "give dL_dtraj or a loss");
  if (B > 0 && (!q0 || !u || !dL_du)) return cs_fail(CS_ERR_INVALID_ARG, "q0, u and dL_du are required");
  if (loss && (r = cs_validate_loss(loss, s->nv))) return r;
  if (B == 0) return CS_OK;
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (s->P.kind == CS_CLOTH)
    return s->real_bytes == 4
               ? launch_cloth_vjp<float>(s, B, H, q0, u, dL_dtraj, loss, L, dL_du, dL_dq0, status, st)
               : launch_cloth_vjp<double>(s, B, H, q0, u, dL_dtraj, loss, L, dL_du, dL_dq0, status, st);
  return s->real_bytes == 4
             ? launch_vjp<float>(s, B, H, q0, u, dL_dtraj, loss, L, dL_du, dL_dq0, status, st)
             : launch_vjp<double>(s, B, H, q0, u, dL_dtraj, loss, L, dL_du, dL_dq0, status, st);
}

cs_status sim_linearize(cs_sim* s, int B, int H, const void* z, const void* v, void* A, void* Bm,
                        int32_t* status, void* stream) {
  cs_status r = check_common(s, B, H);
  if (r) return r;
  if (B == 0) return CS_OK;
  if (!z || !v || !A || !Bm) return cs_fail(CS_ERR_INVALID_ARG, "z, v, A and Bm are required");
  if (s->P.kind == CS_CLOTH) return cs_fail(CS_ERR_UNSUPPORTED, "sim_linearize is built for ropes only");
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  return s->real_bytes == 4 ? launch_linearize<float>(s, B, H, z, v, A, Bm, status, st)
                            : launch_linearize<double>(s, B, H, z, v, A, Bm, status, st);
}

int64_t cs_launch_count(void) {
  const int64_t n = g_launches;
  g_launches = 0;
  return n;
}

const char* cs_last_error(void) { return g_err.c_str(); }

}  // extern "C"
