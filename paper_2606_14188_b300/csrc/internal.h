// Internal host-side definitions shared by the C-ABI translation units.
#pragma once
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "cordsim.h"
#include "cloth_band.cuh"
#include "common.cuh"
#include "rope.cuh"
#include "rope_cta.cuh"

cs_status cs_fail(cs_status s, const std::string& msg);
cs_status cs_cuda_fail(cudaError_t e, const char* where);
void cs_count_launch();

// Argument checks shared by the entry points that take a cs_params or a cs_loss (sim_create,
// sim_rollout_vjp, sim_rollout_vjp_noalloc): kind and sizes, grasp nodes (in range, distinct),
// real type, obstacles, dt and node mass, iteration caps, barrier parameters.  The workspace
// sizes (max_batch, max_horizon) and the checkpoint interval are checked by each caller.
cs_status cs_validate_params(const cs_params* P);
// n_goal within [0, CS_MAX_GOAL] and every goal node within [0, nv)
cs_status cs_validate_loss(const cs_loss* loss, int nv);

struct cs_sim {
  cs_params P;
  int nv, npair, nq;
  int real_bytes;
  void* d_L1 = nullptr;   // rest lengths (stretch)
  void* d_L2 = nullptr;   // rest lengths (bend)
  void* d_ws = nullptr;   // adjoint workspace: ws_stride elements per rollout (checkpoint and
                          // segment records, carry), then the cost and order arrays (vjp_ord_offset)
  size_t ws_stride = 0;   // elements per rollout
  // rope adjoint by the work queue: per rollout max_horizon per-step records (factorisations of the
  // step's adjoint and its smooth solution, fac_stride elements), and the queue state (int32);
  // null when the memory was not available (then the adjoint runs without the queue)
  void* d_fac = nullptr;
  size_t fac_stride = 0;
  void* d_queue = nullptr;
  int sms = 0;
  size_t smem_optin = 0;
  // cloth only: band geometry and the per-CTA workspace slots of the cloth kernels
  cs::ClothDims cd{};
  void* d_slots = nullptr;
  void* d_claim = nullptr;  // int[2]: next rollout to hand out, for launches with more rollouts than
                            // CTAs (the second for the backward part of a two-part launch)
  size_t slot_stride = 0;  // elements per slot
  int nslots = 0;
};

namespace csi {


// the kernels' scene from the parameters, the device rest lengths and an optional loss
template <typename R>
cs::Scene<R> make_scene_from(const cs_params& P, const void* d_L1, const void* d_L2, const cs_loss* loss) {
  cs::Scene<R> S;
  std::memset(&S, 0, sizeof(S));
  S.nv = P.n_nodes;
  S.npair = (P.n_nodes + 1) / 2;
  S.nobs = P.n_obstacles;
  S.grasp[0] = P.grasp_node[0];
  S.grasp[1] = P.grasp_node[1];
  S.kind = P.kind;
  S.rows = P.rows;
  S.cols = P.cols;
  S.fwd_mode = P.fwd_mode;
  S.grad_mode = P.grad_mode;
  S.newton_max = P.newton_max;
  S.ipm_max = P.ipm_max;
  S.ckpt = P.checkpoint_every;
  S.w = (R)(P.node_mass / (P.dt * P.dt));
  S.m = (R)P.node_mass;
  for (int i = 0; i < 3; ++i) S.grav[i] = (R)P.gravity[i];
  S.Dmax = (R)P.D_max;
  S.kh = (R)P.kappa_h;
  S.kc = (R)P.kappa_c;
  S.khard = (R)P.kappa_hard;
  S.kdecay = (R)P.kappa_decay;
  S.mu = (R)P.mu;
  S.rgrasp = (R)P.r_grasp;
  S.rad = (R)P.node_radius;
  S.sig0 = (R)P.sigma0;
  S.ntol = (R)P.newton_tol;
  S.itol = (R)P.ipm_tol;
  S.so = P.second_order ? 1 : 0;
  S.nq = (S.so ? 6 : 3) * P.n_nodes + 6;
  S.dt = (R)P.dt;
  S.cm = (R)(S.so ? P.damp_alpha * P.node_mass / P.dt : 0.0);
  S.cb = (R)(S.so ? P.damp_beta / P.dt : 0.0);
  S.k1 = (R)P.k_stretch;
  S.k2 = (R)P.k_bend;
  S.k3 = (R)P.k_shear;
  for (int o = 0; o < P.n_obstacles; ++o) {
    S.ob_type[o] = P.obstacles[o].type;
    for (int i = 0; i < 6; ++i) S.ob[o][i] = (R)P.obstacles[o].p[i];
  }
  S.L1 = static_cast<const R*>(d_L1);
  S.L2 = static_cast<const R*>(d_L2);
  if (loss) {
    S.has_loss = 1;
    S.n_goal = loss->n_goal;
    for (int g = 0; g < loss->n_goal; ++g) {
      S.goal[g] = loss->goal_nodes[g];
      for (int i = 0; i < 3; ++i) S.goal_pos[g][i] = (R)loss->goal_pos[g][i];
    }
    S.w_goal = (R)loss->w_goal;
    S.w_pen = (R)loss->w_pen;
    S.pen_m = (R)loss->pen_margin;
    S.w_u = (R)loss->w_u;
  }
  return S;
}

template <typename R>
cs::Scene<R> make_scene(const cs_sim* s, const cs_loss* loss) {
  return make_scene_from<R>(s->P, s->d_L1, s->d_L2, loss);
}

inline size_t smem_bytes(const cs_sim* s, int H, bool lin) {
  const size_t rb = (size_t)s->real_bytes;
  const int NP = s->npair <= 32 ? 32 : 64;
  size_t n = cs::ws_size(NP, s->P.n_obstacles, lin ? 1 : H, lin);
  if (lin) n += (size_t)2 * 6 * s->npair * 32 + (size_t)27 * s->nv;
  return n * rb;
}

template <typename Kern>
cs_status prep_kernel(Kern k, size_t smem) {
  cudaError_t e = cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return cs_cuda_fail(e, "cudaFuncSetAttribute");
  return CS_OK;
}

// the adjoint workspace: max_batch blocks of ws_stride elements, then (256-byte aligned) the
// int32 cost [max_batch] and order [max_batch] arrays of the two-part launch
inline size_t vjp_ord_offset(size_t ws_stride, int max_batch, size_t rb) {
  return (ws_stride * (size_t)max_batch * rb + 255) & ~(size_t)255;
}
inline size_t vjp_ws_bytes(size_t ws_stride, int max_batch, size_t rb) {
  return vjp_ord_offset(ws_stride, max_batch, rb) + 2 * sizeof(int32_t) * (size_t)max_batch;
}

inline cs_status check_launch(const char* what) {
  cs_count_launch();
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return cs_cuda_fail(e, what);
  return CS_OK;
}



// launchers (one translation unit per kernel and real type)
template <typename R>
cs_status launch_rollout(cs_sim* s, int B, int H, const void* q0, const void* u, void* traj,
                         void* qH, int32_t* status, int32_t* counters, cudaStream_t st);
template <typename R>
cs_status launch_vjp(cs_sim* s, int B, int H, const void* q0, const void* u, const void* dLdtraj,
                     const cs_loss* loss, void* L, void* dLdu, void* dLdq0, int32_t* status,
                     cudaStream_t st);
template <typename R>
cs_status launch_cloth_rollout(cs_sim* s, int B, int H, const void* q0, const void* u, void* traj, void* qH,
                               int32_t* status, int32_t* counters, cudaStream_t st);
template <typename R>
cs_status launch_cloth_vjp(cs_sim* s, int B, int H, const void* q0, const void* u, const void* dLdtraj,
                           const cs_loss* loss, void* L, void* dLdu, void* dLdq0, int32_t* status,
                           cudaStream_t st);
template <typename R>
int cloth_ctas_per_sm(const cs_sim* s);
template <typename R>
cs_status launch_cloth_packed(const void* jobs, const int* first, int njobs, int total, void* slots,
                              size_t slot_stride, int nslots, size_t smem, size_t scene_off, cudaStream_t st);
template <typename R>
cs_status cloth_packed_prepare(size_t smem, int* ctas_per_sm);

// rest lengths of a cloth's springs in the cloth kernels' order (family by family: structural along
// rows, along columns, the two shear diagonals, bend along rows, along columns)
inline void cloth_rest_lengths(int R, int C, const double* rest, std::vector<double>& L1) {
  auto dist = [&](int a, int b) {
    const double d0 = rest[3 * b] - rest[3 * a], d1 = rest[3 * b + 1] - rest[3 * a + 1],
                 d2 = rest[3 * b + 2] - rest[3 * a + 2];
    return std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  };
  auto id = [&](int r, int c) { return r * C + c; };
  L1.clear();
  for (int r = 0; r < R; ++r) for (int c = 0; c + 1 < C; ++c) L1.push_back(dist(id(r, c), id(r, c + 1)));
  for (int r = 0; r + 1 < R; ++r) for (int c = 0; c < C; ++c) L1.push_back(dist(id(r, c), id(r + 1, c)));
  for (int r = 0; r + 1 < R; ++r) for (int c = 0; c + 1 < C; ++c) L1.push_back(dist(id(r, c), id(r + 1, c + 1)));
  for (int r = 0; r + 1 < R; ++r) for (int c = 0; c + 1 < C; ++c) L1.push_back(dist(id(r, c + 1), id(r + 1, c)));
  for (int r = 0; r < R; ++r) for (int c = 0; c + 2 < C; ++c) L1.push_back(dist(id(r, c), id(r, c + 2)));
  for (int r = 0; r + 2 < R; ++r) for (int c = 0; c < C; ++c) L1.push_back(dist(id(r, c), id(r + 2, c)));
}
template <typename R>
cs_status launch_linearize(cs_sim* s, int B, int H, const void* z, const void* v, void* A,
                           void* Bm, int32_t* status, cudaStream_t st);

}  // namespace csi
