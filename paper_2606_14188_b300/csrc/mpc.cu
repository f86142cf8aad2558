// Served plan solves: request queue, admission by device memory, the scheduler thread that runs
// the running set one evaluation ("tick") at a time on its own stream, CUDA-graph replay of a
// stable set, results delivered through stream host callbacks, per-session warm starts, and the
// warps-per-CTA autotuner of the packed launch.  Contract in include/cordsim.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <cmath>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <deque>
#include <fstream>
#include <map>
#include <memory>
#include <mutex>
#include <sstream>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "cordsim.h"
#include "internal.h"
#include "launch_plan.cuh"

namespace {

int64_t now_ns() {
  return std::chrono::duration_cast<std::chrono::nanoseconds>(
             std::chrono::steady_clock::now().time_since_epoch())
      .count();
}

constexpr size_t kAlign = 256;
size_t al(size_t x) { return (x + kAlign - 1) & ~(kAlign - 1); }

// First-fit allocator over one contiguous range (host-side bookkeeping; the range is device or
// pinned host memory owned by the server).
class Arena {
 public:
  void init(size_t bytes) {
    free_.clear();
    if (bytes) free_[0] = bytes;
  }
  bool alloc(size_t n, size_t* off) {
    for (auto it = free_.begin(); it != free_.end(); ++it) {
      if (it->second < n) continue;
      *off = it->first;
      const size_t rest = it->second - n, o = it->first + n;
      free_.erase(it);
      if (rest) free_[o] = rest;
      return true;
    }
    return false;
  }
  void release(size_t off, size_t n) {
    auto it = free_.emplace(off, n).first;
    auto nx = std::next(it);
    if (nx != free_.end() && it->first + it->second == nx->first) {
      it->second += nx->second;
      free_.erase(nx);
    }
    if (it != free_.begin()) {
      auto pv = std::prev(it);
      if (pv->first + pv->second == it->first) {
        pv->second += it->second;
        free_.erase(it);
      }
    }
  }

 private:
  std::map<size_t, size_t> free_;
};

// device layout of one request (offsets from its arena block)
struct Layout {
  size_t L1, L2, q0, warm, U, M, V, dU, L, status, ws, best, st, total;
  size_t l1_n;           // rest lengths in the L1 region (rope: 128 slots; cloth: every spring)
  size_t ws_stride;      // elements per candidate
  size_t best_bytes;     // best_u (padded) + PlanState: one D2H copy
  // pinned host staging: uploads then the result
  size_t h_L1, h_L2, h_q0, h_warm, h_res, h_total;
};

Layout make_layout(int nv, int H, int Rc, int ck, int rb, size_t l1_n) {
  Layout l{};
  const int nq = 3 * nv + 6;
  size_t o = 0;
  auto take = [&](size_t n) { const size_t at = o; o += al(n); return at; };
  l.l1_n = l1_n;
  l.L1 = take(l1_n * (size_t)rb);
  l.L2 = take(128 * (size_t)rb);
  l.q0 = take((size_t)nq * rb);
  l.warm = take((size_t)H * 6 * rb);
  const size_t nu = (size_t)Rc * H * 6 * rb;
  l.U = take(nu);
  l.M = take(nu);
  l.V = take(nu);
  l.dU = take(nu);
  l.L = take((size_t)Rc * rb);
  l.status = take((size_t)Rc * 4);
  const int nseg = (H + ck - 1) / ck;
  l.ws_stride = (size_t)(nseg + 1 + ck) * cs::rec_len(nv);
  l.ws = take((size_t)Rc * l.ws_stride * rb);
  const size_t bu = ((size_t)H * 6 * rb + 15) & ~(size_t)15;
  l.best_bytes = bu + sizeof(cs::PlanState);
  l.best = take(l.best_bytes);
  l.st = l.best + bu;
  l.total = o;
  o = 0;
  l.h_L1 = take(l1_n * (size_t)rb);
  l.h_L2 = take(128 * (size_t)rb);
  l.h_q0 = take((size_t)nq * rb);
  l.h_warm = take((size_t)H * 6 * rb);
  l.h_res = take(l.best_bytes);
  l.h_total = o;
  return l;
}

struct Req {
  uint64_t ticket = 0;
  cs_mpc_request r{};
  std::vector<double> rest, q0, warm;
  int nv = 0, nq = 0, ppl = 1;   // ppl: rope pairs per lane; 3 for a cloth
  bool cloth = false;
  cs::ClothDims cd{};
  Layout lay{};
  size_t off = 0, poff = 0;
  unsigned char* dev = nullptr;    // device block
  unsigned char* host = nullptr;   // pinned block
  const void* warm_dev = nullptr;
  int warm_H = 0, warm_shift = 0;
  int ticks = 0;
  bool admitted = false, cancelled = false, done = false, released = false;
  bool timed_out = false;          // left because its deadline passed (then cancelled too)
  cs_status err = CS_OK;
  int64_t t_submit = 0, t_start = 0, t_done = 0;
  int64_t deadline_ns = 0;         // steady-clock time after which it leaves; 0: none
};

// a request whose deadline has passed at time `now` (steady clock, ns)
inline bool deadline_passed(const Req& q, int64_t now) {
  return q.deadline_ns > 0 && !q.cancelled && !q.done && now >= q.deadline_ns;
}

struct Session {
  size_t off = 0, bytes = 0;
  int H = 0;
  bool valid = false;
  uint64_t used = 0;   // last use (for eviction)
};

}  // namespace

struct cs_mpc {
  cs_mpc_config cfg{};
  std::string tuner_path;
  int dev = 0, sms = 0, rb = 4;
  size_t smem_optin = 0;
  cudaStream_t stream = nullptr;
  unsigned char* arena_dev = nullptr;
  size_t arena_bytes = 0;
  Arena arena;
  unsigned char* pinned = nullptr;
  size_t pinned_bytes = 0;
  Arena pinned_arena;
  // job table of the running set
  size_t job_bytes = 0;
  unsigned char* d_jobs = nullptr;
  unsigned char* h_jobs = nullptr;
  int* d_first = nullptr;
  int* h_first = nullptr;
  int max_slots = 64;
  std::mutex mu;
  std::condition_variable cv;
  std::deque<std::shared_ptr<Req>> pending;
  std::vector<std::shared_ptr<Req>> running;              // scheduler thread only
  std::unordered_map<uint64_t, std::shared_ptr<Req>> tickets;
  std::unordered_map<uint64_t, Session> sessions;
  unsigned char* session_dev = nullptr;   // plans kept for sessions (own pool, least recently
  size_t session_bytes = 0;               // used evicted when full)
  Arena session_arena;
  uint64_t session_clock = 0;
  uint64_t next_ticket = 1;
  bool stop = false;
  std::thread thread;
  cs_status fatal = CS_OK;
  std::string fatal_msg;
  // tick state (scheduler thread)
  cudaGraphExec_t gexec = nullptr;
  bool graph_valid = false;
  cudaEvent_t tick_ev[2] = {nullptr, nullptr};
  bool set_dirty = false;     // the running set lost members since the last tick
  std::atomic<int64_t> ticks{0}, graph_launches{0}, kernel_launches{0}, graphs_built{0};
  int warps[3] = {1, 1, 1};   // tuned warps per CTA of the packed launch, by pairs per lane
  // cloth candidates: CTA workspace slots shared by the cloth launches of a tick (one stream)
  void* cloth_pool = nullptr;
  size_t cloth_pool_bytes = 0, cloth_stride = 0;
  int cloth_nslots = 0;
  size_t cloth_smem = 0, cloth_scene_off = 0;   // packed cloth launch: shared memory, scene copy
};

namespace {

cs_status cuda_err(cudaError_t e, const char* what) { return cs_cuda_fail(e, what); }

// ---- request validation and copies ---------------------------------------------------------

cs_status check_request(const cs_mpc* m, const cs_mpc_request* q) {
  if (q->params.second_order) return cs_fail(CS_ERR_UNSUPPORTED, "plan solves use the quasi-static step");
  const cs_params& P = q->params;
  if (!q->rest_x || !q->q0) return cs_fail(CS_ERR_INVALID_ARG, "rest_x and q0 are required");
  const bool cloth = P.kind == CS_CLOTH;
  if (P.kind != CS_ROPE && !cloth) return cs_fail(CS_ERR_INVALID_ARG, "unknown kind");
  if (!cloth && (P.n_nodes < 2 || P.n_nodes > 128)) return cs_fail(CS_ERR_INVALID_ARG, "rope n_nodes must be in [2, 128]");
  if (cloth && (P.rows < 1 || P.cols < 2 || P.rows > 256 || P.cols > 256 || P.n_nodes != P.rows * P.cols))
    return cs_fail(CS_ERR_INVALID_ARG, "cloth needs rows >= 1, cols >= 2 and n_nodes = rows * cols");
  for (int i = 0; i < 2; ++i)
    if (P.grasp_node[i] < 0 || P.grasp_node[i] >= P.n_nodes) return cs_fail(CS_ERR_INVALID_ARG, "grasp_node out of range");
  if (P.grasp_node[0] == P.grasp_node[1]) return cs_fail(CS_ERR_INVALID_ARG, "the two grippers must hold different nodes");
  if (P.n_obstacles < 0 || P.n_obstacles > CS_MAX_OBSTACLES) return cs_fail(CS_ERR_INVALID_ARG, "n_obstacles out of range");
  for (int o = 0; o < P.n_obstacles; ++o) {
    const int t = P.obstacles[o].type;
    if (t != CS_PLANE && t != CS_SPHERE && t != CS_BOX) return cs_fail(CS_ERR_INVALID_ARG, "unknown obstacle type");
  }
  if (!(P.dt > 0) || !(P.node_mass > 0)) return cs_fail(CS_ERR_INVALID_ARG, "dt and node_mass must be > 0");
  if (P.checkpoint_every < 0 || P.newton_max < 1 || P.ipm_max < 1)
    return cs_fail(CS_ERR_INVALID_ARG, "checkpoint_every must be >= 0 and iteration caps >= 1");
  if (!(P.kappa_decay > 0 && P.kappa_decay < 1)) return cs_fail(CS_ERR_INVALID_ARG, "kappa_decay must be in (0,1)");
  if (!(P.kappa_c > 0) || !(P.kappa_hard > 0) || P.kappa_hard > P.kappa_c)
    return cs_fail(CS_ERR_INVALID_ARG, "need 0 < kappa_hard <= kappa_c");
  if (q->H < 1 || q->R < 1 || q->G < 1) return cs_fail(CS_ERR_INVALID_ARG, "H, R and G must be >= 1");
  if (q->loss.n_goal < 0 || q->loss.n_goal > CS_MAX_GOAL) return cs_fail(CS_ERR_INVALID_ARG, "n_goal out of range");
  for (int g = 0; g < q->loss.n_goal; ++g)
    if (q->loss.goal_nodes[g] < 0 || q->loss.goal_nodes[g] >= P.n_nodes)
      return cs_fail(CS_ERR_INVALID_ARG, "goal node out of range");
  if (!(q->u_max > 0) || !(q->sigma >= 0) || !(q->lr >= 0)) return cs_fail(CS_ERR_INVALID_ARG, "need u_max > 0, sigma >= 0, lr >= 0");
  if (cloth) {
    cs::ClothDims d = cs::cloth_dims(P.rows, P.cols);
    if (!cs::cloth_fit(d, (size_t)m->rb, m->smem_optin))
      return cs_fail(CS_ERR_INVALID_ARG, "cloth too large for one CTA's shared memory");
    return CS_OK;
  }
  const int ppl = (P.n_nodes + 1) / 2 <= 32 ? 1 : 2;
  const size_t ws = m->rb == 4 ? csi::plan_warp_smem<float>(ppl, P.n_obstacles, q->H)
                               : csi::plan_warp_smem<double>(ppl, P.n_obstacles, q->H);
  if (ws > m->smem_optin) return cs_fail(CS_ERR_INVALID_ARG, "horizon too long for one warp's shared memory");
  return CS_OK;
}

template <typename R>
void put_real(unsigned char* dst, const double* src, size_t n) {
  R* d = reinterpret_cast<R*>(dst);
  for (size_t i = 0; i < n; ++i) d[i] = (R)src[i];
}

void stage_uploads(cs_mpc* m, Req& q) {
  const int nv = q.nv;
  std::vector<double> L1(128, 0.0), L2(128, 0.0);
  auto dist = [&](int a, int b) {
    const double* x = q.rest.data();
    const double d0 = x[3 * b] - x[3 * a], d1 = x[3 * b + 1] - x[3 * a + 1], d2 = x[3 * b + 2] - x[3 * a + 2];
    return std::sqrt(d0 * d0 + d1 * d1 + d2 * d2);
  };
  if (q.cloth) {
    csi::cloth_rest_lengths(q.r.params.rows, q.r.params.cols, q.rest.data(), L1);
  } else {
    for (int j = 0; j + 1 < nv; ++j) L1[j] = dist(j, j + 1);
    for (int j = 0; j + 2 < nv; ++j) L2[j] = dist(j, j + 2);
  }
  auto put = [&](size_t off, const double* src, size_t n) {
    if (m->rb == 4) put_real<float>(q.host + off, src, n);
    else put_real<double>(q.host + off, src, n);
  };
  put(q.lay.h_L1, L1.data(), q.lay.l1_n);
  put(q.lay.h_L2, L2.data(), 128);
  put(q.lay.h_q0, q.q0.data(), q.q0.size());
  if (!q.warm.empty()) put(q.lay.h_warm, q.warm.data(), q.warm.size());
}

cs_status enqueue_uploads(cs_mpc* m, Req& q) {
  const Layout& l = q.lay;
  const size_t rb = (size_t)m->rb;
  struct C { size_t d, h, n; } cps[4] = {{l.L1, l.h_L1, l.l1_n * rb}, {l.L2, l.h_L2, 128 * rb},
                                         {l.q0, l.h_q0, (size_t)q.nq * rb},
                                         {l.warm, l.h_warm, q.warm.empty() ? 0 : (size_t)q.r.H * 6 * rb}};
  for (const C& c : cps) {
    if (!c.n) continue;
    cudaError_t e = cudaMemcpyAsync(q.dev + c.d, q.host + c.h, c.n, cudaMemcpyHostToDevice, m->stream);
    if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync");
  }
  return CS_OK;
}

csi::PlanSpec make_spec(const cs_mpc* m, const Req& q) {
  csi::PlanSpec p{};
  const Layout& l = q.lay;
  p.P = q.r.params;
  p.loss = q.r.loss;
  p.L1 = q.dev + l.L1;
  p.L2 = q.dev + l.L2;
  p.q0 = q.dev + l.q0;
  p.warm = q.warm_dev;
  p.U = q.dev + l.U;
  p.M = q.dev + l.M;
  p.V = q.dev + l.V;
  p.dU = q.dev + l.dU;
  p.L = q.dev + l.L;
  p.status = reinterpret_cast<int32_t*>(q.dev + l.status);
  p.ws = q.dev + l.ws;
  p.best_u = q.dev + l.best;
  p.st = reinterpret_cast<cs::PlanState*>(q.dev + l.st);
  p.ws_stride = l.ws_stride;
  p.seed = (unsigned long long)q.r.seed;
  p.H = q.r.H;
  p.Rc = q.r.R;
  p.G = q.r.G;
  p.warm_H = q.warm_H;
  p.warm_shift = q.warm_shift;
  p.cloth_wg = q.cloth ? q.cd.win_global : 0;
  p.lr = q.r.lr;
  p.sigma = q.r.sigma;
  p.u_max = q.r.u_max;
  (void)m;
  return p;
}

// ---- one tick ------------------------------------------------------------------------------

struct Group {
  int j0 = 0, n = 0, total = 0, nobs = 0, H = 0;
};

// offset of the cloth group's candidate offsets in the first[] table (after the two rope groups)
inline int cloth_first_base(const Group g[3]) { return g[1].n + 1 + g[2].n + 1; }

template <typename R>
cs_status enqueue_tick(cs_mpc* m, const Group g[3], const Group& cg, int njobs, int max_elems, bool count) {
  cs_status r;
  for (int ppl = 1; ppl <= 2; ++ppl) {
    const Group& G = g[ppl];
    if (!G.n) continue;
    const size_t ws = csi::plan_warp_smem<R>(ppl, G.nobs, G.H);
    int warps = m->warps[ppl];
    while (warps > 1 && ws * warps > m->smem_optin) warps >>= 1;
    const int grid = (G.total + warps - 1) / warps;
    r = csi::launch_plan_vjp<R>(m->d_jobs + (size_t)G.j0 * m->job_bytes, m->d_first + (ppl == 1 ? 0 : g[1].n + 1),
                                G.n, G.total, ppl, warps, ws, grid, m->stream);
    if (r) return r;
    if (count) ++m->kernel_launches;
  }
  // cloth requests: one packed launch over the candidates of all of them
  if (cg.n) {
    r = csi::launch_cloth_packed<R>(m->d_jobs + (size_t)cg.j0 * m->job_bytes, m->d_first + cloth_first_base(g), cg.n,
                                    cg.total, m->cloth_pool, m->cloth_stride, m->cloth_nslots, m->cloth_smem,
                                    m->cloth_scene_off, m->stream);
    if (r) return r;
    if (count) ++m->kernel_launches;
  }
  if ((r = csi::launch_plan_select<R>(m->d_jobs, njobs, m->stream))) return r;
  if ((r = csi::launch_plan_adam<R>(m->d_jobs, njobs, max_elems, m->stream))) return r;
  if (count) m->kernel_launches += 2;
  return CS_OK;
}

template <typename R>
cs_status prepare_groups(cs_mpc* m, const Group g[3]) {
  for (int ppl = 1; ppl <= 2; ++ppl) {
    if (!g[ppl].n) continue;
    const size_t ws = csi::plan_warp_smem<R>(ppl, g[ppl].nobs, g[ppl].H);
    int warps = m->warps[ppl];
    while (warps > 1 && ws * warps > m->smem_optin) warps >>= 1;
    cs_status r = csi::plan_prepare<R>(ppl, ws * warps);
    if (r) return r;
  }
  return CS_OK;
}

// the packed cloth kernel's shared memory (the widest running cloth's layout, then the scene copy)
// and a workspace pool of one slot per resident CTA, grown (after the stream drains) when a wider
// cloth joins
template <typename R>
cs_status prepare_cloth(cs_mpc* m, const Group& cg) {
  if (!cg.n) return CS_OK;
  size_t lay = 0, stride = 0;
  for (int j = cg.j0; j < cg.j0 + cg.n; ++j) {
    const Req& q = *m->running[j];
    lay = std::max(lay, cs::cloth_smem_elems(q.cd) * sizeof(R));
    stride = std::max(stride, cs::cloth_ws_elems(q.cd, q.r.params.n_obstacles));
  }
  const size_t scene_off = (lay + 15) & ~(size_t)15;
  const size_t smem = scene_off + cs::plan_scene_bytes<R>();
  if (smem > m->smem_optin) return cs_fail(CS_ERR_INVALID_ARG, "cloth too large for the packed launch");
  int per_sm = 1;
  cs_status r = csi::cloth_packed_prepare<R>(smem, &per_sm);
  if (r) return r;
  const int nslots = per_sm * m->sms;
  const size_t bytes = stride * (size_t)nslots * sizeof(R);
  if (bytes > m->cloth_pool_bytes) {
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_err(e, "cudaStreamSynchronize");
    if (m->cloth_pool) cudaFree(m->cloth_pool);
    m->cloth_pool = nullptr;
    m->cloth_pool_bytes = 0;
    e = cudaMalloc(&m->cloth_pool, bytes);
    if (e != cudaSuccess) return e == cudaErrorMemoryAllocation ? cs_fail(CS_ERR_OOM, "cloth workspace") : cuda_err(e, "cudaMalloc");
    m->cloth_pool_bytes = bytes;
  }
  m->cloth_stride = stride;
  m->cloth_nslots = nslots;
  m->cloth_smem = smem;
  m->cloth_scene_off = scene_off;
  return CS_OK;
}

void CUDART_CB on_result(void* arg);

struct DoneCtx {
  cs_mpc* m;
  std::shared_ptr<Req> q;
};

template <typename R>
cs_status run_tick(cs_mpc* m, const std::vector<std::shared_ptr<Req>>& admitted, bool changed) {
  auto& run = m->running;
  const int n = (int)run.size();
  Group g[3];
  int max_elems = 0;
  if (changed) {
    // running set: pairs-per-lane 1 first, then 2
    std::stable_sort(run.begin(), run.end(), [](const std::shared_ptr<Req>& a, const std::shared_ptr<Req>& b) {
      return a->ppl < b->ppl;
    });
    // the pinned job table may still feed an earlier copy
    cudaError_t e = cudaStreamSynchronize(m->stream);
    if (e != cudaSuccess) return cuda_err(e, "cudaStreamSynchronize");
  }
  int first1 = 0, first2 = 0;
  Group cg;                              // cloth requests (last in the sorted running set)
  for (int j = 0; j < n; ++j) {
    const Req& q = *run[j];
    if (q.cloth) {
      if (!cg.n) cg.j0 = j;
      ++cg.n;
      cg.total += q.r.R;
      max_elems = std::max(max_elems, q.r.R * q.r.H * 6);
      if (changed) csi::plan_fill_job<R>(m->h_jobs + (size_t)j * m->job_bytes, make_spec(m, q));
      continue;
    }
    Group& G = g[q.ppl];
    if (!G.n) G.j0 = j;
    ++G.n;
    G.total += q.r.R;
    G.nobs = std::max(G.nobs, q.r.params.n_obstacles);
    G.H = std::max(G.H, q.r.H);
    max_elems = std::max(max_elems, q.r.R * q.r.H * 6);
    if (changed) {
      csi::plan_fill_job<R>(m->h_jobs + (size_t)j * m->job_bytes, make_spec(m, q));
      if (q.ppl == 1) m->h_first[G.n - 1] = first1, first1 += q.r.R;
      else m->h_first[g[1].n + 1 + G.n - 1] = first2, first2 += q.r.R;
    }
  }
  cs_status r;
  if (changed) {
    m->h_first[g[1].n] = first1;
    m->h_first[g[1].n + 1 + g[2].n] = first2;
    const int cb = cloth_first_base(g);
    int first3 = 0;
    for (int k = 0; k < cg.n; ++k) {
      m->h_first[cb + k] = first3;
      first3 += run[cg.j0 + k]->r.R;
    }
    m->h_first[cb + cg.n] = first3;
    cudaError_t e = cudaMemcpyAsync(m->d_jobs, m->h_jobs, (size_t)n * m->job_bytes, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(m->d_first, m->h_first, sizeof(int) * (size_t)(cb + cg.n + 1), cudaMemcpyHostToDevice,
                          m->stream);
    if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync");
    for (const auto& q : admitted) {
      int j = 0;
      while (run[j] != q) ++j;
      if ((r = csi::launch_plan_init<R>(m->d_jobs, j, 1, q->r.R * q->r.H * 6, m->stream))) return r;
      ++m->kernel_launches;
    }
    if ((r = prepare_groups<R>(m, g))) return r;
    if ((r = prepare_cloth<R>(m, cg))) return r;
    m->graph_valid = false;
  }
  // at most two ticks in flight
  cudaEvent_t ev = m->tick_ev[m->ticks & 1];
  cudaError_t e = cudaEventSynchronize(ev);
  if (e != cudaSuccess) return cuda_err(e, "cudaEventSynchronize");
  if (m->cfg.use_graphs && m->cfg.batched) {
    if (!m->graph_valid) {
      if (m->gexec) cudaGraphExecDestroy(m->gexec);
      m->gexec = nullptr;
      cudaGraph_t graph = nullptr;
      e = cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal);
      if (e != cudaSuccess) return cuda_err(e, "cudaStreamBeginCapture");
      r = enqueue_tick<R>(m, g, cg, n, max_elems, false);
      e = cudaStreamEndCapture(m->stream, &graph);
      if (r) return r;
      if (e != cudaSuccess) return cuda_err(e, "cudaStreamEndCapture");
      e = cudaGraphInstantiate(&m->gexec, graph, 0);
      cudaGraphDestroy(graph);
      if (e != cudaSuccess) return cuda_err(e, "cudaGraphInstantiate");
      m->graph_valid = true;
      ++m->graphs_built;
    }
    e = cudaGraphLaunch(m->gexec, m->stream);
    if (e != cudaSuccess) return cuda_err(e, "cudaGraphLaunch");
    ++m->graph_launches;
    m->kernel_launches += (g[1].n ? 1 : 0) + (g[2].n ? 1 : 0) + (cg.n ? 1 : 0) + 2;
  } else {
    if ((r = enqueue_tick<R>(m, g, cg, n, max_elems, true))) return r;
  }
  e = cudaEventRecord(ev, m->stream);
  if (e != cudaSuccess) return cuda_err(e, "cudaEventRecord");
  ++m->ticks;
  // finished requests: result to the host, session plan kept on the device, then a callback
  for (auto& q : run) {
    if (++q->ticks < q->r.G) continue;
    e = cudaMemcpyAsync(q->host + q->lay.h_res, q->dev + q->lay.best, q->lay.best_bytes, cudaMemcpyDeviceToHost,
                        m->stream);
    if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync");
    if (q->r.session_id) {
      std::lock_guard<std::mutex> lk(m->mu);
      Session& s = m->sessions[q->r.session_id];
      const size_t need = al((size_t)q->r.H * 6 * m->rb);
      if (s.valid && s.bytes != need) {
        m->session_arena.release(s.off, s.bytes);
        s.valid = false;
      }
      while (!s.valid && !m->session_arena.alloc(need, &s.off)) {
        // evict the least recently used other session (stream order keeps its readers first)
        Session* lru = nullptr;
        for (auto& kv : m->sessions)
          if (kv.second.valid && &kv.second != &s && (!lru || kv.second.used < lru->used)) lru = &kv.second;
        if (!lru) break;
        m->session_arena.release(lru->off, lru->bytes);
        lru->valid = false;
      }
      if (!s.valid && m->session_arena.alloc(need, &s.off)) s.valid = true;
      if (s.valid) {
        s.bytes = need;
        s.H = q->r.H;
        s.used = ++m->session_clock;
        e = cudaMemcpyAsync(m->session_dev + s.off, q->dev + q->lay.best, (size_t)q->r.H * 6 * m->rb,
                            cudaMemcpyDeviceToDevice, m->stream);
        if (e != cudaSuccess) return cuda_err(e, "cudaMemcpyAsync");
      }
    }
    e = cudaLaunchHostFunc(m->stream, on_result, new DoneCtx{m, q});
    if (e != cudaSuccess) return cuda_err(e, "cudaLaunchHostFunc");
  }
  return CS_OK;
}

void release_locked(cs_mpc* m, Req& q) {
  if (q.released) return;
  q.released = true;
  if (q.admitted) m->arena.release(q.off, q.lay.total);
}

void CUDART_CB on_result(void* arg) {
  DoneCtx* c = static_cast<DoneCtx*>(arg);
  {
    std::lock_guard<std::mutex> lk(c->m->mu);
    c->q->done = true;
    c->q->t_done = now_ns();
    release_locked(c->m, *c->q);
  }
  c->m->cv.notify_all();
  delete c;
}

void CUDART_CB on_dropped(void* arg) {
  DoneCtx* c = static_cast<DoneCtx*>(arg);
  {
    std::lock_guard<std::mutex> lk(c->m->mu);
    release_locked(c->m, *c->q);
  }
  c->m->cv.notify_all();
  delete c;
}

void fail_all(cs_mpc* m, cs_status s) {
  std::lock_guard<std::mutex> lk(m->mu);
  m->fatal = s;
  m->fatal_msg = cs_last_error();
  for (auto& kv : m->tickets)
    if (!kv.second->done) kv.second->err = s;
  m->cv.notify_all();
}

void scheduler(cs_mpc* m) {
  cudaSetDevice(m->dev);
  while (true) {
    std::vector<std::shared_ptr<Req>> admitted, dropped;
    bool changed = m->set_dirty;
    m->set_dirty = false;
    {
      std::unique_lock<std::mutex> lk(m->mu);
      m->cv.wait(lk, [&] { return m->stop || !m->pending.empty() || !m->running.empty(); });
      if (m->stop) break;
      // deadlines: a queued or running request past its deadline leaves like a cancelled one
      // (at this tick boundary) and its poll reports CS_ERR_TIMEOUT
      {
        const int64_t now = now_ns();
        bool expired = false;
        for (auto& q : m->running)
          if (deadline_passed(*q, now)) { q->cancelled = q->timed_out = true; expired = true; }
        for (auto& q : m->pending)
          if (deadline_passed(*q, now)) { q->cancelled = q->timed_out = true; expired = true; }
        if (expired) m->cv.notify_all();
      }
      for (auto it = m->running.begin(); it != m->running.end();) {
        if ((*it)->cancelled) {
          dropped.push_back(*it);
          it = m->running.erase(it);
          changed = true;
        } else {
          ++it;
        }
      }
      const size_t cap = m->cfg.batched ? (size_t)m->max_slots : 1;
      while (!m->pending.empty() && m->running.size() < cap) {
        std::shared_ptr<Req> q = m->pending.front();
        if (q->cancelled) { m->pending.pop_front(); continue; }
        size_t off = 0;
        if (!m->arena.alloc(q->lay.total, &off)) break;
        q->off = off;
        q->dev = m->arena_dev + off;
        q->admitted = true;
        q->t_start = now_ns();
        // warm start: the request's own, else its session's last plan shifted by one step
        if (!q->warm.empty()) {
          q->warm_dev = q->dev + q->lay.warm;
          q->warm_H = q->r.H;
          q->warm_shift = 0;
        } else if (q->r.session_id) {
          auto s = m->sessions.find(q->r.session_id);
          if (s != m->sessions.end() && s->second.valid) {
            q->warm_dev = m->session_dev + s->second.off;
            q->warm_H = s->second.H;
            q->warm_shift = 1;
            s->second.used = ++m->session_clock;
          }
        }
        m->pending.pop_front();
        m->running.push_back(q);
        admitted.push_back(q);
        changed = true;
      }
      if (m->running.empty() && dropped.empty()) continue;
    }
    cs_status r = CS_OK;
    for (auto& q : dropped) {
      cudaError_t e = cudaLaunchHostFunc(m->stream, on_dropped, new DoneCtx{m, q});
      if (e != cudaSuccess) { r = cuda_err(e, "cudaLaunchHostFunc"); break; }
    }
    for (auto& q : admitted) {
      if (r) break;
      r = enqueue_uploads(m, *q);
    }
    if (!r && !m->running.empty())
      r = m->rb == 4 ? run_tick<float>(m, admitted, changed) : run_tick<double>(m, admitted, changed);
    if (r) {
      fail_all(m, r);
      break;
    }
    // requests that got their last evaluation leave the running set
    bool left = false;
    for (auto it = m->running.begin(); it != m->running.end();) {
      if ((*it)->ticks >= (*it)->r.G) { it = m->running.erase(it); left = true; } else ++it;
    }
    if (left) m->set_dirty = true;
  }
}

// ---- autotuner -----------------------------------------------------------------------------
// Times the packed launch with 1, 2 and 4 warps per CTA on a synthetic running set (straight
// ropes of 64 and 128 nodes above a ground plane, horizon 16, 2 x SMs candidates each) and keeps
// the fastest per pairs-per-lane.  Results are cached in a text file, one line per
// (device, real type, pairs per lane): "<device>|<real bytes>|<ppl> <warps>".

std::string device_name(int dev) {
  cudaDeviceProp p;
  if (cudaGetDeviceProperties(&p, dev) != cudaSuccess) return "unknown";
  std::string s = p.name;
  for (char& c : s)
    if (c == '|' || c == ' ') c = '_';
  return s;
}

void load_tuning(cs_mpc* m, bool found[3]) {
  found[1] = found[2] = false;
  if (m->tuner_path.empty()) return;
  std::ifstream f(m->tuner_path);
  std::string line, key = device_name(m->dev) + "|" + std::to_string(m->rb) + "|";
  while (std::getline(f, line)) {
    if (line.compare(0, key.size(), key) != 0) continue;
    std::istringstream is(line.substr(key.size()));
    int ppl = 0, w = 0;
    if (is >> ppl >> w && (ppl == 1 || ppl == 2) && (w == 1 || w == 2 || w == 4)) {
      m->warps[ppl] = w;
      found[ppl] = true;
    }
  }
}

void save_tuning(cs_mpc* m) {
  if (m->tuner_path.empty()) return;
  std::vector<std::string> keep;
  std::string key = device_name(m->dev) + "|" + std::to_string(m->rb) + "|";
  {
    std::ifstream f(m->tuner_path);
    std::string line;
    while (std::getline(f, line))
      if (line.compare(0, key.size(), key) != 0 && !line.empty()) keep.push_back(line);
  }
  std::ofstream f(m->tuner_path, std::ios::trunc);
  for (auto& l : keep) f << l << "\n";
  for (int ppl = 1; ppl <= 2; ++ppl) f << key << ppl << " " << m->warps[ppl] << "\n";
}

template <typename R>
cs_status tune(cs_mpc* m) {
  const int H = 16, Rc = 2 * m->sms;
  for (int ppl = 1; ppl <= 2; ++ppl) {
    const int nv = ppl == 1 ? 64 : 128;
    cs_params P{};
    P.kind = CS_ROPE;
    P.n_nodes = nv;
    P.grasp_node[0] = 0;
    P.grasp_node[1] = nv - 1;
    P.dt = 0.01;
    P.gravity[2] = -9.81;
    P.node_mass = 0.1 / nv;
    P.k_stretch = 500;
    P.k_shear = 250;
    P.k_bend = 25;
    P.D_max = 1e4;
    P.kappa_h = 0.01;
    P.kappa_c = 1e-4;
    P.kappa_hard = 1e-6;
    P.kappa_decay = 0.2;
    P.mu = 0.5;
    P.r_grasp = 0.01;
    P.node_radius = 0.005;
    P.sigma0 = 1e-3;
    P.n_obstacles = 1;
    P.obstacles[0].type = CS_PLANE;
    P.obstacles[0].p[2] = 1.0;
    P.newton_max = 40;
    P.ipm_max = 80;
    P.newton_tol = 1e-5;
    P.ipm_tol = 1e-6;
    P.checkpoint_every = 4;
    Req q;
    q.nv = nv;
    q.nq = 3 * nv + 6;
    q.r.params = P;
    q.r.H = H;
    q.r.R = Rc;
    q.r.G = 1;
    q.r.u_max = 0.05;
    q.r.sigma = 0.02;
    q.lay = make_layout(nv, H, Rc, P.checkpoint_every, m->rb, 128);
    q.rest.resize(3 * nv);
    q.q0.resize(q.nq);
    for (int j = 0; j < nv; ++j) {
      q.rest[3 * j] = 0.1 + 0.8 * j / (nv - 1);
      q.rest[3 * j + 2] = 0.3;
    }
    for (int i = 0; i < 3 * nv; ++i) q.q0[i] = q.rest[i];
    for (int i = 0; i < 3; ++i) {
      q.q0[3 * nv + i] = q.rest[i];
      q.q0[3 * nv + 3 + i] = q.rest[3 * (nv - 1) + i];
    }
    size_t off = 0, poff = 0;
    if (!m->arena.alloc(q.lay.total, &off)) continue;          // no room to tune: keep 1
    if (!m->pinned_arena.alloc(q.lay.h_total, &poff)) {
      m->arena.release(off, q.lay.total);
      continue;
    }
    q.dev = m->arena_dev + off;
    q.host = m->pinned + poff;
    stage_uploads(m, q);
    cs_status r = enqueue_uploads(m, q);
    csi::plan_fill_job<R>(m->h_jobs, make_spec(m, q));
    m->h_first[0] = 0;
    m->h_first[1] = Rc;
    cudaError_t e = cudaMemcpyAsync(m->d_jobs, m->h_jobs, m->job_bytes, cudaMemcpyHostToDevice, m->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(m->d_first, m->h_first, 2 * sizeof(int), cudaMemcpyHostToDevice, m->stream);
    if (!r && e != cudaSuccess) r = cuda_err(e, "cudaMemcpyAsync");
    if (!r) r = csi::launch_plan_init<R>(m->d_jobs, 0, 1, Rc * H * 6, m->stream);
    const size_t ws = csi::plan_warp_smem<R>(ppl, 1, H);
    float best = 1e30f;
    int bestw = 1;
    cudaEvent_t a = nullptr, b = nullptr;
    if (!r) {
      cudaEventCreate(&a);
      cudaEventCreate(&b);
    }
    for (int w = 1; w <= 4 && !r; w *= 2) {
      if (ws * w > m->smem_optin) break;
      if ((r = csi::plan_prepare<R>(ppl, ws * w))) break;
      const int grid = (Rc + w - 1) / w;
      if ((r = csi::launch_plan_vjp<R>(m->d_jobs, m->d_first, 1, Rc, ppl, w, ws, grid, m->stream))) break;
      cudaEventRecord(a, m->stream);
      for (int rep = 0; rep < 2 && !r; ++rep)
        r = csi::launch_plan_vjp<R>(m->d_jobs, m->d_first, 1, Rc, ppl, w, ws, grid, m->stream);
      cudaEventRecord(b, m->stream);
      e = cudaEventSynchronize(b);
      if (!r && e != cudaSuccess) r = cuda_err(e, "cudaEventSynchronize");
      float ms = 0;
      cudaEventElapsedTime(&ms, a, b);
      if (!r && ms < best) { best = ms; bestw = w; }
    }
    if (a) cudaEventDestroy(a);
    if (b) cudaEventDestroy(b);
    cudaStreamSynchronize(m->stream);
    m->arena.release(off, q.lay.total);
    m->pinned_arena.release(poff, q.lay.h_total);
    if (r) return r;
    m->warps[ppl] = bestw;
  }
  return CS_OK;
}

void destroy_resources(cs_mpc* m) {
  if (m->stream) cudaStreamSynchronize(m->stream);
  if (m->gexec) cudaGraphExecDestroy(m->gexec);
  for (auto& e : m->tick_ev)
    if (e) cudaEventDestroy(e);
  if (m->arena_dev) cudaFree(m->arena_dev);
  if (m->session_dev) cudaFree(m->session_dev);
  if (m->d_jobs) cudaFree(m->d_jobs);
  if (m->d_first) cudaFree(m->d_first);
  if (m->pinned) cudaFreeHost(m->pinned);
  if (m->h_jobs) cudaFreeHost(m->h_jobs);
  if (m->h_first) cudaFreeHost(m->h_first);
  if (m->cloth_pool) cudaFree(m->cloth_pool);
  if (m->stream) cudaStreamDestroy(m->stream);
}

}  // namespace

extern "C" {

cs_status mpc_create(const cs_mpc_config* cfg, cs_mpc** out) {
  if (!cfg || !out) return cs_fail(CS_ERR_INVALID_ARG, "null argument");
  *out = nullptr;
  if (cfg->real_bytes != 4 && cfg->real_bytes != 8) return cs_fail(CS_ERR_INVALID_ARG, "real_bytes must be 4 or 8");
  if (cfg->max_slots < 0) return cs_fail(CS_ERR_INVALID_ARG, "max_slots must be >= 0");
  std::unique_ptr<cs_mpc> m(new cs_mpc());
  m->cfg = *cfg;
  if (cfg->tuner_cache) m->tuner_path = cfg->tuner_cache;
  m->cfg.tuner_cache = nullptr;
  m->rb = cfg->real_bytes;
  m->max_slots = cfg->max_slots ? cfg->max_slots : 64;
  cudaError_t e = cudaGetDevice(&m->dev);
  if (e != cudaSuccess) return cuda_err(e, "cudaGetDevice");
  int v = 0;
  cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, m->dev);
  m->sms = v;
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->dev);
  m->smem_optin = (size_t)v;
  size_t free_b = 0, total_b = 0;
  if ((e = cudaMemGetInfo(&free_b, &total_b)) != cudaSuccess) return cuda_err(e, "cudaMemGetInfo");
  m->arena_bytes = cfg->mem_budget_bytes ? cfg->mem_budget_bytes : free_b / 2;
  m->arena_bytes &= ~(kAlign - 1);
  if (m->arena_bytes < (1u << 20)) return cs_fail(CS_ERR_INVALID_ARG, "memory budget below 1 MiB");
  if (m->arena_bytes > free_b) return cs_fail(CS_ERR_OOM, "memory budget above the free device memory");
  m->job_bytes = m->rb == 4 ? csi::plan_job_bytes<float>() : csi::plan_job_bytes<double>();
  m->job_bytes = (m->job_bytes + 15) & ~(size_t)15;
  m->pinned_bytes = (size_t)64 << 20;
  auto fail = [&](cudaError_t er, const char* what) {
    destroy_resources(m.get());
    return er == cudaErrorMemoryAllocation ? cs_fail(CS_ERR_OOM, what) : cuda_err(er, what);
  };
  if ((e = cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking)) != cudaSuccess) return fail(e, "cudaStreamCreate");
  for (auto& ev : m->tick_ev)
    if ((e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming)) != cudaSuccess) return fail(e, "cudaEventCreate");
  if ((e = cudaMalloc(&m->arena_dev, m->arena_bytes)) != cudaSuccess) return fail(e, "device arena");
  m->session_bytes = (size_t)16 << 20;
  if ((e = cudaMalloc(&m->session_dev, m->session_bytes)) != cudaSuccess) return fail(e, "session plans");
  if ((e = cudaMalloc(&m->d_jobs, m->job_bytes * m->max_slots)) != cudaSuccess) return fail(e, "job table");
  if ((e = cudaMalloc(&m->d_first, sizeof(int) * (m->max_slots + 3))) != cudaSuccess) return fail(e, "job table");
  if ((e = cudaHostAlloc(&m->pinned, m->pinned_bytes, cudaHostAllocDefault)) != cudaSuccess) return fail(e, "pinned staging");
  if ((e = cudaHostAlloc(&m->h_jobs, m->job_bytes * m->max_slots, cudaHostAllocDefault)) != cudaSuccess) return fail(e, "pinned job table");
  if ((e = cudaHostAlloc(&m->h_first, sizeof(int) * (m->max_slots + 3), cudaHostAllocDefault)) != cudaSuccess) return fail(e, "pinned job table");
  m->arena.init(m->arena_bytes);
  m->pinned_arena.init(m->pinned_bytes);
  m->session_arena.init(m->session_bytes);
  bool found[3];
  load_tuning(m.get(), found);
  if (cfg->autotune && !(found[1] && found[2])) {
    cs_status r = m->rb == 4 ? tune<float>(m.get()) : tune<double>(m.get());
    if (r) { destroy_resources(m.get()); return r; }
    save_tuning(m.get());
  }
  cs_mpc* raw = m.release();
  raw->thread = std::thread(scheduler, raw);
  *out = raw;
  return CS_OK;
}

cs_status mpc_submit(cs_mpc* m, const cs_mpc_request* req, uint64_t* ticket) {
  if (!m || !req || !ticket) return cs_fail(CS_ERR_INVALID_ARG, "null argument");
  cs_status r = check_request(m, req);
  if (r) return r;
  auto q = std::make_shared<Req>();
  q->r = *req;
  q->nv = req->params.n_nodes;
  q->nq = 3 * q->nv + 6;
  q->ppl = (q->nv + 1) / 2 <= 32 ? 1 : 2;
  size_t l1_n = 128;
  if (req->params.kind == CS_CLOTH) {
    q->cloth = true;
    q->ppl = 3;                      // after the rope groups in the running set
    q->cd = cs::cloth_dims(req->params.rows, req->params.cols);
    cs::cloth_fit(q->cd, (size_t)m->rb, m->smem_optin);
    l1_n = (size_t)q->cd.nspr;
  }
  q->rest.assign(req->rest_x, req->rest_x + 3 * q->nv);
  q->q0.assign(req->q0, req->q0 + q->nq);
  if (req->warm) q->warm.assign(req->warm, req->warm + 6 * (size_t)req->H);
  q->r.rest_x = q->r.q0 = q->r.warm = nullptr;
  if (q->r.params.checkpoint_every == 0) {
    // automatic: the smallest interval whose candidates' records fit in an eighth of the memory
    // budget, at most about sqrt(H); the result is the same for every interval, only the
    // recomputed steps and the memory differ
    const int kmax = std::max(1, (int)std::lround(std::sqrt((double)req->H)));
    int k = 1;
    while (k < kmax && make_layout(q->nv, req->H, req->R, k, m->rb, l1_n).total > m->arena_bytes / 8) ++k;
    q->r.params.checkpoint_every = k;
  }
  q->lay = make_layout(q->nv, req->H, req->R, q->r.params.checkpoint_every, m->rb, l1_n);
  if (q->lay.total > m->arena_bytes) return cs_fail(CS_ERR_INVALID_ARG, "request larger than the memory budget");
  if (q->lay.h_total > m->pinned_bytes) return cs_fail(CS_ERR_INVALID_ARG, "request larger than the staging memory");
  if (req->deadline_ms < 0) return cs_fail(CS_ERR_INVALID_ARG, "deadline_ms must be >= 0");
  q->t_submit = now_ns();
  if (req->deadline_ms > 0) q->deadline_ns = q->t_submit + (int64_t)req->deadline_ms * 1000000;
  {
    std::unique_lock<std::mutex> lk(m->mu);
    if (m->fatal) return cs_fail(m->fatal, "server failed: " + m->fatal_msg);
    // pinned staging, waiting while finished results hold it
    size_t poff = 0;
    while (!m->pinned_arena.alloc(q->lay.h_total, &poff)) {
      if (m->fatal) return cs_fail(m->fatal, "server failed: " + m->fatal_msg);
      m->cv.wait_for(lk, std::chrono::milliseconds(5));
    }
    q->poff = poff;
    q->host = m->pinned + poff;
    stage_uploads(m, *q);
    q->ticket = m->next_ticket++;
    m->tickets[q->ticket] = q;
    m->pending.push_back(q);
    *ticket = q->ticket;
  }
  m->cv.notify_all();
  return CS_OK;
}

cs_status mpc_poll(cs_mpc* m, uint64_t ticket, int timeout_ms, cs_mpc_result* out) {
  if (!m) return cs_fail(CS_ERR_INVALID_ARG, "null handle");
  std::unique_lock<std::mutex> lk(m->mu);
  auto it = m->tickets.find(ticket);
  if (it == m->tickets.end()) return cs_fail(CS_ERR_INVALID_ARG, "unknown ticket");
  std::shared_ptr<Req> q = it->second;
  auto ready = [&] { return q->done || q->err || (q->cancelled && !q->admitted) || (q->cancelled && q->released); };
  if (!ready()) {
    if (timeout_ms < 0) m->cv.wait(lk, ready);
    else if (timeout_ms > 0) m->cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
  }
  if (q->err) {
    m->tickets.erase(it);
    return cs_fail(q->err, "server failed: " + m->fatal_msg);
  }
  if (q->cancelled && !q->done) {
    if (!ready()) return cs_fail(CS_ERR_PENDING, "cancellation in progress");
    m->pinned_arena.release(q->poff, q->lay.h_total);
    const bool timed_out = q->timed_out;
    m->tickets.erase(it);
    if (timed_out) return cs_fail(CS_ERR_TIMEOUT, "deadline passed before the plan finished");
    return cs_fail(CS_ERR_CANCELLED, "cancelled");
  }
  if (!q->done) return cs_fail(CS_ERR_PENDING, "not done");
  if (!out) return cs_fail(CS_ERR_INVALID_ARG, "null result");
  const unsigned char* res = q->host + q->lay.h_res;
  const size_t bu = ((size_t)q->r.H * 6 * m->rb + 15) & ~(size_t)15;
  cs::PlanState ps;
  std::memcpy(&ps, res + bu, sizeof(ps));
  if (out->u)
    for (int i = 0; i < q->r.H * 6; ++i)
      out->u[i] = m->rb == 4 ? (double)reinterpret_cast<const float*>(res)[i] : reinterpret_cast<const double*>(res)[i];
  out->L = ps.best_it > 0 ? ps.best_L : std::nan("");
  out->status = ps.best_it > 0 ? 0 : (ps.flags ? ps.flags : CS_ST_NONFINITE);
  out->best_iter = ps.best_it;
  out->best_candidate = ps.best_r;
  out->t_submit_ns = q->t_submit;
  out->t_start_ns = q->t_start;
  out->t_done_ns = q->t_done;
  m->pinned_arena.release(q->poff, q->lay.h_total);
  m->tickets.erase(it);
  m->cv.notify_all();
  return CS_OK;
}

cs_status mpc_cancel(cs_mpc* m, uint64_t ticket) {
  if (!m) return cs_fail(CS_ERR_INVALID_ARG, "null handle");
  {
    std::lock_guard<std::mutex> lk(m->mu);
    auto it = m->tickets.find(ticket);
    if (it == m->tickets.end()) return cs_fail(CS_ERR_INVALID_ARG, "unknown ticket");
    if (it->second->done) return CS_OK;   // too late: the result stays available
    it->second->cancelled = true;
  }
  m->cv.notify_all();
  return CS_OK;
}

cs_status mpc_destroy(cs_mpc* m) {
  if (!m) return CS_OK;
  {
    std::lock_guard<std::mutex> lk(m->mu);
    m->stop = true;
  }
  m->cv.notify_all();
  if (m->thread.joinable()) m->thread.join();
  destroy_resources(m);
  delete m;
  return CS_OK;
}

cs_status mpc_stats(cs_mpc* m, int64_t* ticks, int64_t* graph_launches, int64_t* kernel_launches,
                    int64_t* graphs_built) {
  if (!m) return cs_fail(CS_ERR_INVALID_ARG, "null handle");
  std::lock_guard<std::mutex> lk(m->mu);
  if (ticks) *ticks = m->ticks;
  if (graph_launches) *graph_launches = m->graph_launches;
  if (kernel_launches) *kernel_launches = m->kernel_launches;
  if (graphs_built) *graphs_built = m->graphs_built;
  return CS_OK;
}

}  // extern "C"
