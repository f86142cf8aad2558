/*
 * cordsim.h -- C ABI of the B300-native contact-smoothed differentiable rope/cloth simulator.
 *
 * The library implements the simulator of arxiv 2606.14188, Sec. 4.1 ("Differentiable Deformable
 * Object Simulator with Contact Smoothing") and the calls its planners make (Sec. 3, Problem 1:
 * q_{k+1} = f(q_k, u_k); Sec. 4.2: the linearisation A(z,v), B(z,v); Sec. 4.1 eq. (diff-sim):
 * the adjoint dL/dtheta).
 *
 * Conventions for every entry point
 *   - State layout (Sec. 4.1): q = [x_0 .. x_{nv-1}, g_0, g_1], n_q = 3 n_v + 6; node positions
 *     (cloth nodes row-major), then the two 3-D gripper positions.  Controls u = [du_0, du_1]
 *     (n_u = 6): gripper displacement commands, g+ = g + u (kinematic grippers).
 *   - Array arguments are caller-owned DEVICE pointers unless stated otherwise, row-major and
 *     contiguous, in the handle's real type (float when real_bytes = 4, double when 8).
 *     int32 status arrays are device pointers too.  The library never frees caller memory.
 *   - Calls are asynchronous and ordered on the given CUDA stream (`stream` is a cudaStream_t;
 *     NULL = the legacy default stream).  A handle may be used by one stream at a time.
 *   - Every function returns a cs_status.  Argument errors are reported before any launch and
 *     leave outputs untouched; per-rollout numerical failures are reported as bits in status[b]
 *     (CS_ST_*) and do not fail the call.  cs_last_error() gives a message for the calling thread.
 *   - Nothing aborts the process; device loops are bounded by the iteration caps in cs_params.
 */
#ifndef CORDSIM_H
#define CORDSIM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  CS_OK = 0,
  CS_ERR_INVALID_ARG = 1,
  CS_ERR_OOM = 2,
  CS_ERR_NOCONVERGE = 3,
  CS_ERR_NONFINITE = 4,
  CS_ERR_TIMEOUT = 5,
  CS_ERR_PENDING = 6,
  CS_ERR_CUDA = 7,
  CS_ERR_CANCELLED = 8,
  CS_ERR_UNSUPPORTED = 9
} cs_status;

/* per-rollout status bits written to status[b] */
#define CS_ST_NEWTON 1     /* stage-1 Newton reached newton_max before converging          */
#define CS_ST_CONTACT 2    /* stage-2 interior point reached ipm_max / found no interior    */
#define CS_ST_NONFINITE 4  /* a non-finite value appeared                                   */
#define CS_ST_NOTPD 8      /* a stage-2 or adjoint system was not positive definite         */
#define CS_ST_TIMEOUT 16   /* a bounded device-side wait of the adjoint ran out (no result)  */

#define CS_MAX_OBSTACLES 8
#define CS_MAX_GOAL 64

enum { CS_ROPE = 0, CS_CLOTH = 1 };
enum { CS_PLANE = 0, CS_SPHERE = 1, CS_BOX = 2 };
enum { CS_HARD = 0, CS_SMOOTH = 1 };          /* fwd_mode */
enum { CS_SURROGATE = 0, CS_CONSISTENT = 1 }; /* grad_mode */

/* Obstacle: plane p = {n_x, n_y, n_z, offset} (phi = n.x - offset - r, |n| = 1);
 * sphere p = {c_x, c_y, c_z, R}; axis-aligned box p = {c_x, c_y, c_z, h_x, h_y, h_z}. */
typedef struct {
  int type;
  double p[6];
} cs_obstacle;

/* Simulator parameters (Sec. 4.1; values are not printed in the paper and are inputs here). */
typedef struct {
  int kind;                 /* CS_ROPE: chain of n_nodes; CS_CLOTH: rows x cols grid          */
  int n_nodes, rows, cols;
  int grasp_node[2];        /* node a(i) held by gripper i                                   */
  double dt;                /* time step delta t [s]                                         */
  double gravity[3];        /* [m/s^2]                                                       */
  double node_mass;         /* lumped mass per node [kg]; M = node_mass I                    */
  double k_stretch, k_shear, k_bend;  /* spring stiffnesses [N/m]; rest lengths from rest_x  */
  double D_max;             /* grasp stiffness D_max [N/m]                                   */
  double kappa_h;           /* grasp smoothing length kappa in D = D_max exp(-|c|/kappa) [m] */
  double kappa_c;           /* relaxed complementarity s^T lambda = kappa_c [N m]            */
  double kappa_hard;        /* barrier weight at which the nonsmooth SOCP is declared solved */
  double kappa_decay;       /* barrier decrease per path-following stage (0 < . < 1)         */
  double mu;                /* friction coefficient                                          */
  double r_grasp;           /* nonsmooth grasp active while |c_i| <= r_grasp [m]             */
  double node_radius;       /* contact radius of a node [m]                                  */
  double sigma0;            /* interior start of a penetrating contact slack [m]             */
  int n_obstacles;
  cs_obstacle obstacles[CS_MAX_OBSTACLES];
  int fwd_mode;             /* CS_HARD (paper forward) or CS_SMOOTH                          */
  int grad_mode;            /* CS_SURROGATE (paper) or CS_CONSISTENT (smooth fwd + exact grad)*/
  int newton_max, ipm_max;  /* iteration caps                                                */
  double newton_tol;        /* stage-1 stop: max |Newton step| <= newton_tol [m]             */
  double ipm_tol;           /* stage-2 stop: max |Newton step| <= ipm_tol [m]                */
  int checkpoint_every;     /* adjoint checkpoint interval k (>= 1; 0 in sim_create: the
                               smallest interval whose adjoint workspace fits in a quarter of
                               the free device memory, at most about sqrt(max_horizon); 0 in
                               an mpc request: see cs_mpc_request; sim_rollout_vjp_noalloc
                               needs k >= 1)                                                  */
  int real_bytes;           /* 4 = FP32, 8 = FP64                                            */
  int max_batch, max_horizon; /* size the handle's workspace                                 */
  /* Inertial variant (ropes; sim_rollout, sim_rollout_vjp, sim_linearize): the state is
   * q = [x (3 n_v), v (3 n_v), g (6)], n_q = 6 n_v + 6, and a step solves
   * M (x+ - x - dt v)/dt^2 + D (x+ - x)/dt + dE/dx(x+) = tau + sum J^T lam, v+ = (x+ - x)/dt, with
   * Rayleigh damping D = damp_alpha M + damp_beta sum_s k_s u_s u_s^T (the springs' axial
   * stiffness at the step start).  It is the quasi-static step of eq. (dynamics) at v = 0, D = 0.
   * second_order = 0 selects the quasi-static step (the paper's). */
  int second_order;
  double damp_alpha, damp_beta;  /* [1/s], [s], both >= 0                                       */
} cs_params;

/* Planning loss (the paper's cost J is not printed):
 *   L = w_goal sum_{j in goal} |x_j(H) - goal_pos_j|^2
 *     + w_pen sum_{t=1..H} sum_{j, non-plane obstacles o} max(0, pen_margin - phi_jo(q_t))^2
 *     + w_u sum_{t=0..H-1} |u_t|^2 */
typedef struct {
  int n_goal;
  int goal_nodes[CS_MAX_GOAL];
  double goal_pos[CS_MAX_GOAL][3];
  double w_goal, w_pen, pen_margin, w_u;
} cs_loss;

typedef struct cs_sim cs_sim;

/* Create a simulator for one scene.  rest_x: HOST array [n_v][3] of rest node positions (the
 * spring rest lengths are taken from it).  Allocates the handle's device workspace for
 * max_batch rollouts of up to max_horizon steps.  A rope (CS_ROPE) has 2..128 nodes; a cloth
 * (CS_CLOTH) rows x cols nodes, row-major (its node-coupled matrices have half bandwidth
 * 6 cols + 2): the band window sits in shared memory up to 33 columns in FP32 (22 in FP64) and in
 * the handle's global workspace beyond; the other per-rollout arrays in shared memory limit a
 * square cloth to about 66 x 66 in FP32 (46 x 46 in FP64).
 * Errors: CS_ERR_INVALID_ARG (bad sizes, a rope or cloth beyond those limits, unknown kind or
 * obstacle), CS_ERR_OOM, CS_ERR_CUDA. */
cs_status sim_create(const cs_params* params, const double* rest_x, cs_sim** out);

/* Release the handle and its workspace (synchronises the device first).  NULL is accepted. */
cs_status sim_destroy(cs_sim* sim);

/* Forward rollout q_{t+1} = f(q_t, u_t), t = 0..H-1, in fwd_mode (Sec. 3 eq. (dynamics_sim);
 * Sec. 4.1 two-stage solve).
 *   q0   [B][n_q]          initial states
 *   u    [B][H][6]         controls
 *   traj [B][H+1][n_q]     all states (may be NULL)
 *   qH   [B][n_q]          final state (may be NULL)
 *   status [B]             CS_ST_* bits
 * Errors: CS_ERR_INVALID_ARG if B > max_batch, H > max_horizon, or a required pointer is NULL. */
cs_status sim_rollout(cs_sim* sim, int B, int H, const void* q0, const void* u, void* traj,
                      void* qH, int32_t* status, void* stream);

/* sim_rollout with solver instrumentation: counters [B][H][3] (device int32, may be NULL)
 * receives, per rollout and step, the stage-1 Newton iterations, the stage-2 interior-point
 * iterations (summed over the path-following stages) and the step's CS_ST_* bits. */
cs_status sim_rollout_counters(cs_sim* sim, int B, int H, const void* q0, const void* u,
                               void* traj, void* qH, int32_t* status, int32_t* counters,
                               void* stream);

/* Forward rollout + checkpointed adjoint (Sec. 4.1 eq. (diff-sim), composed over the horizon).
 * The forward runs in the nonsmooth model (grad_mode CS_SURROGATE) or the smooth model
 * (CS_CONSISTENT); the backward applies the smooth step's Jacobians along the forward states
 * (the paper's surrogate gradient).  States are checkpointed every checkpoint_every steps and the
 * steps in between are recomputed.
 *   dL_dtraj [B][H+1][n_q] seeds dL/dq_t (may be NULL; then `loss` must be given)
 *   loss     HOST pointer to the planning loss (may be NULL when dL_dtraj is given; if both are
 *            given the seeds are added)
 *   L        [B] loss values (may be NULL)
 *   dL_du    [B][H][6] (required)
 *   dL_dq0   [B][n_q] (may be NULL)
 *   status   [B]
 * A rollout whose status becomes nonzero stops at the failing step: its L is NaN and its dL_du
 * and dL_dq0 are zero.
 * Errors: as sim_rollout; CS_ERR_INVALID_ARG when both dL_dtraj and loss are NULL. */
cs_status sim_rollout_vjp(cs_sim* sim, int B, int H, const void* q0, const void* u,
                          const void* dL_dtraj, const cs_loss* loss, void* L, void* dL_du,
                          void* dL_dq0, int32_t* status, void* stream);

/* Per-step linearisation of the smooth step about a nominal trajectory (Sec. 4.2: A(z,v),
 * B(z,v)), by forward-mode tangents of the implicit two-stage solve.
 *   z  [B][H+1][n_q] nominal states; the stage-1 Newton iteration of step t starts at the node
 *                     positions of z_{t+1} (the root next to the nominal trajectory)
 *   v  [B][H][6]     nominal controls
 *   A  [B][H][n_q][n_q]  A_t[i][j] = d q_{t+1,i} / d q_{t,j}
 *   Bm [B][H][n_q][6]    B_t[i][j] = d q_{t+1,i} / d u_{t,j}
 *   status [B] (OR over the steps; a step whose smooth solve fails or whose H1 or H2 is not
 *               positive definite gets NaN Jacobians)
 * With the handle's per-step records (allocated by sim_create when they fit in half the free
 * device memory) it runs as two launches: the smooth steps with their factorisations, then every
 * tangent direction of a step in one CTA; otherwise one warp per (trajectory, step).
 * Errors: as sim_rollout; CS_ERR_UNSUPPORTED for a cloth (built for ropes), and for the inertial
 * variant without the per-step records. */
cs_status sim_linearize(cs_sim* sim, int B, int H, const void* z, const void* v, void* A,
                        void* Bm, int32_t* status, void* stream);

/* Allocation-free rollout adjoint (no counterpart in the paper; an interface for callers that
 * cannot allocate device memory: a real-time control loop that must not block on a driver
 * allocation, which can take milliseconds and synchronise the device, or a process whose device
 * memory is already owned by another allocator).  Same computation and argument conventions as
 * sim_rollout_vjp, but without a handle: params and rest_x (HOST, [n_v][3]) are passed directly,
 * and the spring rest lengths and checkpoint records live in a file-scope device array of
 * CS_NOALLOC_SCRATCH_BYTES bytes that every GPU loading the library holds until the process
 * exits.  No cudaMalloc, cudaFree or allocating library routine is called.
 *   - The first call on a device looks up the array's device address (cudaGetSymbolAddress) for
 *     that device; make that first call before any stream capture.
 *   - All calls share the array and it keeps the last call's contents; nothing in it needs to
 *     start at zero (each call writes every element it reads).  Calls that overlap on the GPU
 *     (different streams, or different host threads on one device) race on it.
 *   - The rest lengths reach the device through a small kernel launched on `stream` that carries
 *     them in its argument; no host-to-device copy is issued.
 *   - Errors: CS_ERR_INVALID_ARG when the checkpoint records of B rollouts of H steps do not fit
 *     in CS_NOALLOC_SCRATCH_BYTES, checkpoint_every < 1, and the argument errors of sim_create
 *     (parameters) and sim_rollout_vjp (loss, sizes, pointers), checked before any device call;
 *     CS_ERR_UNSUPPORTED for a cloth. */
#define CS_NOALLOC_SCRATCH_BYTES (48u << 20)
cs_status sim_rollout_vjp_noalloc(const cs_params* params, const double* rest_x, int B, int H,
                                  const void* q0, const void* u, const void* dL_dtraj,
                                  const cs_loss* loss, void* L, void* dL_du, void* dL_dq0,
                                  int32_t* status, void* stream);

/* ------------------------------------------------------------------------------------------
 * Served plan solves (MPC).  The paper's planners optimise a nominal control sequence by
 * gradients of the simulator at every MPC update (Sec. 4.2 nominal trajectory generation;
 * Sec. 5 planning experiments); the optimiser is not printed.  A plan solve here:
 *   candidates  u^(0) = clip(w), u^(r) = clip(w + sigma eps^(r)), r = 1..R-1, w the warm start,
 *               eps^(r)[t][d] standard normals from Philox4x32-10 (Salmon et al., SC 2011)
 *               keyed by (seed, r, 6 t + d) through Box-Muller;
 *   iterations  G evaluations (forward + surrogate-gradient adjoint of every candidate, the
 *               planning loss cs_loss); after evaluations 1..G-1 a bias-corrected Adam step
 *               (beta 0.9 / 0.999, eps 1e-8, step lr) and the clip to [-u_max, u_max] on every
 *               candidate whose rollout succeeded;
 *   result      the evaluated candidate with the lowest loss over all evaluations (ties: earlier
 *               evaluation, then lower r).
 * A server owns one CUDA stream and a scheduler thread.  Requests wait in FIFO order until a
 * slot and device memory for them are free, then join the running set at the next tick; every
 * tick runs one evaluation (one packed forward + adjoint launch over the candidates of every
 * running request, then the selection and Adam kernels), replayed from a captured CUDA graph
 * while the running set does not change.  Results are independent of what else is running.
 * ------------------------------------------------------------------------------------------ */
typedef struct cs_mpc cs_mpc;

typedef struct {
  size_t mem_budget_bytes;  /* device memory for running requests; 0 = half the free memory   */
  int max_slots;            /* most requests running at once (0 = 64)                         */
  int real_bytes;           /* 4 (FP32) or 8 (FP64)                                           */
  int batched;              /* 1: continuous batching; 0: one request at a time, no graphs
                               (the one-launch-per-request form)                              */
  int use_graphs;           /* 1: replay captured CUDA graphs while the running set is stable */
  int autotune;             /* 1: time the packed launch's warps per CTA at creation          */
  const char* tuner_cache;  /* file holding tuned launch shapes (read, then written); or NULL  */
} cs_mpc_config;

typedef struct {
  cs_params params;         /* scene and solver settings (real_bytes, max_* are ignored;
                               checkpoint_every = 0: the server picks the smallest interval
                               whose candidates' records fit in an eighth of its memory
                               budget, at most about sqrt(H))                                 */
  const double* rest_x;     /* HOST [n_nodes][3] rest positions                               */
  const double* q0;         /* HOST [n_q] state to plan from                                  */
  const double* warm;       /* HOST [H][6] warm start, or NULL: the session's previous plan
                               shifted by one step (last control repeated), else zeros        */
  cs_loss loss;             /* planning loss                                                  */
  int H, R, G;              /* horizon, candidates, evaluations                               */
  double lr, sigma, u_max;  /* Adam step, candidate spread, control bound                     */
  uint64_t seed;
  uint64_t session_id;      /* nonzero: keep this plan on the device for the session's next
                               request                                                        */
  int deadline_ms;          /* 0: none.  > 0: a request still queued or running this long after
                               mpc_submit leaves at the next tick boundary (its device work
                               stops there, nothing waits on the device) and mpc_poll returns
                               CS_ERR_TIMEOUT for it                                          */
} cs_mpc_request;

typedef struct {
  double* u;                /* caller-owned HOST [H][6]: the plan (filled by mpc_poll)        */
  double L;                 /* its loss                                                       */
  int32_t status;           /* 0; else CS_ST_* bits of the last evaluation when no candidate
                               ever succeeded (u is then the warm start)                      */
  int32_t best_iter;        /* evaluation (1..G) and candidate of the plan                    */
  int32_t best_candidate;
  int64_t t_submit_ns, t_start_ns, t_done_ns;  /* steady clock: submitted, admitted, result on
                                                  the host                                    */
} cs_mpc_result;

/* Create a server on the current device.  Errors: CS_ERR_INVALID_ARG, CS_ERR_OOM, CS_ERR_CUDA. */
cs_status mpc_create(const cs_mpc_config* config, cs_mpc** out);
/* Queue a plan solve of a rope or a cloth; the request and its host arrays are copied before the
 * call returns.  Errors: CS_ERR_INVALID_ARG (sizes, a rope or cloth beyond the limits of
 * sim_create, a request larger than the memory budget). */
cs_status mpc_submit(cs_mpc* mpc, const cs_mpc_request* req, uint64_t* ticket);
/* Wait up to timeout_ms (0: do not wait, < 0: no limit) for a result.  CS_OK fills `out` and
 * forgets the ticket; CS_ERR_PENDING if it is not done yet; CS_ERR_CANCELLED; CS_ERR_TIMEOUT when
 * the request's deadline_ms passed before it finished (the ticket is then forgotten);
 * CS_ERR_INVALID_ARG for an unknown ticket; CS_ERR_CUDA if the server's stream failed. */
cs_status mpc_poll(cs_mpc* mpc, uint64_t ticket, int timeout_ms, cs_mpc_result* out);
/* Cancel a queued or running solve (a running one stops at the next tick boundary). */
cs_status mpc_cancel(cs_mpc* mpc, uint64_t ticket);
/* Stop the scheduler (running solves are abandoned) and release everything. */
cs_status mpc_destroy(cs_mpc* mpc);
/* Counters of a server: ticks run, graph launches, kernel launches, graphs captured. */
cs_status mpc_stats(cs_mpc* mpc, int64_t* ticks, int64_t* graph_launches, int64_t* kernel_launches,
                    int64_t* graphs_built);

/* ------------------------------------------------------------------------------------------
 * Output-feedback SLS observer stage (Sec. 4.2): the Kalman recursion, the observer's closed-loop
 * responses and the closed-loop maps, about B nominal trajectories at once (the consumer of
 * sim_linearize's A_t).  Per trajectory, times 0..N, state dimension n, observation p, control m:
 *   A  [B][N][n][n]   A_j, the dynamics linearisation (sim_linearize's A)
 *   C  [B][N][p][n]   C_j, the observation model's linearisation
 *   E  [B][N][n][nw]  E_j, process disturbance scaling
 *   F  [B][N][p][ne]  F_j, observation disturbance scaling (F_j F_j^T positive definite)
 *   Xi [B][n][n0]     initial state uncertainty
 * A block lower-triangular operator over times 0..N is stored packed: block (k, j),
 * 0 <= j <= k <= N, at index k (k + 1) / 2 + j of T = (N + 1)(N + 2) / 2 blocks, each row-major.
 * Arrays are caller-owned DEVICE pointers in the real type real_bytes names (4 float, 8 double).
 * `workspace` is caller-owned device memory of at least the size the matching *_workspace call
 * returns; these calls allocate nothing.  Calls are asynchronous on `stream`; sizes and pointers
 * are checked before any launch.  Errors: CS_ERR_INVALID_ARG (B < 0, a dimension < 1 or > 4096,
 * real_bytes not 4 or 8, a NULL pointer while B > 0, a workspace too small), CS_ERR_CUDA. */

/* Device bytes of scratch sls_observer needs (0 for invalid sizes). */
size_t sls_observer_workspace(int B, int N, int n, int p, int real_bytes);

/* Kalman recursion (Sec. 4.2 eq. kalman_recursions) and observer responses (eq.
 * backward_propagations):
 *   Pi   [B][N+1][n][n]  Pi_0 = Xi Xi^T,
 *                        Pi_{j+1} = E_j E_j^T + A_j Pi_j A_j^T + A_j Pi_j C_j^T L_{j+1}
 *   L    [B][N][p][n]    L[j] = L_{j+1} = -(F_j F_j^T + C_j Pi_j C_j^T)^{-1} C_j Pi_j A_j^T
 *   PhiX [B][T][n][n]    Phihat^x_{k,k} = I, Phihat^x_{k,j} = Phihat^x_{k,j+1} (A_j + L_{j+1}^T C_j)
 *   PhiY [B][T][n][p]    Phihat^y_{k,j} = Phihat^x_{k,j} L_j^T (j >= 1), Phihat^y_{k,0} = 0
 *   status [B]           CS_ST_NOTPD when an innovation matrix F_j F_j^T + C_j Pi_j C_j^T was not
 *                        positive definite: that step's gain and what follows it are NaN (may be
 *                        NULL)
 * The gain computed from (Pi_j, A_j, C_j) carries the label j+1 and is the one the propagation
 * through A_j uses; Pi and L are the same for every injection time k.  p is limited by the gain
 * solve's shared memory (p^2 + 10 p reals within 200 KB: p <= 221 in FP32, 155 in FP64). */
cs_status sls_observer(int B, int N, int n, int p, int nw, int ne, int n0, int real_bytes,
                       const void* A, const void* C, const void* E, const void* F, const void* Xi,
                       void* Pi, void* L, void* PhiX, void* PhiY, int32_t* status,
                       void* workspace, size_t workspace_bytes, void* stream);

/* Device bytes of scratch sls_kalman_scan needs (0 for invalid sizes). */
size_t sls_kalman_scan_workspace(int B, int N, int n, int p, int real_bytes);

/* The covariances Pi [B][N+1][n][n] of sls_observer by the associative scan of eq.
 * combination_rules with eq. initialization: the elements are the prior (0, 0, Xi Xi^T) and, per
 * step j, (A_j^T, C_j^T (F_j F_j^T)^{-1} C_j, E_j E_j^T); Pi_j is the composition of the first j + 1
 * elements, the later step on the left, formed in ceil(log2(N + 1)) levels (each a batch of
 * products and one LU solve with (I + Dtil Ptil) per element pair).  Same inputs as
 * sls_observer; F_j F_j^T must be positive definite (else CS_ST_NOTPD, and NaN from there);
 * status [B] may be NULL.  n is limited by the LU solve's shared memory (n^2 + 10 n reals within
 * 200 KB: n <= 221 in FP32, 155 in FP64).  Errors: as sls_observer. */
cs_status sls_kalman_scan(int B, int N, int n, int p, int nw, int ne, int n0, int real_bytes,
                          const void* A, const void* C, const void* E, const void* F, const void* Xi,
                          void* Pi, int32_t* status, void* workspace, size_t workspace_bytes,
                          void* stream);

/* Closed-loop response of x_{k+1} = Acl_k x_k + delta_{k+1}, the products that eq.
 * backward_propagations forms, for given closed-loop matrices:
 *   Acl [B][N][n][n];  Phi [B][T][n][n], Phi_{k,k} = I, Phi_{k,j} = Phi_{k,j+1} Acl_j.
 * With Acl_j = A_j + B_j K_j it is the state-feedback response (I - Z (A + B K))^{-1}. */
cs_status sls_response(int B, int N, int n, int real_bytes, const void* Acl, void* Phi,
                       void* stream);

/* Device bytes of scratch sls_closed_loop needs (0 for invalid sizes). */
size_t sls_closed_loop_workspace(int B, int N, int n, int p, int real_bytes);

/* Closed-loop maps (Sec. 4.2) from the state-feedback responses Phibar (the stage before this
 * one; an input) and the observer's, with M = I - Z A (Z the block downshift):
 *   PhiXW [B][T][n][n] = Phibar^x + Phihat^x - Phibar^x M Phihat^x
 *   PhiUW [B][T][m][n] = Phibar^u (I - M Phihat^x)
 *   PhiXE [B][T][n][p] = Phihat^y - Phibar^x M Phihat^y
 *   PhiUE [B][T][m][p] = -Phibar^u M Phihat^y
 * from A [B][N][n][n], PhiBarX [B][T][n][n], PhiBarU [B][T][m][n] and PhiX, PhiY as sls_observer
 * writes them. */
cs_status sls_closed_loop(int B, int N, int n, int m, int p, int real_bytes, const void* A,
                          const void* PhiBarX, const void* PhiBarU, const void* PhiX,
                          const void* PhiY, void* PhiXW, void* PhiUW, void* PhiXE, void* PhiUE,
                          void* workspace, size_t workspace_bytes, void* stream);

/* Device bytes of scratch sls_tubes needs (0 for invalid sizes). */
size_t sls_tubes_workspace(int B, int N, int n, int m, int p, int nw, int ne, int nc, int real_bytes);

/* Reachable tubes and constraint tightening (Sec. 4.2 eq. of_optimization_tightening1/2) from the
 * closed-loop maps sls_closed_loop writes and the disturbance scalings E [B][N][n][nw],
 * F [B][N][p][ne] of sls_observer.  The disturbances w_j, e_j of step j reach time k through the
 * blocks (k, j + 1) (j = 0..k-1); the initial estimation error is not in the sums.
 *   tau    [B][N+1][n+m]  tau_k = sum_j ||[Phi^xw; Phi^uw]_{k,j+1} E_j||_{2,r}
 *                                + ||[Phi^xe; Phi^ue]_{k,j+1} F_j||_{2,r} (row-wise 2-norms of the
 *                         rows of [x_k; u_k]); tau_0 = 0
 *   margin [B][N][nc]     -b_i - c_i^T [z_k; v_k] - sum_j (|c_i^T Phi^w_{k,j+1} E_j|_2 +
 *                         |c_i^T Phi^e_{k,j+1} F_j|_2), k = 0..N-1: the constraint c_i^T [x; u]
 *                         <= -b_i holds for every disturbance in the unit balls when it is >= 0
 *   Ccon [nc][n+m], bcon [nc] (shared by the trajectories), nominal z [B][N+1][n], v [B][N][m];
 *   with nc = 0 these and margin may be NULL.
 * Errors: as sls_closed_loop; nc in [0, 4096]. */
cs_status sls_tubes(int B, int N, int n, int m, int p, int nw, int ne, int nc, int real_bytes,
                    const void* PhiXW, const void* PhiUW, const void* PhiXE, const void* PhiUE,
                    const void* E, const void* F, const void* Ccon, const void* bcon,
                    const void* z, const void* v, void* tau, void* margin, void* workspace,
                    size_t workspace_bytes, void* stream);

/* Conformal radius (Sec. 4.4): scores s_i = ||q_next_i - f_pred_i||_2 of n_cal calibration
 * transitions (q_next [n_cal][dim] the next perceived states, f_pred [n_cal][dim] the model's
 * predictions, e.g. sim_rollout with H = 1), and radius[0] = s_(k), the k-th smallest score with
 * k = ceil((n_cal + 1)(1 - delta / T)) (at least 1; +inf when k > n_cal).  scores [n_cal] may be
 * NULL; radius is a device pointer to one real.  A NaN score sorts as +inf.
 * Errors: CS_ERR_INVALID_ARG (n_cal not in [1, 8192], dim not in [1, 2^20], delta not in (0, 1),
 * T < 1, NULL q_next, f_pred or radius), CS_ERR_CUDA. */
cs_status sls_conformal_radius(int n_cal, int dim, int real_bytes, const void* q_next,
                               const void* f_pred, double delta, int T, void* scores,
                               void* radius, void* stream);

/* ------------------------------------------------------------------------------------------
 * Analytic policy gradient (Sec. 4.3): a policy in the loop of the batched rollout and the
 * gradient of the closed-loop planning loss through the simulator (eq. diff-sim).  The policy,
 * shared by the rollouts, is one tanh hidden layer of `hidden` units,
 *   u = W2 tanh(W1 q + b1) + b2,   theta = [W1 (hidden x n_q), b1 (hidden), W2 (6 x hidden), b2 (6)]
 * (device, the handle's real type, row-major, packed in that order: n_theta = hidden n_q +
 * 7 hidden + 6).  The rollout runs q_{t+1} = f(q_t, pi(q_t)), t = 0..H-1, in the nonsmooth model;
 * the loss is the planning loss `loss` (HOST pointer: goal on q_H, obstacle penalty on q_1..q_H,
 * effort w_u |u_t|^2) of that trajectory, and the gradient is the surrogate one (the smooth step's
 * Jacobians along the nonsmooth trajectory), with the policy's derivatives in the chain.  Each
 * step runs as a one-step sim_rollout and a one-step sim_rollout_vjp (every state a checkpoint).
 *   q0 [B][n_q]; L [B] (may be NULL; NaN for a flagged rollout); dtheta [n_theta], summed over
 *   the rollouts whose status stayed 0; dq0 [B][n_q] (may be NULL; zero for a flagged rollout);
 *   status [B] (may be NULL): the OR of the steps' CS_ST_* bits.
 * Errors: CS_ERR_INVALID_ARG (NULL handle, q0, theta, loss, dtheta or workspace; B not in
 * [1, max_batch]; H < 1; hidden not in [1, 1024]; the loss checks of sim_rollout_vjp; a
 * workspace smaller than apg_workspace()), and those of sim_rollout and sim_rollout_vjp. */
size_t apg_workspace(const cs_sim* sim, int B, int H, int hidden);
cs_status apg_rollout_grad(cs_sim* sim, int B, int H, int hidden, const void* q0, const void* theta,
                           const cs_loss* loss, void* L, void* dtheta, void* dq0, int32_t* status,
                           void* workspace, size_t workspace_bytes, void* stream);

/* Number of kernel launches the library made on the calling thread since the last call
 * (instrumentation for benchmarks). */
int64_t cs_launch_count(void);

/* Message describing the last error on the calling thread ("" if none). */
const char* cs_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* CORDSIM_H */
