// Linearisation of the smooth rope step (arxiv 2606.14188, Sec. 4.2: A_t = dq_{t+1}/dq_t and
// B_t = dq_{t+1}/du_t of the smoothed dynamics at a nominal (z_t, v_t)), in two launches:
//
//   rope_cta_lin_step_kernel  one 64-thread CTA per (trajectory, step) job at a time: the smooth
//                             step at (z_t, v_t), stage 1 started at the nominal next state, then
//                             H2 = dR/dq+ and H1 = dF/dq*, both at the step's solution, factorised
//                             by block Cholesky (a lower block-bidiagonal factor in node pairs), and
//                             a record with the two factors, the node state and the step's scalars;
//   rope_lin_tangent_kernel   one CTA per job: every tangent direction of the step in one pass, a
//                             thread per direction running the forward and backward block sweeps
//                             on the shared factors (broadcast vector reads) with its own
//                             right-hand side in shared memory (a column per thread).
//
// Directions (132 for a 40-node rope): dir < 3 nv node coordinates, then the 6 gripper
// coordinates (columns of A), then the 6 controls (columns of B).  For direction theta,
//   dx*     = H1^-1 (-dF/dtheta)                                 (implicit function theorem on F = 0)
//   dDelta  = H2^-1 (-(dR/dx*) dx* - dR/dtheta)                  (on the stage-2 optimality R = 0)
//   dq+/dtheta = dx* + dDelta on the nodes; the grippers move by g+ = g + u.
#pragma once
#include "rope_cta.cuh"

// cs::rc: the quasi-static step; cs::rci: the inertial variant
#define RC_NS rc
#define RC_SO_ON(S) false
#include "rope_lin_body.cuh"
#undef RC_NS
#undef RC_SO_ON
#define RC_NS rci
#define RC_SO_ON(S) ((S).so != 0)
#include "rope_lin_body.cuh"
#undef RC_NS
#undef RC_SO_ON
