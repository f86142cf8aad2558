// Rope (particle chain) kernels with one CTA of 64 threads per rollout for the whole horizon.
// Thread t owns nodes j = t + 64 k (slots k < NPT): their state in registers, their rows of the
// node-coupled matrices, and their contact pairs with every obstacle.  Springs read the
// neighbouring nodes' values from shared memory; the block cyclic reduction of the node-coupled
// matrices runs with a group of threads per block row at each level.
//
// The computation is that of the one-warp kernels in rope.cuh (arxiv 2606.14188, Sec. 4.1):
//   stage 1  Newton for q* with F(q*) = M(q*-q)/dt^2 + dE(q*) - tau(u) + sum_i d_i (x*_a - g*_i) = 0
//            (eq. dynamics-first-stage; kinematic grippers g* = g + u; d_i the grasp stiffness);
//   stage 2  Delta = argmin 1/2 Delta^T P Delta over the dual friction cones (eq.
//            dynamics-second-stage) by a primal-dual interior point whose central path at kappa is
//            the relaxed complementarity s^T lam = kappa (Sec. 4.1 "Contact Smoothing");
//   adjoint  eq. diff-sim with the total derivative, the smooth step evaluated along the
//            nonsmooth trajectory (the surrogate gradient).
// Spreading a rollout over 64 threads shortens its dependency chains (the contact pairs, the
// spring assembly and the reduction levels run in parallel), which is what bounds a call: the
// slowest rollouts decide when it ends.
#pragma once
#include "common.cuh"
#include "cr.cuh"
#include "rope.cuh"

// cs::rc: the quasi-static step (the paper's); cs::rci: the inertial variant (state [x, v, g])
#define RC_NS rc
#define RC_SO_ON(S) false
#include "rope_cta_body.cuh"
#undef RC_NS
#undef RC_SO_ON
#define RC_NS rci
#define RC_SO_ON(S) ((S).so != 0)
#include "rope_cta_body.cuh"
#undef RC_NS
#undef RC_SO_ON
