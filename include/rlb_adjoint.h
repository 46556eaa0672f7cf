/*
 * rlb_adjoint.h -- exact discrete gradient of a profile misfit through the fused
 * step of librlb (reverse mode, hand-written adjoint kernels, sqrt(T) checkpoints).
 *
 * The paper (arXiv 1211.3286, Sec. V) studies how the relaxation times tau_v,
 * tau_e and tau_eps of the MRT collision (Eqs. 30-35) shape shock-tube profiles.
 * This call differentiates that map: for the FP64 lattice h whose current state
 * g^0 is taken as the initial state, it runs nsteps fused steps forward and
 * returns
 *     J = w_P sum_x (P(x) - P*(x))^2 + w_u sum_x |u(x) - u*(x)|^2
 * of the fields at step nsteps (Eq. 10 plus the recovery of the stored lattice),
 * together with dJ/dtau_v, dJ/dtau_e, dJ/dtau_eps (tau_q is tied to tau_v) and
 * dJ/de0(x), the gradient with respect to the initial energy-density field of an
 * equilibrium initial state g^0 = g^eq(e0, u0) (Eqs. 8-9; u0 and n0 held fixed;
 * g^eq is linear in e0, so dJ/de0 = sum_a lambda^0_a g^0_a / e0).
 *
 * Method: the step is g^{t+1} = C(S g^t; tau) with S the pull stream (linear) and
 * C the per-node collide.  Reverse mode propagates lambda^t = S^T C_g^T lambda^{t+1}
 * (C_g^T lambda is the vector-Jacobian product of the collide, written out by hand;
 * S^T gathers the pushed adjoints, with the clamped pulls of zero-gradient ends
 * adding into the edge node) and accumulates dJ/dtau from C_tau^T lambda per node.
 * States are recomputed per segment from checkpoints taken every
 * `checkpoint_every` steps (<= 0 selects ceil(sqrt(nsteps))), so memory grows as
 * about 2 sqrt(nsteps) states.  f does not enter J (the velocity comes from g), so
 * only g is differentiated.
 *
 * Requirements: precision RLB_FP64; tau_q <= 0 or tau_q == tau_v.  BGK lattices
 * return dJ/dtau_e = dJ/dtau_eps = 0.
 * Arguments: target_P, target_ux, target_uy, target_uz: nodes values each in
 * `where` memory; de0 (nodes values, `where` memory) may be NULL; loss and dtau
 * (3 values) are host memory.  On return the handle holds the forward state at
 * step nsteps.  Synchronises.  RLB_ENONPHYS if the forward run met a
 * non-physical node; RLB_ENOMEM if the checkpoints do not fit.
 */
#ifndef RLB_ADJOINT_H
#define RLB_ADJOINT_H

#include "rlb.h"

#ifdef __cplusplus
extern "C" {
#endif

int rlb_adjoint(rlb_handle* h, int nsteps, int checkpoint_every, const double* target_P, const double* target_ux,
                const double* target_uy, const double* target_uz, double w_P, double w_u, int where, double* loss,
                double* dtau, double* de0);

#ifdef __cplusplus
}
#endif
#endif /* RLB_ADJOINT_H */
