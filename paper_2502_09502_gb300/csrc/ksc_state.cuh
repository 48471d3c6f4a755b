// ksc_state.cuh -- device-resident state of one node solve (restarted FISTA,
// Algorithm 3) and the argument blocks of the kernels that advance it.
#pragma once

#include <stdint.h>

namespace ksc {

enum : int8_t { kFree = 0, kZero = 1, kOne = 2 };
enum : int { kLossLsq = 0, kLossLogistic = 1, kLossSqHinge = 2, kLossPoisson = 3, kLossGamma = 4 };

// termination codes written by the fused restart/gap step
enum : int {
  kRunning = 0,
  kDoneGap = 1,        // in-loop relative gap <= tol_loop
  kDonePruned = 2,     // in-loop dual bound above the incumbent
  kDonePrimal = 3,     // primal below the incumbent
  kDoneMaxIter = 4
};

// Parameters (written by the host before a solve) and evolving scalars of one
// node.  Lives in device memory; every kernel of a FISTA step reads it, the
// last one (the restart/gap step) writes it.
struct NodeDev {
  // ---- parameters
  double lambda2, M, rho, L, invL, tol_loop, incumbent;
  int kp;            // k' = k - |S1|
  int max_iter;
  int restart_on, momentum_on;
  int loss;
  int n_one;         // |S1|: its indices are the first n_one entries of Dev::one_idx
  // ---- state
  int iter;          // t: beta^t is in slot t % 3
  int done;
  int restarts;
  int nnz;           // nonzeros of the newest iterate (written by the prox)
  int qhint;         // candidate count that sufficed at the previous step
  int fallback;      // number of steps that needed the full-pass root finder
  int sparse_steps;  // number of steps whose forward pass gathered nonzero columns
  int pad2;
  double phi;        // momentum counter of Algorithm 3
  double c;          // momentum coefficient phi/(phi+3) of the next step
  double Lcur;       // objective at beta^t (restart test)
  double best_primal, best_dual, gap;
  double g_next;     // g_node(beta^{t+1})            (prox kernel)
  double negconj;    // -F*(-zeta_gamma)              (gradient kernel)
  double gstar;      // G*(X^T zeta_gamma) over the node (prox kernel, dual CTA)
  double theta;      // pooled-block threshold of the last prox
  double last_primal, last_dual;
  // ---- prox selection result (select kernel -> apply kernel)
  unsigned thr_kf;   // float bits of the k'-th largest |w| (top-set key threshold)
  int q;             // min(k', p): size of the top set
  double bnd_a;      // exact |w| of the last top member among keys == thr_kf (-1: all)
  int bnd_i;         // its index (ties broken by ascending index)
  int pad1;
  double l1, s1sq;   // sum |b_F| and sum_{S1} b^2 of the newest iterate
  // eigen-perspective relaxation (App. D.2; 0: the perspective relaxation): lambda2
  // above is then lambda2 + eig, rho and invL those of L - 2 eig
  double eig;
  double bsq_next;   // ||beta^{t+1}||^2 (eig > 0 only)
  // warm-started candidate selection: float-bit key thresholds predicted from the
  // previous step (0 = take every coordinate, i.e. no prediction yet)
  unsigned cguess;   // prox: keys >= cguess are appended by the gradient epilogue
  unsigned dguess;   // dual: |grad| keys >= dguess
  int fast_steps;    // steps whose prox used the predicted candidates
  int dfast_steps;   // steps whose dual term used the predicted candidates
  // ---- certificate (FP64 kernels at exit)
  double cert_f;        // F(X b^) in FP64
  double cert_negconj;  // -F*(-zeta) at zeta = -grad F(X b^)
  double cert_margin_f; // rounding bound of cert_negconj
  double cert_zeta_sq;  // ||zeta||_2^2 (for the X^T zeta error bound)
  double cert_gstar;    // G*(a), a = X^T zeta, FP64
  double cert_margin_g; // rounding bound of cert_gstar
  double cert_g;        // g_node(b^) in FP64 (Algorithm 2)
  double cert_sbar;     // Algorithm 2 break value (relaxed z)
  double cert_dual, cert_primal, cert_gap;
};

// The restart, best-bound and termination logic closing one FISTA step
// (Algorithm 3's objective and restart test, the gap test of Sec. 4.1, the early-termination rules
// of Sec. 4.3), for any node record with these fields (NodeDev, BNode).
// dL (optional): the change L^{t+1} - L^t evaluated as a difference (the batched
// solver's cancellation-free form); otherwise the two values are compared.
template <class N>
__device__ __forceinline__ void fista_step_logic(N* nd, double f, const double* dL = nullptr) {
  const double Lnext = f + 2.0 * nd->lambda2 * nd->g_next;
  const double D = nd->negconj - 2.0 * nd->lambda2 * nd->gstar;
  nd->last_primal = Lnext;
  nd->last_dual = D;
  const bool up = dL ? (*dL >= 0.0) : (Lnext >= nd->Lcur);
  if (nd->restart_on && up) {
    nd->phi = 1.0;
    nd->restarts += 1;
  } else {
    nd->phi += 1.0;
  }
  nd->Lcur = Lnext;
  nd->best_primal = fmin(nd->best_primal, Lnext);
  nd->best_dual = fmax(nd->best_dual, D);
  nd->gap = (nd->best_primal - nd->best_dual) / fmax(fabs(nd->best_primal), 1e-300);
  const int t = nd->iter + 1;
  nd->iter = t;
  int done = kRunning;
  if (isfinite(nd->incumbent)) {
    if (nd->best_dual > nd->incumbent) done = kDonePruned;
    else if (Lnext < nd->incumbent) done = kDonePrimal;
  }
  if (done == kRunning && nd->gap <= nd->tol_loop) done = kDoneGap;
  if (done == kRunning && t - 1 >= nd->max_iter) done = kDoneMaxIter;
  nd->done = done;
  nd->c = nd->momentum_on ? nd->phi / (nd->phi + 3.0) : 0.0;
}

}  // namespace ksc
