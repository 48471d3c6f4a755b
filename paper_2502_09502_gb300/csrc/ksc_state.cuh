// ksc_state.cuh -- device-resident state of one node solve (restarted FISTA,
// Algorithm 3) and the argument blocks of the kernels that advance it.
#pragma once

#include <stdint.h>

namespace ksc {

enum : int8_t { kFree = 0, kZero = 1, kOne = 2 };
enum : int { kLossLsq = 0, kLossLogistic = 1 };

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
  int pad0;
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

}  // namespace ksc
