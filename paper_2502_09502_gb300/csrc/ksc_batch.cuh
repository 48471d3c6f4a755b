// ksc_batch.cuh -- device view of a batched solve: many nodes of one problem
// advance together through restarted FISTA (Algorithm 3), with the two products
// of each step on the tensor cores (k_tcgemm.cu) and one CTA per node for the
// prox, g and the dual term (k_batch.cu).
//
// Precision.  The iterate (beta, u = X beta, G = X^T grad F) is FP64.  The tensor
// cores multiply BF16 X by a difference from a per-node anchor, split into three
// BF16 pieces whose sum is the FP32 value exactly:
//   u^{t+1} = u_ref + X (beta^{t+1} - beta_ref),   G = G_ref + X^T (r - r_ref),
// where u_ref = X beta_ref and G_ref = X^T r_ref come from the double-float
// streaming product (accurate to ~1e-13).  The FP32 accumulation error is then
// relative to the difference, which shrinks as the node converges; an FP32
// product of the full vectors would shift the fixed point of the iteration by
// ~ (L / mu) * 1e-7 and stall above a 1e-6 gap.  Nodes re-anchor at their
// current iterate as their gap falls.
//
// Layout (node-major; rows padded to multiples of 8 elements for TMA):
//   beta      B x 3 x ldp   FP64 iterate slots (cur, prev, new rotate per node)
//   beta_ref  B x ldp       FP64 anchor iterate
//   bpc       P x Bpad x ldp  BF16 pieces of fl32(beta^{t+1} - beta_ref)
//   U         B x 3 x ldn   FP64 u per slot
//   u_ref     B x ldn       FP64 X beta_ref
//   r_ref     B x ldn       FP64 grad F(u_ref)
//   rpc       P x Bpad x ldn  BF16 pieces of fl32(grad F(u_gamma) - r_ref)
//   G, G_ref  B x ldp       FP64 X^T grad F(u_gamma), X^T r_ref
//
// E4M3 X (per-column power-of-two scales s_j, e8 = 1): the products read E4M3 X
// and kTcE4m3Pieces E4M3 pieces of each difference, scaled per node by a power
// of two (k_tcgemm.cu, ksc_tc.h): bpc8 holds the pieces of s_j (beta_j -
// beta_ref_j) (the column scales folded into the vector), rpc8 those of
// grad F(u_gamma) - r_ref (the column scales applied to X^T r in the epilogue);
// rs_fwd / rs_grad hold each node's inverse scale.  The residual differences go
// through rbuf (FP32) with per-CTA maxima in rmaxp, so that the pieces are cut
// once the node's largest entry is known.
#pragma once

#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ksc_launch.h"
#include "ksc_state.cuh"

namespace ksc {

constexpr int kBatchPieces = 3;     // BF16 pieces of an FP32 vector (exact sum)
constexpr int kBatchCap = 2048;     // prox candidates per node in shared memory
constexpr int kBatchMax = 1024;     // nodes per device pass
constexpr int kBProxBlock = 256;    // threads of the per-node prox CTA
static_assert(kBatchCap + 1 >= 2 * kBProxBlock, "the prox's full-pass sums use the prefix buffer");
constexpr int kBThreads = 256;      // residual kernel
constexpr int kBRows = 8;           // rows per residual thread
constexpr int kSlotIdle = 5;        // BNode::done of an empty slot (every kernel skips it)

// one node of a batched solve (field names follow NodeDev: the restart/gap step
// logic is shared)
struct BNode {
  // parameters
  double lambda2, M, rho, invL, tol_loop, incumbent;
  int kp, max_iter, restart_on, momentum_on;
  // state
  int iter, done, restarts, cur;
  int prev, nnz, qhint, fallback;
  double phi, c, Lcur, best_primal, best_dual, gap;
  double g_next, negconj, gstar, theta, last_primal, last_dual;
  double g_cur;        // g_node(beta^t) (the restart test's difference)
  // eigen-perspective relaxation (App. D.2; 0: the perspective relaxation):
  // lambda2 above is then lambda2 + eig, rho and invL those of L - 2 eig
  double eig;
  double bsq_cur, bsq_next;   // ||beta^t||^2, ||beta^{t+1}||^2
  double gthr;                // the last in-loop dual term's k'-th largest |G_F| (0: none yet)
  double ptop;                // the last prox's k'-th largest |w_F| (0: none yet)
};

// FP64 certificate of one node (copied out of the single-node workspace)
struct BCert {
  double primal, dual, gap, g;
};

struct BatchDev {
  int n, p, B, Bpad, loss, P;
  int ldp, ldn;
  int nft;             // loss partials per node (one per 64 rows of X)
  int nrt;             // residual CTAs per node
  int wsm;             // prox keeps w in shared memory (elements), else wbuf
  const float* yf;     // n
  const double* y;     // n
  const int8_t* state; // B x ldp
  double* beta;
  double* beta_ref;
  __nv_bfloat16* bpc;
  double* U;
  double* u_ref;
  double* r_ref;
  __nv_bfloat16* rpc;
  double* G;           // B x ldp: grad at gamma (k_bprox subtracts 2 eig gamma in place for eigen nodes)
  double* G_ref;       // B x ldp: X^T r_ref, exact
  double* wbuf;        // B x ldp, or NULL
  int* slot_cur;       // B: slot of u^t (read by the forward product)
  int* slot_new;       // B: slot the forward product writes
  double* fpart;       // B x nft x 2: sums of F(u^{t+1}) and of F(u^{t+1}) - F(u^t)
  double* ncpart;      // B x nrt
  BNode* nodes;        // B
  BCert* cert;         // B
  double* beta_out;    // B x p (certified iterate, FP64)
  double* z_out;       // B x p (relaxed z)
  // FP64 certificate (Sec. 3.4) of many nodes at once
  const double* colnorm;  // p: column 2-norms of X, rounded up
  double* cert_u;      // B x ldn: X b^
  double* cert_z;      // B x ldn: zeta = -grad F(X b^)
  double* cert_a;      // B x ldp: X^T zeta
  double* cpart;       // B x nrt x 4: F, -F*(-zeta), its rounding weights, ||zeta||^2
  double* dfws;        // kDfWsElems: split partials of the tiled exact product
  int* tile_run;       // per 128 slots: any node running (k_bstep and the host keep it)
  double xfro;         // ||X||_F, rounded up (eigen-perspective certificate)
  double ynorm;        // ||y||_2, rounded up
  // E4M3 X (e8 = 1): see the header comment
  int e8;
  int ldp8, ldn8;      // byte strides of the E4M3 pieces (multiples of 16)
  uint8_t* bpc8;       // kTcE4m3Pieces x Bpad x ldp8
  uint8_t* rpc8;       // kTcE4m3Pieces x Bpad x ldn8
  float* rs_fwd;       // B: inverse scale of the node's forward pieces
  float* rs_grad;      // B: inverse scale of the node's residual pieces
  float* rbuf;         // B x ldn: FP32 residual differences
  float* rmaxp;        // B x nrt: their per-CTA largest magnitudes
  const float* xscale; // p: the column scales s_j
};

__host__ __device__ inline int batch_nrt(int n) { return (n + kBThreads * kBRows - 1) / (kBThreads * kBRows); }

size_t bprox_smem_bytes(int wsm);
cudaError_t batch_prepare(int optin);
void launch_bresid(const BatchDev& d, cudaStream_t s);
// E4M3: the residual differences' pieces from rbuf, once every CTA's maximum is in
void launch_bsplit8_resid(const BatchDev& d, cudaStream_t s);
// E4M3: the pieces of beta slot 1 - beta_ref of the listed nodes (the zero anchor's
// admission product)
void launch_bsplit8_beta(const BatchDev& d, const int* list, int count, cudaStream_t s);
void launch_bprox(const BatchDev& d, cudaStream_t s);
void launch_bstep(const BatchDev& d, cudaStream_t s);
// admission of the slots in `list` (device int array, count entries): beta slots
// 0 and 1 and the anchor from the warm start uploaded into slot 1
void launch_binit_copy(const BatchDev& d, const int* list, int count, cudaStream_t s);
// after the slots' anchors: u slots, F(u^1), g(beta^1), L^1 and the node state;
// zero != 0: after the zero anchor, u^1 is in u slot 1 (the admission product)
void launch_binit_node(const BatchDev& d, const int* list, int count, int zero, cudaStream_t s);
// the zero anchor of the listed slots (beta_ref = 0, u_ref = 0, r_ref = r0 =
// grad F(0), G_ref = G0 = X^T r0, pieces of beta^1) and the slot maps of the
// admission's forward product (admitted rows -> slot 1, others -> their free slot)
void launch_bzero_anchor(const BatchDev& d, const int* list, int count, const double* r0, const double* G0,
                         cudaStream_t s);
// anchors of the listed nodes (device list, count entries) at their current
// iterate: beta_ref = beta^t (mid-solve only), then (after u_ref = X beta_ref)
// r_ref = grad F(u_ref), u slot(s) = u_ref and, mid-solve, fresh in-loop bests
void launch_banchor_copy(const BatchDev& d, const int* list, int count, cudaStream_t s);
void launch_banchor_resid(const BatchDev& d, const int* list, int count, int init, cudaStream_t s);
// FP64 certificates of the listed nodes (device list, count entries): the iterate
// projected onto dom g (into beta_out), then -- after cert_u = X b^ -- zeta, F and
// -F*(-zeta) per row, then -- after cert_a = X^T zeta -- the bound with its
// rounding margins, g(b^), the relaxed z and the gap.  err_a: the product's error
// factor (dfprod_error_factor).
void launch_bcert_prep(const BatchDev& d, const int* list, int count, cudaStream_t s);
void launch_bcert_rows(const BatchDev& d, const int* list, int count, cudaStream_t s);
// err_u: the forward product's error factor (the eigen-perspective bound's margin)
void launch_bcert_final(const BatchDev& d, const int* list, int count, double err_a, double err_u,
                        cudaStream_t s);
// out = A^T vec with A = X (rows n, vec n -> out p) or A = Xc (vec p -> out n),
// double-float products (the single-node streaming kernel; uses d's partials)
void launch_colsum_any(const Dev& d, bool use_xc, const double* vec, double* out, cudaStream_t s);
// D[list[r]] = A^T V[list[r]] for r < R: the same product for many nodes in one
// launch (rows of V and D with strides ldv, ldd), blocked double-float with a
// rigorous error bound (dfprod_error_factor * sum |A V|).  Few nodes split K over
// more CTAs through ws (kDfWsElems doubles).
constexpr int kDfMaxSplits = 16;
constexpr size_t kDfWsElems = (size_t)2 * 608 * 128 * 16;
// kblock: terms per double-float block (a multiple of 32): kDfBlockCert for the
// certificates (the bound below), kDfBlockAnchor for anchors (no bound needed)
constexpr int kDfBlockCert = 64, kDfBlockAnchor = 256;
void launch_dfprod(const Dev& d, bool use_xc, const double* V, int64_t ldv, const int* list, int R, double* D,
                   int64_t ldd, double* ws, int kblock, cudaStream_t s);
int dfprod_splits(int R, int C);
double dfprod_error_factor(int K, int R, int C, int kblock);

}  // namespace ksc
