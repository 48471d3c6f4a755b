// ksc_batch.cuh -- device view of a batched solve: many nodes of one problem
// advance together through restarted FISTA (Algorithm 3), with the two products
// of each step on the tensor cores (k_tcgemm.cu) and one CTA per node for the
// prox, g and the dual term (k_batch.cu).
//
// Layout (node-major; rows padded to multiples of 8 elements for TMA):
//   beta   B x 3 x ldp   FP32 iterate slots (cur, prev, new rotate per node)
//   bpc    P x Bpad x ldp  BF16 pieces of the step dbeta = beta^{t+1} - beta^t
//                        (A of the product X dbeta)
//   U      B x 3 x ldn   FP64 u = X beta per slot, advanced as u^{t+1} = u^t + X dbeta:
//                        the FP32 accumulation error of the product is relative
//                        to the step, not to u (the residual correction that lets
//                        an FP32 iteration reach a 1e-6 certified gap)
//   rpc    P x Bpad x ldn  BF16 pieces of grad F(u_gamma) (A of X^T r)
//   G      B x ldp       FP32 X^T grad F(u_gamma)
#pragma once

#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

#include "ksc_launch.h"
#include "ksc_state.cuh"

namespace ksc {

constexpr int kBatchPieces = 3;     // BF16 pieces of an FP32 vector (exact sum)
constexpr int kBatchCap = 1024;     // prox candidates per node in shared memory
constexpr int kBatchMax = 1024;     // nodes per device pass
constexpr int kBProxBlock = 256;    // threads of the per-node prox CTA
constexpr int kBThreads = 256;      // residual kernel
constexpr int kBRows = 8;           // rows per residual thread

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
};

// FP64 certificate of one node (copied out of the single-node workspace)
struct BCert {
  double primal, dual, gap, g;
};

struct BatchDev {
  int n, p, B, Bpad, loss, P;
  int ldp, ldn;
  int nft;             // forward-product tiles per node (loss partials)
  int nrt;             // residual CTAs per node
  int wsm;             // prox keeps w in shared memory (elements), else wbuf
  const float* yf;     // n
  const int8_t* state; // B x ldp
  float* beta;
  __nv_bfloat16* bpc;
  double* U;
  __nv_bfloat16* rpc;
  float* G;
  float* wbuf;         // B x ldp, or NULL
  int* slot_cur;       // B: slot of u^t (read by the forward product)
  int* slot_new;       // B: slot the forward product writes
  double* fpart;       // B x nft x 2: sums of F(u^{t+1}) and of F(u^{t+1}) - F(u^t)
  double* ncpart;      // B x nrt
  BNode* nodes;        // B
  BCert* cert;         // B
  double* beta_out;    // B x p (certified iterate, FP64)
  double* z_out;       // B x p (relaxed z), or NULL
};

__host__ __device__ inline int batch_nrt(int n) { return (n + kBThreads * kBRows - 1) / (kBThreads * kBRows); }

size_t bprox_smem_bytes(int wsm);
void batch_prepare(int optin);
void launch_bresid(const BatchDev& d, cudaStream_t s);
void launch_bprox(const BatchDev& d, cudaStream_t s);
void launch_bstep(const BatchDev& d, cudaStream_t s);
void launch_binit_split(const BatchDev& d, cudaStream_t s);
void launch_binit_node(const BatchDev& d, cudaStream_t s);
// FP64 certificate of node b through the single-node workspace d
void launch_bcert_load(const BatchDev& bd, int b, const Dev& d, cudaStream_t s);
void launch_bcert_store(const BatchDev& bd, int b, const Dev& d, int want_z, cudaStream_t s);

}  // namespace ksc
