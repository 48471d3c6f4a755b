// ksc_launch.h -- host-side view of one node-solve workspace and the launchers
// of the single-node kernels (restarted FISTA, Algorithm 3; power iteration for
// L; the FP64 weak-duality certificate of Sec. 3.4).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ksc_state.cuh"

namespace ksc {

enum XDtype : int { kXF64 = 0, kXF32 = 1, kXBF16 = 2 };

// Tile shapes (kept in one place: the host sizes workspaces with them).
constexpr int kGradThreads = 256;   // gradient pass: threads per CTA
constexpr int kGradRows = 256;      // gradient pass: rows per CTA (split-n)
constexpr int kFwdThreads = 256;    // forward pass: 8 warps
constexpr int kFwdRows = 32;        // forward pass: 4 rows per warp
constexpr int kFwdChunk = 2048;     // forward pass: staged columns of beta
constexpr int kProxCap = 4096;      // prox candidates (k' + pooled tail) in shared memory

__host__ __device__ inline int cols_per_thread(int xdt) { return xdt == kXF64 ? 2 : (xdt == kXF32 ? 4 : 8); }

struct Dev {
  int xdt;
  const void* X;
  int64_t ldx;
  int n, p;
  int vec;                 // rows are 16-byte aligned: vector loads
  int loss;
  const double* y;         // n
  const double* colnorm;   // p, FP64 column 2-norms rounded up
  int8_t* state;           // p (node coordinate states)
  void* beta;              // 3 slots x p, FP64
  double* u;               // 3 slots x n: X beta in FP64
  double* grad;            // p: X^T grad F(u_gamma) in FP64
  void* wbuf;              // p, FP64 prox scratch
  void* nnz_val;           // p, FP64
  int* nnz_idx;            // p
  int nnz_cap;             // sparse forward pass when nnz <= nnz_cap
  void* ws;                // gradient partials: nrb x p doubles
  int* cnt;                // completion counters (zeroed once; kernels reset them)
  double* ncpart;          // nrb
  double* fpart;           // 4 x nft
  double* u64;             // n   certificate
  double* zeta;            // n
  double* a64;             // p
  double* z64;             // p   relaxed z
  double* b64;             // p   final iterate promoted
  NodeDev* nd;
  void* pow_v;             // p, FP64
  double* pow_lam;         // power-iteration history
  int prox_wsm;            // prox keeps w in shared memory (elements), 0 = global scratch
};

__host__ __device__ inline int grad_ncol(const Dev& d) {
  const int tile = kGradThreads * cols_per_thread(d.xdt);
  return (d.p + tile - 1) / tile;
}
__host__ __device__ inline int grad_nrb(const Dev& d) { return (d.n + kGradRows - 1) / kGradRows; }
__host__ __device__ inline int fwd_ntiles(const Dev& d) { return (d.n + kFwdRows - 1) / kFwdRows; }
size_t prox_smem_bytes(const Dev& d);
// counters layout inside Dev::cnt
__host__ __device__ inline int cnt_grad(const Dev&) { return 0; }
__host__ __device__ inline int cnt_fwd(const Dev& d) { return grad_ncol(d) + 1; }
__host__ __device__ inline int cnt_total(const Dev& d) { return grad_ncol(d) + 8; }

// one FISTA step: gradient pass, prox (+ g, dual TopSum), forward pass + step logic.
// ev (optional): 6 events recorded around the three kernels.
void launch_step(const Dev& d, cudaStream_t s, cudaEvent_t* ev);
// g(beta^1), u^1 = X beta^1 and the objective L^1 (Algorithm 3, lines 1-2)
void launch_init(const Dev& d, cudaStream_t s);
// FP64 certificate at the current iterate (projection onto dom g, u, zeta,
// a = X^T zeta, G*, g, margins)
void launch_certificate(const Dev& d, cudaStream_t s, int want_z);
// one power-iteration step v <- X^T X v / ||X^T X v||, lam[it] = ||X^T X v||
void launch_power_step(const Dev& d, cudaStream_t s, int it);
void launch_power_init(const Dev& d, cudaStream_t s);
// FP64 column norms (rounded up) for the certificate's error bound
void launch_colnorm(const Dev& d, cudaStream_t s);
// set the prox kernels' dynamic shared memory limits once per process
void prox_prepare();

// primitives (one CTA, FP64)
void launch_prox_prim(const double* w, int p, int k, double M, double rho, double* beta,
                      int* top, double* wbuf, cudaStream_t s);
void launch_gvalue_prim(const double* beta, int p, int k, double M, double* g, double* z,
                        cudaStream_t s);
void launch_gstar_prim(const double* a, int p, int k, double M, double* out, cudaStream_t s);

}  // namespace ksc
