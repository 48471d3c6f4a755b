// ksc_launch.h -- host-side view of one node-solve workspace and the launchers
// of the single-node kernels (restarted FISTA, Algorithm 3; power iteration for
// L; the FP64 weak-duality certificate of Sec. 3.4).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "ksc_state.cuh"

namespace ksc {

enum XDtype : int { kXF64 = 0, kXF32 = 1, kXBF16 = 2, kXFP8 = 3 };

// Tile shapes (kept in one place: the host sizes workspaces with them).
constexpr int kGradThreads = 256;   // gradient pass: threads per CTA
constexpr int kGradRows = 256;      // gradient pass: most rows per CTA (split-n)
constexpr int kGradRowsMin = 128;   // gradient pass: fewest rows per CTA the balancing picks
constexpr int kFwdThreads = 256;    // forward pass: 8 warps
constexpr int kFwdRows = 32;        // forward pass: 4 rows per warp
constexpr int kFwdChunk = 2048;     // forward pass: staged columns of beta
constexpr int kProxCap = 4096;      // prox candidates (k' + pooled tail) in shared memory
constexpr int kSegLen = 256;        // prox apply: coordinates per CTA (one compaction segment)
constexpr int kMaxSegSparse = 4096; // sparse forward pass needs p <= kSegLen * this
constexpr int kSpRows = 256;        // sparse forward pass: rows per CTA (one per thread)
constexpr int kSpSplit = 16;        // sparse forward pass: chunks of the nonzero list
constexpr int kSpStage = 1024;      // sparse forward pass: list entries staged per round
constexpr int kLanczosMax = 512;    // Lanczos steps for lambda_max(X^T X)

__host__ __device__ inline int cols_per_thread(int xdt) { return xdt == kXF64 ? 2 : (xdt == kXF32 ? 4 : 8); }   // FP8: 8 per 8-byte load

struct Dev {
  int xdt;
  const void* X;
  int64_t ldx;
  const float* xscale;     // FP8 X: p power-of-two column scales (the matrix is X_ij s_j); else NULL
  const void* Xc;          // column-major copy of X (ldc >= n), for the sparse forward pass
  int64_t ldc;
  int n, p;
  int grow;                // gradient pass: rows per CTA (kGradRowsMin..kGradRows, grad_rows())
  int vec;                 // rows are 16-byte aligned: vector loads
  int loss;
  const double* y;         // n
  const double* colnorm;   // p, FP64 column 2-norms rounded up
  int8_t* state;           // p (node coordinate states)
  int* one_idx;            // p: the indices of S1, ascending (the first NodeDev::n_one)
  void* beta;              // 3 slots x p, FP64
  double* u;               // 3 slots x n: X beta in FP64
  double* grad;            // p: X^T grad F(u_gamma) in FP64
  void* wbuf;              // p, FP64 prox scratch
  int* nnz_idx;            // p: nonzeros of the newest iterate, kSegLen-long segments
  int sp_cap;              // sparse (column-major) forward pass when nnz <= sp_cap
  double* sp_part;         // kSpSplit x n partial products of the sparse forward pass
  int* cnt_sp;             // ceil(n / kSpRows) completion counters
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
  int prox_wsm;            // prox keeps w in shared memory (elements), 0 = global scratch
  // grid prox
  unsigned* key;           // p: float bits of |w| on the free set, 0 elsewhere
  unsigned* dkey;          // p: float bits of |grad| on the free set, 0 elsewhere
  unsigned* hist;          // 2 x 2048: first radix digit of key / dkey (zero between steps)
  unsigned long long* cand_a;  // kProxCap: |w| bits of the predicted prox candidates
  int* cand_i;                 // kProxCap: their indices
  unsigned long long* dcand;   // kProxCap: |grad| bits of the predicted dual candidates
  int* ccount;                 // 2: appended prox / dual candidates (may exceed kProxCap)
  float* bhi;              // p: newest iterate split b = bhi + blo (dense forward pass)
  float* blo;
  int* seg_cnt;            // nseg: nonzeros per apply segment
  int* seg_off;            // nseg + 1: exclusive prefix of seg_cnt
  double* segpart;         // 2 x nseg: sum |b_F| and sum_{S1} b^2 per segment
  double* tbeta;           // kProxCap: |b| of the top set, descending (for Algorithm 2)
  int nseg;
  // Lanczos for lambda_max(X^T X)
  double* vcur;            // p
  double* vprev;           // p
  float* vhi;              // p: vcur = vhi + vlo
  float* vlo;
  double* lz;              // alpha[kLanczosMax], beta[kLanczosMax]
};

__host__ __device__ inline int grad_ncol(const Dev& d) {
  const int tile = kGradThreads * cols_per_thread(d.xdt);
  return (d.p + tile - 1) / tile;
}
__host__ __device__ inline int grad_nrb(const Dev& d) { return (d.n + d.grow - 1) / d.grow; }
__host__ __device__ inline int grad_nrb_max(const Dev& d) { return (d.n + kGradRowsMin - 1) / kGradRowsMin; }
// Rows per CTA of a streaming pass over `rows` x (strips column strips) whose CTAs
// all do equal work: `slots` CTAs run at once (SMs x CTAs per SM), so the pass
// takes whole waves of them; the choice in [kGradRowsMin, kGradRows] (a multiple
// of 4, the main loop's row step) minimises waves x rows per CTA, the larger on ties.
inline int balanced_rows(int rows, int strips, int slots) {
  int best = kGradRows;
  double best_cost = 1e300;
  for (int r = kGradRows; r >= kGradRowsMin; r -= 4) {
    const long long ctas = (long long)((rows + r - 1) / r) * strips;
    const long long waves = (ctas + slots - 1) / slots;
    const double cost = (double)waves * r;
    if (cost < best_cost * (1.0 - 1e-12)) { best_cost = cost; best = r; }
  }
  return best;
}
int grad_rows(const Dev& d);   // balanced_rows for the gradient pass of this problem

// Stop test of the Lanczos iteration for L, taken every 8 steps: theta, prev and
// prev2 are the largest Ritz value now, 8 and 16 steps earlier (<= 0: not yet
// taken).  The Ritz value rises monotonically to lambda_max and L keeps a 1% margin.
// With the rises d1, d2 over the last two 8-step blocks shrinking (q = d2/d1 < 1),
// the geometric tail d2 q / (1 - q) estimates what is left (Aitken); stop once that
// is at most 1e-3 of theta, or a block moves it by at most 1e-5 of itself.  On the
// 20000 x 50000 Toeplitz(0.9) instance this stops after 32 steps, 3e-4 below
// lambda_max (64 steps under the 1e-5 rise alone).
inline bool lanczos_stop(double theta, double prev, double prev2) {
  if (!(prev > 0)) return false;
  const double d2 = theta - prev;
  if (d2 <= 1e-5 * theta && d2 >= -1e-5 * theta) return true;
  if (!(prev2 > 0)) return false;
  const double d1 = prev - prev2;
  if (d1 > 0 && d2 >= 0 && d2 < d1) {
    const double q = d2 / d1;
    return d2 * q / (1.0 - q) <= 1e-3 * theta;
  }
  return false;
}
__host__ __device__ inline int fwd_ntiles(const Dev& d) { return (d.n + kFwdRows - 1) / kFwdRows; }
__host__ __device__ inline int sp_nrb(const Dev& d) { return (d.n + kSpRows - 1) / kSpRows; }
size_t prox_smem_bytes(const Dev& d);
// counters layout inside Dev::cnt
__host__ __device__ inline int cnt_grad(const Dev&) { return 0; }
__host__ __device__ inline int cnt_fwd(const Dev& d) { return grad_ncol(d) + 1; }
__host__ __device__ inline int cnt_apply(const Dev& d) { return grad_ncol(d) + 2; }
__host__ __device__ inline int cnt_lz(const Dev& d) { return grad_ncol(d) + 3; }
// the generic streaming matvec's per-strip counters (max of its column strips over
// the two shapes p x n and n x p)
__host__ __device__ inline int cnt_colsum(const Dev& d) { return grad_ncol(d) + 8; }
__host__ __device__ inline int colsum_strips(const Dev& d) {
  const int tile = kGradThreads * cols_per_thread(d.xdt);
  const int a = (d.n + tile - 1) / tile, b = (d.p + tile - 1) / tile;
  return a > b ? a : b;
}
__host__ __device__ inline int cnt_total(const Dev& d) { return grad_ncol(d) + 8 + colsum_strips(d) + 1; }
// gradient-partials workspace (doubles): max of the two streaming shapes
__host__ __device__ inline size_t ws_elems(const Dev& d) {
  const size_t a = (size_t)((d.n + kGradRowsMin - 1) / kGradRowsMin) * d.p;
  const size_t b = (size_t)((d.p + kGradRowsMin - 1) / kGradRowsMin) * d.n;
  return a > b ? a : b;
}

// one FISTA step: gradient pass (+ prox input and keys), prox select and apply
// (+ g, dual TopSum), forward pass + step logic.  ev (optional): 4 events around
// the gradient pass, the prox kernels and the forward pass.
void launch_step(const Dev& d, cudaStream_t s, cudaEvent_t* ev, bool eig);   // eig: the eigen-perspective step
// g(beta^1), u^1 = X beta^1 and the objective L^1 (the start of Algorithm 3)
void launch_init(const Dev& d, cudaStream_t s);
// FP64 certificate at the current iterate (projection onto dom g, u, zeta,
// a = X^T zeta, G*, g, margins)
void launch_certificate(const Dev& d, cudaStream_t s, int want_z);
// Lanczos on X^T X: start vector (scaled by inv_norm), then step `it`
// (v_{it+1}, alpha_it, beta_it into d.lz)
void launch_lanczos_start(const Dev& d, cudaStream_t s, double inv_norm);
void launch_lanczos_step(const Dev& d, cudaStream_t s, int it);
// split the FP64 vector src into hi + lo floats (grid-wide)
void launch_split(const double* src, float* hi, float* lo, int n, cudaStream_t s);
// FP64 column norms (rounded up) for the certificate's error bound
void launch_colnorm(const Dev& d, cudaStream_t s);
// column-major copy Xc of X
void launch_transpose(const Dev& d, cudaStream_t s);
// BF16 copy of E4M3 rows times their column (per_col) or row scales; padding zeroed
void launch_fp8_to_bf16(const void* src, int64_t ld_src, int rows, int cols, const float* scale, int per_col,
                        void* dst, int64_t ld_dst, cudaStream_t s);
// per row of X: max_j |x_ij| and sum_j |x_ij| (the Poisson / Gamma step constant)
void launch_rowstats(const Dev& d, double* rmax, double* rl1, cudaStream_t s);
// set the kernels' dynamic shared memory limits, once per device (the first call
// on each device does it under a lock; later calls return at once); returns the
// first failing CUDA call's error, and the device is set up again on the next call
cudaError_t prox_prepare();

// primitives (one CTA, FP64)
// prox of g for `count` vectors (device rows with leading dims ldw, ldb), one CTA each
int prox_rows_cap();
// g (Algorithm 2) of `count` device rows of length p (row stride ldb), one CTA per row
void launch_gvalue_rows(const double* beta, int64_t ldb, int p, int count, int k, double M, double* g,
                        cudaStream_t s);
void launch_prox_rows(const double* w, int64_t ldw, double* beta, int64_t ldb, int p, int count, int k,
                      double M, double rho, cudaStream_t s);
void launch_prox_prim(const double* w, int p, int k, double M, double rho, double* beta,
                      int* top, double* wbuf, cudaStream_t s);
void launch_gvalue_prim(const double* beta, int p, int k, double M, double* g, double* z,
                        cudaStream_t s);
void launch_gstar_prim(const double* a, int p, int k, double M, double* out, cudaStream_t s);

}  // namespace ksc
