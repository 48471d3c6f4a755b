// ksc_eig.cu -- the shift of the eigen-perspective relaxation (App. D.2): a
// certified lower bound lambda on lambda_min(X^T X), so that Q = X^T X - lambda I
// is positive semidefinite and the eigen-perspective bound is a valid weak-duality
// bound whatever rounding the computation of lambda met.
//
// A = X^T X is formed in FP64 on the device; lambda_min(A) is bracketed by
// bisection on a shift c, c counting as below lambda_min when the Cholesky
// factorisation of H = A - c I runs to completion.  A completed floating-point
// Cholesky factorisation R of a symmetric H satisfies R^T R = H + dH with
// |dH| <= gamma_{p+1} |R^T| |R| (Higham, Accuracy and Stability of Numerical
// Algorithms, 2nd ed., Thm 10.3; any order of the inner sums, FMA included), so
// H + dH is positive semidefinite and lambda_min(H) >= -||dH||_2 >= -gamma_{p+1}
// ||R||_F^2.  With the rounding of the shifted diagonal (u |H_ii| per entry) and of
// the Gram matrix (|fl(X^T X) - X^T X| <= gamma_n |X|^T |X|, spectral norm at most
// gamma_n ||X||_F^2):
//   lambda_min(X^T X) >= c - gamma_{p+1} ||R||_F^2 - u max_i |H_ii| - gamma_n ||X||_F^2,
// gamma_m = m u / (1 - m u), u = 2^-53.  The certified lambda is that right-hand
// side at the largest shift that factorised, clipped at 0.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <string>
#include <vector>

#include "ksc_common.cuh"
#include "ksc_launch.h"
#include "ksc_problem.h"

#define KE_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return api_fail(e_ == cudaErrorMemoryAllocation ? KSC_ERR_OOM : KSC_ERR_CUDA,          \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

namespace ksc {

namespace {

constexpr int kGramT = 32;

// A(i, k) = sum_r X_ri X_rk for the lower tiles (i >= k tile-wise), stored
// column-major (A[k p + i]); products of FP32/BF16/FP8-times-scale values are
// exact in FP64, the sum runs over r in order
template <typename TX>
__global__ void __launch_bounds__(256) k_gram(const TX* __restrict__ X, int64_t ldx, int n, int p,
                                              const float* __restrict__ xscale, double* __restrict__ A) {
  if (blockIdx.x > blockIdx.y) return;
  __shared__ double Xi[kGramT][kGramT + 1];
  __shared__ double Xk[kGramT][kGramT + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 32 x 8
  const int i0 = blockIdx.y * kGramT, k0 = blockIdx.x * kGramT;
  double acc[4] = {0.0, 0.0, 0.0, 0.0};
  for (int r0 = 0; r0 < n; r0 += kGramT) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int rr = ty + 8 * q, r = r0 + rr;
      const int ci = i0 + tx, ck = k0 + tx;
      double vi = 0.0, vk = 0.0;
      if (r < n && ci < p) {
        vi = xval<double>(X[(size_t)r * ldx + ci]);
        if (is_fp8<TX>()) vi *= (double)xscale[ci];
      }
      if (r < n && ck < p) {
        vk = xval<double>(X[(size_t)r * ldx + ck]);
        if (is_fp8<TX>()) vk *= (double)xscale[ck];
      }
      Xi[rr][tx] = vi;
      Xk[rr][tx] = vk;
    }
    __syncthreads();
#pragma unroll 8
    for (int rr = 0; rr < kGramT; ++rr) {
      const double b = Xk[rr][tx];
#pragma unroll
      for (int q = 0; q < 4; ++q) acc[q] = fma(Xi[rr][ty + 8 * q], b, acc[q]);
    }
    __syncthreads();
  }
  const int k = k0 + tx;
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int i = i0 + ty + 8 * q;
    if (i < p && k < p && k <= i) A[(size_t)k * p + i] = acc[q];
  }
}

// W = A - c I on the lower triangle (column-major)
__global__ void __launch_bounds__(256) k_chol_prep(const double* __restrict__ A, double* __restrict__ W, int p,
                                                   double c) {
  const int k = blockIdx.y;
  for (int i = k + blockIdx.x * 256 + (int)threadIdx.x; i < p; i += gridDim.x * 256) {
    const double v = A[(size_t)k * p + i];
    W[(size_t)k * p + i] = (i == k) ? v - c : v;
  }
}

struct CholState {
  int fail;      // 0, or 1 + the column whose pivot was not positive
  int pad;
  double fro;    // sum of the squares of the factor's entries so far
};

// column j of the factor: pivot sqrt(W_jj), the column below it divided by the
// pivot; one CTA
__global__ void __launch_bounds__(256) k_chol_col(double* __restrict__ W, int p, int j, CholState* st) {
  __shared__ double red[64];
  if (st->fail) return;
  const double dj = W[(size_t)j * p + j];
  if (!(dj > 0.0)) {   // every thread reads the same pivot
    if (threadIdx.x == 0) st->fail = j + 1;
    return;
  }
  const double r = sqrt(dj);
  double s = 0.0;
  double* col = W + (size_t)j * p;
  for (int i = j + 1 + (int)threadIdx.x; i < p; i += 256) {
    const double v = col[i] / r;
    col[i] = v;
    s += v * v;
  }
  s = block_sum<double, 256>(s, red);
  if (threadIdx.x == 0) {
    col[j] = r;
    st->fro += s + r * r;
  }
}

// trailing update W(i, k) -= L(i, j) L(k, j) for j < k <= i: 256 rows x 32
// columns per CTA, coalesced along the rows of each column
__global__ void __launch_bounds__(256) k_chol_upd(double* __restrict__ W, int p, int j, const CholState* st) {
  if (st->fail) return;
  const int kb = j + 1 + blockIdx.y * 32;
  const int ib = j + 1 + blockIdx.x * 256;
  if (ib + 255 < kb) return;   // the tile lies above the diagonal
  __shared__ double lk[32];
  const double* lj = W + (size_t)j * p;
  if (threadIdx.x < 32) lk[threadIdx.x] = (kb + (int)threadIdx.x < p) ? lj[kb + threadIdx.x] : 0.0;
  __syncthreads();
  const int i = ib + (int)threadIdx.x;
  if (i >= p) return;
  const double li = lj[i];
  const int kend = min(min(kb + 32, p), i + 1);
  for (int k = kb; k < kend; ++k) {
    double* w = W + (size_t)k * p + i;
    *w = fma(-li, lk[k - kb], *w);
  }
}

}  // namespace

}  // namespace ksc

using namespace ksc;

// the Gram matrix of a problem and the workspace of its shifted factorisations
struct EigWork {
  ksc_problem* pr = nullptr;
  cudaStream_t s = nullptr;
  int n = 0, p = 0;
  double* A = nullptr;
  double* W = nullptr;
  CholState* st = nullptr;
  double dmin = 0.0, dmax = 0.0, trace = 0.0, xf2 = 0.0;
  ~EigWork() {
    if (A) cudaFree(A);
    if (W) cudaFree(W);
    if (st) cudaFree(st);
  }
};

static ksc_status eig_begin(EigWork* w, ksc_problem* pr, cudaStream_t s) {
  const int n = (int)pr->n, p = (int)pr->p;
  w->pr = pr;
  w->s = s;
  w->n = n;
  w->p = p;
  if (cudaMalloc(&w->A, (size_t)p * p * 8) != cudaSuccess || cudaMalloc(&w->W, (size_t)p * p * 8) != cudaSuccess ||
      cudaMalloc(&w->st, sizeof(CholState)) != cudaSuccess) {
    cudaGetLastError();
    return api_fail(KSC_ERR_OOM, "eigen shift: Gram matrix workspace");
  }
  const Dev& d = pr->dev;
  const dim3 g((p + kGramT - 1) / kGramT, (p + kGramT - 1) / kGramT);
  if (d.xdt == kXF64)
    k_gram<double><<<g, 256, 0, s>>>((const double*)d.X, d.ldx, n, p, nullptr, w->A);
  else if (d.xdt == kXF32)
    k_gram<float><<<g, 256, 0, s>>>((const float*)d.X, d.ldx, n, p, nullptr, w->A);
  else if (d.xdt == kXBF16)
    k_gram<__nv_bfloat16><<<g, 256, 0, s>>>((const __nv_bfloat16*)d.X, d.ldx, n, p, nullptr, w->A);
  else
    k_gram<__nv_fp8_e4m3><<<g, 256, 0, s>>>((const __nv_fp8_e4m3*)d.X, d.ldx, n, p, d.xscale, w->A);
  pr->launches += 1;
  KE_CUDA(cudaGetLastError());
  std::vector<double> diag(p), cn(p);
  KE_CUDA(cudaMemcpy2DAsync(diag.data(), 8, w->A, (size_t)(p + 1) * 8, 8, p, cudaMemcpyDeviceToHost, s));
  KE_CUDA(cudaMemcpyAsync(cn.data(), d.colnorm, (size_t)p * 8, cudaMemcpyDeviceToHost, s));
  KE_CUDA(cudaStreamSynchronize(s));
  w->dmin = w->dmax = diag[0];
  for (int j = 0; j < p; ++j) {
    w->dmin = std::min(w->dmin, diag[j]);
    w->dmax = std::max(w->dmax, diag[j]);
    w->trace += diag[j];
    w->xf2 += cn[j] * cn[j];   // column norms are rounded up
  }
  return KSC_OK;
}

// the rounding terms of the certificate after a factorisation with ||R||_F^2 = fro
static double eig_margin(const EigWork& w, double fro) {
  const double u = 1.1102230246251565e-16;
  auto gamma = [&](double m) { return m * u / (1.0 - m * u); };
  return 1.01 * (gamma(w.p + 1.0) * fro * (1.0 + 1e-7) + u * w.dmax + gamma((double)w.n) * w.xf2 * (1.0 + 1e-7));
}

// factorise A - c I; *cert = the certified lower bound on lambda_min(X^T X) it
// gives (c - margin), or -inf when the factorisation broke down
static ksc_status eig_try(EigWork* w, double c, double* cert) {
  const int p = w->p;
  cudaStream_t s = w->s;
  KE_CUDA(cudaMemsetAsync(w->st, 0, sizeof(CholState), s));
  k_chol_prep<<<dim3((p + 255) / 256 < 32 ? (p + 255) / 256 : 32, p), 256, 0, s>>>(w->A, w->W, p, c);
  for (int j = 0; j < p; ++j) {
    k_chol_col<<<1, 256, 0, s>>>(w->W, p, j, w->st);
    const int m = p - j - 1;
    if (m > 0) k_chol_upd<<<dim3((m + 255) / 256, (m + 31) / 32), 256, 0, s>>>(w->W, p, j, w->st);
  }
  w->pr->launches += 2 * (int64_t)p;
  KE_CUDA(cudaGetLastError());
  CholState h{};
  KE_CUDA(cudaMemcpyAsync(&h, w->st, sizeof h, cudaMemcpyDeviceToHost, s));
  KE_CUDA(cudaStreamSynchronize(s));
  *cert = h.fail == 0 ? c - eig_margin(*w, h.fro) : -INFINITY;
  return KSC_OK;
}

static ksc_status eig_compute(ksc_problem* pr, cudaStream_t s, double* lam) {
  *lam = 0.0;
  if (pr->n < pr->p) return KSC_OK;   // X^T X is singular: the eigen shift is 0
  EigWork w;
  ksc_status rc = eig_begin(&w, pr, s);
  if (rc != KSC_OK) return rc;
  double cert = 0.0;
  if ((rc = eig_try(&w, 0.0, &cert)) != KSC_OK || !(cert > -INFINITY)) return rc;   // singular: no shift
  // bisection on [lo, hi]: lo factorised, hi (at first the smallest diagonal entry,
  // a Rayleigh quotient) did not; to 1e-3 of lo
  double lo = 0.0, best = 0.0, hi = w.dmin;
  for (int it = 0; it < 48 && (lo == 0.0 || hi - lo > 1e-3 * lo); ++it) {
    const double mid = 0.5 * (lo + hi);
    if ((rc = eig_try(&w, mid, &cert)) != KSC_OK) return rc;
    if (cert > -INFINITY) {
      lo = mid;
      best = cert;
    } else {
      hi = mid;
    }
  }
  *lam = std::max(0.0, best);
  return KSC_OK;
}

extern "C" ksc_status ksc_problem_eig_lambda(ksc_problem* pr, void* cuda_stream, double* lambda) {
  if (!pr || !lambda) return api_fail(KSC_ERR_INVALID_ARG, "problem and lambda must be non-NULL");
  if (pr->eig_ready) {
    *lambda = pr->eig_lambda;
    return KSC_OK;
  }
  if (pr->n >= pr->p && pr->p > kEigMaxP)
    return api_fail(KSC_ERR_UNIMPLEMENTED, "eigen shift: p > 8192 with n >= p");
  ksc_status st = ensure_prepared();
  if (st != KSC_OK) return st;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != pr->device && cudaSetDevice(pr->device) != cudaSuccess) return api_fail(KSC_ERR_CUDA, "cudaSetDevice");
  double lam = 0.0;
  st = eig_compute(pr, (cudaStream_t)cuda_stream, &lam);
  if (st != KSC_OK) return st;
  pr->eig_lambda = lam;
  pr->eig_ready = true;
  *lambda = lam;
  return KSC_OK;
}

extern "C" ksc_status ksc_problem_set_eig_lambda(ksc_problem* pr, void* cuda_stream, double lambda) {
  if (!pr) return api_fail(KSC_ERR_INVALID_ARG, "problem is NULL");
  if (!(lambda >= 0.0) || !std::isfinite(lambda)) return api_fail(KSC_ERR_INVALID_ARG, "lambda must be >= 0");
  if (lambda > 0.0) {
    if (pr->n < pr->p) return api_fail(KSC_ERR_INVALID_ARG, "lambda above lambda_min(X^T X) = 0 (n < p)");
    if (pr->p > kEigMaxP) return api_fail(KSC_ERR_UNIMPLEMENTED, "eigen shift: p > 8192 with n >= p");
    ksc_status st = ensure_prepared();
    if (st != KSC_OK) return st;
    int cur = 0;
    cudaGetDevice(&cur);
    if (cur != pr->device && cudaSetDevice(pr->device) != cudaSuccess) return api_fail(KSC_ERR_CUDA, "cudaSetDevice");
    EigWork w;
    if ((st = eig_begin(&w, pr, (cudaStream_t)cuda_stream)) != KSC_OK) return st;
    // the factorisation at lambda plus the margin it is expected to cost
    // (||R||_F^2 <= trace(A - c I) + its rounding)
    const double c = lambda + eig_margin(w, 1.01 * w.trace);
    double cert = 0.0;
    if ((st = eig_try(&w, c, &cert)) != KSC_OK) return st;
    if (!(cert >= lambda)) return api_fail(KSC_ERR_INVALID_ARG, "lambda is not certified below lambda_min(X^T X)");
  }
  pr->eig_lambda = lambda;
  pr->eig_ready = true;
  return KSC_OK;
}
