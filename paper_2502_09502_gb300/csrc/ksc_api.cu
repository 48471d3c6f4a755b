// ksc_api.cu -- the C ABI (include/ksc.h): problem lifetime, the host loop of a
// node solve (CUDA-graph replays of FISTA steps, FP64 certificate, early
// termination), and the FP64 primitives.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "../../include/ksc.h"
#include "ksc_launch.h"
#include "ksc_problem.h"
#include "ksc_state.cuh"

using namespace ksc;

namespace ksc {
size_t prox_smem_limit();
}

// ------------------------------------------------------------------ errors

static thread_local std::string g_err;

static ksc_status fail(ksc_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

// shared with the other translation units of the library
ksc_status ksc_internal_fail(ksc_status st, const char* msg) { return fail(st, msg); }
ksc_status ksc::api_fail(ksc_status st, const std::string& msg) { return fail(st, msg); }

#define KSC_CUDA(call)                                                              \
  do {                                                                              \
    cudaError_t e_ = (call);                                                        \
    if (e_ != cudaSuccess) {                                                        \
      return fail(e_ == cudaErrorMemoryAllocation ? KSC_ERR_OOM : KSC_ERR_CUDA,     \
                  std::string(#call) + ": " + cudaGetErrorString(e_));              \
    }                                                                               \
  } while (0)

// per-device one-time set-up (k_prox.cu keeps the per-device state and its lock)
ksc_status ksc::ensure_prepared() {
  const cudaError_t e = prox_prepare();
  if (e != cudaSuccess) return fail(KSC_ERR_CUDA, std::string("prepare: ") + cudaGetErrorString(e));
  return KSC_OK;
}

// ------------------------------------------------------------------ problem

// kernels per launcher (kept beside the launchers they count)
static constexpr int kLaunchesPerStep = 5;      // gradient, prox select, prox apply, 2 forward
static constexpr int kLaunchesPerCert = 5;      // prep, 2 forward, gradient, final
static constexpr int kLaunchesPerInit = 3;      // g value, split, forward
static constexpr int kLaunchesPerLanczos = 5;   // forward, gradient, three vector phases

// the iterate vectors are FP64 for every storage type of X
static size_t tbytes(int) { return 8; }
static size_t xbytes(int xdt) { return xdt == kXF64 ? 8 : (xdt == kXF32 ? 4 : (xdt == kXFP8 ? 1 : 2)); }

template <typename P>
static ksc_status dmalloc(ksc_problem* pr, P** ptr, size_t bytes) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess)
    return fail(KSC_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  pr->allocs.push_back(v);
  pr->bytes += bytes;
  *ptr = (P*)v;
  return KSC_OK;
}

static void free_problem(ksc_problem* pr) {
  if (!pr) return;
  int cur = 0;
  cudaGetDevice(&cur);
  cudaSetDevice(pr->device);
  if (pr->graph) cudaGraphExecDestroy(pr->graph);
  if (pr->graph_prof) cudaGraphExecDestroy(pr->graph_prof);
  if (pr->graph_eig) cudaGraphExecDestroy(pr->graph_eig);
  if (pr->graph_eig_prof) cudaGraphExecDestroy(pr->graph_eig_prof);
  free_batch(pr->batch);
  for (auto e : pr->events) cudaEventDestroy(e);
  for (void* v : pr->allocs) cudaFree(v);
  cudaSetDevice(cur);
  delete pr;
}

static ksc_status alloc_workspace(ksc_problem* pr) {
  Dev& d = pr->dev;
  const int64_t n = pr->n, p = pr->p;
  const size_t tb = tbytes(pr->xdt);
  ksc_status st;
#define ALLOC(ptr, bytes) \
  if ((st = dmalloc(pr, &(ptr), (bytes))) != KSC_OK) return st
  ALLOC(d.beta, 3 * p * tb);
  ALLOC(d.u, 3 * n * 8);
  ALLOC(d.grad, p * 8);
  ALLOC(d.wbuf, p * tb);
  ALLOC(d.nnz_idx, p * sizeof(int));
  ALLOC(d.ws, ws_elems(d) * 8);
  ALLOC(d.cnt, (size_t)cnt_total(d) * sizeof(int));
  ALLOC(d.ncpart, (size_t)grad_nrb_max(d) * 8);
  ALLOC(d.fpart, (size_t)fwd_ntiles(d) * 4 * 8);
  ALLOC(d.u64, n * 8);
  ALLOC(d.zeta, n * 8);
  ALLOC(d.a64, p * 8);
  ALLOC(d.z64, p * 8);
  ALLOC(d.b64, p * 8);
  double* cn = nullptr;
  ALLOC(cn, p * 8);
  d.colnorm = cn;
  ALLOC(d.state, p);
  ALLOC(d.one_idx, (size_t)p * 4);
  d.nseg = (int)((p + kSegLen - 1) / kSegLen);
  ALLOC(d.key, p * 4);
  ALLOC(d.dkey, p * 4);
  ALLOC(d.hist, 2 * 2048 * 4);
  ALLOC(d.bhi, p * 4);
  ALLOC(d.blo, p * 4);
  ALLOC(d.seg_cnt, (size_t)d.nseg * 4);
  ALLOC(d.seg_off, (size_t)(d.nseg + 1) * 4);
  ALLOC(d.segpart, (size_t)3 * d.nseg * 8);
  ALLOC(d.tbeta, (size_t)kProxCap * 8);
  ALLOC(d.cand_a, (size_t)kProxCap * 8);
  ALLOC(d.cand_i, (size_t)kProxCap * 4);
  ALLOC(d.dcand, (size_t)kProxCap * 8);
  ALLOC(d.ccount, 2 * 4);
  ALLOC(d.vcur, p * 8);
  ALLOC(d.vprev, p * 8);
  ALLOC(d.vhi, p * 4);
  ALLOC(d.vlo, p * 4);
  ALLOC(d.lz, 2 * kLanczosMax * 8);
  ALLOC(d.nd, sizeof(NodeDev));
  ALLOC(d.sp_part, (size_t)kSpSplit * n * 8);
  ALLOC(d.cnt_sp, (size_t)sp_nrb(d) * 4);
  {
    void* xc = nullptr;
    // a multiple of 16 bytes (TMA row stride of the batched products)
    d.ldc = pr->xdt == kXFP8 ? (n + 15) / 16 * 16 : (n + 7) / 8 * 8;
    ALLOC(xc, (size_t)d.ldc * p * xbytes(pr->xdt));
    d.Xc = xc;
  }
#undef ALLOC
  KSC_CUDA(cudaMemset(d.cnt, 0, (size_t)cnt_total(d) * sizeof(int)));
  KSC_CUDA(cudaMemset(d.beta, 0, 3 * p * tb));
  KSC_CUDA(cudaMemset(d.u, 0, 3 * n * 8));
  KSC_CUDA(cudaMemset(d.state, 0, p));
  KSC_CUDA(cudaMemset(d.nd, 0, sizeof(NodeDev)));
  KSC_CUDA(cudaMemset(d.hist, 0, 2 * 2048 * 4));
  KSC_CUDA(cudaMemset(d.cnt_sp, 0, (size_t)sp_nrb(d) * 4));
  KSC_CUDA(cudaMemset(d.ccount, 0, 2 * 4));
  return KSC_OK;
}

// Largest eigenvalue of the symmetric tridiagonal (alpha[0..m), beta[0..m-1))
// by bisection on the Sturm count (number of eigenvalues below x).
static double tridiag_max_eig(const double* alpha, const double* beta, int m) {
  double lo = alpha[0], hi = alpha[0];
  for (int i = 0; i < m; ++i) {
    const double r = (i > 0 ? std::fabs(beta[i - 1]) : 0.0) + (i + 1 < m ? std::fabs(beta[i]) : 0.0);
    lo = std::min(lo, alpha[i] - r);
    hi = std::max(hi, alpha[i] + r);
  }
  auto below = [&](double x) {
    int c = 0;
    double q = alpha[0] - x;
    if (q < 0) ++c;
    for (int i = 1; i < m; ++i) {
      if (q == 0.0) q = 1e-300;
      q = (alpha[i] - x) - beta[i - 1] * beta[i - 1] / q;
      if (q < 0) ++c;
    }
    return c;
  };
  for (int it = 0; it < 200 && hi - lo > 1e-15 * std::fabs(hi); ++it) {
    const double mid = 0.5 * (lo + hi);
    if (below(mid) >= m) hi = mid; else lo = mid;
  }
  return hi;
}

// lambda_max(X^T X) by the Lanczos iteration (FP64 vectors, error-free products):
// the largest Ritz value converges far faster than power iteration on spectra
// with a small relative gap at the top.
static ksc_status lanczos_lmax(ksc_problem* pr, cudaStream_t s) {
  Dev& d = pr->dev;
  double nrm = 0.0;
  for (int64_t j = 0; j < pr->p; ++j) {
    const double v = 1.0 + (double)((unsigned long long)(j + 1) * 2654435761ull % 1000ull) / 1000.0;
    nrm += v * v;
  }
  launch_lanczos_start(d, s, 1.0 / std::sqrt(nrm));
  pr->launches += 1;
  KSC_CUDA(cudaGetLastError());
  std::vector<double> hlz(2 * kLanczosMax);
  const int maxit = (int)std::min<int64_t>(kLanczosMax, pr->p);
  double theta = 0.0, prev = -1.0, prev2 = -1.0;
  int it = 0;
  while (it < maxit) {
    const int upto = std::min(maxit, it + 8);
    for (; it < upto; ++it) launch_lanczos_step(d, s, it);
    pr->launches += (int64_t)kLaunchesPerLanczos * 8;
    KSC_CUDA(cudaGetLastError());
    KSC_CUDA(cudaMemcpyAsync(hlz.data(), d.lz, 2 * kLanczosMax * sizeof(double), cudaMemcpyDeviceToHost, s));
    KSC_CUDA(cudaStreamSynchronize(s));
    int m = it;
    bool breakdown = false;
    for (int j = 0; j < it; ++j) {
      if (!(hlz[kLanczosMax + j] > 1e-13 * std::fabs(hlz[0]) + 1e-300)) { m = j + 1; breakdown = true; break; }
    }
    theta = tridiag_max_eig(hlz.data(), hlz.data() + kLanczosMax, m);
    pr->power_iters = m;
    if (breakdown || lanczos_stop(theta, prev, prev2)) break;
    prev2 = prev;
    prev = theta;
  }
  // F' is 2-Lipschitz for least squares and the squared hinge, 1/4 for logistic;
  // Poisson and Gamma: lambda_max alone here, each node multiplies in its
  // curvature bound (node_lipschitz)
  const double cf = pr->loss == KSC_LOSS_LOGISTIC ? 0.25 : (loss_counts(pr->loss) ? 1.0 : 2.0);
  pr->L = cf * theta * 1.01;
  return KSC_OK;
}

bool ksc::loss_counts(int loss) { return loss == KSC_LOSS_POISSON || loss == KSC_LOSS_GAMMA; }

// Poisson and Gamma regression have no global Lipschitz constant (their curvature
// is e^u, y e^-u).  Every iterate lies in {|b_j| <= M, sum |b_j| <= kM}, where
// |x_i^T b| <= U_i = M min(k max_j |x_ij|, sum_j |x_ij|), and the extrapolated
// point of a step within 3 U_i; there the Hessian of F(X b) is at most
// lambda_max(X^T X) max_i c_i with c_i = e^{3 U_i} or y_i e^{3 U_i}.
double ksc::node_lipschitz(const ksc_problem* pr, double M, int k) {
  if (!loss_counts(pr->loss) || pr->l_fixed) return pr->L;
  double lc = -INFINITY;   // log max_i c_i
  for (int64_t i = 0; i < pr->n; ++i) {
    const double U = M * std::min((double)k * pr->row_max[i], pr->row_l1[i]);
    double l = 3.0 * U * (1.0 + 1e-12);
    if (pr->loss == KSC_LOSS_GAMMA) l += std::log(pr->y_host[i]);
    lc = std::max(lc, l);
  }
  return pr->L * std::exp(lc) * (1.0 + 1e-12);
}

void ksc::project_warm(const ksc_problem* pr, const NodeSetup& ns, double M, int k, double* b) {
  double l1 = 0.0;
  for (int64_t j = 0; j < pr->p; ++j) {
    b[j] = ns.state[j] == kZero ? 0.0 : std::min(M, std::max(-M, b[j]));
    l1 += std::fabs(b[j]);
  }
  if (loss_counts(pr->loss) && l1 > (double)k * M) {
    const double sc = (double)k * M / l1 * (1.0 - 1e-15);
    for (int64_t j = 0; j < pr->p; ++j) b[j] *= sc;
  }
}

extern "C" ksc_status ksc_problem_create(const ksc_problem_desc* desc, void* cuda_stream,
                                         ksc_problem** out) {
  if (!out) return fail(KSC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!desc) return fail(KSC_ERR_INVALID_ARG, "desc is NULL");
  if (desc->n < 1 || desc->p < 1) return fail(KSC_ERR_INVALID_ARG, "n and p must be >= 1");
  if (desc->n > (1ll << 31) - 1 || desc->p > (1ll << 31) - 1)
    return fail(KSC_ERR_INVALID_ARG, "n and p must be < 2^31");
  if (desc->x_dtype != KSC_F64 && desc->x_dtype != KSC_F32 && desc->x_dtype != KSC_BF16 &&
      desc->x_dtype != KSC_FP8_E4M3_COLSCALE)
    return fail(KSC_ERR_INVALID_ARG, "unknown x_dtype");
  if (desc->x_dtype == KSC_FP8_E4M3_COLSCALE) {
    // power-of-two scales: X_ij s_j is exact in FP32 (e4m3 has 4 significant bits)
    if (!desc->col_scale) return fail(KSC_ERR_INVALID_ARG, "FP8 X needs col_scale");
    for (int64_t j = 0; j < desc->p; ++j) {
      const float v = desc->col_scale[j];
      int e = 0;
      const float m = std::frexp(v, &e);
      if (!(v > 0.0f) || !std::isfinite(v) || m != 0.5f || e < -99 || e > 101)
        return fail(KSC_ERR_INVALID_ARG, "col_scale entries must be powers of two in [2^-100, 2^100]");
    }
  }
  if (desc->loss != KSC_LOSS_LSQ && desc->loss != KSC_LOSS_LOGISTIC && desc->loss != KSC_LOSS_SQHINGE &&
      desc->loss != KSC_LOSS_POISSON && desc->loss != KSC_LOSS_GAMMA)
    return fail(KSC_ERR_INVALID_ARG, "unknown loss");
  if (!desc->X || !desc->y) return fail(KSC_ERR_INVALID_ARG, "X and y must be non-NULL");
  const int64_t ldx = desc->ldx == 0 ? desc->p : desc->ldx;
  if (ldx < desc->p) return fail(KSC_ERR_INVALID_ARG, "ldx < p");
  for (int64_t i = 0; i < desc->n; ++i) {
    const double v = desc->y[i];
    if (!std::isfinite(v)) return fail(KSC_ERR_INVALID_ARG, "y has a non-finite entry");
    if ((desc->loss == KSC_LOSS_LOGISTIC || desc->loss == KSC_LOSS_SQHINGE) && v != 1.0 && v != -1.0)
      return fail(KSC_ERR_INVALID_ARG, "logistic and squared-hinge labels must be +1 or -1");
    if (desc->loss == KSC_LOSS_POISSON && !(v >= 0.0))
      return fail(KSC_ERR_INVALID_ARG, "Poisson responses must be >= 0");
    if (desc->loss == KSC_LOSS_GAMMA && !(v > 0.0))
      return fail(KSC_ERR_INVALID_ARG, "Gamma responses must be > 0");
  }
  ksc_status st = ensure_prepared();
  if (st != KSC_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  ksc_problem* pr = new ksc_problem();
  cudaGetDevice(&pr->device);
  pr->n = desc->n;
  pr->p = desc->p;
  pr->ldx = ldx;
  pr->xdt = (int)desc->x_dtype;
  pr->loss = (int)desc->loss;
  pr->y_host.assign(desc->y, desc->y + desc->n);
  Dev& d = pr->dev;
  d.xdt = pr->xdt;
  d.n = (int)pr->n;
  d.p = (int)pr->p;
  d.ldx = ldx;
  d.loss = pr->loss;
  const size_t xb = xbytes(pr->xdt);
  auto bail = [&](ksc_status e) { free_problem(pr); return e; };
  if (desc->x_on_device) {
    pr->X = const_cast<void*>(desc->X);
    pr->own_x = false;
  } else {
    void* xd = nullptr;
    if ((st = dmalloc(pr, &xd, (size_t)(pr->n - 1) * ldx * xb + (size_t)pr->p * xb)) != KSC_OK) return bail(st);
    cudaError_t e = cudaMemcpyAsync(xd, desc->X, ((size_t)(pr->n - 1) * ldx + pr->p) * xb,
                                    cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bail(fail(KSC_ERR_CUDA, std::string("copy X: ") + cudaGetErrorString(e)));
    pr->X = xd;
    pr->own_x = true;
  }
  d.X = pr->X;
  d.xscale = nullptr;
  if (pr->xdt == kXFP8) {
    float* sc = nullptr;
    if ((st = dmalloc(pr, &sc, (size_t)pr->p * 4)) != KSC_OK) return bail(st);
    cudaError_t e = cudaMemcpyAsync(sc, desc->col_scale, (size_t)pr->p * 4, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bail(fail(KSC_ERR_CUDA, std::string("copy col_scale: ") + cudaGetErrorString(e)));
    d.xscale = sc;
  }
  const int cpt = cols_per_thread(pr->xdt);
  d.vec = ((ldx % cpt) == 0 && ((uintptr_t)pr->X % 16) == 0) ? 1 : 0;
  d.grow = grad_rows(d);
  if ((st = dmalloc(pr, &pr->y, pr->n * 8)) != KSC_OK) return bail(st);
  {
    cudaError_t e = cudaMemcpyAsync(pr->y, desc->y, pr->n * 8, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return bail(fail(KSC_ERR_CUDA, std::string("copy y: ") + cudaGetErrorString(e)));
  }
  d.y = pr->y;
  if ((st = alloc_workspace(pr)) != KSC_OK) return bail(st);
  d.sp_cap = std::max(1, d.p / 2);
  // keep w in shared memory when it fits beside the prox buffers
  {
    size_t lim = prox_smem_limit();
    Dev t = d;
    t.prox_wsm = d.p;
    d.prox_wsm = (prox_smem_bytes(t) <= lim) ? d.p : 0;
  }
  launch_transpose(d, s);
  launch_colnorm(d, s);
  pr->launches += 2;
  if (cudaGetLastError() != cudaSuccess) return bail(fail(KSC_ERR_CUDA, "colnorm launch failed"));
  if (desc->lipschitz > 0) {
    pr->L = desc->lipschitz;
    pr->l_fixed = true;
  } else if ((st = lanczos_lmax(pr, s)) != KSC_OK) {
    return bail(st);
  }
  if (loss_counts(pr->loss) && !pr->l_fixed) {
    // the rows' largest entries and absolute sums, for each node's step constant
    double* rs = nullptr;
    if ((st = dmalloc(pr, &rs, (size_t)pr->n * 16)) != KSC_OK) return bail(st);
    launch_rowstats(d, rs, rs + pr->n, s);
    pr->launches += 1;
    pr->row_max.resize(pr->n);
    pr->row_l1.resize(pr->n);
    cudaError_t e1 = cudaMemcpyAsync(pr->row_max.data(), rs, (size_t)pr->n * 8, cudaMemcpyDeviceToHost, s);
    if (e1 == cudaSuccess)
      e1 = cudaMemcpyAsync(pr->row_l1.data(), rs + pr->n, (size_t)pr->n * 8, cudaMemcpyDeviceToHost, s);
    if (e1 != cudaSuccess) return bail(fail(KSC_ERR_CUDA, std::string("row statistics: ") + cudaGetErrorString(e1)));
  }
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail(fail(KSC_ERR_CUDA, std::string("problem setup: ") + cudaGetErrorString(e)));
  if (!(pr->L > 0.0) || !std::isfinite(pr->L)) return bail(fail(KSC_ERR_INVALID_ARG, "X has zero norm"));
  *out = pr;
  return KSC_OK;
}

extern "C" ksc_status ksc_problem_destroy(ksc_problem* problem) {
  free_problem(problem);
  return KSC_OK;
}

extern "C" size_t ksc_problem_bytes(const ksc_problem* problem) {
  if (!problem) return 0;
  return problem->bytes;
}

extern "C" ksc_status ksc_problem_info(const ksc_problem* problem, double* lipschitz, int32_t* power_iters) {
  if (!problem) return fail(KSC_ERR_INVALID_ARG, "problem is NULL");
  if (lipschitz) *lipschitz = problem->L;
  if (power_iters) *power_iters = problem->power_iters;
  return KSC_OK;
}

extern "C" ksc_status ksc_problem_profile(ksc_problem* problem, int32_t enable) {
  if (!problem) return fail(KSC_ERR_INVALID_ARG, "problem is NULL");
  problem->profile = enable != 0;
  return KSC_OK;
}

extern "C" ksc_status ksc_problem_kernel_time(ksc_problem* problem, int32_t kernel, int64_t* launches,
                                              double* total_ms, int32_t reset) {
  if (!problem) return fail(KSC_ERR_INVALID_ARG, "problem is NULL");
  if (kernel < 0 || kernel >= kKernelIds) return fail(KSC_ERR_INVALID_ARG, "unknown kernel id");
  if (launches) *launches = problem->k_launches[kernel];
  if (total_ms) *total_ms = problem->k_ms[kernel];
  if (reset) {
    for (int k = 0; k < kKernelIds; ++k) { problem->k_launches[k] = 0; problem->k_ms[k] = 0.0; }
  }
  return KSC_OK;
}

// ------------------------------------------------------------------ solve

static cudaGraphExec_t* graph_slot(ksc_problem* pr, bool prof, bool eig) {
  return eig ? (prof ? &pr->graph_eig_prof : &pr->graph_eig) : (prof ? &pr->graph_prof : &pr->graph);
}

static ksc_status build_graph(ksc_problem* pr, cudaStream_t s, bool prof, bool eig) {
  cudaGraphExec_t* slot = graph_slot(pr, prof, eig);
  if (*slot) return KSC_OK;
  if (prof && pr->events.empty()) {
    pr->events.resize(kEventsPerStep * kStepsPerGraph);
    for (auto& e : pr->events) KSC_CUDA(cudaEventCreate(&e));
  }
  // capture on a private stream (legacy default stream cannot be captured)
  cudaStream_t cs;
  KSC_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int k = 0; k < kStepsPerGraph; ++k) launch_step(pr->dev, cs, prof ? &pr->events[kEventsPerStep * k] : nullptr, eig);
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(slot, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  (void)s;
  if (e != cudaSuccess) return fail(KSC_ERR_CUDA, std::string("graph capture: ") + cudaGetErrorString(e));
  return KSC_OK;
}

template <typename T>
static void fill_slots(std::vector<unsigned char>& buf, const std::vector<double>& b) {
  buf.resize(b.size() * sizeof(T));
  T* t = (T*)buf.data();
  for (size_t j = 0; j < b.size(); ++j) t[j] = (T)b[j];
}

ksc_status ksc::check_node(const ksc_problem* pr, const ksc_node* node, NodeSetup* ns) {
  if (!node) return fail(KSC_ERR_INVALID_ARG, "node is NULL");
  if (!(node->lambda2 > 0) || !std::isfinite(node->lambda2)) return fail(KSC_ERR_INVALID_ARG, "lambda2 must be > 0");
  if (!(node->M > 0) || !std::isfinite(node->M)) return fail(KSC_ERR_INVALID_ARG, "M must be > 0");
  if (node->k < 0) return fail(KSC_ERR_INVALID_ARG, "k must be >= 0");
  if (node->max_iter <= 0) return fail(KSC_ERR_INVALID_ARG, "max_iter must be > 0");
  if (!(node->rel_gap_tol >= 0) || !std::isfinite(node->rel_gap_tol)) return fail(KSC_ERR_INVALID_ARG, "rel_gap_tol must be >= 0");
  if (node->n_zero < 0 || node->n_one < 0) return fail(KSC_ERR_INVALID_ARG, "negative set size");
  if ((node->n_zero > 0 && !node->fixed_zero) || (node->n_one > 0 && !node->fixed_one))
    return fail(KSC_ERR_INVALID_ARG, "fixed-set pointer is NULL");
  if (node->flags & KSC_FLAG_EIG) {
    if (pr->loss != KSC_LOSS_LSQ) return fail(KSC_ERR_INVALID_ARG, "the eigen-perspective relaxation is for least squares");
    if (!pr->eig_ready) return fail(KSC_ERR_INVALID_ARG, "eigen shift not computed (ksc_problem_eig_lambda)");
  }
  ns->state.assign(pr->p, (int8_t)kFree);
  for (int i = 0; i < node->n_zero; ++i) {
    const int j = node->fixed_zero[i];
    if (j < 0 || j >= pr->p) return fail(KSC_ERR_INVALID_ARG, "fixed_zero index out of range");
    ns->state[j] = kZero;
  }
  for (int i = 0; i < node->n_one; ++i) {
    const int j = node->fixed_one[i];
    if (j < 0 || j >= pr->p) return fail(KSC_ERR_INVALID_ARG, "fixed_one index out of range");
    if (ns->state[j] == kZero) ns->infeasible = true;
    if (ns->state[j] != kOne) ns->n_one += 1;
    ns->state[j] = kOne;
  }
  ns->kp = node->k - ns->n_one;
  if (ns->kp < 0) ns->infeasible = true;
  int nfree = 0;
  for (auto v : ns->state) nfree += (v == kFree);
  const int q = std::min(ns->kp, nfree);
  if (!ns->infeasible && q >= kProxCap)
    return fail(KSC_ERR_UNIMPLEMENTED, "k' = k - |S1| must be < 4096 (prox candidate capacity)");
  if (node->warm_beta)
    for (int64_t j = 0; j < pr->p; ++j)
      if (!std::isfinite(node->warm_beta[j])) return fail(KSC_ERR_INVALID_ARG, "warm_beta has a non-finite entry");
  return KSC_OK;
}

static ksc_status replay(ksc_problem* pr, cudaStream_t s, NodeDev* h) {
  const bool prof = pr->profile;
  cudaGraphExec_t g = *graph_slot(pr, prof, h->eig > 0.0);
  const int before = h->iter;
  KSC_CUDA(cudaGraphLaunch(g, s));
  pr->launches += (int64_t)kLaunchesPerStep * kStepsPerGraph;
  KSC_CUDA(cudaMemcpyAsync(h, pr->dev.nd, sizeof(NodeDev), cudaMemcpyDeviceToHost, s));
  KSC_CUDA(cudaStreamSynchronize(s));
  if (prof) {
    const int steps = std::min(kStepsPerGraph, h->iter - before);
    // events of a step: before the gradient, before the prox's select and apply
    // kernels, before the forward pass, after it
    struct Span { int id, from, to; };
    static constexpr Span spans[] = {{KSC_KERNEL_GRADIENT, 0, 1}, {KSC_KERNEL_PROX, 1, 3},
                                     {KSC_KERNEL_PROX_SELECT, 1, 2}, {KSC_KERNEL_PROX_APPLY, 2, 3},
                                     {KSC_KERNEL_FORWARD, 3, 4}};
    for (int k = 0; k < steps; ++k) {
      for (const Span& sp : spans) {
        float ms = 0.f;
        KSC_CUDA(cudaEventElapsedTime(&ms, pr->events[kEventsPerStep * k + sp.from],
                                      pr->events[kEventsPerStep * k + sp.to]));
        pr->k_ms[sp.id] += ms;
        pr->k_launches[sp.id] += 1;
      }
    }
  }
  return KSC_OK;
}

extern "C" ksc_status ksc_solve_node(ksc_problem* pr, const ksc_node* node, ksc_result* res,
                                     void* cuda_stream) {
  if (!pr) return fail(KSC_ERR_INVALID_ARG, "problem is NULL");
  if (!res) return fail(KSC_ERR_INVALID_ARG, "result is NULL");
  if (node && (node->flags & KSC_FLAG_EIG) && pr->loss == KSC_LOSS_LSQ && !pr->eig_ready) {
    // the certified shift, computed on first use
    double lam = 0.0;
    ksc_status se = ksc_problem_eig_lambda(pr, cuda_stream, &lam);
    if (se != KSC_OK) return se;
  }
  NodeSetup ns;
  ksc_status st = check_node(pr, node, &ns);
  if (st != KSC_OK) return st;
  res->iters = 0;
  res->restarts = 0;
  res->pruned = 0;
  if (ns.infeasible) {
    res->primal = INFINITY;
    res->dual_bound = INFINITY;
    res->rel_gap = 0.0;
    res->pruned = 1;
    res->status = KSC_ERR_INFEASIBLE_NODE;
    return fail(KSC_ERR_INFEASIBLE_NODE, "infeasible node: |S1| > k or S0 and S1 intersect");
  }
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int cur_dev = 0;
  cudaGetDevice(&cur_dev);
  if (cur_dev != pr->device) KSC_CUDA(cudaSetDevice(pr->device));
  Dev& d = pr->dev;
  const int64_t p = pr->p;
  // warm start projected on the node: S0 -> 0, clip to the box (reading of Algorithm
  // 3's start); Poisson / Gamma: scaled into the l1 ball of radius k M as well
  std::vector<double> w0(p, 0.0);
  if (node->warm_beta) {
    for (int64_t j = 0; j < p; ++j) w0[j] = node->warm_beta[j];
    project_warm(pr, ns, node->M, node->k, w0.data());
  }
  const double Lnode = node_lipschitz(pr, node->M, node->k);
  std::vector<unsigned char> wb;
  fill_slots<double>(wb, w0);
  const size_t tb = tbytes(pr->xdt);
  KSC_CUDA(cudaMemcpyAsync(d.state, ns.state.data(), p, cudaMemcpyHostToDevice, s));
  // S1 as an index list: the in-loop dual term visits |S1| coordinates, not all p
  std::vector<int> ones;
  for (int64_t j = 0; j < p; ++j)
    if (ns.state[j] == kOne) ones.push_back((int)j);
  if (!ones.empty())
    KSC_CUDA(cudaMemcpyAsync(d.one_idx, ones.data(), ones.size() * 4, cudaMemcpyHostToDevice, s));
  KSC_CUDA(cudaMemcpyAsync(d.beta, wb.data(), p * tb, cudaMemcpyHostToDevice, s));
  KSC_CUDA(cudaMemcpyAsync((char*)d.beta + p * tb, wb.data(), p * tb, cudaMemcpyHostToDevice, s));
  NodeDev h;
  std::memset(&h, 0, sizeof h);
  // eigen-perspective (App. D.2): lambda2 + eig on the perspective term, the smooth
  // part's constant 2 (lambda_max - eig) <= L - 2 eig
  const double eig = (node->flags & KSC_FLAG_EIG) ? pr->eig_lambda : 0.0;
  const double Ln = Lnode - 2.0 * eig;
  h.eig = eig;
  h.lambda2 = node->lambda2 + eig;
  h.M = node->M;
  h.L = Ln;
  h.invL = 1.0 / Ln;
  h.rho = Ln / (2.0 * h.lambda2);
  h.tol_loop = node->rel_gap_tol;
  h.incumbent = node->incumbent;
  h.kp = ns.kp;
  h.n_one = (int)ones.size();
  h.max_iter = node->max_iter;
  h.restart_on = (node->flags & KSC_FLAG_RESTART_OFF) ? 0 : 1;
  h.momentum_on = (node->flags & KSC_FLAG_MOMENTUM_OFF) ? 0 : 1;
  h.loss = pr->loss;
  h.iter = 1;
  h.qhint = 0;
  h.nnz = (int)p + 1;   // the warm start's support is unknown: dense forward pass
  KSC_CUDA(cudaMemcpyAsync(d.nd, &h, sizeof h, cudaMemcpyHostToDevice, s));
  launch_init(d, s);
  pr->launches += kLaunchesPerInit;
  KSC_CUDA(cudaGetLastError());
  if ((st = build_graph(pr, s, pr->profile, h.eig > 0.0)) != KSC_OK) return st;
  KSC_CUDA(cudaMemcpyAsync(&h, d.nd, sizeof h, cudaMemcpyDeviceToHost, s));
  KSC_CUDA(cudaStreamSynchronize(s));

  const double tol = node->rel_gap_tol;
  const double inc = node->incumbent;
  int pruned = 0;
  ksc_status out_status = KSC_OK;
  for (;;) {
    if ((st = replay(pr, s, &h)) != KSC_OK) return st;
    if (h.done == kRunning) continue;
    // FP64 certificate at the current iterate
    launch_certificate(d, s, res->z != nullptr);
    pr->launches += kLaunchesPerCert;
    KSC_CUDA(cudaGetLastError());
    KSC_CUDA(cudaMemcpyAsync(&h, d.nd, sizeof h, cudaMemcpyDeviceToHost, s));
    KSC_CUDA(cudaStreamSynchronize(s));
    const bool gap_ok = h.cert_gap <= tol;
    const bool prune_ok = std::isfinite(inc) && h.cert_dual > inc;
    if (prune_ok) { pruned = 1; break; }
    if (gap_ok) break;
    if (h.done == kDonePrimal) break;                 // Sec. 4.3 rule (1): branch
    if (h.done == kDoneMaxIter) { out_status = KSC_NOT_CONVERGED; break; }
    // the in-loop test fired on values the FP64 certificate does not confirm:
    // tighten the in-loop tolerance (or the in-loop prune threshold) and go on
    NodeDev upd = h;
    if (h.done == kDoneGap) upd.tol_loop = std::max(h.gap * 0.25, 1e-16);
    if (h.done == kDonePruned) upd.incumbent = inc + 2.0 * std::fabs(h.best_dual - h.cert_dual) + 1e-12 * std::fabs(inc);
    upd.done = kRunning;
    upd.best_dual = h.cert_dual > -INFINITY ? std::max(h.cert_dual, -1e300) : -INFINITY;
    KSC_CUDA(cudaMemcpyAsync(d.nd, &upd, sizeof upd, cudaMemcpyHostToDevice, s));
    h = upd;
  }
  for (int i = 6; i < 12; ++i) pr->last_stats[i] = 0;
  pr->last_stats[0] = h.iter - 1;
  pr->last_stats[1] = h.sparse_steps;
  pr->last_stats[2] = h.fallback;
  pr->last_stats[3] = h.fast_steps;
  pr->last_stats[4] = h.dfast_steps;
  pr->last_stats[5] = pr->power_iters;
  res->primal = h.cert_primal;
  res->dual_bound = h.cert_dual;
  res->rel_gap = h.cert_gap;
  res->iters = h.iter - 1;
  res->restarts = h.restarts;
  res->pruned = pruned;
  res->status = out_status;
  if (res->beta) KSC_CUDA(cudaMemcpyAsync(res->beta, d.b64, p * 8, cudaMemcpyDeviceToHost, s));
  if (res->z) KSC_CUDA(cudaMemcpyAsync(res->z, d.z64, p * 8, cudaMemcpyDeviceToHost, s));
  KSC_CUDA(cudaStreamSynchronize(s));
  if (out_status != KSC_OK) return fail(out_status, "max_iter reached before the gap target");
  return KSC_OK;
}

// ------------------------------------------------------------------ primitives

struct DevBuf {
  void* p = nullptr;
  ~DevBuf() { if (p) cudaFree(p); }
};

static ksc_status prim_check(int64_t p, int32_t k, double M) {
  if (p < 1 || p > (1ll << 30)) return fail(KSC_ERR_INVALID_ARG, "p must be in [1, 2^30]");
  if (k < 0) return fail(KSC_ERR_INVALID_ARG, "k must be >= 0");
  if (!(M > 0) || !std::isfinite(M)) return fail(KSC_ERR_INVALID_ARG, "M must be > 0");
  if (std::min<int64_t>(k, p) >= kProxCap)
    return fail(KSC_ERR_UNIMPLEMENTED, "min(k, p) must be < 4096 (prox candidate capacity)");
  return ensure_prepared();
}

extern "C" ksc_status ksc_prox_g(const double* w, int64_t p, int32_t k, double M, double rho,
                                 double* beta_out, int32_t* top_out) {
  if (!w || !beta_out) return fail(KSC_ERR_INVALID_ARG, "w and beta_out must be non-NULL");
  if (!(rho > 0) || !std::isfinite(rho)) return fail(KSC_ERR_INVALID_ARG, "rho must be > 0");
  ksc_status st = prim_check(p, k, M);
  if (st != KSC_OK) return st;
  for (int64_t j = 0; j < p; ++j)
    if (!std::isfinite(w[j])) return fail(KSC_ERR_INVALID_ARG, "w has a non-finite entry");
  DevBuf bw, bb, bt, bs;
  const int q = (int)std::min<int64_t>(k, p);
  KSC_CUDA(cudaMalloc(&bw.p, p * 8));
  KSC_CUDA(cudaMalloc(&bb.p, p * 8));
  KSC_CUDA(cudaMalloc(&bs.p, p * 8));
  KSC_CUDA(cudaMalloc(&bt.p, (q > 0 ? q : 1) * sizeof(int)));
  KSC_CUDA(cudaMemcpy(bw.p, w, p * 8, cudaMemcpyHostToDevice));
  launch_prox_prim((const double*)bw.p, (int)p, k, M, rho, (double*)bb.p, top_out ? (int*)bt.p : nullptr,
                   (double*)bs.p, 0);
  KSC_CUDA(cudaGetLastError());
  KSC_CUDA(cudaMemcpy(beta_out, bb.p, p * 8, cudaMemcpyDeviceToHost));
  if (top_out && q > 0) KSC_CUDA(cudaMemcpy(top_out, bt.p, q * sizeof(int), cudaMemcpyDeviceToHost));
  return KSC_OK;
}

extern "C" ksc_status ksc_g_value(const double* beta, int64_t p, int32_t k, double M, double* g_out,
                                  double* z_out) {
  if (!beta || !g_out) return fail(KSC_ERR_INVALID_ARG, "beta and g_out must be non-NULL");
  ksc_status st = prim_check(p, k, M);
  if (st != KSC_OK) return st;
  for (int64_t j = 0; j < p; ++j)
    if (!std::isfinite(beta[j])) return fail(KSC_ERR_INVALID_ARG, "beta has a non-finite entry");
  DevBuf bb, bg, bz;
  KSC_CUDA(cudaMalloc(&bb.p, p * 8));
  KSC_CUDA(cudaMalloc(&bg.p, 8));
  KSC_CUDA(cudaMalloc(&bz.p, p * 8));
  KSC_CUDA(cudaMemcpy(bb.p, beta, p * 8, cudaMemcpyHostToDevice));
  launch_gvalue_prim((const double*)bb.p, (int)p, k, M, (double*)bg.p, z_out ? (double*)bz.p : nullptr, 0);
  KSC_CUDA(cudaGetLastError());
  KSC_CUDA(cudaMemcpy(g_out, bg.p, 8, cudaMemcpyDeviceToHost));
  if (z_out) KSC_CUDA(cudaMemcpy(z_out, bz.p, p * 8, cudaMemcpyDeviceToHost));
  return KSC_OK;
}

extern "C" ksc_status ksc_gstar(const double* a, int64_t p, int32_t k, double M, double* out) {
  if (!a || !out) return fail(KSC_ERR_INVALID_ARG, "a and out must be non-NULL");
  if (p < 1 || k < 0 || !(M > 0)) return fail(KSC_ERR_INVALID_ARG, "need p >= 1, k >= 0, M > 0");
  ksc_status st = ensure_prepared();
  if (st != KSC_OK) return st;
  for (int64_t j = 0; j < p; ++j)
    if (!std::isfinite(a[j])) return fail(KSC_ERR_INVALID_ARG, "a has a non-finite entry");
  DevBuf ba, bo;
  KSC_CUDA(cudaMalloc(&ba.p, p * 8));
  KSC_CUDA(cudaMalloc(&bo.p, 8));
  KSC_CUDA(cudaMemcpy(ba.p, a, p * 8, cudaMemcpyHostToDevice));
  launch_gstar_prim((const double*)ba.p, (int)p, k, M, (double*)bo.p, 0);
  KSC_CUDA(cudaGetLastError());
  KSC_CUDA(cudaMemcpy(out, bo.p, 8, cudaMemcpyDeviceToHost));
  return KSC_OK;
}

extern "C" ksc_status ksc_problem_solve_stats(const ksc_problem* problem, int32_t* stats, int32_t n) {
  if (!problem) return fail(KSC_ERR_INVALID_ARG, "problem is NULL");
  if (n < 0 || (n > 0 && !stats)) return fail(KSC_ERR_INVALID_ARG, "bad stats buffer");
  for (int32_t i = 0; i < n; ++i) stats[i] = i < 12 ? problem->last_stats[i] : 0;
  return KSC_OK;
}

extern "C" ksc_status ksc_problem_launch_count(const ksc_problem* problem, int64_t* launches) {
  if (!problem || !launches) return fail(KSC_ERR_INVALID_ARG, "problem and launches must be non-NULL");
  *launches = problem->launches;
  return KSC_OK;
}

extern "C" const char* ksc_last_error(void) { return g_err.c_str(); }

extern "C" const char* ksc_version(void) { return "ksc 0.1 (sm_103a)"; }
