// k_prox.cu -- per-node kernels built on the block prox (ksc_prox.cuh); the prox
// of a FISTA step itself is spread over the GPU in k_prox_grid.cu.
//   k_gvalue_init    g(beta^1) for the initial objective (Algorithm 3)
//   k_cert_final     FP64 G*(a) with its rounding margin, FP64 g(b^), the
//                    certified bound and gap (Sec. 3.4)
//   primitives       prox_{rho^-1 g}, g, g* on one vector (FP64)
#include <mutex>

#include "ksc_common.cuh"
#include "ksc_launch.h"
#include "ksc_prox.cuh"
#include "ksc_state.cuh"

namespace ksc {

// g* primitive shared memory: hist + scratch only
constexpr int kDualCap = 16;

cudaError_t prox_grid_prepare(int optin);   // k_prox_grid.cu
cudaError_t batch_prepare(int optin);       // k_batch.cu
cudaError_t tcx_prepare();                  // k_tcexact.cu

template <typename T>
__global__ void __launch_bounds__(kProxBlock, 1) k_gvalue_init(Dev d) {
  extern __shared__ __align__(16) unsigned char smem[];
  NodeDev* nd = d.nd;
  SegSmem<double> sm = carve_seg_smem<double>(smem, kProxCap, 0);
  const T* b1 = (const T*)d.beta + (size_t)1 * d.p;
  GOut o = gvalue_segment<double, kProxBlock>(d.p, [&](int i) { return to_d(b1[i]); }, d.state,
                                              nd->kp, nd->M, sm, nullptr,
                                              sizeof(T) == 8 ? 1e-12 : 1e-6);
  double bsq = 0.0;
  if (nd->eig > 0.0) {   // eigen-perspective: ||b^1||^2 for the initial objective
    for (int j = threadIdx.x; j < d.p; j += kProxBlock) {
      const double v = to_d(b1[j]);
      bsq += v * v;
    }
    bsq = block_sum<double, kProxBlock>(bsq, sm.red);
  }
  if (threadIdx.x == 0) {
    nd->g_next = o.g;
    nd->bsq_next = bsq;
  }
}

// The certificate's iterate: the final beta promoted to FP64, clipped to the box,
// fixed-to-zero coordinates zeroed, and the free part scaled onto the l1 budget
// k'M when rounding left it a hair outside dom g -- so the primal value reported
// is the objective at a point of the domain.
template <typename T>
__global__ void __launch_bounds__(kProxBlock, 1) k_cert_prep(Dev d) {
  __shared__ double red[64];
  NodeDev* nd = d.nd;
  const int p = d.p;
  const double M = nd->M;
  const T* b = (const T*)d.beta + (size_t)(nd->iter % 3) * p;
  double l1 = 0.0;
  for (int j = threadIdx.x; j < p; j += kProxBlock) {
    const int8_t st = d.state ? d.state[j] : (int8_t)kFree;
    double v = fmin(fmax(to_d(b[j]), -M), M);
    if (st == kZero) v = 0.0;
    d.b64[j] = v;
    if (st == kFree) l1 += fabs(v);
  }
  l1 = block_sum<double, kProxBlock>(l1, red);
  const double budget = (double)(nd->kp > 0 ? nd->kp : 0) * M;
  if (l1 > budget) {
    const double sc = budget > 0.0 ? (budget / l1) * (1.0 - 8.0 * 1.1102230246251565e-16) : 0.0;
    for (int j = threadIdx.x; j < p; j += kProxBlock) {
      const int8_t st = d.state ? d.state[j] : (int8_t)kFree;
      if (st == kFree) d.b64[j] *= sc;
    }
  }
}

template <typename T>
__global__ void __launch_bounds__(kProxBlock, 1) k_cert_final(Dev d, int want_z) {
  extern __shared__ __align__(16) unsigned char smem[];
  NodeDev* nd = d.nd;
  SegSmem<double> sm = carve_seg_smem<double>(smem, kProxCap, 0);
  const int p = d.p;
  const double ur = 1.1102230246251565e-16;
  const double l2 = nd->lambda2, M = nd->M;
  const double scale = 1.0 / (2.0 * l2);
  // eigen-perspective (App. D.2): G* at 2 (X^T y - Q b^) = X^T zeta + 2 eig b^
  const double eig = nd->eig;
  // G*(a) / (2 lambda2) over the node: TopSum_k'(H_M(|a_F|/2l2)) + sum_S1 H_M(a_j/2l2)
  const double gs = gstar_segment<double, kProxBlock>(
      p, [&](int i) { return eig > 0.0 ? d.a64[i] + 2.0 * eig * d.b64[i] : d.a64[i]; }, d.state, nd->kp, M,
      scale, sm);
  // error bound of a = X^T zeta (FP64, any summation order):
  //   |a^_j - a_j| <= gamma_{n+1} sum_i |x_ij zeta_i| <= gamma_{n+1} ||x_j|| ||zeta||
  double cmax = 0.0, amax = 0.0, bsq = 0.0, xf2 = 0.0, y2 = 0.0;
  int n1 = 0;
  for (int j = threadIdx.x; j < p; j += kProxBlock) {
    const int8_t st = d.state ? d.state[j] : (int8_t)kFree;
    if (st != kZero) cmax = fmax(cmax, d.colnorm[j]);
    if (st == kOne) n1 += 1;
    if (eig > 0.0) {
      if (st != kZero) amax = fmax(amax, fabs(d.a64[j]) + 2.0 * eig * fabs(d.b64[j]));
      bsq += d.b64[j] * d.b64[j];
      xf2 += d.colnorm[j] * d.colnorm[j];
    }
  }
  if (eig > 0.0)
    for (int i = threadIdx.x; i < d.n; i += kProxBlock) y2 += d.y[i] * d.y[i];
  cmax = block_max<double, kProxBlock>(cmax, sm.red, 0.0);
  n1 = (int)block_sum<double, kProxBlock>((double)n1, sm.red);
  if (eig > 0.0) {
    amax = block_max<double, kProxBlock>(amax, sm.red, 0.0);
    bsq = block_sum<double, kProxBlock>(bsq, sm.red);
    xf2 = block_sum<double, kProxBlock>(xf2, sm.red);
    y2 = block_sum<double, kProxBlock>(y2, sm.red);
  }
  const double nn = (double)d.n + 2.0;
  const double gam = nn * ur / (1.0 - nn * ur);
  const double znorm = sqrt(nd->cert_zeta_sq) * (1.0 + (nn + 2.0) * ur);
  double eps_a = 1.01 * gam * cmax * znorm;
  double nce = nd->cert_negconj, margin_e = 0.0;
  if (eig > 0.0) {
    // The bound at b^ is ||y||^2 - ||X b^||^2 + eig ||b^||^2 - G*(2 X^T (y - X b^) + 2 eig b^).
    // cert_negconj is ||y||^2 - ||u~||^2 (up to its margin) for u~ = y - zeta/2, and
    // X^T zeta = 2 X^T (y - u~); the forward product u = X b^ (FP64, or error-free
    // products with compensated sums) is within gamma_{p+1} ||x_i|| ||b^|| per row, so
    // ||u~ - X b^|| <= delta = gamma_{p+1} ||X||_F ||b^|| + u ||zeta|| (the rounding of u - y):
    //   | ||u~||^2 - ||X b^||^2 | <= delta (2 ||u~|| + delta),
    //   per coordinate of the G* argument: eps_a + 2 ||x_j|| delta + its own rounding
    const double pp = (double)p + 2.0;
    const double gp = pp * ur / (1.0 - pp * ur);
    const double bnorm = sqrt(bsq) * (1.0 + ((double)p + 4.0) * ur);
    const double xfro = sqrt(xf2 * (1.0 + ((double)p + 4.0) * ur)) * (1.0 + 4.0 * ur);
    const double ynorm = sqrt(y2 * (1.0 + ((double)d.n + 4.0) * ur)) * (1.0 + 4.0 * ur);
    const double delta = (gp * xfro * bnorm + ur * znorm) * 1.01;
    const double unorm = ynorm + 0.5 * znorm;
    margin_e = delta * (2.0 * unorm + delta) + ((double)p + 4.0) * ur * eig * bsq * 1.01;
    eps_a += 2.0 * cmax * delta + 2.0 * ur * (amax + 2.0 * eig * M) * 1.01;
    nce += eig * bsq;
  }
  const int kp = nd->kp;
  const int nsel = (kp < p ? kp : p) + n1;
  // H_M is M-Lipschitz and TopSum is 1-Lipschitz per selected entry; the factors
  // 1/(2 lambda2) and 2 lambda2 cancel.  Plus the rounding of the H_M values
  // (division, square, product) and of their sum.
  const double margin_g = (double)nsel * M * eps_a * (1.0 + 4.0 * ur) +
                          2.0 * l2 * gs * ((double)nsel + 8.0) * 4.0 * ur;
  // g(b^) in FP64 (Algorithm 2) and the relaxed z, at the prepared iterate b64
  GOut go = gvalue_segment<double, kProxBlock>(p, [&](int i) { return d.b64[i]; }, d.state, kp, M,
                                               sm, want_z ? d.z64 : nullptr);
  if (threadIdx.x == 0) {
    const double gst = 2.0 * l2 * gs;
    double dual = nce - nd->cert_margin_f - margin_e - gst - margin_g;
    dual -= 4.0 * ur * (fabs(nce) + gst);
    const double primal = nd->cert_f - eig * bsq + 2.0 * l2 * go.g;
    nd->cert_gstar = gst;
    nd->cert_margin_g = margin_g;
    nd->cert_g = go.g;
    nd->cert_sbar = go.sbar;
    nd->cert_dual = dual;
    nd->cert_primal = primal;
    nd->cert_gap = (primal - dual) / fmax(fabs(primal), 1e-300);
  }
}

// ---------------------------------------------------------------- primitives

__global__ void __launch_bounds__(kProxBlock, 1)
k_prox_prim(const double* w, int p, int k, double M, double rho, double* beta, int* top,
            double* wbuf, int wsm) {
  extern __shared__ __align__(16) unsigned char smem[];
  SegSmem<double> sm = carve_seg_smem<double>(smem, kProxCap, wsm);
  SegIO<double> io;
  io.m = p;
  io.state = nullptr;
  io.w = w;
  io.bc = io.bp = nullptr;
  io.grad = nullptr;
  io.gradf = nullptr;
  io.c = 0.0;
  io.invL = 0.0;
  io.rho = rho;
  io.M = M;
  io.kp = k;
  io.wbuf = wbuf;
  io.beta = beta;
  io.nnz_idx = nullptr;
  io.nnz_val = nullptr;
  io.nnz_cap = 0;
  io.top_out = top;
  io.qhint = 0;
  io.theta0 = -1.0;
  prox_segment<double, kProxBlock>(io, sm);
}

// many independent vectors, one CTA each: row r of w -> row r of beta.  w is read
// in place (every coordinate free, no copy); the first round of candidates is
// sized for a pooled tail of a few times k.
constexpr int kRowsBlock = 256, kRowsCap = 2048;
static_assert(kRowsCap + 1 >= 2 * kRowsBlock && kProxCap + 1 >= 2 * kProxBlock,
              "the prox's full-pass sums use the prefix buffer");

__global__ void __launch_bounds__(kRowsBlock)
k_prox_rows(const double* w, int64_t ldw, double* beta, int64_t ldb, int p, int k, double M, double rho) {
  extern __shared__ __align__(16) unsigned char smem[];
  SegSmem<double> sm = carve_seg_smem<double>(smem, kRowsCap, 0);
  const int64_t r = blockIdx.x;
  SegIO<double> io;
  io.m = p;
  io.state = nullptr;
  io.w = w + r * ldw;
  io.bc = io.bp = nullptr;
  io.grad = nullptr;
  io.gradf = nullptr;
  io.c = 0.0;
  io.invL = 0.0;
  io.rho = rho;
  io.M = M;
  io.kp = k;
  io.wbuf = nullptr;
  io.beta = beta + r * ldb;
  io.nnz_idx = nullptr;
  io.nnz_val = nullptr;
  io.nnz_cap = 0;
  io.top_out = nullptr;
  const int q = k < p ? k : p;
  io.qhint = 4 * q + 64 < kRowsCap ? 4 * q + 64 : kRowsCap;
  io.theta0 = -1.0;
  prox_segment<double, kRowsBlock>(io, sm);
}

// g(b) (Algorithm 2) of many rows, one CTA per row, every coordinate free
__global__ void __launch_bounds__(kRowsBlock)
k_gvalue_rows(const double* beta, int64_t ldb, int p, int k, double M, double* g) {
  extern __shared__ __align__(16) unsigned char smem[];
  SegSmem<double> sm = carve_seg_smem<double>(smem, kRowsCap, 0);
  const double* b = beta + (int64_t)blockIdx.x * ldb;
  const GOut o = gvalue_segment<double, kRowsBlock>(p, [&](int i) { return b[i]; }, nullptr, k, M, sm, nullptr);
  if (threadIdx.x == 0) g[blockIdx.x] = o.g;
}

__global__ void __launch_bounds__(kProxBlock, 1)
k_gvalue_prim(const double* beta, int p, int k, double M, double* g, double* z) {
  extern __shared__ __align__(16) unsigned char smem[];
  SegSmem<double> sm = carve_seg_smem<double>(smem, kProxCap, 0);
  GOut o = gvalue_segment<double, kProxBlock>(p, [&](int i) { return beta[i]; }, nullptr, k, M, sm, z);
  if (threadIdx.x == 0) *g = o.g;
}

__global__ void __launch_bounds__(kProxBlock, 1)
k_gstar_prim(const double* a, int p, int k, double M, double* out) {
  extern __shared__ __align__(16) unsigned char smem[];
  SegSmem<double> sm = carve_seg_smem<double>(smem, kDualCap, 0);
  double s = gstar_segment<double, kProxBlock>(p, [&](int i) { return a[i]; }, nullptr, k, M, 1.0, sm);
  if (threadIdx.x == 0) *out = s;
}

// ---------------------------------------------------------------- launchers

static size_t prox_bytes(int cap, int wsm, int tb) { return seg_smem_bytes(cap, wsm, tb); }

size_t prox_smem_bytes(const Dev& d) { return prox_bytes(kProxCap, d.prox_wsm, 8); }

// per-device set-up state: kernel attributes are per device, so each device is
// prepared once, under one lock shared by every entry point of the library
constexpr int kMaxPrepDevices = 64;
static std::mutex g_prep_mu;
static bool g_prep_done[kMaxPrepDevices] = {};
static size_t g_smem_max[kMaxPrepDevices] = {};

static int current_device() {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxPrepDevices) return -1;
  return dev;
}

cudaError_t prox_prepare() {
  const int dev = current_device();
  if (dev < 0) return cudaErrorInvalidDevice;
  std::lock_guard<std::mutex> lock(g_prep_mu);
  if (g_prep_done[dev]) return cudaSuccess;
  int optin = 0;
  cudaError_t e = cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  const cudaError_t steps[] = {
      prox_grid_prepare(optin),
      batch_prepare(optin),
      cudaFuncSetAttribute(k_gvalue_init<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
      cudaFuncSetAttribute(k_cert_final<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
      cudaFuncSetAttribute(k_prox_prim, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
      cudaFuncSetAttribute(k_prox_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
      cudaFuncSetAttribute(k_prox_rows, cudaFuncAttributePreferredSharedMemoryCarveout, 100),
      cudaFuncSetAttribute(k_gvalue_prim, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
      cudaFuncSetAttribute(k_gvalue_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
      cudaFuncSetAttribute(k_gstar_prim, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
      tcx_prepare(),
  };
  for (cudaError_t st : steps)
    if (st != cudaSuccess) return st;
  g_smem_max[dev] = (size_t)optin;
  g_prep_done[dev] = true;
  return cudaSuccess;
}

size_t prox_smem_limit() {
  const int dev = current_device();
  return dev < 0 ? 0 : g_smem_max[dev];
}

void launch_gvalue_init(const Dev& d, cudaStream_t s) {
  const size_t bytes = prox_bytes(kProxCap, 0, 8);
  k_gvalue_init<double><<<1, kProxBlock, bytes, s>>>(d);
}

void launch_cert_prep(const Dev& d, cudaStream_t s) {
  k_cert_prep<double><<<1, kProxBlock, 0, s>>>(d);
}

void launch_cert_final(const Dev& d, cudaStream_t s, int want_z) {
  const size_t bytes = prox_bytes(kProxCap, 0, 8);
  k_cert_final<double><<<1, kProxBlock, bytes, s>>>(d, want_z);
}

void launch_prox_prim(const double* w, int p, int k, double M, double rho, double* beta, int* top,
                      double* wbuf, cudaStream_t s) {
  // keep w in shared memory when it fits beside the candidate buffers
  const size_t base = prox_bytes(kProxCap, 0, 8);
  int wsm = 0;
  if (base + (size_t)p * 8 + 16 <= prox_smem_limit()) wsm = p;
  k_prox_prim<<<1, kProxBlock, prox_bytes(kProxCap, wsm, 8), s>>>(w, p, k, M, rho, beta, top, wbuf,
                                                                 wsm);
}

int prox_rows_cap() { return kRowsCap; }

void launch_prox_rows(const double* w, int64_t ldw, double* beta, int64_t ldb, int p, int count, int k,
                      double M, double rho, cudaStream_t s) {
  if (count <= 0) return;
  k_prox_rows<<<count, kRowsBlock, prox_bytes(kRowsCap, 0, 8), s>>>(w, ldw, beta, ldb, p, k, M, rho);
}

void launch_gvalue_rows(const double* beta, int64_t ldb, int p, int count, int k, double M, double* g,
                        cudaStream_t s) {
  if (count <= 0) return;
  k_gvalue_rows<<<count, kRowsBlock, prox_bytes(kRowsCap, 0, 8), s>>>(beta, ldb, p, k, M, g);
}

void launch_gvalue_prim(const double* beta, int p, int k, double M, double* g, double* z,
                        cudaStream_t s) {
  k_gvalue_prim<<<1, kProxBlock, prox_bytes(kProxCap, 0, 8), s>>>(beta, p, k, M, g, z);
}

void launch_gstar_prim(const double* a, int p, int k, double M, double* out, cudaStream_t s) {
  k_gstar_prim<<<1, kProxBlock, prox_bytes(kDualCap, 0, 8), s>>>(a, p, k, M, out);
}

}  // namespace ksc
