// ksc_noalloc.cu -- the prox of g and g itself on device buffers with no device
// allocation at all: ksc_prox_g_noalloc (one vector), ksc_prox_g_batch and
// ksc_g_value_batch (many vectors).
//
// Some callers cannot call cudaMalloc: runtimes that own every byte of device
// memory through their own pool and forbid allocations behind their back (a
// serving process that reserved the GPU's memory at start-up, a solver embedded
// in another framework's allocator), and latency-critical loops where an
// allocation's implicit device synchronisation is not acceptable.  This entry point serves them: the caller passes device inputs and
// outputs, and the only scratch the kernel needs (the prox's copy of w when p is
// too large for shared memory) lives in the fixed-size device array below, which
// every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>

#include "../../include/ksc.h"
#include "ksc_launch.h"

ksc_status ksc_internal_fail(ksc_status st, const char* msg);

namespace {

// largest p the allocation-free prox accepts: 2^19 coordinates, 4 MiB of FP64
constexpr int64_t kNoAllocMaxP = int64_t(1) << 19;
constexpr int kMaxDevices = 64;

// file-scope scratch shared by every call on a device (its address is taken on
// the host once per device with cudaGetSymbolAddress; the name itself is only a
// host-side stand-in for the device object)
static __device__ __align__(256) double g_prox_scratch[kNoAllocMaxP];

std::mutex g_mu;
void* g_scratch_ptr[kMaxDevices] = {};
bool g_ready[kMaxDevices] = {};

}  // namespace

// one-time set-up on the current device (the scratch's address and the kernels'
// shared-memory limits); returns the scratch or NULL with the error recorded
static void* prepare_device(ksc_status* st) {
  *st = KSC_OK;
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
    *st = ksc_internal_fail(KSC_ERR_CUDA, "no usable current CUDA device");
    return nullptr;
  }
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_ready[dev]) {
    // each call's own return code is checked, so an error left pending by the
    // caller's earlier work does not fail (or repeat) this set-up
    void* ptr = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&ptr, g_prox_scratch);
    if (e != cudaSuccess) {
      *st = ksc_internal_fail(KSC_ERR_CUDA, cudaGetErrorString(e));
      return nullptr;
    }
    e = ksc::prox_prepare();
    if (e != cudaSuccess) {
      *st = ksc_internal_fail(KSC_ERR_CUDA, cudaGetErrorString(e));
      return nullptr;
    }
    g_scratch_ptr[dev] = ptr;
    g_ready[dev] = true;
  }
  return g_scratch_ptr[dev];
}

extern "C" ksc_status ksc_prox_g_batch(const double* w, int64_t ldw, double* beta_out, int64_t ldb, int64_t p,
                                       int32_t count, int32_t k, double M, double rho, void* cuda_stream) {
  if (count < 0) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "count must be >= 0");
  if (count > 0 && (!w || !beta_out)) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "w and beta_out must be non-NULL");
  if (p < 1 || p > INT32_MAX) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "p must be in [1, 2^31)");
  if (ldw < p || ldb < p) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "ldw and ldb must be >= p");
  // the byte spans below stay within int64: (count - 1) * ld + p <= count * ld <= INT64_MAX / 8
  const int64_t ld_max = INT64_MAX / 8 / (count > 0 ? count : 1);
  if (ldw > ld_max || ldb > ld_max) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "ldw or ldb too large");
  if (k < 0) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "k must be >= 0");
  if (!(M > 0) || !std::isfinite(M)) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "M must be > 0");
  if (!(rho > 0) || !std::isfinite(rho)) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "rho must be > 0");
  if ((k < p ? (int64_t)k : p) >= ksc::prox_rows_cap())
    return ksc_internal_fail(KSC_ERR_UNIMPLEMENTED, "min(k, p) must be < 2048 (per-vector candidate capacity)");
  if (count > 0) {
    const char* a = (const char*)w;
    const char* b = (const char*)beta_out;
    const int64_t wb = ((int64_t)(count - 1) * ldw + p) * 8, bb = ((int64_t)(count - 1) * ldb + p) * 8;
    if (a < b + bb && b < a + wb) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "w and beta_out overlap");
  }
  if (count == 0) return KSC_OK;
  ksc_status st;
  if (!prepare_device(&st)) return st;
  ksc::launch_prox_rows(w, ldw, beta_out, ldb, (int)p, count, k, M, rho, (cudaStream_t)cuda_stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ksc_internal_fail(KSC_ERR_CUDA, cudaGetErrorString(e));
  return KSC_OK;
}

extern "C" ksc_status ksc_g_value_batch(const double* beta, int64_t ldb, int64_t p, int32_t count, int32_t k,
                                        double M, double* g_out, void* cuda_stream) {
  if (count < 0) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "count must be >= 0");
  if (count > 0 && (!beta || !g_out)) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "beta and g_out must be non-NULL");
  if (p < 1 || p > INT32_MAX) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "p must be in [1, 2^31)");
  if (ldb < p) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "ldb must be >= p");
  const int64_t ld_max = INT64_MAX / 8 / (count > 0 ? count : 1);
  if (ldb > ld_max) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "ldb too large");
  if (k < 0) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "k must be >= 0");
  if (!(M > 0) || !std::isfinite(M)) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "M must be > 0");
  if ((k < p ? (int64_t)k : p) >= ksc::prox_rows_cap())
    return ksc_internal_fail(KSC_ERR_UNIMPLEMENTED, "min(k, p) must be < 2048 (per-vector candidate capacity)");
  if (count == 0) return KSC_OK;
  ksc_status st;
  if (!prepare_device(&st)) return st;
  ksc::launch_gvalue_rows(beta, ldb, (int)p, count, k, M, g_out, (cudaStream_t)cuda_stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ksc_internal_fail(KSC_ERR_CUDA, cudaGetErrorString(e));
  return KSC_OK;
}

extern "C" ksc_status ksc_prox_g_noalloc(const double* w, int64_t p, int32_t k, double M,
                                         double rho, double* beta_out, int32_t* top_out,
                                         void* cuda_stream) {
  if (!w || !beta_out) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "w and beta_out must be non-NULL");
  if (p < 1) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "p must be >= 1");
  if (p > kNoAllocMaxP)
    return ksc_internal_fail(KSC_ERR_INVALID_ARG,
                             "p exceeds the allocation-free maximum of 524288 coordinates");
  if (k < 0) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "k must be >= 0");
  if (!(M > 0) || !std::isfinite(M)) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "M must be > 0");
  if (!(rho > 0) || !std::isfinite(rho)) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "rho must be > 0");
  if ((k < p ? (int64_t)k : p) >= ksc::kProxCap)
    return ksc_internal_fail(KSC_ERR_UNIMPLEMENTED,
                             "min(k, p) must be < 4096 (prox candidate capacity)");
  ksc_status st;
  void* scratch = prepare_device(&st);
  if (!scratch) return st;
  // every entry of the scratch that the kernel reads it has written first in the
  // same call, so nothing needs clearing between calls
  ksc::launch_prox_prim(w, (int)p, k, M, rho, beta_out, top_out, (double*)scratch,
                        (cudaStream_t)cuda_stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ksc_internal_fail(KSC_ERR_CUDA, cudaGetErrorString(e));
  return KSC_OK;
}
