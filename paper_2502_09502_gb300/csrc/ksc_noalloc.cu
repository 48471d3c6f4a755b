// ksc_noalloc.cu -- ksc_prox_g_noalloc: the prox of g on device buffers, with no
// device allocation at all.
//
// Some callers cannot call cudaMalloc: code running while a CUDA graph is being
// captured (cudaMalloc is not capturable), runtimes that own every byte of device
// memory through their own pool and forbid outside allocations, and latency-
// critical loops where an allocation's implicit device synchronisation is not
// acceptable.  This entry point serves them: the caller passes device inputs and
// outputs, and the only scratch the kernel needs (the prox's copy of w when p is
// too large for shared memory) lives in the fixed-size device array below, which
// every GPU that loads the library holds until the process exits.
#include <cuda_runtime.h>

#include <cmath>
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
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return ksc_internal_fail(KSC_ERR_CUDA, "no usable current CUDA device");
  void* scratch = nullptr;
  {
    // one-time set-up on this device (the device is current): the scratch
    // address and the kernel's shared-memory limit
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_ready[dev]) {
      cudaError_t e = cudaGetSymbolAddress(&g_scratch_ptr[dev], g_prox_scratch);
      if (e != cudaSuccess) {
        g_scratch_ptr[dev] = nullptr;
        return ksc_internal_fail(KSC_ERR_CUDA, cudaGetErrorString(e));
      }
      ksc::prox_prepare();
      e = cudaGetLastError();
      if (e != cudaSuccess) return ksc_internal_fail(KSC_ERR_CUDA, cudaGetErrorString(e));
      g_ready[dev] = true;
    }
    scratch = g_scratch_ptr[dev];
  }
  // every entry of the scratch that the kernel reads it has written first in the
  // same call, so nothing needs clearing between calls
  ksc::launch_prox_prim(w, (int)p, k, M, rho, beta_out, top_out, (double*)scratch,
                        (cudaStream_t)cuda_stream);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return ksc_internal_fail(KSC_ERR_CUDA, cudaGetErrorString(e));
  return KSC_OK;
}
