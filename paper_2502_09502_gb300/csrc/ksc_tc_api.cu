// ksc_tc_api.cu -- ksc_tc_gemm, ksc_tc_gemm_sk, ksc_tc_gemm_e4m3 and ksc_tc_exact: the batched
// solver's tensor-core products on caller-owned device buffers, exported so that
// tests can check them on their own.
#include <cuda_runtime.h>

#include <string>

#include "../../include/ksc.h"
#include "ksc_launch.h"
#include "ksc_tc.h"
#include "ksc_tcx.h"

ksc_status ksc_internal_fail(ksc_status st, const char* msg);

using namespace ksc;

extern "C" ksc_status ksc_tc_gemm(const void* A, int32_t pieces, int32_t m, int32_t m_pad, int32_t k,
                                  int64_t lda, const void* B, int32_t n, int64_t ldb, float* D, int64_t ldd,
                                  int32_t tile_n, void* cuda_stream) {
  if (!A || !B || !D) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "NULL operand");
  if (ldd < n || (ldd % 4) != 0 || ((uintptr_t)D % 16) != 0)
    return ksc_internal_fail(KSC_ERR_INVALID_ARG, "ldd must be >= n, a multiple of 4, D 16-byte aligned");
  TcPlan plan;
  const char* why = "";
  if (!tc_plan(&plan, A, pieces, m, m_pad, k, lda, B, n, ldb, tile_n, &why))
    return ksc_internal_fail(KSC_ERR_INVALID_ARG, why);
  cudaStream_t s = (cudaStream_t)cuda_stream;
  tc_clear_error(s);
  TcEpi e{};
  e.out = D;
  e.ldo = ldd;
  tc_launch(plan, e, kTcStore, s);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (err != cudaSuccess)
    return ksc_internal_fail(KSC_ERR_CUDA, (std::string("tensor-core product: ") + cudaGetErrorString(err)).c_str());
  int word = 0;
  cudaMemcpy(&word, tc_error_word(), sizeof word, cudaMemcpyDeviceToHost);
  if (word != 0) return ksc_internal_fail(KSC_ERR_TIMEOUT, "tensor-core product: a device wait gave up");
  return KSC_OK;
}

extern "C" ksc_status ksc_tc_gemm_sk(const void* A, int32_t pieces, int32_t m, int32_t m_pad, int32_t k,
                                     int64_t lda, const void* B, int32_t n, int64_t ldb, float* D, int64_t ldd,
                                     int32_t tile_n, int32_t grid, void* cuda_stream) {
  if (!A || !B || !D) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "NULL operand");
  if (ldd < n || (ldd % 4) != 0 || ((uintptr_t)D % 16) != 0)
    return ksc_internal_fail(KSC_ERR_INVALID_ARG, "ldd must be >= n, a multiple of 4, D 16-byte aligned");
  if (grid < 1 || grid > 4096) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "grid must be in [1, 4096]");
  TcPlan plan;
  const char* why = "";
  if (!tc_plan(&plan, A, pieces, m, m_pad, k, lda, B, n, ldb, tile_n, &why) ||
      !tc_plan_stream_k(&plan, grid, &why))
    return ksc_internal_fail(KSC_ERR_INVALID_ARG, why);
  float* ws = nullptr;
  if (cudaMalloc(&ws, tc_skws_floats(grid, tile_n) * sizeof(float)) != cudaSuccess)
    return ksc_internal_fail(KSC_ERR_OOM, "stream-K partials");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  tc_clear_error(s);
  TcEpi e{};
  e.out = D;
  e.ldo = ldd;
  e.skws = ws;
  tc_launch(plan, e, kTcStore, s);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  cudaFree(ws);
  if (err != cudaSuccess)
    return ksc_internal_fail(KSC_ERR_CUDA, (std::string("stream-K product: ") + cudaGetErrorString(err)).c_str());
  int word = 0;
  cudaMemcpy(&word, tc_error_word(), sizeof word, cudaMemcpyDeviceToHost);
  if (word != 0) return ksc_internal_fail(KSC_ERR_TIMEOUT, "stream-K product: a device wait gave up");
  return KSC_OK;
}

extern "C" ksc_status ksc_tc_gemm_e4m3(const void* A, int32_t m, int32_t m_pad, int32_t k, int64_t lda,
                                       const void* B, int32_t n, int64_t ldb, const float* row_scale,
                                       const float* col_scale, float* D, int64_t ldd, int32_t tile_n, int32_t grid,
                                       void* cuda_stream) {
  if (!A || !B || !D || !row_scale) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "NULL operand");
  if (ldd < n || (ldd % 4) != 0 || ((uintptr_t)D % 16) != 0)
    return ksc_internal_fail(KSC_ERR_INVALID_ARG, "ldd must be >= n, a multiple of 4, D 16-byte aligned");
  if (grid < 0 || grid > 4096) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "grid must be in [0, 4096]");
  TcPlan plan;
  const char* why = "";
  if (!tc_plan(&plan, A, kTcE4m3Pieces, m, m_pad, k, lda, B, n, ldb, tile_n, &why, 1) ||
      (grid > 0 && !tc_plan_stream_k(&plan, grid, &why)))
    return ksc_internal_fail(KSC_ERR_INVALID_ARG, why);
  float* ws = nullptr;
  if (grid > 0 && cudaMalloc(&ws, tc_skws_floats(grid, tile_n) * sizeof(float)) != cudaSuccess)
    return ksc_internal_fail(KSC_ERR_OOM, "stream-K partials");
  cudaStream_t s = (cudaStream_t)cuda_stream;
  tc_clear_error(s);
  TcEpi e{};
  e.out = D;
  e.ldo = ldd;
  e.skws = ws;
  e.rscale = row_scale;
  e.cscale = col_scale;
  tc_launch(plan, e, kTcStore, s);
  cudaError_t err = cudaGetLastError();
  if (err == cudaSuccess) err = cudaStreamSynchronize(s);
  if (ws) cudaFree(ws);
  if (err != cudaSuccess)
    return ksc_internal_fail(KSC_ERR_CUDA, (std::string("E4M3 product: ") + cudaGetErrorString(err)).c_str());
  int word = 0;
  cudaMemcpy(&word, tc_error_word(), sizeof word, cudaMemcpyDeviceToHost);
  if (word != 0) return ksc_internal_fail(KSC_ERR_TIMEOUT, "E4M3 product: a device wait gave up");
  return KSC_OK;
}

extern "C" ksc_status ksc_tc_exact(const void* A, int32_t c, int32_t k, int64_t lda, const double* V, int32_t r,
                                   int64_t ldv, double* D, int64_t ldd, double* err_factor, void* cuda_stream) {
  if (!A || !V || !D) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "NULL operand");
  if (c < 1 || k < 1 || r < 1 || r > kTcxMaxR) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "sizes out of range");
  if (lda < k || ldv < k || ldd < c) return ksc_internal_fail(KSC_ERR_INVALID_ARG, "row strides too small");
  cudaError_t e = prox_prepare();
  if (e != cudaSuccess) return ksc_internal_fail(KSC_ERR_CUDA, cudaGetErrorString(e));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  TcxSlices x;
  TcxVecs v;
  const char* why = "";
  if (!tcx_slices_build(&x, A, c, k, lda, s, &why)) return ksc_internal_fail(KSC_ERR_OOM, why);
  if (!tcx_vecs_alloc(&v, r, k, &why)) {
    tcx_slices_free(&x);
    return ksc_internal_fail(KSC_ERR_OOM, why);
  }
  tcx_clear_error(s);
  tcx_product(x, v, V, ldv, nullptr, r, D, ldd, s);
  e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  int word = 0;
  if (e == cudaSuccess) e = cudaMemcpy(&word, tcx_error_word(), sizeof word, cudaMemcpyDeviceToHost);
  if (err_factor) *err_factor = tcx_error_factor(x);
  tcx_slices_free(&x);
  tcx_vecs_free(&v);
  if (e != cudaSuccess)
    return ksc_internal_fail(KSC_ERR_CUDA, (std::string("exact product: ") + cudaGetErrorString(e)).c_str());
  if (word != 0) return ksc_internal_fail(KSC_ERR_TIMEOUT, "exact product: a device wait gave up");
  return KSC_OK;
}
