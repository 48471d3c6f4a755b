// k_dfprod.cu -- the exact (double-float) product of X with many nodes' FP64
// vectors at once: the anchors of the batched solver (u_ref = X beta_ref,
// G_ref = X^T r_ref) and its FP64 certificates (X b^, X^T zeta; Sec. 3.4), with a
// rigorous a-priori error bound for the certificate's margin.
#include <cuda_bf16.h>

#include "ksc_batch.cuh"
#include "ksc_common.cuh"
#include "ksc_launch.h"

namespace ksc {

// ----------------------------------------------------------- batched exact product
// D[list[r]][c] = sum_k A[k][c] V[list[r]][k] for the rows r < R of a node list
// (A row-major K x C with leading dim lda): the exact products of many nodes in
// one launch.  Each CTA stages a 32 x 128 tile of A once for 16 node vectors
// (split into float hi + lo).  Within a block of K_b consecutive k the terms
// are summed in double-float (df_add); each block result hi + lo is added to an
// FP64 accumulator.  Error bound (u = 2^-24, U = 2^-53, S = sum_k |A[k][c] V[k]|):
//   |D - exact| <= [ (K_b^2/2 + 6 K_b + 5) u^2 + (blocks + splits + 2) U ] * 1.01 * S,
// K_b = kblock (a multiple of 32; the certificates use 64, the anchors, which need
// accuracy but no rigorous bound, 256 -- fewer FP64 block sums): per block the lo word collects the exact TwoSum and product errors
// with its own rounding (<= u^2 (K_b^2/2 + 6 K_b + 4) S_block), the split of V costs
// u^2 S, and the FP64 conversions and sums add the U terms.  With K split over
// gridDim.z CTAs the partial sums go to ws and k_dfsum adds them in split order.
// Every output element sums its terms in an order fixed by K alone.
constexpr int kDfCols = 128, kDfNodes = 16, kDfK = 32;

template <typename TX>
__global__ void __launch_bounds__(256, 3) k_dfprod(const TX* __restrict__ A, int64_t lda, int K, int C,
                                                const double* __restrict__ V, int64_t ldv,
                                                const int* __restrict__ list, int R, double* __restrict__ D,
                                                int64_t ldd, int kchunk, int kblock, double* __restrict__ ws) {
  __shared__ __align__(16) float As[kDfK][kDfCols + 4];
  __shared__ float Vh[kDfNodes][kDfK + 1];
  __shared__ float Vl[kDfNodes][kDfK + 1];
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;   // 4 columns x 2 nodes per thread
  const int c0 = blockIdx.x * kDfCols, r0 = blockIdx.y * kDfNodes;
  const int kb = blockIdx.z * kchunk, ke = min(K, kb + kchunk);
  float hi[2][4], lo[2][4];
  double acc[2][4];
#pragma unroll
  for (int q = 0; q < 2; ++q)
#pragma unroll
    for (int j = 0; j < 4; ++j) { hi[q][j] = 0.f; lo[q][j] = 0.f; acc[q][j] = 0.0; }
  // the next chunk's A and V are loaded into registers while the current one is
  // multiplied (16 A elements and 2 V entries per thread)
  constexpr int kAPer = kDfK * kDfCols / 256, kVPer = kDfNodes * kDfK / 256;
  float ra[kAPer];
  double rv[kVPer];
  auto load = [&](int k0) {
#pragma unroll
    for (int t = 0; t < kAPer; ++t) {
      const int e = (int)threadIdx.x + t * 256;
      const int k = k0 + e / kDfCols, c = c0 + e % kDfCols;
      ra[t] = (k < ke && c < C) ? xval<float>(A[(size_t)k * lda + c]) : 0.f;
    }
#pragma unroll
    for (int t = 0; t < kVPer; ++t) {
      const int e = (int)threadIdx.x + t * 256;
      const int r = r0 + e / kDfK, k = k0 + e % kDfK;
      rv[t] = (r < R && k < ke) ? V[(size_t)list[r] * ldv + k] : 0.0;
    }
  };
  if (kb < ke) load(kb);
  for (int k0 = kb; k0 < ke; k0 += kDfK) {
#pragma unroll
    for (int t = 0; t < kAPer; ++t) {
      const int e = (int)threadIdx.x + t * 256;
      As[e / kDfCols][e % kDfCols] = ra[t];
    }
    int nz = 0;
#pragma unroll
    for (int t = 0; t < kVPer; ++t) {
      const int e = (int)threadIdx.x + t * 256;
      const float h = (float)rv[t];
      Vh[e / kDfK][e % kDfK] = h;
      Vl[e / kDfK][e % kDfK] = (float)(rv[t] - (double)h);
      nz |= rv[t] != 0.0;
    }
    // a chunk where every node's vector is zero adds nothing (sparse iterates:
    // the nodes of one problem concentrate on the same columns)
    const bool any = __syncthreads_or(nz) != 0;
    if (k0 + kDfK < ke) load(k0 + kDfK);
    if (any) {
#pragma unroll 4
      for (int kk = 0; kk < kDfK; ++kk) {
        const float4 a = *reinterpret_cast<const float4*>(&As[kk][tx * 4]);
        const float av[4] = {a.x, a.y, a.z, a.w};
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          const float vh = Vh[ty * 2 + q][kk], vl = Vl[ty * 2 + q][kk];
#pragma unroll
          for (int j = 0; j < 4; ++j) df_add(hi[q][j], lo[q][j], av[j], vh, vl);
        }
      }
    }
    __syncthreads();
    if (((k0 - kb + kDfK) % kblock) == 0 || k0 + kDfK >= ke) {   // close the block
#pragma unroll
      for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          acc[q][j] += (double)hi[q][j] + (double)lo[q][j];
          hi[q][j] = 0.f;
          lo[q][j] = 0.f;
        }
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const int r = r0 + ty * 2 + q;
    if (r >= R) continue;
    double* drow = ws ? ws + ((size_t)blockIdx.z * R + r) * C : D + (size_t)list[r] * ldd;
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int c = c0 + tx * 4 + j;
      if (c < C) drow[c] = acc[q][j];
    }
  }
}

// D[list[r]][c] = sum over splits z (in order) of ws[z][r][c]
__global__ void __launch_bounds__(256) k_dfsum(const double* __restrict__ ws, int splits, int R, int C,
                                               const int* __restrict__ list, double* __restrict__ D, int64_t ldd) {
  const int r = blockIdx.y;
  for (int c = blockIdx.x * 256 + (int)threadIdx.x; c < C; c += gridDim.x * 256) {
    double t = 0.0;
    for (int z = 0; z < splits; ++z) t += ws[((size_t)z * R + r) * C + c];
    D[(size_t)list[r] * ldd + c] = t;
  }
}

// K splits so that few nodes still fill ~4 CTAs per SM; splits x tiles stays below
// 2 x 608, so the split partials fit kDfWsElems doubles
int dfprod_splits(int R, int C) {
  const int tiles = ((C + kDfCols - 1) / kDfCols) * ((R + kDfNodes - 1) / kDfNodes);
  if (tiles >= 4 * 152) return 1;
  const int sp = (4 * 152 + tiles - 1) / tiles;
  return sp < kDfMaxSplits ? sp : kDfMaxSplits;
}

double dfprod_error_factor(int K, int R, int C, int kblock) {
  const double u = 5.9604644775390625e-08, U = 1.1102230246251565e-16;
  const int splits = dfprod_splits(R, C);
  const double kb = kblock;
  const double blocks = (double)((K + kblock - 1) / kblock) + splits;
  return 1.01 * ((kb * kb / 2 + 6 * kb + 5) * u * u + (blocks + splits + 2) * U);
}

// D rows = A^T V rows for the listed nodes (A = X: V of length n, D of length p;
// A = Xc: V of length p, D of length n); ws: dfprod_ws_elems doubles when the
// product is split over K (few nodes)
void launch_dfprod(const Dev& d, bool use_xc, const double* V, int64_t ldv, const int* list, int R, double* D,
                   int64_t ldd, double* ws, int kblock, cudaStream_t s) {
  if (R <= 0) return;
  const int K = use_xc ? d.p : d.n, C = use_xc ? d.n : d.p;
  const int64_t lda = use_xc ? d.ldc : d.ldx;
  const void* A = use_xc ? d.Xc : d.X;
  const int splits = ws ? dfprod_splits(R, C) : 1;
  // split ranges are whole 32-row chunks; blocks (<= kDfBlock terms) restart in every split
  const int kchunk = ((K + splits - 1) / splits + kDfK - 1) / kDfK * kDfK;
  dim3 grid((C + kDfCols - 1) / kDfCols, (R + kDfNodes - 1) / kDfNodes, splits);
  double* w = splits > 1 ? ws : nullptr;
  if (d.xdt == kXF64)
    k_dfprod<double><<<grid, 256, 0, s>>>((const double*)A, lda, K, C, V, ldv, list, R, D, ldd, kchunk, kblock, w);
  else if (d.xdt == kXF32)
    k_dfprod<float><<<grid, 256, 0, s>>>((const float*)A, lda, K, C, V, ldv, list, R, D, ldd, kchunk, kblock, w);
  else
    k_dfprod<__nv_bfloat16><<<grid, 256, 0, s>>>((const __nv_bfloat16*)A, lda, K, C, V, ldv, list, R, D, ldd,
                                                 kchunk, kblock, w);
  if (splits > 1) {
    dim3 g2((C + 255) / 256 < 64 ? (C + 255) / 256 : 64, R);
    k_dfsum<<<g2, 256, 0, s>>>(ws, splits, R, C, list, D, ldd);
  }
}

}  // namespace ksc
