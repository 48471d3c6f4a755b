// k_tcexact.cu -- exact products of BF16 X with many FP64 vectors on the
// tensor cores (ksc_tcx.h): the anchors and certificates of the batched solver.
//
// One CTA computes a 128 x kTcxBN tile of D^T (128 rows c of A, kTcxBN vectors)
// over a range of K blocks of 64 (grid: vector tiles, row tiles, K splits):
//   warp 0      TMA producer: per K block the 3 slices of the 128 rows of A and
//               the 6 slices of the kTcxBN vectors land in one shared-memory
//               stage (128-byte swizzle);
//   warp 1      allocates 512 TMEM columns (two buffers of 8 diagonals x kTcxBN
//               FP32 columns) and issues, from one thread, the 18 slice-pair MMAs
//               (M = 128, N = kTcxBN, K = 16) of each K step, pair (t, s) into
//               diagonal t + s of the block's buffer; one commit frees the stage,
//               one hands the buffer to the drain;
//   warps 2..9  drain: per block, tcgen05.ld of the 8 diagonals (exact integers
//               below 2^24 in FP32), added into two 64-bit integers per output
//               (hi: diagonals 0-1 in units of 2^-8, lo: 2-7 in units of 2^-40
//               of the block's leading weight); the buffer is released to the MMA
//               warp at once, so one block drains while the next multiplies.
// At the end the drain converts (hi, lo) to FP64 with the row and vector
// exponents, or stores them as split partials that k_tcx_finish sums exactly.
// Every wait is bounded (%globaltimer); a wait that gives up sets the error
// word, raises the CTA's abort flag, and the CTA drains its copies and MMAs
// before it frees TMEM and exits.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <vector>

#include "ksc_tcptx.cuh"
#include "ksc_tcx.h"

namespace ksc {

constexpr int kTcxBM = 128;                 // rows of A per tile (TMEM lanes)
constexpr int kTcxBK = 64;                  // K block: one 128-byte swizzle row of BF16
constexpr int kTcxDiag = kTcxXSlices + kTcxVSlices - 1;    // 8 diagonals t + s
constexpr int kTcxBufs = 2;                 // TMEM accumulator buffers
constexpr uint32_t kTcxTmemCols = 512;
static_assert(kTcxBufs * kTcxDiag * kTcxBN <= (int)kTcxTmemCols, "TMEM holds both buffers");
constexpr uint32_t kTcxATile = kTcxBM * 128;        // bytes of one A slice per stage
constexpr uint32_t kTcxBTile = kTcxBN * 128;        // bytes of one vector slice per stage
constexpr uint32_t kTcxStageTx = kTcxXSlices * kTcxATile + kTcxVSlices * kTcxBTile;
constexpr int kTcxStages = 3;
constexpr int kTcxDrainWarps = 8;                   // two per TMEM lane quadrant
constexpr int kTcxThreads = 64 + 32 * kTcxDrainWarps;
constexpr int kTcxNodesPerThread = kTcxBN / 2;      // each drain warp takes half the vectors
constexpr int kTcxSmem = kTcxStages * (int)kTcxStageTx + 1024 + 256;
constexpr int kTcxMinBlocksPerSplit = 8;

__device__ int g_tcx_err;

// ------------------------------------------------------------------ slicing

// exponent e with 2^e <= m < 2^(e+1) of a positive normal float / double, from
// its bits (m = 0: 0)
__device__ __forceinline__ int exp_of(float m) {
  return m > 0.0f ? (int)((__float_as_uint(m) >> 23) & 0xffu) - 127 : 0;
}
__device__ __forceinline__ int exp_of(double m) {
  return m > 0.0 ? (int)((__double_as_longlong(m) >> 52) & 0x7ff) - 1023 : 0;
}
// 2^k for -1022 <= k <= 1023, built from its bits (exact)
__host__ __device__ __forceinline__ double pow2d(int k) {
  union { long long i; double d; } u;
  u.i = (long long)(k + 1023) << 52;
  return u.d;
}

// A slices, one CTA per row c of A (rows C..Cpad-1 written as zeros): e_c from the
// largest |a|; |a| 2^(23 - e_c) < 2^24 truncated to an integer q, slices
// q >> 16, (q >> 8) & 255, q & 255 with the sign of a; the truncated remainder
// (nonzero only for |a| < 2^(e_c - 16)) is counted (mode 0) or written as an
// exact residual entry at the row's offset (mode 1).
__global__ void __launch_bounds__(256) k_tcx_slice_rows(const __nv_bfloat16* __restrict__ A, int64_t lda, int C,
                                                        int K, __nv_bfloat16* __restrict__ sl, int64_t ld,
                                                        int Cpad, int* __restrict__ ex, int* __restrict__ cnt,
                                                        const int* __restrict__ off, int* __restrict__ rk,
                                                        double* __restrict__ rv, int mode) {
  __shared__ float red[256 / 32];
  __shared__ int wcnt[256 / 32];
  const int c = blockIdx.x;
  const __nv_bfloat16* row = A + (size_t)c * lda;
  float m = 0.0f;
  if (c < C)
    for (int k = threadIdx.x; k < K; k += 256) m = fmaxf(m, fabsf(__bfloat162float(row[k])));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.0f;
#pragma unroll
  for (int w = 0; w < 256 / 32; ++w) m = fmaxf(m, red[w]);
  const int e = exp_of(m);
  const double scale = pow2d(23 - e), unit = pow2d(e - 23);   // exact powers of two
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // residual entries are numbered in order of k (deterministic)
  int running = (mode == 1 && c < C) ? off[c] : 0, total = 0;
  for (int k0 = 0; k0 < (int)ld; k0 += 256) {
    const int k = k0 + (int)threadIdx.x;
    float a = 0.0f;
    if (c < C && k < K) a = __bfloat162float(row[k]);
    const double ma = (double)fabsf(a) * scale;     // < 2^24, exact
    const double qf = trunc(ma);
    const unsigned q = (unsigned)qf;
    const float sg = a < 0.0f ? -1.0f : 1.0f;
    if (k < (int)ld) {
      const size_t o = (size_t)c * ld + k;
      const size_t ps = (size_t)Cpad * ld;
      sl[o] = __float2bfloat16_rn(sg * (float)(q >> 16));
      sl[o + ps] = __float2bfloat16_rn(sg * (float)((q >> 8) & 255u));
      sl[o + 2 * ps] = __float2bfloat16_rn(sg * (float)(q & 255u));
    }
    const double rem = ma - qf;                     // exact: the bits below 2^(e - 23)
    const bool has = rem != 0.0;
    const unsigned bal = __ballot_sync(0xffffffffu, has);
    if (lane == 0) wcnt[warp] = __popc(bal);
    __syncthreads();
    int before = 0, chunk = 0;
#pragma unroll
    for (int w = 0; w < 256 / 32; ++w) {
      before += w < warp ? wcnt[w] : 0;
      chunk += wcnt[w];
    }
    if (mode == 1 && has) {
      const int pos = running + before + __popc(bal & ((1u << lane) - 1u));
      rk[pos] = k;
      rv[pos] = (double)sg * rem * unit;            // exact: a = sg (q + rem) 2^(e - 23)
    }
    running += chunk;
    total += chunk;
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (ex) ex[c] = e;
    if (mode == 0 && c < C) cnt[c] = total;
  }
}

// vector slices, one CTA per listed vector r < Rt (rows r >= R written as zeros):
// f_r from the largest |v|; |v| 2^(47 - f_r) < 2^48 truncated to an integer q,
// slices q >> 40, (q >> 32) & 255, ..., q & 255 with the sign of v
__global__ void __launch_bounds__(256) k_tcx_slice_vecs(const double* __restrict__ V, int64_t ldv,
                                                        const int* __restrict__ list, int R, int K,
                                                        __nv_bfloat16* __restrict__ sl, int64_t ld, int Npad,
                                                        int* __restrict__ ev) {
  __shared__ double red[256 / 32];
  const int r = blockIdx.x;
  const double* row = r < R ? V + (size_t)(list ? list[r] : r) * ldv : nullptr;
  double m = 0.0;
  if (row)
    for (int k = threadIdx.x; k < K; k += 256) m = fmax(m, fabs(row[k]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = m;
  __syncthreads();
  m = 0.0;
#pragma unroll
  for (int w = 0; w < 256 / 32; ++w) m = fmax(m, red[w]);
  const int f = exp_of(m);
  const double s0 = pow2d(-f), s1 = pow2d(47);    // exact powers of two (two steps: -f may be 1023)
  for (int k = threadIdx.x; k < (int)ld; k += 256) {
    const double v = (row && k < K) ? row[k] : 0.0;
    const unsigned long long q = (unsigned long long)(fabs(v) * s0 * s1);   // < 2^48, truncated
    const float sg = v < 0.0 ? -1.0f : 1.0f;
    const size_t o = (size_t)r * ld + k;
    const size_t ps = (size_t)Npad * ld;
#pragma unroll
    for (int s = 0; s < kTcxVSlices; ++s)
      sl[o + s * ps] = __float2bfloat16_rn(sg * (float)((q >> (8 * (kTcxVSlices - 1 - s))) & 255ull));
  }
  if (threadIdx.x == 0) ev[r] = f;
}

// ------------------------------------------------------------------ product

struct TcxShape {
  int C, Cpad, R, Npad, nkb, kbs;   // kbs: K blocks per split (blockIdx.z)
};

struct TcxOut {
  double* D;
  int64_t ldd;
  const int* list;
  const int* ex;
  const int* ev;
  long long* part;   // split partials (gridDim.z > 1): ((z Rt + r) C + c) pairs, Rt = gridDim.x kTcxBN
};

// instruction descriptor for M = 128, N = kTcxBN (kind::f16, BF16 A and B, FP32 D)
constexpr uint32_t kTcxIdesc = tc_idesc(kTcxBM, kTcxBN);

__global__ void __launch_bounds__(kTcxThreads, 1)
    k_tcx(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcxShape sh,
          TcxOut out) {
  constexpr int S = kTcxStages;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + S * kTcxXSlices * kTcxATile;
  uint64_t* full = (uint64_t*)(sB + S * kTcxVSlices * kTcxBTile);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;           // kTcxBufs: the block's diagonals are in TMEM
  uint64_t* drained = accf + kTcxBufs;  // kTcxBufs: the drain has read them
  uint64_t* drainend = drained + kTcxBufs;
  uint32_t* tmem_slot = (uint32_t*)(drainend + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  // blockIdx.x runs over the vector tiles, so the CTAs that share a tile of X's
  // slices run together and X streams from DRAM about once
  const int c0 = blockIdx.y * kTcxBM, r0 = blockIdx.x * kTcxBN;
  const int kb0 = blockIdx.z * sh.kbs;
  const int nb = max(0, min(sh.nkb, kb0 + sh.kbs) - kb0);

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < kTcxBufs; ++i) {
      mbar_init(&accf[i], 1);
      mbar_init(&drained[i], kTcxDrainWarps);
    }
    mbar_init(drainend, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, kTcxTmemCols);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
      int issued = 0;
      for (int i = 0; i < nb; ++i) {
        const int s = i % S;
        const uint32_t ph = (uint32_t)(i / S) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
          atomicExch(&g_tcx_err, 1);
          *abort_flag = 1;
          break;
        }
        mbar_expect_tx(&full[s], kTcxStageTx);
        const int kx = (kb0 + i) * kTcxBK;
#pragma unroll
        for (int t = 0; t < kTcxXSlices; ++t)
          tma_load_2d(sA + (s * kTcxXSlices + t) * kTcxATile, &tmA, &full[s], kx, t * sh.Cpad + c0);
#pragma unroll
        for (int v = 0; v < kTcxVSlices; ++v)
          tma_load_2d(sB + (s * kTcxVSlices + v) * kTcxBTile, &tmB, &full[s], kx, v * sh.Npad + r0);
        issued = i + 1;
      }
      if (*abort_flag) {
        // let the copies already issued land before the CTA leaves
        for (int i = issued - S < 0 ? 0 : issued - S; i < issued; ++i) {
          volatile int never = 0;
          mbar_wait(&full[i % S], (uint32_t)(i / S) & 1u, &never);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      bool ok = true;
      for (int i = 0; i < nb; ++i) {
        const int s = i % S;
        const int buf = i % kTcxBufs;
        if (!mbar_wait(&full[s], (uint32_t)(i / S) & 1u, abort_flag) ||
            (i >= kTcxBufs && !mbar_wait(&drained[buf], (uint32_t)(i / kTcxBufs - 1) & 1u, abort_flag))) {
          atomicExch(&g_tcx_err, 2);
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dbase = tmem + (uint32_t)(buf * kTcxDiag * kTcxBN);
#pragma unroll
        for (int kk = 0; kk < kTcxBK / 16; ++kk) {
#pragma unroll
          for (int t = 0; t < kTcxXSlices; ++t) {
            const uint64_t ad = sw128_desc(smem_u32(sA + (s * kTcxXSlices + t) * kTcxATile) + kk * 32);
#pragma unroll
            for (int v = 0; v < kTcxVSlices; ++v) {
              const int d = t + v;
              // the first pair of diagonal d in the block starts it afresh
              const uint32_t acc = (kk == 0 && t == (d > kTcxVSlices - 1 ? d - (kTcxVSlices - 1) : 0)) ? 0u : 1u;
              umma_bf16(dbase + (uint32_t)(d * kTcxBN), ad,
                        sw128_desc(smem_u32(sB + (s * kTcxVSlices + v) * kTcxBTile) + kk * 32), kTcxIdesc, acc);
            }
          }
        }
        umma_commit(&empty[s]);
        umma_commit(&accf[buf]);
      }
      if (!ok) {
        // wait for the MMAs already issued before TMEM is released
        umma_commit(drainend);
        volatile int never = 0;
        mbar_wait(drainend, 0, &never);
      }
    }
    __syncwarp();
  } else {
    const int qd = warp & 3;                 // TMEM lanes 32 qd .. 32 qd + 31
    const int half = (warp - 2) >> 2;        // vectors half * 16 .. half * 16 + 15 of the tile
    const int c = c0 + 32 * qd + lane;
    long long zh[kTcxNodesPerThread], zl[kTcxNodesPerThread];
#pragma unroll
    for (int j = 0; j < kTcxNodesPerThread; ++j) { zh[j] = 0; zl[j] = 0; }
    const uint32_t lanes = (uint32_t)(32 * qd) << 16;
    bool ok = true;
    for (int i = 0; i < nb; ++i) {
      const int buf = i % kTcxBufs;
      ok = __all_sync(0xffffffffu, mbar_wait(&accf[buf], (uint32_t)(i / kTcxBufs) & 1u, abort_flag) ? 1 : 0) != 0;
      if (!ok) break;
      tc_fence_after();
      const uint32_t tb = tmem + lanes + (uint32_t)(buf * kTcxDiag * kTcxBN + half * kTcxNodesPerThread);
      uint32_t a[16], b[16];
      // diagonals 0, 1: hi += acc_0 2^8 + acc_1 (below 2^31: int32)
      tmem_ld16_nowait(tb + 0 * kTcxBN, a);
      tmem_ld16_nowait(tb + 1 * kTcxBN, b);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j)
        zh[j] += (long long)(__float2int_rz(__uint_as_float(a[j])) * 256 + __float2int_rz(__uint_as_float(b[j])));
      // diagonals 6, 7 in units of 2^-40: acc_6 2^-8 + acc_7 2^-16 (below 2^16),
      // rounded to an int32 on the FP32 pipe (64-bit conversions would run on the
      // slow FP64 one)
      tmem_ld16_nowait(tb + 6 * kTcxBN, a);
      tmem_ld16_nowait(tb + 7 * kTcxBN, b);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j)
        zl[j] += (long long)__float2int_rn(__fmaf_rn(__uint_as_float(a[j]), 0.00390625f,
                                                     __uint_as_float(b[j]) * 1.52587890625e-05f));
      // diagonals 2, 3: acc_2 2^24 + acc_3 2^16
      tmem_ld16_nowait(tb + 2 * kTcxBN, a);
      tmem_ld16_nowait(tb + 3 * kTcxBN, b);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j)
        zl[j] += ((long long)__float2int_rz(__uint_as_float(a[j])) << 24) +
                 ((long long)__float2int_rz(__uint_as_float(b[j])) << 16);
      // diagonals 4, 5: acc_4 2^8 + acc_5
      tmem_ld16_nowait(tb + 4 * kTcxBN, a);
      tmem_ld16_nowait(tb + 5 * kTcxBN, b);
      tmem_wait_ld();
#pragma unroll
      for (int j = 0; j < 16; ++j)
        zl[j] += (long long)(__float2int_rz(__uint_as_float(a[j])) * 256) + (long long)__float2int_rz(__uint_as_float(b[j]));
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&drained[buf]);
    }
    if (!ok) {
      atomicExch(&g_tcx_err, 3);
      *abort_flag = 1;
    } else if (c < sh.C) {
      const int rb = r0 + half * kTcxNodesPerThread;
      if (gridDim.z == 1) {
        const double sc = pow2d(out.ex[c] - 7);
#pragma unroll
        for (int j = 0; j < kTcxNodesPerThread; ++j) {
          const int r = rb + j;
          if (r < sh.R) {
            // value = 2^(e_c + f_r - 14) (hi 2^-8 + lo 2^-40), hi 2^-8 exact in FP64
            const double v = ((double)zh[j] * 0.00390625 + (double)zl[j] * 9.094947017729282e-13) * sc *
                             pow2d(out.ev[r] - 7);
            out.D[(int64_t)(out.list ? out.list[r] : r) * out.ldd + c] = v;
          }
        }
      } else {
        const int64_t Rt = (int64_t)gridDim.x * kTcxBN;
#pragma unroll
        for (int j = 0; j < kTcxNodesPerThread; ++j) {
          long long* pp = out.part + 2 * (((int64_t)blockIdx.z * Rt + rb + j) * sh.C + c);
          pp[0] = zh[j];
          pp[1] = zl[j];
        }
      }
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, kTcxTmemCols);
}

// split partials summed exactly (64-bit integers), converted like the drain does
__global__ void __launch_bounds__(256) k_tcx_finish(const long long* __restrict__ part, int splits, int Rt, int C,
                                                    int R, const int* __restrict__ ex, const int* __restrict__ ev,
                                                    const int* __restrict__ list, double* __restrict__ D,
                                                    int64_t ldd) {
  const int r = blockIdx.y;
  for (int c = blockIdx.x * 256 + (int)threadIdx.x; c < C; c += gridDim.x * 256) {
    long long h = 0, l = 0;
    for (int z = 0; z < splits; ++z) {
      const long long* pp = part + 2 * (((int64_t)z * Rt + r) * C + c);
      h += pp[0];
      l += pp[1];
    }
    const double v = ((double)h * 0.00390625 + (double)l * 9.094947017729282e-13) * pow2d(ex[c] - 7) *
                     pow2d(ev[r] - 7);
    D[(int64_t)(list ? list[r] : r) * ldd + c] = v;
  }
}

// the exact residuals of A (entries below 2^(e_c - 16)): D[c] += sum res v[k], FP64
__global__ void __launch_bounds__(256) k_tcx_resid(const int* __restrict__ rows, const int* __restrict__ ptr,
                                                   const int* __restrict__ rk, const double* __restrict__ rv,
                                                   int nrr, const double* __restrict__ V, int64_t ldv,
                                                   const int* __restrict__ list, double* __restrict__ D,
                                                   int64_t ldd) {
  const int q = blockIdx.x * 256 + (int)threadIdx.x;
  if (q >= nrr) return;
  const int r = blockIdx.y;
  const int64_t vr = list ? list[r] : r;
  const double* v = V + vr * ldv;
  double s = 0.0;
  for (int e = ptr[q]; e < ptr[q + 1]; ++e) s += rv[e] * v[rk[e]];
  D[vr * ldd + rows[q]] += s;
}

// ------------------------------------------------------------------ host

static PFN_cuTensorMapEncodeTiled_v12000 tcx_encode_fn() {
  static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
  static bool tried = false;
  if (!tried) {
    tried = true;
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = (PFN_cuTensorMapEncodeTiled_v12000)p;
  }
  return fn;
}

static bool tcx_map(void* out, const void* base, uint64_t inner, uint64_t rows, int64_t ld, uint32_t box_rows,
                    const char** why) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = tcx_encode_fn();
  if (!fn) {
    *why = "cuTensorMapEncodeTiled is not available from the driver";
    return false;
  }
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * 2};
  cuuint32_t box[2] = {(cuuint32_t)kTcxBK, box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn((CUtensorMap*)out, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *why = "cuTensorMapEncodeTiled rejected the slice layout";
    return false;
  }
  return true;
}

static int64_t round_up(int64_t a, int64_t b) { return (a + b - 1) / b * b; }

cudaError_t tcx_prepare() {
  return cudaFuncSetAttribute(k_tcx, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcxSmem);
}

void tcx_slices_free(TcxSlices* x) {
  void* ptrs[] = {x->sl, x->ex, x->res_rows, x->res_ptr, x->res_k, x->res_v};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  *x = TcxSlices{};
}

bool tcx_slices_build(TcxSlices* x, const void* A, int C, int K, int64_t lda, cudaStream_t s, const char** why) {
  tcx_slices_free(x);
  if (C <= 0 || K <= 0 || lda < K) {
    *why = "empty or malformed operand";
    return false;
  }
  x->C = C;
  x->K = K;
  x->Cpad = (int)round_up(C, kTcxBM);
  x->ld = round_up(K, kTcxBK);
  const size_t sl_elems = (size_t)kTcxXSlices * x->Cpad * x->ld;
  int* cnt = nullptr;
  int* off = nullptr;
  auto fail = [&](const char* m) {
    if (cnt) cudaFree(cnt);
    if (off) cudaFree(off);
    tcx_slices_free(x);
    *why = m;
    return false;
  };
  if (cudaMalloc(&x->sl, sl_elems * 2) != cudaSuccess || cudaMalloc(&x->ex, (size_t)x->Cpad * 4) != cudaSuccess ||
      cudaMalloc(&cnt, (size_t)C * 4) != cudaSuccess || cudaMalloc(&off, (size_t)C * 4) != cudaSuccess)
    return fail("out of device memory for the slices of X");
  const __nv_bfloat16* a = (const __nv_bfloat16*)A;
  k_tcx_slice_rows<<<x->Cpad, 256, 0, s>>>(a, lda, C, K, x->sl, x->ld, x->Cpad, x->ex, cnt, nullptr, nullptr,
                                           nullptr, 0);
  std::vector<int> hc(C), ho(C);
  if (cudaMemcpyAsync(hc.data(), cnt, (size_t)C * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return fail("slicing X failed");
  int64_t tot = 0;
  std::vector<int> rows, ptr;
  for (int c = 0; c < C; ++c) {
    ho[c] = (int)tot;
    if (hc[c] > 0) {
      rows.push_back(c);
      ptr.push_back((int)tot);
      x->res_max = std::max(x->res_max, hc[c]);
    }
    tot += hc[c];
  }
  if (tot > INT32_MAX) return fail("too many residual entries");
  ptr.push_back((int)tot);
  x->nres = (int)tot;
  x->nrr = (int)rows.size();
  if (x->nres > 0) {
    if (cudaMalloc(&x->res_k, (size_t)x->nres * 4) != cudaSuccess ||
        cudaMalloc(&x->res_v, (size_t)x->nres * 8) != cudaSuccess ||
        cudaMalloc(&x->res_rows, (size_t)x->nrr * 4) != cudaSuccess ||
        cudaMalloc(&x->res_ptr, (size_t)(x->nrr + 1) * 4) != cudaSuccess)
      return fail("out of device memory for the residuals of X");
    if (cudaMemcpyAsync(off, ho.data(), (size_t)C * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(x->res_rows, rows.data(), (size_t)x->nrr * 4, cudaMemcpyHostToDevice, s) != cudaSuccess ||
        cudaMemcpyAsync(x->res_ptr, ptr.data(), (size_t)(x->nrr + 1) * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
      return fail("copying the residual index failed");
    k_tcx_slice_rows<<<C, 256, 0, s>>>(a, lda, C, K, x->sl, x->ld, x->Cpad, nullptr, nullptr, off, x->res_k,
                                       x->res_v, 1);
  }
  if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess)
    return fail("slicing X failed");
  cudaFree(cnt);
  cudaFree(off);
  cnt = off = nullptr;
  if (!tcx_map(x->tm, x->sl, (uint64_t)K, (uint64_t)kTcxXSlices * x->Cpad, x->ld, kTcxBM, why)) {
    const char* m = *why;
    return fail(m);
  }
  x->bytes = sl_elems * 2 + (size_t)x->Cpad * 4 + (size_t)x->nres * 12 + (size_t)(2 * x->nrr + 1) * 4;
  x->ok = true;
  return true;
}

void tcx_vecs_free(TcxVecs* v) {
  void* ptrs[] = {v->sl, v->ev, v->part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  *v = TcxVecs{};
}

static int tcx_nsm() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0) n = 152;
  return n;
}

bool tcx_vecs_alloc(TcxVecs* v, int Rcap, int K, const char** why) {
  tcx_vecs_free(v);
  if (Rcap <= 0 || Rcap > kTcxMaxR || K <= 0) {
    *why = "vector count or length out of range";
    return false;
  }
  v->Rcap = Rcap;
  v->K = K;
  v->Npad = (int)round_up(Rcap, kTcxBN);
  v->ld = round_up(K, kTcxBK);
  // split partials: splits x tiles stays below 4 x SMs (tcx_plan), 128 x kTcxBN pairs a tile
  v->part_pairs = (size_t)4 * tcx_nsm() * kTcxBM * kTcxBN;
  const size_t sl_elems = (size_t)kTcxVSlices * v->Npad * v->ld;
  if (cudaMalloc(&v->sl, sl_elems * 2) != cudaSuccess || cudaMalloc(&v->ev, (size_t)v->Npad * 4) != cudaSuccess ||
      cudaMalloc(&v->part, v->part_pairs * 16) != cudaSuccess) {
    tcx_vecs_free(v);
    *why = "out of device memory for the vector slices";
    return false;
  }
  if (!tcx_map(v->tm, v->sl, (uint64_t)K, (uint64_t)kTcxVSlices * v->Npad, v->ld, kTcxBN, why)) {
    tcx_vecs_free(v);
    return false;
  }
  v->bytes = sl_elems * 2 + (size_t)v->Npad * 4 + v->part_pairs * 16;
  v->ok = true;
  return true;
}

// grid of one product: row tiles, vector tiles, K splits (more splits while the
// tiles leave SMs idle, each split at least kTcxMinBlocksPerSplit K blocks)
struct TcxPlan {
  int tc, tr, nkb, splits, kbs;
};
static TcxPlan tcx_plan(const TcxSlices& x, int R) {
  TcxPlan p;
  p.tc = (x.C + kTcxBM - 1) / kTcxBM;
  p.tr = (R + kTcxBN - 1) / kTcxBN;
  p.nkb = (x.K + kTcxBK - 1) / kTcxBK;
  const int tiles = p.tc * p.tr, nsm = tcx_nsm();
  int sp = 1;
  if (tiles < 2 * nsm) sp = (2 * nsm + tiles - 1) / tiles;
  sp = std::min(sp, std::max(1, p.nkb / kTcxMinBlocksPerSplit));
  p.kbs = (p.nkb + sp - 1) / sp;
  p.splits = (p.nkb + p.kbs - 1) / p.kbs;
  return p;
}

int tcx_launches(const TcxSlices& x, int R) {
  const TcxPlan p = tcx_plan(x, R);
  return 2 + (p.splits > 1) + (x.nrr > 0);
}

double tcx_error_factor(const TcxSlices& x) {
  const double K = (double)x.K;
  return 1.01 * (sqrt(K) * ldexp(1.0, -47) + ldexp(1.0, -54) * (K / 64.0 + 1.0) +
                 (4.0 + (double)x.res_max) * ldexp(1.0, -53));
}

int* tcx_error_word() {
  int* p = nullptr;
  cudaGetSymbolAddress((void**)&p, g_tcx_err);
  return p;
}

void tcx_clear_error(cudaStream_t s) {
  int* p = tcx_error_word();
  if (p) cudaMemsetAsync(p, 0, sizeof(int), s);
}

void tcx_product(const TcxSlices& x, TcxVecs& v, const double* V, int64_t ldv, const int* list, int R, double* D,
                 int64_t ldd, cudaStream_t s) {
  if (R <= 0) return;
  const TcxPlan p = tcx_plan(x, R);
  const int Rt = p.tr * kTcxBN;
  k_tcx_slice_vecs<<<Rt, 256, 0, s>>>(V, ldv, list, R, x.K, v.sl, v.ld, v.Npad, v.ev);
  TcxShape sh{x.C, x.Cpad, R, v.Npad, p.nkb, p.kbs};
  TcxOut out{D, ldd, list, x.ex, v.ev, v.part};
  dim3 grid(p.tr, p.tc, p.splits);
  k_tcx<<<grid, kTcxThreads, kTcxSmem, s>>>(*(const CUtensorMap*)x.tm, *(const CUtensorMap*)v.tm, sh, out);
  if (p.splits > 1) {
    dim3 g2((x.C + 255) / 256 < 64 ? (x.C + 255) / 256 : 64, R);
    k_tcx_finish<<<g2, 256, 0, s>>>(v.part, p.splits, Rt, x.C, R, x.ex, v.ev, list, D, ldd);
  }
  if (x.nrr > 0) {
    dim3 g3((x.nrr + 255) / 256, R);
    k_tcx_resid<<<g3, 256, 0, s>>>(x.res_rows, x.res_ptr, x.res_k, x.res_v, x.nrr, V, ldv, list, D, ldd);
  }
}

}  // namespace ksc
