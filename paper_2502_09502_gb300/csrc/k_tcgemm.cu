// k_tcgemm.cu -- the batched solver's products on the 5th-generation tensor cores.
//
// One CTA computes a 128 x BN tile of D = sum_q A_q B^T (ksc_tc.h):
//   warp 0      TMA producer: per 64-wide K block, the P pieces of the 128 A rows
//               and the BN rows of B land in one shared-memory stage (128-byte
//               swizzle), signalled on the stage's "full" mbarrier;
//   warp 1      allocates the TMEM accumulator (128 lanes x BN FP32 columns) and,
//               from one thread, issues tcgen05.mma (M = 128, N = BN, K = 16; four
//               per piece per K block) and tcgen05.commit to free each stage;
//   warps 2..5  epilogue: tcgen05.ld of their 32 TMEM lanes (one output row per
//               thread): row-major FP32 stores, or FP64 anchor + D with the loss
//               partials of the row.
// Every wait is bounded (%globaltimer); a wait that gives up sets the error word,
// raises the CTA's abort flag and the CTA drains its copies and MMAs before it
// frees TMEM and exits.
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdint.h>

#include "ksc_state.cuh"
#include "ksc_tc.h"
#include "ksc_tcptx.cuh"

namespace ksc {

constexpr int kTcThreads = 192;
constexpr int kTcBM = 128;
constexpr int kTcBK = 64;                       // 64 BF16 = one 128-byte swizzle row
constexpr uint32_t kTcATile = kTcBM * 128;      // bytes of one A piece per stage
constexpr int kTcSmemMax = 232448 - 2048;       // opt-in limit minus alignment and barriers

__device__ int g_tc_err;

__host__ __device__ constexpr int tc_stage_bytes(int P, int BN) { return P * (int)kTcATile + BN * 128; }
__host__ __device__ constexpr int tc_stages(int P, int BN) {
  return (kTcSmemMax / tc_stage_bytes(P, BN)) > 6 ? 6 : (kTcSmemMax / tc_stage_bytes(P, BN));
}
__host__ __device__ constexpr int tc_smem_bytes(int P, int BN) {
  return tc_stages(P, BN) * tc_stage_bytes(P, BN) + 1024 + 256;
}
__host__ __device__ constexpr uint32_t tc_tmem_cols(int BN) {
  return BN <= 32 ? 32u : BN <= 64 ? 64u : BN <= 128 ? 128u : BN <= 256 ? 256u : 512u;
}

// E4M3 plans keep two accumulators per tile: pieces [0, kTcE4m3Hi) in the tile's
// first BN TMEM columns, the rest (cut from the residual scaled by 2^kTcE4m3Shift)
// in the next BN; the epilogue adds them as hi + 2^-kTcE4m3Shift lo
template <int E8>
__device__ __forceinline__ void tmem_ld_tile16(uint32_t taddr, int bn, float* v) {
  tmem_ld16(taddr, v);
  if (E8) {
    float w[16];
    tmem_ld16(taddr + (uint32_t)bn, w);
    constexpr float lo = 1.0f / (float)(1 << kTcE4m3Shift);
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = fmaf(w[i], lo, v[i]);
  }
}

// F_i(u) in FP32 (summed in FP64 by the caller)
__device__ __forceinline__ float loss_term(float u, float y, int loss) {
  if (loss == kLossLsq) {
    const float r = u - y;
    return r * r;
  }
  if (loss == kLossPoisson) return expf(u) - y * u;
  if (loss == kLossGamma) return y * expf(-u) + u;
  const float t = -y * u;
  return fmaxf(t, 0.0f) + log1pf(expf(-fabsf(t)));
}

// F_i(u) added to an FP64 sum (least squares, squared hinge: the difference
// u - y or 1 - y u cancels near the fit) or to an FP32 one (logistic)
__device__ __forceinline__ void add_loss(double u, float y, int loss, double& fd, float& fa) {
  if (loss == kLossLsq) {
    const double r = u - (double)y;
    fd += r * r;
  } else if (loss == kLossSqHinge) {
    const double m = fmax(0.0, 1.0 - (double)y * u);
    fd += m * m;
  } else {
    fa += loss_term((float)u, y, loss);
  }
}

// F_i(u + d) - F_i(u) without cancellation: least squares d (2 (u - y) + d);
// squared hinge with s = 1 - y u, t = -y d: t (2 s + t) where s and s + t are
// both positive, else max(0, s + t)^2 - max(0, s)^2; Poisson e^u expm1(d) - y d;
// Gamma y e^-u expm1(-d) + d; logistic
// log1p(expm1(-y d) sigma(-y u)), since
// (1 + e^{-y(u+d)}) / (1 + e^{-y u}) = 1 + (e^{-y d} - 1) e^{-y u} / (1 + e^{-y u})
__device__ __forceinline__ float loss_change(double u, float d, float y, int loss) {
  if (loss == kLossLsq) {
    const float r = (float)(u - (double)y);
    return d * (2.0f * r + d);
  }
  if (loss == kLossSqHinge) {
    const float s = (float)(1.0 - (double)y * u), t = -y * d;
    if (s > 0.0f && s + t > 0.0f) return t * (2.0f * s + t);
    const float m = fmaxf(s, 0.0f), mn = fmaxf(s + t, 0.0f);
    return mn * mn - m * m;
  }
  // far from u (|d| > 16) the plain difference: expm1 could overflow, and there is
  // no cancellation to avoid
  if (fabsf(d) > 16.0f) return loss_term((float)(u + (double)d), y, loss) - loss_term((float)u, y, loss);
  if (loss == kLossPoisson) return expf((float)u) * expm1f(d) - y * d;            // e^u (e^d - 1) - y d
  if (loss == kLossGamma) return y * expf(-(float)u) * expm1f(-d) + d;         // y e^-u (e^-d - 1) + d
  const float s = 1.0f / (1.0f + expf(y * (float)u));   // sigma(-y u)
  return log1pf(expm1f(-y * d) * s);
}

// ------------------------------------------------------------------ kernel

// bk: elements per K block of 128 bytes (64 BF16 or 128 E4M3)
struct TcShape {
  int M, Mpad, N, K, bk;
};

// row pointers of the epilogue and one 16-column chunk of it (nc = first column
// of the chunk, a multiple of 16), shared by both schedules and the fix-up
struct EpiRow {
  float* orow;
  const double* brow;
  double* o64;
  const double* uin;
  double* uout;
  bool ok;
};

template <int MODE>
__device__ __forceinline__ EpiRow epi_row(const TcShape& sh, const TcEpi& ep, int m) {
  EpiRow r{nullptr, nullptr, nullptr, nullptr, nullptr, m < sh.M};
  if (!r.ok) return r;
  if (MODE == kTcStore) {
    r.orow = ep.out + (int64_t)m * ep.ldo;
  } else if (MODE == kTcAdd) {
    r.brow = ep.base + (int64_t)m * ep.ldb;
    r.o64 = ep.out64 + (int64_t)m * ep.ldo;
  } else {
    r.brow = ep.base + (int64_t)m * ep.ldb;
    r.uin = ep.u64 + (int64_t)m * ep.ldo + (int64_t)ep.slot_in[m] * ep.slot_stride;
    r.uout = ep.u64 + (int64_t)m * ep.ldo + (int64_t)ep.slot_out[m] * ep.slot_stride;
  }
  return r;
}

// PART: write the loss partials when the chunk closes its 64-column group (the
// fix-up kernel sums its four chunks across threads and writes them itself)
template <int MODE, bool PART = true>
__device__ __forceinline__ void epi_chunk(const TcShape& sh, const TcEpi& ep, const EpiRow& r, int m, int nc,
                                          float* v, double& fsum, double& dsum) {
  if (!r.ok || nc >= sh.N) return;
  const bool whole = nc + 16 <= sh.N;   // rows are 64-byte aligned (strides padded to 8 elements)
  if (ep.rscale != nullptr) {
    // E4M3 operands: undo the row's power-of-two scale and apply the columns'
    // (both exact in FP32)
    const float rs = ep.rscale[m];
#pragma unroll
    for (int i = 0; i < 16; ++i)
      v[i] *= (ep.cscale != nullptr && nc + i < sh.N) ? rs * ep.cscale[nc + i] : rs;
  }
  if (MODE == kTcStore) {
#pragma unroll
    for (int i = 0; i < 16; ++i)
      if (nc + i < sh.N) r.orow[nc + i] = v[i];
  } else if (MODE == kTcAdd) {
    if (whole) {
      const double2* b2 = reinterpret_cast<const double2*>(r.brow + nc);
      double2* o2 = reinterpret_cast<double2*>(r.o64 + nc);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const double2 b = b2[i];
        o2[i] = make_double2(b.x + (double)v[2 * i], b.y + (double)v[2 * i + 1]);
      }
    } else {
#pragma unroll 4
      for (int i = 0; i < 16; ++i)
        if (nc + i < sh.N) r.o64[nc + i] = r.brow[nc + i] + (double)v[i];
    }
  } else if (whole) {
    float fa = 0.0f, da = 0.0f;
    double fd = 0.0;
    const double2* u2 = reinterpret_cast<const double2*>(r.uin + nc);
    const double2* b2 = reinterpret_cast<const double2*>(r.brow + nc);
    double2* w2 = reinterpret_cast<double2*>(r.uout + nc);
    const float4* y4 = reinterpret_cast<const float4*>(ep.y + nc);
#pragma unroll 2
    for (int i = 0; i < 8; ++i) {
      const double2 uo = u2[i], b = b2[i];
      const float4 yq = __ldg(&y4[i >> 1]);
      const float y0 = (i & 1) ? yq.z : yq.x, y1 = (i & 1) ? yq.w : yq.y;
      const double un0 = b.x + (double)v[2 * i], un1 = b.y + (double)v[2 * i + 1];
      w2[i] = make_double2(un0, un1);
      add_loss(un0, y0, ep.loss, fd, fa);
      add_loss(un1, y1, ep.loss, fd, fa);
      da += loss_change(uo.x, (float)(un0 - uo.x), y0, ep.loss) + loss_change(uo.y, (float)(un1 - uo.y), y1, ep.loss);
    }
    fsum += (double)fa + fd;
    dsum += (double)da;
    if (PART && (((nc + 16) & 63) == 0 || nc + 16 >= sh.N)) {
      double* pp = ep.part + 2 * ((int64_t)m * ep.npart + (nc >> 6));
      pp[0] = fsum;
      pp[1] = dsum;
      fsum = 0.0;
      dsum = 0.0;
    }
  } else {
    float fa = 0.0f, da = 0.0f;
    double fd = 0.0;
#pragma unroll 4
    for (int i = 0; i < 16; ++i) {
      if (nc + i < sh.N) {
        const double uo = r.uin[nc + i];
        const double un = r.brow[nc + i] + (double)v[i];
        r.uout[nc + i] = un;
        const float yi = __ldg(&ep.y[nc + i]);
        add_loss(un, yi, ep.loss, fd, fa);
        da += loss_change(uo, (float)(un - uo), yi, ep.loss);
      }
    }
    fsum += (double)fa + fd;
    dsum += (double)da;
    if (PART && (((nc + 16) & 63) == 0 || nc + 16 >= sh.N)) {   // one pair of partials per 64 columns
      double* pp = ep.part + 2 * ((int64_t)m * ep.npart + (nc >> 6));
      pp[0] = fsum;
      pp[1] = dsum;
      fsum = 0.0;
      dsum = 0.0;
    }
  }
}

// ------------------------------------------------------------------ stream-K

constexpr int kSkMaxMTiles = 8;   // M <= 1024

// The work assignment, computed identically by every CTA of both kernels from the
// tile flags (which do not change between them): active M tiles in order, tiles
// numbered N-major (CTAs that run at the same time share B tiles in L2), K blocks
// of every tile consecutive; CTA c owns iterations [c I / G, (c+1) I / G).
struct SkMap {
  int act[kSkMaxMTiles];
  int A, nN, KB, G;
  int64_t I;
};

__device__ __forceinline__ void sk_map(const TcShape& sh, const TcEpi& ep, int bn, int G, SkMap& mp) {
  const int nM = (sh.M + kTcBM - 1) / kTcBM;
  mp.A = 0;
  for (int t = 0; t < nM && t < kSkMaxMTiles; ++t)
    if (ep.tile_active == nullptr || ep.tile_active[t] != 0) mp.act[mp.A++] = t;
  mp.nN = (sh.N + bn - 1) / bn;
  mp.KB = (sh.K + sh.bk - 1) / sh.bk;
  mp.G = G;
  mp.I = (int64_t)mp.A * mp.nN * mp.KB;
}
__device__ __forceinline__ int64_t sk_begin(const SkMap& mp, int c) { return (int64_t)c * mp.I / mp.G; }
__device__ __forceinline__ int sk_owner(const SkMap& mp, int64_t i) { return (int)(((i + 1) * mp.G - 1) / mp.I); }

// E8: A and B hold E4M3 bytes (kind::f8f6f4) instead of BF16 (kind::f16)
template <int P, int BN, int MODE, int E8>
__global__ void __launch_bounds__(kTcThreads, 1)
    k_tcgemm(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcShape sh,
             TcEpi ep) {
  // every row of this M tile belongs to a finished node: nothing to compute
  if (ep.tile_active != nullptr && ep.tile_active[blockIdx.y] == 0) return;
  constexpr int S = tc_stages(P, BN);
  constexpr uint32_t B_TILE = BN * 128;
  constexpr uint32_t STAGE_TX = P * kTcATile + B_TILE;
  constexpr uint32_t TCOLS = tc_tmem_cols((E8 ? 2 : 1) * BN);
  static_assert(S >= 2, "at least two pipeline stages");
  static_assert(BN % 16 == 0 && BN >= 16 && BN <= 256, "MMA N for M = 128");
  static_assert(!E8 || BN <= 128, "two E4M3 accumulators of BN columns each");

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + S * P * kTcATile;
  uint64_t* full = (uint64_t*)(sB + S * B_TILE);
  uint64_t* empty = full + S;
  uint64_t* accf = empty + S;
  uint64_t* drain = accf + 1;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m0 = blockIdx.y * kTcBM, n0 = blockIdx.x * BN;
  const int nkb = (sh.K + sh.bk - 1) / sh.bk;

  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    mbar_init(accf, 1);
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
      int issued = 0;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % S;
        const uint32_t ph = (uint32_t)(kb / S) & 1u;
        if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
          atomicExch(&g_tc_err, 1);
          *abort_flag = 1;
          break;
        }
        mbar_expect_tx(&full[s], STAGE_TX);
#pragma unroll
        for (int q = 0; q < P; ++q)
          tma_load_2d(sA + (s * P + q) * kTcATile, &tmA, &full[s], kb * sh.bk, q * sh.Mpad + m0);
        tma_load_2d(sB + s * B_TILE, &tmB, &full[s], kb * sh.bk, n0);
        issued = kb + 1;
      }
      if (*abort_flag) {
        // let the copies already issued land before the CTA leaves
        for (int kb = issued - S < 0 ? 0 : issued - S; kb < issued; ++kb) {
          volatile int never = 0;
          mbar_wait(&full[kb % S], (uint32_t)(kb / S) & 1u, &never);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = E8 ? tc_idesc_e4m3(kTcBM, BN) : tc_idesc(kTcBM, BN);
      bool ok = true;
      for (int kb = 0; kb < nkb; ++kb) {
        const int s = kb % S;
        const uint32_t ph = (uint32_t)(kb / S) & 1u;
        if (!mbar_wait(&full[s], ph, abort_flag)) {
          atomicExch(&g_tc_err, 2);
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t b_addr = smem_u32(sB + s * B_TILE);
#pragma unroll
        for (int q = 0; q < P; ++q) {
          const uint32_t a_addr = smem_u32(sA + (s * P + q) * kTcATile);
#pragma unroll
          for (int kk = 0; kk < 4; ++kk) {   // 32 bytes of the 128-byte row per MMA
            const bool lo = E8 && q >= kTcE4m3Hi;   // the second accumulator's pieces
            const uint32_t acc = (kb | (lo ? q - kTcE4m3Hi : q) | kk) != 0 ? 1u : 0u;
            if (E8)
              umma_e4m3(tmem + (lo ? (uint32_t)BN : 0u), sw128_desc(a_addr + kk * 32),
                        sw128_desc(b_addr + kk * 32), idesc, acc);
            else
              umma_bf16(tmem, sw128_desc(a_addr + kk * 32), sw128_desc(b_addr + kk * 32), idesc, acc);
          }
        }
        umma_commit(&empty[s]);
      }
      if (ok) {
        umma_commit(accf);
      } else {
        // wait for the MMAs already issued before TMEM is released
        umma_commit(drain);
        volatile int never = 0;
        mbar_wait(drain, 0, &never);
      }
    }
    __syncwarp();
  } else {
    const int qd = warp & 3;   // TMEM lanes 32 qd .. 32 qd + 31
    const int m = m0 + 32 * qd + lane;
    // warp-uniform: tcgen05.ld is a warp-collective instruction
    const bool ok = __all_sync(0xffffffffu, mbar_wait(accf, 0, abort_flag) ? 1 : 0) != 0;
    tc_fence_after();
    if (ok) {
      const EpiRow er = epi_row<MODE>(sh, ep, m);
      double fsum = 0.0, dsum = 0.0;
      const uint32_t tbase = tmem + ((uint32_t)(32 * qd) << 16);
#pragma unroll 1
      for (int c = 0; c < BN; c += 16) {
        float v[16];
        tmem_ld_tile16<E8>(tbase + (uint32_t)c, BN, v);
        epi_chunk<MODE>(sh, ep, er, m, n0 + c, v, fsum, dsum);
      }
    } else {
      atomicExch(&g_tc_err, 3);
      *abort_flag = 1;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, TCOLS);
}

__host__ __device__ constexpr uint32_t tc_tmem_cols2(int BN) {
  return 2 * BN <= 32 ? 32u : 2 * BN <= 64 ? 64u : 2 * BN <= 128 ? 128u : 2 * BN <= 256 ? 256u : 512u;
}

// partial tile layout in skws: [slot][chunk of 16 columns][128 rows][16]
__device__ __forceinline__ float* sk_part(float* ws, int bn, int slot, int chunk, int row) {
  return ws + (((size_t)slot * (bn / 16) + chunk) * kTcBM + row) * 16;
}

// epilogue warps of the stream-K kernel: two per TMEM lane quadrant (each on half
// of the columns, a multiple of 64) when the tile is at least 128 wide
__host__ __device__ constexpr int sk_epi_warps(int BN) { return BN >= 128 ? 8 : 4; }
__host__ __device__ constexpr int sk_threads(int BN) { return 64 + 32 * sk_epi_warps(BN); }

template <int P, int BN, int MODE, int E8>
__global__ void __launch_bounds__(sk_threads(BN), 1)
    k_tcgemm_sk(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcShape sh,
                TcEpi ep) {
  constexpr int S = tc_stages(P, BN);
  constexpr uint32_t B_TILE = BN * 128;
  constexpr uint32_t STAGE_TX = P * kTcATile + B_TILE;
  constexpr int AW = (E8 ? 2 : 1) * BN;   // TMEM columns of one tile's accumulator(s)
  constexpr uint32_t TCOLS = tc_tmem_cols2(AW);
  static_assert(S >= 2, "at least two pipeline stages");
  static_assert(2 * AW <= 512, "two buffers of the tile's accumulators in TMEM");
  SkMap mp;
  sk_map(sh, ep, BN, gridDim.x, mp);
  const int c = blockIdx.x;
  const int64_t ib = sk_begin(mp, c), ie = sk_begin(mp, c + 1);
  if (mp.I == 0 || ib >= ie) return;   // nothing to do (uniform over the CTA)
  const int t_first = (int)(ib / mp.KB);

  extern __shared__ unsigned char smem_raw[];
  unsigned char* smem = (unsigned char*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  unsigned char* sA = smem;
  unsigned char* sB = smem + S * P * kTcATile;
  uint64_t* full = (uint64_t*)(sB + S * B_TILE);
  uint64_t* empty = full + S;
  uint64_t* tfull = empty + S;     // [2]: accumulator buffer ready for the epilogue
  uint64_t* tempty = tfull + 2;    // [2]: epilogue done with the buffer
  uint64_t* drain = tempty + 2;
  uint32_t* tmem_slot = (uint32_t*)(drain + 1);
  volatile int* abort_flag = (volatile int*)(tmem_slot + 1);

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) {
    for (int i = 0; i < S; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], sk_epi_warps(BN));   // one arrive per epilogue warp
    }
    mbar_init(drain, 1);
    *abort_flag = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) tmem_alloc(tmem_slot, TCOLS);
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  if (warp == 0) {
    if (lane == 0) {
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmA) : "memory");
      asm volatile("prefetch.tensormap [%0];" ::"l"((uint64_t)&tmB) : "memory");
      int64_t g = 0;
      bool ok = true;
      for (int64_t i = ib; i < ie && ok;) {
        const int t = (int)(i / mp.KB), kb0 = (int)(i % mp.KB);
        const int kb1 = (int)((ie - i) < (int64_t)(mp.KB - kb0) ? kb0 + (ie - i) : mp.KB);
        const int m0 = mp.act[t % mp.A] * kTcBM, n0 = (t / mp.A) * BN;
        for (int kb = kb0; kb < kb1; ++kb, ++g) {
          const int s = (int)(g % S);
          const uint32_t ph = (uint32_t)(g / S) & 1u;
          if (!mbar_wait(&empty[s], ph ^ 1u, abort_flag)) {
            atomicExch(&g_tc_err, 4);
            *abort_flag = 1;
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], STAGE_TX);
#pragma unroll
          for (int q = 0; q < P; ++q)
            tma_load_2d(sA + (s * P + q) * kTcATile, &tmA, &full[s], kb * sh.bk, q * sh.Mpad + m0);
          tma_load_2d(sB + s * B_TILE, &tmB, &full[s], kb * sh.bk, n0);
        }
        i += kb1 - kb0;
      }
      if (!ok) {
        for (int64_t gg = g - S < 0 ? 0 : g - S; gg < g; ++gg) {
          volatile int never = 0;
          mbar_wait(&full[gg % S], (uint32_t)(gg / S) & 1u, &never);
        }
      }
    }
    __syncwarp();
  } else if (warp == 1) {
    if (lane == 0) {
      constexpr uint32_t idesc = E8 ? tc_idesc_e4m3(kTcBM, BN) : tc_idesc(kTcBM, BN);
      int64_t g = 0;
      int sg = 0;
      bool ok = true;
      for (int64_t i = ib; i < ie && ok; ++sg) {
        const int kb0 = (int)(i % mp.KB);
        const int kb1 = (int)((ie - i) < (int64_t)(mp.KB - kb0) ? kb0 + (ie - i) : mp.KB);
        const int ab = sg & 1;
        if (!mbar_wait(&tempty[ab], ((uint32_t)(sg >> 1) & 1u) ^ 1u, abort_flag)) {
          atomicExch(&g_tc_err, 5);
          *abort_flag = 1;
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t dt = tmem + (uint32_t)(ab * AW);
        for (int kb = kb0; kb < kb1; ++kb, ++g) {
          const int s = (int)(g % S);
          const uint32_t ph = (uint32_t)(g / S) & 1u;
          if (!mbar_wait(&full[s], ph, abort_flag)) {
            atomicExch(&g_tc_err, 6);
            *abort_flag = 1;
            ok = false;
            break;
          }
          tc_fence_after();
          const uint32_t b_addr = smem_u32(sB + s * B_TILE);
#pragma unroll
          for (int q = 0; q < P; ++q) {
            const uint32_t a_addr = smem_u32(sA + (s * P + q) * kTcATile);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) {   // 32 bytes of the 128-byte row per MMA
              const bool lo = E8 && q >= kTcE4m3Hi;   // the second accumulator's pieces
              const uint32_t acc = ((kb - kb0) | (lo ? q - kTcE4m3Hi : q) | kk) != 0 ? 1u : 0u;
              if (E8)
                umma_e4m3(dt + (lo ? (uint32_t)BN : 0u), sw128_desc(a_addr + kk * 32),
                          sw128_desc(b_addr + kk * 32), idesc, acc);
              else
                umma_bf16(dt, sw128_desc(a_addr + kk * 32), sw128_desc(b_addr + kk * 32), idesc, acc);
            }
          }
          umma_commit(&empty[s]);
        }
        if (ok) umma_commit(&tfull[ab]);
        i += kb1 - kb0;
      }
      if (!ok) {
        umma_commit(drain);
        volatile int never = 0;
        mbar_wait(drain, 0, &never);
      }
    }
    __syncwarp();
  } else {
    constexpr int EW = sk_epi_warps(BN);
    constexpr int CW = BN * 4 / EW;      // columns per epilogue warp
    const int qd = warp & 3;             // TMEM lanes 32 qd .. 32 qd + 31
    const int c_lo = ((warp - 2) / 4) * CW;
    const int row = 32 * qd + lane;
    int sg = 0;
    for (int64_t i = ib; i < ie; ++sg) {
      const int t = (int)(i / mp.KB), kb0 = (int)(i % mp.KB);
      const int kb1 = (int)((ie - i) < (int64_t)(mp.KB - kb0) ? kb0 + (ie - i) : mp.KB);
      const int m0 = mp.act[t % mp.A] * kTcBM, n0 = (t / mp.A) * BN;
      const int ab = sg & 1;
      const bool ok = __all_sync(0xffffffffu, mbar_wait(&tfull[ab], (uint32_t)(sg >> 1) & 1u, abort_flag) ? 1 : 0) != 0;
      if (!ok) {
        atomicExch(&g_tc_err, 7);
        *abort_flag = 1;
        break;
      }
      tc_fence_after();
      const uint32_t tbase = tmem + ((uint32_t)(32 * qd) << 16) + (uint32_t)(ab * AW);
      if (kb0 == 0 && kb1 == mp.KB) {   // the whole tile: the epilogue
        const int m = m0 + row;
        const EpiRow er = epi_row<MODE>(sh, ep, m);
        double fsum = 0.0, dsum = 0.0;
#pragma unroll 1
        for (int cc = c_lo; cc < c_lo + CW; cc += 16) {
          float v[16];
          tmem_ld_tile16<E8>(tbase + (uint32_t)cc, BN, v);
          epi_chunk<MODE>(sh, ep, er, m, n0 + cc, v, fsum, dsum);
        }
      } else {                          // part of the tile: FP32 partial for the fix-up kernel
        const int slot = t == t_first ? 2 * c : 2 * c + 1;
#pragma unroll 1
        for (int cc = c_lo; cc < c_lo + CW; cc += 16) {
          float v[16];
          tmem_ld_tile16<E8>(tbase + (uint32_t)cc, BN, v);
          float4* dst = reinterpret_cast<float4*>(sk_part(ep.skws, BN, slot, cc / 16, row));
#pragma unroll
          for (int j = 0; j < 4; ++j) dst[j] = make_float4(v[4 * j], v[4 * j + 1], v[4 * j + 2], v[4 * j + 3]);
        }
      }
      tc_fence_before();
      __syncwarp();
      if (lane == 0) mbar_arrive(&tempty[ab]);
      i += kb1 - kb0;
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 1) tmem_dealloc(tmem, TCOLS);
}

// the tiles whose K blocks span several CTAs: one CTA per CTA boundary inside a
// tile (the first such boundary of each tile does its work) and per 64 columns
// (blockIdx.y; one loss-partial group), summing the partial tiles in CTA order
// and applying the epilogue
template <int BN, int MODE>
__global__ void __launch_bounds__(kTcBM * 4) k_tcgemm_fix(TcShape sh, TcEpi ep, int G) {
  __shared__ double sp[2][4][kTcBM];
  SkMap mp;
  sk_map(sh, ep, BN, G, mp);
  const int c = blockIdx.x + 1;
  if (mp.I == 0 || c >= G) return;
  const int64_t b = sk_begin(mp, c);
  if (b >= mp.I || b % mp.KB == 0) return;
  const int t = (int)(b / mp.KB);
  const int64_t t0 = (int64_t)t * mp.KB;
  if (sk_begin(mp, c - 1) > t0) return;   // an earlier boundary lies inside this tile
  const int clo = sk_owner(mp, t0), chi = sk_owner(mp, t0 + mp.KB - 1);
  const int m0 = mp.act[t % mp.A] * kTcBM, n0 = (t / mp.A) * BN;
  // one thread per row and 16-column chunk of the CTA's 64 columns
  const int row = (int)threadIdx.x % kTcBM, q4 = (int)threadIdx.x / kTcBM;
  const int m = m0 + row;
  const EpiRow er = epi_row<MODE>(sh, ep, m);
  double fsum = 0.0, dsum = 0.0;
  const int cc = (int)blockIdx.y * 64 + q4 * 16;
  if (cc < BN) {
    float v[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) v[j] = 0.0f;
    for (int q = clo; q <= chi; ++q) {
      if (sk_begin(mp, q) == sk_begin(mp, q + 1)) continue;   // an empty range (fewer iterations than CTAs)
      const int slot = sk_begin(mp, q) >= t0 ? 2 * q : 2 * q + 1;
      const float4* src = reinterpret_cast<const float4*>(sk_part(ep.skws, BN, slot, cc / 16, row));
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float4 x = src[j];
        v[4 * j] += x.x;
        v[4 * j + 1] += x.y;
        v[4 * j + 2] += x.z;
        v[4 * j + 3] += x.w;
      }
    }
    epi_chunk<MODE, false>(sh, ep, er, m, n0 + cc, v, fsum, dsum);
  }
  if (MODE == kTcAnchor) {
    // the 64-column group's loss partials: its four chunks added in column order,
    // as the product's own epilogue adds them
    sp[0][q4][row] = fsum;
    sp[1][q4][row] = dsum;
    __syncthreads();
    const int g0 = n0 + (int)blockIdx.y * 64;
    if (q4 == 0 && er.ok && g0 < sh.N) {
      double f = sp[0][0][row], dd = sp[1][0][row];
#pragma unroll
      for (int k = 1; k < 4; ++k) {
        f += sp[0][k][row];
        dd += sp[1][k][row];
      }
      double* pp = ep.part + 2 * ((int64_t)m * ep.npart + (g0 >> 6));
      pp[0] = f;
      pp[1] = dd;
    }
  }
}

// ------------------------------------------------------------------ host

static PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
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

// e8: E4M3 bytes (128 per swizzle row) instead of BF16 (64)
static bool make_map(void* out, const void* base, uint64_t inner, uint64_t rows, int64_t ld, uint32_t box_rows,
                     int e8, const char** why) {
  PFN_cuTensorMapEncodeTiled_v12000 fn = encode_fn();
  if (!fn) {
    *why = "cuTensorMapEncodeTiled is not available from the driver";
    return false;
  }
  cuuint64_t dims[2] = {inner, rows};
  cuuint64_t strides[1] = {(cuuint64_t)ld * (e8 ? 1 : 2)};
  cuuint32_t box[2] = {(cuuint32_t)(e8 ? 128 : kTcBK), box_rows};
  cuuint32_t estr[2] = {1, 1};
  CUresult r = fn((CUtensorMap*)out, e8 ? CU_TENSOR_MAP_DATA_TYPE_UINT8 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2,
                  const_cast<void*>(base), dims, strides,
                  box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                  CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    *why = "cuTensorMapEncodeTiled rejected the operand layout";
    return false;
  }
  return true;
}

bool tc_plan(TcPlan* plan, const void* A, int P, int M, int Mpad, int K, int64_t lda, const void* B, int N,
             int64_t ldb, int bn, const char** why, int e8) {
  plan->ok = 0;
  if (!e8 && (P < 1 || P > 3)) { *why = "BF16 pieces must be 1, 2 or 3"; return false; }
  if (e8 && P != kTcE4m3Pieces) { *why = "E4M3 products take KSC_E4M3_PIECES pieces"; return false; }
  if (e8 && bn > 128) { *why = "E4M3 tile width must be 64 or 128 (two accumulators)"; return false; }
  if (bn != 64 && bn != 128 && bn != 256) { *why = "tile width must be 64, 128 or 256"; return false; }
  if (M <= 0 || N <= 0 || K <= 0) { *why = "empty product"; return false; }
  if (Mpad % kTcBM != 0 || Mpad < M) { *why = "Mpad must be a multiple of 128 and >= M"; return false; }
  const int64_t es = e8 ? 1 : 2;
  if ((lda * es) % 16 != 0 || (ldb * es) % 16 != 0 || lda < K || ldb < K) {
    *why = "row strides must be >= K and multiples of 16 bytes";
    return false;
  }
  if (((uintptr_t)A % 16) != 0 || ((uintptr_t)B % 16) != 0) { *why = "operands must be 16-byte aligned"; return false; }
  if (!make_map(plan->tmA, A, (uint64_t)K, (uint64_t)P * Mpad, lda, kTcBM, e8, why)) return false;
  if (!make_map(plan->tmB, B, (uint64_t)K, (uint64_t)N, ldb, (uint32_t)bn, e8, why)) return false;
  plan->e8 = e8 ? 1 : 0;
  plan->P = P;
  plan->M = M;
  plan->Mpad = Mpad;
  plan->N = N;
  plan->K = K;
  plan->bn = bn;
  plan->ok = 1;
  plan->sk = 0;
  plan->grid = 0;
  return true;
}

bool tc_plan_stream_k(TcPlan* plan, int grid, const char** why) {
  if (!plan->ok) { *why = "plan the product first"; return false; }
  if (plan->M > kSkMaxMTiles * kTcBM) { *why = "stream-K schedule takes M <= 1024"; return false; }
  if (grid < 1) { *why = "grid must be >= 1"; return false; }
  plan->sk = 1;
  plan->grid = grid;
  return true;
}

size_t tc_skws_floats(int grid, int bn) { return (size_t)2 * grid * kTcBM * bn; }

template <int P, int BN, int MODE, int E8>
static void launch_one(const TcPlan& g, const TcEpi& e, cudaStream_t s) {
  constexpr int bytes = tc_smem_bytes(P, BN);
  TcShape sh{g.M, g.Mpad, g.N, g.K, E8 ? 128 : kTcBK};
  if (g.sk) {
    static bool attr_sk = false;
    if (!attr_sk) {
      cudaFuncSetAttribute(k_tcgemm_sk<P, BN, MODE, E8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
      attr_sk = true;
    }
    k_tcgemm_sk<P, BN, MODE, E8><<<g.grid, sk_threads(BN), bytes, s>>>(*(const CUtensorMap*)g.tmA,
                                                                  *(const CUtensorMap*)g.tmB, sh, e);
    if (g.grid > 1) k_tcgemm_fix<BN, MODE><<<dim3(g.grid - 1, (BN + 63) / 64), kTcBM * 4, 0, s>>>(sh, e, g.grid);
    return;
  }
  static bool attr = false;
  if (!attr) {
    cudaFuncSetAttribute(k_tcgemm<P, BN, MODE, E8>, cudaFuncAttributeMaxDynamicSharedMemorySize, bytes);
    attr = true;
  }
  dim3 grid((g.N + BN - 1) / BN, (g.M + kTcBM - 1) / kTcBM);
  k_tcgemm<P, BN, MODE, E8><<<grid, kTcThreads, bytes, s>>>(*(const CUtensorMap*)g.tmA,
                                                            *(const CUtensorMap*)g.tmB, sh, e);
}

template <int P, int MODE, int E8 = 0>
static void launch_bn(const TcPlan& g, const TcEpi& e, cudaStream_t s) {
  if (g.bn == 64) launch_one<P, 64, MODE, E8>(g, e, s);
  else if (g.bn == 128 || E8) launch_one<P, 128, MODE, E8>(g, e, s);   // E4M3 plans: bn <= 128
  else launch_one<P, E8 ? 128 : 256, MODE, E8>(g, e, s);
}

template <int MODE>
static void launch_p(const TcPlan& g, const TcEpi& e, cudaStream_t s) {
  if (g.e8) launch_bn<kTcE4m3Pieces, MODE, 1>(g, e, s);
  else if (g.P == 1) launch_bn<1, MODE>(g, e, s);
  else if (g.P == 2) launch_bn<2, MODE>(g, e, s);
  else launch_bn<3, MODE>(g, e, s);
}

void tc_launch(const TcPlan& plan, const TcEpi& epi, int mode, cudaStream_t s) {
  if (mode == kTcAnchor) launch_p<kTcAnchor>(plan, epi, s);
  else if (mode == kTcAdd) launch_p<kTcAdd>(plan, epi, s);
  else launch_p<kTcStore>(plan, epi, s);
}

int* tc_error_word() {
  void* p = nullptr;
  cudaGetSymbolAddress(&p, g_tc_err);
  return (int*)p;
}

void tc_clear_error(cudaStream_t s) { cudaMemsetAsync(tc_error_word(), 0, sizeof(int), s); }

}  // namespace ksc
