// ksc_common.cuh -- device building blocks shared by the kernels of the library:
// warp/block reductions and scans, key bit maps, the block-wide MSD radix select
// and the block bitonic sort used by the segmented prox (Alg. 1 / Lemma 3.3).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp8.h>
#include <stdint.h>

namespace ksc {

constexpr int kWarp = 32;

// ----------------------------------------------------------------- scalars

__device__ __forceinline__ double to_d(double x) { return x; }
__device__ __forceinline__ double to_d(float x) { return (double)x; }
__device__ __forceinline__ double to_d(__nv_bfloat16 x) { return (double)__bfloat162float(x); }
__device__ __forceinline__ float to_f(float x) { return x; }
__device__ __forceinline__ float to_f(__nv_bfloat16 x) { return __bfloat162float(x); }
__device__ __forceinline__ float to_f(double x) { return (float)x; }

// ------------------------------------------------------- warp/block reduce

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_max(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}
template <typename T>
__device__ __forceinline__ T warp_min(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v = min(v, __shfl_xor_sync(0xffffffffu, v, o));
  return v;
}

// Block-wide reductions; `red` is a shared scratch of >= 32 elements of T.  All
// threads receive the result.  Deterministic (fixed tree order).
template <typename T, int BLOCK>
__device__ __forceinline__ T block_sum(T v, T* red) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_sum(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T t = (threadIdx.x < BLOCK / 32) ? red[threadIdx.x] : T(0);
  if (w == 0) t = warp_sum(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  T r = red[0];
  __syncthreads();
  return r;
}
template <typename T, int BLOCK>
__device__ __forceinline__ T block_max(T v, T* red, T lowest) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_max(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T t = (threadIdx.x < BLOCK / 32) ? red[threadIdx.x] : lowest;
  if (w == 0) t = warp_max(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  T r = red[0];
  __syncthreads();
  return r;
}
template <typename T, int BLOCK>
__device__ __forceinline__ T block_min(T v, T* red, T highest) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  v = warp_min(v);
  __syncthreads();
  if (lane == 0) red[w] = v;
  __syncthreads();
  T t = (threadIdx.x < BLOCK / 32) ? red[threadIdx.x] : highest;
  if (w == 0) t = warp_min(t);
  if (threadIdx.x == 0) red[0] = t;
  __syncthreads();
  T r = red[0];
  __syncthreads();
  return r;
}

// Exclusive prefix sum over the block in thread order (warp shuffles + one
// shared pass over warp totals).  `red` holds >= 33 elements.  Returns this
// thread's exclusive prefix; *total receives the block total.
template <typename T, int BLOCK>
__device__ __forceinline__ T block_exclusive_scan(T v, T* red, T* total) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  T incl = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    T n = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += n;
  }
  __syncthreads();
  if (lane == 31) red[w] = incl;
  __syncthreads();
  if (w == 0) {
    T t = (lane < BLOCK / 32) ? red[lane] : T(0);
    T ti = t;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      T n = __shfl_up_sync(0xffffffffu, ti, o);
      if (lane >= o) ti += n;
    }
    red[lane] = ti - t;            // exclusive warp offsets
    if (lane == 31) red[32] = ti;  // block total
  }
  __syncthreads();
  T r = red[w] + incl - v;
  *total = red[32];
  __syncthreads();
  return r;
}

// --------------------------------------------------------------- key bits
// Non-negative floating keys compare like their bit patterns as unsigned ints.

template <typename T> struct Bits;
template <> struct Bits<float> {
  using U = uint32_t;
  static __device__ __forceinline__ U of(float x) { return __float_as_uint(x); }
  static __device__ __forceinline__ float val(U u) { return __uint_as_float(u); }
};
template <> struct Bits<double> {
  using U = unsigned long long;
  static __device__ __forceinline__ U of(double x) { return (U)__double_as_longlong(x); }
  static __device__ __forceinline__ double val(U u) { return __longlong_as_double((long long)u); }
};

// ---------------------------------------------------------- radix select
// Block-wide selection of the q-th largest of m non-negative keys (1 <= q <= m)
// by most-significant-digit radix passes of 11 bits over the key bits.
// `load(i)` returns the key bits of element i.  hist: shared, >= 2048 uint32.
// sh: shared int scratch >= 40.  Result: thr = bits of the q-th largest key,
// gt = #keys > thr, eq = #keys == thr.

template <typename U>
struct SelectResult {
  U thr;
  int gt;
  int eq;
};

// first (optional): the histogram of the first digit (key >> (BITS - 11)), already
// counted elsewhere -- it replaces the first pass over the keys.
template <typename U, int BLOCK, typename Load>
__device__ SelectResult<U> block_select(int m, int q, Load load, unsigned* hist, int* sh,
                                        const unsigned* first = nullptr) {
  constexpr int BITS = (int)sizeof(U) * 8;
  constexpr int DIG = 11;
  constexpr int NB = 1 << DIG;
  constexpr int PER = NB / BLOCK;   // bins per thread
  static_assert(NB % BLOCK == 0 && PER >= 1, "block_select: 2048 bins over the block");
  U prefix = 0;
  int q_rem = q, gt = 0, eq = 0;
  int hi = BITS;
  while (hi > 0) {
    const int w = hi < DIG ? hi : DIG;
    const int lo = hi - w;
    const U himask = (hi >= BITS) ? (U)0 : (~(U)0 << hi);
    const bool given = (hi == BITS) && first != nullptr;
    for (int b = threadIdx.x; b < NB; b += BLOCK) hist[b] = given ? __ldcg(&first[b]) : 0u;
    __syncthreads();
    // warp-uniform loop; lanes with the same bin are aggregated (__match_any_sync)
    // so that runs of equal keys (e.g. zeros) do not serialise on one counter.  The
    // next key is loaded before this one is binned: its global loads overlap the
    // match and the atomic instead of waiting behind them
    const int mm = given ? 0 : m;
    U kn = ((int)threadIdx.x < mm) ? load((int)threadIdx.x) : (U)0;
    for (int base = 0; base < mm; base += BLOCK) {
      const int i = base + (int)threadIdx.x;
      const U k = kn;
      if (i + BLOCK < mm) kn = load(i + BLOCK);
      int bin = -1;
      if (i < mm && (k & himask) == (prefix & himask)) bin = (int)((k >> lo) & (U)((1u << w) - 1u));
      const unsigned peers = __match_any_sync(0xffffffffu, bin);
      if (bin >= 0 && (threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1))
        atomicAdd(&hist[bin], (unsigned)__popc(peers));
    }
    __syncthreads();
    // thread t owns bins NB-1-PER*t down to NB-PER*(t+1): thread order is
    // descending bin order, so an exclusive scan gives the count above a bin.
    const int btop = NB - 1 - PER * (int)threadIdx.x;
    int cnt[PER];
    int own = 0;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      cnt[k] = (int)hist[btop - k];
      own += cnt[k];
    }
    int tot;
    int run = block_exclusive_scan<int, BLOCK>(own, sh, &tot);
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      if (run < q_rem && q_rem <= run + cnt[k]) { sh[36] = btop - k; sh[37] = run; sh[38] = cnt[k]; }
      run += cnt[k];
    }
    __syncthreads();
    const int bin = sh[36], cab = sh[37];
    eq = sh[38];
    __syncthreads();
    prefix |= ((U)bin) << lo;
    gt += cab;
    q_rem -= cab;
    hi = lo;
    if (hi > DIG && eq <= 32) {
      // at most 32 keys share the prefix and two or more passes remain: gather
      // them (hist is free until the next pass) and rank them directly.  The
      // q_rem-th largest key t of the bin has #{> t} < q_rem <= #{>= t}.
      U* keys = reinterpret_cast<U*>(hist + 4);   // 32 keys, then the result at keys[32]
      if (threadIdx.x == 0) hist[0] = 0u;
      __syncthreads();
      const U mask = ~(U)0 << hi;
      for (int i = threadIdx.x; i < m; i += BLOCK) {
        const U k = load(i);
        if ((k & mask) == prefix) {
          const unsigned pos = atomicAdd(&hist[0], 1u);
          if (pos < 32u) keys[pos] = k;
        }
      }
      __syncthreads();
      if (threadIdx.x < (unsigned)eq) {
        const U kt = keys[threadIdx.x];
        int ngt = 0, neq = 0;
        for (int s = 0; s < eq; ++s) {
          const U ks = keys[s];
          ngt += ks > kt;
          neq += ks == kt;
        }
        if (ngt < q_rem && q_rem <= ngt + neq) {   // equal keys write equal values
          keys[32] = kt;
          hist[1] = (unsigned)ngt;
          hist[2] = (unsigned)neq;
        }
      }
      __syncthreads();
      prefix = keys[32];
      gt += (int)hist[1];
      eq = (int)hist[2];
      __syncthreads();
      break;
    }
  }
  return SelectResult<U>{prefix, gt, eq};
}

// ---------------------------------------------------------- bitonic sort
// In-place descending sort of N (power of two) values in shared memory.  Sorting
// non-negative doubles as their 64-bit patterns gives the same order with integer
// compares (sort_desc_nonneg), which matters where FP64 issue is slow.
template <typename T, int BLOCK>
__device__ void block_bitonic_sort_desc(T* s, int N) {
  for (int size = 2; size <= N; size <<= 1) {
    for (int stride = size >> 1; stride > 0; stride >>= 1) {
      for (int i = threadIdx.x; i < (N >> 1); i += BLOCK) {
        const int lo = 2 * i - (i & (stride - 1));
        const int hi = lo + stride;
        const bool desc = ((lo & size) == 0);
        T a = s[lo], b = s[hi];
        if ((a < b) == desc) { s[lo] = b; s[hi] = a; }
      }
      __syncthreads();
    }
  }
}

// descending sort of N non-negative doubles (padding: +0.0)
template <int BLOCK>
__device__ __forceinline__ void sort_desc_nonneg(double* s, int N) {
  block_bitonic_sort_desc<unsigned long long, BLOCK>(reinterpret_cast<unsigned long long*>(s), N);
}

// the bit pattern of a non-negative double: ordered like the value
__device__ __forceinline__ unsigned long long nnbits(double x) { return (unsigned long long)__double_as_longlong(x); }

// ---------------------------------------------------------- double-float products

// X entries read in their storage type, as A
template <typename A> __device__ __forceinline__ A xval(float x) { return (A)x; }
template <typename A> __device__ __forceinline__ A xval(double x) { return (A)x; }
template <typename A> __device__ __forceinline__ A xval(__nv_bfloat16 x) { return (A)__bfloat162float(x); }
// FP8 e4m3 values are exact in half and float
template <typename A> __device__ __forceinline__ A xval(__nv_fp8_e4m3 x) { return (A)(float)x; }
template <typename TX> __host__ __device__ constexpr bool is_fp8() { return false; }
template <> __host__ __device__ constexpr bool is_fp8<__nv_fp8_e4m3>() { return true; }
// one element of X, streamed (evict-first)
template <typename TX> __device__ __forceinline__ TX ldcs_x(const TX* p) { return __ldcs(p); }
template <> __device__ __forceinline__ __nv_fp8_e4m3 ldcs_x(const __nv_fp8_e4m3* p) {
  __nv_fp8_e4m3 v;
  v.__x = (__nv_fp8_storage_t)__ldcs(reinterpret_cast<const unsigned char*>(p));
  return v;
}

// Double-float accumulation of x * (rh + rl) into hi + lo.  x*rh = p + e exactly
// (e by fma); hi + p = s + err exactly (Knuth's TwoSum); lo collects err, e and
// x*rl, whose own rounding is ~u^2 of the sum.  The result hi + lo (taken in
// double) is accurate to ~1e-13 relative.  __fmul_rn/__fadd_rn/__fsub_rn are never
// contracted into an FMA, which would break the exactness of p and of TwoSum.
__device__ __forceinline__ void df_add(float& hi, float& lo, float x, float rh, float rl) {
  const float p = __fmul_rn(x, rh);
  const float e = fmaf(x, rh, -p);
  const float s = __fadd_rn(hi, p);
  const float bp = __fsub_rn(s, hi);
  const float err = __fadd_rn(__fsub_rn(hi, __fsub_rn(s, bp)), __fsub_rn(p, bp));
  hi = s;
  lo = __fadd_rn(lo, __fadd_rn(err, fmaf(x, rl, e)));
}

// ---------------------------------------------------------- Huber

__device__ __forceinline__ double huber(double a, double M) {
  double t = fabs(a);
  return t <= M ? 0.5 * t * t : M * t - 0.5 * M * M;
}

}  // namespace ksc
