// k_prox_grid.cu -- the prox of one FISTA step (the proximal step of Algorithm 3) spread over
// the GPU, and the Lanczos iteration that gives L.
//
// prox_{rho^-1 g}(w) = w - rho^-1 prox_{rho g*}(rho w) (Moreau, Sec. 3.3).  With the
// Huber weight on the top k' positions only, PAVA (Alg. 1 + 4) pools at most one
// block across positions k'/k'+1: the result is fixed by the top-k' set and one
// threshold theta, the root of the monotone piecewise-linear
//   Phi(t) = sum_top (t + min(rho t, M) - a)_+ - sum_tail (a - t)_+,   a = |w|,
// top coordinates get |b| = min(M, rho a/(1+rho), a - theta), the rest max(0, a - theta).
//
//  gradient pass epilogue (k_matvec.cu): w (FP64), 32-bit selection keys = float
//      bits of |w| (monotone: fl(a) > fl(b) implies a > b), first radix digit
//      histogram -- fused into the CTA that finishes each column strip.
//  k_prox_select (2 CTAs): the candidates predicted from the previous step (or
//      integer radix passes) give the top-k' set; ties of the float key are broken
//      exactly on |w| then index (Alg. 1 order); the top-Q candidates are sorted as
//      64-bit patterns of |w| (bitonic, warp blocks in registers) and one warp's
//      k-ary search over the breakpoints {a_j, theta_t, M/rho} of Phi (integer
//      compares of their bit patterns) finds the linear piece holding the root.
//      Q grows if the pooled block reaches below the candidates; beyond the
//      shared-memory capacity a bracketed Newton iteration over full passes is
//      used.  CTA 1: the in-loop dual term G*(X^T zeta_gamma) (Lemma 3.1 on the
//      node) from keys of |grad|, with S1 read from its index list.
//  k_prox_apply (grid): b, its float split for the dense forward pass, the
//      nonzero list (one compaction segment per CTA, ascending index), sum |b_F|,
//      and in the last CTA g(b) by the water-filling of Algorithm 2.
#include "ksc_common.cuh"
#include "ksc_launch.h"
#include "ksc_prox.cuh"
#include "ksc_state.cuh"

namespace ksc {

constexpr int kSelBlock = 1024;

struct SelSmem {
  unsigned hist[2048];
  int sh[64];
  double red[64];
  unsigned long long cand[kProxCap];   // bit patterns of non-negative doubles
  double pref[kProxCap + 1];
  double tb[kProxCap];
  int cidx[kProxCap];
  unsigned long long tkey[kProxCap];   // the top set (and its ties), sorted in Alg. 1 order
  int tidx[kProxCap];
  double rsum[2];
  int rcnt[2 + 16];
  double rt[2];                  // root search: result, and the scalars below
  unsigned long long rtb[2];     // bit patterns of the point t and of t + min(rho t, M)
  int rflag[2];                  // done, pooled count
  double cs[2];                  // per-call scalars computed once: rho / (1 + rho), 1 / (2 lambda2)
  double root[2];
  int flag[2];
};

__device__ __forceinline__ double dval(unsigned long long b) { return __longlong_as_double((long long)b); }
__device__ __forceinline__ unsigned long long dbits(double x) { return (unsigned long long)__double_as_longlong(x); }

// Bitonic sort into descending order: PAIRS ranks by key, ties by ascending index
// (Alg. 1's order); otherwise keys alone (non-negative doubles compare like their
// bits).  N is a power of two <= kProxCap.  With kSelBlock threads, each of
// W = min(N/32, 32) warps holds a block of B = N/W consecutive elements in
// registers (R = B/32 per lane: element base + 32 r + lane); the merge stages
// whose stride is below B run there (strides >= 32 inside a thread, smaller ones
// by warp shuffles), the wider ones through shared memory.
__device__ __forceinline__ bool rank_gt(unsigned long long ka, int ia, unsigned long long kb, int ib, bool pairs) {
  return ka > kb || (pairs && ka == kb && ia < ib);
}

template <bool PAIRS>
__device__ void smem_merge_stage(unsigned long long* s, int* ix, int N, int size, int stride) {
  for (int i = threadIdx.x; i < (N >> 1); i += kSelBlock) {
    const int lo = 2 * i - (i & (stride - 1));
    const int hi = lo + stride;
    const bool desc = ((lo & size) == 0);
    const unsigned long long a = s[lo], b = s[hi];
    const int ia = PAIRS ? ix[lo] : 0, ib = PAIRS ? ix[hi] : 0;
    if (rank_gt(a, ia, b, ib, PAIRS) != desc) {
      s[lo] = b;
      s[hi] = a;
      if (PAIRS) {
        ix[lo] = ib;
        ix[hi] = ia;
      }
    }
  }
  __syncthreads();
}

template <bool PAIRS>
__device__ void bitonic_desc(unsigned long long* s, int* ix, int N) {
  if (N < 64) {   // a single small block: shared memory only
    for (int size = 2; size <= N; size <<= 1)
      for (int stride = size >> 1; stride > 0; stride >>= 1) smem_merge_stage<PAIRS>(s, ix, N, size, stride);
    return;
  }
  const int W = N / 32 < 32 ? N / 32 : 32;
  const int R = N / (32 * W);   // 1, 2 or 4
  const int B = 32 * R;
  const int warp = (int)threadIdx.x >> 5, lane = (int)threadIdx.x & 31;
  const bool act = warp < W;
  const int base = warp * B;
  unsigned long long k[4] = {0ull, 0ull, 0ull, 0ull};
  int id[4] = {0, 0, 0, 0};
  auto load = [&]() {
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (r < R) {
        k[r] = s[base + 32 * r + lane];
        if (PAIRS) id[r] = ix[base + 32 * r + lane];
      }
  };
  auto store = [&]() {
#pragma unroll
    for (int r = 0; r < 4; ++r)
      if (r < R) {
        s[base + 32 * r + lane] = k[r];
        if (PAIRS) ix[base + 32 * r + lane] = id[r];
      }
  };
  // in-thread compare-exchange of registers ra < rb (elements e and e + 32 (rb - ra))
  auto cx = [&](int ra, int rb, int size) {
    const int e = base + 32 * ra + lane;
    const bool desc = ((e & size) == 0);
    if (rank_gt(k[ra], id[ra], k[rb], id[rb], PAIRS) != desc) {
      const unsigned long long t = k[ra];
      k[ra] = k[rb];
      k[rb] = t;
      const int u = id[ra];
      id[ra] = id[rb];
      id[rb] = u;
    }
  };
  auto reg_stages = [&](int size, int stride_hi) {
    for (int stride = stride_hi; stride > 0; stride >>= 1) {
      if (stride >= 64) {          // R = 4: registers 0-2, 1-3
        cx(0, 2, size);
        cx(1, 3, size);
      } else if (stride == 32) {   // registers 0-1 (and 2-3)
        cx(0, 1, size);
        if (R == 4) cx(2, 3, size);
      } else {
        const bool is_lo = (lane & stride) == 0;
#pragma unroll
        for (int r = 0; r < 4; ++r)
          if (r < R) {
            const unsigned long long b = __shfl_xor_sync(0xffffffffu, k[r], stride);
            const int ib = PAIRS ? __shfl_xor_sync(0xffffffffu, id[r], stride) : 0;
            const int e = base + 32 * r + lane;
            const bool desc = ((e & size) == 0);
            const bool a_first = rank_gt(k[r], id[r], b, ib, PAIRS);
            if ((is_lo == desc) != a_first) {
              k[r] = b;
              id[r] = ib;
            }
          }
      }
    }
  };
  if (act) {
    load();
    for (int size = 2; size <= B; size <<= 1) reg_stages(size, size >> 1);
    store();
  }
  __syncthreads();
  for (int size = 2 * B; size <= N; size <<= 1) {
    for (int stride = size >> 1; stride >= B; stride >>= 1) smem_merge_stage<PAIRS>(s, ix, N, size, stride);
    if (act) {
      load();
      reg_stages(size, B >> 1);
      store();
    }
    __syncthreads();
  }
}

__device__ void sort_u64_desc(unsigned long long* s, int N) { bitonic_desc<false>(s, nullptr, N); }

// descending by value, ascending by index
__device__ void sort_pairs_desc(unsigned long long* s, int* ix, int N) { bitonic_desc<true>(s, ix, N); }

// prefix sums pref[0..C] of the candidate values
__device__ void prefix_values(SelSmem& sm, int C) {
  const int per = (C + kSelBlock - 1) / kSelBlock;
  const int s0 = threadIdx.x * per;
  double loc = 0.0;
  for (int j = 0; j < per; ++j) if (s0 + j < C) loc += dval(sm.cand[s0 + j]);
  double tot;
  double ex = block_exclusive_scan<double, kSelBlock>(loc, sm.red, &tot);
  for (int j = 0; j < per; ++j) if (s0 + j < C) { sm.pref[s0 + j] = ex; ex += dval(sm.cand[s0 + j]); }
  if (threadIdx.x == 0) sm.pref[C] = tot;
  __syncthreads();
}

// Phi on the sorted candidates (valid for t >= the smallest candidate); also the
// active sets of the piece that holds t.
struct Piece {
  double phi, SA, SB;
  int nA, nB;
};

__device__ Piece phi_at(const SelSmem& sm, double th, int q, int C, double rho, double M) {
  // th, theta_t and a_j are non-negative doubles: their bit patterns compare alike
  // (integer compares; FP64 issues at 1/64 of the FP32 rate)
  const unsigned long long tk = dbits(th);
  int lo = 0, hi = q;   // first top t with theta_t < th (theta_t non-increasing)
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (dbits(sm.tb[mid]) < tk) hi = mid; else lo = mid + 1;
  }
  const int t0 = lo;
  lo = q; hi = C;       // first tail j with a_j <= th
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (sm.cand[mid] <= tk) hi = mid; else lo = mid + 1;
  }
  Piece e;
  e.nA = q - t0;
  e.SA = sm.pref[q] - sm.pref[t0];
  e.nB = lo - q;
  e.SB = sm.pref[lo] - sm.pref[q];
  e.phi = (double)e.nA * (th + fmin(rho * th, M)) - e.SA - (e.SB - (double)e.nB * th);
  return e;
}

// First index in [lo, hi) where a predicate that is monotone in the index (false
// ... false true ... true) holds, hi if none: one warp, 32 probes per round.
template <class Pred>
__device__ int warp_first_true(int lo, int hi, Pred pred) {
  const int lane = (int)threadIdx.x & 31;
  while (lo < hi) {
    const int step = (hi - lo + 31) / 32;
    const int j = lo + lane * step;
    const unsigned m = __ballot_sync(0xffffffffu, j < hi && pred(j));
    if (m == 0u) {
      const int last = (hi - 1 - lo) / step < 31 ? (hi - 1 - lo) / step : 31;   // the last probe below hi
      lo += last * step + 1;
    } else {
      const int f = __ffs(m) - 1;
      hi = lo + f * step;                    // the first true probe
      if (f > 0) lo += (f - 1) * step + 1;   // past the last false one
    }
  }
  return lo;
}

// Root of Phi on [floorv, inf) by search over the two sorted breakpoint
// sequences (one warp: every lane returns the same).  Returns false when
// Phi(floorv) > 0 and floorv is a true floor (the pooled block reaches below the
// candidates).
__device__ bool root_search(const SelSmem& sm, int q, int C, double floorv, bool floor_is_zero,
                            double rho, double M, double* theta) {
  if (!floor_is_zero && phi_at(sm, floorv, q, C, rho, M).phi > 0.0) return false;
  double lo = floorv, hi = INFINITY;
  // tail breakpoints a_j, j in [q, C): Phi(a_j) is non-increasing in j
  int a = warp_first_true(q, C, [&](int j) { return phi_at(sm, dval(sm.cand[j]), q, C, rho, M).phi <= 0.0; });
  if (a < C) lo = fmax(lo, dval(sm.cand[a]));
  if (a > q) hi = fmin(hi, dval(sm.cand[a - 1]));
  // top breakpoints theta_t, t in [0, q): non-increasing in t
  a = warp_first_true(0, q, [&](int t) { return phi_at(sm, sm.tb[t], q, C, rho, M).phi <= 0.0; });
  if (a < q && sm.tb[a] >= floorv) lo = fmax(lo, sm.tb[a]);
  if (a > 0) hi = fmin(hi, sm.tb[a - 1]);
  const double thM = M / rho;
  if (thM >= floorv) {
    const double v = phi_at(sm, thM, q, C, rho, M).phi;
    if (v <= 0.0) lo = fmax(lo, thM);
    if (v >= 0.0) hi = fmin(hi, thM);
  }
  double th;
  if (!(hi > lo)) {
    th = isinf(hi) ? lo : hi;
  } else {
    const double mid = 0.5 * (lo + hi);
    const Piece e = phi_at(sm, mid, q, C, rho, M);
    th = (rho * mid < M) ? (e.SA + e.SB) / ((double)e.nA * (1.0 + rho) + (double)e.nB)
                         : (e.SA + e.SB - (double)e.nA * M) / (double)(e.nA + e.nB);
    th = fmin(fmax(th, lo), hi);
  }
  *theta = th;
  return true;
}

// the magnitude a selection key stands for: |w_i| on the free set; key 0 marks a
// coordinate off the free set (or one below the float range), taken as 0
__device__ __forceinline__ double key_value(unsigned kk, const double* w, int i) {
  return kk == 0u ? 0.0 : fabs(__ldcg(&w[i]));
}

// membership of coordinate i in the top set (exact Alg. 1 order)
__device__ __forceinline__ bool in_top(unsigned kk, double a, int i, unsigned thr, int q,
                                       double bnd_a, int bnd_i) {
  if (q <= 0) return false;
  if (kk != thr) return kk > thr;
  return bnd_a < 0.0 || a > bnd_a || (a == bnd_a && i <= bnd_i);
}

// Two counts and two FP64 sums over the block.  FP64 issues at 1/64 of the FP32
// rate here, so every thread's sums go through shared memory to one warp (each
// value added once) instead of a tree in every thread; the order is fixed.
__device__ __forceinline__ void block_reduce_cs(int& na, double& sa, int& nb, double& sb, SelSmem& sm) {
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  na = __reduce_add_sync(0xffffffffu, na);
  nb = __reduce_add_sync(0xffffffffu, nb);
  sm.pref[threadIdx.x] = sa;
  sm.pref[kSelBlock + threadIdx.x] = sb;
  if (lane == 0) {
    sm.sh[w] = na;
    sm.sh[32 + w] = nb;
  }
  __syncthreads();
  if (w == 0) {
    double a = 0.0, b = 0.0;
    for (int v = 0; v < kSelBlock / 32; ++v) {
      a += sm.pref[32 * v + lane];
      b += sm.pref[kSelBlock + 32 * v + lane];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      a += __shfl_xor_sync(0xffffffffu, a, o);
      b += __shfl_xor_sync(0xffffffffu, b, o);
    }
    const int ca = __reduce_add_sync(0xffffffffu, lane < kSelBlock / 32 ? sm.sh[lane] : 0);
    const int cb = __reduce_add_sync(0xffffffffu, lane < kSelBlock / 32 ? sm.sh[32 + lane] : 0);
    if (lane == 0) {
      sm.rsum[0] = a;
      sm.rsum[1] = b;
      sm.rcnt[0] = ca;
      sm.rcnt[1] = cb;
    }
  }
  __syncthreads();
  sa = sm.rsum[0];
  sb = sm.rsum[1];
  na = sm.rcnt[0];
  nb = sm.rcnt[1];
  __syncthreads();
}

// Root of Phi on [floorv, top_max] over the unsorted candidates (the top set is
// {key > bk} + {key == bk, index <= bi}, Alg. 1 order).  Every thread evaluates
// the counts and sums of Phi's linear piece at the broadcast point -- top members
// active where a < t + min(rho t, M), tail members where a > t, by integer
// compares of bit patterns -- together with the nearest keys on either side of t
// (tail) and of t + min(rho t, M) (top), which bound that piece; thread 0 alone
// does the scalar FP64 work (FP64 issues at 1/64 of the FP32 rate): the Newton
// point of the piece is the root when no key separates it from t (no second
// pass to confirm it), bisection when it leaves the bracket, warm-started at the
// previous step's threshold.  The first pass also evaluates Phi at the floor.
// false when Phi(floorv) > 0 (the pooled block reaches below the candidates).
__device__ bool root_unsorted(SelSmem& sm, int cc, unsigned long long bk, int bi, double floorv, bool all,
                              double top_max, double t0, double rho, double M, double* root, int* pooled) {
  using ULL = unsigned long long;
  __shared__ int s_cnt[4][32];
  __shared__ ULL s_x[4][32];
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  constexpr int NW = kSelBlock / 32;
  // thread 0's state
  double lo = floorv, hi = top_max, t = 0.0;
  if (threadIdx.x == 0) {
    t = (t0 > lo && t0 < hi) ? t0 : 0.5 * (lo + hi);
    sm.rtb[0] = dbits(t);
    sm.rtb[1] = dbits(t + fmin(rho * t, M));
    sm.rflag[0] = 0;
  }
  const ULL fb = dbits(floorv), hfb = dbits(floorv + fmin(rho * floorv, M));
  __syncthreads();
  for (int it = 0; it < 200; ++it) {
    const bool first = it == 0 && !all;   // Phi at the floor too
    const ULL tb = sm.rtb[0], hb = sm.rtb[1];
    int c[4] = {0, 0, 0, 0};              // nA, nB at t; nA, nB at the floor
    double sum[4] = {0.0, 0.0, 0.0, 0.0};
    ULL tl = 0ull, tg = ~0ull, al = 0ull, ag = ~0ull;
    for (int j = threadIdx.x; j < cc; j += kSelBlock) {
      const ULL k = sm.cand[j];
      const double v = dval(k);
      const bool top = k > bk || (k == bk && sm.cidx[j] <= bi);
      if (top) {
        if (k < hb) { c[0] += 1; sum[0] += v; al = k > al ? k : al; }
        else ag = k < ag ? k : ag;
        if (first && k < hfb) { c[2] += 1; sum[2] += v; }
      } else {
        if (k > tb) { c[1] += 1; sum[1] += v; tg = k < tg ? k : tg; }
        else tl = k > tl ? k : tl;
        if (first && k > fb) { c[3] += 1; sum[3] += v; }
      }
    }
    // block reduction: counts and extremes per warp, the FP64 sums through shared
    // memory to one warp (fixed order)
#pragma unroll
    for (int i = 0; i < 4; ++i) c[i] = __reduce_add_sync(0xffffffffu, c[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      ULL v;
      v = __shfl_xor_sync(0xffffffffu, tl, o); tl = v > tl ? v : tl;
      v = __shfl_xor_sync(0xffffffffu, al, o); al = v > al ? v : al;
      v = __shfl_xor_sync(0xffffffffu, tg, o); tg = v < tg ? v : tg;
      v = __shfl_xor_sync(0xffffffffu, ag, o); ag = v < ag ? v : ag;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) sm.pref[i * kSelBlock + threadIdx.x] = sum[i];
    if (lane == 0) {
#pragma unroll
      for (int i = 0; i < 4; ++i) s_cnt[i][wid] = c[i];
      s_x[0][wid] = tl;
      s_x[1][wid] = al;
      s_x[2][wid] = tg;
      s_x[3][wid] = ag;
    }
    __syncthreads();
    if (wid == 0) {
      double a[4] = {0.0, 0.0, 0.0, 0.0};
      for (int v = 0; v < NW; ++v)
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] += sm.pref[i * kSelBlock + 32 * v + lane];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1)
#pragma unroll
        for (int i = 0; i < 4; ++i) a[i] += __shfl_xor_sync(0xffffffffu, a[i], o);
      int n[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) n[i] = __reduce_add_sync(0xffffffffu, lane < NW ? s_cnt[i][lane] : 0);
      ULL x0 = lane < NW ? s_x[0][lane] : 0ull, x1 = lane < NW ? s_x[1][lane] : 0ull;
      ULL x2 = lane < NW ? s_x[2][lane] : ~0ull, x3 = lane < NW ? s_x[3][lane] : ~0ull;
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        ULL v;
        v = __shfl_xor_sync(0xffffffffu, x0, o); x0 = v > x0 ? v : x0;
        v = __shfl_xor_sync(0xffffffffu, x1, o); x1 = v > x1 ? v : x1;
        v = __shfl_xor_sync(0xffffffffu, x2, o); x2 = v < x2 ? v : x2;
        v = __shfl_xor_sync(0xffffffffu, x3, o); x3 = v < x3 ? v : x3;
      }
      if (lane == 0) {
        // thread 0: the scalar step
        int done = 0;
        double res = t;
        if (first) {
          const double hf = dval(hfb);
          const double phif = (double)n[2] * hf - a[2] - (a[3] - (double)n[3] * floorv);
          if (phif > 0.0) done = 2;               // the root lies below the candidates
          else if (phif == 0.0) { done = 1; res = floorv; }
        }
        if (!done) {
          const double phi = (double)n[0] * dval(hb) - a[0] - (a[1] - (double)n[1] * t);
          if (phi == 0.0) {
            done = 1;
          } else {
            if (phi < 0.0) lo = t; else hi = t;
            const bool capped = rho * t >= M;
            const double den = capped ? (double)(n[0] + n[1]) : (double)n[0] * (1.0 + rho) + (double)n[1];
            const double tn = den > 0.0 ? (capped ? (a[0] + a[1] - (double)n[0] * M) : (a[0] + a[1])) / den
                                        : 0.5 * (lo + hi);
            const bool ok = den > 0.0 && tn > lo && tn < hi;
            if (ok) {
              // the Newton point is the root when it lies on the same linear piece:
              // no tail key in (tn, t] or (t, tn], no top key between the two h values
              const double hn = tn + fmin(rho * tn, M);
              const ULL cb = dbits(tn), hcb = dbits(hn);
              bool same = (rho * tn >= M) == capped;
              if (tn < t) same = same && x0 <= cb && x1 < hcb;
              else same = same && x2 > cb && x3 >= hcb;
              if (same) { done = 1; res = tn; }
              t = tn;
            } else {
              t = 0.5 * (lo + hi);
            }
            if (!done && (hi - lo <= 2e-16 * hi || it == 199)) { done = 1; res = ok ? tn : hi; }
          }
        }
        sm.rflag[0] = done;
        sm.rflag[1] = n[1];
        sm.rt[0] = res;
        sm.rtb[0] = dbits(t);
        sm.rtb[1] = dbits(t + fmin(rho * t, M));
      }
    }
    __syncthreads();
    const int done = sm.rflag[0];
    if (done) {
      *root = sm.rt[0];
      *pooled = sm.rflag[1];
      __syncthreads();
      return done == 1;
    }
  }
  return false;   // not reached: thread 0 ends the search by iteration 199
}

// Root of Phi over full passes of w (pooled blocks wider than the candidate
// capacity), the same search as root_unsorted: every thread sums the active
// members of its coordinates -- the float key of |w| decides most of them, the
// FP64 value (compared as bits) only where the key ties with the boundary's or
// the point's -- and thread 0 alone runs the Newton / bisection scalars, from the
// previous step's threshold.  Phi(hi0) > 0; Phi(0) <= 0 always.
__device__ double root_fullpass_global(const Dev& d, SelSmem& sm, int q, unsigned thr, double bnd_a, int bnd_i,
                                       double hi0, double t0, double rho, double M) {
  const int p = d.p;
  const double* w = (const double*)d.wbuf;
  double lo = 0.0, hi = hi0, t = 0.0;
  int pnA = -1, pnB = -1;
  double pSA = 0.0, pSB = 0.0;
  bool pcap = false;
  if (threadIdx.x == 0) {
    t = (t0 > lo && t0 < hi) ? t0 : 0.5 * hi;
    sm.rtb[0] = dbits(t);
    sm.rtb[1] = dbits(t + fmin(rho * t, M));
    sm.rflag[1] = (int)(__float_as_uint((float)t) & 0x7fffffffu);
    sm.rflag[0] = 0;
  }
  __syncthreads();
  for (int it = 0; it < 200; ++it) {
    const unsigned long long tb = sm.rtb[0], hb = sm.rtb[1];
    const unsigned kt = (unsigned)sm.rflag[1];
    int nA = 0, nB = 0;
    double SA = 0.0, SB = 0.0;
    for (int i = threadIdx.x; i < p; i += kSelBlock) {
      const unsigned kk = __ldcg(&d.key[i]);
      if (kk == 0u || (kk < kt && kk < thr)) continue;   // off the free set, or below both the point and the top set
      const bool maybe_top = kk >= thr;
      double a = 0.0;
      bool top = false;
      if (maybe_top) {
        a = fabs(__ldcg(&w[i]));
        top = in_top(kk, a, i, thr, q, bnd_a, bnd_i);
      }
      if (top) {
        if (dbits(a) < hb) { nA += 1; SA += a; }
      } else if (kk >= kt) {
        if (!maybe_top) a = fabs(__ldcg(&w[i]));
        if (dbits(a) > tb) { nB += 1; SB += a; }
      }
    }
    block_reduce_cs(nA, SA, nB, SB, sm);
    if (threadIdx.x == 0) {
      const bool capped = rho * t >= M;
      const double phi = (double)nA * dval(hb) - SA - (SB - (double)nB * t);
      int done = 0;
      double res = t;
      if (phi == 0.0 || (nA == pnA && nB == pnB && capped == pcap && SA == pSA && SB == pSB)) {
        done = 1;
      } else {
        if (phi < 0.0) lo = t; else hi = t;
        const double den = capped ? (double)(nA + nB) : (double)nA * (1.0 + rho) + (double)nB;
        const double tn = den > 0.0 ? (capped ? (SA + SB - (double)nA * M) : (SA + SB)) / den : 0.5 * (lo + hi);
        const bool ok = tn > lo && tn < hi;
        if (hi - lo <= 2e-16 * hi || it == 199) {
          done = 1;
          res = ok ? tn : hi;
        } else {
          pnA = ok ? nA : -1;
          pnB = nB;
          pSA = SA;
          pSB = SB;
          pcap = capped;
          t = ok ? tn : 0.5 * (lo + hi);
        }
      }
      sm.rflag[0] = done;
      sm.rt[0] = res;
      sm.rtb[0] = dbits(t);
      sm.rtb[1] = dbits(t + fmin(rho * t, M));
      // the float key below which no coordinate can exceed t: fl32 rounds to nearest,
      // so key(a) < key(t) implies a < t
      sm.rflag[1] = (int)(__float_as_uint((float)t) & 0x7fffffffu);
    }
    __syncthreads();
    if (sm.rflag[0]) {
      const double r = sm.rt[0];
      __syncthreads();
      return r;
    }
  }
  return sm.rt[0];
}

// next step's candidate floor: with x the smallest value of a fixed ladder whose
// count of candidates at or above x theta stays within `want` (the top set and
// about 1.5 times the pooled block) and whose x theta is not below this list's
// floor, 0.98 x theta -- the candidates then reach a little below the pooled
// block the next step is likely to need; 0 (every free coordinate) when theta is 0
__device__ unsigned next_floor_key(SelSmem& sm, int cc, double theta, int want, unsigned long long floor_now) {
  constexpr int NX = 16;
  if (!(theta > 0.0) || !isfinite(theta)) return 0u;
  unsigned long long* thr = sm.tkey + kProxCap - 16;   // past any top set of the fast path
  if (threadIdx.x < NX) {
    const double xs[NX] = {0.999, 0.995, 0.99, 0.985, 0.98, 0.97, 0.96, 0.94,
                           0.92,  0.89,  0.85, 0.8,   0.7,  0.6,  0.5,  0.3};
    thr[threadIdx.x] = dbits(xs[threadIdx.x] * theta);
    sm.rcnt[2 + threadIdx.x] = 0;
  }
  __syncthreads();
  int c[NX];
#pragma unroll
  for (int m = 0; m < NX; ++m) c[m] = 0;
  for (int j = threadIdx.x; j < cc; j += kSelBlock) {
    const unsigned long long k = sm.cand[j];
#pragma unroll
    for (int m = 0; m < NX; ++m) c[m] += k >= thr[m];
  }
#pragma unroll
  for (int m = 0; m < NX; ++m) {
    c[m] = __reduce_add_sync(0xffffffffu, c[m]);
    if ((threadIdx.x & 31) == 0) atomicAdd(&sm.rcnt[2 + m], c[m]);
  }
  __syncthreads();
  // counts below the current list's floor are unknown: the ladder stops there
  int pick = 0;
#pragma unroll
  for (int m = 0; m < NX; ++m)
    if (sm.rcnt[2 + m] <= want && thr[m] >= floor_now) pick = m;
  const unsigned key = __float_as_uint((float)(0.98 * dval(thr[pick]))) & 0x7fffffffu;
  __syncthreads();
  return key;
}

__device__ void prox_select_cta(const Dev& d, NodeDev* nd, SelSmem& sm, int q) {
  const int p = d.p;
  const double rho = nd->rho, M = nd->M;
  if (threadIdx.x == 0) sm.cs[0] = rho / (1.0 + rho);   // once, not in every thread
  __syncthreads();
  const double shrink = sm.cs[0];
  const unsigned* key = d.key;
  const double* w = (const double*)d.wbuf;
  auto kload = [&](int i) -> unsigned { return __ldcg(&key[i]); };
  unsigned thr = 0xffffffffu;
  double bnd_a = -1.0, theta = INFINITY;
  int bnd_i = 0x7fffffff, qused = 0, fb = 0;
  bool sorted_top = false;
  unsigned next_guess = 0u;
  // ---- fast path: the candidates predicted from the previous step (every free
  // coordinate with key >= cguess, appended by the gradient epilogue)
  bool done = false;
  const int cc = __ldcg(&d.ccount[0]);
  const unsigned cg = nd->cguess;
  if (q > 0 && cc <= kProxCap && (cc >= q + 1 || cg == 0u)) {
    for (int j = threadIdx.x; j < cc; j += kSelBlock) {
      sm.cand[j] = __ldcg(&d.cand_a[j]);
      sm.cidx[j] = __ldcg(&d.cand_i[j]);
    }
    __syncthreads();
    if (cc <= q) {
      // every free coordinate is in the top set (the rest of it are zeros)
      const int N = next_pow2(cc > 0 ? cc : 1);
      for (int j = cc + threadIdx.x; j < N; j += kSelBlock) { sm.cand[j] = 0ull; sm.cidx[j] = 0x7fffffff; }
      __syncthreads();
      sort_pairs_desc(sm.cand, sm.cidx, N);   // |w| descending, index ascending (Alg. 1)
      thr = 0u;
      bnd_a = -1.0;
      theta = 0.0;
      for (int t = threadIdx.x; t < q; t += kSelBlock) {
        const double a = t < cc ? dval(sm.cand[t]) : 0.0;
        const double mg = fmin(fmin(M, shrink * a), a);
        d.tbeta[t] = mg > 0.0 ? mg : 0.0;
      }
      done = true;
    } else {
      // the top set in Alg. 1 order (|w| descending, index ascending): every candidate
      // at or above a floor that holds at least q of them, sorted -- the floor is just
      // below the previous step's boundary value (the top set moves little), else
      // the q-th largest by radix selection
      auto cload = [&](int i) -> unsigned long long { return sm.cand[i]; };
      auto gather = [&](unsigned long long fk) {
        if (threadIdx.x == 0) sm.flag[0] = 0;
        __syncthreads();
        for (int j = threadIdx.x; j < cc; j += kSelBlock) {
          if (sm.cand[j] >= fk) {
            const int pos = atomicAdd(&sm.flag[0], 1);
            if (pos < kProxCap - 16) {
              sm.tkey[pos] = sm.cand[j];
              sm.tidx[pos] = sm.cidx[j];
            }
          }
        }
        __syncthreads();
        return sm.flag[0];
      };
      int G = 0;
      const double pb = nd->bnd_a;
      if (pb > 0.0 && isfinite(pb)) {
        G = gather(dbits(0.98 * pb));
        if (G < q || G > 1024) G = 0;      // too few (the set grew) or too many to sort cheaply
      }
      if (G == 0) {
        const SelectResult<unsigned long long> R =
            block_select<unsigned long long, kSelBlock>(cc, q, cload, sm.hist, sm.sh);
        G = gather(R.thr);
      }
      __syncthreads();
      if (G <= kProxCap - 16) {   // else: massive ties at the boundary, left to the full path below
      const int NG = next_pow2(G);
      for (int j = G + threadIdx.x; j < NG; j += kSelBlock) { sm.tkey[j] = 0ull; sm.tidx[j] = 0x7fffffff; }
      __syncthreads();
      sort_pairs_desc(sm.tkey, sm.tidx, NG);
      const unsigned long long bk = sm.tkey[q - 1];
      const int bi = sm.tidx[q - 1];
      // the root of Phi over the unsorted candidates (floor: every coordinate off the
      // candidate list has a key below cg, hence |w| below the float value of cg)
      const bool all = (cg == 0u);
      const double floorv = all ? 0.0 : (double)__uint_as_float(cg);
      double th = 0.0;
      int pooled = 0;
      const bool fnd = root_unsorted(sm, cc, bk, bi, floorv, all, dval(sm.tkey[0]), nd->theta, rho, M,
                                     &th, &pooled);
      if (fnd) {
        theta = th;
        bnd_a = dval(bk);
        bnd_i = bi;
        thr = __float_as_uint((float)bnd_a) & 0x7fffffffu;   // the key of the boundary element
        qused = cc;
        for (int t = threadIdx.x; t < q; t += kSelBlock) {
          const double a = dval(sm.tkey[t]);
          const double mg = fmin(fmin(M, shrink * a), a - theta);
          d.tbeta[t] = mg > 0.0 ? mg : 0.0;
        }
        __syncthreads();   // the top set's reads are done before its tail is reused
        // next step's list: about 1.5 times the top set and pooled block
        const int want = (q + pooled) + (q + pooled) / 2 + 32;
        next_guess = next_floor_key(sm, cc, theta, want < kProxCap ? want : kProxCap, dbits(floorv));
        done = true;
      }
      __syncthreads();
      }
    }
  }
  if (q > 0 && !done) {
    const SelectResult<unsigned> Rk = block_select<unsigned, kSelBlock>(p, q, kload, sm.hist, sm.sh, d.hist);
    thr = Rk.thr;
    const int need = q - Rk.gt, eq = Rk.eq;
    if (need < eq && eq <= kProxCap && thr != 0u) {
      // exact order among equal float keys: |w| descending, then index ascending
      if (threadIdx.x == 0) sm.flag[0] = 0;
      __syncthreads();
      for (int i = threadIdx.x; i < p; i += kSelBlock) {
        if (__ldcg(&key[i]) == thr) {
          const int pos = atomicAdd(&sm.flag[0], 1);
          sm.cand[pos] = dbits(fabs(__ldcg(&w[i])));
          sm.cidx[pos] = i;
        }
      }
      __syncthreads();
      const int N = next_pow2(eq);
      for (int j = eq + threadIdx.x; j < N; j += kSelBlock) { sm.cand[j] = 0ull; sm.cidx[j] = 0x7fffffff; }
      __syncthreads();
      sort_pairs_desc(sm.cand, sm.cidx, N);
      bnd_a = dval(sm.cand[need - 1]);
      bnd_i = sm.cidx[need - 1];
      __syncthreads();
    }
    if (q == p || thr == 0u) {
      theta = 0.0;   // no tail (or only zeros in it): no isotonic violation
    } else {
      int Q = nd->qhint > q + 1 ? nd->qhint : q + 1;
      if (Q > p) Q = p;
      bool found = false;
      double last_floor = INFINITY;
      while (!found && Q <= kProxCap) {
        unsigned thrQ = 0u;
        int C = p;
        if (Q < p) {
          const SelectResult<unsigned> RQ =
              block_select<unsigned, kSelBlock>(p, Q, kload, sm.hist, sm.sh, d.hist);
          thrQ = RQ.thr;
          C = RQ.gt + RQ.eq;
        }
        if (C > kProxCap) break;
        if (threadIdx.x == 0) sm.flag[0] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < p; i += kSelBlock) {
          const unsigned kk = __ldcg(&key[i]);
          if (Q >= p || kk >= thrQ) {
            const int pos = atomicAdd(&sm.flag[0], 1);
            sm.cand[pos] = dbits(key_value(kk, w, i));
          }
        }
        __syncthreads();
        const int N = next_pow2(C);
        for (int j = C + threadIdx.x; j < N; j += kSelBlock) sm.cand[j] = 0ull;
        __syncthreads();
        sort_u64_desc(sm.cand, N);
        prefix_values(sm, C);
        for (int t = threadIdx.x; t < q; t += kSelBlock) sm.tb[t] = top_break(dval(sm.cand[t]), rho, M);
        __syncthreads();
        const double floorv = (Q < p) ? dval(sm.cand[C - 1]) : 0.0;
        double th = 0.0;
        const bool fnd = threadIdx.x < 32 && root_search(sm, q, C, floorv, Q >= p, rho, M, &th);
        if (threadIdx.x == 0) {
          sm.flag[1] = fnd ? 1 : 0;
          sm.root[0] = th;
        }
        __syncthreads();
        found = sm.flag[1] != 0;
        theta = sm.root[0];
        qused = C;
        last_floor = floorv;
        __syncthreads();
        if (!found) {   // grow, and try the full capacity before giving up
          if (Q >= p || Q >= kProxCap) break;
          Q = 4 * Q;
          if (Q > kProxCap) Q = kProxCap;
          if (Q > p) Q = p;
        }
      }
      if (found) {
        sorted_top = true;
      } else {
        fb = 1;
        theta = root_fullpass_global(d, sm, q, thr, bnd_a, bnd_i,
                                     isinf(last_floor) ? (double)__uint_as_float(thr) * 2.0 + 1e-300
                                                       : last_floor, nd->theta, rho, M);
      }
    }
    // |b| on the top set, descending (its order is the order of |w|), for Alg. 2
    if (!sorted_top) {
      if (threadIdx.x == 0) sm.flag[0] = 0;
      __syncthreads();
      const int C = Rk.gt + Rk.eq;
      if (C <= kProxCap) {
        for (int i = threadIdx.x; i < p; i += kSelBlock) {
          const unsigned kk = __ldcg(&key[i]);
          if (kk >= thr) sm.cand[atomicAdd(&sm.flag[0], 1)] = dbits(key_value(kk, w, i));
        }
        __syncthreads();
        const int N = next_pow2(C);
        for (int j = C + threadIdx.x; j < N; j += kSelBlock) sm.cand[j] = 0ull;
        __syncthreads();
        sort_u64_desc(sm.cand, N);
      } else {  // massive ties of the float key: its value stands for the tied ones
        for (int i = threadIdx.x; i < p; i += kSelBlock) {
          const unsigned kk = __ldcg(&key[i]);
          if (kk > thr) sm.cand[atomicAdd(&sm.flag[0], 1)] = dbits(key_value(kk, w, i));
        }
        __syncthreads();
        for (int j = Rk.gt + threadIdx.x; j < q; j += kSelBlock)
          sm.cand[j] = dbits((double)__uint_as_float(thr));
        const int N = next_pow2(q);
        for (int j = q + threadIdx.x; j < N; j += kSelBlock) sm.cand[j] = 0ull;
        __syncthreads();
        sort_u64_desc(sm.cand, N);
      }
    }
    for (int t = threadIdx.x; t < q; t += kSelBlock) {
      const double a = dval(sm.cand[t]);
      const double mg = fmin(fmin(M, shrink * a), a - theta);
      d.tbeta[t] = mg > 0.0 ? mg : 0.0;
    }
    // next step's guess from the threshold just found
    next_guess = (theta > 0.0 && isfinite(theta))
                     ? (__float_as_uint((float)(0.95 * theta)) & 0x7fffffffu) : 0u;
  }
  if (threadIdx.x == 0) {
    nd->cguess = next_guess;
    nd->fast_steps += done ? 1 : 0;
    d.ccount[0] = 0;
    nd->theta = theta;
    nd->thr_kf = thr;
    nd->bnd_a = bnd_a;
    nd->bnd_i = bnd_i;
    nd->q = q;
    int h = qused / 2;
    if (h < q + 64) h = q + 64;
    nd->qhint = h;
    nd->fallback += fb;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 2048; b += kSelBlock) d.hist[b] = 0u;   // ready for the next step
}

// In-loop dual term (Sec. 3.4) at zeta_gamma: a = X^T zeta_gamma = -grad;
// G*(a)/(2 lambda2) = TopSum_k'(H_M(|a_F|/2l2)) + sum_S1 H_M(|a_j|/2l2).
__device__ void dual_cta(const Dev& d, NodeDev* nd, SelSmem& sm, int q) {
  const int p = d.p;
  if (threadIdx.x == 0) sm.cs[1] = 1.0 / (2.0 * nd->lambda2);   // once, not in every thread
  __syncthreads();
  const double scale = sm.cs[1], M = nd->M;
  const double* g = d.grad;
  // S1 from its index list (a scan of the p states would be a chain of dependent
  // loads per thread: ~50 loads deep at p = 50000)
  double s1 = 0.0;
  const int n1 = nd->n_one;
  for (int t = threadIdx.x; t < n1; t += kSelBlock) s1 += huber(fabs(g[d.one_idx[t]]) * scale, M);
  {
    int c0 = 0, c1 = 0;
    double unused = 0.0;
    block_reduce_cs(c0, s1, c1, unused, sm);
  }
  double s = 0.0;
  unsigned next_guess = 0u;
  const int dc = __ldcg(&d.ccount[1]);
  const unsigned dg = nd->dguess;
  if (q > 0 && dc <= kProxCap && (dc >= q || dg == 0u)) {
    // the predicted candidates hold the top-k' magnitudes of the gradient (at a
    // KKT point many of them are nearly equal: the list can be long): the k'-th
    // largest by radix selection, H_M over the larger ones, the ties at its value
    for (int j = threadIdx.x; j < dc; j += kSelBlock) sm.cand[j] = __ldcg(&d.dcand[j]);
    __syncthreads();
    const int top = q < dc ? q : dc;
    if (top > 0) {
      auto cload = [&](int i) -> unsigned long long { return sm.cand[i]; };
      const SelectResult<unsigned long long> R =
          block_select<unsigned long long, kSelBlock>(dc, top, cload, sm.hist, sm.sh);
      int nb = 0, nz = 0;
      double b = 0.0, z = 0.0;
      for (int j = threadIdx.x; j < dc; j += kSelBlock)
        if (sm.cand[j] > R.thr) b += huber(dval(sm.cand[j]) * scale, M);
      block_reduce_cs(nb, b, nz, z, sm);
      if (threadIdx.x == 0) {
        const double tv = dval(R.thr);
        sm.rt[1] = b + (double)(top - R.gt) * huber(tv * scale, M);
        sm.rflag[1] = (int)(__float_as_uint((float)(0.995 * tv)) & 0x7fffffffu);
      }
      __syncthreads();
      s = sm.rt[1];
      next_guess = (unsigned)sm.rflag[1];
    }
    if (threadIdx.x == 0) nd->dfast_steps += 1;
  } else if (q > 0) {
    auto kload = [&](int i) -> unsigned { return __ldcg(&d.dkey[i]); };
    const SelectResult<unsigned> R =
        block_select<unsigned, kSelBlock>(p, q, kload, sm.hist, sm.sh, d.hist + 2048);
    for (int i = threadIdx.x; i < p; i += kSelBlock)
      if (__ldcg(&d.dkey[i]) > R.thr) s += huber(fabs(g[i]) * scale, M);
    s = block_sum<double, kSelBlock>(s, sm.red);
    const int need = q - R.gt;
    if (need > 0) {
      if (R.eq <= kProxCap) {   // the `need` largest exact values among equal float keys
        if (threadIdx.x == 0) sm.flag[0] = 0;
        __syncthreads();
        for (int i = threadIdx.x; i < p; i += kSelBlock) {
          const unsigned kk = __ldcg(&d.dkey[i]);
          if (kk == R.thr) sm.cand[atomicAdd(&sm.flag[0], 1)] = dbits(key_value(kk, g, i));
        }
        __syncthreads();
        const int N = next_pow2(R.eq);
        for (int j = R.eq + threadIdx.x; j < N; j += kSelBlock) sm.cand[j] = 0ull;
        __syncthreads();
        sort_u64_desc(sm.cand, N);
        double b = 0.0;
        for (int j = threadIdx.x; j < need; j += kSelBlock) b += huber(dval(sm.cand[j]) * scale, M);
        s += block_sum<double, kSelBlock>(b, sm.red);
      } else {
        s += (double)need * huber((double)__uint_as_float(R.thr) * scale, M);
      }
    }
    next_guess = __float_as_uint(0.995f * __uint_as_float(R.thr)) & 0x7fffffffu;
  }
  // eigen-perspective (App. D.2): the in-loop dual point -2 Q gamma adds eig ||gamma||^2
  // to -F*(-zeta) (||y||^2 - ||X gamma||^2 + eig ||gamma||^2)
  double gsq = 0.0;
  const double eig = nd->eig;
  if (eig > 0.0) {
    const int t = nd->iter;
    const double* bc = (const double*)d.beta + (size_t)(t % 3) * p;
    const double* bp = (const double*)d.beta + (size_t)((t + 2) % 3) * p;
    const double c = nd->c;
    for (int j = threadIdx.x; j < p; j += kSelBlock) {
      const double g = bc[j] + c * (bc[j] - bp[j]);
      gsq += g * g;
    }
    int c0 = 0, c1 = 0;
    double unused = 0.0;
    block_reduce_cs(c0, gsq, c1, unused, sm);
  }
  if (threadIdx.x == 0) {
    nd->gstar = s1 + s;
    if (eig > 0.0) nd->negconj += eig * gsq;
    nd->dguess = next_guess;
    d.ccount[1] = 0;
  }
  __syncthreads();
  for (int b = threadIdx.x; b < 2048; b += kSelBlock) d.hist[2048 + b] = 0u;
}

__global__ void __launch_bounds__(kSelBlock, 1) k_prox_select(Dev d) {
  NodeDev* nd = d.nd;
  if (nd->done) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  SelSmem& sm = *reinterpret_cast<SelSmem*>(smem_raw);
  const int kp = nd->kp;
  const int q = kp <= 0 ? 0 : (kp < d.p ? kp : d.p);
  if (blockIdx.x == 0) prox_select_cta(d, nd, sm, q);
  else dual_cta(d, nd, sm, q);
}

// ------------------------------------------------------------------ apply

__global__ void __launch_bounds__(kSegLen) k_prox_apply(Dev d) {
  NodeDev* nd = d.nd;
  if (nd->done) return;
  __shared__ double red[64];
  __shared__ int shi[64];
  __shared__ int wcnt[kSegLen / 32];
  __shared__ int s_last;
  const int p = d.p, seg = blockIdx.x;
  const int j = seg * kSegLen + (int)threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nxt = (nd->iter + 1) % 3;
  double* bn = (double*)d.beta + (size_t)nxt * p;
  const double theta = nd->theta, rho = nd->rho, M = nd->M, bnd_a = nd->bnd_a;
  const double shrink = rho / (1.0 + rho);
  const unsigned thr = nd->thr_kf;
  const int q = nd->q, bnd_i = nd->bnd_i;
  double l1 = 0.0, s1 = 0.0, bsq = 0.0;
  bool nz = false;
  if (j < p) {
    const int8_t st = d.state ? d.state[j] : (int8_t)kFree;
    const double w = ((const double*)d.wbuf)[j];
    double b;
    if (st == kFree) {
      const double a = fabs(w);
      double mag = in_top(d.key[j], a, j, thr, q, bnd_a, bnd_i) ? fmin(fmin(M, shrink * a), a - theta)
                                                                 : fmax(0.0, a - theta);
      if (!(mag > 0.0)) mag = 0.0;
      b = w < 0.0 ? -mag : mag;
      l1 = mag;
      bsq = mag * mag;
    } else if (st == kZero) {
      b = 0.0;
    } else {   // z_j = 1: argmin 1/2 (b - w)^2 + b^2/(2 rho) on the box
      b = fmin(fmax(rho * w / (1.0 + rho), -M), M);
      s1 = b * b;
    }
    bn[j] = b;
    const float hi = (float)b;
    d.bhi[j] = hi;
    d.blo[j] = (float)(b - (double)hi);
    nz = b != 0.0;
  }
  // ordered compaction of this segment's nonzeros
  const unsigned bal = __ballot_sync(0xffffffffu, nz);
  if (lane == 0) wcnt[warp] = __popc(bal);
  __syncthreads();
  int base = 0, tot = 0;
  for (int k = 0; k < kSegLen / 32; ++k) {
    if (k < warp) base += wcnt[k];
    tot += wcnt[k];
  }
  if (nz) d.nnz_idx[seg * kSegLen + base + __popc(bal & ((1u << lane) - 1u))] = j;
  l1 = block_sum<double, kSegLen>(l1, red);
  s1 = block_sum<double, kSegLen>(s1, red);
  const bool eig = nd->eig > 0.0;   // eigen-perspective: ||b^{t+1}||^2 for the objective
  if (eig) bsq = block_sum<double, kSegLen>(bsq, red);
  if (threadIdx.x == 0) {
    d.seg_cnt[seg] = tot;
    d.segpart[seg] = l1;
    d.segpart[d.nseg + seg] = s1;
    if (eig) d.segpart[2 * d.nseg + seg] = bsq;
  }
  __threadfence();
  __syncthreads();
  const int ci = cnt_apply(d);
  if (threadIdx.x == 0) s_last = (atomicAdd(&d.cnt[ci], 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  // last CTA: segment offsets, totals, and g(b) by Algorithm 2's water-filling on
  // the top set (its |b| in descending order from the select kernel)
  int running = 0;
  for (int b0 = 0; b0 < d.nseg; b0 += kSegLen) {
    const int i = b0 + (int)threadIdx.x;
    const int v = i < d.nseg ? __ldcg(&d.seg_cnt[i]) : 0;
    int t2;
    const int ex = block_exclusive_scan<int, kSegLen>(v, shi, &t2);
    if (i < d.nseg) d.seg_off[i] = running + ex;
    running += t2;
  }
  double L1 = 0.0, S1 = 0.0, BQ = 0.0;
  for (int i = threadIdx.x; i < d.nseg; i += kSegLen) {
    L1 += __ldcg(&d.segpart[i]);
    S1 += __ldcg(&d.segpart[d.nseg + i]);
    if (eig) BQ += __ldcg(&d.segpart[2 * d.nseg + i]);
  }
  L1 = block_sum<double, kSegLen>(L1, red);
  S1 = block_sum<double, kSegLen>(S1, red);
  if (eig) BQ = block_sum<double, kSegLen>(BQ, red);
  if (threadIdx.x == 0) {
    d.seg_off[d.nseg] = running;
    nd->nnz = running;
    nd->l1 = L1;
    nd->s1sq = S1;
    const int kp = nd->kp;
    double g = 0.0, sq = 0.0, cum = 0.0;
    bool brk = false;
    for (int t = 0; t < q; ++t) {
      const double bt = __ldcg(&d.tbeta[t]);
      const double sbar = (L1 - cum) / (double)(kp - t);
      if (sbar >= bt) {
        g = 0.5 * (sq + (double)(kp - t) * sbar * sbar);
        brk = true;
        break;
      }
      sq += bt * bt;
      cum += bt;
    }
    if (!brk) {
      if (q < kp) {
        const double sbar = fmax(0.0, (L1 - cum) / (double)(kp - q));
        g = 0.5 * (sq + (double)(kp - q) * sbar * sbar);
      } else {
        g = 0.5 * sq;
      }
    }
    nd->g_next = 0.5 * S1 + g;
    nd->bsq_next = BQ + S1;
    d.cnt[ci] = 0;
  }
}

// ------------------------------------------------------------------ Lanczos

constexpr int kVecBlock = 256;

__host__ __device__ inline int vec_grid(int n) {
  const int g = (n + kVecBlock - 1) / kVecBlock;
  return g < 1216 ? g : 1216;   // 8 CTAs per SM; partials fit the segment arrays
}

__global__ void __launch_bounds__(kVecBlock) k_split(const double* src, float* hi, float* lo, int n) {
  for (int i = blockIdx.x * kVecBlock + threadIdx.x; i < n; i += gridDim.x * kVecBlock) {
    const double v = src[i];
    const float h = (float)v;
    hi[i] = h;
    lo[i] = (float)(v - (double)h);
  }
}

__global__ void __launch_bounds__(kVecBlock) k_lz_start(Dev d, double inv_norm) {
  for (int i = blockIdx.x * kVecBlock + threadIdx.x; i < d.p; i += gridDim.x * kVecBlock) {
    const double v = (1.0 + (double)((unsigned long long)(i + 1) * 2654435761ull % 1000ull) / 1000.0) * inv_norm;
    d.vcur[i] = v;
    d.vprev[i] = 0.0;
    const float h = (float)v;
    d.vhi[i] = h;
    d.vlo[i] = (float)(v - (double)h);
  }
}

// phase 0: w = X^T X v - beta_{it-1} v_prev, alpha = w.v
// phase 1: w -= alpha v, beta = ||w||
// phase 2: v_prev = v, v = w / beta (and its float split)
template <int PHASE>
__global__ void __launch_bounds__(kVecBlock) k_lz(Dev d, int it) {
  __shared__ double red[64];
  __shared__ int s_last;
  double* w = (double*)d.wbuf;
  const double* alpha = d.lz;
  const double* beta = d.lz + kLanczosMax;
  double acc = 0.0;
  const double bprev = (PHASE == 0 && it > 0) ? beta[it - 1] : 0.0;
  const double al = (PHASE == 1) ? alpha[it] : 0.0;
  const double inv_b = (PHASE == 2) ? (beta[it] > 0.0 ? 1.0 / beta[it] : 0.0) : 0.0;
  for (int i = blockIdx.x * kVecBlock + threadIdx.x; i < d.p; i += gridDim.x * kVecBlock) {
    if (PHASE == 0) {
      const double v = d.grad[i] - bprev * d.vprev[i];
      w[i] = v;
      acc += v * d.vcur[i];
    } else if (PHASE == 1) {
      const double v = w[i] - al * d.vcur[i];
      w[i] = v;
      acc += v * v;
    } else {
      const double v = w[i] * inv_b;
      d.vprev[i] = d.vcur[i];
      d.vcur[i] = v;
      const float h = (float)v;
      d.vhi[i] = h;
      d.vlo[i] = (float)(v - (double)h);
    }
  }
  if (PHASE == 2) return;
  acc = block_sum<double, kVecBlock>(acc, red);
  if (threadIdx.x == 0) d.segpart[blockIdx.x] = acc;
  __threadfence();
  __syncthreads();
  const int ci = cnt_lz(d);
  if (threadIdx.x == 0) s_last = (atomicAdd(&d.cnt[ci], 1) == (int)gridDim.x - 1);
  __syncthreads();
  if (!s_last) return;
  __threadfence();
  double s = 0.0;
  for (int b = threadIdx.x; b < (int)gridDim.x; b += kVecBlock) s += __ldcg(&d.segpart[b]);
  s = block_sum<double, kVecBlock>(s, red);
  if (threadIdx.x == 0) {
    if (PHASE == 0) d.lz[it] = s;
    else d.lz[kLanczosMax + it] = sqrt(s);
    d.cnt[ci] = 0;
  }
}

// ------------------------------------------------------------------ launchers

void launch_fwd_raw(const Dev& d, cudaStream_t s);   // k_matvec.cu
void launch_grad_raw(const Dev& d, cudaStream_t s);

cudaError_t prox_grid_prepare(int optin) {
  return cudaFuncSetAttribute(k_prox_select, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)sizeof(SelSmem) < optin ? (int)sizeof(SelSmem) : optin);
}

void launch_prox_select(const Dev& d, cudaStream_t s) {
  k_prox_select<<<2, kSelBlock, sizeof(SelSmem), s>>>(d);
}

void launch_prox_apply(const Dev& d, cudaStream_t s) {
  k_prox_apply<<<d.nseg, kSegLen, 0, s>>>(d);
}

void launch_split(const double* src, float* hi, float* lo, int n, cudaStream_t s) {
  k_split<<<vec_grid(n), kVecBlock, 0, s>>>(src, hi, lo, n);
}

void launch_lanczos_start(const Dev& d, cudaStream_t s, double inv_norm) {
  k_lz_start<<<vec_grid(d.p), kVecBlock, 0, s>>>(d, inv_norm);
}

void launch_lanczos_step(const Dev& d, cudaStream_t s, int it) {
  launch_fwd_raw(d, s);
  launch_grad_raw(d, s);
  const int g = vec_grid(d.p);
  k_lz<0><<<g, kVecBlock, 0, s>>>(d, it);
  k_lz<1><<<g, kVecBlock, 0, s>>>(d, it);
  k_lz<2><<<g, kVecBlock, 0, s>>>(d, it);
}

}  // namespace ksc
