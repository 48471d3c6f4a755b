// ksc_prox.cuh -- block-level (one CTA per segment) exact proximal operator of
// the perspective term and the value of g, for one node.
//
// prox_{rho^-1 g}(w) = w - rho^-1 prox_{rho g*}(rho w)     (Moreau, Sec. 3.3)
// prox_{rho g*} is the Huber-isotonic regression of Lemma 3.3 on the sorted
// |rho w|, solved by PAVA in the paper (Alg. 1 + Alg. 4).  With the Huber
// weight rho on the top k' positions only, the unconstrained block values are
// non-increasing on each side of position k', so PAVA pools at most ONE block
// straddling k'/k'+1.  Its value v = rho * theta is the root of the monotone,
// piecewise-linear
//   Phi(theta) = sum_{t in top} (theta + min(rho theta, M) - a_t)_+
//              - sum_{j in tail} (a_j - theta)_+,        a = |w|,
// and in primal terms the prox is
//   top k':  |b| = min(M, rho a/(1+rho), a - theta)   (ridge shrink / box / pool)
//   tail:    |b| = max(0, a - theta)                    (soft threshold).
// The kernel finds theta exactly: a radix select gives the top-Q magnitudes
// (Q = k' + candidate tail), a bitonic sort orders them, and a prefix scan over
// the breakpoints {a_j, theta^b_t, M/rho} brackets the root, where Phi is linear.
// If the pooled block reaches past the candidates, Q grows; past the shared
// memory capacity a full-pass bracketed Newton iteration on the same Phi is used.
#pragma once

#include "ksc_common.cuh"
#include "ksc_state.cuh"

namespace ksc {

constexpr int kProxBlock = 1024;

// Shared-memory carve for one segment.  cap: candidate capacity (power of 2).
template <typename T>
struct SegSmem {
  unsigned* hist;   // 2048
  int* sh;          // 64
  double* red;      // 64
  double* cand;     // cap
  double* pref;     // cap + 1
  int* cidx;        // cap (index payload for ordered outputs)
  T* wsm;           // segment values in shared memory, or nullptr (global scratch)
  int cap;
};

__host__ __device__ inline size_t seg_smem_bytes(int cap, int wsm_elems, int tbytes) {
  return 2048 * 4 + 64 * 4 + 64 * 8 + (size_t)cap * 8 + (size_t)(cap + 1) * 8 + (size_t)cap * 4 +
         (size_t)wsm_elems * tbytes + 64;
}

template <typename T>
__device__ inline SegSmem<T> carve_seg_smem(unsigned char* base, int cap, int wsm_elems) {
  SegSmem<T> s;
  size_t off = 0;
  s.hist = (unsigned*)(base + off); off += 2048 * 4;
  s.sh = (int*)(base + off); off += 64 * 4;
  s.red = (double*)(base + off); off += 64 * 8;
  s.cand = (double*)(base + off); off += (size_t)cap * 8;
  s.pref = (double*)(base + off); off += (size_t)(cap + 1) * 8;
  s.cidx = (int*)(base + off); off += (size_t)cap * 4;
  off = (off + 15) & ~(size_t)15;
  s.wsm = wsm_elems > 0 ? (T*)(base + off) : nullptr;
  s.cap = cap;
  return s;
}

template <typename T>
__device__ __forceinline__ typename Bits<T>::U abs_bits(T x) {
  using U = typename Bits<T>::U;
  const U mask = ~((U)1 << (sizeof(U) * 8 - 1));
  return Bits<T>::of(x) & mask;
}

__device__ __forceinline__ int next_pow2(int x) {
  int n = 1;
  while (n < x) n <<= 1;
  return n;
}

// breakpoint of a top element: theta where theta + min(rho theta, M) = a
__device__ __forceinline__ double top_break(double a, double rho, double M) {
  return (a * rho <= M * (1.0 + rho)) ? a / (1.0 + rho) : a - M;
}

// Exclusive prefix sums pref[0..Q] of cand[0..Q) (double), block-wide.
template <int BLOCK>
__device__ void block_prefix(const double* cand, double* pref, int Q, double* red) {
  const int per = (Q + BLOCK - 1) / BLOCK;
  const int s0 = threadIdx.x * per;
  double loc = 0.0;
  for (int j = 0; j < per; ++j) if (s0 + j < Q) loc += cand[s0 + j];
  double tot;
  double ex = block_exclusive_scan<double, BLOCK>(loc, red, &tot);
  for (int j = 0; j < per; ++j) if (s0 + j < Q) { pref[s0 + j] = ex; ex += cand[s0 + j]; }
  if (threadIdx.x == 0) pref[Q] = tot;
  __syncthreads();
}

// Phi evaluated from the sorted candidate list (valid for theta >= floor).
struct PhiEval {
  double phi;
  int nA, nB;
  double SA, SB;
};

__device__ __forceinline__ PhiEval phi_sorted(double th, const double* cand, const double* pref,
                                              int q, int Q, double rho, double M) {
  // top member t is active iff a_t < h(theta) = theta + min(rho theta, M) (h is the
  // inverse of top_break); all values are non-negative, so the searches compare bits
  const double h = th + fmin(rho * th, M);
  const unsigned long long hb = nnbits(h), tb = nnbits(th);
  const unsigned long long* cb = reinterpret_cast<const unsigned long long*>(cand);
  // t0: first t in [0,q) with cand[t] < h (cand descending)
  int lo = 0, hi = q;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cb[mid] < hb) hi = mid; else lo = mid + 1;
  }
  const int t0 = lo;
  // j0: first j in [q,Q) with cand[j] <= th
  lo = q; hi = Q;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cb[mid] <= tb) hi = mid; else lo = mid + 1;
  }
  const int j0 = lo;
  PhiEval e;
  e.nA = q - t0;
  e.SA = pref[q] - pref[t0];
  e.nB = j0 - q;
  e.SB = pref[j0] - pref[q];
  e.phi = (double)e.nA * h - e.SA - (e.SB - (double)e.nB * th);
  return e;
}

// Root of the linear piece with the given active sets.
__device__ __forceinline__ double solve_piece(int nA, double SA, int nB, double SB, bool rho_branch,
                                              double rho, double M) {
  if (rho_branch) return (SA + SB) / ((double)nA * (1.0 + rho) + (double)nB);
  return (SA + SB - (double)nA * M) / (double)(nA + nB);
}

// Bracket the root on the sorted candidates.  Returns false if the root lies
// below `floorv` (more candidates needed).  All threads call it.  The top
// breakpoints, M/rho and the floor are evaluated one per thread; the tail
// breakpoints cand[q..Q) (descending, all >= floorv) have Phi(cand[j])
// non-increasing in j, so the first j with Phi <= 0 is found by a BLOCK-ary
// search (two rounds for Q <= BLOCK^2) instead of evaluating every one.
template <int BLOCK>
__device__ bool root_from_sorted(const double* cand, const double* pref, int q, int Q, double floorv,
                                 double rho, double M, double* red, int* sh, double* theta_out) {
  const double thM = M / rho;
  double lo = -1.0, hi = INFINITY;
  for (int e = threadIdx.x; e < q + 2; e += BLOCK) {
    double th;
    if (e < q) th = top_break(cand[e], rho, M);
    else if (e == q) th = floorv;
    else th = thM;
    if (th < floorv) continue;
    PhiEval v = phi_sorted(th, cand, pref, q, Q, rho, M);
    if (v.phi <= 0.0) lo = fmax(lo, th);
    if (v.phi >= 0.0) hi = fmin(hi, th);
  }
  // J: first j in [q, Q) with Phi(cand[j]) <= 0, or Q.  Invariant: J in [a, b],
  // Phi(cand[j]) > 0 for j < a.
  int a = q, b = Q;
  while (a < b) {
    const int len = b - a;
    const int step = (len + BLOCK - 1) / BLOCK;
    const int j = a + (int)threadIdx.x * step;
    int first = b;
    if (j < b && phi_sorted(cand[j], cand, pref, q, Q, rho, M).phi <= 0.0) first = j;
    first = block_min<int, BLOCK>(first, sh, b);
    if (first < b) {
      const int na = first - step + 1;
      a = na > a ? na : a;
      b = first;
    } else {
      a = a + ((len - 1) / step) * step + 1;
    }
  }
  const int J = a;
  if (J < Q) {
    lo = fmax(lo, cand[J]);
    if (phi_sorted(cand[J], cand, pref, q, Q, rho, M).phi >= 0.0) hi = fmin(hi, cand[J]);
  }
  if (J > q) hi = fmin(hi, cand[J - 1]);
  lo = block_max<double, BLOCK>(lo, red, -1.0);
  hi = block_min<double, BLOCK>(hi, red, INFINITY);
  if (lo < floorv) return false;  // Phi(floor) > 0: the pooled block extends below the candidates
  double th;
  if (!(hi > lo)) {
    th = hi <= lo ? (isinf(hi) ? lo : hi) : lo;
  } else {
    const double mid = 0.5 * (lo + hi);
    PhiEval v = phi_sorted(mid, cand, pref, q, Q, rho, M);
    th = solve_piece(v.nA, v.SA, v.nB, v.SB, rho * mid < M, rho, M);
    th = fmin(fmax(th, lo), hi);
  }
  *theta_out = th;
  return true;
}

// ------------------------------------------------------------------------
// Appending to a shared list: one shared-memory atomic per warp (a leader adds
// the warp's count) instead of one per element, which serialised on the single
// counter when thousands of coordinates qualified.  Every lane of the warp must
// call it (take = false for lanes with nothing to add); returns the lane's slot
// or -1.
__device__ __forceinline__ int warp_append(bool take, int* counter) {
  const unsigned bal = __ballot_sync(0xffffffffu, take);
  if (bal == 0u) return -1;
  const int lane = threadIdx.x & 31, leader = __ffs(bal) - 1;
  int base = 0;
  if (lane == leader) base = atomicAdd(counter, __popc(bal));
  base = __shfl_sync(0xffffffffu, base, leader);
  return take ? base + __popc(bal & ((1u << lane) - 1u)) : -1;
}

// ------------------------------------------------------------------------
// The prox of one segment.

template <typename T>
struct SegIO {
  int m;
  const int8_t* state;       // nullptr: all coordinates free
  const T* w;                // direct input, or nullptr to form w from the FISTA state:
  const T* bc;               //   gamma = bc + c (bc - bp);  w = gamma - grad / L
  const T* bp;
  const double* grad;         // FP64 gradient, or
  const float* gradf;         //   FP32 gradient (batched solves)
  double c, invL;
  double rho, M;
  int kp;
  T* wbuf;                   // global scratch (length m) used when sm.wsm == nullptr
  T* beta;                   // output, length m
  int* nnz_idx;              // optional ordered compaction of beta's nonzeros
  T* nnz_val;
  int nnz_cap;               // 0: do not compact
  int* top_out;              // optional: the top-k' indices in sorted order
  int qhint;                 // candidates to start from; above the capacity: full pass
  double theta0;             // previous theta (warm start of the full pass), or <= 0
  double topk_hint = 0.0;    // previous k'-th largest |w| (> 0: gather above it first), or <= 0
};

struct SegOut {
  double g, theta, l1, sbar;
  double topk;               // this call's k'-th largest |w| (the next call's topk_hint)
  int nnz, qused, fallback;
};

// Full-pass root of Phi, for pooled blocks wider than the candidate capacity.
// T members: keys > thr_k plus need_k of the keys equal to thr_k; tail: the rest.
// Each pass evaluates Phi at theta from all m keys (integer compares on the key
// bits; FP64 adds only for the active keys) together with the nearest keys on
// either side of theta (tail) and of h(theta) (top): these bound the linear piece
// of Phi through theta.  The Newton point c of that piece is Phi's root when no
// breakpoint separates c from theta, which ends the iteration (usually one or two
// passes from the previous step's theta); otherwise c, or the bisection point
// when c leaves the bracket, is the next theta.  Phi(0) <= 0 <= Phi(hi0).
// scratch: >= (BLOCK/32 + 2) * 8 64-bit words of shared memory; dsum: 2 BLOCK
// doubles of shared memory (the candidates' prefix-sum buffer, free here).
// *nb_out: the active tail count at the root.
template <int BLOCK, typename KeyBits>
__device__ double root_fullpass(int m, KeyBits keybits, double thr_k, int need_k, int eq_k, double hi0,
                                double th0, double rho, double M, unsigned long long* scratch, double* dsum,
                                int* nb_out) {
  // FP64 issues at 1/64 of the FP32 rate here: the FP64 sums go through shared
  // memory (dsum: 2 BLOCK doubles) to one warp (each value added once), and thread
  // 0 alone runs the scalar Newton / bisection logic, broadcasting the next point's
  // bit patterns
  using ULL = unsigned long long;
  constexpr int NW = BLOCK / 32;
  static_assert((NW + 2) * 8 <= 1024, "root_fullpass scratch: the 2048-word histogram");
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  const ULL thr_b = nnbits(thr_k);
  ULL* wpart = scratch;                                        // NW x 8 warp partials
  ULL* bc = wpart + NW * 8;                                    // broadcast: th, h bits, done, nB
  // thread 0's state
  double lo = 0.0, hi = hi0, th = (th0 > 0.0 && th0 < hi0) ? th0 : hi0;
  if (threadIdx.x == 0) {
    bc[0] = nnbits(th);
    bc[1] = nnbits(th + fmin(rho * th, M));
    bc[2] = 0ull;
  }
  __syncthreads();
  for (int it = 0; it < 100; ++it) {
    const ULL tb = bc[0], hb = bc[1];
    long long nA = 0, nB = 0;
    double SA = 0.0, SB = 0.0;
    // tail: max key <= theta, min key > theta; top: max key < h, min key >= h
    ULL tl = 0ull, tg = ~0ull, al = 0ull, ag = ~0ull;
    for (int i = threadIdx.x; i < m; i += BLOCK) {
      const ULL kb = keybits(i);
      if (kb > thr_b) {
        if (kb < hb) { ++nA; SA += __longlong_as_double((long long)kb); al = kb > al ? kb : al; }
        else ag = kb < ag ? kb : ag;
      } else if (kb < thr_b) {
        if (kb > tb) { ++nB; SB += __longlong_as_double((long long)kb); tg = kb < tg ? kb : tg; }
        else tl = kb > tl ? kb : tl;
      }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      nA += __shfl_xor_sync(0xffffffffu, nA, o);
      nB += __shfl_xor_sync(0xffffffffu, nB, o);
      ULL v;
      v = __shfl_xor_sync(0xffffffffu, tl, o); tl = v > tl ? v : tl;
      v = __shfl_xor_sync(0xffffffffu, al, o); al = v > al ? v : al;
      v = __shfl_xor_sync(0xffffffffu, tg, o); tg = v < tg ? v : tg;
      v = __shfl_xor_sync(0xffffffffu, ag, o); ag = v < ag ? v : ag;
    }
    dsum[threadIdx.x] = SA;
    dsum[BLOCK + threadIdx.x] = SB;
    if (lane == 0) {
      ULL* w = wpart + wid * 8;
      w[0] = (ULL)nA; w[1] = (ULL)nB;
      w[4] = tl; w[5] = tg; w[6] = al; w[7] = ag;
    }
    __syncthreads();
    if (wid == 0) {   // fixed order: the same sums on every call
      double sa = 0.0, sb = 0.0;
      for (int k = lane; k < BLOCK; k += 32) { sa += dsum[k]; sb += dsum[BLOCK + k]; }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        sa += __shfl_xor_sync(0xffffffffu, sa, o);
        sb += __shfl_xor_sync(0xffffffffu, sb, o);
      }
      if (lane == 0) {
        long long a0 = 0, b0 = 0;
        ULL x4 = 0ull, x5 = ~0ull, x6 = 0ull, x7 = ~0ull;
        const ULL* w = wpart;
        for (int k = 0; k < NW; ++k, w += 8) {
          a0 += (long long)w[0]; b0 += (long long)w[1];
          x4 = w[4] > x4 ? w[4] : x4; x5 = w[5] < x5 ? w[5] : x5;
          x6 = w[6] > x6 ? w[6] : x6; x7 = w[7] < x7 ? w[7] : x7;
        }
        // the keys equal to thr_k: need_k of them in the top set, eq_k - need_k in the tail
        if (need_k > 0) {
          if (thr_b < hb) { a0 += need_k; sa += (double)need_k * thr_k; x6 = thr_b > x6 ? thr_b : x6; }
          else x7 = thr_b < x7 ? thr_b : x7;
        }
        if (eq_k > need_k) {
          if (thr_b > tb) { b0 += eq_k - need_k; sb += (double)(eq_k - need_k) * thr_k; x5 = thr_b < x5 ? thr_b : x5; }
          else x4 = thr_b > x4 ? thr_b : x4;
        }
        const double h = __longlong_as_double((long long)hb);
        const double phi = (double)a0 * h - sa - (sb - (double)b0 * th);
        ULL done = 0ull;
        double res = th;
        if (phi == 0.0) {
          done = 1ull;
        } else {
          if (phi < 0.0) lo = th; else hi = th;
          const bool rb = rho * th < M;
          const double c = solve_piece((int)a0, sa, (int)b0, sb, rb, rho, M);
          if (a0 + b0 > 0 && c > lo && c < hi) {
            const double hc = c + fmin(rho * c, M);
            const ULL cb = nnbits(c), hcb = nnbits(hc);
            bool same = (rho * c < M) == rb;
            if (c < th) same = same && x4 <= cb && x6 < hcb;   // no key in (c, th] (tail) or [h(c), h(th)) (top)
            else same = same && x5 > cb && x7 >= hcb;         // no key in (th, c] (tail) or [h(th), h(c)) (top)
            if (same) { done = 1ull; res = c; }
            th = c;
          } else {
            th = 0.5 * (lo + hi);
          }
          if (!done && !(hi - lo > 2e-16 * hi)) { done = 1ull; res = hi; }
          if (!done && it == 99) { done = 1ull; res = th; }
        }
        bc[0] = nnbits(done ? res : th);
        bc[1] = nnbits(th + fmin(rho * th, M));
        bc[2] = done;
        bc[3] = (ULL)b0;
      }
    }
    __syncthreads();
    if (bc[2]) {
      const double r = __longlong_as_double((long long)bc[0]);
      *nb_out = (int)(long long)bc[3];
      __syncthreads();
      return r;
    }
  }
  return __longlong_as_double((long long)bc[0]);
}

template <typename T, int BLOCK>
__device__ SegOut prox_segment(const SegIO<T>& io, const SegSmem<T>& sm) {
  static_assert(sizeof(T) == 8, "prox_segment: FP64 segments (64-bit key bits)");
  using B = Bits<T>;
  using U = typename B::U;
  const int m = io.m;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  // a direct input with every coordinate free is read in place (no copy)
  const bool direct = io.w != nullptr && io.state == nullptr && sm.wsm == nullptr && io.wbuf == nullptr;
  T* wv = direct ? const_cast<T*>(io.w) : (sm.wsm ? sm.wsm : io.wbuf);
  const double rho = io.rho, M = io.M;

  // pass 1: w (rounded to T), the fixed coordinates' outputs
  double s1sq = 0.0;
  for (int i = direct ? m : threadIdx.x; i < m; i += BLOCK) {
    double w;
    if (io.w) w = to_d(io.w[i]);
    else {
      const double b = to_d(io.bc[i]);
      const double gi = io.grad ? io.grad[i] : (double)io.gradf[i];
      w = b + io.c * (b - to_d(io.bp[i])) - gi * io.invL;
    }
    const int8_t st = io.state ? io.state[i] : (int8_t)kFree;
    if (st == kFree) {
      wv[i] = (T)w;
    } else {
      wv[i] = T(0);
      if (st == kZero) {
        io.beta[i] = T(0);
      } else {  // z_j = 1: argmin 1/2 (b - w)^2 + 1/(2 rho) b^2 on the box
        double b = fmin(fmax(rho * w / (1.0 + rho), -M), M);
        T bt = (T)b;
        io.beta[i] = bt;
        s1sq += to_d(bt) * to_d(bt);
      }
    }
  }
  s1sq = block_sum<double, BLOCK>(s1sq, sm.red);

  auto keybits = [&](int i) -> U { return abs_bits<T>(wv[i]); };
  auto keyval = [&](int i) -> double { return fabs(to_d(wv[i])); };

  SegOut out;
  out.fallback = 0;
  out.qused = 0;
  const int kp = io.kp;
  const int q = kp < m ? kp : m;
  double thr_k = INFINITY;
  int need_k = 0, eq_k = 0;
  double theta = INFINITY;   // k' = 0: every free coordinate is soft-thresholded to 0
  bool cand_sorted = false;  // cand[0..q) holds the top-q values, descending

  out.topk = 0.0;
  if (q > 0) {
    // the k'-th largest |w|: from the keys at or above 0.99 times the previous
    // call's (one pass to gather them; the top set moves little between FISTA
    // steps) when they number at least k' and fit the candidates, else by radix
    // passes over all m.  Both give the same threshold and counts: every key equal
    // to it or above is among the gathered ones.
    SelectResult<U> Rk;
    bool have = false;
    if (io.topk_hint > 0.0 && q < m) {
      const U fk = abs_bits<T>((T)(0.99 * io.topk_hint));
      if (threadIdx.x == 0) sm.sh[40] = 0;
      __syncthreads();
      for (int i0 = 0; i0 < m; i0 += BLOCK) {   // warp-uniform trip count (warp_append)
        const int i = i0 + (int)threadIdx.x;
        const U kb = i < m ? keybits(i) : U(0);
        const int pos = warp_append(i < m && kb >= fk, &sm.sh[40]);
        if (pos >= 0 && pos < sm.cap) sm.cand[pos] = to_d(B::val(kb));
      }
      __syncthreads();
      const int cnt = sm.sh[40];
      __syncthreads();
      if (cnt >= q && cnt <= sm.cap) {
        auto cbits = [&](int j) -> U { return abs_bits<T>((T)sm.cand[j]); };
        Rk = block_select<U, BLOCK>(cnt, q, cbits, sm.hist, sm.sh);
        have = true;
      }
    }
    if (!have) Rk = block_select<U, BLOCK>(m, q, keybits, sm.hist, sm.sh);
    thr_k = to_d(B::val(Rk.thr));
    out.topk = thr_k;
    need_k = q - Rk.gt;
    eq_k = Rk.eq;
    if (q == m) {
      theta = 0.0;  // no tail: no isotonic violation
    } else {
      int Q = io.qhint > q + 1 ? io.qhint : q + 1;
      if (Q > m) Q = m;
      // the previous call's pooled tail did not fit the candidates: straight to the full pass
      const bool wide = Q > sm.cap;
      bool found = false;
      double last_floor = INFINITY;
      while (!wide && !found && Q <= sm.cap) {
        double floorv = 0.0;
        if (Q < m) {
          SelectResult<U> RQ = block_select<U, BLOCK>(m, Q, keybits, sm.hist, sm.sh);
          floorv = to_d(B::val(RQ.thr));
          if (threadIdx.x == 0) sm.sh[40] = 0;
          __syncthreads();
          for (int i0 = 0; i0 < m; i0 += BLOCK) {
            const int i = i0 + (int)threadIdx.x;
            const U kb = i < m ? keybits(i) : U(0);
            const int pos = warp_append(i < m && kb > RQ.thr, &sm.sh[40]);
            if (pos >= 0) sm.cand[pos] = to_d(B::val(kb));
          }
          __syncthreads();
          for (int j = RQ.gt + threadIdx.x; j < Q; j += BLOCK) sm.cand[j] = floorv;
        } else {
          for (int i = threadIdx.x; i < m; i += BLOCK) sm.cand[i] = keyval(i);
        }
        const int N = next_pow2(Q);
        for (int j = Q + threadIdx.x; j < N; j += BLOCK) sm.cand[j] = 0.0;
        __syncthreads();
        sort_desc_nonneg<BLOCK>(sm.cand, N);
        block_prefix<BLOCK>(sm.cand, sm.pref, Q, sm.red);
        found = root_from_sorted<BLOCK>(sm.cand, sm.pref, q, Q, floorv, rho, M, sm.red, sm.sh, &theta);
        out.qused = Q;
        last_floor = floorv;
        if (!found) {
          if (Q == m) break;  // cannot happen: Phi(0) <= 0
          Q = (4 * Q < m) ? 4 * Q : m;
        }
      }
      if (found) {
        cand_sorted = true;
        // the next call's candidate count: the top set, twice the pooled tail found
        // here, and a margin (the pooled block moves little between FISTA steps)
        int lo2 = q, hi2 = out.qused;
        while (lo2 < hi2) {
          const int mid = (lo2 + hi2) >> 1;
          if (sm.cand[mid] <= theta) hi2 = mid; else lo2 = mid + 1;
        }
        const int next = q + 2 * (lo2 - q) + 32;
        out.qused = next < out.qused ? next : out.qused;
      } else {
        out.fallback = 1;
        int nb = 0;
        // Phi(last_floor) > 0 when the candidates were tried; Phi(thr_k) >= 0 always
        const double hi0 = isinf(last_floor) ? thr_k : last_floor;
        theta = root_fullpass<BLOCK>(m, keybits, thr_k, need_k, eq_k, hi0, io.theta0, rho, M,
                                     reinterpret_cast<unsigned long long*>(sm.hist), sm.pref, &nb);
        // the pooled tail at the root sizes the next call (above the capacity: full pass again)
        out.qused = q + 2 * nb + 32;
      }
    }
  }
  out.theta = theta;

  // ---- ordered passes: warp w owns the contiguous chunk [w*chunk, (w+1)*chunk)
  const int nw = BLOCK / 32;
  const int chunk = (((m + nw - 1) / nw) + 31) & ~31;
  const int c0 = wid * chunk;
  const int c1 = min(m, c0 + chunk);
  const bool tie_split = (q > 0) && (need_k < eq_k);
  int tie_base = 0;
  if (tie_split) {  // rank of tied keys in index order
    int cnt = 0;
    for (int base = c0; base < c1; base += 32) {
      const int i = base + lane;
      const bool t = (i < c1) && keyval(i) == thr_k && (io.state == nullptr || io.state[i] == kFree);
      cnt += __popc(__ballot_sync(0xffffffffu, t));
    }
    int tot;
    int ex = block_exclusive_scan<int, BLOCK>(lane == 0 ? cnt : 0, sm.sh, &tot);
    tie_base = __shfl_sync(0xffffffffu, ex, 0);
  }
  // main output pass.  Magnitudes and thresholds are non-negative, so the
  // membership tests compare bit patterns; FP64 arithmetic runs only for the
  // coordinates that come out nonzero (the top set and the tail above theta).
  const double shrink = rho / (1.0 + rho);
  const unsigned long long thr_b = nnbits(thr_k), theta_b = nnbits(theta);
  double l1 = 0.0;
  int nzc = 0, tie_run = 0;
  for (int base = c0; base < c1; base += 32) {
    const int i = base + lane;
    const bool valid = i < c1;
    const int8_t st = (valid && io.state) ? io.state[i] : (int8_t)kFree;
    const T wt = valid ? wv[i] : T(0);
    const unsigned long long ab = valid ? (unsigned long long)abs_bits<T>(wt) : 0ull;   // |w| bits, integer ops
    bool tie = valid && st == kFree && q > 0 && ab == thr_b;
    int tie_rank = 0;
    if (tie_split) {
      const unsigned bal = __ballot_sync(0xffffffffu, tie);
      tie_rank = tie_base + tie_run + __popc(bal & ((1u << lane) - 1u));
      tie_run += __popc(bal);
    }
    bool nz = false;
    if (valid) {
      if (st == kFree) {
        const bool in_top = (q > 0) && (ab > thr_b || (tie && (!tie_split || tie_rank < need_k)));
        double mag = 0.0;
        if (in_top || ab > theta_b) {
          const double a = fabs(to_d(wt));
          mag = in_top ? fmin(fmin(M, shrink * a), a - theta) : a - theta;
          if (!(mag > 0.0)) mag = 0.0;
        }
        T bt = T(0);
        if (mag > 0.0) {
          bt = (T)(to_d(wt) < 0 ? -mag : mag);
          l1 += fabs(to_d(bt));
          nz = true;
        }
        io.beta[i] = bt;
      } else {
        nz = to_d(io.beta[i]) != 0.0;
      }
    }
    nzc += __popc(__ballot_sync(0xffffffffu, nz));
  }
  l1 = block_sum<double, BLOCK>(l1, sm.red);
  {
    int tot;
    int ex = block_exclusive_scan<int, BLOCK>(lane == 0 ? nzc : 0, sm.sh, &tot);
    const int nz_base = __shfl_sync(0xffffffffu, ex, 0);
    out.nnz = tot;
    if (io.nnz_cap > 0 && tot <= io.nnz_cap) {
      __syncthreads();
      int run = 0;
      for (int base = c0; base < c1; base += 32) {
        const int i = base + lane;
        T v = (i < c1) ? io.beta[i] : T(0);
        const bool nz = to_d(v) != 0.0;
        const unsigned bal = __ballot_sync(0xffffffffu, nz);
        if (nz) {
          const int pos = nz_base + run + __popc(bal & ((1u << lane) - 1u));
          io.nnz_idx[pos] = i;
          io.nnz_val[pos] = v;
        }
        run += __popc(bal);
      }
    }
  }
  out.l1 = l1;

  // ---- g(beta) (Algorithm 2) on the prox output: the top-k' of |beta| are the
  // top-k' of |w| (the prox preserves the order of the magnitudes), and
  // |b_t| = min(M, rho a_t/(1+rho), a_t - theta) is monotone in a_t.
  double g = 0.5 * s1sq, sbar = 0.0;
  if (q > sm.cap) g = NAN;  // the host rejects k' beyond the candidate capacity
  if (q > 0 && q <= sm.cap) {
    if (!cand_sorted) {  // gather the top-q values and sort them
      if (threadIdx.x == 0) sm.sh[40] = 0;
      __syncthreads();
      const U tb = B::of((T)thr_k);
      for (int i0 = 0; i0 < m; i0 += BLOCK) {
        const int i = i0 + (int)threadIdx.x;
        const U kb = i < m ? keybits(i) : U(0);
        const int pos = warp_append(i < m && kb > tb, &sm.sh[40]);
        if (pos >= 0) sm.cand[pos] = to_d(B::val(kb));
      }
      __syncthreads();
      for (int j = (q - need_k) + threadIdx.x; j < q; j += BLOCK) sm.cand[j] = thr_k;
      const int N = next_pow2(q);
      for (int j = q + threadIdx.x; j < N; j += BLOCK) sm.cand[j] = 0.0;
      __syncthreads();
      sort_desc_nonneg<BLOCK>(sm.cand, N);
    }
    // |b_t| into cand (in place), prefix sums in pref
    for (int t = threadIdx.x; t < q; t += BLOCK) {
      const double a = sm.cand[t];
      double mg = fmin(fmin(M, shrink * a), a - theta);
      sm.cand[t] = mg > 0.0 ? to_d((T)mg) : 0.0;
    }
    __syncthreads();
    block_prefix<BLOCK>(sm.cand, sm.pref, q, sm.red);
    int jst = q;
    for (int j = threadIdx.x; j < q; j += BLOCK) {
      const double sb = (l1 - sm.pref[j]) / (double)(kp - j);
      if (sb >= sm.cand[j]) jst = min(jst, j);
    }
    jst = block_min<int, BLOCK>(jst, sm.sh, q);
    double sq = 0.0;
    for (int j = threadIdx.x; j < jst; j += BLOCK) sq += sm.cand[j] * sm.cand[j];
    sq = block_sum<double, BLOCK>(sq, sm.red);
    sbar = (jst < kp) ? fmax(0.0, (l1 - sm.pref[jst]) / (double)(kp - jst)) : 0.0;
    g += 0.5 * (sq + (double)(kp - jst) * sbar * sbar);
  }
  out.g = g;
  out.sbar = sbar;

  // ---- optional: the top-k' indices in sorted order (stable: ties by index)
  if (io.top_out && q > 0 && q <= sm.cap) {
    if (threadIdx.x == 0) sm.sh[40] = 0;
    __syncthreads();
    // members: keys > thr_k, plus the first need_k tied keys in index order
    int run = 0;
    for (int base = c0; base < c1; base += 32) {
      const int i = base + lane;
      const bool valid = i < c1;
      const bool fr = valid && (io.state == nullptr || io.state[i] == kFree);
      const double a = valid ? keyval(i) : 0.0;
      const bool tie = fr && a == thr_k;
      const unsigned bal = __ballot_sync(0xffffffffu, tie);
      const int rank = tie_base + run + __popc(bal & ((1u << lane) - 1u));
      run += __popc(bal);
      const bool mem = fr && (a > thr_k || (tie && (!tie_split || rank < need_k)));
      const int pos = warp_append(mem, &sm.sh[40]);
      if (pos >= 0) {
        sm.cand[pos] = a;
        sm.cidx[pos] = i;
      }
    }
    __syncthreads();
    const int N = next_pow2(q);
    for (int j = q + threadIdx.x; j < N; j += BLOCK) { sm.cand[j] = 0.0; sm.cidx[j] = 0x7fffffff; }
    __syncthreads();
    // bitonic sort of (value desc, index asc)
    for (int size = 2; size <= N; size <<= 1) {
      for (int stride = size >> 1; stride > 0; stride >>= 1) {
        for (int i = threadIdx.x; i < (N >> 1); i += BLOCK) {
          const int lo = 2 * i - (i & (stride - 1));
          const int hi = lo + stride;
          const bool desc = ((lo & size) == 0);
          const double a = sm.cand[lo], b = sm.cand[hi];
          const unsigned long long ab = nnbits(a), bb = nnbits(b);
          const int ia = sm.cidx[lo], ib = sm.cidx[hi];
          const bool a_before_b = (ab > bb) || (ab == bb && ia < ib);
          if (a_before_b != desc) {
            sm.cand[lo] = b; sm.cand[hi] = a; sm.cidx[lo] = ib; sm.cidx[hi] = ia;
          }
        }
        __syncthreads();
      }
    }
    for (int t = threadIdx.x; t < q; t += BLOCK) io.top_out[t] = sm.cidx[t];
    __syncthreads();
  }
  return out;
}

// ------------------------------------------------------------------------
// g(beta) of a node by Algorithm 2 (partial sort to the top k', water-filling).
// Optionally the relaxed z (from the proof of Thm 3.6): z_j = min(1, |b_j|/sbar)
// on the free coordinates, 1 on S1, 0 on S0.

struct GOut {
  double g, sbar, l1;
  int infeasible;
};

// slack: relative tolerance of the domain test (|b| <= M, sum|b| <= k'M) for an
// iterate stored in a narrower type than FP64.
template <typename T, int BLOCK, typename LoadB>
__device__ GOut gvalue_segment(int m, LoadB loadb, const int8_t* state, int kp, double M,
                               const SegSmem<T>& sm, double* z_out, double slack = 1e-12) {
  using B = Bits<double>;
  using U = typename B::U;
  double l1 = 0.0, s1sq = 0.0, linf = 0.0;
  int bad = 0;
  for (int i = threadIdx.x; i < m; i += BLOCK) {
    const int8_t st = state ? state[i] : (int8_t)kFree;
    const double b = loadb(i);
    if (st == kFree) { l1 += fabs(b); linf = fmax(linf, fabs(b)); }
    else if (st == kOne) { s1sq += b * b; linf = fmax(linf, fabs(b)); }
    else if (b != 0.0) bad = 1;
  }
  l1 = block_sum<double, BLOCK>(l1, sm.red);
  s1sq = block_sum<double, BLOCK>(s1sq, sm.red);
  linf = block_max<double, BLOCK>(linf, sm.red, 0.0);
  bad = block_max<int, BLOCK>(bad, sm.sh, 0);
  GOut o;
  o.l1 = l1;
  o.sbar = 0.0;
  o.infeasible = 0;
  const double kM = (double)(kp > 0 ? kp : 0) * M;
  if (bad || kp < 0 || linf > M * (1.0 + slack) || l1 > kM * (1.0 + slack)) {
    o.infeasible = 1;
    o.g = INFINITY;
  } else {
    double g = 0.5 * s1sq, sbar = 0.0;
    const int q = kp < m ? kp : m;
    if (q > sm.cap) g = NAN;  // the host rejects k' beyond the candidate capacity
    if (q > 0 && q <= sm.cap) {
      auto keybits = [&](int i) -> U {
        const int8_t st = state ? state[i] : (int8_t)kFree;
        return st == kFree ? B::of(fabs(loadb(i))) : (U)0;
      };
      SelectResult<U> R = block_select<U, BLOCK>(m, q, keybits, sm.hist, sm.sh);
      if (threadIdx.x == 0) sm.sh[40] = 0;
      __syncthreads();
      for (int i0 = 0; i0 < m; i0 += BLOCK) {
        const int i = i0 + (int)threadIdx.x;
        const U kb = i < m ? keybits(i) : U(0);
        const int pos = warp_append(i < m && kb > R.thr, &sm.sh[40]);
        if (pos >= 0) sm.cand[pos] = B::val(kb);
      }
      __syncthreads();
      const double thr = B::val(R.thr);
      for (int j = R.gt + threadIdx.x; j < q; j += BLOCK) sm.cand[j] = thr;
      const int N = next_pow2(q);
      for (int j = q + threadIdx.x; j < N; j += BLOCK) sm.cand[j] = 0.0;
      __syncthreads();
      sort_desc_nonneg<BLOCK>(sm.cand, N);
      block_prefix<BLOCK>(sm.cand, sm.pref, q, sm.red);
      int jst = q;
      for (int j = threadIdx.x; j < q; j += BLOCK) {
        const double sb = (l1 - sm.pref[j]) / (double)(kp - j);
        if (sb >= sm.cand[j]) jst = min(jst, j);
      }
      jst = block_min<int, BLOCK>(jst, sm.sh, q);
      double sq = 0.0;
      for (int j = threadIdx.x; j < jst; j += BLOCK) sq += sm.cand[j] * sm.cand[j];
      sq = block_sum<double, BLOCK>(sq, sm.red);
      sbar = (jst < kp) ? fmax(0.0, (l1 - sm.pref[jst]) / (double)(kp - jst)) : 0.0;
      g += 0.5 * (sq + (double)(kp - jst) * sbar * sbar);
    }
    o.g = g;
    o.sbar = sbar;
  }
  if (z_out) {
    for (int i = threadIdx.x; i < m; i += BLOCK) {
      const int8_t st = state ? state[i] : (int8_t)kFree;
      const double b = fabs(loadb(i));
      double z;
      if (st == kOne) z = 1.0;
      else if (st == kZero) z = 0.0;
      else if (o.sbar > 0.0) z = fmin(1.0, b / o.sbar);
      else z = b > 0.0 ? 1.0 : 0.0;
      z_out[i] = z;
    }
  }
  __syncthreads();
  return o;
}

// ------------------------------------------------------------------------
// TopSum_{k'}(H_M(|a_F| * scale)) + sum_{S1} H_M(|a_j| * scale)   (Lemma 3.1 on
// the node, with the separable-sum rule for S1).  Keys are read in T.

// hint (> 0): the previous call's k'-th largest |a_F|; every free |a_j| at or above
// 0.99 hint is gathered in one pass, and when at least k' of them (and at most the
// candidate capacity) are found the selection runs on those in shared memory
// instead of in radix passes over all m.  *thr_out (optional): this call's k'-th
// largest |a_F|, the next call's hint.
template <typename T, int BLOCK, typename LoadA>
__device__ double gstar_segment(int m, LoadA loada, const int8_t* state, int kp, double M,
                                double scale, const SegSmem<T>& sm, double hint = 0.0,
                                double* thr_out = nullptr) {
  using B = Bits<T>;
  using U = typename B::U;
  double s1 = 0.0;
#pragma unroll 4
  for (int i = threadIdx.x; i < m; i += BLOCK)
    if (state && state[i] == kOne) s1 += huber(fabs(to_d(loada(i))) * scale, M);
  s1 = block_sum<double, BLOCK>(s1, sm.red);
  const int q = kp < m ? kp : m;
  if (q <= 0) return s1;
  auto keybits = [&](int i) -> U {
    const int8_t st = state ? state[i] : (int8_t)kFree;
    return st == kFree ? abs_bits<T>(loada(i)) : (U)0;
  };
  if (hint > 0.0) {
    const U fk = abs_bits<T>((T)(0.99 * hint));
    if (threadIdx.x == 0) sm.sh[40] = 0;
    __syncthreads();
    for (int i0 = 0; i0 < m; i0 += BLOCK) {
      const int i = i0 + (int)threadIdx.x;
      const U kb = i < m ? keybits(i) : U(0);
      const int pos = warp_append(i < m && kb >= fk, &sm.sh[40]);
      if (pos >= 0 && pos < sm.cap) sm.cand[pos] = to_d(B::val(kb));
    }
    __syncthreads();
    const int cnt = sm.sh[40];
    __syncthreads();
    if (cnt >= q && cnt <= sm.cap) {
      auto cbits = [&](int j) -> U { return abs_bits<T>((T)sm.cand[j]); };
      SelectResult<U> R = block_select<U, BLOCK>(cnt, q, cbits, sm.hist, sm.sh);
      const double thr = to_d(B::val(R.thr));
      double s = 0.0;
      for (int j = threadIdx.x; j < cnt; j += BLOCK) {
        const U kb = cbits(j);
        if (kb > R.thr) s += huber(sm.cand[j] * scale, M);
      }
      s = block_sum<double, BLOCK>(s, sm.red);
      if (thr_out) *thr_out = thr;
      return s1 + s + (double)(q - R.gt) * huber(thr * scale, M);
    }
  }
  SelectResult<U> R = block_select<U, BLOCK>(m, q, keybits, sm.hist, sm.sh);
  const double thr = to_d(B::val(R.thr));
  double s = 0.0;
#pragma unroll 4
  for (int i = threadIdx.x; i < m; i += BLOCK) {
    U kb = keybits(i);
    if (kb > R.thr) s += huber(to_d(B::val(kb)) * scale, M);
  }
  s = block_sum<double, BLOCK>(s, sm.red);
  if (thr_out) *thr_out = thr;
  return s1 + s + (double)(q - R.gt) * huber(thr * scale, M);
}

}  // namespace ksc
