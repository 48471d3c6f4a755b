// k_batch.cu -- the per-node kernels of a batched FISTA step (Algorithm 3 over B
// nodes of one problem).  Between them run the two tensor-core products of
// k_tcgemm.cu, each on a difference from the node's anchor (ksc_batch.cuh):
//
//   k_bresid   u_gamma = u_t + c (u_t - u_{t-1}) (linearity: no extra pass over X),
//              r - r_ref = grad F(u_gamma) - grad F(u_ref) without cancellation,
//              its BF16 pieces, and the terms of -F*(-zeta_gamma),
//              zeta_gamma = -grad F(u_gamma) (App. D.1), per CTA
//   [tensor]   G = G_ref + X^T (r - r_ref)                       (FP64 out)
//   k_bprox    one CTA per node: w = gamma - G/L, the exact prox of g_node (block
//              radix select + bitonic sort + breakpoint scan, Alg. 1 + 4 in the
//              threshold form), g(beta^{t+1}) (Alg. 2), the in-loop dual term
//              G*(X^T zeta_gamma) (Lemma 3.1 on the node), and the BF16 pieces of
//              beta^{t+1} - beta_ref
//   [tensor]   u^{t+1} = u_ref + X (beta^{t+1} - beta_ref) (FP64), partials of
//              F(u^{t+1}) and of its change F(u^{t+1}) - F(u^t)
//   k_bstep    the restart test on L^{t+1} - L^t (a sum of changes, free of the
//              cancellation of two nearly equal objective values) and the gap
//              test per node (the step logic shared with the single-node solver)
#include "ksc_batch.cuh"
#include "ksc_common.cuh"
#include "ksc_tc.h"
#include "ksc_prox.cuh"
#include "ksc_state.cuh"

namespace ksc {

// ------------------------------------------------------------------ helpers

// v = hi + mid + lo exactly (P = 3): each remainder is exact in FP32 and holds at
// most 16, then 8, significant bits
__device__ __forceinline__ void split_store(float v, __nv_bfloat16* dst, size_t piece_stride, int P) {
  const __nv_bfloat16 h = __float2bfloat16_rn(v);
  dst[0] = h;
  if (P > 1) {
    const float r1 = __fsub_rn(v, __bfloat162float(h));
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    dst[piece_stride] = m;
    if (P > 2) dst[2 * piece_stride] = __float2bfloat16_rn(__fsub_rn(r1, __bfloat162float(m)));
  }
}

// E4M3 pieces of v (already scaled below 256 in magnitude): each piece is the
// E4M3 rounding (to nearest) of what the previous pieces left, which FP32 holds
// exactly; pieces kTcE4m3Hi.. are cut from that remainder times 2^kTcE4m3Shift
// (the product's second accumulator), so that no entry stops at the smallest
// E4M3 subnormal: the pieces carry v to about 2^-30 of 256
__device__ __forceinline__ void split8_store(float v, uint8_t* dst, size_t piece_stride) {
#pragma unroll
  for (int q = 0; q < kTcE4m3Pieces; ++q) {
    if (q == kTcE4m3Hi) v *= (float)(1 << kTcE4m3Shift);
    const __nv_fp8_e4m3 h(v);
    dst[q * piece_stride] = h.__x;
    v = __fsub_rn(v, float(h));
  }
}

// the power-of-two exponent e that puts amax * 2^e in [128, 256) (0 for 0)
__device__ __forceinline__ int e8_exponent(double amax) {
  if (!(amax > 0.0)) return 0;
  int ex;
  frexp(amax, &ex);   // amax = f 2^ex, f in [0.5, 1)
  const int e = 8 - ex;
  return e < -120 ? -120 : (e > 120 ? 120 : e);
}

__device__ __forceinline__ float softplusf(float x) { return fmaxf(x, 0.0f) + log1pf(expf(-fabsf(x))); }

__device__ __forceinline__ double sigmoid_d(double t) {
  return t >= 0 ? 1.0 / (1.0 + exp(-t)) : exp(t) / (1.0 + exp(t));
}

// F_i(u) in FP64
__device__ __forceinline__ double loss_d(double u, double y, int loss) {
  if (loss == kLossLsq) {
    const double r = u - y;
    return r * r;
  }
  if (loss == kLossSqHinge) {
    const double m = fmax(0.0, 1.0 - y * u);
    return m * m;
  }
  if (loss == kLossPoisson) return exp(u) - y * u;
  if (loss == kLossGamma) return y * exp(-u) + u;
  const double t = -y * u;
  return t > 0 ? t + log1p(exp(-t)) : log1p(exp(t));
}

// The represented matrix of E4M3 X in BF16: dst[r][c] = src[r][c] * scale (the
// scale of column c when per_col, else of row r), exact (4 significant bits times
// a power of two); the padding columns [cols, ld_dst) are zeroed
__global__ void __launch_bounds__(256) k_fp8_to_bf16(const __nv_fp8_e4m3* src, int64_t ld_src, int rows, int cols,
                                                     const float* scale, int per_col, __nv_bfloat16* dst,
                                                     int64_t ld_dst) {
  const int r = blockIdx.x;   // one CTA per row (rows can exceed the 65535 limit of grid y)
  for (int64_t c = threadIdx.x; c < ld_dst; c += 256) {
    float v = 0.0f;
    if (c < cols) v = float(src[(int64_t)r * ld_src + c]) * (per_col ? scale[c] : scale[r]);
    dst[(int64_t)r * ld_dst + c] = __float2bfloat16_rn(v);
  }
}

void launch_fp8_to_bf16(const void* src, int64_t ld_src, int rows, int cols, const float* scale, int per_col,
                        void* dst, int64_t ld_dst, cudaStream_t s) {
  k_fp8_to_bf16<<<rows, 256, 0, s>>>((const __nv_fp8_e4m3*)src, ld_src, rows, cols, scale, per_col,
                                     (__nv_bfloat16*)dst, ld_dst);
}

// ------------------------------------------------------------------ residual

__global__ void __launch_bounds__(kBThreads) k_bresid(BatchDev d) {
  __shared__ double red[64];
  const int b = blockIdx.y;
  const BNode* nd = d.nodes + b;
  if (nd->done != kRunning) return;
  const double c = nd->c;
  const double* Uc = d.U + ((size_t)b * 3 + nd->cur) * d.ldn;
  const double* Up = d.U + ((size_t)b * 3 + nd->prev) * d.ldn;
  const double* Ur = d.u_ref + (size_t)b * d.ldn;
  const size_t pstride = (size_t)d.Bpad * d.ldn;
  __nv_bfloat16* rrow = d.e8 ? nullptr : d.rpc + (size_t)b * d.ldn;
  float* rb = d.e8 ? d.rbuf + (size_t)b * d.ldn : nullptr;
  float amax = 0.0f;
  double nc = 0.0;
  const int i0 = blockIdx.x * kBThreads * kBRows;
#pragma unroll 2
  for (int r = 0; r < kBRows; ++r) {
    const int i = i0 + r * kBThreads + (int)threadIdx.x;
    if (i < d.n) {
      const double uc = __ldg(&Uc[i]);
      const double ug = uc + c * (uc - __ldg(&Up[i]));
      const double du = ug - __ldg(&Ur[i]);
      const float y = __ldg(&d.yf[i]);
      float dr, term;
      if (d.loss == kLossLsq) {
        dr = (float)(2.0 * du);                          // grad F = 2 (u - y)
        const double z = -2.0 * (ug - (double)y);        // zeta = -grad F (FP64: u - y cancels)
        nc += (double)y * z - 0.25 * z * z;              // -F*(-zeta), App. D.1
        term = 0.0f;
      } else if (d.loss == kLossSqHinge) {
        // grad F = -2 y max(0, 1 - y u): where both margins are positive the
        // difference is 2 (u - u_ref) exactly; elsewhere from the two margins
        const double mg = fmax(0.0, 1.0 - (double)y * ug);
        const double mr = fmax(0.0, 1.0 - (double)y * __ldg(&Ur[i]));
        dr = (mg > 0.0 && mr > 0.0) ? (float)(2.0 * du) : (float)(-2.0 * (double)y * (mg - mr));
        const double z = 2.0 * (double)y * mg;          // zeta = -grad F, y zeta = 2 m >= 0
        nc += (double)y * z - 0.25 * z * z;
        term = 0.0f;
      } else if (d.loss == kLossPoisson) {
        // grad F = e^u - y: the difference e^{u_ref} expm1(u - u_ref) without
        // cancellation (far from the anchor, where expm1 would overflow, the plain
        // difference, which has none to lose); -F*(-zeta) = e^u (1 - u)
        const float eg = expf((float)ug);
        dr = fabs(du) > 16.0 ? eg - expf((float)__ldg(&Ur[i])) : expf((float)__ldg(&Ur[i])) * expm1f((float)du);
        term = eg * (1.0f - (float)ug);
      } else if (d.loss == kLossGamma) {
        // grad F = 1 - y e^-u: the difference -y e^{-u_ref} expm1(-(u - u_ref));
        // with w = y e^-u, -F*(-zeta) = w (1 + u)
        const float wg = y * expf(-(float)ug);
        dr = fabs(du) > 16.0 ? -(wg - y * expf(-(float)__ldg(&Ur[i])))
                             : -y * expf(-(float)__ldg(&Ur[i])) * expm1f(-(float)du);
        term = wg * (1.0f + (float)ug);
      } else {
        // grad F = -y sigma(t), t = -y u;  sigma(t) - sigma(t_ref)
        //   = sigma(t) (1 - sigma(t_ref)) (1 - e^{-(t - t_ref)}),
        // or, far from the anchor (|t - t_ref| > 16: e^{-(t - t_ref)} can overflow,
        // and the two values differ by orders of magnitude), the plain difference
        const float t = -y * (float)ug;
        const float tr = -y * (float)__ldg(&Ur[i]);
        const float dt = (float)(-(double)y * du);
        const float s = 1.0f / (1.0f + expf(-t));
        if (fabsf(dt) > 16.0f) {
          dr = -y * (s - 1.0f / (1.0f + expf(-tr)));
        } else {
          const float sr = 1.0f / (1.0f + expf(tr));    // 1 - sigma(t_ref)
          dr = -y * (s * sr * (-expm1f(-dt)));
        }
        // binary entropy of q = zeta_i y_i = sigma(t)
        term = s * softplusf(-t) + (1.0f - s) * softplusf(t);
      }
      if (d.e8) {
        rb[i] = dr;
        amax = fmaxf(amax, fabsf(dr));
      } else {
        split_store(dr, rrow + i, pstride, d.P);
      }
      nc += (double)term;
    }
  }
  nc = block_sum<double, kBThreads>(nc, red);
  if (threadIdx.x == 0) d.ncpart[(size_t)b * d.nrt + blockIdx.x] = nc;
  if (d.e8) {
    const double am = block_max<double, kBThreads>((double)amax, red, 0.0);
    if (threadIdx.x == 0) d.rmaxp[(size_t)b * d.nrt + blockIdx.x] = (float)am;
  }
}

// E4M3 pieces of the residual differences: the node's largest |dr| from the
// residual CTAs' maxima, then the same rows as the residual kernel
__global__ void __launch_bounds__(kBThreads) k_bsplit8_resid(BatchDev d) {
  const int b = blockIdx.y;
  if (d.nodes[b].done != kRunning) return;
  float amax = 0.0f;
  for (int t = 0; t < d.nrt; ++t) amax = fmaxf(amax, d.rmaxp[(size_t)b * d.nrt + t]);
  const int e = e8_exponent((double)amax);
  const float sc = scalbnf(1.0f, e);
  if (blockIdx.x == 0 && threadIdx.x == 0) d.rs_grad[b] = scalbnf(1.0f, -e);
  const float* rb = d.rbuf + (size_t)b * d.ldn;
  uint8_t* row = d.rpc8 + (size_t)b * d.ldn8;
  const size_t pstride = (size_t)d.Bpad * d.ldn8;
  const int i0 = blockIdx.x * kBThreads * kBRows;
  for (int r = 0; r < kBRows; ++r) {
    const int i = i0 + r * kBThreads + (int)threadIdx.x;
    if (i < d.n) split8_store(rb[i] * sc, row + i, pstride);
  }
}

// E4M3 pieces of s_j (beta_j - beta_ref_j) for one node (one CTA of BLOCK
// threads): its largest magnitude first, then the pieces; returns the inverse scale
template <int BLOCK>
__device__ float split8_beta_row(const BatchDev& d, int b, const double* bn, const double* br, double* red) {
  double amax = 0.0;
  for (int j = threadIdx.x; j < d.p; j += BLOCK) {
    const double x = bn[j], r = br[j];
    if (((__double_as_longlong(x) | __double_as_longlong(r)) << 1) != 0)
      amax = fmax(amax, fabs((x - r) * (double)d.xscale[j]));
  }
  amax = block_max<double, BLOCK>(amax, red, 0.0);
  const int e = e8_exponent(amax);
  const double sc = ldexp(1.0, e);
  uint8_t* row = d.bpc8 + (size_t)b * d.ldp8;
  const size_t pstride = (size_t)d.Bpad * d.ldp8;
  for (int j = threadIdx.x; j < d.p; j += BLOCK) {
    const double x = bn[j], r = br[j];
    const float v = ((__double_as_longlong(x) | __double_as_longlong(r)) << 1) == 0
                        ? 0.0f
                        : (float)((x - r) * ((double)d.xscale[j] * sc));
    split8_store(v, row + j, pstride);
  }
  return scalbnf(1.0f, -e);
}

__global__ void __launch_bounds__(256) k_bsplit8_beta(BatchDev d, const int* list) {
  __shared__ double red[64];
  const int b = list[blockIdx.x];
  const double* b1 = d.beta + ((size_t)b * 3 + 1) * d.ldp;
  const double* br = d.beta_ref + (size_t)b * d.ldp;
  const float rs = split8_beta_row<256>(d, b, b1, br, red);
  if (threadIdx.x == 0) d.rs_fwd[b] = rs;
}

// ------------------------------------------------------------------ prox

__global__ void __launch_bounds__(kBProxBlock) k_bprox(BatchDev d) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x;
  BNode* nd = d.nodes + b;
  const int cur = nd->cur, prev = nd->prev, nw = 3 - cur - prev;
  if (nd->done != kRunning) {
    if (threadIdx.x == 0) d.slot_new[b] = nw;
    return;
  }
  SegSmem<double> sm = carve_seg_smem<double>(smem, kBatchCap, d.wsm);
  const int p = d.p;
  const int8_t* st = d.state + (size_t)b * d.ldp;
  double* brow = d.beta + (size_t)b * 3 * d.ldp;
  double* G = d.G + (size_t)b * d.ldp;
  const double lambda2 = nd->lambda2, M = nd->M;
  const int kp = nd->kp;
  const double eig = nd->eig;
  double gsq = 0.0;
  if (eig > 0.0) {
    // eigen-perspective (App. D.2): the smooth part b^T Q b - 2 y^T X b + ||y||^2
    // has the gradient X^T grad F(X gamma) - 2 eig gamma at the momentum point
    const double* bc = brow + (size_t)cur * d.ldp;
    const double* bp = brow + (size_t)prev * d.ldp;
    const double c = nd->c;
    for (int j = threadIdx.x; j < p; j += kBProxBlock) {
      const double g = bc[j] + c * (bc[j] - bp[j]);
      G[j] -= 2.0 * eig * g;
      gsq += g * g;
    }
    gsq = block_sum<double, kBProxBlock>(gsq, sm.red);
    __syncthreads();
  }
  // in-loop dual term at gamma: a = X^T zeta_gamma = -G, |a| = |G|
  double gthr = 0.0;
  const double gs = gstar_segment<double, kBProxBlock>(p, [&](int i) { return G[i]; }, st, kp, M,
                                                       0.5 / lambda2, sm, nd->gthr, &gthr);
  SegIO<double> io;
  io.m = p;
  io.state = st;
  io.w = nullptr;
  io.bc = brow + (size_t)cur * d.ldp;
  io.bp = brow + (size_t)prev * d.ldp;
  io.grad = G;
  io.gradf = nullptr;
  io.c = nd->c;
  io.invL = nd->invL;
  io.rho = nd->rho;
  io.M = M;
  io.kp = kp;
  io.wbuf = d.wbuf ? d.wbuf + (size_t)b * d.ldp : nullptr;
  io.beta = brow + (size_t)nw * d.ldp;
  io.nnz_idx = nullptr;
  io.nnz_val = nullptr;
  io.nnz_cap = 0;
  io.top_out = nullptr;
  io.qhint = nd->qhint;
  io.theta0 = nd->theta;
  io.topk_hint = nd->ptop;
  const SegOut o = prox_segment<double, kBProxBlock>(io, sm);
  __syncthreads();
  // BF16 pieces of fl32(beta^{t+1} - beta_ref) (E4M3: pieces of s_j times it)
  const size_t pstride = (size_t)d.Bpad * d.ldp;
  __nv_bfloat16* prow = d.bpc + (size_t)b * d.ldp;
  const double* bn = io.beta;
  const double* br = d.beta_ref + (size_t)b * d.ldp;
  double bsq = 0.0;
  if (d.e8) {
    const float rs = split8_beta_row<kBProxBlock>(d, b, bn, br, sm.red);
    if (threadIdx.x == 0) d.rs_fwd[b] = rs;
  }
  for (int j = d.e8 ? p : (int)threadIdx.x; j < p; j += kBProxBlock) {
    const double x = bn[j], r = br[j];
    // both zero (most coordinates of a sparse iterate): no FP64 arithmetic
    const float v = ((__double_as_longlong(x) | __double_as_longlong(r)) << 1) == 0 ? 0.0f : (float)(x - r);
    split_store(v, prow + j, pstride, d.P);
    if (eig > 0.0) bsq += x * x;
  }
  if (eig > 0.0) bsq = block_sum<double, kBProxBlock>(bsq, sm.red);
  if (threadIdx.x == 0) {
    double nc = 0.0;
    for (int t = 0; t < d.nrt; ++t) nc += d.ncpart[(size_t)b * d.nrt + t];
    // -F*(-zeta) at zeta = -2 Q gamma: ||y||^2 - ||X gamma||^2 + eig ||gamma||^2
    nd->negconj = nc + eig * gsq;
    nd->bsq_next = bsq;
    nd->gstar = gs;
    nd->gthr = gthr;
    nd->ptop = o.topk;
    nd->g_next = o.g;
    nd->theta = o.theta;
    nd->nnz = o.nnz;
    nd->qhint = o.qused;
    nd->fallback += o.fallback;
    d.slot_new[b] = nw;
  }
}

// ------------------------------------------------------------------ step

__global__ void __launch_bounds__(128) k_bstep(BatchDev d) {
  // one block per 128 slots (the products' M tile)
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  int run = 0;
  if (b < d.B && d.nodes[b].done == kRunning) {
    BNode* nd = d.nodes + b;
    double f = 0.0, df = 0.0;
    const double* fp = d.fpart + (size_t)2 * b * d.nft;
    for (int t = 0; t < d.nft; ++t) {
      f += fp[2 * t];
      df += fp[2 * t + 1];
    }
    // L^{t+1} - L^t = sum_i [F_i(u^{t+1}) - F_i(u^t)] + 2 lambda2 (g(beta^{t+1}) - g(beta^t))
    double dL = df + 2.0 * nd->lambda2 * (nd->g_next - nd->g_cur);
    if (nd->eig > 0.0) {   // eigen-perspective: - eig ||beta||^2 in the objective
      f -= nd->eig * nd->bsq_next;
      dL -= nd->eig * (nd->bsq_next - nd->bsq_cur);
    }
    fista_step_logic(nd, f, &dL);
    nd->g_cur = nd->g_next;
    nd->bsq_cur = nd->bsq_next;
    nd->prev = nd->cur;
    nd->cur = d.slot_new[b];
    d.slot_cur[b] = nd->cur;
    run = nd->done == kRunning;
  }
  // the next step's products skip the tile once all its nodes have stopped
  run = __syncthreads_or(run);
  if (threadIdx.x == 0) d.tile_run[blockIdx.x] = run;
}

// ------------------------------------------------------------------ admission

// beta^0 = beta^1 = beta_ref = the projected warm start (uploaded into slot 1)
__global__ void __launch_bounds__(256) k_binit_copy(BatchDev d, const int* list) {
  const int b = list[blockIdx.y];
  double* brow = d.beta + (size_t)b * 3 * d.ldp;
  for (int j = blockIdx.x * 256 + (int)threadIdx.x; j < d.p; j += gridDim.x * 256) {
    const double v = brow[(size_t)d.ldp + j];
    brow[j] = v;
    d.beta_ref[(size_t)b * d.ldp + j] = v;
  }
}

// u^0 = u^1 = u_ref (set by the anchor) -- or, after the zero anchor, u^1 from the
// admission product in slot 1, copied to slot 0 --, F(u^1) in FP64, g(beta^1)
// (Alg. 2), L^1 = F(u^1) + 2 lambda2 g(beta^1)  (the initial objective of Algorithm 3)
__global__ void __launch_bounds__(kBProxBlock) k_binit_node(BatchDev d, const int* list, int zero) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = list[blockIdx.x];
  BNode* nd = d.nodes + b;
  SegSmem<double> sm = carve_seg_smem<double>(smem, kBatchCap, 0);
  double* U = d.U + (size_t)b * 3 * d.ldn;
  const double* ur = zero ? U + d.ldn : d.u_ref + (size_t)b * d.ldn;
  double f = 0.0;
  for (int i = threadIdx.x; i < d.n; i += kBProxBlock) {
    f += loss_d(ur[i], d.y[i], d.loss);
    if (zero) U[i] = ur[i];
  }
  f = block_sum<double, kBProxBlock>(f, sm.red);
  const double* b1 = d.beta + ((size_t)b * 3 + 1) * d.ldp;
  const int8_t* st = d.state + (size_t)b * d.ldp;
  const GOut o = gvalue_segment<double, kBProxBlock>(d.p, [&](int i) { return b1[i]; }, st, nd->kp, nd->M, sm,
                                                     nullptr, 1e-12);
  double bsq = 0.0;
  if (nd->eig > 0.0) {
    for (int j = threadIdx.x; j < d.p; j += kBProxBlock) bsq += b1[j] * b1[j];
    bsq = block_sum<double, kBProxBlock>(bsq, sm.red);
  }
  if (threadIdx.x == 0) {
    // eigen-perspective: F(u) - eig ||beta||^2 + 2 (lambda2 + eig) g(beta)
    const double L1 = f - nd->eig * bsq + 2.0 * nd->lambda2 * o.g;
    nd->bsq_cur = bsq;
    nd->bsq_next = bsq;
    nd->g_next = o.g;
    nd->g_cur = o.g;
    nd->Lcur = L1;
    nd->best_primal = L1;
    nd->best_dual = -INFINITY;
    nd->gap = INFINITY;
    nd->phi = 1.0;
    nd->c = nd->momentum_on ? 0.25 : 0.0;
    nd->iter = 1;
    nd->done = kRunning;
    nd->restarts = 0;
    nd->last_primal = L1;
    nd->last_dual = -INFINITY;
    nd->cur = 1;
    nd->prev = 0;
    nd->nnz = d.p;
    nd->qhint = 0;
    nd->fallback = 0;
    d.slot_cur[b] = 1;
    d.slot_new[b] = 2;
  }
}

// ------------------------------------------------------------------ anchors

// The zero anchor of an admission: beta_ref = 0, u_ref = X 0 = 0 exactly,
// r_ref = grad F(0), G_ref = X^T grad F(0) (the same for every node: computed
// once per workspace, exactly), and the BF16 pieces of beta^1 - 0 for the
// admission's forward product u^1 = X beta^1 (FP32 accumulation; the node's first
// exact anchor comes when its gap falls to the anchor threshold).
__global__ void __launch_bounds__(256) k_bzero_anchor(BatchDev d, const int* list, const double* r0,
                                                      const double* G0) {
  const int b = list[blockIdx.y];
  const size_t pstride = (size_t)d.Bpad * d.ldp;
  const double* b1 = d.beta + ((size_t)b * 3 + 1) * d.ldp;
  for (int j = blockIdx.x * 256 + (int)threadIdx.x; j < d.p; j += gridDim.x * 256) {
    d.beta_ref[(size_t)b * d.ldp + j] = 0.0;
    d.G_ref[(size_t)b * d.ldp + j] = G0[j];
    if (!d.e8) split_store((float)b1[j], d.bpc + (size_t)b * d.ldp + j, pstride, d.P);
  }
  for (int i = blockIdx.x * 256 + (int)threadIdx.x; i < d.n; i += gridDim.x * 256) {
    d.u_ref[(size_t)b * d.ldn + i] = 0.0;
    d.r_ref[(size_t)b * d.ldn + i] = r0[i];
  }
}

// slot maps of the admission product: admitted rows write u^1 into slot 1; every
// other row writes its free slot (3 - cur - prev), which no step reads
__global__ void k_bslots_admit(BatchDev d, const int* list, int count) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < d.B) {
    const BNode* nd = d.nodes + t;
    d.slot_new[t] = 3 - nd->cur - nd->prev;
    d.slot_cur[t] = nd->cur;
  }
}
__global__ void k_bslots_admitted(BatchDev d, const int* list, int count) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t < count) {
    d.slot_new[list[t]] = 1;
    d.slot_cur[list[t]] = 1;
  }
}

__global__ void __launch_bounds__(256) k_banchor_copy(BatchDev d, const int* list) {
  const int b = list[blockIdx.y];
  const BNode* nd = d.nodes + b;
  const double* src = d.beta + ((size_t)b * 3 + nd->cur) * d.ldp;
  double* dst = d.beta_ref + (size_t)b * d.ldp;
  for (int j = blockIdx.x * 256 + (int)threadIdx.x; j < d.p; j += gridDim.x * 256) dst[j] = src[j];
}

// r_ref = grad F(u_ref) in FP64; the u slot(s) of the current iterate take the
// accurate u_ref.  Mid-solve, the in-loop best values restart: those recorded
// against the old anchor carry its rounding, and a running minimum (maximum)
// keeps a value that rounding pushed down (up).
__global__ void __launch_bounds__(256) k_banchor_resid(BatchDev d, const int* list, int init) {
  const int b = list[blockIdx.y];
  BNode* nd = d.nodes + b;
  if (!init && blockIdx.x == 0 && threadIdx.x == 0) {
    nd->best_primal = INFINITY;
    nd->best_dual = -INFINITY;
  }
  const double* ur = d.u_ref + (size_t)b * d.ldn;
  double* rr = d.r_ref + (size_t)b * d.ldn;
  double* U = d.U + (size_t)b * 3 * d.ldn;
  const int cur = nd->cur;
  for (int i = blockIdx.x * 256 + (int)threadIdx.x; i < d.n; i += gridDim.x * 256) {
    const double u = ur[i], y = d.y[i];
    rr[i] = d.loss == kLossLsq       ? 2.0 * (u - y)
            : d.loss == kLossSqHinge ? -2.0 * y * fmax(0.0, 1.0 - y * u)
            : d.loss == kLossPoisson ? exp(u) - y
            : d.loss == kLossGamma   ? 1.0 - y * exp(-u)
                                     : -y * sigmoid_d(-y * u);
    if (init) {
      U[i] = u;
      U[(size_t)d.ldn + i] = u;
    } else {
      U[(size_t)cur * d.ldn + i] = u;
    }
  }
}

// ------------------------------------------------------------------ certificates

// The certificate's iterate (as in the single-node certificate): the newest beta
// clipped to the box, fixed-to-zero coordinates zeroed, and the free part scaled
// onto the l1 budget k'M when rounding left it a hair outside dom g.
__global__ void __launch_bounds__(256) k_bcert_prep(BatchDev d, const int* list) {
  __shared__ double red[64];
  const int b = list[blockIdx.x];
  const BNode* nd = d.nodes + b;
  const double M = nd->M;
  const double* src = d.beta + ((size_t)b * 3 + nd->cur) * d.ldp;
  const int8_t* st = d.state + (size_t)b * d.ldp;
  double* dst = d.beta_out + (size_t)b * d.p;
  double l1 = 0.0;
  for (int j = threadIdx.x; j < d.p; j += 256) {
    double v = fmin(fmax(src[j], -M), M);
    if (st[j] == kZero) v = 0.0;
    dst[j] = v;
    if (st[j] == kFree) l1 += fabs(v);
  }
  l1 = block_sum<double, 256>(l1, red);
  const double budget = (double)(nd->kp > 0 ? nd->kp : 0) * M;
  if (l1 > budget) {
    const double sc = budget > 0.0 ? (budget / l1) * (1.0 - 8.0 * 1.1102230246251565e-16) : 0.0;
    for (int j = threadIdx.x; j < d.p; j += 256)
      if (st[j] == kFree) dst[j] *= sc;
  }
}

// per row, in FP64: F(u), zeta = -grad F(u), -F*(-zeta) (App. D.1) with the
// weights of its rounding bound, ||zeta||^2
__global__ void __launch_bounds__(kBThreads) k_bcert_rows(BatchDev d, const int* list) {
  __shared__ double red[64];
  const int b = list[blockIdx.y];
  const double* u = d.cert_u + (size_t)b * d.ldn;
  double* z = d.cert_z + (size_t)b * d.ldn;
  double f = 0.0, nc = 0.0, mg = 0.0, zsq = 0.0;
  const int i0 = blockIdx.x * kBThreads * kBRows;
  for (int r = 0; r < kBRows; ++r) {
    const int i = i0 + r * kBThreads + (int)threadIdx.x;
    if (i >= d.n) break;
    const double ui = u[i], yi = d.y[i];
    if (d.loss == kLossLsq) {
      const double res = ui - yi;
      f += res * res;
      const double zi = -2.0 * res;
      z[i] = zi;
      nc += yi * zi - 0.25 * zi * zi;
      mg += fabs(yi * zi) + 0.25 * zi * zi;
      zsq += zi * zi;
    } else if (d.loss == kLossSqHinge) {
      const double m = fmax(0.0, 1.0 - yi * ui);
      f += m * m;
      const double zi = 2.0 * yi * m;   // y zeta = 2 m >= 0: inside dom F*
      z[i] = zi;
      nc += yi * zi - 0.25 * zi * zi;
      mg += fabs(yi * zi) + 0.25 * zi * zi;
      zsq += zi * zi;
    } else if (d.loss == kLossPoisson || d.loss == kLossGamma) {
      // zeta = -grad F(u); -F*(-zeta) evaluated at this FP64 zeta as the conjugate
      // defines it (App. D.1, the Gamma argument read at -zeta): z = y - zeta or
      // (1 + zeta) / y, minus h(z) (times y for Gamma), h(z) = z log z - z
      const bool poi = d.loss == kLossPoisson;
      const double e = poi ? exp(ui) : yi * exp(-ui);
      f += poi ? e - yi * ui : e + ui;
      const double zi = poi ? yi - e : e - 1.0;
      z[i] = zi;
      const double w = poi ? yi - zi : 1.0 + zi;        // >= 0 by monotone rounding
      const double arg = poi ? w : w / yi;
      const double lg = arg > 0.0 ? log(arg) : 0.0;
      nc -= arg > 0.0 ? w * lg - w : 0.0;
      mg += 4.0 * (fabs(w * lg) + fabs(w)) + 4.0 * fabs(w);
      zsq += zi * zi;
    } else {
      const double t = -yi * ui;
      f += t > 0 ? t + log1p(exp(-t)) : log1p(exp(t));
      const double sg = sigmoid_d(t);
      const double zi = yi * sg;
      z[i] = zi;
      double h = 0.0;
      if (sg > 0.0) h -= sg * log(sg);
      if (sg < 1.0) h -= (1.0 - sg) * log1p(-sg);
      nc += h;
      // |term| plus the rounding of one entropy term in units of u (log() within
      // 2 ulp, 1-q, two products): the margin is (n+8) u * sum(mg)
      const double ql = sg > 0.0 ? fabs(sg * log(sg)) : 0.0;
      const double pl = sg < 1.0 ? fabs((1.0 - sg) * log1p(-sg)) : 0.0;
      mg += h + 8.0 + 16.0 * (ql + pl);
      zsq += zi * zi;
    }
  }
  f = block_sum<double, kBThreads>(f, red);
  nc = block_sum<double, kBThreads>(nc, red);
  mg = block_sum<double, kBThreads>(mg, red);
  zsq = block_sum<double, kBThreads>(zsq, red);
  if (threadIdx.x == 0) {
    double* cp = d.cpart + ((size_t)b * d.nrt + blockIdx.x) * 4;
    cp[0] = f;
    cp[1] = nc;
    cp[2] = mg;
    cp[3] = zsq;
  }
}

// the bound: G*(a) / (2 lambda2) over the node (Lemma 3.1 with the node's sets),
// the rounding margins of -F*(-zeta) and of a = X^T zeta (err_a * ||x_j|| ||zeta||
// per coordinate, H_M M-Lipschitz, TopSum 1-Lipschitz per selected entry), g(b^)
// by Algorithm 2 with the relaxed z, the primal value and the gap
__global__ void __launch_bounds__(kBProxBlock) k_bcert_final(BatchDev d, const int* list, double err_a,
                                                             double err_u) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = list[blockIdx.x];
  const BNode* nd = d.nodes + b;
  SegSmem<double> sm = carve_seg_smem<double>(smem, kBatchCap, 0);
  const int p = d.p;
  const int8_t* st = d.state + (size_t)b * d.ldp;
  const double ur = 1.1102230246251565e-16;
  const double l2 = nd->lambda2, M = nd->M;
  const int kp = nd->kp;
  double f = 0.0, nc = 0.0, mgs = 0.0, zs = 0.0;
  if (threadIdx.x == 0) {
    for (int t = 0; t < d.nrt; ++t) {
      const double* cp = d.cpart + ((size_t)b * d.nrt + t) * 4;
      f += cp[0];
      nc += cp[1];
      mgs += cp[2];
      zs += cp[3];
    }
  }
  const double* a = d.cert_a + (size_t)b * d.ldp;
  const double* bh = d.beta_out + (size_t)b * p;
  // eigen-perspective (App. D.2): G* at 2 (X^T y - Q b^) = X^T zeta + 2 eig b^
  const double eig = nd->eig;
  const double gs = gstar_segment<double, kBProxBlock>(
      p, [&](int i) { return eig > 0.0 ? a[i] + 2.0 * eig * bh[i] : a[i]; }, st, kp, M, 0.5 / l2, sm);
  double cmax = 0.0, amax = 0.0, bsq = 0.0;
  int n1 = 0;
  for (int j = threadIdx.x; j < p; j += kBProxBlock) {
    if (st[j] != kZero) {
      cmax = fmax(cmax, d.colnorm[j]);
      amax = fmax(amax, fabs(a[j]) + 2.0 * eig * fabs(bh[j]));
    }
    if (st[j] == kOne) n1 += 1;
    bsq += bh[j] * bh[j];
  }
  cmax = block_max<double, kBProxBlock>(cmax, sm.red, 0.0);
  amax = block_max<double, kBProxBlock>(amax, sm.red, 0.0);
  bsq = block_sum<double, kBProxBlock>(bsq, sm.red);
  n1 = (int)block_sum<double, kBProxBlock>((double)n1, sm.red);
  const GOut go = gvalue_segment<double, kBProxBlock>(p, [&](int i) { return bh[i]; }, st, kp, M, sm,
                                                      d.z_out + (size_t)b * p);
  if (threadIdx.x == 0) {
    const double nn = (double)d.n + 8.0;
    const double margin_f = 1.01 * nn * ur * mgs + (d.loss != kLossLogistic ? 4.0 * ur * mgs : 0.0);
    const double znorm = sqrt(zs) * (1.0 + ((double)d.n + 4.0) * ur);
    double eps_a = err_a * cmax * znorm + 1e-30;
    double nce = nc, margin_e = 0.0;
    if (eig > 0.0) {
      // The bound at b^ is ||y||^2 - ||X b^||^2 + eig ||b^||^2 - G*(2 X^T (y - X b^)
      // + 2 eig b^).  nc is ||y||^2 - ||u~||^2 exactly (up to margin_f) for
      // u~ = y - zeta/2, and X^T zeta = 2 X^T (y - u~); with
      // ||u~ - X b^|| <= delta = err_u ||X||_F ||b^|| (the exact product's bound,
      // row by row by Cauchy-Schwarz) + u ||zeta|| (the rounding of u - y):
      //   | ||u~||^2 - ||X b^||^2 | <= delta (2 ||u~|| + delta),
      //   per coordinate |a - a_computed| <= eps_a + 2 ||x_j|| delta + rounding of the sum
      const double bnorm = sqrt(bsq) * (1.0 + ((double)p + 4.0) * ur);
      const double delta = (err_u * d.xfro * bnorm + ur * znorm) * 1.01;
      const double unorm = d.ynorm + 0.5 * znorm;
      margin_e = delta * (2.0 * unorm + delta) + ((double)p + 4.0) * ur * eig * bsq * 1.01;
      eps_a += 2.0 * cmax * delta + 2.0 * ur * (amax + 2.0 * eig * M) * 1.01;
      nce = nc + eig * bsq;
    }
    const int nsel = (kp < p ? kp : p) + n1;
    const double margin_g = (double)nsel * M * eps_a * (1.0 + 4.0 * ur) + 2.0 * l2 * gs * ((double)nsel + 8.0) * 4.0 * ur;
    const double gst = 2.0 * l2 * gs;
    double dual = nce - margin_f - margin_e - gst - margin_g;
    dual -= 4.0 * ur * (fabs(nce) + gst);
    const double primal = f - eig * bsq + 2.0 * l2 * go.g;
    BCert c;
    c.primal = primal;
    c.dual = dual;
    c.gap = (primal - dual) / fmax(fabs(primal), 1e-300);
    c.g = go.g;
    d.cert[b] = c;
  }
}

// ------------------------------------------------------------------ launchers

size_t bprox_smem_bytes(int wsm) { return seg_smem_bytes(kBatchCap, wsm, 8); }

cudaError_t batch_prepare(int optin) {
  const cudaError_t steps[] = {
      cudaFuncSetAttribute(k_bprox, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
      // all of the unified L1 as shared memory: 4 node CTAs of ~50 KB per SM instead of 3
      cudaFuncSetAttribute(k_bprox, cudaFuncAttributePreferredSharedMemoryCarveout, 100),
      cudaFuncSetAttribute(k_binit_node, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
      cudaFuncSetAttribute(k_bcert_final, cudaFuncAttributeMaxDynamicSharedMemorySize, optin),
  };
  for (cudaError_t st : steps)
    if (st != cudaSuccess) return st;
  return cudaSuccess;
}

static int vec_blocks(int m) {
  const int g = (m + 255) / 256;
  return g < 64 ? g : 64;
}

void launch_bresid(const BatchDev& d, cudaStream_t s) {
  k_bresid<<<dim3(d.nrt, d.B), kBThreads, 0, s>>>(d);
}

void launch_bsplit8_resid(const BatchDev& d, cudaStream_t s) {
  k_bsplit8_resid<<<dim3(d.nrt, d.B), kBThreads, 0, s>>>(d);
}

void launch_bsplit8_beta(const BatchDev& d, const int* list, int count, cudaStream_t s) {
  k_bsplit8_beta<<<count, 256, 0, s>>>(d, list);
}

void launch_bprox(const BatchDev& d, cudaStream_t s) {
  k_bprox<<<d.B, kBProxBlock, bprox_smem_bytes(d.wsm), s>>>(d);
}

void launch_bstep(const BatchDev& d, cudaStream_t s) { k_bstep<<<(d.B + 127) / 128, 128, 0, s>>>(d); }

void launch_binit_copy(const BatchDev& d, const int* list, int count, cudaStream_t s) {
  k_binit_copy<<<dim3(vec_blocks(d.p), count), 256, 0, s>>>(d, list);
}

void launch_binit_node(const BatchDev& d, const int* list, int count, int zero, cudaStream_t s) {
  k_binit_node<<<count, kBProxBlock, bprox_smem_bytes(0), s>>>(d, list, zero);
}

void launch_bzero_anchor(const BatchDev& d, const int* list, int count, const double* r0, const double* G0,
                         cudaStream_t s) {
  k_bzero_anchor<<<dim3(vec_blocks(d.n > d.p ? d.n : d.p), count), 256, 0, s>>>(d, list, r0, G0);
  k_bslots_admit<<<(d.B + 255) / 256, 256, 0, s>>>(d, list, count);
  k_bslots_admitted<<<(count + 255) / 256, 256, 0, s>>>(d, list, count);
}

void launch_banchor_copy(const BatchDev& d, const int* list, int count, cudaStream_t s) {
  k_banchor_copy<<<dim3(vec_blocks(d.p), count), 256, 0, s>>>(d, list);
}

void launch_banchor_resid(const BatchDev& d, const int* list, int count, int init, cudaStream_t s) {
  k_banchor_resid<<<dim3(vec_blocks(d.n), count), 256, 0, s>>>(d, list, init);
}

void launch_bcert_prep(const BatchDev& d, const int* list, int count, cudaStream_t s) {
  k_bcert_prep<<<count, 256, 0, s>>>(d, list);
}

void launch_bcert_rows(const BatchDev& d, const int* list, int count, cudaStream_t s) {
  k_bcert_rows<<<dim3(d.nrt, count), kBThreads, 0, s>>>(d, list);
}

void launch_bcert_final(const BatchDev& d, const int* list, int count, double err_a, double err_u,
                        cudaStream_t s) {
  k_bcert_final<<<count, kBProxBlock, bprox_smem_bytes(0), s>>>(d, list, err_a, err_u);
}

}  // namespace ksc
