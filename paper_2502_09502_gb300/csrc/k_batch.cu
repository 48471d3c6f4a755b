// k_batch.cu -- the per-node kernels of a batched FISTA step (Algorithm 3 over B
// nodes of one problem).  Between them run the two tensor-core products of
// k_tcgemm.cu:
//
//   k_bresid   u_gamma = u_t + c (u_t - u_{t-1}) (linearity: no extra pass over X),
//              r = grad F(u_gamma), its BF16 pieces (A of X^T r), and the terms of
//              -F*(-zeta_gamma), zeta_gamma = -r (App. D), per CTA
//   [tensor]   G = X^T r                      (node-major rows, FP32)
//   k_bprox    one CTA per node: w = gamma - G/L, the exact prox of g_node (block
//              radix select + bitonic sort + breakpoint scan, Alg. 1 + 4 in the
//              threshold form), g(beta^{t+1}) (Alg. 2), the in-loop dual term
//              G*(X^T zeta_gamma) (Lemma 3.1 on the node), and the BF16 pieces of
//              the step dbeta = beta^{t+1} - beta^t
//   [tensor]   u^{t+1} = u^t + X dbeta (FP64), partials of F(u^{t+1}) and of its
//              change F(u^{t+1}) - F(u^t)
//   k_bstep    the restart test on L^{t+1} - L^t (a sum of changes, free of the
//              cancellation of two nearly equal objective values) and the gap
//              test per node (the step logic shared with the single-node solver)
#include "ksc_batch.cuh"
#include "ksc_common.cuh"
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

__device__ __forceinline__ float softplusf(float x) { return fmaxf(x, 0.0f) + log1pf(__expf(-fabsf(x))); }

// ------------------------------------------------------------------ residual

__global__ void __launch_bounds__(kBThreads) k_bresid(BatchDev d) {
  __shared__ double red[64];
  const int b = blockIdx.y;
  const BNode* nd = d.nodes + b;
  if (nd->done != kRunning) return;
  const double c = nd->c;
  const double* Uc = d.U + ((size_t)b * 3 + nd->cur) * d.ldn;
  const double* Up = d.U + ((size_t)b * 3 + nd->prev) * d.ldn;
  const size_t pstride = (size_t)d.Bpad * d.ldn;
  __nv_bfloat16* rrow = d.rpc + (size_t)b * d.ldn;
  double nc = 0.0;
  const int i0 = blockIdx.x * kBThreads * kBRows;
#pragma unroll 4
  for (int r = 0; r < kBRows; ++r) {
    const int i = i0 + r * kBThreads + (int)threadIdx.x;
    if (i < d.n) {
      const double uc = __ldg(&Uc[i]);
      const float ug = (float)(uc + c * (uc - __ldg(&Up[i])));
      const float y = __ldg(&d.yf[i]);
      float res, term;
      if (d.loss == kLossLsq) {
        res = 2.0f * (ug - y);          // grad F
        const float z = -res;           // zeta = -grad F
        term = y * z - 0.25f * z * z;   // -F*(-zeta), App. D.1
      } else {
        const float t = -y * ug;
        const float s = 1.0f / (1.0f + __expf(-t));   // sigma(t)
        res = -y * s;
        // binary entropy of q = zeta_i y_i = s:  s softplus(-t) + (1-s) softplus(t)
        term = s * softplusf(-t) + (1.0f - s) * softplusf(t);
      }
      split_store(res, rrow + i, pstride, d.P);
      nc += (double)term;
    }
  }
  nc = block_sum<double, kBThreads>(nc, red);
  if (threadIdx.x == 0) d.ncpart[(size_t)b * d.nrt + blockIdx.x] = nc;
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
  SegSmem<float> sm = carve_seg_smem<float>(smem, kBatchCap, d.wsm);
  const int p = d.p;
  const int8_t* st = d.state + (size_t)b * d.ldp;
  float* brow = d.beta + (size_t)b * 3 * d.ldp;
  const float* G = d.G + (size_t)b * d.ldp;
  const double lambda2 = nd->lambda2, M = nd->M;
  const int kp = nd->kp;
  // in-loop dual term at gamma: a = X^T zeta_gamma = -G, |a| = |G|
  const double gs = gstar_segment<float, kBProxBlock>(p, [&](int i) { return G[i]; }, st, kp, M,
                                                      0.5 / lambda2, sm);
  SegIO<float> io;
  io.m = p;
  io.state = st;
  io.w = nullptr;
  io.bc = brow + (size_t)cur * d.ldp;
  io.bp = brow + (size_t)prev * d.ldp;
  io.grad = nullptr;
  io.gradf = G;
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
  const SegOut o = prox_segment<float, kBProxBlock>(io, sm);
  __syncthreads();
  // BF16 pieces of the step beta^{t+1} - beta^t
  const size_t pstride = (size_t)d.Bpad * d.ldp;
  __nv_bfloat16* prow = d.bpc + (size_t)b * d.ldp;
  const float* bn = io.beta;
  const float* bc = io.bc;
  for (int j = threadIdx.x; j < p; j += kBProxBlock) split_store(__fsub_rn(bn[j], bc[j]), prow + j, pstride, d.P);
  if (threadIdx.x == 0) {
    double nc = 0.0;
    for (int t = 0; t < d.nrt; ++t) nc += d.ncpart[(size_t)b * d.nrt + t];
    nd->negconj = nc;
    nd->gstar = gs;
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
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= d.B) return;
  BNode* nd = d.nodes + b;
  if (nd->done != kRunning) return;
  double f = 0.0, df = 0.0;
  const double* fp = d.fpart + (size_t)2 * b * d.nft;
  for (int t = 0; t < d.nft; ++t) {
    f += fp[2 * t];
    df += fp[2 * t + 1];
  }
  // L^{t+1} - L^t = sum_i [F_i(u^{t+1}) - F_i(u^t)] + 2 lambda2 (g(beta^{t+1}) - g(beta^t))
  const double dL = df + 2.0 * nd->lambda2 * (nd->g_next - nd->g_cur);
  fista_step_logic(nd, f, &dL);
  nd->g_cur = nd->g_next;
  nd->prev = nd->cur;
  nd->cur = d.slot_new[b];
  d.slot_cur[b] = nd->cur;
}

// ------------------------------------------------------------------ init

// beta^0 = beta^1 = the projected warm start (uploaded into slot 1): copy to slot
// 0, pieces of slot 1, u slot 0 = 0; the forward product then writes
// u^1 = 0 + X beta^1 into slot 1
__global__ void __launch_bounds__(256) k_binit_split(BatchDev d) {
  const int b = blockIdx.y;
  const int j = blockIdx.x * 256 + (int)threadIdx.x;
  float* brow = d.beta + (size_t)b * 3 * d.ldp;
  if (j < d.p) {
    const float v = brow[(size_t)d.ldp + j];
    brow[j] = v;
    split_store(v, d.bpc + (size_t)b * d.ldp + j, (size_t)d.Bpad * d.ldp, d.P);
  }
  if (j < d.n) d.U[(size_t)b * 3 * d.ldn + j] = 0.0;
  if (j == 0) {
    d.slot_cur[b] = 0;
    d.slot_new[b] = 1;
  }
}

// u^0 = u^1, g(beta^1) (Alg. 2) and L^1 = F(u^1) + 2 lambda2 g(beta^1)
__global__ void __launch_bounds__(kBProxBlock) k_binit_node(BatchDev d) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int b = blockIdx.x;
  BNode* nd = d.nodes + b;
  double* U1 = d.U + ((size_t)b * 3 + 1) * d.ldn;
  double* U0 = d.U + ((size_t)b * 3 + 0) * d.ldn;
  for (int i = threadIdx.x; i < d.n; i += kBProxBlock) U0[i] = U1[i];
  SegSmem<float> sm = carve_seg_smem<float>(smem, kBatchCap, 0);
  const float* b1 = d.beta + ((size_t)b * 3 + 1) * d.ldp;
  const int8_t* st = d.state + (size_t)b * d.ldp;
  const GOut o = gvalue_segment<float, kBProxBlock>(d.p, [&](int i) { return (double)b1[i]; }, st, nd->kp,
                                                    nd->M, sm, nullptr, 1e-6);
  if (threadIdx.x == 0) {
    double f = 0.0;
    const double* fp = d.fpart + (size_t)2 * b * d.nft;
    for (int t = 0; t < d.nft; ++t) f += fp[2 * t];
    const double L1 = f + 2.0 * nd->lambda2 * o.g;   // Algorithm 3 line 2
    nd->g_next = o.g;
    nd->g_cur = o.g;
    d.slot_cur[b] = 1;
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
  }
}

// ------------------------------------------------------------------ certificate bridge

// node b's state and newest iterate into the single-node workspace (FP64 slot 1)
__global__ void __launch_bounds__(256) k_bcert_load(BatchDev bd, int b, Dev d) {
  const BNode* nb = bd.nodes + b;
  const float* src = bd.beta + ((size_t)b * 3 + nb->cur) * bd.ldp;
  const int8_t* st = bd.state + (size_t)b * bd.ldp;
  double* dst = (double*)d.beta + (size_t)1 * d.p;
  for (int j = blockIdx.x * 256 + (int)threadIdx.x; j < d.p; j += gridDim.x * 256) {
    dst[j] = (double)src[j];
    d.state[j] = st[j];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    NodeDev* nd = d.nd;
    nd->lambda2 = nb->lambda2;
    nd->M = nb->M;
    nd->kp = nb->kp;
    nd->iter = 1;          // the certificate reads slot iter % 3
    nd->nnz = d.p + 1;     // dense FP64 forward pass over the promoted iterate
    nd->loss = bd.loss;
  }
}

__global__ void __launch_bounds__(256) k_bcert_store(BatchDev bd, int b, Dev d, int want_z) {
  double* bo = bd.beta_out + (size_t)b * bd.p;
  double* zo = want_z && bd.z_out ? bd.z_out + (size_t)b * bd.p : nullptr;
  for (int j = blockIdx.x * 256 + (int)threadIdx.x; j < d.p; j += gridDim.x * 256) {
    bo[j] = d.b64[j];
    if (zo) zo[j] = d.z64[j];
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    const NodeDev* nd = d.nd;
    BCert c;
    c.primal = nd->cert_primal;
    c.dual = nd->cert_dual;
    c.gap = nd->cert_gap;
    c.g = nd->cert_g;
    bd.cert[b] = c;
  }
}

// ------------------------------------------------------------------ launchers

size_t bprox_smem_bytes(int wsm) { return seg_smem_bytes(kBatchCap, wsm, 4); }

void batch_prepare(int optin) {
  cudaFuncSetAttribute(k_bprox, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
  cudaFuncSetAttribute(k_binit_node, cudaFuncAttributeMaxDynamicSharedMemorySize, optin);
}

void launch_bresid(const BatchDev& d, cudaStream_t s) {
  k_bresid<<<dim3(d.nrt, d.B), kBThreads, 0, s>>>(d);
}

void launch_bprox(const BatchDev& d, cudaStream_t s) {
  k_bprox<<<d.B, kBProxBlock, bprox_smem_bytes(d.wsm), s>>>(d);
}

void launch_bstep(const BatchDev& d, cudaStream_t s) { k_bstep<<<(d.B + 127) / 128, 128, 0, s>>>(d); }

void launch_binit_split(const BatchDev& d, cudaStream_t s) {
  const int m = d.p > d.n ? d.p : d.n;
  k_binit_split<<<dim3((m + 255) / 256, d.B), 256, 0, s>>>(d);
}

void launch_binit_node(const BatchDev& d, cudaStream_t s) {
  k_binit_node<<<d.B, kBProxBlock, bprox_smem_bytes(0), s>>>(d);
}

void launch_bcert_load(const BatchDev& bd, int b, const Dev& d, cudaStream_t s) {
  const int g = (d.p + 255) / 256;
  k_bcert_load<<<g < 304 ? g : 304, 256, 0, s>>>(bd, b, d);
}

void launch_bcert_store(const BatchDev& bd, int b, const Dev& d, int want_z, cudaStream_t s) {
  const int g = (d.p + 255) / 256;
  k_bcert_store<<<g < 304 ? g : 304, 256, 0, s>>>(bd, b, d, want_z);
}

}  // namespace ksc
