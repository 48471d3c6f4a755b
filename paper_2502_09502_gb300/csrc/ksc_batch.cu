// ksc_batch.cu -- batched solves: sessions of node slots of one problem
// (ksc_session.h) and ksc_solve_batch on top of them.
//
// Nodes with BF16 X advance in lock step through restarted FISTA (Algorithm 3):
// per step one residual kernel, the product X^T (r - r_ref) on the tensor cores,
// one prox CTA per node, the product X (beta - beta_ref) on the tensor cores,
// and the per-node step logic -- 16 steps per CUDA-graph replay.  Anchors
// (u_ref = X beta_ref, G_ref = X^T grad F(u_ref)) come from the double-float
// streaming product at admission and again as a node's gap falls.  A node whose
// in-loop test fires is frozen; its FP64 certificate (Sec. 3.4) is computed
// through the single-node workspace, and the node either finishes or resumes with
// a tighter in-loop tolerance, exactly as in ksc_solve_node.  Nodes the batched
// path does not take (X not BF16, k' beyond the per-node candidate capacity) are
// solved one by one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include "ksc_batch.cuh"
#include "ksc_problem.h"
#include "ksc_session.h"
#include "ksc_tc.h"
#include "ksc_tcx.h"

namespace ksc {

struct BatchWs {
  int Bcap = 0;      // nodes the buffers hold
  int Bpad = 0;      // Bcap rounded up to 128 (row stride of the BF16 pieces)
  int ldp = 0, ldn = 0;
  int B = -1;        // nodes of the current plans and graphs
  int bn_fwd = 0, bn_grad = 0;
  int sk_fwd = 0, sk_grad = 0;   // stream-K schedule chosen for each product
  int nsm = 0;                   // SMs (persistent CTAs of a stream-K product)
  float* skws = nullptr;         // stream-K partial tiles (shared by both products)
  double* r0 = nullptr;          // grad F(0) (n) and G0 = X^T grad F(0) (p), exact: the zero anchor
  double* G0 = nullptr;
  bool zero_ready = false;
  std::vector<void*> allocs;
  size_t bytes = 0;
  BatchDev bd{};
  int* dlist = nullptr;   // device slot list for admissions (Bcap ints)
  TcPlan fwd{}, grad{};
  cudaGraphExec_t graph = nullptr;
  cudaGraphExec_t graph_prof = nullptr;   // the same steps with events between the kernels
  std::vector<cudaEvent_t> events;        // 6 per step of graph_prof
  cudaEvent_t ph0 = nullptr, ph1 = nullptr;   // around certificate / anchor phases (profiling)
  const void* Xb = nullptr;   // X with a TMA-compatible row stride (the problem's, or a copy)
  int64_t ldxb = 0;
  // exact products of anchors and certificates on the tensor cores (k_tcexact.cu):
  // slices of X (forward: rows of X, K = p) and of Xc (gradient: columns of X,
  // K = n), and of the listed nodes' vectors; built for the problem-owned
  // workspace of ksc_solve_batch and branch and bound (server sessions keep the
  // streaming double-float product and its smaller footprint)
  bool tcx = false;
  TcxSlices xs_fwd, xs_grad;
  TcxVecs vs_fwd, vs_grad;
};

void free_batch(BatchWs* ws) {
  if (!ws) return;
  tcx_slices_free(&ws->xs_fwd);
  tcx_slices_free(&ws->xs_grad);
  tcx_vecs_free(&ws->vs_fwd);
  tcx_vecs_free(&ws->vs_grad);
  if (ws->graph) cudaGraphExecDestroy(ws->graph);
  if (ws->graph_prof) cudaGraphExecDestroy(ws->graph_prof);
  for (auto e : ws->events) cudaEventDestroy(e);
  if (ws->ph0) cudaEventDestroy(ws->ph0);
  if (ws->ph1) cudaEventDestroy(ws->ph1);
  for (void* v : ws->allocs) cudaFree(v);
  delete ws;
}

size_t Session::bytes() const { return ws ? ws->bytes : 0; }

}  // namespace ksc

using namespace ksc;

namespace {

constexpr int kBatchStepsPerGraph = 16;
constexpr int kLaunchesPerBatchStep = 5;   // residual, X^T r, prox, X beta, step
constexpr int kLaunchesPerBatchCert = 5;   // prep, X b^, rows, X^T zeta, final (per fired group)
constexpr int kLaunchesPerAnchor = 4;      // copy, X beta_ref, grad F, X^T r_ref
// admissions of at least this many nodes start from the zero anchor (one forward
// product for all of them instead of two exact products per node)
constexpr int kZeroAnchorMin = 32;
// relative accuracy of the in-loop gap: the FP32 loss and entropy terms (summed in
// FP64) carry ~1e-8; a tighter in-loop tolerance could never be met
constexpr double kInLoopFloor = 3e-8;

#define KB_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return api_fail(e_ == cudaErrorMemoryAllocation ? KSC_ERR_OOM : KSC_ERR_CUDA,          \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

BNode* hnodes(Session* se) { return (BNode*)se->hn_raw.data(); }
BCert* hcerts(Session* se) { return (BCert*)se->hc_raw.data(); }

template <typename P>
ksc_status balloc(BatchWs* ws, P** ptr, size_t bytes) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess)
    return api_fail(KSC_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  ws->allocs.push_back(v);
  ws->bytes += bytes;
  *ptr = (P*)v;
  return KSC_OK;
}

bool batch_supported(const ksc_problem* pr) { return pr->xdt == kXBF16 || pr->xdt == kXFP8; }

int pad8(int64_t v) { return (int)((v + 7) / 8 * 8); }
int pad16(int64_t v) { return (int)((v + 15) / 16 * 16); }

int sm_count() {
  int dev = 0, n = 0;
  cudaGetDevice(&dev);
  if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n < 1) n = 1;
  return n;
}

static size_t xelem(const ksc_problem* pr) { return pr->xdt == kXFP8 ? 1 : 2; }
bool needs_xcopy(const ksc_problem* pr) {
  return !((pr->ldx * xelem(pr)) % 16 == 0 && ((uintptr_t)pr->X % 16) == 0);
}

// workspace bytes for `need` slots (the allocations of alloc_ws)
size_t ws_bytes(const ksc_problem* pr, int need) {
  const size_t n = pr->n, p = pr->p;
  const size_t ldp = pad8(p), ldn = pad8(n), Bc = need, Bp = (need + 127) / 128 * 128;
  const size_t nft = (n + 63) / 64;
  size_t b = 0;
  b += Bc * ldp;                                // state
  b += Bc * 3 * ldp * 8 + Bc * ldp * 8;         // beta slots, beta_ref
  const bool e8 = pr->xdt == kXFP8;
  if (e8) {
    b += (size_t)kTcE4m3Pieces * Bp * (pad16(p) + pad16(n));                 // E4M3 pieces
    b += Bc * ldn * 4 + Bc * batch_nrt((int)n) * 4 + 2 * Bc * 4;            // rbuf, rmaxp, scales
  } else {
    b += (size_t)kBatchPieces * Bp * (ldp + ldn) * 2;                       // BF16 pieces
  }
  b += Bc * 3 * ldn * 8 + 2 * Bc * ldn * 8;     // u slots, u_ref, r_ref
  b += 2 * Bc * ldp * 8;                        // G, G_ref
  b += 2 * Bc * 4 + Bc * nft * 16 + Bc * batch_nrt((int)n) * 8;
  b += Bc * (sizeof(BNode) + sizeof(BCert)) + 2 * Bc * p * 8 + Bc * 4 + n * 12;
  b += 2 * Bc * ldn * 8 + Bc * ldp * 8 + Bc * batch_nrt((int)n) * 32;   // certificate vectors
  b += kDfWsElems * 8;                          // split partials of the exact product
  b += (size_t)(Bc + 127) / 128 * 4;            // tile flags
  b += tc_skws_floats(sm_count(), 256) * 4;     // stream-K partial tiles
  b += (ldn + ldp) * 8;                         // zero anchor r0, G0
  if (p > 2048) b += Bc * ldp * 8;              // prox scratch
  if (needs_xcopy(pr)) b += n * (e8 ? pad16(p) : ldp * 2);
  return b;
}

bool tcx_enabled();

ksc_status alloc_ws(ksc_problem* pr, int need, cudaStream_t s, BatchWs** out, bool exact_tc) {
  BatchWs* ws = new BatchWs();
  *out = ws;
  const int n = (int)pr->n, p = (int)pr->p;
  ws->Bcap = need;
  ws->Bpad = (need + 127) / 128 * 128;
  ws->ldp = pad8(p);
  ws->ldn = pad8(n);
  const int Bc = ws->Bcap, Bp = ws->Bpad, P = kBatchPieces;
  const size_t ldp = ws->ldp, ldn = ws->ldn;
  const int nft = (n + 63) / 64;
  BatchDev& d = ws->bd;
  ksc_status st;
#define BA(ptr, bytes) \
  if ((st = balloc(ws, &(ptr), (bytes))) != KSC_OK) return st
  int8_t* state = nullptr;
  BA(state, (size_t)Bc * ldp);
  d.state = state;
  BA(d.beta, (size_t)Bc * 3 * ldp * 8);
  BA(d.beta_ref, (size_t)Bc * ldp * 8);
  const bool e8 = pr->xdt == kXFP8;
  d.e8 = e8 ? 1 : 0;
  d.ldp8 = pad16(p);
  d.ldn8 = pad16(n);
  if (e8) {
    if (!tcx_enabled())
      return api_fail(KSC_ERR_UNIMPLEMENTED, "batched solves on E4M3 X take the tensor-core exact products");
    d.bpc = nullptr;
    d.rpc = nullptr;
    BA(d.bpc8, (size_t)kTcE4m3Pieces * Bp * d.ldp8);
    BA(d.rpc8, (size_t)kTcE4m3Pieces * Bp * d.ldn8);
    BA(d.rbuf, (size_t)Bc * ldn * 4);
    BA(d.rmaxp, (size_t)Bc * batch_nrt(n) * 4);
    BA(d.rs_fwd, (size_t)Bc * 4);
    BA(d.rs_grad, (size_t)Bc * 4);
    d.xscale = pr->dev.xscale;
  } else {
    BA(d.bpc, (size_t)P * Bp * ldp * 2);
    BA(d.rpc, (size_t)P * Bp * ldn * 2);
  }
  BA(d.U, (size_t)Bc * 3 * ldn * 8);
  BA(d.u_ref, (size_t)Bc * ldn * 8);
  BA(d.r_ref, (size_t)Bc * ldn * 8);
  BA(d.G, (size_t)Bc * ldp * 8);
  BA(d.G_ref, (size_t)Bc * ldp * 8);
  BA(d.slot_cur, (size_t)Bc * 4);
  BA(d.slot_new, (size_t)Bc * 4);
  BA(d.fpart, (size_t)Bc * nft * 2 * 8);
  BA(d.ncpart, (size_t)Bc * batch_nrt(n) * 8);
  BA(d.nodes, (size_t)Bc * sizeof(BNode));
  BA(d.cert, (size_t)Bc * sizeof(BCert));
  BA(d.beta_out, (size_t)Bc * p * 8);
  BA(d.z_out, (size_t)Bc * p * 8);
  BA(ws->dlist, (size_t)Bc * 4);
  BA(d.cert_u, (size_t)Bc * ldn * 8);
  BA(d.cert_z, (size_t)Bc * ldn * 8);
  BA(d.cert_a, (size_t)Bc * ldp * 8);
  BA(d.cpart, (size_t)Bc * batch_nrt(n) * 4 * 8);
  BA(d.dfws, kDfWsElems * 8);
  BA(d.tile_run, (size_t)(Bc + 127) / 128 * 4);
  ws->nsm = sm_count();
  BA(ws->skws, tc_skws_floats(ws->nsm, 256) * 4);
  BA(ws->r0, ldn * 8);
  BA(ws->G0, ldp * 8);
  KB_CUDA(cudaMemsetAsync(d.tile_run, 1, (size_t)(Bc + 127) / 128 * 4, s));   // nonzero: run every tile
  d.colnorm = pr->dev.colnorm;
  float* yf = nullptr;
  BA(yf, (size_t)n * 4);
  d.yf = yf;
  double* yd = nullptr;
  BA(yd, (size_t)n * 8);
  d.y = yd;
  // w of the prox in shared memory for short segments, else in (L2-resident) global scratch
  d.wsm = p <= 2048 ? p : 0;
  d.wbuf = nullptr;
  if (d.wsm == 0) BA(d.wbuf, (size_t)Bc * ldp * 8);
  // X for the TMA loads: row stride a multiple of 16 bytes, 16-byte aligned base
  if (!needs_xcopy(pr)) {
    ws->Xb = pr->X;
    ws->ldxb = pr->ldx;
  } else {
    // row stride in elements (BF16: ldp, E4M3: ldp8), a multiple of 16 bytes
    const size_t es = xelem(pr), lde = e8 ? (size_t)d.ldp8 : ldp;
    void* xb = nullptr;
    BA(xb, (size_t)n * lde * es);
    KB_CUDA(cudaMemcpy2DAsync(xb, lde * es, pr->X, pr->ldx * es, (size_t)p * es, n, cudaMemcpyDeviceToDevice, s));
    ws->Xb = xb;
    ws->ldxb = (int64_t)lde;
  }
#undef BA
  // every row the products read must be finite: zero the buffers once (E4M3 0x00 is +0)
  if (e8) {
    KB_CUDA(cudaMemsetAsync(d.bpc8, 0, (size_t)kTcE4m3Pieces * Bp * d.ldp8, s));
    KB_CUDA(cudaMemsetAsync(d.rpc8, 0, (size_t)kTcE4m3Pieces * Bp * d.ldn8, s));
    KB_CUDA(cudaMemsetAsync(d.rs_fwd, 0, (size_t)Bc * 4, s));
    KB_CUDA(cudaMemsetAsync(d.rs_grad, 0, (size_t)Bc * 4, s));
  } else {
    KB_CUDA(cudaMemsetAsync(d.bpc, 0, (size_t)P * Bp * ldp * 2, s));
    KB_CUDA(cudaMemsetAsync(d.rpc, 0, (size_t)P * Bp * ldn * 2, s));
  }
  KB_CUDA(cudaMemsetAsync(d.beta, 0, (size_t)Bc * 3 * ldp * 8, s));
  KB_CUDA(cudaMemsetAsync(d.U, 0, (size_t)Bc * 3 * ldn * 8, s));
  KB_CUDA(cudaMemsetAsync(d.u_ref, 0, (size_t)Bc * ldn * 8, s));
  KB_CUDA(cudaMemsetAsync(d.G_ref, 0, (size_t)Bc * ldp * 8, s));
  {
    std::vector<float> yh(n);
    for (int i = 0; i < n; ++i) yh[i] = (float)pr->y_host[i];
    KB_CUDA(cudaMemcpyAsync(yf, yh.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    KB_CUDA(cudaMemcpyAsync(yd, pr->y_host.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
    // ||X||_F and ||y||_2 rounded up, for the eigen-perspective certificate
    std::vector<double> cn(p);
    KB_CUDA(cudaMemcpyAsync(cn.data(), pr->dev.colnorm, (size_t)p * 8, cudaMemcpyDeviceToHost, s));
    KB_CUDA(cudaStreamSynchronize(s));
    const double ur = 1.1102230246251565e-16;
    double xf2 = 0.0, y2 = 0.0;
    for (int j = 0; j < p; ++j) xf2 += cn[j] * cn[j];
    for (int i = 0; i < n; ++i) y2 += pr->y_host[i] * pr->y_host[i];
    d.xfro = std::sqrt(xf2 * (1.0 + (p + 4.0) * ur)) * (1.0 + 4.0 * ur);
    d.ynorm = std::sqrt(y2 * (1.0 + (n + 4.0) * ur)) * (1.0 + 4.0 * ur);
  }
  d.n = n;
  d.p = p;
  d.loss = pr->loss;
  d.P = P;
  d.ldp = ws->ldp;
  d.ldn = ws->ldn;
  d.nrt = batch_nrt(n);
  d.nft = nft;
  d.Bpad = ws->Bpad;
  d.B = Bc;
  if ((exact_tc || e8) && tcx_enabled()) {
    const char* why = "";
    bool ok;
    if (e8) {
      // the slices are cut from the represented matrix X_ij s_j, exact in BF16
      // (4 significant bits times a power of two), held only while they are built
      void* t = nullptr;
      KB_CUDA(cudaMalloc(&t, std::max((size_t)n * d.ldp8, (size_t)p * d.ldn8) * 2));
      launch_fp8_to_bf16(pr->X, pr->ldx, n, p, pr->dev.xscale, 1, t, (int64_t)d.ldp8, s);
      ok = cudaGetLastError() == cudaSuccess;
      if (!ok) why = "the represented matrix could not be formed";
      ok = ok && tcx_slices_build(&ws->xs_fwd, t, n, p, d.ldp8, s, &why);
      if (ok) {
        launch_fp8_to_bf16(pr->dev.Xc, pr->dev.ldc, p, n, pr->dev.xscale, 0, t, (int64_t)d.ldn8, s);
        ok = cudaGetLastError() == cudaSuccess;
        if (!ok) why = "the represented matrix could not be formed";
        ok = ok && tcx_slices_build(&ws->xs_grad, t, p, n, d.ldn8, s, &why);
      }
      const cudaError_t se = cudaStreamSynchronize(s);
      cudaFree(t);
      KB_CUDA(se);
    } else {
      ok = tcx_slices_build(&ws->xs_fwd, pr->X, n, p, pr->ldx, s, &why) &&
           tcx_slices_build(&ws->xs_grad, pr->dev.Xc, p, n, pr->dev.ldc, s, &why);
    }
    if (!ok || !tcx_vecs_alloc(&ws->vs_fwd, Bc, p, &why) || !tcx_vecs_alloc(&ws->vs_grad, Bc, n, &why))
      return api_fail(KSC_ERR_OOM, std::string("exact tensor-core products: ") + why);
    ws->tcx = true;
    ws->bytes += ws->xs_fwd.bytes + ws->xs_grad.bytes + ws->vs_fwd.bytes + ws->vs_grad.bytes;
  }
  return KSC_OK;
}

// KSC_EXACT_PRODUCT=stream keeps the streaming double-float product for anchors and
// certificates (for comparisons); by default they run on the tensor cores
bool tcx_enabled() {
  const char* e = std::getenv("KSC_EXACT_PRODUCT");
  return !(e && std::strcmp(e, "stream") == 0);
}

// exact products of many nodes' vectors: D rows = X V rows (fwd, V of length p) or
// X^T V rows (V of length n), on the tensor cores when the workspace holds the
// slices of X, else the streaming double-float product; returns the error
// factor of the result (|D - exact| <= f ||x_c|| ||v||)
double exact_product(ksc_problem* pr, BatchWs* ws, bool fwd, const double* V, int64_t ldv, int R, double* D,
                     int64_t ldd, int kblock, cudaStream_t s) {
  const BatchDev& d = ws->bd;
  if (ws->tcx) {
    const TcxSlices& x = fwd ? ws->xs_fwd : ws->xs_grad;
    tcx_product(x, fwd ? ws->vs_fwd : ws->vs_grad, V, ldv, ws->dlist, R, D, ldd, s);
    pr->launches += tcx_launches(x, R);
    return tcx_error_factor(x);
  }
  // (E4M3 X always has the slices: alloc_ws refuses it otherwise; the streaming
  // product reads F64, F32 and BF16 X only)
  launch_dfprod(pr->dev, fwd, V, ldv, ws->dlist, R, D, ldd, d.dfws, kblock, s);
  pr->launches += 1 + (dfprod_splits(R, fwd ? d.n : d.p) > 1);
  return fwd ? dfprod_error_factor(d.p, R, d.n, kblock) : dfprod_error_factor(d.n, R, d.p, kblock);
}

TcEpi fwd_epi(const BatchWs* ws) {
  const BatchDev& d = ws->bd;
  TcEpi e{};
  e.base = d.u_ref;
  e.ldb = d.ldn;
  e.u64 = d.U;
  e.ldo = 3 * (int64_t)d.ldn;
  e.slot_in = d.slot_cur;
  e.slot_out = d.slot_new;
  e.slot_stride = d.ldn;
  e.y = d.yf;
  e.loss = d.loss;
  e.npart = d.nft;
  e.part = d.fpart;
  e.tile_active = d.tile_run;
  e.skws = ws->skws;
  if (d.e8) e.rscale = d.rs_fwd;
  return e;
}

TcEpi grad_epi(const BatchWs* ws) {
  const BatchDev& d = ws->bd;
  TcEpi e{};
  e.base = d.G_ref;
  e.ldb = d.ldp;
  e.out64 = d.G;
  e.ldo = d.ldp;
  e.tile_active = d.tile_run;
  e.skws = ws->skws;
  if (d.e8) {
    e.rscale = d.rs_grad;
    e.cscale = d.xscale;
  }
  return e;
}

// one batched step; ev (optional): 6 events around its 5 kernels
void enqueue_step(const BatchWs* ws, cudaStream_t s, const cudaEvent_t* ev) {
  auto mark = [&](int i) {
    if (ev) cudaEventRecordWithFlags(ev[i], s, cudaEventRecordExternal);
  };
  mark(0);
  launch_bresid(ws->bd, s);
  if (ws->bd.e8) launch_bsplit8_resid(ws->bd, s);
  mark(1);
  tc_launch(ws->grad, grad_epi(ws), kTcAdd, s);
  mark(2);
  launch_bprox(ws->bd, s);
  mark(3);
  tc_launch(ws->fwd, fwd_epi(ws), kTcAnchor, s);
  mark(4);
  launch_bstep(ws->bd, s);
  mark(5);
}

ksc_status capture(BatchWs* ws, bool prof) {
  cudaGraphExec_t* slot = prof ? &ws->graph_prof : &ws->graph;
  if (*slot) {
    cudaGraphExecDestroy(*slot);
    *slot = nullptr;
  }
  if (prof && ws->events.empty()) {
    ws->events.resize(6 * kBatchStepsPerGraph);
    for (auto& e : ws->events) KB_CUDA(cudaEventCreate(&e));
  }
  cudaStream_t cs;
  KB_CUDA(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
  cudaGraph_t g = nullptr;
  cudaError_t e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    for (int k = 0; k < kBatchStepsPerGraph; ++k) enqueue_step(ws, cs, prof ? &ws->events[6 * k] : nullptr);
    e = cudaStreamEndCapture(cs, &g);
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(slot, g, 0);
  if (g) cudaGraphDestroy(g);
  cudaStreamDestroy(cs);
  if (e != cudaSuccess) return api_fail(KSC_ERR_CUDA, std::string("batch graph capture: ") + cudaGetErrorString(e));
  return KSC_OK;
}

// tensor maps, tile widths (timed once per slot count) and the step graphs
ksc_status plan_batch(ksc_problem* pr, BatchWs* ws, int B, cudaStream_t s) {
  if (ws->B == B && ws->graph) return KSC_OK;
  BatchDev& d = ws->bd;
  d.B = B;
  const char* why = "";
  const Dev& sd = pr->dev;
  auto make = [&](int bf, int bg) -> bool {
    if (d.e8)
      return tc_plan(&ws->fwd, d.bpc8, kTcE4m3Pieces, B, ws->Bpad, d.p, d.ldp8, ws->Xb, d.n, ws->ldxb, bf, &why,
                     1) &&
             tc_plan(&ws->grad, d.rpc8, kTcE4m3Pieces, B, ws->Bpad, d.n, d.ldn8, sd.Xc, d.p, sd.ldc, bg, &why, 1);
    return tc_plan(&ws->fwd, d.bpc, d.P, B, ws->Bpad, d.p, d.ldp, ws->Xb, d.n, ws->ldxb, bf, &why) &&
           tc_plan(&ws->grad, d.rpc, d.P, B, ws->Bpad, d.n, d.ldn, sd.Xc, d.p, sd.ldc, bg, &why);
  };
  // autotune: time each tile width of each product (their outputs go to scratch:
  // u slot 2 and G of every row, before any node is admitted)
  cudaEvent_t e0, e1;
  KB_CUDA(cudaEventCreate(&e0));
  KB_CUDA(cudaEventCreate(&e1));
  float best_f = 1e30f, best_g = 1e30f;
  int bf = 128, bg = 128, sf = 0, sg = 0;
  std::vector<int> two(B, 2), zero(B, 0);
  KB_CUDA(cudaMemcpyAsync(d.slot_new, two.data(), (size_t)B * 4, cudaMemcpyHostToDevice, s));
  KB_CUDA(cudaMemcpyAsync(d.slot_cur, zero.data(), (size_t)B * 4, cudaMemcpyHostToDevice, s));
  // tile width x schedule (one CTA per tile, or stream-K over the SMs).  The
  // environment variable KSC_TC_SCHEDULE = tiled | stream_k restricts the choice
  // to one schedule (profilers distort the timings the choice is made on).
  const char* sched = std::getenv("KSC_TC_SCHEDULE");
  const int sk_lo = (sched && std::strcmp(sched, "stream_k") == 0) ? 1 : 0;
  const int sk_hi = (sched && std::strcmp(sched, "tiled") == 0) ? 0 : 1;
  // KSC_TC_TILE_FWD / KSC_TC_TILE_GRAD = 64 | 128 | 256 fix one product's tile width
  // (the other product's candidates are still timed)
  auto fixed_tile = [](const char* name) {
    const char* v = std::getenv(name);
    return v ? std::atoi(v) : 0;
  };
  const int fix_f = fixed_tile("KSC_TC_TILE_FWD"), fix_g = fixed_tile("KSC_TC_TILE_GRAD");
  for (int bn : kTcBNs) {
    if (d.e8 && bn > 128) continue;   // E4M3 tiles: two accumulators, at most 128 wide
    const int bnf = fix_f ? fix_f : bn, bng = fix_g ? fix_g : bn;
    for (int sk = sk_lo; sk <= sk_hi; ++sk) {
      bool ok = make(bnf, bng);
      if (ok && sk) ok = tc_plan_stream_k(&ws->fwd, ws->nsm, &why) && tc_plan_stream_k(&ws->grad, ws->nsm, &why);
      if (!ok) {
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        return api_fail(KSC_ERR_INVALID_ARG, std::string("batched products: ") + why);
      }
      for (int rep = 0; rep < 5; ++rep) {   // the first of each is a warm-up; the best of four counts
        float ms = 0.f;
        KB_CUDA(cudaEventRecord(e0, s));
        tc_launch(ws->fwd, fwd_epi(ws), kTcAnchor, s);
        KB_CUDA(cudaEventRecord(e1, s));
        KB_CUDA(cudaEventSynchronize(e1));
        KB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && ms < best_f) { best_f = ms; bf = bnf; sf = sk; }
        KB_CUDA(cudaEventRecord(e0, s));
        tc_launch(ws->grad, grad_epi(ws), kTcAdd, s);
        KB_CUDA(cudaEventRecord(e1, s));
        KB_CUDA(cudaEventSynchronize(e1));
        KB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
        if (rep > 0 && ms < best_g) { best_g = ms; bg = bng; sg = sk; }
      }
      pr->launches += sk ? 20 : 10;
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!make(bf, bg) || (sf && !tc_plan_stream_k(&ws->fwd, ws->nsm, &why)) ||
      (sg && !tc_plan_stream_k(&ws->grad, ws->nsm, &why)))
    return api_fail(KSC_ERR_INVALID_ARG, std::string("batched products: ") + why);
  ws->bn_fwd = bf;
  ws->bn_grad = bg;
  ws->sk_fwd = sf;
  ws->sk_grad = sg;
  ksc_status st;
  if ((st = capture(ws, false)) != KSC_OK) return st;
  if ((st = capture(ws, true)) != KSC_OK) return st;
  ws->B = B;
  return KSC_OK;
}

// device time of a phase of the host loop (profiling only): mark(true) before,
// mark(false) after; the elapsed time goes to kernel id `kid`
struct Phase {
  ksc_problem* pr;
  BatchWs* ws;
  cudaStream_t s;
  int kid;
  int count = 0;
  bool on = false;
  void begin() {
    if (!pr->profile) return;
    if (!ws->ph0) {
      cudaEventCreate(&ws->ph0);
      cudaEventCreate(&ws->ph1);
    }
    cudaEventRecord(ws->ph0, s);
    on = true;
  }
  void end() {
    if (!on) return;
    cudaEventRecord(ws->ph1, s);
    cudaEventSynchronize(ws->ph1);
    float ms = 0.f;
    cudaEventElapsedTime(&ms, ws->ph0, ws->ph1);
    pr->k_ms[kid] += ms;
    pr->k_launches[kid] += count;
    on = false;
  }
};

ksc_status check_tc(cudaStream_t s) {
  int word = 0;
  KB_CUDA(cudaMemcpyAsync(&word, tc_error_word(), sizeof word, cudaMemcpyDeviceToHost, s));
  KB_CUDA(cudaStreamSynchronize(s));
  if (word != 0) return api_fail(KSC_ERR_TIMEOUT, "tensor-core product: a device wait gave up");
  return KSC_OK;
}

// anchors of the listed slots at their current iterates (init: at the warm starts
// in slot 1).  Many nodes share one tiled exact product; a few take the streaming
// product, one node at a time.
constexpr int kAnchorTiled = 24;

ksc_status anchor(Session* se, const std::vector<int>& list, bool init) {
  if (list.empty()) return KSC_OK;
  BatchWs* ws = se->ws;
  const BatchDev& d = ws->bd;
  const Dev& sd = se->pr->dev;
  cudaStream_t s = se->s;
  const int cnt = (int)list.size();
  KB_CUDA(cudaMemcpyAsync(ws->dlist, list.data(), (size_t)cnt * 4, cudaMemcpyHostToDevice, s));
  if (!init) launch_banchor_copy(d, ws->dlist, cnt, s);
  const bool tiled = cnt >= kAnchorTiled || ws->tcx;
  if (tiled) {
    exact_product(se->pr, ws, true, d.beta_ref, d.ldp, cnt, d.u_ref, d.ldn, kDfBlockAnchor, s);
  } else {
    for (int b : list) launch_colsum_any(sd, true, d.beta_ref + (size_t)b * d.ldp, d.u_ref + (size_t)b * d.ldn, s);
  }
  launch_banchor_resid(d, ws->dlist, cnt, init ? 1 : 0, s);
  if (tiled) {
    exact_product(se->pr, ws, false, d.r_ref, d.ldn, cnt, d.G_ref, d.ldp, kDfBlockAnchor, s);
  } else {
    for (int b : list) launch_colsum_any(sd, false, d.r_ref + (size_t)b * d.ldn, d.G_ref + (size_t)b * d.ldp, s);
  }
  se->pr->launches += tiled ? kLaunchesPerAnchor - 2 : 2 + 2 * cnt;
  se->anchors += cnt;
  return KSC_OK;   // the list buffer's next upload is ordered after these kernels
}

}  // namespace

// ------------------------------------------------------------------ sessions

namespace ksc {

size_t session_bytes(const ksc_problem* pr, int slots) { return ws_bytes(pr, slots); }

ksc_status session_open(Session* se, ksc_problem* pr, int slots, bool use_problem_ws, cudaStream_t s) {
  if (slots < 1 || slots > kBatchMax) return api_fail(KSC_ERR_INVALID_ARG, "session slots out of range");
  if (!batch_supported(pr)) return api_fail(KSC_ERR_UNIMPLEMENTED, "batched solves need BF16 X");
  se->pr = pr;
  se->s = s;
  se->B = slots;
  ksc_status st;
  if (use_problem_ws) {
    if (!pr->batch || pr->batch->Bcap < slots) {
      if (pr->batch) {
        pr->bytes -= pr->batch->bytes;
        free_batch(pr->batch);
        pr->batch = nullptr;
      }
      BatchWs* ws = nullptr;
      st = alloc_ws(pr, std::max(slots, 128), s, &ws, true);
      if (st != KSC_OK) {
        free_batch(ws);
        return st;
      }
      pr->batch = ws;
      pr->bytes += ws->bytes;
    }
    se->ws = pr->batch;
    se->own_ws = false;
  } else {
    BatchWs* ws = nullptr;
    st = alloc_ws(pr, slots, s, &ws, false);
    if (st != KSC_OK) {
      free_batch(ws);
      return st;
    }
    se->ws = ws;
    se->own_ws = true;
  }
  if ((st = plan_batch(pr, se->ws, slots, s)) != KSC_OK) return st;
  // every slot starts empty
  se->slot.assign(slots, SlotHost());
  se->hn_raw.assign((size_t)slots * sizeof(BNode), 0);
  se->hc_raw.assign((size_t)slots * sizeof(BCert), 0);
  BNode* hn = hnodes(se);
  for (int b = 0; b < slots; ++b) {
    hn[b].done = kSlotIdle;
    hn[b].cur = 1;
    hn[b].prev = 0;
  }
  KB_CUDA(cudaMemcpyAsync(se->ws->bd.nodes, hn, (size_t)slots * sizeof(BNode), cudaMemcpyHostToDevice, s));
  KB_CUDA(cudaStreamSynchronize(s));
  return KSC_OK;
}

void session_close(Session* se) {
  if (se->own_ws) free_batch(se->ws);
  se->ws = nullptr;
  se->slot.clear();
}

int session_free_slots(const Session* se) {
  int f = 0;
  for (const auto& sl : se->slot) f += sl.busy ? 0 : 1;
  return f;
}

int session_running(const Session* se) {
  int r = 0;
  for (const auto& sl : se->slot) r += (sl.busy && !sl.fin) ? 1 : 0;
  return r;
}

// tiles with a running node (k_bstep clears a tile's flag when its last node stops)
ksc_status upload_tile_flags(Session* se) {
  const int tiles = (se->B + 127) / 128;
  se->tile_flags.assign(tiles, 0);
  for (int b = 0; b < se->B; ++b)
    if (se->slot[b].busy && !se->slot[b].fin) se->tile_flags[b / 128] = 1;
  KB_CUDA(cudaMemcpyAsync(se->ws->bd.tile_run, se->tile_flags.data(), (size_t)tiles * 4, cudaMemcpyHostToDevice,
                          se->s));
  return KSC_OK;
}

// r0 = grad F(0) and G0 = X^T r0 (exact double-float product), once per workspace
ksc_status zero_anchor_prepare(Session* se) {
  BatchWs* ws = se->ws;
  if (ws->zero_ready) return KSC_OK;
  ksc_problem* pr = se->pr;
  const int n = (int)pr->n;
  std::vector<double> r0(n);
  for (int i = 0; i < n; ++i)
    // grad F at u = 0: least squares -2 y, squared hinge -2 y (margin 1), logistic
    // -y/2, Poisson 1 - y (e^0 - y), Gamma 1 - y (1 - y e^0)
    r0[i] = pr->loss == KSC_LOSS_LOGISTIC ? -0.5 * pr->y_host[i]
            : loss_counts(pr->loss)       ? 1.0 - pr->y_host[i]
                                          : -2.0 * pr->y_host[i];
  cudaStream_t s = se->s;
  KB_CUDA(cudaMemcpyAsync(ws->r0, r0.data(), (size_t)n * 8, cudaMemcpyHostToDevice, s));
  const int zero_row = 0;
  KB_CUDA(cudaMemcpyAsync(ws->dlist, &zero_row, 4, cudaMemcpyHostToDevice, s));
  // G0 = X^T r0 by the workspace's exact product (the tensor-core slices when it
  // holds them -- always for FP8 X, which the streaming product cannot read)
  exact_product(pr, ws, false, ws->r0, ws->ldn, 1, ws->G0, ws->ldp, kDfBlockAnchor, s);
  KB_CUDA(cudaGetLastError());
  ws->zero_ready = true;
  return KSC_OK;
}

ksc_status session_admit(Session* se, const std::vector<const ksc_node*>& nodes, const std::vector<const NodeSetup*>& ns,
                         const std::vector<int>& want_z, std::vector<int>* slots) {
  const int cnt = (int)nodes.size();
  slots->clear();
  if (cnt == 0) return KSC_OK;
  if (cnt > session_free_slots(se)) return api_fail(KSC_ERR_ADMISSION, "no free slot");
  ksc_problem* pr = se->pr;
  BatchWs* ws = se->ws;
  BatchDev& d = ws->bd;
  const int p = (int)pr->p;
  const size_t ldp = ws->ldp;
  cudaStream_t s = se->s;
  BNode* hn = hnodes(se);
  // the nodes' state and warm-start rows are staged on the host in chunks of at
  // most 64 MB; each run of consecutive slots goes to the device in one copy per
  // array (a pageable source is staged by the copy before it returns, so the
  // buffers can be refilled without waiting for the device)
  const int chunk = (int)std::max<size_t>(1, ((size_t)64 << 20) / (ldp * 9));
  std::vector<int8_t> hs;
  std::vector<double> hb;
  int next = 0;
  for (int c0 = 0; c0 < cnt; c0 += chunk) {
    const int cn = std::min(chunk, cnt - c0);
    hs.assign((size_t)cn * ldp, (int8_t)kZero);
    hb.assign((size_t)cn * ldp, 0.0);
    for (int i = c0; i < c0 + cn; ++i) {
      while (se->slot[next].busy) ++next;
      const int b = next++;
      slots->push_back(b);
      const ksc_node* nd = nodes[i];
      const NodeSetup& setup = *ns[i];
      int8_t* hsr = hs.data() + (size_t)(i - c0) * ldp;
      double* hbr = hb.data() + (size_t)(i - c0) * ldp;
      std::memcpy(hsr, setup.state.data(), p);
      if (nd->warm_beta) {
        std::memcpy(hbr, nd->warm_beta, (size_t)p * 8);
        project_warm(pr, setup, nd->M, nd->k, hbr);
      }
      BNode& h = hn[b];
      std::memset(&h, 0, sizeof h);
      // eigen-perspective (App. D.2): lambda2 + eig on the perspective term, the
      // smooth part's constant 2 (lambda_max - eig) <= L - 2 eig
      const double eig = (nd->flags & KSC_FLAG_EIG) ? pr->eig_lambda : 0.0;
      const double Ln = node_lipschitz(pr, nd->M, nd->k) - 2.0 * eig;
      h.lambda2 = nd->lambda2 + eig;
      h.eig = eig;
      h.M = nd->M;
      h.rho = Ln / (2.0 * h.lambda2);
      h.invL = 1.0 / Ln;
      h.tol_loop = nd->rel_gap_tol;
      h.incumbent = nd->incumbent;
      h.kp = setup.kp;
      h.max_iter = nd->max_iter;
      h.restart_on = (nd->flags & KSC_FLAG_RESTART_OFF) ? 0 : 1;
      h.momentum_on = (nd->flags & KSC_FLAG_MOMENTUM_OFF) ? 0 : 1;
      h.done = kSlotIdle;   // k_binit_node starts it
      h.cur = 1;
      h.prev = 0;
      SlotHost& sl = se->slot[b];
      sl = SlotHost();
      sl.busy = true;
      sl.want_z = want_z[i];
      sl.tol = nd->rel_gap_tol;
      sl.inc = nd->incumbent;
      sl.anchor_gap = std::max(1e-3, 100.0 * nd->rel_gap_tol);
    }
    for (int i0 = c0; i0 < c0 + cn;) {
      int i1 = i0 + 1;
      while (i1 < c0 + cn && (*slots)[i1] == (*slots)[i1 - 1] + 1) ++i1;
      const int b0 = (*slots)[i0];
      const size_t run = (size_t)(i1 - i0);
      KB_CUDA(cudaMemcpyAsync((void*)(d.state + (size_t)b0 * ldp), hs.data() + (size_t)(i0 - c0) * ldp, run * ldp,
                              cudaMemcpyHostToDevice, s));
      KB_CUDA(cudaMemcpy2DAsync(d.beta + ((size_t)b0 * 3 + 1) * ldp, 3 * ldp * 8, hb.data() + (size_t)(i0 - c0) * ldp,
                                ldp * 8, ldp * 8, run, cudaMemcpyHostToDevice, s));
      KB_CUDA(cudaMemcpyAsync(d.nodes + b0, hn + b0, run * sizeof(BNode), cudaMemcpyHostToDevice, s));
      i0 = i1;
    }
  }
  KB_CUDA(cudaMemcpyAsync(ws->dlist, slots->data(), (size_t)cnt * 4, cudaMemcpyHostToDevice, s));
  launch_binit_copy(d, ws->dlist, cnt, s);
  pr->launches += 1;
  ksc_status st;
  const bool zero = cnt >= kZeroAnchorMin;
  if (zero) {
    // the zero anchor and one forward product for all admitted nodes (instead of
    // two exact products per node)
    if ((st = zero_anchor_prepare(se)) != KSC_OK) return st;
    KB_CUDA(cudaMemcpyAsync(ws->dlist, slots->data(), (size_t)cnt * 4, cudaMemcpyHostToDevice, s));
    launch_bzero_anchor(d, ws->dlist, cnt, ws->r0, ws->G0, s);
    if (d.e8) launch_bsplit8_beta(d, ws->dlist, cnt, s);
    if ((st = upload_tile_flags(se)) != KSC_OK) return st;
    tc_launch(ws->fwd, fwd_epi(ws), kTcAnchor, s);
    pr->launches += 4 + ws->sk_fwd;
  } else {
    if ((st = anchor(se, *slots, true)) != KSC_OK) return st;
  }
  KB_CUDA(cudaMemcpyAsync(ws->dlist, slots->data(), (size_t)cnt * 4, cudaMemcpyHostToDevice, s));
  launch_binit_node(d, ws->dlist, cnt, zero ? 1 : 0, s);
  pr->launches += 1;
  KB_CUDA(cudaGetLastError());
  return KSC_OK;   // stream order: the next replay runs after the admission
}

bool session_advance(Session* se, ksc_status* st) {
  *st = KSC_OK;
  if (session_running(se) == 0) return false;
  ksc_problem* pr = se->pr;
  if ((*st = upload_tile_flags(se)) != KSC_OK) return false;
  cudaError_t e = cudaGraphLaunch(pr->profile ? se->ws->graph_prof : se->ws->graph, se->s);
  if (e != cudaSuccess) {
    *st = api_fail(KSC_ERR_CUDA, std::string("batch graph launch: ") + cudaGetErrorString(e));
    return false;
  }
  pr->launches += (int64_t)(kLaunchesPerBatchStep + se->ws->bd.e8 + se->ws->sk_fwd + se->ws->sk_grad) *
                  kBatchStepsPerGraph;
  return true;
}

ksc_status session_collect(Session* se, std::vector<int>* finished) {
  ksc_problem* pr = se->pr;
  BatchWs* ws = se->ws;
  BatchDev& d = ws->bd;
  cudaStream_t s = se->s;
  const int B = se->B;
  BNode* hn = hnodes(se);
  BCert* hc = hcerts(se);
  KB_CUDA(cudaMemcpyAsync(hn, d.nodes, (size_t)B * sizeof(BNode), cudaMemcpyDeviceToHost, s));
  ksc_status st;
  if ((st = check_tc(s)) != KSC_OK) return st;
  if (pr->profile) {
    for (int k = 0; k < kBatchStepsPerGraph; ++k)
      for (int j = 0; j < 5; ++j) {
        float ms = 0.f;
        KB_CUDA(cudaEventElapsedTime(&ms, ws->events[6 * k + j], ws->events[6 * k + j + 1]));
        pr->k_ms[KSC_KERNEL_B_RESID + j] += ms;
        pr->k_launches[KSC_KERNEL_B_RESID + j] += 1;
      }
  }
  // nodes whose in-loop test fired, and nodes that have sat near their target for
  // a while without firing (their in-loop values can be off by the FP32 rounding
  // of the loss terms, ~1e-8 relative): certify both
  std::vector<int> fired;
  for (int b = 0; b < B; ++b) {
    const SlotHost& sl = se->slot[b];
    if (!sl.busy || sl.fin) continue;
    const BNode& h = hn[b];
    const bool stopped = h.done != kRunning;
    const bool overdue = h.iter - sl.last_cert >= 128 && h.gap <= 10.0 * sl.tol;
    if (stopped || overdue) fired.push_back(b);
  }
  // FP64 certificates of the nodes whose in-loop test fired
  Phase cert_phase{pr, ws, s, KSC_KERNEL_B_CERT};
  cert_phase.count = (int)fired.size();
  if (!fired.empty()) cert_phase.begin();
  if (!fired.empty()) {
    const int R = (int)fired.size();
    const Dev& sd = pr->dev;
    KB_CUDA(cudaMemcpyAsync(ws->dlist, fired.data(), (size_t)R * 4, cudaMemcpyHostToDevice, s));
    launch_bcert_prep(d, ws->dlist, R, s);
    const double err_u = exact_product(pr, ws, true, d.beta_out, d.p, R, d.cert_u, d.ldn, kDfBlockCert, s);
    launch_bcert_rows(d, ws->dlist, R, s);
    const double err_a = exact_product(pr, ws, false, d.cert_z, d.ldn, R, d.cert_a, d.ldp, kDfBlockCert, s);
    launch_bcert_final(d, ws->dlist, R, err_a, err_u, s);
    pr->launches += kLaunchesPerBatchCert - 2;
    se->certificates += R;
    KB_CUDA(cudaGetLastError());
    cert_phase.end();
    KB_CUDA(cudaMemcpyAsync(hc, d.cert, (size_t)B * sizeof(BCert), cudaMemcpyDeviceToHost, s));
    KB_CUDA(cudaStreamSynchronize(s));
  }
  Phase anchor_phase{pr, ws, s, KSC_KERNEL_B_ANCHOR};
  anchor_phase.begin();
  const int64_t anchors0 = se->anchors;
  bool upload = false;
  for (int b : fired) {
    SlotHost& sl = se->slot[b];
    const BNode& h = hn[b];
    const BCert& c = hc[b];
    sl.last_cert = h.iter;
    bool done = false;
    if (std::isfinite(sl.inc) && c.dual > sl.inc) { sl.pruned = 1; done = true; }
    else if (c.gap <= sl.tol) done = true;
    else if (h.done == kDonePrimal) done = true;                       // Sec. 4.3 rule (1): branch
    else if (h.done == kDoneMaxIter) { sl.status = KSC_NOT_CONVERGED; done = true; }
    if (done) {
      sl.fin = true;
      finished->push_back(b);
      if (h.done == kRunning) {   // certified while running: stop it on the device
        hn[b].done = kDoneGap;
        upload = true;
      }
      continue;
    }
    // the in-loop test fired on values the certificate does not confirm: go on
    // from the certificate's exact values (not from in-loop bests that rounding
    // may have moved past them), with a tighter in-loop tolerance
    BNode upd = h;
    // halve the in-loop tolerance (bounded below: an in-loop gap near the rounding
    // floor is noise, and chasing it would keep the node from ever stopping)
    if (h.done == kDoneGap)
      upd.tol_loop = std::max(0.5 * std::min(h.tol_loop, std::max(h.gap, 0.0)), std::max(1e-3 * sl.tol, kInLoopFloor));
    if (h.done == kDonePruned) upd.incumbent = sl.inc + 2.0 * std::fabs(h.best_dual - c.dual) + 1e-12 * std::fabs(sl.inc);
    upd.done = kRunning;
    upd.best_dual = c.dual > -INFINITY ? std::max(c.dual, -1e300) : -INFINITY;
    if (std::isfinite(c.primal)) upd.best_primal = c.primal;
    upd.gap = (upd.best_primal - upd.best_dual) / std::max(std::fabs(upd.best_primal), 1e-300);
    hn[b] = upd;
    upload = true;
  }
  // hn mirrors the device array (copied after the replay; only the certificate
  // kernels ran since, and they do not write nodes): one upload of every change
  if (upload) {
    KB_CUDA(cudaMemcpyAsync(d.nodes, hn, (size_t)B * sizeof(BNode), cudaMemcpyHostToDevice, s));
    KB_CUDA(cudaStreamSynchronize(s));
  }
  // anchors of running nodes whose gap fell (or that ran long without one)
  std::vector<int> alist;
  for (int b = 0; b < B; ++b) {
    SlotHost& sl = se->slot[b];
    const BNode& h = hn[b];
    if (!sl.busy || sl.fin || h.done != kRunning) continue;
    const bool by_gap = h.gap > 0.0 && h.gap <= sl.anchor_gap;
    const bool by_age = h.iter - sl.last_anchor >= 256 && h.gap > sl.tol;
    if (by_gap || by_age) {
      alist.push_back(b);
      sl.last_anchor = h.iter;
      sl.anchors += 1;
      if (by_gap) sl.anchor_gap = std::max(h.gap * 0.03, sl.tol * 1e-3);
    }
  }
  if ((st = anchor(se, alist, false)) != KSC_OK) return st;
  anchor_phase.count = (int)(se->anchors - anchors0);
  anchor_phase.end();
  KB_CUDA(cudaGetLastError());
  return KSC_OK;   // the anchors run while the host fetches results and launches the next replay
}

ksc_status session_fetch(Session* se, int b, ksc_result* r) {
  SlotHost& sl = se->slot[b];
  if (!sl.busy || !sl.fin) return api_fail(KSC_ERR_INVALID_ARG, "slot has no finished node");
  const BNode h = hnodes(se)[b];
  const BCert c = hcerts(se)[b];
  const BatchDev& d = se->ws->bd;
  const int p = d.p;
  r->primal = c.primal;
  r->dual_bound = c.dual;
  r->rel_gap = c.gap;
  r->iters = h.iter - 1;
  r->restarts = h.restarts;
  r->pruned = sl.pruned;
  r->status = sl.status;
  if (r->beta) KB_CUDA(cudaMemcpyAsync(r->beta, d.beta_out + (size_t)b * p, (size_t)p * 8, cudaMemcpyDeviceToHost, se->s));
  if (r->z) KB_CUDA(cudaMemcpyAsync(r->z, d.z_out + (size_t)b * p, (size_t)p * 8, cudaMemcpyDeviceToHost, se->s));
  // empty the slot: every kernel skips it
  BNode idle = h;
  idle.done = kSlotIdle;
  KB_CUDA(cudaMemcpyAsync(d.nodes + b, &idle, sizeof idle, cudaMemcpyHostToDevice, se->s));
  // the caller's arrays may be pinned (then the copies are asynchronous): results
  // must be in host memory on return
  if (r->beta || r->z) KB_CUDA(cudaStreamSynchronize(se->s));
  hnodes(se)[b] = idle;
  sl = SlotHost();
  return KSC_OK;
}

}  // namespace ksc

// ------------------------------------------------------------------ ksc_solve_batch

extern "C" ksc_status ksc_solve_batch(ksc_problem* pr, const ksc_node* nodes, int32_t count, ksc_result* results,
                                      void* cuda_stream) {
  if (!pr || (count > 0 && (!nodes || !results)) || count < 0) return api_fail(KSC_ERR_INVALID_ARG, "bad arguments");
  if (count == 0) return KSC_OK;
  ksc_status st = ensure_prepared();
  if (st != KSC_OK) return st;
  cudaStream_t s = (cudaStream_t)cuda_stream;
  int cur_dev = 0;
  cudaGetDevice(&cur_dev);
  if (cur_dev != pr->device) KB_CUDA(cudaSetDevice(pr->device));
  // the eigen shift, computed on first use
  for (int32_t i = 0; i < count; ++i)
    if ((nodes[i].flags & KSC_FLAG_EIG) && !pr->eig_ready) {
      double lam = 0.0;
      if ((st = ksc_problem_eig_lambda(pr, cuda_stream, &lam)) != KSC_OK) return st;
      break;
    }
  // validate every node first: nothing runs on a bad batch
  std::vector<NodeSetup> setups(count);
  std::vector<int> batch, single;
  ksc_status first = KSC_OK;
  for (int32_t i = 0; i < count; ++i) {
    if ((st = check_node(pr, &nodes[i], &setups[i])) != KSC_OK) return st;
    ksc_result* r = &results[i];
    r->iters = 0;
    r->restarts = 0;
    r->pruned = 0;
    if (setups[i].infeasible) {
      r->primal = INFINITY;
      r->dual_bound = INFINITY;
      r->rel_gap = 0.0;
      r->pruned = 1;
      r->status = KSC_ERR_INFEASIBLE_NODE;
      if (first == KSC_OK) first = KSC_ERR_INFEASIBLE_NODE;
      continue;
    }
    const bool eig_fp8 = (nodes[i].flags & KSC_FLAG_EIG) && pr->xdt == kXFP8;
    if (batch_supported(pr) && !eig_fp8 && std::min<int64_t>(setups[i].kp, pr->p) < kBatchCap) batch.push_back(i);
    else single.push_back(i);
  }
  // nodes with more free support entries run longer: grouping them in the same
  // 128-slot tiles lets the products skip the tiles of the faster nodes sooner
  std::stable_sort(batch.begin(), batch.end(), [&](int a, int b) { return setups[a].kp > setups[b].kp; });
  int64_t iters = 0, anchors = 0, certs = 0, fallbacks = 0;
  int tiles[4] = {0, 0, 0, 0};   // the products' tile widths and schedules (last pass)
  for (size_t g0 = 0; g0 < batch.size(); g0 += kBatchMax) {
    const int cnt = (int)std::min<size_t>(kBatchMax, batch.size() - g0);
    Session se;
    if ((st = session_open(&se, pr, cnt, true, s)) != KSC_OK) return st;
    std::vector<const ksc_node*> nv;
    std::vector<const NodeSetup*> sv;
    std::vector<int> wz, slots;
    for (int i = 0; i < cnt; ++i) {
      const int idx = batch[g0 + i];
      nv.push_back(&nodes[idx]);
      sv.push_back(&setups[idx]);
      wz.push_back(results[idx].z != nullptr);
    }
    if ((st = session_admit(&se, nv, sv, wz, &slots)) != KSC_OK) return st;
    std::vector<int> fin;
    while (session_running(&se) > 0) {
      if (!session_advance(&se, &st)) {
        if (st != KSC_OK) return st;
        break;
      }
      if ((st = session_collect(&se, &fin)) != KSC_OK) return st;
    }
    if (g0 == 0) pr->batch_state.assign((size_t)count * 10, NAN);
    // the certified iterates (and relaxed z) of the whole group in one copy each
    bool any_beta = false, any_z = false;
    int smax = 0;
    for (int i = 0; i < cnt; ++i) {
      any_beta |= results[batch[g0 + i]].beta != nullptr;
      any_z |= results[batch[g0 + i]].z != nullptr;
      smax = std::max(smax, slots[i] + 1);
    }
    std::vector<double> hbeta, hz;
    const size_t pp = (size_t)pr->p;
    if (any_beta) {
      hbeta.resize((size_t)smax * pp);
      KB_CUDA(cudaMemcpyAsync(hbeta.data(), se.ws->bd.beta_out, hbeta.size() * 8, cudaMemcpyDeviceToHost, s));
    }
    if (any_z) {
      hz.resize((size_t)smax * pp);
      KB_CUDA(cudaMemcpyAsync(hz.data(), se.ws->bd.z_out, hz.size() * 8, cudaMemcpyDeviceToHost, s));
    }
    if (any_beta || any_z) KB_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < cnt; ++i) {
      const int idx = batch[g0 + i];
      const BNode& h = hnodes(&se)[slots[i]];
      double* bs = &pr->batch_state[(size_t)idx * 10];
      bs[0] = h.tol_loop;
      bs[1] = h.best_primal;
      bs[2] = h.best_dual;
      bs[3] = h.gap;
      bs[4] = h.last_primal;
      bs[5] = h.last_dual;
      bs[6] = h.g_cur;
      bs[7] = h.restarts;
      bs[8] = h.iter - 1;
      bs[9] = hcerts(&se)[slots[i]].gap;
      fallbacks += h.fallback;
      ksc_result* rr = &results[idx];
      double* ub = rr->beta;
      double* uz = rr->z;
      rr->beta = nullptr;
      rr->z = nullptr;
      st = session_fetch(&se, slots[i], rr);
      rr->beta = ub;
      rr->z = uz;
      if (st != KSC_OK) return st;
      if (ub) std::memcpy(ub, hbeta.data() + (size_t)slots[i] * pp, pp * 8);
      if (uz) std::memcpy(uz, hz.data() + (size_t)slots[i] * pp, pp * 8);
      iters += results[idx].iters;
      if (first == KSC_OK && results[idx].status != KSC_OK) first = results[idx].status;
    }
    anchors += se.anchors;
    certs += se.certificates;
    tiles[0] = se.ws->bn_fwd;
    tiles[1] = se.ws->sk_fwd;
    tiles[2] = se.ws->bn_grad;
    tiles[3] = se.ws->sk_grad;
    session_close(&se);
  }
  if (!batch.empty()) {
    for (int i = 0; i < 12; ++i) pr->last_stats[i] = 0;
    for (int i = 0; i < 4; ++i) pr->last_stats[8 + i] = tiles[i];
    pr->last_stats[0] = (int32_t)std::min<int64_t>(iters, INT32_MAX);
    pr->last_stats[2] = (int32_t)std::min<int64_t>(fallbacks, INT32_MAX);
    pr->last_stats[5] = pr->power_iters;
    pr->last_stats[6] = (int32_t)std::min<int64_t>(certs, INT32_MAX);
    pr->last_stats[7] = (int32_t)std::min<int64_t>(anchors, INT32_MAX);
  }
  for (int i : single) {
    st = ksc_solve_node(pr, &nodes[i], &results[i], cuda_stream);
    if (st != KSC_OK && st != KSC_NOT_CONVERGED && st != KSC_ERR_INFEASIBLE_NODE) return st;
    if (first == KSC_OK && st != KSC_OK) first = st;
  }
  if (first != KSC_OK && first != KSC_ERR_INFEASIBLE_NODE)
    return api_fail(first, "a node reached max_iter before the gap target");
  if (first == KSC_ERR_INFEASIBLE_NODE) return api_fail(first, "a node is infeasible: |S1| > k or S0 and S1 intersect");
  return KSC_OK;
}

extern "C" ksc_status ksc_problem_batch_node_state(const ksc_problem* pr, int32_t index, double* state, int32_t n) {
  if (!pr || (n > 0 && !state) || n < 0) return api_fail(KSC_ERR_INVALID_ARG, "bad arguments");
  if (index < 0 || (size_t)index * 10 >= pr->batch_state.size() || std::isnan(pr->batch_state[(size_t)index * 10]))
    return api_fail(KSC_ERR_INVALID_ARG, "index is not a node of the last batched call");
  for (int32_t i = 0; i < n; ++i) state[i] = i < 10 ? pr->batch_state[(size_t)index * 10 + i] : 0.0;
  return KSC_OK;
}
