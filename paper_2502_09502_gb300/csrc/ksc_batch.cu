// ksc_batch.cu -- ksc_solve_batch: many nodes of one problem solved together.
//
// Nodes with BF16 X advance in lock step through restarted FISTA (Algorithm 3):
// per step one residual kernel, the product X^T r on the tensor cores, one prox
// CTA per node, the product X beta on the tensor cores, and the per-node step
// logic -- 16 steps per CUDA-graph replay.  A node whose in-loop test fires is
// frozen; its FP64 certificate (Sec. 3.4) is computed through the single-node
// workspace, and the node either finishes or resumes with a tighter in-loop
// tolerance, exactly as in ksc_solve_node.  Nodes the batched path does not take
// (X not BF16, k' beyond the per-node candidate capacity) are solved one by one.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>
#include <vector>

#include "ksc_batch.cuh"
#include "ksc_problem.h"
#include "ksc_tc.h"

namespace ksc {

struct BatchWs {
  int Bcap = 0;      // nodes the buffers hold
  int Bpad = 0;      // Bcap rounded up to 128 (row stride of the BF16 pieces)
  int ldp = 0, ldn = 0;
  int B = -1;        // nodes of the current plans and graph
  int bn_fwd = 0, bn_grad = 0;
  int nft_max = 0;
  std::vector<void*> allocs;
  size_t bytes = 0;
  BatchDev bd{};
  TcPlan fwd{}, grad{};
  cudaGraphExec_t graph = nullptr;
  cudaGraphExec_t graph_prof = nullptr;   // the same steps with events between the kernels
  std::vector<cudaEvent_t> events;        // 6 per step of graph_prof
  const void* Xb = nullptr;   // X with a TMA-compatible row stride (the problem's, or a copy)
  int64_t ldxb = 0;
};

void free_batch(BatchWs* ws) {
  if (!ws) return;
  if (ws->graph) cudaGraphExecDestroy(ws->graph);
  if (ws->graph_prof) cudaGraphExecDestroy(ws->graph_prof);
  for (auto e : ws->events) cudaEventDestroy(e);
  for (void* v : ws->allocs) cudaFree(v);
  delete ws;
}

}  // namespace ksc

using namespace ksc;

namespace {

constexpr int kBatchStepsPerGraph = 16;
constexpr int kLaunchesPerBatchStep = 5;   // residual, X^T r, prox, X beta, step
constexpr int kLaunchesPerBatchCert = 7;   // load, 5 certificate kernels, store

#define KB_CUDA(call)                                                                        \
  do {                                                                                       \
    cudaError_t e_ = (call);                                                                 \
    if (e_ != cudaSuccess)                                                                   \
      return api_fail(e_ == cudaErrorMemoryAllocation ? KSC_ERR_OOM : KSC_ERR_CUDA,          \
                      std::string(#call) + ": " + cudaGetErrorString(e_));                   \
  } while (0)

template <typename P>
ksc_status balloc(ksc_problem* pr, BatchWs* ws, P** ptr, size_t bytes) {
  void* v = nullptr;
  cudaError_t e = cudaMalloc(&v, bytes > 0 ? bytes : 16);
  if (e != cudaSuccess)
    return api_fail(KSC_ERR_OOM, std::string("cudaMalloc(") + std::to_string(bytes) + "): " + cudaGetErrorString(e));
  ws->allocs.push_back(v);
  ws->bytes += bytes;
  pr->bytes += bytes;
  *ptr = (P*)v;
  return KSC_OK;
}

bool batch_supported(const ksc_problem* pr) { return pr->xdt == kXBF16; }

// buffers for up to `need` nodes
ksc_status ensure_ws(ksc_problem* pr, int need, cudaStream_t s) {
  BatchWs* ws = pr->batch;
  if (ws && ws->Bcap >= need) return KSC_OK;
  if (ws) {
    pr->bytes -= ws->bytes;
    free_batch(ws);
    pr->batch = nullptr;
  }
  ws = new BatchWs();
  pr->batch = ws;
  const int n = (int)pr->n, p = (int)pr->p;
  ws->Bcap = need;
  ws->Bpad = (need + 127) / 128 * 128;
  ws->ldp = (p + 7) / 8 * 8;
  ws->ldn = (n + 7) / 8 * 8;
  ws->nft_max = (n + 63) / 64;   // loss partials: one per 64 columns
  const int Bc = ws->Bcap, Bp = ws->Bpad, P = kBatchPieces;
  const size_t ldp = ws->ldp, ldn = ws->ldn;
  BatchDev& d = ws->bd;
  ksc_status st;
#define BA(ptr, bytes) \
  if ((st = balloc(pr, ws, &(ptr), (bytes))) != KSC_OK) return st
  int8_t* state = nullptr;
  BA(state, (size_t)Bc * ldp);
  d.state = state;
  BA(d.beta, (size_t)Bc * 3 * ldp * 4);
  BA(d.bpc, (size_t)P * Bp * ldp * 2);
  BA(d.U, (size_t)Bc * 3 * ldn * 8);
  BA(d.rpc, (size_t)P * Bp * ldn * 2);
  BA(d.G, (size_t)Bc * ldp * 4);
  BA(d.slot_cur, (size_t)Bc * 4);
  BA(d.slot_new, (size_t)Bc * 4);
  BA(d.fpart, (size_t)Bc * ws->nft_max * 2 * 8);
  BA(d.ncpart, (size_t)Bc * batch_nrt(n) * 8);
  BA(d.nodes, (size_t)Bc * sizeof(BNode));
  BA(d.cert, (size_t)Bc * sizeof(BCert));
  BA(d.beta_out, (size_t)Bc * p * 8);
  BA(d.z_out, (size_t)Bc * p * 8);
  float* yf = nullptr;
  BA(yf, (size_t)n * 4);
  d.yf = yf;
  // w of the prox in shared memory when it fits (4 CTAs per SM at p = 5000)
  d.wsm = bprox_smem_bytes(p) <= 200 * 1024 ? p : 0;
  d.wbuf = nullptr;
  if (d.wsm == 0) BA(d.wbuf, (size_t)Bc * ldp * 4);
  // X for the TMA loads: row stride a multiple of 16 bytes, 16-byte aligned base
  if ((pr->ldx * 2) % 16 == 0 && ((uintptr_t)pr->X % 16) == 0) {
    ws->Xb = pr->X;
    ws->ldxb = pr->ldx;
  } else {
    void* xb = nullptr;
    BA(xb, (size_t)n * ldp * 2);
    KB_CUDA(cudaMemcpy2DAsync(xb, ldp * 2, pr->X, pr->ldx * 2, (size_t)p * 2, n, cudaMemcpyDeviceToDevice, s));
    ws->Xb = xb;
    ws->ldxb = (int64_t)ldp;
  }
#undef BA
  // every row the products read must be finite: zero the pieces once
  KB_CUDA(cudaMemsetAsync(d.bpc, 0, (size_t)P * Bp * ldp * 2, s));
  KB_CUDA(cudaMemsetAsync(d.rpc, 0, (size_t)P * Bp * ldn * 2, s));
  KB_CUDA(cudaMemsetAsync(d.beta, 0, (size_t)Bc * 3 * ldp * 4, s));
  KB_CUDA(cudaMemsetAsync(d.U, 0, (size_t)Bc * 3 * ldn * 8, s));
  {
    std::vector<float> yh(n);
    for (int i = 0; i < n; ++i) yh[i] = (float)pr->y_host[i];
    KB_CUDA(cudaMemcpyAsync(yf, yh.data(), (size_t)n * 4, cudaMemcpyHostToDevice, s));
    KB_CUDA(cudaStreamSynchronize(s));
  }
  d.n = n;
  d.p = p;
  d.loss = pr->loss;
  d.P = P;
  d.ldp = ws->ldp;
  d.ldn = ws->ldn;
  d.nrt = batch_nrt(n);
  d.nft = ws->nft_max;
  d.Bpad = ws->Bpad;
  return KSC_OK;
}

TcEpi fwd_epi(const BatchWs* ws) {
  const BatchDev& d = ws->bd;
  TcEpi e{};
  e.u64 = d.U;
  e.ldo = 3 * (int64_t)d.ldn;
  e.slot_in = d.slot_cur;
  e.slot_out = d.slot_new;
  e.slot_stride = d.ldn;
  e.y = d.yf;
  e.loss = d.loss;
  e.npart = d.nft;
  e.part = d.fpart;
  return e;
}

TcEpi grad_epi(const BatchWs* ws) {
  TcEpi e{};
  e.out = ws->bd.G;
  e.ldo = ws->bd.ldp;
  return e;
}

// one batched step; ev (optional): 6 events around its 5 kernels
void enqueue_step(const BatchWs* ws, cudaStream_t s, const cudaEvent_t* ev) {
  auto mark = [&](int i) {
    if (ev) cudaEventRecordWithFlags(ev[i], s, cudaEventRecordExternal);
  };
  mark(0);
  launch_bresid(ws->bd, s);
  mark(1);
  tc_launch(ws->grad, grad_epi(ws), kTcStore, s);
  mark(2);
  launch_bprox(ws->bd, s);
  mark(3);
  tc_launch(ws->fwd, fwd_epi(ws), kTcDelta, s);
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

// tensor maps, tile widths (timed once per batch size) and the step graph for B nodes
ksc_status plan_batch(ksc_problem* pr, int B, cudaStream_t s) {
  BatchWs* ws = pr->batch;
  if (ws->B == B && ws->graph) return KSC_OK;
  BatchDev& d = ws->bd;
  d.B = B;
  const char* why = "";
  const Dev& sd = pr->dev;
  auto make = [&](int bf, int bg) -> bool {
    return tc_plan(&ws->fwd, d.bpc, d.P, B, ws->Bpad, d.p, d.ldp, ws->Xb, d.n, ws->ldxb, bf, &why) &&
           tc_plan(&ws->grad, d.rpc, d.P, B, ws->Bpad, d.n, d.ldn, sd.Xc, d.p, sd.ldc, bg, &why);
  };
  // autotune: time each tile width of each product on the current buffers
  cudaEvent_t e0, e1;
  KB_CUDA(cudaEventCreate(&e0));
  KB_CUDA(cudaEventCreate(&e1));
  float best_f = 1e30f, best_g = 1e30f;
  int bf = 128, bg = 128;
  for (int bn : kTcBNs) {
    if (!make(bn, bn)) {
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      return api_fail(KSC_ERR_INVALID_ARG, std::string("batched products: ") + why);
    }
    KB_CUDA(cudaMemsetAsync(d.slot_new, 0, (size_t)B * 4, s));
    KB_CUDA(cudaMemsetAsync(d.slot_cur, 0, (size_t)B * 4, s));
    for (int rep = 0; rep < 3; ++rep) {
      KB_CUDA(cudaEventRecord(e0, s));
      tc_launch(ws->fwd, fwd_epi(ws), kTcDelta, s);
      KB_CUDA(cudaEventRecord(e1, s));
      KB_CUDA(cudaEventSynchronize(e1));
      float ms = 0.f;
      KB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0 && ms < best_f) { best_f = ms; bf = bn; }
      KB_CUDA(cudaEventRecord(e0, s));
      tc_launch(ws->grad, grad_epi(ws), kTcStore, s);
      KB_CUDA(cudaEventRecord(e1, s));
      KB_CUDA(cudaEventSynchronize(e1));
      KB_CUDA(cudaEventElapsedTime(&ms, e0, e1));
      if (rep > 0 && ms < best_g) { best_g = ms; bg = bn; }
    }
    pr->launches += 6;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (!make(bf, bg)) return api_fail(KSC_ERR_INVALID_ARG, std::string("batched products: ") + why);
  ws->bn_fwd = bf;
  ws->bn_grad = bg;
  // the step graphs (plain, and with events for ksc_problem_kernel_time)
  ksc_status st;
  if ((st = capture(ws, false)) != KSC_OK) return st;
  if ((st = capture(ws, true)) != KSC_OK) return st;
  ws->B = B;
  return KSC_OK;
}

ksc_status check_tc(cudaStream_t s) {
  int word = 0;
  KB_CUDA(cudaMemcpyAsync(&word, tc_error_word(), sizeof word, cudaMemcpyDeviceToHost, s));
  KB_CUDA(cudaStreamSynchronize(s));
  if (word != 0) return api_fail(KSC_ERR_TIMEOUT, "tensor-core product: a device wait gave up");
  return KSC_OK;
}

struct Job {
  int idx;            // position in the caller's arrays
  NodeSetup ns;
};

// solve up to kBatchMax nodes in one device pass
ksc_status solve_group(ksc_problem* pr, const ksc_node* nodes, ksc_result* results, std::vector<Job>& jobs,
                       cudaStream_t s) {
  const int B = (int)jobs.size();
  const int p = (int)pr->p;
  ksc_status st;
  if ((st = ensure_ws(pr, std::max(B, pr->batch ? pr->batch->Bcap : 0), s)) != KSC_OK) return st;
  BatchWs* ws = pr->batch;
  BatchDev& d = ws->bd;
  d.B = B;
  const size_t ldp = ws->ldp;
  // per-node inputs: coordinate states, projected warm starts (slot 1), parameters
  {
    std::vector<int8_t> hs((size_t)B * ldp, (int8_t)kZero);
    std::vector<float> hb((size_t)B * ldp, 0.0f);
    std::vector<BNode> hn(B);
    for (int b = 0; b < B; ++b) {
      const ksc_node* nd = &nodes[jobs[b].idx];
      const NodeSetup& ns = jobs[b].ns;
      std::memcpy(&hs[(size_t)b * ldp], ns.state.data(), p);
      if (nd->warm_beta)
        for (int j = 0; j < p; ++j)
          hb[(size_t)b * ldp + j] =
              ns.state[j] == kZero ? 0.0f : (float)std::min(nd->M, std::max(-nd->M, nd->warm_beta[j]));
      BNode& h = hn[b];
      std::memset(&h, 0, sizeof h);
      h.lambda2 = nd->lambda2;
      h.M = nd->M;
      h.rho = pr->L / (2.0 * nd->lambda2);
      h.invL = 1.0 / pr->L;
      h.tol_loop = nd->rel_gap_tol;
      h.incumbent = nd->incumbent;
      h.kp = ns.kp;
      h.max_iter = nd->max_iter;
      h.restart_on = (nd->flags & KSC_FLAG_RESTART_OFF) ? 0 : 1;
      h.momentum_on = (nd->flags & KSC_FLAG_MOMENTUM_OFF) ? 0 : 1;
    }
    KB_CUDA(cudaMemcpy2DAsync((void*)d.state, ldp, hs.data(), ldp, (size_t)p, B, cudaMemcpyHostToDevice, s));
    KB_CUDA(cudaMemcpy2DAsync(d.beta + ldp, 3 * ldp * 4, hb.data(), ldp * 4, ldp * 4, B, cudaMemcpyHostToDevice, s));
    KB_CUDA(cudaMemcpyAsync(d.nodes, hn.data(), (size_t)B * sizeof(BNode), cudaMemcpyHostToDevice, s));
  }
  if ((st = plan_batch(pr, B, s)) != KSC_OK) return st;
  tc_clear_error(s);
  launch_binit_split(d, s);
  tc_launch(ws->fwd, fwd_epi(ws), kTcDelta, s);
  launch_binit_node(d, s);
  pr->launches += 3;
  KB_CUDA(cudaGetLastError());

  std::vector<BNode> hn(B);
  std::vector<BCert> hc(B);
  std::vector<char> fin(B, 0);
  std::vector<int> pruned(B, 0);
  std::vector<ksc_status> status(B, KSC_OK);
  int remaining = B;
  while (remaining > 0) {
    KB_CUDA(cudaGraphLaunch(pr->profile ? ws->graph_prof : ws->graph, s));
    pr->launches += (int64_t)kLaunchesPerBatchStep * kBatchStepsPerGraph;
    KB_CUDA(cudaMemcpyAsync(hn.data(), d.nodes, (size_t)B * sizeof(BNode), cudaMemcpyDeviceToHost, s));
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
    std::vector<int> fired;
    for (int b = 0; b < B; ++b)
      if (!fin[b] && hn[b].done != kRunning) fired.push_back(b);
    if (fired.empty()) continue;
    // FP64 certificates of the nodes whose in-loop test fired
    for (int b : fired) {
      const int want_z = results[jobs[b].idx].z != nullptr;
      launch_bcert_load(d, b, pr->dev, s);
      launch_certificate(pr->dev, s, want_z);
      launch_bcert_store(d, b, pr->dev, want_z, s);
      pr->launches += kLaunchesPerBatchCert;
    }
    KB_CUDA(cudaGetLastError());
    KB_CUDA(cudaMemcpyAsync(hc.data(), d.cert, (size_t)B * sizeof(BCert), cudaMemcpyDeviceToHost, s));
    KB_CUDA(cudaStreamSynchronize(s));
    for (int b : fired) {
      const ksc_node* nd = &nodes[jobs[b].idx];
      const double tol = nd->rel_gap_tol, inc = nd->incumbent;
      const BNode& h = hn[b];
      const BCert& c = hc[b];
      bool done = false;
      if (std::isfinite(inc) && c.dual > inc) { pruned[b] = 1; done = true; }
      else if (c.gap <= tol) done = true;
      else if (h.done == kDonePrimal) done = true;                       // Sec. 4.3 rule (1): branch
      else if (h.done == kDoneMaxIter) { status[b] = KSC_NOT_CONVERGED; done = true; }
      if (done) {
        fin[b] = 1;
        --remaining;
        continue;
      }
      // the in-loop test fired on values the certificate does not confirm
      BNode upd = h;
      if (h.done == kDoneGap) upd.tol_loop = std::max(h.gap * 0.25, 1e-16);
      if (h.done == kDonePruned) upd.incumbent = inc + 2.0 * std::fabs(h.best_dual - c.dual) + 1e-12 * std::fabs(inc);
      upd.done = kRunning;
      upd.best_dual = c.dual > -INFINITY ? std::max(c.dual, -1e300) : -INFINITY;
      KB_CUDA(cudaMemcpyAsync(d.nodes + b, &upd, sizeof upd, cudaMemcpyHostToDevice, s));
      hn[b] = upd;
    }
    KB_CUDA(cudaStreamSynchronize(s));
  }
  // results
  for (int b = 0; b < B; ++b) {
    ksc_result* r = &results[jobs[b].idx];
    r->primal = hc[b].primal;
    r->dual_bound = hc[b].dual;
    r->rel_gap = hc[b].gap;
    r->iters = hn[b].iter - 1;
    r->restarts = hn[b].restarts;
    r->pruned = pruned[b];
    r->status = status[b];
    if (r->beta) KB_CUDA(cudaMemcpyAsync(r->beta, d.beta_out + (size_t)b * p, (size_t)p * 8, cudaMemcpyDeviceToHost, s));
    if (r->z) KB_CUDA(cudaMemcpyAsync(r->z, d.z_out + (size_t)b * p, (size_t)p * 8, cudaMemcpyDeviceToHost, s));
  }
  KB_CUDA(cudaStreamSynchronize(s));
  int64_t it = 0;
  for (int b = 0; b < B; ++b) it += hn[b].iter - 1;
  pr->last_stats[0] = (int32_t)std::min<int64_t>(it, INT32_MAX);
  return KSC_OK;
}

}  // namespace

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
  // validate every node first: nothing runs on a bad batch
  std::vector<Job> batch;
  std::vector<int> single;
  ksc_status first = KSC_OK;
  for (int32_t i = 0; i < count; ++i) {
    Job j;
    j.idx = i;
    if ((st = check_node(pr, &nodes[i], &j.ns)) != KSC_OK) return st;
    ksc_result* r = &results[i];
    r->iters = 0;
    r->restarts = 0;
    r->pruned = 0;
    if (j.ns.infeasible) {
      r->primal = INFINITY;
      r->dual_bound = INFINITY;
      r->rel_gap = 0.0;
      r->pruned = 1;
      r->status = KSC_ERR_INFEASIBLE_NODE;
      if (first == KSC_OK) first = KSC_ERR_INFEASIBLE_NODE;
      continue;
    }
    if (batch_supported(pr) && std::min<int64_t>(j.ns.kp, pr->p) < kBatchCap) batch.push_back(std::move(j));
    else single.push_back(i);
  }
  for (size_t g0 = 0; g0 < batch.size(); g0 += kBatchMax) {
    std::vector<Job> grp(std::make_move_iterator(batch.begin() + g0),
                         std::make_move_iterator(batch.begin() + std::min(batch.size(), g0 + kBatchMax)));
    if ((st = solve_group(pr, nodes, results, grp, s)) != KSC_OK) return st;
    for (auto& j : grp)
      if (first == KSC_OK && results[j.idx].status != KSC_OK) first = results[j.idx].status;
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
