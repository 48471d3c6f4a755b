// ksc_server.cu -- the serving loop: dual-bound requests for nodes of many
// problems, continuous batching on one GPU.
//
// A worker thread owns one batched session (ksc_session.h) per problem with
// pending work.  Each round it
//   1. takes the newly submitted requests,
//   2. opens sessions while the budget allows (problem bytes + session workspace),
//   3. admits pending nodes into free slots of their problem's session,
//   4. launches one graph replay (16 FISTA steps) on every session with running
//      nodes -- each session on its own stream, so the replays overlap on the
//      device -- and only then
//   5. collects each session: certificates, re-anchors, finished slots; results
//      go back to their requests and the slots are free for the next round,
//   6. closes sessions with nothing left to do, returning their budget.
// Problems whose X is not BF16 run one node at a time through ksc_solve_node.
#include <cuda_runtime.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "../../include/ksc.h"
#include "ksc_batch.cuh"
#include "ksc_problem.h"
#include "ksc_session.h"

using namespace ksc;

namespace {

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

struct Request {
  uint64_t ticket = 0;
  ksc_problem* pr = nullptr;
  ksc_node node{};
  std::vector<int32_t> zero, one;
  std::vector<double> warm;
  NodeSetup ns;
  bool batched = false;
  // result
  bool done = false;
  ksc_status status = KSC_OK;
  std::string err;
  ksc_result res{};
  std::vector<double> beta, z;
  double t_submit = 0.0, t_done = 0.0;
  bool counted_wait = false;
};

using ReqP = std::shared_ptr<Request>;

struct Sess {
  Session se;
  cudaStream_t s = nullptr;
  size_t bytes = 0;
  std::deque<ReqP> pending;
  std::vector<ReqP> slot_req;
};

}  // namespace

struct ksc_server {
  int device = 0;
  size_t budget = 0;
  int slots = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::thread worker;
  bool stop = false;
  uint64_t next_ticket = 1;
  std::deque<ReqP> incoming;
  std::unordered_map<uint64_t, ReqP> reqs;
  std::unordered_map<uint64_t, double> latency;
  int64_t stats[6] = {0, 0, 0, 0, 0, 0};
  // worker-only state
  std::map<ksc_problem*, Sess*> sessions;
  std::deque<ReqP> waiting;
  size_t used = 0;
};

namespace {

void complete(ksc_server* sv, const ReqP& r, ksc_status st, const std::string& err) {
  std::lock_guard<std::mutex> lk(sv->mu);
  r->status = st;
  r->err = err;
  r->done = true;
  r->t_done = now_s();
  sv->stats[0] += 1;
  sv->cv_done.notify_all();
}

void close_session(ksc_server* sv, ksc_problem* pr) {
  auto it = sv->sessions.find(pr);
  if (it == sv->sessions.end()) return;
  Sess* ss = it->second;
  session_close(&ss->se);
  if (ss->s) cudaStreamDestroy(ss->s);
  sv->used -= ss->bytes;
  delete ss;
  sv->sessions.erase(it);
}

void fail_session(ksc_server* sv, ksc_problem* pr, ksc_status st) {
  Sess* ss = sv->sessions[pr];
  const std::string msg = ksc_last_error();
  for (auto& r : ss->slot_req)
    if (r) complete(sv, r, st, msg);
  for (auto& r : ss->pending) complete(sv, r, st, msg);
  ss->pending.clear();
  close_session(sv, pr);
}

void run_single(ksc_server* sv, const ReqP& r, cudaStream_t s) {
  r->res.beta = r->beta.data();
  r->res.z = r->z.data();
  const ksc_status st = ksc_solve_node(r->pr, &r->node, &r->res, s);
  complete(sv, r, st, st == KSC_OK ? std::string() : std::string(ksc_last_error()));
}

void worker_loop(ksc_server* sv) {
  cudaSetDevice(sv->device);
  cudaStream_t single_stream = nullptr;
  cudaStreamCreateWithFlags(&single_stream, cudaStreamNonBlocking);
  for (;;) {
    std::deque<ReqP> fresh;
    {
      std::unique_lock<std::mutex> lk(sv->mu);
      bool busy = !sv->waiting.empty();
      for (auto& kv : sv->sessions) busy = busy || session_running(&kv.second->se) > 0 || !kv.second->pending.empty();
      if (!busy && sv->incoming.empty() && !sv->stop)
        sv->cv_work.wait_for(lk, std::chrono::milliseconds(50));
      if (sv->stop) break;
      fresh.swap(sv->incoming);
    }
    // 1. route new requests
    for (auto& r : fresh) {
      if (!r->batched) {
        run_single(sv, r, single_stream);
        continue;
      }
      auto it = sv->sessions.find(r->pr);
      if (it != sv->sessions.end()) it->second->pending.push_back(r);
      else sv->waiting.push_back(r);
    }
    // 2. open sessions while the budget allows (arrival order)
    for (auto it = sv->waiting.begin(); it != sv->waiting.end();) {
      ReqP r = *it;
      auto sit = sv->sessions.find(r->pr);
      if (sit != sv->sessions.end()) {
        sit->second->pending.push_back(r);
        it = sv->waiting.erase(it);
        continue;
      }
      const size_t need = ksc_problem_bytes(r->pr) + session_bytes(r->pr, sv->slots);
      if (need > sv->budget) {
        complete(sv, r, KSC_ERR_ADMISSION, "problem and session workspace exceed the server's HBM budget");
        it = sv->waiting.erase(it);
        continue;
      }
      if (sv->used + need > sv->budget) {
        if (!r->counted_wait) {
          r->counted_wait = true;
          std::lock_guard<std::mutex> lk(sv->mu);
          sv->stats[4] += 1;
        }
        ++it;
        continue;
      }
      Sess* ss = new Sess();
      cudaStreamCreateWithFlags(&ss->s, cudaStreamNonBlocking);
      ksc_status st = session_open(&ss->se, r->pr, sv->slots, false, ss->s);
      if (st != KSC_OK) {
        const std::string msg = ksc_last_error();
        session_close(&ss->se);
        cudaStreamDestroy(ss->s);
        delete ss;
        complete(sv, r, st, msg);
        it = sv->waiting.erase(it);
        continue;
      }
      ss->bytes = need;
      ss->slot_req.assign(sv->slots, nullptr);
      sv->used += need;
      sv->sessions[r->pr] = ss;
      {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stats[2] += 1;
        if ((int64_t)sv->used > sv->stats[3]) sv->stats[3] = (int64_t)sv->used;
      }
      ss->pending.push_back(r);
      it = sv->waiting.erase(it);
    }
    // 3. admit pending nodes into free slots
    std::vector<ksc_problem*> broken;
    for (auto& kv : sv->sessions) {
      Sess* ss = kv.second;
      const int k = std::min<int>(session_free_slots(&ss->se), (int)ss->pending.size());
      if (k <= 0) continue;
      const bool was_running = session_running(&ss->se) > 0;
      std::vector<const ksc_node*> nv;
      std::vector<const NodeSetup*> sv_ns;
      std::vector<int> wz, got;
      std::vector<ReqP> batch;
      for (int i = 0; i < k; ++i) {
        ReqP r = ss->pending.front();
        ss->pending.pop_front();
        nv.push_back(&r->node);
        sv_ns.push_back(&r->ns);
        wz.push_back(1);
        batch.push_back(r);
      }
      ksc_status st = session_admit(&ss->se, nv, sv_ns, wz, &got);
      if (st != KSC_OK) {
        const std::string msg = ksc_last_error();
        for (auto& r : batch) complete(sv, r, st, msg);
        broken.push_back(kv.first);
        continue;
      }
      for (int i = 0; i < k; ++i) ss->slot_req[got[i]] = batch[i];
      if (was_running) {
        std::lock_guard<std::mutex> lk(sv->mu);
        sv->stats[5] += k;
      }
    }
    for (auto* pr : broken) fail_session(sv, pr, KSC_ERR_CUDA);
    broken.clear();
    // 4. one replay per session with running nodes, all enqueued before any wait
    std::vector<ksc_problem*> advanced;
    for (auto& kv : sv->sessions) {
      ksc_status st;
      if (session_advance(&kv.second->se, &st)) advanced.push_back(kv.first);
      else if (st != KSC_OK) broken.push_back(kv.first);
    }
    if (!advanced.empty()) {
      std::lock_guard<std::mutex> lk(sv->mu);
      sv->stats[1] += (int64_t)advanced.size();
    }
    // 5. collect
    for (auto* pr : advanced) {
      Sess* ss = sv->sessions[pr];
      std::vector<int> fin;
      ksc_status st = session_collect(&ss->se, &fin);
      if (st != KSC_OK) {
        broken.push_back(pr);
        continue;
      }
      for (int b : fin) {
        ReqP r = ss->slot_req[b];
        ss->slot_req[b] = nullptr;
        if (!r) continue;
        r->res.beta = r->beta.data();
        r->res.z = r->z.data();
        st = session_fetch(&ss->se, b, &r->res);
        complete(sv, r, st == KSC_OK ? r->res.status : st,
                 st == KSC_OK ? std::string() : std::string(ksc_last_error()));
      }
    }
    for (auto* pr : broken) fail_session(sv, pr, KSC_ERR_CUDA);
    // 6. close idle sessions
    std::vector<ksc_problem*> idle;
    for (auto& kv : sv->sessions)
      if (session_running(&kv.second->se) == 0 && kv.second->pending.empty()) idle.push_back(kv.first);
    for (auto* pr : idle) close_session(sv, pr);
  }
  // shutdown: unfinished requests end with a timeout status
  std::vector<ksc_problem*> all;
  for (auto& kv : sv->sessions) all.push_back(kv.first);
  for (auto* pr : all) {
    Sess* ss = sv->sessions[pr];
    for (auto& r : ss->slot_req)
      if (r) complete(sv, r, KSC_ERR_TIMEOUT, "server destroyed before the request finished");
    for (auto& r : ss->pending) complete(sv, r, KSC_ERR_TIMEOUT, "server destroyed before the request finished");
    ss->pending.clear();
    close_session(sv, pr);
  }
  for (auto& r : sv->waiting) complete(sv, r, KSC_ERR_TIMEOUT, "server destroyed before the request finished");
  sv->waiting.clear();
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    for (auto& r : sv->incoming) {
      r->status = KSC_ERR_TIMEOUT;
      r->err = "server destroyed before the request finished";
      r->done = true;
    }
    sv->incoming.clear();
    sv->cv_done.notify_all();
  }
  if (single_stream) cudaStreamDestroy(single_stream);
}

}  // namespace

extern "C" ksc_status ksc_server_create(size_t hbm_budget_bytes, int32_t max_slots, ksc_server** out) {
  if (!out) return api_fail(KSC_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (max_slots < 1 || max_slots > kBatchMax) return api_fail(KSC_ERR_INVALID_ARG, "max_slots must be in 1..1024");
  if (hbm_budget_bytes == 0) return api_fail(KSC_ERR_INVALID_ARG, "hbm_budget_bytes must be > 0");
  ksc_status st = ensure_prepared();
  if (st != KSC_OK) return st;
  ksc_server* sv = new ksc_server();
  cudaGetDevice(&sv->device);
  sv->budget = hbm_budget_bytes;
  sv->slots = max_slots;
  sv->worker = std::thread(worker_loop, sv);
  *out = sv;
  return KSC_OK;
}

extern "C" ksc_status ksc_server_submit(ksc_server* sv, ksc_problem* pr, const ksc_node* node, uint64_t* ticket) {
  if (!sv || !pr || !node || !ticket) return api_fail(KSC_ERR_INVALID_ARG, "NULL argument");
  auto r = std::make_shared<Request>();
  r->pr = pr;
  r->node = *node;
  if (node->n_zero > 0 && node->fixed_zero) r->zero.assign(node->fixed_zero, node->fixed_zero + node->n_zero);
  if (node->n_one > 0 && node->fixed_one) r->one.assign(node->fixed_one, node->fixed_one + node->n_one);
  if (node->warm_beta) r->warm.assign(node->warm_beta, node->warm_beta + pr->p);
  r->node.fixed_zero = r->zero.empty() ? nullptr : r->zero.data();
  r->node.fixed_one = r->one.empty() ? nullptr : r->one.data();
  r->node.warm_beta = r->warm.empty() ? nullptr : r->warm.data();
  ksc_status st = check_node(pr, &r->node, &r->ns);
  if (st != KSC_OK) return st;
  r->beta.assign(pr->p, 0.0);
  r->z.assign(pr->p, 0.0);
  r->batched = pr->xdt == kXBF16 && !r->ns.infeasible && std::min<int64_t>(r->ns.kp, pr->p) < kBatchCap;
  r->t_submit = now_s();
  std::lock_guard<std::mutex> lk(sv->mu);
  r->ticket = sv->next_ticket++;
  *ticket = r->ticket;
  sv->reqs[r->ticket] = r;
  if (r->ns.infeasible) {
    r->res.primal = INFINITY;
    r->res.dual_bound = INFINITY;
    r->res.rel_gap = 0.0;
    r->res.pruned = 1;
    r->res.status = KSC_ERR_INFEASIBLE_NODE;
    r->status = KSC_ERR_INFEASIBLE_NODE;
    r->done = true;
    r->t_done = r->t_submit;
    sv->stats[0] += 1;
    return KSC_OK;
  }
  sv->incoming.push_back(r);
  sv->cv_work.notify_one();
  return KSC_OK;
}

extern "C" ksc_status ksc_server_poll(ksc_server* sv, uint64_t ticket, ksc_result* result, int32_t timeout_ms) {
  if (!sv || !result) return api_fail(KSC_ERR_INVALID_ARG, "NULL argument");
  std::unique_lock<std::mutex> lk(sv->mu);
  auto it = sv->reqs.find(ticket);
  if (it == sv->reqs.end()) return api_fail(KSC_ERR_INVALID_ARG, "unknown or released ticket");
  ReqP r = it->second;
  auto ready = [&] { return r->done; };
  if (timeout_ms < 0) sv->cv_done.wait(lk, ready);
  else if (!sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready))
    return api_fail(KSC_ERR_TIMEOUT, "request not finished within the timeout");
  double* ub = result->beta;
  double* uz = result->z;
  *result = r->res;
  result->beta = ub;
  result->z = uz;
  const int64_t p = r->pr->p;
  const bool has_vectors = r->status == KSC_OK || r->status == KSC_NOT_CONVERGED;
  if (ub && has_vectors) std::copy(r->beta.begin(), r->beta.begin() + p, ub);
  if (uz && has_vectors) std::copy(r->z.begin(), r->z.begin() + p, uz);
  if (!has_vectors) result->status = r->status;
  sv->latency[ticket] = r->t_done - r->t_submit;
  sv->reqs.erase(it);
  const ksc_status st = r->status;
  const std::string err = r->err;
  lk.unlock();
  if (st != KSC_OK) return api_fail(st, err.empty() ? std::string("request ended with a non-OK status") : err);
  return KSC_OK;
}

extern "C" ksc_status ksc_server_latency(ksc_server* sv, uint64_t ticket, double* seconds) {
  if (!sv || !seconds) return api_fail(KSC_ERR_INVALID_ARG, "NULL argument");
  std::lock_guard<std::mutex> lk(sv->mu);
  auto it = sv->latency.find(ticket);
  if (it == sv->latency.end()) return api_fail(KSC_ERR_INVALID_ARG, "ticket not polled yet");
  *seconds = it->second;
  return KSC_OK;
}

extern "C" ksc_status ksc_server_stats(ksc_server* sv, int64_t* stats, int32_t n) {
  if (!sv || (n > 0 && !stats) || n < 0) return api_fail(KSC_ERR_INVALID_ARG, "bad arguments");
  std::lock_guard<std::mutex> lk(sv->mu);
  for (int32_t i = 0; i < n; ++i) stats[i] = i < 6 ? sv->stats[i] : 0;
  return KSC_OK;
}

extern "C" ksc_status ksc_server_destroy(ksc_server* sv) {
  if (!sv) return KSC_OK;
  {
    std::lock_guard<std::mutex> lk(sv->mu);
    sv->stop = true;
    sv->cv_work.notify_all();
  }
  if (sv->worker.joinable()) sv->worker.join();
  delete sv;
  return KSC_OK;
}
