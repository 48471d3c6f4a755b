// ksc_bnb.cu -- ksc_bnb_solve: a minimal best-first branch and bound for Eq. (1)
// around the batched node solver (Sec. 5.3, App. B.3).
//
// The node relaxations run in one batched session with continuous batching: the
// host keeps a best-bound-first queue of open nodes and, after every graph replay,
// certifies and collects the finished ones, decides prune / close / branch, and
// refills the free slots at once -- children of a node start one replay after it
// finishes, beside nodes that are still iterating.  Incumbent searches (the
// restricted problem on a node's leading support) share the same slots.
// Host code only: every arithmetic step of a solve runs in the session kernels.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstring>
#include <queue>
#include <string>
#include <vector>

#include "../../include/ksc.h"
#include "ksc_batch.cuh"
#include "ksc_problem.h"
#include "ksc_session.h"

namespace ksc {
namespace {

struct OpenNode {
  std::vector<int32_t> zero, one;   // S0, S1 (sorted)
  double bound;                     // certified bound of the parent (a valid lower bound here)
  std::vector<int32_t> wi;          // warm start: the parent's nonzeros
  std::vector<double> wv;
  bool plain = false;               // solve without the incumbent rules (a resumed node)
};

struct ByBound {
  bool operator()(const OpenNode* a, const OpenNode* b) const { return a->bound > b->bound; }
};

struct Job {
  bool busy = false;
  bool heuristic = false;
  OpenNode* node = nullptr;         // the node a relaxation slot solves (owned)
  double bound = -INFINITY;         // lower bound that holds while it runs
};

double elapsed(std::chrono::steady_clock::time_point t0) {
  return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
}

}  // namespace
}  // namespace ksc

extern "C" ksc_status ksc_bnb_solve(ksc_problem* pr, const ksc_bnb_params* prm, ksc_bnb_result* res,
                                    void* cuda_stream) {
  using namespace ksc;
  if (!pr || !prm || !res) return api_fail(KSC_ERR_INVALID_ARG, "problem, params and result must be non-NULL");
  if (!(prm->lambda2 > 0) || !std::isfinite(prm->lambda2)) return api_fail(KSC_ERR_INVALID_ARG, "lambda2 must be > 0");
  if (!(prm->M > 0) || !std::isfinite(prm->M)) return api_fail(KSC_ERR_INVALID_ARG, "M must be > 0");
  if (prm->k < 1) return api_fail(KSC_ERR_INVALID_ARG, "k must be >= 1");
  if (prm->k >= kBatchCap) return api_fail(KSC_ERR_UNIMPLEMENTED, "k must be below 2048");
  if (prm->batch < 1 || prm->batch > kBatchMax) return api_fail(KSC_ERR_INVALID_ARG, "batch must be in [1, 1024]");
  if (!(prm->opt_gap >= 0) || !(prm->node_rel_gap > 0) || prm->node_max_iter < 1 || prm->max_nodes < 0 ||
      !(prm->time_limit_s >= 0))
    return api_fail(KSC_ERR_INVALID_ARG, "opt_gap >= 0, node_rel_gap > 0, node_max_iter >= 1, limits >= 0");
  if (pr->xdt != kXBF16 && pr->xdt != kXFP8)
    return api_fail(KSC_ERR_UNIMPLEMENTED, "branch and bound needs BF16 or FP8 X (batched solver)");
  if (pr->xdt == kXFP8 && (prm->node_flags & KSC_FLAG_EIG))
    return api_fail(KSC_ERR_UNIMPLEMENTED, "the eigen-perspective relaxation runs on BF16 X");
  ksc_status st = ensure_prepared();
  if (st != KSC_OK) return st;
  int cur_dev = 0;
  cudaGetDevice(&cur_dev);
  if (cur_dev != pr->device && cudaSetDevice(pr->device) != cudaSuccess)
    return api_fail(KSC_ERR_CUDA, "cannot select the problem's device");
  const auto t0 = std::chrono::steady_clock::now();
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (prm->node_flags & KSC_FLAG_EIG) {   // the eigen shift, computed on first use
    if (pr->loss != KSC_LOSS_LSQ) return api_fail(KSC_ERR_INVALID_ARG, "the eigen-perspective relaxation is for least squares");
    double lam = 0.0;
    if ((st = ksc_problem_eig_lambda(pr, cuda_stream, &lam)) != KSC_OK) return st;
  }
  const int p = (int)pr->p;
  const int k = prm->k;

  // column norms for the branching score (second-order loss increase of b_j -> 0)
  std::vector<double> cn(p);
  if (cudaMemcpy(cn.data(), pr->dev.colnorm, (size_t)p * 8, cudaMemcpyDeviceToHost) != cudaSuccess)
    return api_fail(KSC_ERR_CUDA, "column norms");
  const double curv = pr->loss == KSC_LOSS_LOGISTIC ? 0.25 : 1.0;

  Session se;
  if ((st = session_open(&se, pr, prm->batch, true, s)) != KSC_OK) return st;
  std::vector<Job> job(prm->batch);
  std::priority_queue<OpenNode*, std::vector<OpenNode*>, ByBound> open;
  std::vector<OpenNode*> heur;     // pending incumbent searches (S1 = support)
  auto free_all = [&]() {
    while (!open.empty()) { delete open.top(); open.pop(); }
    for (OpenNode* h : heur) delete h;
    heur.clear();
    for (Job& j : job) { delete j.node; j.node = nullptr; }
    session_close(&se);
  };

  double inc = INFINITY;
  std::vector<double> inc_beta(p, 0.0), beta(p);
  int64_t nodes = 0, pruned = 0, closed = 0, heuristics = 0, replays = 0, max_open = 0;
  open.push(new OpenNode{{}, {}, -INFINITY, {}, {}});
  const double tiny = 1e-300;
  auto prunable = [&](double bound) { return std::isfinite(inc) && inc - bound <= prm->opt_gap * std::fabs(inc); };
  // the smallest certified bound of the leaves taken off the tree (pruned within the
  // gap, or closed): a leaf pruned within opt_gap may hold points below the
  // incumbent, down to its bound, so the tree's lower bound keeps it
  double done_lb = INFINITY;
  auto lower_bound = [&]() {
    double lb = open.empty() ? INFINITY : open.top()->bound;
    for (const Job& j : job)
      if (j.busy && !j.heuristic) lb = std::min(lb, j.bound);
    return std::min(std::min(lb, done_lb), inc);
  };
  bool certified = false;

  for (;;) {
    // ---- refill free slots: incumbent searches first, then the best open nodes
    std::vector<ksc_node> kn;
    std::vector<NodeSetup> setup;
    std::vector<std::pair<bool, OpenNode*>> who;
    std::vector<std::vector<double>> warms;
    const int nfree = session_free_slots(&se);
    const bool budget_left = prm->max_nodes == 0 || nodes < prm->max_nodes;
    const bool time_left = prm->time_limit_s == 0 || elapsed(t0) < prm->time_limit_s;
    while ((int)who.size() < nfree && time_left) {
      OpenNode* on = nullptr;
      bool h = false;
      if (!heur.empty()) {
        on = heur.back();
        heur.pop_back();
        h = true;
      } else if (!open.empty() && budget_left) {
        on = open.top();
        open.pop();
        if (prunable(on->bound)) {
          ++pruned;
          done_lb = std::min(done_lb, on->bound);
          delete on;
          continue;
        }
      } else {
        break;
      }
      who.push_back({h, on});
    }
    kn.resize(who.size());
    setup.resize(who.size());
    warms.resize(who.size());
    for (size_t i = 0; i < who.size(); ++i) {
      OpenNode* on = who[i].second;
      warms[i].assign(p, 0.0);
      for (size_t t = 0; t < on->wi.size(); ++t) warms[i][on->wi[t]] = on->wv[t];
      ksc_node& nd = kn[i];
      std::memset(&nd, 0, sizeof nd);
      nd.lambda2 = prm->lambda2;
      nd.M = prm->M;
      nd.k = who[i].first ? (int32_t)on->one.size() : k;
      nd.fixed_zero = on->zero.empty() ? nullptr : on->zero.data();
      nd.n_zero = (int32_t)on->zero.size();
      nd.fixed_one = on->one.empty() ? nullptr : on->one.data();
      nd.n_one = (int32_t)on->one.size();
      nd.warm_beta = warms[i].data();
      nd.incumbent = (who[i].first || on->plain) ? INFINITY : inc;
      nd.rel_gap_tol = prm->node_rel_gap;
      nd.max_iter = prm->node_max_iter;
      nd.flags = prm->node_flags;
      if ((st = check_node(pr, &nd, &setup[i])) != KSC_OK) { free_all(); return st; }
    }
    if (!who.empty()) {
      std::vector<const ksc_node*> nv;
      std::vector<const NodeSetup*> sv;
      std::vector<int> wz(who.size(), 0), slots;
      for (size_t i = 0; i < who.size(); ++i) { nv.push_back(&kn[i]); sv.push_back(&setup[i]); }
      if ((st = session_admit(&se, nv, sv, wz, &slots)) != KSC_OK) { free_all(); return st; }
      for (size_t i = 0; i < who.size(); ++i) {
        Job& j = job[slots[i]];
        j.busy = true;
        j.heuristic = who[i].first;
        j.node = who[i].second;
        j.bound = who[i].second->bound;
      }
    }
    max_open = std::max<int64_t>(max_open, (int64_t)open.size());
    // ---- stop?
    const double lb = lower_bound();
    if (std::isfinite(inc) && inc - lb <= prm->opt_gap * std::max(std::fabs(inc), tiny) && heur.empty()) {
      certified = true;
      break;
    }
    if (session_running(&se) == 0) {
      if (open.empty() && heur.empty()) { certified = std::isfinite(inc); break; }
      if (!budget_left || !time_left) break;
      continue;   // admitted nothing new but nodes remain (they were pruned above)
    }
    // ---- one replay, then the finished nodes
    if (!session_advance(&se, &st)) {
      if (st != KSC_OK) { free_all(); return st; }
    } else {
      ++replays;
    }
    std::vector<int> fin;
    if ((st = session_collect(&se, &fin)) != KSC_OK) { free_all(); return st; }
    for (int b : fin) {
      ksc_result r;
      std::memset(&r, 0, sizeof r);
      r.beta = beta.data();
      if ((st = session_fetch(&se, b, &r)) != KSC_OK) { free_all(); return st; }
      Job& j = job[b];
      OpenNode* on = j.node;
      j.node = nullptr;
      j.busy = false;
      if (j.heuristic) {
        ++heuristics;
        if (std::isfinite(r.primal) && r.primal < inc) { inc = r.primal; inc_beta = beta; }
        delete on;
        continue;
      }
      ++nodes;
      const double bound = std::max(r.dual_bound, on->bound);   // both are valid lower bounds
      if (r.status == KSC_ERR_INFEASIBLE_NODE || r.pruned || prunable(bound)) {
        ++pruned;
        if (r.status != KSC_ERR_INFEASIBLE_NODE) done_lb = std::min(done_lb, bound);
        delete on;
        continue;
      }
      // free coordinates of the relaxed solution, largest |b_j| first
      std::vector<char> fixed(p, 0);
      for (int32_t z : on->zero) fixed[z] = 1;
      for (int32_t o : on->one) fixed[o] = 2;
      std::vector<int32_t> nzf;
      for (int jj = 0; jj < p; ++jj)
        if (!fixed[jj] && beta[jj] != 0.0) nzf.push_back(jj);
      const int kp = k - (int)on->one.size();
      // a relaxed solution with at most k' free nonzeros is feasible for Eq. (1):
      // its certified primal is an incumbent; the node is solved when certified,
      // otherwise (stopped early by the incumbent rule) it resumes without the rules
      if ((int)nzf.size() <= kp) {
        if (std::isfinite(r.primal) && r.primal < inc) { inc = r.primal; inc_beta = beta; }
        if (r.status == KSC_OK && r.rel_gap <= prm->node_rel_gap) {
          ++closed;
          done_lb = std::min(done_lb, bound);
          delete on;
        } else if (on->plain) {
          ++closed;   // solved without the rules and still not certified (iteration cap): its point is the incumbent candidate
          done_lb = std::min(done_lb, bound);
          delete on;
        } else {
          on->bound = bound;
          on->plain = true;
          on->wi.clear();
          on->wv.clear();
          for (int jj = 0; jj < p; ++jj)
            if (beta[jj] != 0.0) { on->wi.push_back(jj); on->wv.push_back(beta[jj]); }
          open.push(on);
        }
        continue;
      }
      std::sort(nzf.begin(), nzf.end(), [&](int32_t a, int32_t c) {
        const double fa = std::fabs(beta[a]), fc = std::fabs(beta[c]);
        return fa != fc ? fa > fc : a < c;
      });
      const int take = std::min<int>(std::max(kp, 0), (int)nzf.size());
      // incumbent search on S1 + the k' leading free coordinates
      OpenNode* h = new OpenNode{{}, on->one, -INFINITY, {}, {}};
      for (int t = 0; t < take; ++t) h->one.push_back(nzf[t]);
      std::sort(h->one.begin(), h->one.end());
      for (int32_t jj : h->one) { h->wi.push_back(jj); h->wv.push_back(beta[jj]); }
      if (!h->one.empty()) heur.push_back(h);
      else delete h;
      // branch on the leading free coordinate with the largest second-order loss
      // increase of setting it to zero
      int bj = -1;
      double best = -1.0;
      for (int t = 0; t < std::max(take, std::min<int>(1, (int)nzf.size())); ++t) {
        const int32_t jj = nzf[t];
        const double sc = beta[jj] * beta[jj] * (curv * cn[jj] * cn[jj] + prm->lambda2);
        if (sc > best) { best = sc; bj = jj; }
      }
      if (bj < 0) { delete on; continue; }   // unreachable: nzf has more than k' >= 0 entries
      std::vector<int32_t> wi;
      std::vector<double> wv;
      for (int jj = 0; jj < p; ++jj)
        if (beta[jj] != 0.0) { wi.push_back(jj); wv.push_back(beta[jj]); }
      OpenNode* a = new OpenNode{on->zero, on->one, bound, {}, {}};   // z_j = 0
      a->zero.insert(std::upper_bound(a->zero.begin(), a->zero.end(), bj), bj);
      for (size_t t = 0; t < wi.size(); ++t)
        if (wi[t] != bj) { a->wi.push_back(wi[t]); a->wv.push_back(wv[t]); }
      open.push(a);
      if ((int)on->one.size() + 1 <= k) {                             // z_j = 1
        OpenNode* c = new OpenNode{on->zero, on->one, bound, wi, wv};
        c->one.insert(std::upper_bound(c->one.begin(), c->one.end(), bj), bj);
        open.push(c);
      }
      delete on;
    }
  }
  const double lb = lower_bound();
  res->incumbent = inc;
  res->lower_bound = lb;
  res->gap = std::isfinite(inc) ? (inc - lb) / std::max(std::fabs(inc), tiny) : INFINITY;
  res->nodes = nodes;
  res->pruned = pruned;
  res->closed = closed;
  res->heuristic_solves = heuristics;
  res->replays = replays;
  res->max_open = max_open;
  res->certified = certified ? 1 : 0;
  if (res->beta) std::memcpy(res->beta, inc_beta.data(), (size_t)p * 8);
  free_all();
  res->seconds = elapsed(t0);
  return KSC_OK;
}
