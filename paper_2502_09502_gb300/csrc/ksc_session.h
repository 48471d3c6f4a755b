// ksc_session.h -- a batched-solve session: a fixed set of node slots of one
// problem that advance together (k_batch.cu, k_tcgemm.cu).  Slots are filled and
// emptied between graph replays, so one session serves both ksc_solve_batch (all
// slots filled once) and the server's continuous batching (slots refilled as
// nodes finish).
#pragma once

#include <cuda_runtime.h>

#include <vector>

#include "../../include/ksc.h"
#include "ksc_problem.h"

namespace ksc {

struct BatchWs;

struct SlotHost {
  bool busy = false;       // holds a node (running, or finished and not yet fetched)
  bool fin = false;        // finished: certificate final
  int want_z = 0;
  double tol = 0.0, inc = 0.0;
  double anchor_gap = 0.0; // re-anchor when the in-loop gap falls below this
  int last_anchor = 0;     // iteration of the last anchor
  int last_cert = 0;       // iteration of the last certificate
  int anchors = 0;
  int pruned = 0;
  ksc_status status = KSC_OK;
};

struct Session {
  ksc_problem* pr = nullptr;
  BatchWs* ws = nullptr;
  bool own_ws = false;     // a server session owns its workspace; ksc_solve_batch borrows the problem's
  cudaStream_t s = nullptr;
  int B = 0;
  std::vector<SlotHost> slot;
  std::vector<char> hn_raw;    // host mirror of the BNode array
  std::vector<char> hc_raw;    // host mirror of the BCert array
  int64_t anchors = 0;         // anchor products issued (statistics)
  int64_t certificates = 0;
  std::vector<int> tile_flags; // staging of the per-tile running flags
  size_t bytes() const;
};

// slots: nodes advanced together (<= kBatchMax).  use_problem_ws: borrow (and
// grow) the problem's cached workspace instead of owning one.
ksc_status session_open(Session* se, ksc_problem* pr, int slots, bool use_problem_ws, cudaStream_t s);
void session_close(Session* se);
// workspace bytes a session of `slots` slots allocates for problem pr
size_t session_bytes(const ksc_problem* pr, int slots);
// fill free slots with validated nodes (ns: from check_node, feasible);
// slot ids are returned in *slots
ksc_status session_admit(Session* se, const std::vector<const ksc_node*>& nodes,
                         const std::vector<const NodeSetup*>& ns, const std::vector<int>& want_z,
                         std::vector<int>* slots);
// enqueue one graph replay (16 steps) if any slot is running; returns whether it did
bool session_advance(Session* se, ksc_status* st);
// wait for the replay, certify the nodes whose in-loop test fired, re-anchor
// converging nodes; slots that finished are appended to *finished
ksc_status session_collect(Session* se, std::vector<int>* finished);
// result of a finished slot (beta and z copied to the result's arrays when
// non-NULL); frees the slot
ksc_status session_fetch(Session* se, int slot, ksc_result* r);
int session_free_slots(const Session* se);
int session_running(const Session* se);

}  // namespace ksc
