// ksc_problem.h -- the library's view of a problem handle, shared by the C-ABI
// translation units (single-node loop in ksc_api.cu, batched loop in
// ksc_batch.cu).
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/ksc.h"
#include "ksc_launch.h"
#include "ksc_state.cuh"

namespace ksc {
struct BatchWs;
void free_batch(BatchWs* ws);
}  // namespace ksc

static constexpr int kStepsPerGraph = 16;
static constexpr int kEigMaxP = 8192;   // largest p of the eigen shift's Cholesky test
static constexpr int kKernelIds = 12;   // KSC_KERNEL_* ids of ksc_problem_kernel_time
static constexpr int kEventsPerStep = 5;  // profiling events around the kernels of one FISTA step

struct ksc_problem {
  int device = 0;
  int64_t n = 0, p = 0, ldx = 0;
  int xdt = 0;
  int loss = 0;
  bool own_x = false;
  void* X = nullptr;
  double* y = nullptr;
  std::vector<double> y_host;
  double L = 0.0;
  int power_iters = 0;
  size_t bytes = 0;
  ksc::Dev dev{};
  std::vector<void*> allocs;
  cudaGraphExec_t graph = nullptr;
  cudaGraphExec_t graph_prof = nullptr;
  cudaGraphExec_t graph_eig = nullptr;        // the eigen-perspective step
  cudaGraphExec_t graph_eig_prof = nullptr;
  bool profile = false;
  std::vector<cudaEvent_t> events;   // 4 per step of the profiling graph
  int64_t k_launches[kKernelIds] = {};
  double k_ms[kKernelIds] = {};
  int64_t launches = 0;   // every kernel launch issued for this problem
  int32_t last_stats[12] = {0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0, 0};
  ksc::BatchWs* batch = nullptr;   // batched-solve workspace (created on first use)
  std::vector<double> batch_state; // 10 in-loop values per node of the last batched call
  double eig_lambda = 0.0;         // certified lower bound on lambda_min(X^T X)
  bool eig_ready = false;          // eig_lambda computed (ksc_problem_eig_lambda)
  // Poisson and Gamma regression: L above is lambda_max(X^T X) * 1.01 (or the
  // caller's constant, l_fixed); each node multiplies it by its curvature bound
  // from the rows' largest entries and absolute sums
  bool l_fixed = false;
  std::vector<double> row_max, row_l1;
};

namespace ksc {

// a node's coordinate states and reduced budget, validated
struct NodeSetup {
  std::vector<int8_t> state;
  int kp = 0;
  int n_one = 0;
  bool infeasible = false;
};

ksc_status check_node(const ksc_problem* pr, const ksc_node* node, NodeSetup* ns);
// the step constant L of Algorithm 3 for a node (the problem's L, or for Poisson /
// Gamma regression that L times max_i c_i, c_i = e^{3 U_i} or y_i e^{3 U_i},
// U_i = M min(k max_j |x_ij|, sum_j |x_ij|))
double node_lipschitz(const ksc_problem* pr, double M, int k);
// warm start of a node in place: S0 coordinates 0, every coordinate clipped to the
// box, and for Poisson / Gamma regression scaled into sum |b_j| <= k M
void project_warm(const ksc_problem* pr, const NodeSetup& ns, double M, int k, double* b);
bool loss_counts(int loss);
ksc_status ensure_prepared();
ksc_status api_fail(ksc_status st, const std::string& msg);

}  // namespace ksc
