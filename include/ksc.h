/*
 * ksc.h -- C ABI of the GB300 (sm_103a) library that computes certified dual
 * bounds for the perspective relaxation of the k-sparse, box-constrained,
 * ridge-regularised GLM (Liu et al., "Scalable First-order Method for
 * Certifying Optimal k-Sparse GLMs", arXiv 2502.09502).
 *
 * The problem (Sec. 1, Eq. (1)):
 *     min_b  F(X b) + lambda2 ||b||^2   s.t.  ||b||_inf <= M,  ||b||_0 <= k,
 * with F the least-squares loss ||u - y||^2 or the logistic loss
 * sum_i log(1 + exp(-y_i u_i)), y_i in {-1, +1} (App. D.1).  A branch-and-bound
 * node fixes some z_j to 0 (S0: b_j = 0) and some to 1 (S1: b_j free in the box,
 * outside the cardinality budget), leaving k' = k - |S1| (App. B.3).
 *
 * The library solves the node's perspective relaxation P_conv (Sec. 2, Eq. (4))
 * in the composite form min_b F(X b) + 2 lambda2 g(b) (Sec. 3, Eq. (5)-(6)) by
 * restarted FISTA (Algorithm 3) with the exact prox of g (Algorithm 1 + 4 via
 * the Moreau identity of Sec. 3.3; g itself by Algorithm 2), and certifies the
 * weak-duality bound  D = -F*(-zeta) - G*(X^T zeta),  zeta = -grad F(X b^),
 * G = 2 lambda2 g, G* from Lemma 3.1 (Sec. 3.4).  The certificate is evaluated
 * in FP64 with a rigorous rounding-error margin subtracted, so D never exceeds
 * P_conv(node) <= P_MIP(node) because of rounding.
 *
 * Conventions for every call:
 *   - Return value: a ksc_status; no C++ exception crosses the ABI.  On an error
 *     the message is available from ksc_last_error() (thread-local).
 *   - Ownership: the caller owns every host array and result buffer it passes;
 *     the library owns the device copies, workspaces and resident iterates it
 *     allocates, and frees them in the matching destroy call.
 *   - Layout: X is row-major n x p with leading dimension ldx >= p (elements);
 *     vectors are dense, 0-based, in the original coordinate order.
 *   - Streams: `cuda_stream` is a cudaStream_t passed as void* (NULL = the
 *     legacy default stream); all device work of a call is ordered on it.
 *     Calls are blocking: they return once results are in host memory.
 *   - Devices: all device work runs on the device that is current when the
 *     problem (or server) is created.
 */
#ifndef KSC_H
#define KSC_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  KSC_OK = 0,
  KSC_ERR_INVALID_ARG = 1,      /* a null pointer, size or parameter out of range   */
  KSC_ERR_OOM = 2,              /* a device allocation failed                       */
  KSC_ERR_ADMISSION = 3,        /* a request does not fit the server's HBM budget   */
  KSC_ERR_INFEASIBLE_NODE = 4,  /* |S1| > k or S0 and S1 intersect                  */
  KSC_NOT_CONVERGED = 5,        /* max_iter reached; dual_bound is still certified  */
  KSC_ERR_TIMEOUT = 6,          /* a bounded wait expired (device or host side)     */
  KSC_ERR_CUDA = 7,             /* a CUDA runtime error; see ksc_last_error()       */
  KSC_ERR_UNIMPLEMENTED = 8     /* the requested combination is not built           */
} ksc_status;

typedef enum {
  KSC_LOSS_LSQ = 0,             /* F(u) = ||u - y||^2                     (App. D.1) */
  KSC_LOSS_LOGISTIC = 1,        /* F(u) = sum log(1 + exp(-y_i u_i)), y = +-1        */
  KSC_LOSS_SQHINGE = 2,         /* F(u) = sum max(0, 1 - y_i u_i)^2, y = +-1         */
  KSC_LOSS_POISSON = 3,         /* F(u) = sum e^{u_i} - y_i u_i, y >= 0 (App. D.1)  */
  KSC_LOSS_GAMMA = 4            /* F(u) = sum y_i e^{-u_i} + u_i, y > 0 (App. D.1)  */
} ksc_loss;

typedef enum {
  KSC_F64 = 0,                  /* X in double                                      */
  KSC_F32 = 1,                  /* X in float                                       */
  KSC_BF16 = 2,                 /* X in bfloat16 bits; the problem is the stored X  */
  KSC_FP8_E4M3_COLSCALE = 3     /* X in FP8 e4m3 bits with a per-column scale s_j, a
                                   power of two in [2^-100, 2^100]; the problem's matrix
                                   is X_ij * s_j, exact in FP32 (single-node and
                                   batched solvers, branch and bound)                */
  /* X is streamed from HBM in its storage type.  The iterate vectors (beta, X beta,
     the gradient) are FP64 for every type; products with FP32/BF16 X are made
     error-free (exact product error by fma, compensated sums). */
} ksc_dtype;

/* Node flags (ksc_node.flags): the ablations of Fig. 3. */
#define KSC_FLAG_RESTART_OFF  0x1u   /* plain FISTA: never reset the momentum       */
#define KSC_FLAG_MOMENTUM_OFF 0x2u   /* proximal gradient (ISTA): no momentum       */
#define KSC_FLAG_EIG          0x4u   /* eigen-perspective relaxation (App. D.2), least
                                        squares only: Q = X^T X - lambda I and lambda2 +
                                        lambda on the perspective term, lambda the
                                        problem's certified shift (ksc_problem_eig_lambda,
                                        computed on first use by ksc_solve_node,
                                        ksc_solve_batch and ksc_bnb_solve;
                                        ksc_server_submit refuses such a node with
                                        KSC_ERR_INVALID_ARG until it is known).  Both
                                        the single-node path (every storage type) and
                                        the batched path (BF16 X) run it             */

typedef struct ksc_problem ksc_problem;
typedef struct ksc_server ksc_server;

/* Problem data (Sec. 1): X (n x p, row-major), y (n), loss. */
typedef struct {
  int64_t n, p;
  ksc_dtype x_dtype;
  const void* X;        /* x_on_device = 0: host pointer, copied to the device.
                           x_on_device = 1: device pointer, BORROWED -- it must stay
                           valid and unchanged until ksc_problem_destroy.          */
  int64_t ldx;          /* leading dimension in elements, >= p; 0 means p         */
  const double* y;      /* host pointer, length n, always copied; logistic and
                           squared hinge: +-1; Poisson: >= 0; Gamma: > 0          */
  ksc_loss loss;
  int32_t x_on_device;
  double lipschitz;     /* > 0: the step constant L of Algorithm 3 to use.
                           <= 0: L = c_f * theta * 1.01, c_f = 2 (least squares,
                           squared hinge) or 1/4 (logistic), theta the largest Ritz
                           value of Lanczos on X^T X, checked every 8 steps and
                           stopped when the geometric extrapolation of its remaining
                           rise from the last three checks (Aitken) is at most 1e-3
                           of it, or a check moves it by at most 1e-5.  theta is a lower
                           estimate of lambda_max, so L is an estimate, not a proven
                           upper bound; L only changes the iteration's path, every
                           reported bound is valid for any L.  Poisson and Gamma:
                           their curvature is unbounded, so each node's L is
                           theta * 1.01 * max_i c_i, c_i = e^{3 U_i} (Poisson) or
                           y_i e^{3 U_i} (Gamma), U_i = M min(k max_j |x_ij|,
                           sum_j |x_ij|) -- the curvature over every point the
                           iteration evaluates (its iterates satisfy |b_j| <= M,
                           sum |b_j| <= kM; warm starts are scaled into that set);
                           a caller's L > 0 is used for every node as given     */
  const float* col_scale; /* KSC_FP8_E4M3_COLSCALE: host pointer, p scales (copied);
                           NULL for the other types                                */
} ksc_problem_desc;

/* Create a problem: copies (or borrows) X, copies y, computes L on the device.
 * Errors: KSC_ERR_INVALID_ARG (null pointers, n or p < 1, ldx < p, unknown enum,
 * logistic labels not +-1, FP8 X without power-of-two column scales),
 * KSC_ERR_OOM, KSC_ERR_CUDA.  *out is NULL on error. */
ksc_status ksc_problem_create(const ksc_problem_desc* desc, void* cuda_stream,
                              ksc_problem** out);
/* Free every device buffer the problem owns.  NULL is accepted. */
ksc_status ksc_problem_destroy(ksc_problem* problem);
/* Device bytes the problem holds now (X copy if owned, y, workspaces). */
size_t ksc_problem_bytes(const ksc_problem* problem);
/* L (Algorithm 3's step constant) and the number of Lanczos steps taken for it
 * (power_iters; 0 when the caller gave L in ksc_problem_desc.lipschitz). */
ksc_status ksc_problem_info(const ksc_problem* problem, double* lipschitz,
                            int32_t* power_iters);

/* The shift lambda of the eigen-perspective relaxation (App. D.2): a certified
 * lower bound on lambda_min(X^T X) (0 when n < p), so that Q = X^T X - lambda I is
 * positive semidefinite whatever the rounding.  A = X^T X is formed in FP64 and
 * bracketed by bisection on shifts c whose Cholesky factorisation of A - c I runs
 * to completion (to 1e-3 relative); lambda is the last such c minus the rounding
 * bound of the factorisation and of A (Higham, Thm 10.3).  Computed once per
 * problem, then returned from the cache.  Errors: KSC_ERR_INVALID_ARG (NULL),
 * KSC_ERR_UNIMPLEMENTED (n >= p > 8192), KSC_ERR_OOM (2 p^2 doubles of workspace),
 * KSC_ERR_CUDA. */
ksc_status ksc_problem_eig_lambda(ksc_problem* problem, void* cuda_stream, double* lambda);
/* Make lambda the problem's eigen shift after certifying it: lambda = 0 is always
 * accepted; lambda > 0 when the Cholesky factorisation of X^T X - c I, c = lambda
 * plus its rounding margin, runs to completion (the test of
 * ksc_problem_eig_lambda).  Errors: KSC_ERR_INVALID_ARG (NULL problem, lambda < 0
 * or not finite, lambda not certified below lambda_min), KSC_ERR_UNIMPLEMENTED
 * (p > 8192), KSC_ERR_OOM, KSC_ERR_CUDA. */
ksc_status ksc_problem_set_eig_lambda(ksc_problem* problem, void* cuda_stream, double lambda);

/* One branch-and-bound node (App. B.3) with its parameters (Sec. 1, Sec. 4.2). */
typedef struct {
  double lambda2;            /* > 0                                                  */
  double M;                  /* > 0, box |b_j| <= M                                  */
  int32_t k;                 /* >= 0 cardinality budget                              */
  const int32_t* fixed_zero; /* S0 indices (host), may be NULL when n_zero = 0       */
  int32_t n_zero;
  const int32_t* fixed_one;  /* S1 indices (host), may be NULL when n_one = 0        */
  int32_t n_one;
  const double* warm_beta;   /* host, length p, or NULL for 0.  S0 entries are set to
                                0 and all entries clipped to [-M, M] before use      */
  double incumbent;          /* +inf: none.  Otherwise the early-termination rules of
                                Sec. 4.3: stop when the certified bound exceeds it
                                (pruned) or the primal value falls below it          */
  double rel_gap_tol;        /* (primal - dual)/|primal| target, e.g. 1e-6 (Sec. 4.2) */
  int32_t max_iter;          /* > 0 */
  uint32_t flags;            /* KSC_FLAG_*                                           */
} ksc_node;

typedef struct {
  double* beta;        /* caller-owned host array, length p, or NULL: final iterate   */
  double* z;           /* caller-owned host array, length p, or NULL: relaxed z that
                          attains g(beta) (from the proof of Thm 3.6)                 */
  double primal;       /* F(X b) + 2 lambda2 g_node(b), FP64 (upper bound on P_conv)  */
  double dual_bound;   /* certified FP64 lower bound on P_conv(node) <= P_MIP(node)   */
  double rel_gap;      /* (primal - dual_bound) / max(|primal|, 1e-300)               */
  int32_t iters;       /* FISTA steps taken                                           */
  int32_t restarts;    /* momentum resets (Algorithm 3's restart test)                      */
  int32_t pruned;      /* 1 if dual_bound > incumbent                                 */
  ksc_status status;   /* KSC_OK (gap met, or an incumbent rule fired),
                          KSC_NOT_CONVERGED, KSC_ERR_INFEASIBLE_NODE                  */
} ksc_result;

/* Solve one node to its gap target and certify the bound (blocking).
 * Infeasible node (|S1| > k or S0 and S1 overlap): result->status and the return
 * value are KSC_ERR_INFEASIBLE_NODE, dual_bound = +inf (the node can be pruned). */
ksc_status ksc_solve_node(ksc_problem* problem, const ksc_node* node, ksc_result* result,
                          void* cuda_stream);

/* Solve `count` nodes of one problem together (blocking); result[i] belongs to
 * node[i].  Each result equals what ksc_solve_node returns for that node, within
 * the stated tolerance.  Returns the first non-OK per-node status, else KSC_OK.
 * With BF16 or FP8 X the nodes advance in lock step (up to 1024 per device pass):
 * both products of every FISTA step run on the tensor cores for all nodes at once
 * (FP8: KSC_E4M3_PIECES E4M3 pieces of each difference against E4M3 X), on differences from
 * per-node anchor points whose products are exact, and every reported bound is the
 * FP64 certificate.  Other storage types (and nodes with k' >= 2048, and
 * eigen-perspective nodes on FP8 X) are solved one by one by the single-node path.  The problem's
 * batched workspace is allocated on first use and kept (ksc_problem_bytes). */
ksc_status ksc_solve_batch(ksc_problem* problem, const ksc_node* nodes, int32_t count,
                           ksc_result* results, void* cuda_stream);

/* ---- branch and bound ------------------------------------------------------ */

/* Best-first branch and bound for Eq. (1) (the minimal framework of Sec. 5.3 and
 * App. B.3): node lower bounds are the certified bounds of the node relaxations,
 * computed by the batched solver with continuous batching (one session of
 * `batch` slots: a finished node's children take free slots at once, best bound
 * first), the node's early-termination rules (Sec. 5.3: primal below the
 * incumbent -> stop and branch; bound above it -> prune) use the incumbent of the
 * moment the node starts.  Incumbents: at every processed node the support
 * S1 + the k' largest free |b_j| of its relaxed solution is solved as a
 * restricted problem (a node with S1 = that support and k = its size, whose
 * relaxation is the box-constrained ridge on the support), in the same slots; its
 * certified primal value is the objective of a feasible point.  Branching: on the
 * free coordinate of that support whose removal raises the objective most to
 * second order, b_j^2 (c ||x_j||^2 + lambda2), c = 1 (least squares) or 1/4
 * (logistic).  A node whose relaxed solution already has at most k' free
 * nonzeros and a certified gap closes (its value is a feasible objective).
 * Stops when (incumbent - lower bound) / max(|incumbent|, 1e-300) <= opt_gap, when
 * every node is pruned or closed, or at max_nodes node solves (0: none) or
 * time_limit_s seconds (0: none).  Needs BF16 or FP8 X (KSC_ERR_UNIMPLEMENTED
 * otherwise; the eigen-perspective flag needs BF16); k < 2048; 1 <= batch <= 1024. */
typedef struct {
  double lambda2, M;
  int32_t k;
  double opt_gap;          /* relative optimality gap to certify, e.g. 1e-4 */
  int64_t max_nodes;       /* node relaxations to solve at most (0 = no limit) */
  double time_limit_s;     /* wall-clock limit (0 = no limit) */
  int32_t batch;           /* session slots (nodes in flight) */
  double node_rel_gap;     /* rel_gap_tol of every node solve */
  int32_t node_max_iter;   /* max_iter of every node solve */
  uint32_t node_flags;     /* KSC_FLAG_* of every node solve (KSC_FLAG_EIG: the
                              eigen-perspective node bounds of App. D.2) */
} ksc_bnb_params;

typedef struct {
  double* beta;            /* caller-owned, length p (or NULL): the incumbent */
  double incumbent;        /* its objective F(X beta) + lambda2 ||beta||^2 (+inf if none) */
  double lower_bound;      /* certified lower bound on the optimum of Eq. (1) */
  double gap;              /* (incumbent - lower_bound) / max(|incumbent|, 1e-300) */
  int64_t nodes;           /* node relaxations solved */
  int64_t pruned;          /* nodes pruned by their bound (at start or after solving) */
  int64_t closed;          /* nodes whose relaxation was already feasible */
  int64_t heuristic_solves;
  int64_t replays;         /* lock-step graph replays (16 steps each) */
  int64_t max_open;        /* largest number of open nodes */
  double seconds;
  int32_t certified;       /* 1: gap <= opt_gap (or nothing left open) */
} ksc_bnb_result;

ksc_status ksc_bnb_solve(ksc_problem* problem, const ksc_bnb_params* params, ksc_bnb_result* result,
                         void* cuda_stream);

/* ---- primitives (host pointers, FP64, one GPU launch each) -------------- */

/* beta = prox_{rho^-1 g}(w) (Moreau identity, Sec. 3.3; Alg. 1 + 4), with the
 * cardinality budget k and box M.  top_out (optional, length min(k, p)) receives
 * the indices of the k largest |w| in descending order, ties by ascending index --
 * the set J of Lemma 3.3 in the order of the sort of Alg. 1. */
ksc_status ksc_prox_g(const double* w, int64_t p, int32_t k, double M, double rho,
                      double* beta_out, int32_t* top_out);
/* g(beta) by Algorithm 2 (+inf outside dom g: |b_j| > M or sum|b| > kM beyond a
 * 1e-12 relative slack); z_out (optional, length p) receives the relaxed z. */
ksc_status ksc_g_value(const double* beta, int64_t p, int32_t k, double M, double* g_out,
                       double* z_out);
/* g*(a) = TopSum_k(H_M(a)) (Lemma 3.1). */
ksc_status ksc_gstar(const double* a, int64_t p, int32_t k, double M, double* out);

/* Allocation-free variant of ksc_prox_g on DEVICE buffers (the paper has no
 * counterpart: this is a deployment convenience).  For callers that must not call
 * cudaMalloc -- runtimes that manage all device memory through their own pools
 * and forbid allocations outside them, loops that cannot afford the implicit
 * synchronisation of an allocation.  w (p doubles), beta_out (p doubles) and
 * top_out (min(k, p) int32, or NULL) are device pointers owned by the caller; the
 * results equal ksc_prox_g's.  Work is enqueued on cuda_stream; the call returns
 * without waiting.  No cudaMalloc, cudaFree or allocating library routine is
 * called: the scratch is a fixed device array of 2^19 doubles (4 MiB) that every
 * GPU loading the library holds until exit, so p above 524288 is rejected with
 * KSC_ERR_INVALID_ARG.  The first call on a device does a one-time set-up (the
 * scratch's device address and a kernel attribute): make it before any stream
 * capture.  All calls on a device share the scratch, so calls that may overlap on
 * the GPU (different streams without ordering) race; order them on one stream.
 * A CUDA error already pending on the calling thread when the call is made (from
 * the caller's earlier asynchronous work) is reported, and cleared, by this call
 * as KSC_ERR_CUDA.  Non-finite entries of w give unspecified (but bounded-time)
 * results. */
ksc_status ksc_prox_g_noalloc(const double* w, int64_t p, int32_t k, double M, double rho,
                              double* beta_out, int32_t* top_out, void* cuda_stream);

/* The prox of ksc_prox_g (Moreau identity, Sec. 3.3; Alg. 1 + 4 in their
 * threshold form) for `count` independent vectors of length p at once, on DEVICE
 * buffers: row r of beta_out (p doubles at beta_out + r * ldb) = prox_{rho^-1 g}
 * of row r of w (p doubles at w + r * ldw), every row with the same k, M, rho.
 * This is the throughput form of the paper's prox timing experiment (Sec. 5.1,
 * Fig. 1: many vectors instead of one).  The caller owns both buffers; they must
 * not overlap (KSC_ERR_INVALID_ARG).  ldw, ldb >= p.  min(k, p) must be below 2048
 * (KSC_ERR_UNIMPLEMENTED; ksc_prox_g takes up to 4095).  count = 0 does nothing.
 * One CTA per row; work is enqueued on cuda_stream and the call returns without
 * waiting.  No device memory is allocated (w is read in place); the first call
 * on a device does the one-time set-up of ksc_prox_g_noalloc.  Results agree with
 * ksc_prox_g to rounding (the two kernels order their FP64 sums differently).
 * ldw and ldb above INT64_MAX / 8 / count are rejected (KSC_ERR_INVALID_ARG).  A
 * CUDA error already pending on the calling thread is reported (and cleared) by
 * this call as KSC_ERR_CUDA.  Non-finite entries of w give unspecified (but
 * bounded-time) results. */
ksc_status ksc_prox_g_batch(const double* w, int64_t ldw, double* beta_out, int64_t ldb, int64_t p,
                            int32_t count, int32_t k, double M, double rho, void* cuda_stream);

/* g(beta) of ksc_g_value (Algorithm 2, Sec. 3.2; +inf outside dom g: some
 * |beta_j| > M or sum |beta_j| > kM) for `count` independent vectors of length p
 * at once, on DEVICE buffers: g_out[r] (a device array of count doubles) = g of
 * row r of beta (p doubles at beta + r * ldb).  The throughput form of the
 * g-value evaluation the restart test of Algorithm 3 needs every step (the
 * paper's g experiment, many vectors instead of one).  ldb >= p (and at most
 * INT64_MAX / 8 / count); min(k, p) must be below 2048 (KSC_ERR_UNIMPLEMENTED).
 * count = 0 does nothing.  One CTA per row; work is enqueued on cuda_stream and
 * the call returns without waiting; no device memory is allocated.  Results agree
 * with ksc_g_value to rounding.  A CUDA error already pending on the calling
 * thread is reported (and cleared) as KSC_ERR_CUDA. */
ksc_status ksc_g_value_batch(const double* beta, int64_t ldb, int64_t p, int32_t count, int32_t k, double M,
                             double* g_out, void* cuda_stream);

/* ---- serving -------------------------------------------------------------- */

/* A request loop on the current device for dual-bound solves of many nodes of
 * many problems (continuous batching).  A worker thread keeps one batched session
 * of max_slots node slots per problem with pending work; nodes that arrive while
 * others run take free slots between CUDA-graph replays (16 FISTA steps), the
 * sessions of different problems run on their own streams and overlap on the
 * device, and finished slots are refilled at once.  A session is opened only
 * while the bytes of its problem (ksc_problem_bytes) plus the session's own
 * workspace, summed over the open sessions, stay within hbm_budget_bytes;
 * requests of other problems wait.  Problems whose X is not BF16 are solved one
 * node at a time by the single-node path on the worker.  While a problem has
 * requests in a server, the caller must not solve on it directly, nor destroy it.
 * max_slots in 1..1024.  KSC_ERR_INVALID_ARG on bad arguments. */
ksc_status ksc_server_create(size_t hbm_budget_bytes, int32_t max_slots, ksc_server** out);
/* Queue one node (non-blocking); the node and its arrays are copied.  *ticket
 * identifies the request.  KSC_ERR_INVALID_ARG for a malformed node (nothing is
 * queued); KSC_ERR_ADMISSION when the problem alone exceeds the budget. */
ksc_status ksc_server_submit(ksc_server* server, ksc_problem* problem, const ksc_node* node,
                             uint64_t* ticket);
/* Wait up to timeout_ms (< 0: forever) for a request.  When done, fills *result
 * (beta and z copied to the caller's arrays when non-NULL, length p), releases
 * the ticket and returns the node's status (KSC_OK, KSC_NOT_CONVERGED,
 * KSC_ERR_INFEASIBLE_NODE, or the error that ended it).  KSC_ERR_TIMEOUT when
 * the wait expires (the request stays queued); KSC_ERR_INVALID_ARG for an
 * unknown or released ticket. */
ksc_status ksc_server_poll(ksc_server* server, uint64_t ticket, ksc_result* result, int32_t timeout_ms);
/* Seconds from submission to completion of a polled request (kept until the
 * server is destroyed). */
ksc_status ksc_server_latency(ksc_server* server, uint64_t ticket, double* seconds);
/* Server counters into stats[0..n): 0 completed requests, 1 graph replays,
 * 2 sessions opened, 3 peak budgeted bytes, 4 requests that waited for budget,
 * 5 requests admitted into a session that was already running. */
ksc_status ksc_server_stats(ksc_server* server, int64_t* stats, int32_t n);
/* Stop the worker (requests not yet finished end with KSC_ERR_TIMEOUT) and free
 * every session. */
ksc_status ksc_server_destroy(ksc_server* server);

/* The tensor-core product of the batched solver, exported so that it can be
 * tested on its own.  The paper has no counterpart: it is the product X beta (and
 * X^T r) of Algorithm 3 for many nodes at once, with each node's FP32 vector split
 * into `pieces` BF16 vectors whose sum is exact.
 *   D[i][j] = sum_{q < pieces} sum_{t < k} A[q * m_pad + i][t] * B[j][t]   (FP32 accumulation)
 * A, B: device BF16 arrays, row-major with row strides lda, ldb (elements; >= k and
 * multiples of 8), 16-byte aligned; A has pieces * m_pad rows (m_pad a multiple of
 * 128; rows m..m_pad-1 of each piece are read but not stored).  D: device FP32,
 * m rows of stride ldd (>= n, a multiple of 4), 16-byte aligned, caller-owned.
 * pieces in 1..3, tile_n (columns of B per CTA) in {64, 128, 256}.  Blocks until
 * the product is done.  KSC_ERR_INVALID_ARG for shapes outside these rules,
 * KSC_ERR_TIMEOUT when a device wait of the kernel gave up (nothing is left
 * running), KSC_ERR_CUDA on a runtime error. */
ksc_status ksc_tc_gemm(const void* A, int32_t pieces, int32_t m, int32_t m_pad, int32_t k, int64_t lda,
                       const void* B, int32_t n, int64_t ldb, float* D, int64_t ldd, int32_t tile_n,
                       void* cuda_stream);
/* The same product with the stream-K schedule of the batched solver: the
 * 128 x tile_n tiles times their K blocks of 64 are split evenly over `grid`
 * persistent CTAs (1..4096); tiles that span several CTAs are summed from FP32
 * partials in CTA order by a second kernel.  Arguments and errors as
 * ksc_tc_gemm; m <= 1024.  Allocates (and frees) the partials' device buffer. */
ksc_status ksc_tc_gemm_sk(const void* A, int32_t pieces, int32_t m, int32_t m_pad, int32_t k, int64_t lda,
                          const void* B, int32_t n, int64_t ldb, float* D, int64_t ldd, int32_t tile_n,
                          int32_t grid, void* cuda_stream);

/* E4M3 pieces of each vector row in the batched solver's products for FP8 X. */
#define KSC_E4M3_PIECES 5
/* The batched solver's product for E4M3 X (FP8 with power-of-two column scales),
 * exported so that it can be tested on its own; the paper has no counterpart (its
 * products are FP64).  KSC_E4M3_PIECES E4M3 pieces of each row of the vectors, scaled by a
 * power of two per row, against E4M3 B, on the tensor cores (kind::f8f6f4); the
 * first three pieces and the last two go to separate accumulators, the latter
 * weighted by 2^-12 (they carry the remainder of the first three times 2^12):
 *   S_q[i][j] = sum_{t < k} A[q * m_pad + i][t] * B[j][t]
 *   D[i][j] = row_scale[i] * col_scale[j] * (sum_{q < 3} S_q + 2^-12 sum_{q >= 3} S_q)
 * (FP32 accumulation).  A, B: device E4M3 bytes, row-major with row strides lda,
 * ldb (bytes; >= k and multiples of 16), 16-byte aligned; A has
 * KSC_E4M3_PIECES * m_pad rows (m_pad a multiple of
 * 128; rows m..m_pad-1 of each piece are read but not stored).  row_scale: device
 * FP32, m entries; col_scale: device FP32, n entries, or NULL for 1.  D: device
 * FP32, m rows of stride ldd (>= n, a multiple of 4), 16-byte aligned.  tile_n in
 * {64, 128}; grid 0: one CTA per tile, else the stream-K schedule over `grid`
 * CTAs (m <= 1024; allocates and frees the partials' buffer).  Blocks until done.
 * Errors as ksc_tc_gemm. */
ksc_status ksc_tc_gemm_e4m3(const void* A, int32_t m, int32_t m_pad, int32_t k, int64_t lda, const void* B,
                            int32_t n, int64_t ldb, const float* row_scale, const float* col_scale, float* D,
                            int64_t ldd, int32_t tile_n, int32_t grid, void* cuda_stream);

/* The exact product of the batched solver's anchors and certificates (Sec. 3.4:
 * the bound needs X^T zeta to a known accuracy) on the tensor cores, on DEVICE
 * buffers owned by the caller, exported so that tests can check it on its own:
 *   D[i][j] = sum_l A[j][l] V[i][l],   i < r, j < c,
 * A BF16 (c x k, row stride lda elements: X for X v, the transpose of X for
 * X^T v), V FP64 (r x k, row stride ldv), D FP64 (r x c, row stride ldd).  Both
 * operands are split into 8-bit fixed-point slices (one exponent per row of A and
 * per vector), every slice product is summed exactly, and
 *   |D[i][j] - exact| <= eps ||A_j||_2 ||V_i||_2,
 * eps written to *err_factor (optional; about 1e-12 for k = 10^4).  r <= 1024.
 * Allocates and frees its slices; blocks until done.  KSC_ERR_INVALID_ARG on
 * NULL pointers or bad sizes, KSC_ERR_OOM, KSC_ERR_CUDA, KSC_ERR_TIMEOUT when a
 * device wait gave up. */
ksc_status ksc_tc_exact(const void* A, int32_t c, int32_t k, int64_t lda, const double* V, int32_t r,
                        int64_t ldv, double* D, int64_t ldd, double* err_factor, void* cuda_stream);

/* ---- profiling ------------------------------------------------------------ */

/* Kernel ids for ksc_problem_kernel_time. */
#define KSC_KERNEL_GRADIENT 0   /* X^T grad F(u) pass (one per FISTA step)           */
#define KSC_KERNEL_PROX     1   /* segmented prox + g + dual TopSum (one per step)   */
#define KSC_KERNEL_FORWARD  2   /* X b pass + restart/gap step (one per step)        */
/* batched solves (ksc_solve_batch), one launch each per batched step:          */
#define KSC_KERNEL_B_RESID  3   /* u_gamma, grad F, its BF16 pieces, -F* terms       */
#define KSC_KERNEL_B_GRAD   4   /* tensor-core X^T r for every node                  */
#define KSC_KERNEL_B_PROX   5   /* one prox / g / dual-term CTA per node             */
#define KSC_KERNEL_B_FWD    6   /* tensor-core X beta for every node + loss partials */
#define KSC_KERNEL_B_STEP   7   /* restart / gap step per node                       */
#define KSC_KERNEL_B_CERT   8   /* FP64 certificates between replays (per node)       */
#define KSC_KERNEL_B_ANCHOR 9   /* exact anchor products between replays (per node)   */
/* the two kernels of KSC_KERNEL_PROX (single-node solves), timed separately:   */
#define KSC_KERNEL_PROX_SELECT 10 /* threshold: top-k' select, candidate sort, root */
#define KSC_KERNEL_PROX_APPLY  11 /* output pass, nonzero list, g (grid-wide)       */
/* Enable (1) or disable (0) CUDA-event timing of each kernel launch of the
 * problem's solves; accumulated totals are read with ksc_problem_kernel_time. */
ksc_status ksc_problem_profile(ksc_problem* problem, int32_t enable);
/* Launch count and summed device milliseconds of one kernel since the last reset;
 * reset != 0 clears the counters after reading. */
ksc_status ksc_problem_kernel_time(ksc_problem* problem, int32_t kernel, int64_t* launches,
                                   double* total_ms, int32_t reset);

/* Statistics of the last ksc_solve_node (or batched ksc_solve_batch) on this
 * problem, written to stats[0..n):
 *   0  FISTA steps taken (batched: summed over the nodes)
 *   1  steps whose forward pass streamed only the nonzero columns of X
 *   2  steps whose prox needed the full-pass root finder (pooled block > 4096)
 *   3  steps whose prox used the candidates predicted from the previous step
 *   4  steps whose dual term used the predicted candidates
 *   5  Lanczos steps taken for L when the problem was created
 *   6  batched: FP64 certificates computed (one per in-loop stop)
 *   7  batched: anchor products computed (exact X beta_ref and X^T r_ref)
 *   8  batched: tile width of the X beta product (columns of X per CTA)
 *   9  batched: 1 if that product ran the stream-K schedule
 *  10  batched: tile width of the X^T r product
 *  11  batched: 1 if that product ran the stream-K schedule
 * Entries 1-4 are 0 after a batched solve, 6-11 after a single-node one; entries
 * beyond 12 are set to 0.  n < 0 or a NULL stats with n > 0 is rejected. */
ksc_status ksc_problem_solve_stats(const ksc_problem* problem, int32_t* stats, int32_t n);

/* In-loop state of node `index` of the last batched ksc_solve_batch call on this
 * problem, for diagnosing convergence (the values the gap and restart tests saw
 * when the node stopped), written to state[0..n):
 *   0  in-loop tolerance   1  best primal    2  best dual       3  in-loop gap
 *   4  last primal         5  last dual      6  g of the iterate 7 restarts
 *   8  FISTA steps         9  certificate gap
 * KSC_ERR_INVALID_ARG when index is outside the last batch (or it was not
 * batched). */
ksc_status ksc_problem_batch_node_state(const ksc_problem* problem, int32_t index, double* state, int32_t n);

/* Number of kernel launches the library has issued for this problem (setup,
 * every kernel node of every replayed step graph, certificates). */
ksc_status ksc_problem_launch_count(const ksc_problem* problem, int64_t* launches);

/* Thread-local text of the last error of a call made on this thread. */
const char* ksc_last_error(void);
/* Library version string. */
const char* ksc_version(void);

#ifdef __cplusplus
}
#endif
#endif
