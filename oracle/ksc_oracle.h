/*
 * ksc_oracle.h -- plain FP64 CPU oracle for the perspective relaxation of the
 * k-sparse, box-constrained, ridge-regularised GLM (arXiv 2502.09502).
 *
 * TEST INFRASTRUCTURE ONLY.  This code is the slow, obviously-correct
 * reference that the CUDA library is compared against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it.  It
 * shares no code, header, table or helper with the CUDA path.
 *
 * Every routine is a definition written out, or the paper's method restated
 * from its mathematics, in FP64:
 *   - Huber function H_M ............................ Sec. 3.1
 *   - g*(a) = TopSum_k(H_M(a)) ...................... Lemma 3.1
 *   - prox_{rho g*}: sign/order reduction to an isotonic regression (Lemma 3.3)
 *     solved by pooling adjacent violators (the method of App. A), stack form
 *   - prox_{rho^-1 g} by the Moreau decomposition ... Sec. 3.3
 *   - g(beta) in closed form ........................ Theorem 3.6
 *   - restarted accelerated proximal gradient ....... Algorithm 3 (Sec. 3)
 *   - safe lower bound by weak duality .............. Sec. 3.4, with the GLM
 *     conjugates of App. D.1
 *
 * Node form (branch-and-bound, App. B.3): coordinates carry a state
 *   KSO_FREE (z_j in [0,1]), KSO_ZERO (z_j = 0, beta_j = 0) or KSO_ONE
 *   (z_j = 1).  With k' = k - |ONE|, the node's implicit function is
 *   g_node(b) = 1/2 sum_{ONE} b_j^2 (|b_j| <= M) + g_{k'}(b_FREE) + [b_ZERO = 0].
 *
 * Readings of passages where the paper is ambiguous are listed in the header
 * comment of ksc_oracle.c.
 */
#ifndef KSC_ORACLE_H
#define KSC_ORACLE_H
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* losses (App. D.1): least squares ||u - y||^2, logistic sum log(1 + e^{-y u}),
 * squared hinge sum max(0, 1 - y u)^2 (y in {-1, +1} for those two), Poisson
 * sum e^u - y u (y >= 0), Gamma sum y e^{-u} + u (y > 0) */
enum { KSO_LOSS_LSQ = 0, KSO_LOSS_LOGISTIC = 1, KSO_LOSS_SQHINGE = 2, KSO_LOSS_POISSON = 3, KSO_LOSS_GAMMA = 4 };
enum { KSO_X_F64 = 0, KSO_X_F32 = 1 };
enum { KSO_FREE = 0, KSO_ZERO = 1, KSO_ONE = 2 };
enum {
  KSO_CONVERGED = 0,     /* relative gap <= tol                       */
  KSO_MAX_ITER = 1,      /* iteration cap reached; bound still valid  */
  KSO_PRUNED = 2,        /* dual bound above the incumbent            */
  KSO_PRIMAL_BELOW = 3,  /* primal value below the incumbent          */
  KSO_INFEASIBLE = 4     /* |ONE| > k                                 */
};

/* Huber function H_M (Sec. 3.1). */
double kso_huber(double a, double M);
/* prox_{c H_M}(x) = argmin_v 1/2 (v-x)^2 + c H_M(v), c >= 0. */
double kso_huber_prox(double x, double c, double M);

/* prox_{rho g*}(mu) (Sec. 3.3, Lemma 3.3, App. A).  perm (optional, length p)
 * receives the sort order pi: perm[r] = index of the r-th largest |mu|
 * (ties broken by ascending index).  Returns 0. */
int kso_prox_gstar(const double *mu, int64_t p, int64_t k, double rho, double M,
                   double *alpha, int64_t *perm);
/* prox_{rho^-1 g}(w) = w - rho^-1 prox_{rho g*}(rho w)  (Moreau, Sec. 3.3). */
int kso_prox_g(const double *w, int64_t p, int64_t k, double rho, double M,
               double *beta, int64_t *perm);
/* g(beta) by Theorem 3.6; z (optional, length p) receives the minimising
 * relaxed z.  Returns +inf when beta is outside dom g (relative slack 1e-12). */
double kso_g_value(const double *beta, int64_t p, int64_t k, double M, double *z);
/* g*(a) = TopSum_k(H_M(a)), Lemma 3.1. */
double kso_gstar(const double *a, int64_t p, int64_t k, double M);

/* Node versions (state: length p, values KSO_FREE/ZERO/ONE, or NULL = all free). */
int kso_prox_g_node(const double *w, int64_t p, const int8_t *state, int64_t k,
                    double rho, double M, double *beta, int64_t *top_order);
double kso_g_node(const double *beta, int64_t p, const int8_t *state, int64_t k,
                  double M, double *z);
/* G*(a) for G = 2 lambda2 g_node: 2 lambda2 [sum_ONE H_M(a_j/2l2) + TopSum_k'(H_M(a_F/2l2))]. */
double kso_Gstar_node(const double *a, int64_t p, const int8_t *state, int64_t k,
                      double lambda2, double M);

/* GLM losses F(u) (App. D.1), their gradients and -F*(-zeta). */
double kso_loss(int loss, const double *u, const double *y, int64_t n);
void kso_loss_grad(int loss, const double *u, const double *y, int64_t n, double *grad);
double kso_neg_conj(int loss, const double *zeta, const double *y, int64_t n);

/* Threads the matrix-vector products use: 1, or OpenMP's count in the build made
 * with -fopenmp (the all-cores timing of the benchmark's CPU baseline). */
int kso_threads(void);
/* Row-major X (n x p, leading dimension ldx) in FP64 or FP32 (promoted exactly). */
void kso_matvec(const void *X, int xdt, int64_t n, int64_t p, int64_t ldx,
                const double *v, double *out);               /* out = X v   */
void kso_rmatvec(const void *X, int xdt, int64_t n, int64_t p, int64_t ldx,
                 const double *r, double *out);              /* out = X^T r */
/* lambda_max(X^T X) by power iteration (relative change < tol). */
double kso_power_iteration(const void *X, int xdt, int64_t n, int64_t p, int64_t ldx,
                           double tol, int64_t max_iter, int64_t *iters_out);

typedef struct {
  const void *X; int32_t x_dtype; int64_t n, p, ldx;
  const double *y; int32_t loss;
  double lambda2, M; int64_t k;
  const int8_t *state;     /* length p or NULL */
  const double *warm;      /* length p or NULL */
  double L;                /* <= 0: c_f * lambda_max(X^T X) * (1 + 1e-6); Poisson and
                              Gamma: the curvature bound of reading R22 */
  double tol;              /* relative gap target                      */
  int64_t max_iter;
  int32_t restart, momentum;   /* Algorithm 3 as printed: both 1      */
  double incumbent;        /* +inf: no early termination              */
  double eig;              /* least squares only: 0 = the perspective
                              relaxation; lambda in (0, lambda_min(X^T X)]
                              = the eigen-perspective relaxation of App. D.2
                              with Q = X^T X - lambda I, lambda_eig =
                              lambda2 + lambda                         */
} kso_solve_args;

typedef struct {
  double primal, dual, gap, L;
  int64_t iters, restarts;
  int32_t status;
} kso_solve_out;

/* Restarted FISTA (Algorithm 3) on the node problem, with the weak-duality
 * bound of Sec. 3.4 evaluated at zeta = -grad F(X beta^t) after every step.
 * beta (length p) and z (length p, optional) receive the final iterate and its
 * relaxed z; trace (optional, 2*max_iter doubles) receives (primal, dual)
 * per iteration. */
int kso_solve(const kso_solve_args *a, double *beta, double *z, double *trace,
              kso_solve_out *out);
/* The weak-duality bound -F*(-zeta) - G*(X^T zeta) at zeta = -grad F(X beta);
 * with eig > 0 the eigen-perspective bound of App. D.2 at zeta = -2 Q beta. */
double kso_dual_bound(const kso_solve_args *a, const double *beta);
/* The primal value F(X beta) + 2 lambda2 g_node(beta); with eig > 0
 * ||X beta - y||^2 - eig ||beta||^2 + 2 (lambda2 + eig) g_node(beta). */
double kso_primal(const kso_solve_args *a, const double *beta);

#ifdef __cplusplus
}
#endif
#endif
