/*
 * ksc_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see
 * ksc_oracle.h).  Single-threaded, no blocking, no fusion: each routine is the
 * definition it computes (H_M, g*, the losses and their conjugates, the bound)
 * or, for the prox, g and the solver, the paper's method restated from its
 * mathematics (Lemma 3.1, Lemma 3.3, Theorem 3.6, Sec. 3.3, Algorithm 3).
 *
 * Readings of passages where the paper is ambiguous, garbled or silent:
 *  R1  Sign of zeta in the safe bound (Sec. 3.4): weak duality is written as
 *      -F*(-zeta) - G*(X^T zeta); the tight choice, and the one the conjugate
 *      list of App. D.1 and the eigen bound of App. D.2 are written for, is
 *      zeta = -grad F(X beta).  The oracle uses zeta = -grad F.
 *  R2  Node subproblem (App. B.3 "use Algorithm 3 at each node"): fixed-to-zero
 *      coordinates are removed, fixed-to-one coordinates carry lambda2 b^2 with
 *      |b| <= M and leave the budget, k' = k - |ONE|.  Its conjugate follows
 *      from Lemma 3.1 with the separable-sum and scaling rules of App. D.
 *  R3  L (Algorithm 3 input) = c_f lambda_max(X^T X) (1 + 1e-6), c_f = 2 for
 *      least squares (F = ||u-y||^2) and squared hinge (F'' <= 2 where it
 *      exists, F' 2-Lipschitz), 1/4 for logistic.
 *  R4  Relative gap (Sec. 4.2, eps = 1e-6): (primal - dual) / max(|primal|, 1e-300).
 *  R5  Algorithm 4 as printed has typos (an uninitialised first block value, a
 *      loop bound n for p, v_prev for nu_prev, a look-forward test against the
 *      current element); the stack form of the pooling below needs none of it.
 *  R6  Block value of a merged block: prox_{(P_b/N_b) H_M}(S_b/N_b) (App. A).
 *  R7  Ties in the sort of Algorithm 1 / 2: descending |.|, ties by ascending
 *      index (the prox value does not depend on it; the order output does).
 *  R8  Algorithm 3 prints its initial objective as f(beta^1, y); read
 *      F(X beta^1) + 2 lambda2 g(beta^1), the objective its restart test uses.
 *  R9  Alg. 2 assumes beta in dom g; outside a 1e-12 relative slack it returns
 *      +inf (the value of g there, by the convention of Sec. 3).
 *  R10 Warm start: S0 coordinates set to 0 and all coordinates clipped to
 *      [-M, M] before the first step (Algorithm 3 starts from beta^0 = beta^1).
 *  R22 Poisson and Gamma regression (App. D.1): their curvature e^u (Poisson)
 *      and y e^-u (Gamma) is unbounded, so Algorithm 3's fixed step needs a bound
 *      on u over the points it evaluates.  Every iterate lies in dom g_node, inside
 *      {|b_j| <= M, sum |b_j| <= kM}, where |x_i^T b| <= U_i = M TopSum_k(|x_i|);
 *      the extrapolated point b^t + c (b^t - b^{t-1}), 0 <= c < 1, has
 *      |x_i^T b| < 3 U_i, and so has every point of the segment the step's descent
 *      inequality uses.  Hence L = lambda_max(X^T X) max_i c_i with c_i =
 *      e^{3 U_i} (Poisson) or y_i e^{3 U_i} (Gamma).  The warm start is clipped to
 *      the box and, for these two losses, scaled into sum |b_j| <= kM.  The
 *      printed conjugate of the Gamma loss, y h((1 - zeta)/y), is F*(+zeta); with
 *      zeta = -grad F (R1) the bound takes F*(-zeta) = sum y h((1 + zeta)/y),
 *      h(z) = z log z - z (h(0) = 0, +inf for z < 0).
 *  R20 Eigen-perspective bound (App. D.2): the objective keeps its constant
 *      ||y||^2 (so that the bound is one of ||X b - y||^2 + lambda2 ||b||^2 and
 *      equals the Sec. 3.4 bound at lambda = 0): F(b) = b^T Q b and G(b) =
 *      -2 y^T X b + ||y||^2 + 2 lambda_eig g(b), whence the bound
 *      ||y||^2 - b^T Q b - 2 lambda_eig g*((X^T y - Q b) / lambda_eig); the
 *      printed final inequality carries the signs of -F* and -G* as +.  The
 *      smooth part that Algorithm 3 steps on is b^T Q b - 2 y^T X b + ||y||^2,
 *      with gradient 2 X^T (X b - y) - 2 lambda b and Lipschitz constant
 *      2 (lambda_max - lambda); the prox is that of 2 lambda_eig g.  With fixed
 *      sets the same g_node replaces g (R2).
 */
#include "ksc_oracle.h"

#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* ---------------------------------------------------------------- Huber */

/* H_M(a): 1/2 a^2 if |a| <= M, M|a| - M^2/2 otherwise (Sec. 3.1). */
double kso_huber(double a, double M) {
  double t = fabs(a);
  if (t <= M) return 0.5 * t * t;
  return M * t - 0.5 * M * M;
}

/* prox_{c H_M}(x): stationarity v - x + c H_M'(v) = 0 with H_M'(v) = clip(v, -M, M).
 * For |x| <= M(1+c) the minimiser lies in the quadratic piece: v = x/(1+c);
 * otherwise in the linear piece: v = x - c M sgn(x). */
double kso_huber_prox(double x, double c, double M) {
  double t = fabs(x);
  double v = (t <= M * (1.0 + c)) ? t / (1.0 + c) : t - c * M;
  return x < 0 ? -v : v;
}

/* ------------------------------------------------- magnitude order */

typedef struct { double mag; int64_t idx; } kso_entry;

/* Order of the magnitudes used by the prox and by g: descending |v|, equal
 * magnitudes by ascending index (reading R7). */
static int by_magnitude(const void *pa, const void *pb) {
  const kso_entry *a = (const kso_entry *)pa, *b = (const kso_entry *)pb;
  if (a->mag != b->mag) return (a->mag > b->mag) ? -1 : 1;
  return (a->idx > b->idx) - (a->idx < b->idx);
}

static kso_entry *magnitude_order(const double *v, int64_t p) {
  kso_entry *e = (kso_entry *)malloc((size_t)(p > 0 ? p : 1) * sizeof(kso_entry));
  for (int64_t j = 0; j < p; ++j) { e[j].mag = fabs(v[j]); e[j].idx = j; }
  qsort(e, (size_t)p, sizeof(kso_entry), by_magnitude);
  return e;
}

/* ------------------------------------------- prox of rho g* (Sec. 3.3) */

/* prox_{rho g*}(mu) = argmin_a 1/2 ||a - mu||^2 + rho TopSum_k(H_M(a)), with
 * g* in the form of Lemma 3.1.
 *
 * Reduction (Lemma 3.3 and its proof): the minimiser keeps the signs of mu and
 * the order of |mu|, so a_j = sgn(mu_j) nu_(r) where r is the rank of |mu_j|
 * and nu is non-increasing in r.  For non-increasing nu >= 0 the top-k sum is
 * the sum over the first k ranks, so with m_r the r-th largest |mu| the problem
 * becomes an isotonic regression with separable convex terms:
 *
 *     min_{nu_1 >= ... >= nu_p}  sum_r 1/2 (nu_r - m_r)^2 + c_r H_M(nu_r),
 *     c_r = rho for r <= k, 0 otherwise                       (Algorithm 1).
 *
 * It is solved by pooling adjacent violators (the method of Algorithm 4,
 * App. A), here in its textbook stack form: ranks enter left to right as
 * singleton blocks; while the newest block's value exceeds the value of the
 * block before it, the two are merged.  A block B carries its count N_B, the
 * sum S_B of its m_r and the sum P_B of its c_r; completing the square,
 * sum_{r in B} 1/2 (v - m_r)^2 + c_r H_M(v) = N_B [1/2 (v - S_B/N_B)^2 +
 * (P_B/N_B) H_M(v)] + const, so its value is prox_{(P_B/N_B) H_M}(S_B/N_B)
 * (reading R6).  The objective is strictly convex, so the pooled solution is
 * the unique minimiser whatever the merge order. */
typedef struct { double cnt, msum, csum, value; int64_t last; } kso_block;

static double block_value(const kso_block *b, double M) {
  return kso_huber_prox(b->msum / b->cnt, b->csum / b->cnt, M);
}

int kso_prox_gstar(const double *mu, int64_t p, int64_t k, double rho, double M,
                   double *alpha, int64_t *perm) {
  if (p <= 0) return 0;
  kso_entry *ord = magnitude_order(mu, p);
  kso_block *stack = (kso_block *)malloc((size_t)p * sizeof(kso_block));
  int64_t top = -1;                      /* index of the newest block */
  for (int64_t r = 0; r < p; ++r) {
    kso_block nb;
    nb.cnt = 1.0;
    nb.msum = ord[r].mag;
    nb.csum = (r < k) ? rho : 0.0;
    nb.last = r;
    nb.value = block_value(&nb, M);
    stack[++top] = nb;
    while (top > 0 && stack[top].value > stack[top - 1].value) {
      kso_block *lo = &stack[top - 1];
      const kso_block *hi = &stack[top];
      lo->cnt += hi->cnt;
      lo->msum += hi->msum;
      lo->csum += hi->csum;
      lo->last = hi->last;
      lo->value = block_value(lo, M);
      --top;
    }
  }
  /* each rank takes its block's value; a_j = sgn(mu_j) nu_(rank of j) */
  int64_t r = 0;
  for (int64_t b = 0; b <= top; ++b) {
    for (; r <= stack[b].last; ++r) {
      int64_t j = ord[r].idx;
      double s = (mu[j] > 0) ? 1.0 : ((mu[j] < 0) ? -1.0 : 0.0);
      alpha[j] = s * stack[b].value;
      if (perm) perm[r] = j;
    }
  }
  free(stack);
  free(ord);
  return 0;
}

/* Moreau decomposition (Sec. 3.3): prox_{rho^-1 g}(w) = w - rho^-1 prox_{rho g*}(rho w).
 * Where prox_{rho g*} leaves a coordinate unchanged (a_j = mu_j: ranks outside
 * the pooled block past the top k, and every coordinate when k = 0, where g is
 * the indicator of {0}) the decomposition gives beta_j = w_j - rho w_j / rho = 0
 * exactly; it is set to 0 rather than to the rounding residue of that
 * difference (reading R14). */
int kso_prox_g(const double *w, int64_t p, int64_t k, double rho, double M,
               double *beta, int64_t *perm) {
  if (p <= 0) return 0;
  double *mu = (double *)malloc((size_t)p * sizeof(double));
  double *a = (double *)malloc((size_t)p * sizeof(double));
  for (int64_t j = 0; j < p; ++j) mu[j] = rho * w[j];
  kso_prox_gstar(mu, p, k, rho, M, a, perm);
  for (int64_t j = 0; j < p; ++j) beta[j] = (a[j] == mu[j]) ? 0.0 : w[j] - a[j] / rho;
  free(mu);
  free(a);
  return 0;
}

/* ------------------------------------------------- g (Theorem 3.6) */

/* g(beta) = min_z 1/2 sum_j beta_j^2 / z_j over sum z <= k, 0 <= z <= 1,
 * |beta_j| <= M z_j (Sec. 3.1), +inf outside dom g (reading R9).
 *
 * Theorem 3.6 (Algorithm 2) gives the minimiser in closed form: with the
 * magnitudes in descending order, the t largest take z = 1 and the rest share
 * the remaining budget in proportion to their size, z_j = |beta_j| / s with the
 * level s = (sum of the other magnitudes) / (k - t); t is the first count at
 * which the next magnitude does not exceed that level.  Then
 * g = 1/2 sum_{top t} beta_j^2 + 1/2 (k - t) s^2.  When every magnitude past
 * the top t is zero the level is 0 and so is z there. */
double kso_g_value(const double *beta, int64_t p, int64_t k, double M, double *z) {
  double l1 = 0.0, linf = 0.0;
  for (int64_t j = 0; j < p; ++j) {
    double t = fabs(beta[j]);
    l1 += t;
    if (t > linf) linf = t;
  }
  if (z) for (int64_t j = 0; j < p; ++j) z[j] = 0.0;
  if (linf > M * (1.0 + 1e-12) || l1 > (double)k * M * (1.0 + 1e-12)) return INFINITY;
  if (p == 0 || k <= 0) return 0.0;
  kso_entry *ord = magnitude_order(beta, p);
  double rest = l1;          /* sum of the magnitudes not yet given z = 1 */
  double g = 0.0, level = 0.0;
  int64_t t = 0;             /* number of coordinates with z = 1 */
  int found = 0;
  for (; t < k; ++t) {
    double next = (t < p) ? ord[t].mag : 0.0;
    level = rest / (double)(k - t);
    if (next <= level) { found = 1; break; }
    g += 0.5 * next * next;
    rest -= next;
  }
  if (found) g += 0.5 * (double)(k - t) * level * level;
  if (z) {
    for (int64_t r = 0; r < p; ++r) {
      int64_t j = ord[r].idx;
      if (r < t) z[j] = 1.0;
      else z[j] = (found && level > 0.0) ? ord[r].mag / level : 0.0;
    }
  }
  free(ord);
  return g;
}

/* sum of the k largest |v_j| */
static double kso_gstar_abs_topsum(const double *v, int64_t p, int64_t k) {
  if (p <= 0 || k <= 0) return 0.0;
  kso_entry *ord = magnitude_order(v, p);
  double s = 0.0;
  for (int64_t r = 0; r < k && r < p; ++r) s += ord[r].mag;
  free(ord);
  return s;
}

/* Lemma 3.1: g*(a) = sum of the k largest H_M(a_j). */
double kso_gstar(const double *a, int64_t p, int64_t k, double M) {
  if (p <= 0 || k <= 0) return 0.0;
  kso_entry *ord = magnitude_order(a, p);          /* H_M is increasing in |a| */
  double s = 0.0;
  for (int64_t r = 0; r < k && r < p; ++r) s += kso_huber(ord[r].mag, M);
  free(ord);
  return s;
}

/* ----------------------------------------------------------- node forms */

static int64_t count_state(const int8_t *state, int64_t p, int8_t v) {
  int64_t c = 0;
  if (!state) return (v == KSO_FREE) ? p : 0;
  for (int64_t j = 0; j < p; ++j) c += (state[j] == v);
  return c;
}

int kso_prox_g_node(const double *w, int64_t p, const int8_t *state, int64_t k,
                    double rho, double M, double *beta, int64_t *top_order) {
  int64_t nf = count_state(state, p, KSO_FREE);
  int64_t kp = k - count_state(state, p, KSO_ONE);
  if (kp < 0) return -1;
  double *wf = (double *)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(double));
  double *bf = (double *)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(double));
  int64_t *map = (int64_t *)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(int64_t));
  int64_t *perm = (int64_t *)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(int64_t));
  int64_t q = 0;
  for (int64_t j = 0; j < p; ++j) {
    int8_t st = state ? state[j] : KSO_FREE;
    if (st == KSO_FREE) { wf[q] = w[j]; map[q] = j; ++q; }
    else if (st == KSO_ZERO) beta[j] = 0.0;
    else {  /* z_j = 1: argmin 1/2 (b-w)^2 + rho^-1 1/2 b^2, |b| <= M */
      double b = rho * w[j] / (1.0 + rho);
      beta[j] = (b > M) ? M : ((b < -M) ? -M : b);
    }
  }
  kso_prox_g(wf, nf, kp, rho, M, bf, perm);
  for (int64_t r = 0; r < nf; ++r) beta[map[r]] = bf[r];
  if (top_order)
    for (int64_t r = 0; r < kp && r < nf; ++r) top_order[r] = map[perm[r]];
  free(wf); free(bf); free(map); free(perm);
  return 0;
}

double kso_g_node(const double *beta, int64_t p, const int8_t *state, int64_t k,
                  double M, double *z) {
  int64_t nf = count_state(state, p, KSO_FREE);
  int64_t kp = k - count_state(state, p, KSO_ONE);
  if (kp < 0) return INFINITY;
  double g = 0.0;
  double *bf = (double *)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(double));
  double *zf = (double *)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(double));
  int64_t *map = (int64_t *)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(int64_t));
  int64_t q = 0;
  for (int64_t j = 0; j < p; ++j) {
    int8_t st = state ? state[j] : KSO_FREE;
    if (st == KSO_FREE) { bf[q] = beta[j]; map[q] = j; ++q; }
    else if (st == KSO_ZERO) {
      if (beta[j] != 0.0) g = INFINITY;
      if (z) z[j] = 0.0;
    } else {
      if (fabs(beta[j]) > M * (1.0 + 1e-12)) g = INFINITY;
      g += 0.5 * beta[j] * beta[j];
      if (z) z[j] = 1.0;
    }
  }
  g += kso_g_value(bf, nf, kp, M, z ? zf : NULL);
  if (z) for (int64_t r = 0; r < nf; ++r) z[map[r]] = zf[r];
  free(bf); free(zf); free(map);
  return g;
}

double kso_Gstar_node(const double *a, int64_t p, const int8_t *state, int64_t k,
                      double lambda2, double M) {
  int64_t nf = count_state(state, p, KSO_FREE);
  int64_t kp = k - count_state(state, p, KSO_ONE);
  if (kp < 0) return -INFINITY;
  double c = 2.0 * lambda2, one = 0.0;
  double *af = (double *)malloc((size_t)(nf > 0 ? nf : 1) * sizeof(double));
  int64_t q = 0;
  for (int64_t j = 0; j < p; ++j) {
    int8_t st = state ? state[j] : KSO_FREE;
    if (st == KSO_FREE) af[q++] = a[j] / c;
    else if (st == KSO_ONE) one += kso_huber(a[j] / c, M);
    /* ZERO: the indicator of {b_j = 0} has conjugate 0 */
  }
  double t = c * (one + kso_gstar(af, nf, kp, M));
  free(af);
  return t;
}

/* --------------------------------------------------------------- losses */

static double log1pexp(double t) {                 /* log(1 + e^t), stable  */
  return (t > 0) ? t + log1p(exp(-t)) : log1p(exp(t));
}

double kso_loss(int loss, const double *u, const double *y, int64_t n) {
  double f = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (loss == KSO_LOSS_LSQ) { double r = u[i] - y[i]; f += r * r; }
    else if (loss == KSO_LOSS_SQHINGE) { double m = fmax(0.0, 1.0 - y[i] * u[i]); f += m * m; }
    else if (loss == KSO_LOSS_POISSON) f += exp(u[i]) - y[i] * u[i];
    else if (loss == KSO_LOSS_GAMMA) f += y[i] * exp(-u[i]) + u[i];
    else f += log1pexp(-y[i] * u[i]);
  }
  return f;
}

void kso_loss_grad(int loss, const double *u, const double *y, int64_t n, double *grad) {
  for (int64_t i = 0; i < n; ++i) {
    if (loss == KSO_LOSS_LSQ) grad[i] = 2.0 * (u[i] - y[i]);
    else if (loss == KSO_LOSS_SQHINGE) grad[i] = -2.0 * y[i] * fmax(0.0, 1.0 - y[i] * u[i]);
    else if (loss == KSO_LOSS_POISSON) grad[i] = exp(u[i]) - y[i];
    else if (loss == KSO_LOSS_GAMMA) grad[i] = 1.0 - y[i] * exp(-u[i]);
    else {  /* d/du log(1+exp(-y u)) = -y sigma(-y u) */
      double t = -y[i] * u[i];
      double sig = (t >= 0) ? 1.0 / (1.0 + exp(-t)) : exp(t) / (1.0 + exp(t));
      grad[i] = -y[i] * sig;
    }
  }
}

/* -F*(-zeta), App. D.1.  Least squares: y^T zeta - ||zeta||^2 / 4.
 * Logistic (y in {-1,+1}): with q = zeta / y, -sum[(1-q)log(1-q) + q log q],
 * 0 log 0 = 0, and -inf outside q in [0,1].
 * Squared hinge (y in {-1,+1}): F*(-zeta) = sum h(-y_i zeta_i) with
 * h(z) = z + z^2/4 for z <= 0 and +inf for z > 0, so -F*(-zeta) =
 * sum [y_i zeta_i - zeta_i^2 / 4] (y_i^2 = 1) on y_i zeta_i >= 0, -inf elsewhere.
 * Poisson (y >= 0): F*(-zeta) = sum h(y_i - zeta_i); Gamma (y > 0):
 * F*(-zeta) = sum y_i h((1 + zeta_i) / y_i) (reading R22); h(z) = z log z - z,
 * h(0) = 0, and -F*(-zeta) = -inf where an argument is negative. */
static double hlog(double z) { return z > 0.0 ? z * log(z) - z : 0.0; }

double kso_neg_conj(int loss, const double *zeta, const double *y, int64_t n) {
  double t = 0.0;
  for (int64_t i = 0; i < n; ++i) {
    if (loss == KSO_LOSS_POISSON) {
      const double z = y[i] - zeta[i];
      if (z < 0.0) return -INFINITY;
      t -= hlog(z);
      continue;
    }
    if (loss == KSO_LOSS_GAMMA) {
      const double z = (1.0 + zeta[i]) / y[i];
      if (z < 0.0) return -INFINITY;
      t -= y[i] * hlog(z);
      continue;
    }
    if (loss == KSO_LOSS_LSQ) t += y[i] * zeta[i] - 0.25 * zeta[i] * zeta[i];
    else if (loss == KSO_LOSS_SQHINGE) {
      double z = -y[i] * zeta[i];
      if (z > 0.0) return -INFINITY;
      t -= z + 0.25 * z * z;
    } else {
      double q = zeta[i] / y[i];
      if (q < 0.0 || q > 1.0) return -INFINITY;
      double h = 0.0;
      if (q > 0.0) h += q * log(q);
      if (q < 1.0) h += (1.0 - q) * log(1.0 - q);
      t -= h;
    }
  }
  return t;
}

/* ------------------------------------------------------------- matvecs */

static double xat(const void *X, int xdt, int64_t ldx, int64_t i, int64_t j) {
  if (xdt == KSO_X_F32) return (double)((const float *)X)[i * ldx + j];
  return ((const double *)X)[i * ldx + j];
}

/* Threads of the all-cores build (-fopenmp): the rows of X v, and blocks of
 * columns of X^T r, are independent; every output element is summed in the same
 * order as in the single-threaded build, so both builds give identical results. */
int kso_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

void kso_matvec(const void *X, int xdt, int64_t n, int64_t p, int64_t ldx,
                const double *v, double *out) {
#pragma omp parallel for schedule(static)
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < p; ++j) s += xat(X, xdt, ldx, i, j) * v[j];
    out[i] = s;
  }
}

void kso_rmatvec(const void *X, int xdt, int64_t n, int64_t p, int64_t ldx,
                 const double *r, double *out) {
  /* out[j] = sum_i X[i][j] r[i], i ascending, one block of 256 columns at a time */
#pragma omp parallel for schedule(static)
  for (int64_t j0 = 0; j0 < p; j0 += 256) {
    const int64_t j1 = (j0 + 256 < p) ? j0 + 256 : p;
    for (int64_t j = j0; j < j1; ++j) out[j] = 0.0;
    for (int64_t i = 0; i < n; ++i)
      for (int64_t j = j0; j < j1; ++j) out[j] += xat(X, xdt, ldx, i, j) * r[i];
  }
}

double kso_power_iteration(const void *X, int xdt, int64_t n, int64_t p, int64_t ldx,
                           double tol, int64_t max_iter, int64_t *iters_out) {
  double *v = (double *)malloc((size_t)p * sizeof(double));
  double *u = (double *)malloc((size_t)n * sizeof(double));
  double *w = (double *)malloc((size_t)p * sizeof(double));
  double nrm = 0.0;
  for (int64_t j = 0; j < p; ++j) {      /* fixed, generic start vector */
    v[j] = 1.0 + (double)((uint64_t)(j + 1) * 2654435761ull % 1000ull) / 1000.0;
    nrm += v[j] * v[j];
  }
  nrm = sqrt(nrm);
  for (int64_t j = 0; j < p; ++j) v[j] /= nrm;
  double lam = 0.0;
  int64_t it = 0;
  for (it = 1; it <= max_iter; ++it) {
    kso_matvec(X, xdt, n, p, ldx, v, u);
    kso_rmatvec(X, xdt, n, p, ldx, u, w);
    double s = 0.0;
    for (int64_t j = 0; j < p; ++j) s += w[j] * w[j];
    s = sqrt(s);                         /* ||X^T X v|| with ||v|| = 1 */
    if (s == 0.0) { lam = 0.0; break; }
    for (int64_t j = 0; j < p; ++j) v[j] = w[j] / s;
    double prev = lam;
    lam = s;
    if (it > 1 && fabs(lam - prev) <= tol * lam) break;
  }
  if (iters_out) *iters_out = it > max_iter ? max_iter : it;
  free(v); free(u); free(w);
  return lam;
}

/* ------------------------------------------- restarted FISTA (Sec. 3) */

/* Poisson and Gamma (reading R22): max_i c_i, c_i = e^{3 U_i} or y_i e^{3 U_i},
 * U_i = M TopSum_k(|x_i|), the largest |x_i^T b| over |b_j| <= M, sum |b_j| <= kM. */
static double curvature_bound(const kso_solve_args *a) {
  double *row = (double *)malloc((size_t)(a->p > 0 ? a->p : 1) * sizeof(double));
  double c = 0.0;
  for (int64_t i = 0; i < a->n; ++i) {
    for (int64_t j = 0; j < a->p; ++j) row[j] = fabs(xat(a->X, a->x_dtype, a->ldx, i, j));
    const double U = a->M * kso_gstar_abs_topsum(row, a->p, a->k);
    const double ci = (a->loss == KSO_LOSS_GAMMA ? a->y[i] : 1.0) * exp(3.0 * U);
    if (ci > c) c = ci;
  }
  free(row);
  return c;
}

/* Lipschitz constant of beta -> grad F(X beta) (readings R3, R22). */
static double lipschitz(const kso_solve_args *a) {
  if (a->L > 0) return a->L;
  double lmax = kso_power_iteration(a->X, a->x_dtype, a->n, a->p, a->ldx, 1e-10, 10000, NULL);
  if (a->loss == KSO_LOSS_POISSON || a->loss == KSO_LOSS_GAMMA)
    return lmax * (1.0 + 1e-6) * curvature_bound(a);
  double cf = (a->loss == KSO_LOSS_LOGISTIC) ? 0.25 : 2.0;
  if (a->eig > 0) return 2.0 * (lmax * (1.0 + 1e-6) - a->eig);   /* R20 */
  return cf * lmax * (1.0 + 1e-6);
}

static double sumsq(const double *v, int64_t m) {
  double s = 0.0;
  for (int64_t i = 0; i < m; ++i) s += v[i] * v[i];
  return s;
}

/* Objective of the node problem at beta, given u = X beta:
 * F(u) + 2 lambda2 g_node(beta); with eig > 0 the eigen-perspective objective
 * b^T Q b - 2 y^T X b + ||y||^2 + 2 lambda_eig g_node(b) = ||u - y||^2 - eig ||b||^2
 * + 2 (lambda2 + eig) g_node(b) (R20). */
static double objective_at(const kso_solve_args *a, const double *beta, const double *u) {
  double f = kso_loss(a->loss, u, a->y, a->n);
  double g = kso_g_node(beta, a->p, a->state, a->k, a->M, NULL);
  if (a->eig > 0) return f - a->eig * sumsq(beta, a->p) + 2.0 * (a->lambda2 + a->eig) * g;
  return f + 2.0 * a->lambda2 * g;
}

/* Weak-duality bound of Sec. 3.4 at zeta = -grad F(u), u = X beta (reading R1):
 * -F*(-zeta) - G*_node(X^T zeta), G = 2 lambda2 g_node. */
static double bound_at(const kso_solve_args *a, const double *u) {
  int64_t n = a->n, p = a->p;
  double *zeta = (double *)malloc((size_t)n * sizeof(double));
  double *xz = (double *)malloc((size_t)p * sizeof(double));
  kso_loss_grad(a->loss, u, a->y, n, zeta);
  for (int64_t i = 0; i < n; ++i) zeta[i] = -zeta[i];
  kso_rmatvec(a->X, a->x_dtype, n, p, a->ldx, zeta, xz);
  double d = kso_neg_conj(a->loss, zeta, a->y, n)
           - kso_Gstar_node(xz, p, a->state, a->k, a->lambda2, a->M);
  free(zeta);
  free(xz);
  return d;
}

/* Eigen-perspective bound of App. D.2 at beta, given u = X beta (R20):
 * ||y||^2 - b^T Q b - G*_node(2 (X^T y - Q b)), Q b = X^T u - eig b, G* the
 * conjugate of 2 lambda_eig g_node. */
static double eig_bound_at(const kso_solve_args *a, const double *beta, const double *u) {
  int64_t n = a->n, p = a->p;
  double *qb = (double *)malloc((size_t)p * sizeof(double));
  double *arg = (double *)malloc((size_t)p * sizeof(double));
  kso_rmatvec(a->X, a->x_dtype, n, p, a->ldx, u, qb);
  for (int64_t j = 0; j < p; ++j) qb[j] -= a->eig * beta[j];
  kso_rmatvec(a->X, a->x_dtype, n, p, a->ldx, a->y, arg);
  double bqb = 0.0;
  for (int64_t j = 0; j < p; ++j) {
    bqb += beta[j] * qb[j];
    arg[j] = 2.0 * (arg[j] - qb[j]);
  }
  double d = sumsq(a->y, n) - bqb
           - kso_Gstar_node(arg, p, a->state, a->k, a->lambda2 + a->eig, a->M);
  free(qb);
  free(arg);
  return d;
}

static double lower_bound_at(const kso_solve_args *a, const double *beta, const double *u) {
  return (a->eig > 0) ? eig_bound_at(a, beta, u) : bound_at(a, u);
}

double kso_primal(const kso_solve_args *a, const double *beta) {
  double *u = (double *)malloc((size_t)a->n * sizeof(double));
  kso_matvec(a->X, a->x_dtype, a->n, a->p, a->ldx, beta, u);
  double v = objective_at(a, beta, u);
  free(u);
  return v;
}

double kso_dual_bound(const kso_solve_args *a, const double *beta) {
  double *u = (double *)malloc((size_t)a->n * sizeof(double));
  kso_matvec(a->X, a->x_dtype, a->n, a->p, a->ldx, beta, u);
  double d = lower_bound_at(a, beta, u);
  free(u);
  return d;
}

/* Algorithm 3: accelerated proximal gradient on F(X b) + 2 lambda2 g_node(b)
 * with step 1/L, momentum weight phi/(phi+3) and a restart of the momentum
 * counter whenever the objective does not decrease (Sec. 3, Fig. 3); after each
 * step the bound of Sec. 3.4 at the new iterate gives the gap of Sec. 4.2 (R4)
 * and the early-termination rules of Sec. 4.3 (R12).  The prox of the step is
 * the prox of rho^-1 g_node with rho = L / (2 lambda2): a step of length 1/L on
 * 2 lambda2 g_node.  The first iterate is the projected warm start (R10) and the
 * first objective is the objective at it (R8). */
int kso_solve(const kso_solve_args *a, double *beta, double *z, double *trace,
              kso_solve_out *out) {
  int64_t n = a->n, p = a->p;
  memset(out, 0, sizeof(*out));
  if (a->k - count_state(a->state, p, KSO_ONE) < 0) {
    out->status = KSO_INFEASIBLE; out->dual = INFINITY; out->primal = INFINITY;
    return 0;
  }
  const double L = lipschitz(a);
  const double lam = a->lambda2 + (a->eig > 0 ? a->eig : 0.0);   /* lambda_eig, R20 */
  const double rho = L / (2.0 * lam);
  out->L = L;
  double *b_old = (double *)malloc((size_t)p * sizeof(double));   /* b^{t-1} */
  double *b = (double *)malloc((size_t)p * sizeof(double));       /* b^t     */
  double *v = (double *)malloc((size_t)p * sizeof(double));       /* extrapolated point, then the gradient step */
  double *grad = (double *)malloc((size_t)p * sizeof(double));
  double *u = (double *)malloc((size_t)n * sizeof(double));
  double *r = (double *)malloc((size_t)n * sizeof(double));
  double l1 = 0.0;
  for (int64_t j = 0; j < p; ++j) {
    double x = a->warm ? a->warm[j] : 0.0;
    if (a->state && a->state[j] == KSO_ZERO) x = 0.0;
    b_old[j] = b[j] = fmin(fmax(x, -a->M), a->M);
    l1 += fabs(b[j]);
  }
  if ((a->loss == KSO_LOSS_POISSON || a->loss == KSO_LOSS_GAMMA) && l1 > (double)a->k * a->M)
    for (int64_t j = 0; j < p; ++j) b_old[j] = b[j] = b[j] * ((double)a->k * a->M / l1);   /* R22 */
  kso_matvec(a->X, a->x_dtype, n, p, a->ldx, b, u);
  double obj = objective_at(a, b, u);
  double phi = 1.0, D = -INFINITY, gap = INFINITY;
  int64_t t = 0, restarts = 0;
  int32_t status = KSO_MAX_ITER;
  for (t = 1; t <= a->max_iter; ++t) {
    /* extrapolation */
    const double c = a->momentum ? phi / (phi + 3.0) : 0.0;
    for (int64_t j = 0; j < p; ++j) v[j] = b[j] + c * (b[j] - b_old[j]);
    /* gradient of the smooth part at the extrapolated point */
    kso_matvec(a->X, a->x_dtype, n, p, a->ldx, v, u);
    kso_loss_grad(a->loss, u, a->y, n, r);
    kso_rmatvec(a->X, a->x_dtype, n, p, a->ldx, r, grad);
    if (a->eig > 0)                                  /* Q = X^T X - eig I, R20 */
      for (int64_t j = 0; j < p; ++j) grad[j] -= 2.0 * a->eig * v[j];
    /* proximal step */
    for (int64_t j = 0; j < p; ++j) v[j] -= grad[j] / L;
    memcpy(b_old, b, (size_t)p * sizeof(double));
    kso_prox_g_node(v, p, a->state, a->k, rho, a->M, b, NULL);
    /* objective, restart test, bound and gap at the new iterate */
    kso_matvec(a->X, a->x_dtype, n, p, a->ldx, b, u);
    const double obj_new = objective_at(a, b, u);
    if (a->restart && obj_new >= obj) { phi = 1.0; ++restarts; }
    else phi += 1.0;
    obj = obj_new;
    D = lower_bound_at(a, b, u);
    gap = (obj - D) / fmax(fabs(obj), 1e-300);
    if (trace) { trace[2 * (t - 1)] = obj; trace[2 * (t - 1) + 1] = D; }
    if (isfinite(a->incumbent)) {
      if (D > a->incumbent) { status = KSO_PRUNED; break; }
      if (obj < a->incumbent) { status = KSO_PRIMAL_BELOW; break; }
    }
    if (gap <= a->tol) { status = KSO_CONVERGED; break; }
  }
  if (t > a->max_iter) t = a->max_iter;
  memcpy(beta, b, (size_t)p * sizeof(double));
  if (z) kso_g_node(b, p, a->state, a->k, a->M, z);
  out->primal = obj; out->dual = D; out->gap = gap;
  out->iters = t; out->restarts = restarts; out->status = status;
  free(b_old); free(b); free(v); free(grad); free(u); free(r);
  return 0;
}
