/*
 * ksc_oracle.c -- plain FP64 CPU oracle (TEST INFRASTRUCTURE ONLY; see
 * ksc_oracle.h).  Single-threaded, no blocking, no fusion: each routine is the
 * paper's definition or algorithm written out step by step.
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
 *  R5  Algorithm 4 typos: nu_1 := nuhat_1; loop bound n := p; v_prev := nu_prev;
 *      the look-forward test reads "j < p and nu <= nuhat_{j+1}".
 *  R6  Block value of a merged block: prox_{(P_b/N_b) H_M}(S_b/N_b) (App. A).
 *  R7  Ties in the sort of Algorithm 1 / 2: descending |.|, ties by ascending
 *      index (the prox value does not depend on it; the order output does).
 *  R8  Algorithm 3 line 2 prints L^1 = f(beta^1, y); read f(X beta^1, y) +
 *      2 lambda2 g(beta^1), the same objective as line 10.
 *  R9  Alg. 2 assumes beta in dom g; outside a 1e-12 relative slack it returns
 *      +inf (the value of g there, by the convention of Sec. 3).
 *  R10 Warm start: S0 coordinates set to 0 and all coordinates clipped to
 *      [-M, M] before the first step (Algorithm 3 starts from beta^0 = beta^1).
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

/* ------------------------------------------------------------ sorting */

typedef struct { double key; int64_t idx; } kso_pair;

/* descending key, ties by ascending index (reading R7) */
static int cmp_desc_stable(const void *pa, const void *pb) {
  const kso_pair *a = (const kso_pair *)pa, *b = (const kso_pair *)pb;
  if (a->key > b->key) return -1;
  if (a->key < b->key) return 1;
  return (a->idx < b->idx) ? -1 : (a->idx > b->idx);
}

static kso_pair *sorted_abs(const double *v, int64_t p) {
  kso_pair *s = (kso_pair *)malloc((size_t)(p > 0 ? p : 1) * sizeof(kso_pair));
  for (int64_t j = 0; j < p; ++j) { s[j].key = fabs(v[j]); s[j].idx = j; }
  qsort(s, (size_t)p, sizeof(kso_pair), cmp_desc_stable);
  return s;
}

/* ------------------------------------------------- Algorithm 1 + 4 (PAVA) */

int kso_prox_gstar(const double *mu, int64_t p, int64_t k, double rho, double M,
                   double *alpha, int64_t *perm) {
  if (p <= 0) return 0;
  /* line 3: SpecialSort -- m[r] = |mu_{pi(r)}| in non-increasing order */
  kso_pair *s = sorted_abs(mu, p);
  double *m = (double *)malloc((size_t)p * sizeof(double));
  double *w = (double *)malloc((size_t)p * sizeof(double));     /* rho_j  */
  double *nuhat = (double *)malloc((size_t)p * sizeof(double));
  for (int64_t r = 0; r < p; ++r) {
    m[r] = s[r].key;
    w[r] = (r < k) ? rho : 0.0;                                 /* line 1 */
    nuhat[r] = kso_huber_prox(m[r], w[r], M);                   /* lines 7-9 */
  }
  /* lines 11-14 via Algorithm 4 (1-based block arrays as printed) */
  double *P = (double *)malloc((size_t)(p + 1) * sizeof(double));
  double *S = (double *)malloc((size_t)(p + 1) * sizeof(double));
  double *N = (double *)malloc((size_t)(p + 1) * sizeof(double));
  double *nu = (double *)malloc((size_t)(p + 1) * sizeof(double));
  int64_t *rr = (int64_t *)malloc((size_t)(p + 1) * sizeof(int64_t));
  int64_t b = 1;
  P[1] = w[0]; S[1] = m[0]; N[1] = 1.0; nu[1] = nuhat[0]; rr[1] = 1;
  double nu_prev = nuhat[0];
  int64_t j = 2;                                   /* 1-based element index */
  while (j <= p) {
    b = b + 1;
    P[b] = w[j - 1]; S[b] = m[j - 1]; N[b] = 1.0;
    double v = nuhat[j - 1];
    if (v > nu_prev) {                             /* isotonic violation    */
      b = b - 1;
      P[b] += w[j - 1]; S[b] += m[j - 1]; N[b] += 1.0;
      v = kso_huber_prox(S[b] / N[b], P[b] / N[b], M);
      while (j < p && v <= nuhat[j]) {             /* look forward (R5)     */
        j = j + 1;
        P[b] += w[j - 1]; S[b] += m[j - 1]; N[b] += 1.0;
        v = kso_huber_prox(S[b] / N[b], P[b] / N[b], M);
      }
      while (b > 1 && nu[b - 1] < v) {             /* look backward         */
        b = b - 1;
        P[b] += P[b + 1]; S[b] += S[b + 1]; N[b] += N[b + 1];
        v = kso_huber_prox(S[b] / N[b], P[b] / N[b], M);
      }
    }
    nu[b] = v; rr[b] = j;
    nu_prev = v; j = j + 1;
  }
  /* expand block values back over their elements */
  int64_t start = 0;
  for (int64_t l = 1; l <= b; ++l) {
    for (int64_t q = start; q < rr[l]; ++q) nuhat[q] = nu[l];
    start = rr[l];
  }
  /* line 16: sgn(mu) .* pi^{-1}(nuhat) */
  for (int64_t r = 0; r < p; ++r) {
    int64_t i = s[r].idx;
    double sg = (mu[i] > 0) ? 1.0 : ((mu[i] < 0) ? -1.0 : 0.0);
    alpha[i] = sg * nuhat[r];
    if (perm) perm[r] = i;
  }
  free(P); free(S); free(N); free(nu); free(rr);
  free(m); free(w); free(nuhat); free(s);
  return 0;
}

/* Moreau identity (Sec. 3.3): prox_{rho^-1 g}(w) = w - rho^-1 prox_{rho g*}(rho w).
 * Where prox_{rho g*} leaves a coordinate unchanged (alpha_j = mu_j: the tail
 * outside the pooled block, and every coordinate when k = 0, where g is the
 * indicator of {0}) the identity gives beta_j = w_j - rho w_j / rho = 0 exactly;
 * it is set to 0 rather than to the rounding residue of that difference. */
int kso_prox_g(const double *w, int64_t p, int64_t k, double rho, double M,
               double *beta, int64_t *perm) {
  if (p <= 0) return 0;
  double *mu = (double *)malloc((size_t)p * sizeof(double));
  double *al = (double *)malloc((size_t)p * sizeof(double));
  for (int64_t j = 0; j < p; ++j) mu[j] = rho * w[j];
  kso_prox_gstar(mu, p, k, rho, M, al, perm);
  for (int64_t j = 0; j < p; ++j) beta[j] = (al[j] == mu[j]) ? 0.0 : w[j] - al[j] / rho;
  free(mu); free(al);
  return 0;
}

/* ------------------------------------------------------ Algorithm 2 (g) */

double kso_g_value(const double *beta, int64_t p, int64_t k, double M, double *z) {
  double l1 = 0.0, linf = 0.0;
  for (int64_t j = 0; j < p; ++j) {
    double t = fabs(beta[j]);
    l1 += t;
    if (t > linf) linf = t;
  }
  if (z) for (int64_t j = 0; j < p; ++j) z[j] = 0.0;
  /* dom g: |b_j| <= M and sum |b_j| <= k M (reading R9) */
  if (linf > M * (1.0 + 1e-12) || l1 > (double)k * M * (1.0 + 1e-12)) return INFINITY;
  if (p == 0 || k <= 0) return 0.0;
  kso_pair *s = sorted_abs(beta, p);               /* line 2 (full sort)    */
  double sum = l1;                                 /* line 3                */
  double g = 0.0, sbar = 0.0;
  int64_t jstar = -1;                              /* 0-based break position */
  for (int64_t j = 0; j < k; ++j) {                /* lines 5-8             */
    double bj = (j < p) ? s[j].key : 0.0;
    sbar = sum / (double)(k - j);
    if (sbar >= bj) {                              /* psi_{j:k} = sbar      */
      g += 0.5 * (double)(k - j) * sbar * sbar;
      jstar = j;
      break;
    }
    g += 0.5 * bj * bj;                            /* psi_j = |b_j|         */
    sum -= bj;
  }
  /* relaxed z (from the proof of Thm 3.6): z = 1 where psi_j = |b_j|, and
   * z_j = |b_j| / sbar on the rest of the coordinates */
  if (z) {
    int64_t fixed = (jstar < 0) ? (k < p ? k : p) : jstar;
    for (int64_t r = 0; r < p; ++r) {
      int64_t i = s[r].idx;
      if (r < fixed) z[i] = 1.0;
      else z[i] = (sbar > 0.0) ? s[r].key / sbar : 0.0;
    }
  }
  free(s);
  return g;
}

/* Lemma 3.1: g*(a) = sum of the k largest H_M(a_j). */
double kso_gstar(const double *a, int64_t p, int64_t k, double M) {
  if (p <= 0 || k <= 0) return 0.0;
  kso_pair *s = sorted_abs(a, p);                  /* H_M monotone in |a|  */
  double t = 0.0;
  for (int64_t r = 0; r < k && r < p; ++r) t += kso_huber(s[r].key, M);
  free(s);
  return t;
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
    else f += log1pexp(-y[i] * u[i]);
  }
  return f;
}

void kso_loss_grad(int loss, const double *u, const double *y, int64_t n, double *grad) {
  for (int64_t i = 0; i < n; ++i) {
    if (loss == KSO_LOSS_LSQ) grad[i] = 2.0 * (u[i] - y[i]);
    else if (loss == KSO_LOSS_SQHINGE) grad[i] = -2.0 * y[i] * fmax(0.0, 1.0 - y[i] * u[i]);
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
 * sum [y_i zeta_i - zeta_i^2 / 4] (y_i^2 = 1) on y_i zeta_i >= 0, -inf elsewhere. */
double kso_neg_conj(int loss, const double *zeta, const double *y, int64_t n) {
  double t = 0.0;
  for (int64_t i = 0; i < n; ++i) {
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

void kso_matvec(const void *X, int xdt, int64_t n, int64_t p, int64_t ldx,
                const double *v, double *out) {
  for (int64_t i = 0; i < n; ++i) {
    double s = 0.0;
    for (int64_t j = 0; j < p; ++j) s += xat(X, xdt, ldx, i, j) * v[j];
    out[i] = s;
  }
}

void kso_rmatvec(const void *X, int xdt, int64_t n, int64_t p, int64_t ldx,
                 const double *r, double *out) {
  for (int64_t j = 0; j < p; ++j) out[j] = 0.0;
  for (int64_t i = 0; i < n; ++i)
    for (int64_t j = 0; j < p; ++j) out[j] += xat(X, xdt, ldx, i, j) * r[i];
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

/* ------------------------------------------------------ Algorithm 3 */

static double lipschitz(const kso_solve_args *a) {
  if (a->L > 0) return a->L;
  double lmax = kso_power_iteration(a->X, a->x_dtype, a->n, a->p, a->ldx, 1e-10, 10000, NULL);
  double cf = (a->loss == KSO_LOSS_LOGISTIC) ? 0.25 : 2.0;
  if (a->eig > 0) return 2.0 * (lmax * (1.0 + 1e-6) - a->eig);   /* R20 */
  return cf * lmax * (1.0 + 1e-6);
}

static double sumsq(const double *v, int64_t m) {
  double s = 0.0;
  for (int64_t i = 0; i < m; ++i) s += v[i] * v[i];
  return s;
}

double kso_primal(const kso_solve_args *a, const double *beta) {
  double *u = (double *)malloc((size_t)a->n * sizeof(double));
  kso_matvec(a->X, a->x_dtype, a->n, a->p, a->ldx, beta, u);
  double f = kso_loss(a->loss, u, a->y, a->n);
  double g = kso_g_node(beta, a->p, a->state, a->k, a->M, NULL);
  free(u);
  if (a->eig > 0)   /* b^T Q b - 2 y^T X b + ||y||^2 + 2 lambda_eig g(b), R20 */
    return f - a->eig * sumsq(beta, a->p) + 2.0 * (a->lambda2 + a->eig) * g;
  return f + 2.0 * a->lambda2 * g;
}

/* App. D.2: ||y||^2 - b^T Q b - G*_node(2 (X^T y - Q b)) with Q b = X^T X b - eig b
 * and G*_node the conjugate of 2 lambda_eig g_node (R20). */
static double eig_dual_bound(const kso_solve_args *a, const double *beta) {
  int64_t n = a->n, p = a->p;
  double *u = (double *)malloc((size_t)n * sizeof(double));
  double *qb = (double *)malloc((size_t)p * sizeof(double));
  double *xty = (double *)malloc((size_t)p * sizeof(double));
  kso_matvec(a->X, a->x_dtype, n, p, a->ldx, beta, u);
  kso_rmatvec(a->X, a->x_dtype, n, p, a->ldx, u, qb);
  for (int64_t j = 0; j < p; ++j) qb[j] -= a->eig * beta[j];          /* Q b */
  kso_rmatvec(a->X, a->x_dtype, n, p, a->ldx, a->y, xty);
  double bqb = 0.0;
  for (int64_t j = 0; j < p; ++j) {
    bqb += beta[j] * qb[j];
    xty[j] = 2.0 * (xty[j] - qb[j]);                                  /* a */
  }
  double d = sumsq(a->y, n) - bqb
           - kso_Gstar_node(xty, p, a->state, a->k, a->lambda2 + a->eig, a->M);
  free(u); free(qb); free(xty);
  return d;
}

double kso_dual_bound(const kso_solve_args *a, const double *beta) {
  if (a->eig > 0) return eig_dual_bound(a, beta);
  int64_t n = a->n, p = a->p;
  double *u = (double *)malloc((size_t)n * sizeof(double));
  double *zeta = (double *)malloc((size_t)n * sizeof(double));
  double *xz = (double *)malloc((size_t)p * sizeof(double));
  kso_matvec(a->X, a->x_dtype, n, p, a->ldx, beta, u);
  kso_loss_grad(a->loss, u, a->y, n, zeta);
  for (int64_t i = 0; i < n; ++i) zeta[i] = -zeta[i];        /* reading R1 */
  kso_rmatvec(a->X, a->x_dtype, n, p, a->ldx, zeta, xz);
  double d = kso_neg_conj(a->loss, zeta, a->y, n)
           - kso_Gstar_node(xz, p, a->state, a->k, a->lambda2, a->M);
  free(u); free(zeta); free(xz);
  return d;
}

int kso_solve(const kso_solve_args *a, double *beta, double *z, double *trace,
              kso_solve_out *out) {
  int64_t n = a->n, p = a->p;
  memset(out, 0, sizeof(*out));
  int64_t kp = a->k - count_state(a->state, p, KSO_ONE);
  if (kp < 0) {
    out->status = KSO_INFEASIBLE; out->dual = INFINITY; out->primal = INFINITY;
    return 0;
  }
  double L = lipschitz(a);
  double lam = a->lambda2 + (a->eig > 0 ? a->eig : 0.0);   /* lambda_eig, R20 */
  double rho = L / (2.0 * lam);
  out->L = L;
  double *bprev = (double *)malloc((size_t)p * sizeof(double));
  double *bcur = (double *)malloc((size_t)p * sizeof(double));
  double *gam = (double *)malloc((size_t)p * sizeof(double));
  double *grad = (double *)malloc((size_t)p * sizeof(double));
  double *u = (double *)malloc((size_t)n * sizeof(double));
  double *r = (double *)malloc((size_t)n * sizeof(double));
  /* line 1 (with a warm start, reading R10) */
  for (int64_t j = 0; j < p; ++j) {
    double b = a->warm ? a->warm[j] : 0.0;
    if (a->state && a->state[j] == KSO_ZERO) b = 0.0;
    b = (b > a->M) ? a->M : ((b < -a->M) ? -a->M : b);
    bprev[j] = bcur[j] = b;
  }
  double phi = 1.0;
  double Lcur = kso_primal(a, bcur);                          /* line 2, R8 */
  double D = -INFINITY, gap = INFINITY;
  int64_t t = 0, restarts = 0;
  int32_t status = KSO_MAX_ITER;
  for (t = 1; t <= a->max_iter; ++t) {
    double c = a->momentum ? phi / (phi + 3.0) : 0.0;
    for (int64_t j = 0; j < p; ++j) gam[j] = bcur[j] + c * (bcur[j] - bprev[j]);  /* line 5 */
    kso_matvec(a->X, a->x_dtype, n, p, a->ldx, gam, u);
    kso_loss_grad(a->loss, u, a->y, n, r);
    kso_rmatvec(a->X, a->x_dtype, n, p, a->ldx, r, grad);   /* grad F(gamma) */
    if (a->eig > 0)                                          /* - 2 eig gamma, R20 */
      for (int64_t j = 0; j < p; ++j) grad[j] -= 2.0 * a->eig * gam[j];
    for (int64_t j = 0; j < p; ++j) gam[j] -= grad[j] / L;  /* line 7 */
    memcpy(bprev, bcur, (size_t)p * sizeof(double));
    kso_prox_g_node(gam, p, a->state, a->k, rho, a->M, bcur, NULL);  /* line 8 */
    double Lnext = kso_primal(a, bcur);                     /* line 10 */
    if (a->restart && Lnext >= Lcur) { phi = 1.0; ++restarts; }       /* line 11 */
    else phi = phi + 1.0;
    Lcur = Lnext;
    D = kso_dual_bound(a, bcur);                            /* Sec. 3.4 */
    gap = (Lcur - D) / fmax(fabs(Lcur), 1e-300);            /* R4 */
    if (trace) { trace[2 * (t - 1)] = Lcur; trace[2 * (t - 1) + 1] = D; }
    if (isfinite(a->incumbent)) {                           /* Sec. 4.3 rules */
      if (D > a->incumbent) { status = KSO_PRUNED; break; }
      if (Lcur < a->incumbent) { status = KSO_PRIMAL_BELOW; break; }
    }
    if (gap <= a->tol) { status = KSO_CONVERGED; break; }
  }
  if (t > a->max_iter) t = a->max_iter;
  memcpy(beta, bcur, (size_t)p * sizeof(double));
  if (z) kso_g_node(bcur, p, a->state, a->k, a->M, z);
  out->primal = Lcur; out->dual = D; out->gap = gap;
  out->iters = t; out->restarts = restarts; out->status = status;
  free(bprev); free(bcur); free(gam); free(grad); free(u); free(r);
  return 0;
}
