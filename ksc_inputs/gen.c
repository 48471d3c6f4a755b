/*
 * gen.c -- seeded synthetic design matrices for the k-sparse GLM workloads.
 *
 * Shared by the tests, the benchmark and both sides of every parity check; it
 * holds none of the solver's arithmetic.  Rows follow the paper's generator
 * (App. B.2): x_i ~ N(0, Sigma) with Toeplitz Sigma_jl = r^|j-l|, realised as
 * the stationary AR(1) recursion x_i1 = e_i1, x_ij = r x_i,j-1 + sqrt(1-r^2) e_ij,
 * followed by column standardisation (mean 0, squared norm n).
 *
 * Gaussians e_ij come from Box-Muller over Philox4x32-10 (Salmon, Moraes,
 * Dror, Shaw, "Parallel random numbers: as easy as 1, 2, 3", SC'11), keyed by
 * (seed, stream) and counted by (pair index, row).  The result depends only on
 * (n, p, r, seed): rows are produced in fixed blocks and column statistics are
 * combined in block order, whatever the number of threads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KSG_ROWS_PER_BLOCK 64

/* ------------------------------------------------------------ Philox */

static inline void mulhilo32(uint32_t a, uint32_t b, uint32_t *hi, uint32_t *lo) {
  uint64_t prod = (uint64_t)a * (uint64_t)b;
  *hi = (uint32_t)(prod >> 32);
  *lo = (uint32_t)prod;
}

void ksg_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  uint32_t c0 = ctr_in[0], c1 = ctr_in[1], c2 = ctr_in[2], c3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    uint32_t hi0, lo0, hi1, lo1;
    mulhilo32(0xD2511F53u, c0, &hi0, &lo0);
    mulhilo32(0xCD9E8D57u, c2, &hi1, &lo1);
    uint32_t n0 = hi1 ^ c1 ^ k0, n1 = lo1, n2 = hi0 ^ c3 ^ k1, n3 = lo0;
    c0 = n0; c1 = n1; c2 = n2; c3 = n3;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  out[0] = c0; out[1] = c1; out[2] = c2; out[3] = c3;
}

/* Two N(0,1) draws from one Philox block: 53-bit uniforms in (0,1), Box-Muller. */
static inline void gauss2(uint32_t key0, uint32_t key1, uint32_t c0, uint32_t c1,
                          double *z0, double *z1) {
  uint32_t ctr[4] = {c0, c1, 0u, 0u}, key[2] = {key0, key1}, o[4];
  ksg_philox4x32_10(ctr, key, o);
  uint64_t a = ((uint64_t)o[0] << 21) ^ (uint64_t)(o[1] >> 11);
  uint64_t b = ((uint64_t)o[2] << 21) ^ (uint64_t)(o[3] >> 11);
  a &= ((1ull << 53) - 1); b &= ((1ull << 53) - 1);
  double u1 = ((double)a + 0.5) * (1.0 / 9007199254740992.0);
  double u2 = ((double)b + 0.5) * (1.0 / 9007199254740992.0);
  double rad = sqrt(-2.0 * log(u1));
  double ang = 6.283185307179586476925286766559 * u2;
  *z0 = rad * cos(ang);
  *z1 = rad * sin(ang);
}

/* Uniform doubles in (0,1), four per call of gen; used for labels and sets. */
void ksg_uniform(uint64_t seed, uint32_t stream, int64_t count, double *out) {
  uint32_t key[2] = {(uint32_t)seed ^ (uint32_t)(seed >> 32), stream};
  for (int64_t q = 0; q < count; q += 2) {
    uint32_t ctr[4] = {(uint32_t)(q >> 1), (uint32_t)((uint64_t)q >> 33), 0xA5A5A5A5u, 0u};
    uint32_t o[4];
    ksg_philox4x32_10(ctr, key, o);
    uint64_t a = (((uint64_t)o[0] << 21) ^ (o[1] >> 11)) & ((1ull << 53) - 1);
    uint64_t b = (((uint64_t)o[2] << 21) ^ (o[3] >> 11)) & ((1ull << 53) - 1);
    out[q] = ((double)a + 0.5) * (1.0 / 9007199254740992.0);
    if (q + 1 < count) out[q + 1] = ((double)b + 0.5) * (1.0 / 9007199254740992.0);
  }
}

/* Standard normals, stream-keyed, for noise vectors. */
void ksg_normal(uint64_t seed, uint32_t stream, int64_t count, double *out) {
  uint32_t k0 = (uint32_t)seed ^ (uint32_t)(seed >> 32);
  for (int64_t q = 0; q < count; q += 2) {
    double z0, z1;
    gauss2(k0, stream, (uint32_t)(q >> 1), 0x5EEDu + (uint32_t)((uint64_t)q >> 33), &z0, &z1);
    out[q] = z0;
    if (q + 1 < count) out[q + 1] = z1;
  }
}

/* One AR(1) row in double. */
static void make_row(int64_t i, int64_t p, double r, uint32_t k0, double *row) {
  const uint32_t stream = 1u;
  double s = sqrt(1.0 - r * r);
  double prev = 0.0;
  for (int64_t j = 0; j < p; j += 2) {
    double z0, z1;
    gauss2(k0, stream, (uint32_t)(j >> 1), (uint32_t)i, &z0, &z1);
    double x0 = (j == 0) ? z0 : r * prev + s * z0;
    row[j] = x0;
    prev = x0;
    if (j + 1 < p) {
      double x1 = r * prev + s * z1;
      row[j + 1] = x1;
      prev = x1;
    }
  }
}

/* round-to-nearest-even float -> bfloat16 bits */
static inline uint16_t f32_to_bf16(float f) {
  uint32_t u;
  memcpy(&u, &f, 4);
  if ((u & 0x7f800000u) == 0x7f800000u) return (uint16_t)(u >> 16);
  uint32_t lsb = (u >> 16) & 1u;
  u += 0x7fffu + lsb;
  return (uint16_t)(u >> 16);
}

typedef struct {
  int64_t n, p; double r; uint32_t k0;
  int out_dtype; void *X;
  const double *mean, *scale;
  double *blk_sum, *blk_sq;      /* [nblocks][p] column partials (pass 1) */
  const double *beta_star; double *xb;
  int64_t next_block, nblocks;
  int pass;
  pthread_mutex_t mu;
} job_t;

static void *worker(void *arg) {
  job_t *J = (job_t *)arg;
  int64_t p = J->p;
  double *row = (double *)malloc((size_t)p * sizeof(double));
  for (;;) {
    pthread_mutex_lock(&J->mu);
    int64_t b = J->next_block++;
    pthread_mutex_unlock(&J->mu);
    if (b >= J->nblocks) break;
    int64_t i0 = b * KSG_ROWS_PER_BLOCK;
    int64_t i1 = i0 + KSG_ROWS_PER_BLOCK;
    if (i1 > J->n) i1 = J->n;
    if (J->pass == 1) {
      double *cs = J->blk_sum + b * p, *cq = J->blk_sq + b * p;
      memset(cs, 0, (size_t)p * sizeof(double));
      memset(cq, 0, (size_t)p * sizeof(double));
      for (int64_t i = i0; i < i1; ++i) {
        make_row(i, p, J->r, J->k0, row);
        for (int64_t j = 0; j < p; ++j) { cs[j] += row[j]; cq[j] += row[j] * row[j]; }
      }
    } else {
      for (int64_t i = i0; i < i1; ++i) {
        make_row(i, p, J->r, J->k0, row);
        double acc = 0.0;
        for (int64_t j = 0; j < p; ++j) {
          double x = (row[j] - J->mean[j]) * J->scale[j];
          if (J->out_dtype == 0) {
            ((double *)J->X)[i * p + j] = x;
          } else if (J->out_dtype == 1) {
            float f = (float)x;
            ((float *)J->X)[i * p + j] = f;
            x = (double)f;
          } else {
            uint16_t h = f32_to_bf16((float)x);
            ((uint16_t *)J->X)[i * p + j] = h;
            uint32_t u = (uint32_t)h << 16;
            float f;
            memcpy(&f, &u, 4);
            x = (double)f;
          }
          if (J->beta_star && J->beta_star[j] != 0.0) acc += x * J->beta_star[j];
        }
        if (J->xb) J->xb[i] = acc;
      }
    }
  }
  free(row);
  return NULL;
}

/* X (n x p row-major) in out_dtype (0 f64, 1 f32, 2 bf16 bits); the stored
 * values are the standardised doubles rounded to that type.  If beta_star and
 * xb are given, xb = X_stored beta_star in double. */
int ksg_make_X(int64_t n, int64_t p, double r, uint64_t seed, int out_dtype, void *X,
               const double *beta_star, double *xb, int nthreads) {
  if (n <= 0 || p <= 0 || r < 0.0 || r >= 1.0) return -1;
  if (nthreads < 1) nthreads = 1;
  job_t J;
  memset(&J, 0, sizeof J);
  J.n = n; J.p = p; J.r = r;
  J.k0 = (uint32_t)seed ^ (uint32_t)(seed >> 32);
  J.out_dtype = out_dtype; J.X = X;
  J.nblocks = (n + KSG_ROWS_PER_BLOCK - 1) / KSG_ROWS_PER_BLOCK;
  J.blk_sum = (double *)malloc((size_t)(J.nblocks * p) * sizeof(double));
  J.blk_sq = (double *)malloc((size_t)(J.nblocks * p) * sizeof(double));
  double *mean = (double *)calloc((size_t)p, sizeof(double));
  double *scale = (double *)calloc((size_t)p, sizeof(double));
  if (!J.blk_sum || !J.blk_sq || !mean || !scale) return -2;
  pthread_mutex_init(&J.mu, NULL);
  pthread_t *th = (pthread_t *)malloc((size_t)nthreads * sizeof(pthread_t));
  for (int pass = 1; pass <= 2; ++pass) {
    J.pass = pass;
    J.next_block = 0;
    if (pass == 2) {
      J.mean = mean; J.scale = scale;
      J.beta_star = beta_star; J.xb = xb;
    }
    for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, worker, &J);
    for (int t = 0; t < nthreads; ++t) pthread_join(th[t], NULL);
    if (pass == 1) {
      for (int64_t j = 0; j < p; ++j) {
        double s = 0.0, q = 0.0;
        for (int64_t b = 0; b < J.nblocks; ++b) { s += J.blk_sum[b * p + j]; q += J.blk_sq[b * p + j]; }
        double m = s / (double)n;
        double ss = q - (double)n * m * m;           /* sum (x - m)^2 */
        mean[j] = m;
        scale[j] = (ss > 0.0) ? sqrt((double)n / ss) : 1.0;
      }
    }
  }
  pthread_mutex_destroy(&J.mu);
  free(th); free(J.blk_sum); free(J.blk_sq); free(mean); free(scale);
  return 0;
}
