/*
 * or_gibbs.c -- Markov-dependent consumers of the buffered RNG object, in
 * FP64, and a thread harness over chain ranges for timing.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Every chain is one stream (one BatchRNG object, Sec. 2.2) whose id is the
 * global chain id; chains never share draws, so a chain range split across
 * threads (or devices) gives identical results.
 *
 *  - triangle (Sec. 1, Eq. 1 and Fig. 1): start (x, y) as given, then per
 *    sweep x <- U[0, 1-y), y <- U[0, 1-x), each uniform a 53-bit FP64 draw.
 *  - normal-gamma: observations with sufficient statistics (n, xbar,
 *    S = sum (x - xbar)^2); priors mu ~ N(mu0, 1/prec0), tau ~ Gamma(a0, b0)
 *    (rate).  Per sweep tau | mu ~ Gamma(a0 + n/2, b0 + SS/2) with
 *    SS = S + n (xbar - mu)^2, then mu | tau ~ N((prec0 mu0 + tau n xbar)/P,
 *    1/P), P = prec0 + n tau.
 *  - LDA document-topic step (Sec. 1, LDA paragraph and footnote): per sweep
 *    theta_d ~ Dirichlet(alpha_d), every component its own stream.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"
#include "or_internal.h"

int or_gibbs_triangle(uint64_t seed, uint64_t chain_offset, uint32_t n_chains, uint32_t n_sweeps,
                      double *xy, uint64_t *pos, double *mom, uint32_t buf_len) {
  if (buf_len == 0 || chain_offset + n_chains > 0x100000000ull) return OR_EINVAL;
  for (uint32_t c = 0; c < n_chains; ++c) {
    or_batchrng g;
    uint64_t start[OR_NDOM] = {0, 0, 0, 0, pos[c]};
    uint32_t len[OR_NDOM] = {0, 0, 0, 0, buf_len};
    or_batchrng_init(&g, seed, (uint32_t)(chain_offset + c), start, len);
    double x = xy[2 * c], y = xy[2 * c + 1];
    double *m = mom + 5 * (uint64_t)c;
    for (uint32_t it = 0; it < n_sweeps; ++it) {
      x = (1.0 - y) * or_get_u64(&g);
      y = (1.0 - x) * or_get_u64(&g);
      m[0] += x;
      m[1] += y;
      m[2] += x * x;
      m[3] += y * y;
      m[4] += x * y;
    }
    xy[2 * c] = x;
    xy[2 * c + 1] = y;
    uint64_t end[OR_NDOM];
    or_batchrng_free(&g, end);
    pos[c] = end[OR_DOM_U64];
  }
  return OR_OK;
}

int or_gibbs_normal_gamma(uint64_t seed, uint64_t chain_offset, uint32_t n_chains,
                          uint32_t n_sweeps, const float *prior, const float *nobs,
                          const float *xbar, const float *sc, double *state, uint64_t *pos,
                          double *mom, double *trace, uint32_t buf_len) {
  if (buf_len == 0 || chain_offset + n_chains > 0x100000000ull) return OR_EINVAL;
  const float a0 = prior[0];
  const double b0 = prior[1], mu0 = prior[2], prec0 = prior[3];
  int n_reject = 0;
  for (uint32_t c = 0; c < n_chains; ++c) {
    or_batchrng g;
    uint64_t start[OR_NDOM] = {pos[2 * c + 1], pos[2 * c], 0, 0, 0};
    uint32_t len[OR_NDOM] = {buf_len, buf_len, 0, 0, 0};
    or_batchrng_init(&g, seed, (uint32_t)(chain_offset + c), start, len);
    const double n = nobs[c], xb = xbar[c], S = sc[c];
    /* the Gamma shape is formed in FP32, as the parameter array of a
     * varying-parameter draw would hold it */
    const float shape = a0 + 0.5f * nobs[c];
    double mu = state[2 * c], tau = state[2 * c + 1];
    double *m = mom + 4 * (uint64_t)c;
    for (uint32_t it = 0; it < n_sweeps; ++it) {
      double dm = xb - mu;
      double SS = S + n * dm * dm;
      int rej = 0;
      double kappa = 0.0;
      double G = or_get_gamma(&g, shape, NULL, NULL, &rej, &kappa);
      n_reject += rej;
      tau = G / (b0 + 0.5 * SS);
      double P = prec0 + n * tau;
      double mean = (prec0 * mu0 + tau * n * xb) / P;
      double z = or_get_gaussian(&g, NULL);
      mu = mean + z / sqrt(P);
      m[0] += mu;
      m[1] += tau;
      m[2] += mu * mu;
      m[3] += tau * tau;
      if (trace) {
        double *tr = trace + 5 * ((uint64_t)c * n_sweeps + it);
        tr[0] = G;
        tr[1] = kappa;
        tr[2] = z;
        tr[3] = tau;
        tr[4] = mu;
      }
    }
    state[2 * c] = mu;
    state[2 * c + 1] = tau;
    uint64_t end[OR_NDOM];
    or_batchrng_free(&g, end);
    pos[2 * c] = end[OR_DOM_N];
    pos[2 * c + 1] = end[OR_DOM_U];
  }
  return n_reject ? OR_EREJECT : OR_OK;
}

int or_gibbs_lda(uint64_t seed, uint64_t doc_offset, uint32_t n_docs, uint32_t K,
                 uint32_t n_sweeps, const float *alpha, double *theta, double *logs,
                 double *cond, uint64_t *pos, double *mom, double *trace, uint32_t buf_len) {
  if (buf_len == 0 || K == 0 || (doc_offset + n_docs) * (uint64_t)K > 0x100000000ull)
    return OR_EINVAL;
  int n_domain = 0, n_reject = 0;
  or_batchrng *comp = (or_batchrng *)malloc(sizeof(or_batchrng) * K);
  double *l = (double *)malloc(sizeof(double) * K);
  for (uint32_t d = 0; d < n_docs; ++d) {
    for (uint32_t k = 0; k < K; ++k) {
      uint64_t idx = (uint64_t)d * K + k;
      uint64_t start[OR_NDOM] = {pos[2 * idx + 1], pos[2 * idx], 0, 0, 0};
      uint32_t len[OR_NDOM] = {buf_len, buf_len, 0, 0, 0};
      or_batchrng_init(&comp[k], seed, (uint32_t)((doc_offset + d) * K + k), start, len);
    }
    const float *a = alpha + (uint64_t)d * K;
    double *th = theta + (uint64_t)d * K;
    double *m = mom + (uint64_t)d * K;
    for (uint32_t k = 0; k < K; ++k) l[k] = NAN;
    for (uint32_t it = 0; it < n_sweeps; ++it) {
      double *cd = cond ? cond + (uint64_t)d * K : NULL;
      or_dirichlet_row(comp, K, a, th, l, cd, &n_domain, &n_reject);
      for (uint32_t k = 0; k < K; ++k) m[k] += th[k];
      if (trace) {
        double *tr = trace + 2 * ((uint64_t)d * n_sweeps + it) * K;
        for (uint32_t k = 0; k < K; ++k) {
          tr[2 * k] = l[k];
          tr[2 * k + 1] = cd ? cd[k] : 0.0;
        }
      }
    }
    if (logs)
      for (uint32_t k = 0; k < K; ++k) logs[(uint64_t)d * K + k] = l[k];
    for (uint32_t k = 0; k < K; ++k) {
      uint64_t idx = (uint64_t)d * K + k;
      uint64_t end[OR_NDOM];
      or_batchrng_free(&comp[k], end);
      pos[2 * idx] = end[OR_DOM_N];
      pos[2 * idx + 1] = end[OR_DOM_U];
    }
  }
  free(comp);
  free(l);
  if (n_domain) return OR_EDOMAIN;
  return n_reject ? OR_EREJECT : OR_OK;
}

/* ---- thread harness: contiguous chain ranges, one per thread ---------- */

typedef struct {
  int model;
  uint64_t seed, offset;
  uint32_t n, K, sweeps, buf_len;
  const float *prior, *nobs, *xbar, *sc, *alpha;
  double *a, *b; /* model outputs */
  double *logs, *cond, *trace;
  uint64_t *pos;
  int status;
  /* mixed stream */
  uint32_t S, s0, s1;
  uint64_t n_draws;
  const uint8_t *tag;
  const float *p0, *p1;
  uint32_t *words;
} or_job;

static void *or_run(void *arg) {
  or_job *j = (or_job *)arg;
  switch (j->model) {
  case 0:
    j->status = or_gibbs_triangle(j->seed, j->offset, j->n, j->sweeps, j->a, j->pos, j->b,
                                  j->buf_len);
    break;
  case 1:
    j->status = or_gibbs_normal_gamma(j->seed, j->offset, j->n, j->sweeps, j->prior, j->nobs,
                                      j->xbar, j->sc, j->a, j->pos, j->b, j->trace, j->buf_len);
    break;
  case 2:
    j->status = or_gibbs_lda(j->seed, j->offset, j->n, j->K, j->sweeps, j->alpha, j->a,
                             j->logs, j->cond, j->pos, j->b, j->trace, j->buf_len);
    break;
  default:
    j->status = or_mixed_streams(j->seed, j->S, j->s0, j->s1, j->pos, j->n_draws, j->tag, j->p0,
                                 j->p1, j->a, j->words, j->cond, j->buf_len);
  }
  return NULL;
}

static int or_spawn(or_job *jobs, int nthreads) {
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, or_run, &jobs[t]);
  int status = OR_OK;
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(th[t], NULL);
    if (jobs[t].status != OR_OK && status == OR_OK) status = jobs[t].status;
  }
  free(th);
  return status;
}

static void range_of(uint32_t n, int nthreads, int t, uint32_t *b, uint32_t *e) {
  uint64_t lo = (uint64_t)n * t / nthreads, hi = (uint64_t)n * (t + 1) / nthreads;
  *b = (uint32_t)lo;
  *e = (uint32_t)hi;
}

int or_gibbs_triangle_mt(uint64_t seed, uint64_t chain_offset, uint32_t n_chains,
                         uint32_t n_sweeps, double *xy, uint64_t *pos, double *mom,
                         uint32_t buf_len, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  or_job *jobs = (or_job *)calloc(nthreads, sizeof(or_job));
  for (int t = 0; t < nthreads; ++t) {
    uint32_t b, e;
    range_of(n_chains, nthreads, t, &b, &e);
    jobs[t] = (or_job){.model = 0, .seed = seed, .offset = chain_offset + b, .n = e - b,
                       .sweeps = n_sweeps, .buf_len = buf_len, .a = xy + 2 * (uint64_t)b,
                       .b = mom + 5 * (uint64_t)b, .pos = pos + b};
  }
  int st = or_spawn(jobs, nthreads);
  free(jobs);
  return st;
}

int or_gibbs_normal_gamma_mt(uint64_t seed, uint64_t chain_offset, uint32_t n_chains,
                             uint32_t n_sweeps, const float *prior, const float *nobs,
                             const float *xbar, const float *sc, double *state, uint64_t *pos,
                             double *mom, double *trace, uint32_t buf_len, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  or_job *jobs = (or_job *)calloc(nthreads, sizeof(or_job));
  for (int t = 0; t < nthreads; ++t) {
    uint32_t b, e;
    range_of(n_chains, nthreads, t, &b, &e);
    jobs[t] = (or_job){.model = 1, .seed = seed, .offset = chain_offset + b, .n = e - b,
                       .sweeps = n_sweeps, .buf_len = buf_len, .prior = prior,
                       .nobs = nobs + b, .xbar = xbar + b, .sc = sc + b,
                       .a = state + 2 * (uint64_t)b, .b = mom + 4 * (uint64_t)b,
                       .pos = pos + 2 * (uint64_t)b,
                       .trace = trace ? trace + 5 * (uint64_t)b * n_sweeps : NULL};
  }
  int st = or_spawn(jobs, nthreads);
  free(jobs);
  return st;
}

int or_gibbs_lda_mt(uint64_t seed, uint64_t doc_offset, uint32_t n_docs, uint32_t K,
                    uint32_t n_sweeps, const float *alpha, double *theta, double *logs,
                    double *cond, uint64_t *pos, double *mom, double *trace, uint32_t buf_len,
                    int nthreads) {
  if (nthreads < 1) nthreads = 1;
  or_job *jobs = (or_job *)calloc(nthreads, sizeof(or_job));
  for (int t = 0; t < nthreads; ++t) {
    uint32_t b, e;
    range_of(n_docs, nthreads, t, &b, &e);
    uint64_t o = (uint64_t)b * K;
    jobs[t] = (or_job){.model = 2, .seed = seed, .offset = doc_offset + b, .n = e - b, .K = K,
                       .sweeps = n_sweeps, .buf_len = buf_len, .alpha = alpha + o,
                       .a = theta + o, .b = mom + o, .pos = pos + 2 * o,
                       .logs = logs ? logs + o : NULL, .cond = cond ? cond + o : NULL,
                       .trace = trace ? trace + 2 * o * n_sweeps : NULL};
  }
  int st = or_spawn(jobs, nthreads);
  free(jobs);
  return st;
}

int or_mixed_mt(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const uint8_t *tag,
                const float *p0, const float *p1, double *out, uint32_t *words, double *cond,
                uint32_t buf_len, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  or_job *jobs = (or_job *)calloc(nthreads, sizeof(or_job));
  for (int t = 0; t < nthreads; ++t) {
    uint32_t b, e;
    range_of(S, nthreads, t, &b, &e);
    jobs[t] = (or_job){.model = 3, .seed = seed, .S = S, .s0 = b, .s1 = e, .n_draws = n,
                       .tag = tag, .p0 = p0, .p1 = p1, .a = out, .words = words, .pos = pos,
                       .buf_len = buf_len, .cond = cond};
  }
  int st = or_spawn(jobs, nthreads);
  free(jobs);
  return st;
}
