/*
 * or_batchrng.c -- the paper's buffered RNG object and the varying-parameter
 * distributions built on it, in FP64.  TEST INFRASTRUCTURE ONLY (oracle.h).
 *
 * The object follows Sec. 2.2 member for member: per reducible distribution
 * a buffer_length, a buffer and a buffer_counter; the constructor fills every
 * buffer; a Get* call refills its buffer from the core engine when the
 * counter has reached the end, resets the counter, and returns
 * buffer[counter++].  Irreducible distributions (Gamma, Laplace, Weibull) are
 * composed from the reducible Get* calls (Sec. 2.2, Sec. 2.1 key concept 1).
 *
 * Readings where the paper is silent (Gamma source withheld, Sec. 3 note;
 * Laplace/Weibull formulas not given, Sec. 2.2):
 *   Gamma(alpha, 1): Marsaglia & Tsang (2000).  a = alpha (alpha >= 1) or
 *     alpha + 1 (alpha < 1); d = a - 1/3; c = 1/sqrt(9d).  Each attempt takes
 *     one Gaussian z; t = 1 + c z; if t <= 0 the attempt ends; otherwise
 *     v = t^3, one U' is taken and the attempt accepts iff
 *     ln U' < z^2/2 + d (1 - v + ln v), giving d v.  For alpha < 1 one more
 *     U' is taken after the accept and the result is d v U'^(1/alpha).
 *     After 64 attempts the draw is NaN (never reached in practice).
 *   Laplace(mu, b): one exponential e, then one uniform u; mu - b e if
 *     u < 1/2, else mu + b e.
 *   Weibull(k, lambda): lambda e^(1/k) for one exponential e.
 * An invalid parameter gives NaN and consumes nothing.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"
#include "or_internal.h"

/* ---- the buffered object --------------------------------------------- */

static void or_fill(or_batchrng *g, uint32_t dom) {
  or_buffer *b = &g->buf[dom];
  or_elem_values(g->seed, dom, g->stream, b->first, b->length, b->buffer, b->words);
}

void or_batchrng_init(or_batchrng *g, uint64_t seed, uint32_t stream, const uint64_t *start,
                      const uint32_t *length) {
  g->seed = seed;
  g->stream = stream;
  for (uint32_t d = 0; d < OR_NDOM; ++d) {
    or_buffer *b = &g->buf[d];
    b->length = length[d];
    b->counter = 0;
    b->first = start[d];
    b->buffer = b->length ? (double *)malloc(sizeof(double) * b->length) : NULL;
    b->words = b->length ? (uint32_t *)malloc(sizeof(uint32_t) * b->length) : NULL;
    if (b->length) or_fill(g, d);
  }
}

void or_batchrng_free(or_batchrng *g, uint64_t *end) {
  for (uint32_t d = 0; d < OR_NDOM; ++d) {
    or_buffer *b = &g->buf[d];
    if (end) end[d] = b->first + b->counter;
    free(b->buffer);
    free(b->words);
    b->buffer = NULL;
    b->words = NULL;
  }
}

double or_get(or_batchrng *g, uint32_t dom, uint32_t *word) {
  or_buffer *b = &g->buf[dom];
  if (b->length == 0) abort(); /* the caller disabled a domain it uses */
  if (b->counter == b->length) {
    b->first += b->length;
    b->counter = 0;
    or_fill(g, dom);
  }
  if (word) *word = b->words[b->counter];
  return b->buffer[b->counter++];
}

/* GetUniform returns U in [0,1); the open-left U' = U + 2^-24 is exact */
double or_get_uniform(or_batchrng *g, uint32_t *word) { return or_get(g, OR_DOM_U, word); }
double or_get_uniform_open(or_batchrng *g) { return or_get(g, OR_DOM_U, NULL) + 0x1p-24; }
double or_get_log_uniform(or_batchrng *g) { return or_log(or_get_uniform_open(g)); }
double or_get_gaussian(or_batchrng *g, uint32_t *word) { return or_get(g, OR_DOM_N, word); }
double or_get_exponential(or_batchrng *g, uint32_t *word) { return or_get(g, OR_DOM_E, word); }
double or_get_u64(or_batchrng *g) { return or_get(g, OR_DOM_U64, NULL); }

int or_mt_accept(double alpha, double z, double u_open) {
  double a = alpha < 1.0 ? alpha + 1.0 : alpha;
  double d = a - 1.0 / 3.0;
  double c = 1.0 / sqrt(9.0 * d);
  double t = 1.0 + c * z;
  if (t <= 0.0) return -1;
  double v = t * t * t;
  return or_log(u_open) < 0.5 * z * z + d * ((1.0 - v) + or_log(v));
}

double or_get_gamma(or_batchrng *g, float alpha_f, uint32_t *first_word, double *log_y,
                    int *rejected, double *cond) {
  double alpha = (double)alpha_f;
  double a = alpha < 1.0 ? alpha + 1.0 : alpha;
  double d = a - 1.0 / 3.0;
  double c = 1.0 / sqrt(9.0 * d);
  for (int attempt = 0; attempt < OR_GAMMA_MAX_ATTEMPTS; ++attempt) {
    uint32_t w;
    double z = or_get_gaussian(g, &w);
    if (attempt == 0 && first_word) *first_word = w;
    double t = 1.0 + c * z;
    if (t <= 0.0) continue;
    double v = t * t * t;
    double u = or_get_uniform_open(g);
    if (or_log(u) < 0.5 * z * z + d * ((1.0 - v) + or_log(v))) {
      double y = d * v;
      double ly = log(y);
      /* conditioning of d v in the Gaussian z (3 |c z| / t) and of the boost
       * exponent L = ln(u_b)/alpha: a diagnostic for FP32 comparisons */
      double kappa = 3.0 * fabs(c * z) / t;
      if (alpha < 1.0) {
        double ub = or_get_uniform_open(g);
        y = y * pow(ub, 1.0 / alpha);
        ly = ly + log(ub) / alpha;
        kappa += fabs(log(ub) / alpha);
      }
      if (log_y) *log_y = ly;
      if (cond) *cond = kappa;
      return y;
    }
  }
  if (rejected) *rejected = 1;
  if (log_y) *log_y = NAN;
  if (cond) *cond = 0.0;
  return NAN;
}

/* ---- bulk varying-parameter streams ----------------------------------- */

static int finite_f(float x) { return isfinite(x); }

/* open stream s positioned at pos[3s..3s+2] (U, N, E) with buffers of L */
static void open_stream(or_batchrng *g, uint64_t seed, uint32_t s, const uint64_t *pos3,
                        uint32_t L) {
  uint64_t start[OR_NDOM] = {pos3[0], pos3[1], pos3[2], 0, 0};
  uint32_t len[OR_NDOM] = {L, L, L, 0, 0};
  or_batchrng_init(g, seed, s, start, len);
}

static void close_stream(or_batchrng *g, uint64_t *pos3) {
  uint64_t end[OR_NDOM];
  or_batchrng_free(g, end);
  pos3[0] = end[0];
  pos3[1] = end[1];
  pos3[2] = end[2];
}

/* one draw of distribution `tag` with parameters (p0, p1); returns the value,
 * sets *word to the first raw word it consumed (0 if none), and counts
 * errors. */
static double draw_tagged(or_batchrng *g, unsigned tag, float p0, float p1, uint32_t *word,
                          double *cond, int *n_domain, int *n_reject) {
  uint32_t w = 0;
  double out = NAN, kappa = 0.0;
  switch (tag) {
  case 0: /* Uniform[a, b) = a + (b - a) U */
    if (finite_f(p0) && finite_f(p1) && p0 <= p1) {
      double u = or_get_uniform(g, &w);
      out = (double)p0 + ((double)p1 - (double)p0) * u;
    } else ++*n_domain;
    break;
  case 1: /* Normal(mu, sigma) = mu + sigma z */
    if (finite_f(p0) && finite_f(p1) && p1 > 0.0f) {
      double z = or_get_gaussian(g, &w);
      out = (double)p0 + (double)p1 * z;
    } else ++*n_domain;
    break;
  case 2: /* Exponential(rate lambda) = E / lambda */
    if (finite_f(p0) && p0 > 0.0f) {
      double e = or_get_exponential(g, &w);
      out = e / (double)p0;
    } else ++*n_domain;
    break;
  case 3: /* Gamma(alpha, 1) */
    if (finite_f(p0) && p0 > 0.0f) {
      int rej = 0;
      out = or_get_gamma(g, p0, &w, NULL, &rej, &kappa);
      if (rej) ++*n_reject;
    } else ++*n_domain;
    break;
  case 4: /* Laplace(mu, b) */
    if (finite_f(p0) && finite_f(p1) && p1 > 0.0f) {
      double e = or_get_exponential(g, &w);
      double u = or_get_uniform(g, NULL);
      out = u < 0.5 ? (double)p0 - (double)p1 * e : (double)p0 + (double)p1 * e;
    } else ++*n_domain;
    break;
  case 5: /* Weibull(shape k, scale lambda) = lambda E^(1/k) */
    if (finite_f(p0) && finite_f(p1) && p0 > 0.0f && p1 > 0.0f) {
      double e = or_get_exponential(g, &w);
      out = (double)p1 * pow(e, 1.0 / (double)p0);
      kappa = fabs(log(e) / (double)p0);
    } else ++*n_domain;
    break;
  case 6: /* Poisson(lambda): inversion of one U for small means, else PTRS */
    if (finite_f(p0) && p0 > 0.0f && p0 <= OR_POISSON_MAX_LAMBDA) {
      if (p0 <= OR_INVERSION_MAX_MEAN) {
        double u = or_get_uniform(g, &w);
        out = or_poisson_inv((double)p0, u);
      } else {
        int rej = 0;
        out = or_poisson_ptrs(g, (double)p0, &w, &rej);
        if (rej) ++*n_reject;
      }
    } else ++*n_domain;
    break;
  case 7: /* Binomial(n, p): inversion of one U for small means, else BTRD */
    if (finite_f(p0) && p0 >= 0.0f && p0 == floorf(p0) && p0 <= 16777216.0f && finite_f(p1) &&
        p1 >= 0.0f && p1 <= 1.0f) {
      if ((double)p0 * fmin((double)p1, 1.0 - (double)p1) <= OR_INVERSION_MAX_MEAN) {
        double u = or_get_uniform(g, &w);
        out = or_binomial_inv((double)p0, (double)p1, u);
      } else {
        int rej = 0;
        out = or_binomial_btrd(g, (double)p0, (double)p1, &w, &rej);
        if (rej) ++*n_reject;
      }
    } else ++*n_domain;
    break;
  default:
    ++*n_domain;
  }
  if (word) *word = w;
  if (cond) *cond = kappa;
  return out;
}

/* ---- large means: transformed rejection (Hormann 1993) ----------------- */
/*
 * Both samplers run in FP64 with the oracle's own log (or_log), IEEE sqrt,
 * floor and division, every operation in the order written and without
 * contraction; ln k! comes from or_lfact.  A sampler that runs out of
 * attempts (64, as the Gamma sampler; never seen) gives NaN.
 */

#define OR_HALF_LOG_2PI 0x1.d67f1c864beb5p-1 /* ln(2 pi) / 2 */

/* Stirling's series of ln Gamma(x), x >= 17, to the x^-7 term (the next term,
 * 1/(1188 x^9), is below 1e-14): (x - 1/2) ln x - x + ln(2 pi)/2
 * + 1/(12x) - 1/(360x^3) + 1/(1260x^5) - 1/(1680x^7). */
static double or_stirling_tail(double x) {
  const double inv = 1.0 / x;
  const double inv2 = inv * inv;
  return inv * (1.0 / 12.0 - inv2 * (1.0 / 360.0 - inv2 * (1.0 / 1260.0 - inv2 * (1.0 / 1680.0))));
}

/* ln k! for an integer k >= 0: the log of the exact product for k <= 15
 * (15! < 2^53), Stirling's series of ln Gamma(k + 1) above */
double or_lfact(double k) {
  if (k <= 15.0) {
    double f = 1.0;
    for (double i = 2.0; i <= k; i += 1.0) f = f * i;
    return or_log(f);
  }
  const double x = k + 1.0;
  return ((x - 0.5) * or_log(x) - x) + (OR_HALF_LOG_2PI + or_stirling_tail(x));
}

/* f_c(k) = ln k! - (k + 1/2) ln(k + 1) + (k + 1) - ln(2 pi)/2, the correction
 * term of Stirling's formula that BTRD uses */
static double or_stirling_fc(double k) {
  if (k <= 15.0) {
    const double x = k + 1.0;
    return ((or_lfact(k) - (k + 0.5) * or_log(x)) + x) - OR_HALF_LOG_2PI;
  }
  return or_stirling_tail(k + 1.0);
}

/* PTRS for Poisson(lam), lam >= 10 (here > 64): per attempt U from the U
 * domain [0, 1) (shifted by -1/2) and V = U' in (0, 1]; an attempt with
 * 1/2 - |U| = 0 is rejected (the transformation is unbounded there). */
double or_poisson_ptrs(or_batchrng *g, double lam, uint32_t *word, int *rejected) {
  const double slam = sqrt(lam);
  const double loglam = or_log(lam);
  const double b = 0.931 + 2.53 * slam;
  const double a = -0.059 + 0.02483 * b;
  const double inv_alpha = 1.1239 + 1.1328 / (b - 3.4);
  const double vr = 0.9277 - 3.6224 / (b - 2.0);
  for (int attempt = 0; attempt < OR_GAMMA_MAX_ATTEMPTS; ++attempt) {
    uint32_t w0;
    const double u = or_get_uniform(g, &w0) - 0.5;
    const double v = or_get_uniform_open(g);
    if (attempt == 0 && word) *word = w0;
    const double us = 0.5 - fabs(u);
    if (us == 0.0) continue;
    const double k = floor(((2.0 * a) / us + b) * u + lam + 0.43);
    if (us >= 0.07 && v <= vr) return k;
    if (k < 0.0 || (us < 0.013 && v > us)) continue;
    if ((or_log(v) + or_log(inv_alpha)) - or_log(a / (us * us) + b) <= ((-lam) + k * loglam) - or_lfact(k))
      return k;
  }
  *rejected = 1;
  return NAN;
}

/* BTRD for Binomial(n, p), n min(p, 1 - p) >= 10 (here > 64), on
 * p' = min(p, 1 - p) (n - k when p > 1/2).  Per attempt V = U' in (0, 1];
 * unless V <= 0.86 v_r, one more element: U from [0, 1) (shifted by -1/2)
 * when V >= v_r, else V' = U' v_r. */
double or_binomial_btrd(or_batchrng *g, double n, double p_in, uint32_t *word, int *rejected) {
  const int flip = p_in > 0.5;
  const double p = flip ? 1.0 - p_in : p_in;
  const double q = 1.0 - p;
  const double m = floor((n + 1.0) * p);
  const double r = p / q;
  const double nr = (n + 1.0) * r;
  const double npq = (n * p) * q;
  const double spq = sqrt(npq);
  const double b = 1.15 + 2.53 * spq;
  const double a = (-0.0873 + 0.0248 * b) + 0.01 * p;
  const double c = n * p + 0.5;
  const double alpha = (2.83 + 5.1 / b) * spq;
  const double vr = 0.92 - 4.2 / b;
  const double urvr = 0.86 * vr;
  for (int attempt = 0; attempt < OR_GAMMA_MAX_ATTEMPTS; ++attempt) {
    uint32_t w0;
    double v = or_get_uniform(g, &w0) + 0x1p-24; /* U' */
    if (attempt == 0 && word) *word = w0;
    double u, k;
    if (v <= urvr) {
      u = v / vr - 0.43;
      k = floor(((2.0 * a) / (0.5 - fabs(u)) + b) * u + c);
      return flip ? n - k : k;
    }
    if (v >= vr) {
      u = or_get_uniform(g, NULL) - 0.5;
    } else {
      u = v / vr - 0.93;
      u = (u < 0.0 ? -0.5 : 0.5) - u;
      v = or_get_uniform_open(g) * vr;
    }
    const double us = 0.5 - fabs(u);
    if (us == 0.0) continue;
    k = floor(((2.0 * a) / us + b) * u + c);
    if (k < 0.0 || k > n) continue;
    v = (v * alpha) / (a / (us * us) + b);
    const double km = fabs(k - m);
    if (km <= 15.0) { /* f(k)/f(m) by its recursion */
      double f = 1.0;
      if (m < k) {
        for (double i = m + 1.0; i <= k; i += 1.0) f = f * (nr / i - r);
      } else if (m > k) {
        for (double i = k + 1.0; i <= m; i += 1.0) v = v * (nr / i - r);
      }
      if (v <= f) return flip ? n - k : k;
      continue;
    }
    v = or_log(v); /* squeeze on the log scale */
    const double rho = (km / npq) * (((km / 3.0 + 0.625) * km + 1.0 / 6.0) / npq + 0.5);
    const double t = -(km * km) / (2.0 * npq);
    if (v < t - rho) return flip ? n - k : k;
    if (v > t + rho) continue;
    const double nm = (n - m) + 1.0;
    const double h = ((m + 0.5) * or_log((m + 1.0) / (r * nm)) + or_stirling_fc(m)) + or_stirling_fc(n - m);
    const double nk = (n - k) + 1.0;
    if (v <= (((h + (n + 1.0) * or_log(nm / nk)) + (k + 0.5) * or_log((nk * r) / (k + 1.0))) -
              or_stirling_fc(k)) - or_stirling_fc(n - k))
      return flip ? n - k : k;
  }
  *rejected = 1;
  return NAN;
}

double or_poisson_inv(double lambda, double u) {
  double p = or_exp(-lambda);
  double F = p;
  int k = 0;
  while (!(u < F) && k < OR_POISSON_MAX_K) {
    ++k;
    p = (p * lambda) / (double)k;
    if (p == 0.0) break; /* the tail underflowed: nothing left to add */
    F = F + p;
  }
  return (double)k;
}

double or_binomial_inv(double n, double p, double u) {
  const int flip = p > 0.5;
  const double q = flip ? 1.0 - p : p;
  double pk = or_exp(n * or_log(1.0 - q));
  const double r = q / (1.0 - q);
  double F = pk;
  int k = 0;
  while (!(u < F) && (double)k < n) {
    ++k;
    pk = (pk * (((n - (double)k) + 1.0) * r)) / (double)k;
    if (pk == 0.0) break; /* the tail underflowed: nothing left to add */
    F = F + pk;
  }
  return flip ? n - (double)k : (double)k;
}

static int status_of(int n_domain, int n_reject) {
  if (n_domain) return OR_EDOMAIN;
  if (n_reject) return OR_EREJECT;
  return OR_OK;
}

int or_mixed_streams(uint64_t seed, uint32_t S, uint32_t s_begin, uint32_t s_end, uint64_t *pos,
                     uint64_t n, const uint8_t *tag, const float *p0, const float *p1,
                     double *out, uint32_t *words, double *cond, uint32_t buf_len) {
  int n_domain = 0, n_reject = 0;
  if (S == 0 || buf_len == 0) return OR_EINVAL;
  for (uint32_t s = s_begin; s < s_end && s < S; ++s) {
    if ((uint64_t)s >= n) break;
    or_batchrng g;
    open_stream(&g, seed, s, pos + 3 * (uint64_t)s, buf_len);
    for (uint64_t i = s; i < n; i += S) {
      uint32_t w;
      double k;
      out[i] = draw_tagged(&g, tag[i], p0[i], p1 ? p1[i] : 0.0f, &w, &k, &n_domain, &n_reject);
      if (words) words[i] = w;
      if (cond) cond[i] = k;
    }
    close_stream(&g, pos + 3 * (uint64_t)s);
  }
  return status_of(n_domain, n_reject);
}

int or_mixed(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const uint8_t *tag,
             const float *p0, const float *p1, double *out, uint32_t *words, double *cond,
             uint32_t buf_len) {
  return or_mixed_streams(seed, S, 0, S, pos, n, tag, p0, p1, out, words, cond, buf_len);
}

/* single-distribution streams: the mixed stream with a constant tag */
static int single(unsigned tagv, uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n,
                  const float *p0, const float *p1, double *out, uint32_t *words, double *cond,
                  uint32_t buf_len) {
  int n_domain = 0, n_reject = 0;
  if (S == 0 || buf_len == 0) return OR_EINVAL;
  for (uint32_t s = 0; s < S && (uint64_t)s < n; ++s) {
    or_batchrng g;
    open_stream(&g, seed, s, pos + 3 * (uint64_t)s, buf_len);
    for (uint64_t i = s; i < n; i += S) {
      uint32_t w;
      double k;
      out[i] = draw_tagged(&g, tagv, p0[i], p1 ? p1[i] : 0.0f, &w, &k, &n_domain, &n_reject);
      if (words) words[i] = w;
      if (cond) cond[i] = k;
    }
    close_stream(&g, pos + 3 * (uint64_t)s);
  }
  return status_of(n_domain, n_reject);
}

int or_uniform(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *a,
               const float *b, double *out, uint32_t *words, uint32_t buf_len) {
  return single(0, seed, S, pos, n, a, b, out, words, NULL, buf_len);
}
/* U[a, b) in FP64 from the 53-bit U64 domain: Sec. 2.2's GetUniform at
 * double precision, a + (b - a) U64 with one U64 element per valid draw,
 * rounded as fma(b - a, U64, a): the difference rounded once, then the
 * product and sum rounded together (C99 fma, correctly rounded).
 * pos64[s] is stream s's U64 position (separate from its U, N, E positions).
 * Needs finite a <= b; otherwise NaN, word 0, nothing consumed. */
int or_uniform_f64(uint64_t seed, uint32_t S, uint64_t *pos64, uint64_t n, const double *a,
                   const double *b, double *out, uint32_t *words, uint32_t buf_len) {
  int n_domain = 0;
  for (uint32_t s = 0; s < S && (uint64_t)s < n; ++s) {
    or_batchrng g;
    uint64_t start[OR_NDOM] = {0, 0, 0, 0, pos64[s]};
    uint32_t len[OR_NDOM] = {0, 0, 0, 0, buf_len};
    or_batchrng_init(&g, seed, s, start, len);
    for (uint64_t i = s; i < n; i += S) {
      uint32_t w = 0;
      double v = NAN;
      if (isfinite(a[i]) && isfinite(b[i]) && a[i] <= b[i]) {
        const double u = or_get(&g, OR_DOM_U64, &w);
        v = fma(b[i] - a[i], u, a[i]);
      } else {
        ++n_domain;
      }
      out[i] = v;
      if (words) words[i] = w;
    }
    uint64_t end[OR_NDOM];
    or_batchrng_free(&g, end);
    pos64[s] = end[OR_DOM_U64];
  }
  return status_of(n_domain, 0);
}
int or_normal(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *mu,
              const float *sigma, double *out, uint32_t *words, uint32_t buf_len) {
  return single(1, seed, S, pos, n, mu, sigma, out, words, NULL, buf_len);
}
int or_exponential(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *lambda,
                   double *out, uint32_t *words, uint32_t buf_len) {
  return single(2, seed, S, pos, n, lambda, NULL, out, words, NULL, buf_len);
}
int or_gamma(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *alpha,
             double *out, uint32_t *words, double *cond, uint32_t buf_len) {
  return single(3, seed, S, pos, n, alpha, NULL, out, words, cond, buf_len);
}
int or_laplace(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *mu,
               const float *scale, double *out, uint32_t *words, uint32_t buf_len) {
  return single(4, seed, S, pos, n, mu, scale, out, words, NULL, buf_len);
}
int or_weibull(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *shape,
               const float *scale, double *out, uint32_t *words, double *cond, uint32_t buf_len) {
  return single(5, seed, S, pos, n, shape, scale, out, words, cond, buf_len);
}

int or_poisson(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *lambda,
               double *out, uint32_t *words, uint32_t buf_len) {
  return single(6, seed, S, pos, n, lambda, NULL, out, words, NULL, buf_len);
}
int or_binomial(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *trials,
                const float *prob, double *out, uint32_t *words, uint32_t buf_len) {
  return single(7, seed, S, pos, n, trials, prob, out, words, NULL, buf_len);
}

/* Dirichlet (Sec. 1 footnote): y_k ~ Gamma(alpha_k, 1), x_k = y_k / sum y.
 * The normalisation is taken on log y_k (x_k = exp(l_k - M) / sum exp(l_j - M),
 * M = max l), the same quotient without underflow of tiny y_k. */
void or_dirichlet_row(or_batchrng *comp, uint32_t K, const float *alpha, double *out,
                      double *scratch_l, double *cond, int *n_domain, int *n_reject) {
  for (uint32_t k = 0; k < K; ++k) {
    if (!(finite_f(alpha[k]) && alpha[k] > 0.0f)) {
      ++*n_domain;
      for (uint32_t j = 0; j < K; ++j) out[j] = NAN;
      return;
    }
  }
  int rej = 0;
  for (uint32_t k = 0; k < K; ++k)
    or_get_gamma(&comp[k], alpha[k], NULL, &scratch_l[k], &rej, cond ? &cond[k] : NULL);
  if (rej) {
    ++*n_reject;
    for (uint32_t j = 0; j < K; ++j) out[j] = NAN;
    return;
  }
  double M = scratch_l[0];
  for (uint32_t k = 1; k < K; ++k) M = scratch_l[k] > M ? scratch_l[k] : M;
  double sum = 0.0;
  for (uint32_t k = 0; k < K; ++k) sum += exp(scratch_l[k] - M);
  for (uint32_t k = 0; k < K; ++k) out[k] = exp(scratch_l[k] - M) / sum;
}

int or_dirichlet(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n_rows, uint32_t K,
                 const float *alpha, double *out, double *logs, double *cond, uint32_t buf_len) {
  if (S == 0 || K == 0 || S % K != 0 || buf_len == 0) return OR_EINVAL;
  uint32_t R = S / K;
  int n_domain = 0, n_reject = 0;
  or_batchrng *comp = (or_batchrng *)malloc(sizeof(or_batchrng) * K);
  double *l = (double *)malloc(sizeof(double) * K);
  for (uint32_t r = 0; r < R && (uint64_t)r < n_rows; ++r) {
    for (uint32_t k = 0; k < K; ++k)
      open_stream(&comp[k], seed, r * K + k, pos + 3 * ((uint64_t)r * K + k), buf_len);
    for (uint64_t i = r; i < n_rows; i += R) {
      for (uint32_t k = 0; k < K; ++k) l[k] = NAN;
      or_dirichlet_row(comp, K, alpha + i * K, out + i * K, l, cond ? cond + i * K : NULL,
                       &n_domain, &n_reject);
      if (logs)
        for (uint32_t k = 0; k < K; ++k) logs[i * K + k] = l[k];
    }
    for (uint32_t k = 0; k < K; ++k) close_stream(&comp[k], pos + 3 * ((uint64_t)r * K + k));
  }
  free(comp);
  free(l);
  return status_of(n_domain, n_reject);
}
