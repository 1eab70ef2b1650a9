/*
 * or_internal.h -- the oracle's buffered RNG object (Sec. 2.2 class members),
 * shared by the oracle's own source files only.  TEST INFRASTRUCTURE ONLY.
 */
#ifndef BRNG_OR_INTERNAL_H
#define BRNG_OR_INTERNAL_H

#include <stdint.h>

#include "oracle.h"

typedef struct {
  uint32_t length;  /* buffer_length                                   */
  uint32_t counter; /* buffer_counter: index of the next element        */
  uint64_t first;   /* element index (in the domain) held by buffer[0]  */
  double *buffer;   /* buffer: converted deviates                        */
  uint32_t *words;  /* the raw word each buffered element owns           */
} or_buffer;

typedef struct {
  uint64_t seed;   /* engine state: key                               */
  uint32_t stream; /* engine state: stream id (counter word 2)        */
  or_buffer buf[OR_NDOM];
} or_batchrng;

void or_batchrng_init(or_batchrng *g, uint64_t seed, uint32_t stream, const uint64_t *start,
                      const uint32_t *length);
void or_batchrng_free(or_batchrng *g, uint64_t *end);
double or_get(or_batchrng *g, uint32_t dom, uint32_t *word);
double or_get_uniform(or_batchrng *g, uint32_t *word);
double or_get_uniform_open(or_batchrng *g);
double or_get_log_uniform(or_batchrng *g);
double or_get_gaussian(or_batchrng *g, uint32_t *word);
double or_get_exponential(or_batchrng *g, uint32_t *word);
double or_get_u64(or_batchrng *g);
double or_get_gamma(or_batchrng *g, float alpha, uint32_t *first_word, double *log_y,
                    int *rejected, double *cond);
double or_poisson_ptrs(or_batchrng *g, double lam, uint32_t *word, int *rejected);
double or_binomial_btrd(or_batchrng *g, double n, double p, uint32_t *word, int *rejected);
void or_dirichlet_row(or_batchrng *comp, uint32_t K, const float *alpha, double *out,
                      double *l, double *cond, int *n_domain, int *n_reject);

#endif
