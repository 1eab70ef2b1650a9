/*
 * or_philox.c -- the oracle's core engine and base conversions.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * Core engine (Sec. 2.2: "the existence of at least a vectorized RNG for
 * uniform distribution"; Sec. 3 item 2, alternative core RNGs): Philox4x32
 * with 10 rounds as published by Salmon et al. (SC'11).  Each round maps the
 * counter (c0,c1,c2,c3) with key (k0,k1) to
 *     (hi(M1*c2) ^ c1 ^ k0,  lo(M1*c2),  hi(M0*c0) ^ c3 ^ k1,  lo(M0*c0))
 * and the key is bumped by the Weyl constants (W0, W1) between rounds.
 *
 * Base conversions (Sec. 2.1 key concept 2, reducible distributions), for a
 * 32-bit word w and k = w >> 8 (its top 24 bits):
 *     U  = k * 2^-24          in [0, 1)   (uniform buffer, U[a,b) transform)
 *     U' = (k + 1) * 2^-24    in (0, 1]   (wherever a logarithm is taken)
 *     U64 = ((wa >> 5) * 2^26 + (wb >> 6)) * 2^-53 in [0, 1)
 *     Gaussian pair from (w0, w1): r = sqrt(-2 ln U'(w0)), a = 2 U(w1),
 *         (z_even, z_odd) = (r cos(pi a), r sin(pi a))      (Box-Muller)
 *     exponential: -ln U'(w)
 */
#include <math.h>
#include <stdint.h>

#include "oracle.h"

#define OR_M0 0xD2511F53u
#define OR_M1 0xCD9E8D57u
#define OR_W0 0x9E3779B9u
#define OR_W1 0xBB67AE85u

void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c0 = ctr[0], c1 = ctr[1], c2 = ctr[2], c3 = ctr[3];
  uint32_t k0 = key[0], k1 = key[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += OR_W0;
      k1 += OR_W1;
    }
    uint64_t p0 = (uint64_t)OR_M0 * (uint64_t)c0;
    uint64_t p1 = (uint64_t)OR_M1 * (uint64_t)c2;
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    c0 = hi1 ^ c1 ^ k0;
    c1 = lo1;
    c2 = hi0 ^ c3 ^ k1;
    c3 = lo0;
  }
  out[0] = c0;
  out[1] = c1;
  out[2] = c2;
  out[3] = c3;
}

static void or_block(uint64_t seed, uint32_t domain, uint32_t stream, uint64_t block,
                     uint32_t w[4]) {
  uint32_t ctr[4] = {(uint32_t)block, domain, stream, (uint32_t)(block >> 32)};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  or_philox4x32_10(ctr, key, w);
}

void or_philox_words(uint64_t seed, uint32_t domain, uint32_t stream, uint64_t first_block,
                     uint64_t n_blocks, uint32_t *out) {
  for (uint64_t b = 0; b < n_blocks; ++b) or_block(seed, domain, stream, first_block + b, out + 4 * b);
}

static double or_u(uint32_t w) { return (double)(w >> 8) * 0x1p-24; }
static double or_uopen(uint32_t w) { return (double)((w >> 8) + 1u) * 0x1p-24; }

/* the raw word an element "owns": its own slot for U/N/E, the first of its
 * pair for U64 */
uint32_t or_elem_word(uint64_t seed, uint32_t domain, uint32_t stream, uint64_t j) {
  uint32_t w[4];
  if (domain == OR_DOM_U64) {
    or_block(seed, domain, stream, j / 2, w);
    return w[2 * (j % 2)];
  }
  or_block(seed, domain, stream, j / 4, w);
  return w[j % 4];
}

double or_elem_value(uint64_t seed, uint32_t domain, uint32_t stream, uint64_t j) {
  uint32_t w[4];
  switch (domain) {
  case OR_DOM_U:
    or_block(seed, domain, stream, j / 4, w);
    return or_u(w[j % 4]);
  case OR_DOM_E:
    or_block(seed, domain, stream, j / 4, w);
    return -or_log(or_uopen(w[j % 4]));
  case OR_DOM_N: {
    or_block(seed, domain, stream, j / 4, w);
    unsigned pair = (unsigned)(j % 4) / 2;
    double r = sqrt(-2.0 * or_log(or_uopen(w[2 * pair])));
    double s, c;
    or_sincospi(2.0 * or_u(w[2 * pair + 1]), &s, &c);
    return (j % 2 == 0) ? r * c : r * s;
  }
  case OR_DOM_U64: {
    or_block(seed, domain, stream, j / 2, w);
    uint32_t wa = w[2 * (j % 2)], wb = w[2 * (j % 2) + 1];
    return ((double)(wa >> 5) * 67108864.0 + (double)(wb >> 6)) * 0x1p-53;
  }
  default:
    return NAN;
  }
}

void or_elem_values(uint64_t seed, uint32_t domain, uint32_t stream, uint64_t j0, uint64_t n,
                    double *out, uint32_t *words) {
  for (uint64_t i = 0; i < n; ++i) {
    if (out) out[i] = or_elem_value(seed, domain, stream, j0 + i);
    if (words) words[i] = or_elem_word(seed, domain, stream, j0 + i);
  }
}
