/*
 * or_math.c -- FP64 natural log and sin/cos of pi*a for the oracle.
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The Gamma sampler's accept/reject decision (Sec. 2.2 "GetGamma", taken
 * here as Marsaglia-Tsang) depends on logarithms, and the Gaussian buffer on
 * a logarithm and sin/cos.  Library log/sin differ by an ulp between C
 * libraries and devices, so the oracle fixes its own versions, each a plain
 * textbook method with a fixed number of terms and a fixed order of IEEE
 * operations.  This file must be compiled without floating-point contraction
 * (-ffp-contract=off) and without -ffast-math.
 *
 * log:  x = m * 2^e with m in [sqrt(1/2), sqrt(2)); s = (m-1)/(m+1);
 *       ln m = 2 atanh s = 2 (s + s^3/3 + s^5/5 + ...), series through s^25
 *       (|s| <= 0.1716, so the first dropped term is below 2^-60 relative);
 *       ln x = e*ln2_hi + (e*ln2_lo + ln m), ln2 split so e*ln2_hi is exact.
 * exp:  (for the Poisson inversion's e^-lambda) x = k ln2 + r with
 *       k = floor(x (1/ln2) + 1/2), r = (x - k ln2_hi) - k ln2_lo
 *       (k ln2_hi exact), |r| <= 0.35; e^r by its Taylor series through
 *       r^16/16! (first dropped term below 2^-74 relative), Horner in r;
 *       times 2^k (exact for results in the normal range).
 * sincospi: a reduced exactly by multiples of 1/2 to r in [-1/4, 1/4];
 *       y = pi*r; Taylor series of sin y through y^23 and cos y through y^22
 *       (|y| <= pi/4), evaluated by Horner in y^2; quadrant swap/sign.
 */
#include <math.h>
#include <stdint.h>
#include <string.h>

#include "oracle.h"

/* ln 2 = OR_LN2_HI + OR_LN2_LO; OR_LN2_HI has 32 significant bits */
static const double OR_LN2_HI = 0x1.62e42fee00000p-1;
static const double OR_LN2_LO = 0x1.a39ef35793c76p-33;
static const double OR_SQRT_HALF = 0x1.6a09e667f3bcdp-1;
static const double OR_PI = 0x1.921fb54442d18p+1;

double or_log(double x) {
  if (!(x > 0.0)) return x == 0.0 ? -INFINITY : NAN;
  if (isinf(x)) return x;
  uint64_t bits;
  memcpy(&bits, &x, sizeof bits);
  int e = 0;
  if ((bits >> 52) == 0) { /* subnormal: scale into the normal range */
    x = x * 0x1p54;
    memcpy(&bits, &x, sizeof bits);
    e = -54;
  }
  /* x = m * 2^(E-1022) with m in [0.5, 1) */
  e += (int)((bits >> 52) & 0x7ff) - 1022;
  uint64_t mbits = (bits & 0x000fffffffffffffull) | 0x3fe0000000000000ull;
  double m;
  memcpy(&m, &mbits, sizeof m);
  if (m < OR_SQRT_HALF) { /* move m into [sqrt(1/2), sqrt(2)) */
    m = m * 2.0;
    e = e - 1;
  }
  double s = (m - 1.0) / (m + 1.0);
  double s2 = s * s;
  /* p = sum_{k=0}^{12} s2^k / (2k+1), Horner from the top term */
  double p = 1.0 / 25.0;
  p = p * s2 + 1.0 / 23.0;
  p = p * s2 + 1.0 / 21.0;
  p = p * s2 + 1.0 / 19.0;
  p = p * s2 + 1.0 / 17.0;
  p = p * s2 + 1.0 / 15.0;
  p = p * s2 + 1.0 / 13.0;
  p = p * s2 + 1.0 / 11.0;
  p = p * s2 + 1.0 / 9.0;
  p = p * s2 + 1.0 / 7.0;
  p = p * s2 + 1.0 / 5.0;
  p = p * s2 + 1.0 / 3.0;
  double lnm = 2.0 * s + (2.0 * s) * (s2 * p);
  double fe = (double)e;
  return fe * OR_LN2_HI + (fe * OR_LN2_LO + lnm);
}

/* e^x for -708 <= x <= 709 (NaN for NaN; 0 below, inf above) */
double or_exp(double x) {
  if (isnan(x)) return x;
  if (x < -708.0) return 0.0;
  if (x > 709.0) return INFINITY;
  const double k = floor(x * 0x1.71547652b82fep+0 + 0.5); /* nearest multiple of ln 2 */
  const double r = (x - k * OR_LN2_HI) - k * OR_LN2_LO;
  double p = 0x1.ae7f3e733b81fp-45;      /* 1/16! */
  p = p * r + 0x1.ae7f3e733b81fp-41;     /* 1/15! */
  p = p * r + 0x1.93974a8c07c9dp-37;     /* 1/14! */
  p = p * r + 0x1.6124613a86d09p-33;     /* 1/13! */
  p = p * r + 0x1.1eed8eff8d898p-29;     /* 1/12! */
  p = p * r + 0x1.ae64567f544e4p-26;     /* 1/11! */
  p = p * r + 0x1.27e4fb7789f5cp-22;     /* 1/10! */
  p = p * r + 0x1.71de3a556c734p-19;     /* 1/9!  */
  p = p * r + 0x1.a01a01a01a01ap-16;     /* 1/8!  */
  p = p * r + 0x1.a01a01a01a01ap-13;     /* 1/7!  */
  p = p * r + 0x1.6c16c16c16c17p-10;     /* 1/6!  */
  p = p * r + 0x1.1111111111111p-7;      /* 1/5!  */
  p = p * r + 0x1.5555555555555p-5;      /* 1/4!  */
  p = p * r + 0x1.5555555555555p-3;      /* 1/3!  */
  p = p * r + 0.5;                       /* 1/2!  */
  p = p * r + 1.0;
  p = p * r + 1.0;
  return ldexp(p, (int)k);
}

void or_exp_many(uint64_t n, const double *x, double *out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = or_exp(x[i]);
}

/* sin y and cos y for |y| <= pi/4 by their Taylor series */
static void or_sincos_kernel(double y, double *s, double *c) {
  double y2 = y * y;
  /* sin y = y + y*y2*( -1/3! + y2*( 1/5! - ... + y2*(1/23!) ) ) */
  double ps = -0x1.761b41316381ap-75; /* -1/23! */
  ps = ps * y2 + 0x1.71b8ef6dcf572p-66; /*  1/21! */
  ps = ps * y2 - 0x1.2f49b46814157p-57; /* -1/19! */
  ps = ps * y2 + 0x1.952c77030ad4ap-49; /*  1/17! */
  ps = ps * y2 - 0x1.ae7f3e733b81fp-41; /* -1/15! */
  ps = ps * y2 + 0x1.6124613a86d09p-33; /*  1/13! */
  ps = ps * y2 - 0x1.ae64567f544e4p-26; /* -1/11! */
  ps = ps * y2 + 0x1.71de3a556c734p-19; /*  1/9!  */
  ps = ps * y2 - 0x1.a01a01a01a01ap-13; /* -1/7!  */
  ps = ps * y2 + 0x1.1111111111111p-7;  /*  1/5!  */
  ps = ps * y2 - 0x1.5555555555555p-3;  /* -1/3!  */
  *s = y + (y * y2) * ps;
  /* cos y = 1 + y2*( -1/2! + y2*( 1/4! - ... + y2*(-1/22!) ) ) */
  double pc = -0x1.0ce396db7f853p-70;   /* -1/22! */
  pc = pc * y2 + 0x1.e542ba4020225p-62; /*  1/20! */
  pc = pc * y2 - 0x1.6827863b97d97p-53; /* -1/18! */
  pc = pc * y2 + 0x1.ae7f3e733b81fp-45; /*  1/16! */
  pc = pc * y2 - 0x1.93974a8c07c9dp-37; /* -1/14! */
  pc = pc * y2 + 0x1.1eed8eff8d898p-29; /*  1/12! */
  pc = pc * y2 - 0x1.27e4fb7789f5cp-22; /* -1/10! */
  pc = pc * y2 + 0x1.a01a01a01a01ap-16; /*  1/8!  */
  pc = pc * y2 - 0x1.6c16c16c16c17p-10; /* -1/6!  */
  pc = pc * y2 + 0x1.5555555555555p-5;  /*  1/4!  */
  pc = pc * y2 - 0.5;                   /* -1/2!  */
  *c = 1.0 + y2 * pc;
}

void or_sincospi(double a, double *s, double *c) {
  /* n = nearest multiple of 1/2 (as an integer count of halves); exact for
   * the dyadic arguments the Gaussian buffer uses (a = k * 2^-23). */
  double n = floor(2.0 * a + 0.5);
  double r = a - 0.5 * n; /* exact: |r| <= 1/4 */
  double ss, cc;
  or_sincos_kernel(OR_PI * r, &ss, &cc);
  long q = ((long)fmod(n, 4.0) + 4) % 4;
  switch (q) {
  case 0: *s = ss; *c = cc; break;
  case 1: *s = cc; *c = -ss; break;
  case 2: *s = -ss; *c = -cc; break;
  default: *s = -cc; *c = ss; break;
  }
}

void or_log_many(uint64_t n, const double *x, double *out) {
  for (uint64_t i = 0; i < n; ++i) out[i] = or_log(x[i]);
}

void or_sincospi_many(uint64_t n, const double *a, double *s, double *c) {
  for (uint64_t i = 0; i < n; ++i) or_sincospi(a[i], &s[i], &c[i]);
}
