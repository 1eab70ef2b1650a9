// brng_rejection32.cuh -- one attempt of Hormann's transformed-rejection
// samplers (PTRS for Poisson, BTRD for Binomial; W. Hormann, "The generation
// of binomial random variates", J. Statist. Comput. Simul. 46, 1993, and
// "The transformed rejection method for generating Poisson random
// variables", Insurance: Mathematics and Economics 12, 1993), decided in
// FP32 and float-float arithmetic where that decision provably equals the
// FP64 evaluation of the same attempt (brng_fp64.cuh), and reported
// undecided otherwise, for the caller to redo in FP64.
//
// Each attempt makes up to four kinds of decision, each certified its own way:
//  * comparisons of a grid value (every U element is a multiple of 2^-24)
//    with a threshold: exact thresholds on the grid where the threshold is a
//    constant; float-float thresholds with a 2^-34 band where it depends on
//    the parameters;
//  * k = floor(X) of the hat transform X = (2a/us + b) u + c: X is evaluated
//    in float-float around its integer part (taken exactly from the
//    parameters), and k is kept only when X lies farther than a bound on
//    |X_ff - X_fp64| from every integer;
//  * the product test of BTRD's recursion (|k - m| <= 15): float-float, with
//    a relative band of 2^-30;
//  * the log-scale tests: FP32, with every logarithm taken in a form whose
//    argument is known to a few rounding errors (log1p(t) for ratios near 1,
//    the factorials through g(t) = (1+t) log1p(t) - t), CUDA's logf and
//    log1pf (at most 1 ulp), and a band of 32u or 64u times the sum of the
//    magnitudes of the terms (twice or more the worst-case FP32 error), plus
//    the FP64 evaluation's own rounding.
// The bands are several times the error bounds stated with each decision, so
// an attempt is reported decided only when the FP64 evaluation cannot decide
// it otherwise; the checked build recomputes every decided attempt in FP64
// and counts any difference as a violation.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "brng_ff.cuh"

namespace brng {

struct Attempt32 {
  float k;   // the count; -1 rejected; kUndecided: redo the attempt in FP64
  int used;  // U elements the attempt consumed (when decided)
};

// us >= 0.07 and us < 0.013 (the doubles) on the 2^-24 grid: us = j 2^-24
// compares with 0.07 as j >= 1174406 and with 0.013 as j < 218104.
constexpr float kUs007 = 0x1.1eb86p-4f;  // 1174406 * 2^-24
constexpr float kUs013 = 0x1.a9fcp-7f;   //  218104 * 2^-24
constexpr float kGrid = 0x1p-24f;
constexpr float kHalfLn2Pi32 = 0.918938533f;

// ln Gamma(x) - ((x - 1/2) ln x - x + ln(2 pi)/2) by Stirling's series
// through x^-7, for x >= 17 (the same terms as the FP64 evaluation; the FP32
// value is within 4u of 0.005 there).
__device__ __forceinline__ float stirling_tail32(float x) {
  const float inv = __fdiv_rn(1.0f, x);
  const float inv2 = __fmul_rn(inv, inv);
  float t = __fmul_rn(inv2, 1.0f / 1680.0f);
  t = __fmul_rn(inv2, __fadd_rn(1.0f / 1260.0f, -t));
  t = __fmul_rn(inv2, __fadd_rn(1.0f / 360.0f, -t));
  return __fmul_rn(inv, __fadd_rn(1.0f / 12.0f, -t));
}

// floor(Y) for |Y| < lim (<= 2^24), certified: false (undecided) when Y is
// within ek of an integer.
__device__ __forceinline__ bool cert_floor(FF Y, float ek, float lim, float* fy) {
  if (!(fabsf(Y.hi) < lim)) return false;
  *fy = ff_floor(Y);
  return ff_frac_gap(Y, *fy) > ek;
}

// ---- PTRS ---------------------------------------------------------------
// One attempt for Poisson(lam), 64 < lam <= 1e7, from u0 (U, [0, 1)) and
// v = U' (u1 + 2^-24, (0, 1]); always consumes 2 elements.
__device__ __forceinline__ Attempt32 ptrs_attempt32(float lam, float u0, float v) {
  Attempt32 r{-1.0f, 2};
  const float u = __fadd_rn(u0, -0.5f);      // exact
  const float us = __fadd_rn(0.5f, -fabsf(u));  // exact, on the grid
  if (us == 0.0f || (us < kUs013 && v > us)) return r;  // rejections whatever k is

  // b, a in float-float (b: 4 operations, a: 6; within 2^-37 relative)
  const FF slam = ff_sqrt(ff_from(lam));
  const FF b = ff_add(ff_const(0.931), ff_mul(ff_const(2.53), slam));
  const FF a = ff_add(ff_const(-0.059), ff_mul(ff_const(0.02483), b));
  // X - floor(lam) = (2a/us + b) u + (lam - floor(lam)) + 0.43; u and us are
  // exact, so |X_ff - X*| <= 2^-36 (|T| + 1); the FP64 evaluation is within
  // 2^-49 (|T| + lam) of X*.
  const FF T = ff_mul_f(ff_add(ff_div_f(ff_scale2(a), us), b), u);
  const float Li = floorf(lam);
  const float Lf = __fadd_rn(lam, -Li);  // exact
  const FF Y = ff_add(T, ff_add_f(ff_const(0.43), Lf));
  const float ek = __fmaf_rn(fabsf(T.hi) + 1.0f, 0x1p-36f, __fmul_rn(lam, 0x1p-46f));
  const bool negative = __fadd_rn(Y.hi, Li) < -2.0f - 2.0f * ek;  // k < 0 whatever the rounding
  float fy;
  const bool known = !negative && cert_floor(Y, ek, 0x1p22f, &fy);
  const float k = known ? __fadd_rn(Li, fy) : 0.0f;  // exact: integers below 2^24
  const float b32 = b.hi;

  if (us >= kUs007) {  // the squeeze: v <= vr accepts k (k > lam - 0.74 b > 0 here)
    // vr in FP32 from b (within 2^-37): 3 roundings and the constants' 2,
    // |vr_32 - vr| <= 3u; the band is 8u
    const float vr = __fadd_rn(0.9277f, -__fdiv_rn(3.6224f, __fadd_rn(b32, -2.0f)));
    const float dv = __fadd_rn(v, -vr);
    if (known && dv <= -8.0f * kGrid) {
      r.k = k;
      return r;
    }
    if (!(dv > 8.0f * kGrid)) {
      r.k = kUndecided;
      return r;
    }
  }
  if (negative) return r;
  if (!known) {
    r.k = kUndecided;
    return r;
  }
  if (k < 0.0f) return r;
  if (k < 16.0f) {  // ln k! outside the Stirling form below (k + 1 <= 2^24 is exact)
    r.k = kUndecided;
    return r;
  }

  // log(v) + log(1/alpha) - log(a/us^2 + b) <= -lam + k log(lam) - log k!
  const float a32 = a.hi;
  const float ia = __fadd_rn(1.1239f, __fdiv_rn(1.1328f, __fadd_rn(b32, -3.4f)));
  const float A = __fadd_rn(__fdiv_rn(a32, __fmul_rn(us, us)), b32);
  const float lv = logf(v), lia = logf(ia), lA = logf(A);
  const float lhs = __fadd_rn(__fadd_rn(lv, lia), -lA);
  // with x = k + 1, d = x - lam, t = d / lam and ln k! by Stirling at x:
  //   rhs = -lam g(t) + log1p(t)/2 - (ln lam + ln 2pi)/2 - tail(x),
  //   g(t) = (1+t) log1p(t) - t = (t^2/2) sum_j 2 (-t)^j / ((j+1)(j+2))
  const float x = __fadd_rn(k, 1.0f);
  const float d = __fadd_rn(__fadd_rn(x, -Li), -Lf);  // x - Li exact
  const float t = __fdiv_rn(d, lam);
  float G, L1, sG;
  if (fabsf(t) < 0.125f) {  // series to t^7 (remainder below 2^-29 relative)
    L1 = log1pf(t);
    float h = -1.0f / 36.0f;
    h = __fmaf_rn(h, t, 1.0f / 28.0f);
    h = __fmaf_rn(h, t, -1.0f / 21.0f);
    h = __fmaf_rn(h, t, 1.0f / 15.0f);
    h = __fmaf_rn(h, t, -0.1f);
    h = __fmaf_rn(h, t, 1.0f / 6.0f);
    h = __fmaf_rn(h, t, -1.0f / 3.0f);
    h = __fmaf_rn(h, t, 1.0f);
    G = __fmul_rn(__fmul_rn(__fmul_rn(d, t), 0.5f), h);
    sG = 0.0f;
  } else {  // |t| >= 1/8: no cancellation beyond a factor 18
    L1 = logf(__fdiv_rn(x, lam));
    G = __fadd_rn(__fmul_rn(x, L1), -d);
    sG = __fadd_rn(fabsf(__fmul_rn(x, L1)), fabsf(d));
  }
  const float lnlam = logf(lam);
  const float C = __fmaf_rn(0.5f, lnlam, kHalfLn2Pi32);
  const float rhs = __fadd_rn(__fadd_rn(__fadd_rn(__fmul_rn(0.5f, L1), -G), -C), -stirling_tail32(x));
  const float diff = __fadd_rn(lhs, -rhs);
  const float mag = fabsf(lv) + fabsf(lia) + fabsf(lA) + fabsf(lhs) + fabsf(G) + sG + fabsf(L1) + fabsf(C) +
                    fabsf(rhs) + fabsf(diff) + 1.0f;
  // the FP64 evaluation sums -lam, k ln lam and ln k! (each up to ~2e8)
  const float e64 = 0x1p-47f * (lam + x * (2.0f * fabsf(lnlam) + fabsf(L1) + 2.0f));
  // Each term's FP32 error is at most 12u times its magnitude (logf, log1pf
  // within 1 ulp = 2u relative; the largest factor, 11.5u, on x |L1| and |d|
  // of the |t| >= 1/8 form), so 32u (2^-19) times the sum is twice the bound.
  const float band = __fmaf_rn(mag, 0x1p-19f, e64);
  if (diff <= -band) {
    r.k = k;
  } else if (!(diff > band)) {
    r.k = kUndecided;
  }
  return r;
}

// g1(x) = x - log1p(x) >= 0 for x > -1/2: the series x^2 (1/2 - x/3 + ...)
// through x^9 for |x| < 1/8 (remainder below 2^-26 relative), else the
// difference (which loses at most a factor 16 to cancellation there).
__device__ __forceinline__ float g1_32(float x) {
  if (fabsf(x) < 0.125f) {
    float s = -1.0f / 9.0f;
    s = __fmaf_rn(s, x, 0.125f);
    s = __fmaf_rn(s, x, -1.0f / 7.0f);
    s = __fmaf_rn(s, x, 1.0f / 6.0f);
    s = __fmaf_rn(s, x, -0.2f);
    s = __fmaf_rn(s, x, 0.25f);
    s = __fmaf_rn(s, x, -1.0f / 3.0f);
    s = __fmaf_rn(s, x, 0.5f);
    return __fmul_rn(__fmul_rn(x, x), s);
  }
  return __fadd_rn(x, -log1pf(x));
}

// ---- BTRD ---------------------------------------------------------------
// m = floor((n+1) p), its fraction, and c = n p + 1/2 split at its integer
// part, exactly, from p = M 2^-sh (M the 24-bit significand): n p 2^sh and
// (n+1) p 2^sh are integers below 2^49.
struct BtrdExact {
  float ci;   // floor(n p + 1/2)
  FF cfr;     // n p + 1/2 - ci, exactly
  FF np;      // n p, exactly
  float m;    // floor((n + 1) p)
  float fr;   // (n + 1) p - m, rounded once
  FF fr_ff;   // (n + 1) p - m, exactly
};

__device__ __forceinline__ FF ull_to_ff(unsigned long long v, float scale) {  // v < 2^49, scale 2^-j
  const float hi = __ull2float_rn(v);
  const long long rest = static_cast<long long>(v) - static_cast<long long>(__float2ull_rn(hi));
  return FF{__fmul_rn(hi, scale), __fmul_rn(__ll2float_rn(rest), scale)};
}

__device__ __forceinline__ BtrdExact btrd_exact(float n, float p) {  // p in [2^-18, 1/2]
  const uint32_t pb = __float_as_uint(p);
  const unsigned long long M = (pb & 0x7fffffu) | 0x800000u;
  const int sh = 150 - static_cast<int>(pb >> 23);  // 24..41
  const float scale = __uint_as_float(static_cast<uint32_t>(127 - sh) << 23);
  const unsigned long long mask = (1ull << sh) - 1ull;
  const unsigned long long N = __float2ull_rn(n);
  const unsigned long long P = N * M;
  const unsigned long long C = P + (1ull << (sh - 1));
  const unsigned long long R = P + M;
  BtrdExact e;
  e.ci = __ull2float_rn(C >> sh);
  e.cfr = ull_to_ff(C & mask, scale);
  e.np = ull_to_ff(P, scale);
  e.m = __ull2float_rn(R >> sh);
  e.fr_ff = ull_to_ff(R & mask, scale);
  e.fr = e.fr_ff.hi;
  return e;
}

// One attempt for Binomial(n, p_in), n min(p, 1-p) > 64, n <= 2^24, from
// u0 (first element; v = u0 + 2^-24) and u1 (second, read only when used).
__device__ __forceinline__ Attempt32 btrd_attempt32(float n, float p_in, float u0, float u1) {
  Attempt32 r{-1.0f, 1};
  const float v0 = __fadd_rn(u0, kGrid);       // exact
  const bool flip = p_in > 0.5f;
  const float p = flip ? __fadd_rn(1.0f, -p_in) : p_in;  // exact
  const FF q = fast_two_sum(1.0f, -p);         // 1 - p exactly
  const BtrdExact e = btrd_exact(n, p);
  // per-draw constants in float-float (each within ~2^-43 relative)
  const FF npq = ff_mul(e.np, q);
  const FF spq = ff_sqrt(npq);
  const FF b = ff_add(ff_const(1.15), ff_mul(ff_const(2.53), spq));
  const FF a = ff_add(ff_add(ff_const(-0.0873), ff_mul(ff_const(0.0248), b)), ff_mul_f(ff_const(0.01), p));
  const FF vr = ff_sub(ff_const(0.92), ff_div(ff_const(4.2), b));
  const FF urvr = ff_mul(ff_const(0.86), vr);
  const FF a2 = ff_scale2(a);
  constexpr float kBand = 0x1p-34f;  // thresholds below 1, known to ~2^-43

  const float d1 = ff_sub(urvr, ff_from(v0)).hi;
  if (!(fabsf(d1) > kBand)) {
    r.k = kUndecided;
    return r;
  }
  if (d1 > 0.0f) {  // v < urvr: the immediate accept, one element
    const FF u = ff_add(ff_div(ff_from(v0), vr), ff_const(-0.43));
    const FF us = ff_add_f(ff_neg(ff_abs(u)), 0.5f);  // >= 0.07
    const FF A2 = ff_div(a2, us);
    const FF T = ff_mul(ff_add(A2, b), u);
    const FF Y = ff_add(T, e.cfr);
    // |u| error <= 2^-37: |dX| <= 2^-36 (|T| + b + |2a/us| / us) + the FP64 sum's 2^-48 |X|
    const float ek = __fmaf_rn(fabsf(T.hi) + b.hi + 1.0f + __fdiv_rn(fabsf(A2.hi), us.hi), 0x1p-36f,
                               __fmul_rn(e.ci + fabsf(T.hi), 0x1p-48f));
    const float top = __fadd_rn(n, -e.ci);  // exact
    float fy;
    if (!cert_floor(Y, ek, 0x1p24f, &fy) || fy < -e.ci || fy > top) {
      r.k = kUndecided;  // (k outside [0, n] cannot occur for us >= 0.07; kept as a guard)
      return r;
    }
    const float k = __fadd_rn(e.ci, fy);  // exact, in [0, n]
    r.k = flip ? __fadd_rn(n, -k) : k;
    return r;
  }

  r.used = 2;
  const float d2 = ff_sub(ff_from(v0), vr).hi;  // v - vr
  if (!(fabsf(d2) > kBand)) {
    r.k = kUndecided;
    return r;
  }
  FF u, V;
  const bool exact_u = d2 > 0.0f;
  if (exact_u) {  // v >= vr: u from the second element, exactly
    u = ff_from(__fadd_rn(u1, -0.5f));
    V = ff_from(v0);
  } else {
    const FF w = ff_add(ff_div(ff_from(v0), vr), ff_const(-0.93));
    if (!(fabsf(w.hi) > kBand)) {
      r.k = kUndecided;
      return r;
    }
    u = ff_add_f(ff_neg(w), w.hi < 0.0f ? -0.5f : 0.5f);
    V = ff_mul_f(vr, __fadd_rn(u1, kGrid));
  }
  const FF us = ff_add_f(ff_neg(ff_abs(u)), 0.5f);
  if (us.hi == 0.0f) {  // only for u1 = 0 in the exact case
    r.k = -1.0f;
    return r;
  }
  const FF A2 = ff_div(a2, us);
  const FF T = ff_mul(ff_add(A2, b), u);
  const FF Y = ff_add(T, e.cfr);
  // bound on |us_ff - us| / us: us is exact when u is
  const float rel_us = exact_u ? 0.0f : __fdiv_rn(0x1p-36f, us.hi);
  const float ek = __fmaf_rn(fabsf(T.hi) + b.hi + 1.0f + fabsf(A2.hi) * rel_us * 0x1p36f, 0x1p-36f,
                             __fmul_rn(e.ci + fabsf(T.hi), 0x1p-48f));
  // k = ci + floor(Y); k < 0 or k > n rejects, decided on floor(Y) against
  // the exact integers -ci and n - ci
  const float top = __fadd_rn(n, -e.ci);  // exact
  if (Y.hi > top + 2.0f + 2.0f * ek || Y.hi < -e.ci - 2.0f - 2.0f * ek) {
    r.k = -1.0f;
    return r;
  }
  float fy;
  if (!cert_floor(Y, ek, 0x1p24f, &fy)) {
    r.k = kUndecided;
    return r;
  }
  if (fy < -e.ci || fy > top) {
    r.k = -1.0f;
    return r;
  }
  const float k = __fadd_rn(e.ci, fy);  // exact, in [0, n]
  const float res = flip ? __fadd_rn(n, -k) : k;
  const float m = e.m;
  const float km = fabsf(__fadd_rn(k, -m));  // exact
  const FF rr = ff_div(ff_from(p), q);
  const FF Aq = ff_add(ff_div(a, ff_mul(us, us)), b);
  const FF alpha = ff_mul(ff_add(ff_const(2.83), ff_div(ff_const(5.1), b)), spq);
  FF Vs = ff_div(ff_mul(V, alpha), Aq);
  const float rel_v = __fmaf_rn(4.0f, rel_us, 0x1p-34f);  // relative error bound of Vs

  if (km <= 15.0f) {  // f(k) / f(m) by the recursion, <= 15 factors of ~2^-38 each
    const FF nr = ff_add(ff_mul_f(rr, n), rr);  // (n + 1) r
    FF f = ff_from(1.0f);
    if (m < k) {
      for (float i = __fadd_rn(m, 1.0f); i <= k; i = __fadd_rn(i, 1.0f)) f = ff_mul(f, ff_sub(ff_div_f(nr, i), rr));
    } else if (m > k) {
      for (float i = __fadd_rn(k, 1.0f); i <= m; i = __fadd_rn(i, 1.0f))
        Vs = ff_mul(Vs, ff_sub(ff_div_f(nr, i), rr));
    }
    const float dd = ff_sub(Vs, f).hi;
    const float band = __fmul_rn(fmaxf(fabsf(Vs.hi), fabsf(f.hi)), __fadd_rn(0x1p-30f, rel_v));
    r.k = dd <= -band ? res : (dd > band ? -1.0f : kUndecided);
    return r;
  }

  // the squeeze on the log scale
  const float lv = __fadd_rn(logf(Vs.hi), __fdiv_rn(Vs.lo, Vs.hi));
  const float npq32 = npq.hi;
  const float rho = __fmul_rn(__fdiv_rn(km, npq32),
                              __fadd_rn(__fdiv_rn(__fadd_rn(__fmul_rn(__fadd_rn(__fdiv_rn(km, 3.0f), 0.625f), km),
                                                            1.0f / 6.0f),
                                                  npq32),
                                        0.5f));
  const float t = -__fdiv_rn(__fmul_rn(km, km), __fmul_rn(2.0f, npq32));
  const float lo = __fadd_rn(t, -rho), hi = __fadd_rn(t, rho);
  // t within 4u, rho within 12u, lv within 2u |lv| + rel_v: 32u covers twice
  const float es = __fmaf_rn(fabsf(t) + rho + fabsf(lv) + 1.0f, 0x1p-19f, rel_v);
  if (lv < lo - es) {
    r.k = res;
    return r;
  }
  if (lv > hi + es) {
    r.k = -1.0f;
    return r;
  }
  if (!(lv > lo + es && lv < hi - es) || k < 16.0f || __fadd_rn(n, -k) < 16.0f) {
    r.k = kUndecided;
    return r;
  }

  // the exact bound: h + (n+1) ln(nm/nk) + (k+1/2) ln(nk r/(k+1)) - fc(k) - fc(n-k),
  // h = (m+1/2) ln((m+1)/(r nm)) + fc(m) + fc(n-m), each ratio near 1 through log1p:
  //   (m+1)/(r nm) = 1 + (q - fr)/(p nm),  nm/nk = 1 + x1, x1 = (k - m)/nk,
  //   nk r/(k+1) = 1 + x2, x2 = (fr + p + m - k - 1)/(q (k+1)).
  // The two middle terms are each about (k - m)/q and cancel to O(1), so they
  // are split as Lin - Quad with g1(x) = x - log1p(x) >= 0:
  //   Lin  = (n+1) x1 + (k+1/2) x2           in float-float (the cancellation),
  //   Quad = (n+1) g1(x1) + (k+1/2) g1(x2)   in FP32 (two non-negative terms).
  const float q32 = q.hi;
  const float nm = __fadd_rn(__fadd_rn(n, -m), 1.0f);  // exact
  const float nk = __fadd_rn(__fadd_rn(n, -k), 1.0f);  // exact
  const float k1 = __fadd_rn(k, 1.0f);
  const float La = log1pf(__fdiv_rn(__fadd_rn(q32, -e.fr), __fmul_rn(p, nm)));
  const float hA = __fmul_rn(__fadd_rn(m, 0.5f), La);
  const float h = __fadd_rn(__fadd_rn(hA, stirling_tail32(__fadd_rn(m, 1.0f))), stirling_tail32(nm));
  const FF x1 = ff_div_f(ff_from(__fadd_rn(k, -m)), nk);
  const FF num = ff_add(ff_add_f(e.fr_ff, p), ff_from(__fadd_rn(__fadd_rn(m, -k), -1.0f)));
  const FF qk1 = ff_mul_f(q, k1);
  const FF x2 = ff_div(num, qk1);
  const FF P1 = ff_add(ff_mul_f(x1, n), x1);                  // (n + 1) x1
  const FF P2 = ff_add(ff_mul_f(x2, k), ff_mul_f(x2, 0.5f));  // (k + 1/2) x2
  const float Lin = ff_add(P1, P2).hi;
  // 1 + x2 near 0: the ratio nk p / (q (k+1)) is the better-conditioned argument
  const float g2 = x2.hi < -0.5f ? __fadd_rn(x2.hi, -logf(__fdiv_rn(__fmul_rn(nk, p), qk1.hi))) : g1_32(x2.hi);
  const float g1v = g1_32(x1.hi);
  const float Quad = __fadd_rn(__fmaf_rn(n, g1v, g1v), __fmul_rn(__fadd_rn(k, 0.5f), g2));
  const float bound = __fadd_rn(__fadd_rn(__fadd_rn(__fadd_rn(h, Lin), -Quad), -stirling_tail32(k1)),
                                -stirling_tail32(nk));
  const float diff = __fadd_rn(lv, -bound);
  const float S = fabsf(hA) + fabsf(h) + fabsf(Lin) + Quad + fabsf(bound) + fabsf(diff) + 4.0f;
  // the FP64 evaluation rounds the middle terms (each up to |A1|, |A2|) on their own
  const float e64 = __fmaf_rn(fabsf(P1.hi) + fabsf(P2.hi), 0x1p-46f, 0x1p-26f);
  const float band = __fmaf_rn(S, 0x1p-18f, e64) + __fmaf_rn(4.0f * fabsf(lv), 0x1p-24f, rel_v);
  r.k = diff <= -band ? res : (diff > band ? -1.0f : kUndecided);
  return r;
}

}  // namespace brng
