// brng_fp64.cuh -- FP64 natural log and sin/cos(pi a) for the Gamma accept
// recheck, written so that each is a fixed sequence of IEEE double
// operations (explicit __d*_rn intrinsics: never contracted into FMA).
//
// Why: a Gamma attempt's accept/reject decision is a comparison of two
// logarithmic expressions.  The FP32 fast path takes it when its margin is
// clearly away from zero; otherwise the decision is recomputed in FP64 from
// the same Philox bits.  For that decision to be the one a reference FP64
// computation takes, both must evaluate the same expression with the same
// elementary functions, so these functions are defined by their method, not
// by a math library:
//
//  log(x):  x = m 2^e, m in [sqrt(1/2), sqrt(2)); s = (m - 1)/(m + 1);
//           ln m = 2 atanh s = 2s + 2s s^2 (1/3 + s^2/5 + ... + s^22/25)
//           (Horner from the s^22/25 term); ln x = e ln2_hi + (e ln2_lo + ln m)
//           with ln2_hi holding 32 significant bits of ln 2.
//  sincospi(a): n = floor(2a + 1/2), r = a - n/2 (exact for dyadic a),
//           y = pi r, Taylor series of sin y to y^23 and cos y to y^22 by
//           Horner in y^2, then the quadrant n mod 4 swaps/negates.
//  exp(x):  (the Poisson inversion's e^-lambda) k = floor(x (1/ln2) + 1/2),
//           r = (x - k ln2_hi) - k ln2_lo, e^r by Taylor through r^16/16!
//           (Horner in r), times 2^k.
#pragma once

namespace brng {

__device__ __forceinline__ double dlog(double x) {
  if (!(x > 0.0)) return x == 0.0 ? -__longlong_as_double(0x7ff0000000000000ll)
                                  : __longlong_as_double(0x7ff8000000000000ll);
  long long bits = __double_as_longlong(x);
  if ((bits >> 52) >= 0x7ff) return x;  // +inf
  int e = 0;
  if ((bits >> 52) == 0) {  // subnormal: scale by 2^54
    x = __dmul_rn(x, 0x1p54);
    bits = __double_as_longlong(x);
    e = -54;
  }
  e += static_cast<int>((bits >> 52) & 0x7ff) - 1022;
  double m = __longlong_as_double((bits & 0x000fffffffffffffll) | 0x3fe0000000000000ll);
  if (m < 0x1.6a09e667f3bcdp-1) {
    m = __dmul_rn(m, 2.0);
    e -= 1;
  }
  const double s = __ddiv_rn(__dadd_rn(m, -1.0), __dadd_rn(m, 1.0));
  const double s2 = __dmul_rn(s, s);
  double p = 1.0 / 25.0;
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 23.0);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 21.0);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 19.0);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 17.0);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 15.0);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 13.0);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 11.0);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 9.0);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 7.0);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 5.0);
  p = __dadd_rn(__dmul_rn(p, s2), 1.0 / 3.0);
  const double two_s = __dmul_rn(2.0, s);
  const double lnm = __dadd_rn(two_s, __dmul_rn(two_s, __dmul_rn(s2, p)));
  const double fe = static_cast<double>(e);
  return __dadd_rn(__dmul_rn(fe, 0x1.62e42fee00000p-1),
                   __dadd_rn(__dmul_rn(fe, 0x1.a39ef35793c76p-33), lnm));
}

// e^x for -708 <= x <= 709 (NaN for NaN; 0 below, inf above)
__device__ __forceinline__ double dexp(double x) {
  if (x != x) return x;
  if (x < -708.0) return 0.0;
  if (x > 709.0) return __longlong_as_double(0x7ff0000000000000ll);
  const double k = floor(__dadd_rn(__dmul_rn(x, 0x1.71547652b82fep+0), 0.5));
  const double r = __dadd_rn(__dadd_rn(x, -__dmul_rn(k, 0x1.62e42fee00000p-1)),
                             -__dmul_rn(k, 0x1.a39ef35793c76p-33));
  double p = 0x1.ae7f3e733b81fp-45;                      // 1/16!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.ae7f3e733b81fp-41);  // 1/15!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.93974a8c07c9dp-37);  // 1/14!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.6124613a86d09p-33);  // 1/13!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.1eed8eff8d898p-29);  // 1/12!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.ae64567f544e4p-26);  // 1/11!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.27e4fb7789f5cp-22);  // 1/10!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.71de3a556c734p-19);  // 1/9!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.a01a01a01a01ap-16);  // 1/8!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.a01a01a01a01ap-13);  // 1/7!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.6c16c16c16c17p-10);  // 1/6!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.1111111111111p-7);   // 1/5!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.5555555555555p-5);   // 1/4!
  p = __dadd_rn(__dmul_rn(p, r), 0x1.5555555555555p-3);   // 1/3!
  p = __dadd_rn(__dmul_rn(p, r), 0.5);
  p = __dadd_rn(__dmul_rn(p, r), 1.0);
  p = __dadd_rn(__dmul_rn(p, r), 1.0);
  return ldexp(p, static_cast<int>(k));
}

// Poisson(lambda) by inversion of u in FP64: the smallest k with u < F(k),
// F(k) = p_0 + ... + p_k left to right, p_0 = e^-lambda, p_j = (p_{j-1} lambda) / j;
// the search stops when p underflows or at k = kmax.
__device__ __forceinline__ double poisson_inv64(double lambda, double u, int kmax) {
  double p = dexp(-lambda);
  double F = p;
  int k = 0;
  while (!(u < F) && k < kmax) {
    ++k;
    p = __ddiv_rn(__dmul_rn(p, lambda), static_cast<double>(k));
    if (p == 0.0) break;
    F = __dadd_rn(F, p);
  }
  return static_cast<double>(k);
}

// Binomial(n, p) by inversion of u in FP64 on q = min(p, 1 - p): the smallest
// k with u < F(k), F summed left to right from p_0 = exp(n log(1 - q)),
// p_k = (p_{k-1} ((n - k + 1) r)) / k, r = q / (1 - q); n - k when p > 1/2.
__device__ __forceinline__ double binomial_inv64(double n, double p, double u) {
  const bool flip = p > 0.5;
  const double q = flip ? __dadd_rn(1.0, -p) : p;
  const double omq = __dadd_rn(1.0, -q);
  double pk = dexp(__dmul_rn(n, dlog(omq)));
  const double r = __ddiv_rn(q, omq);
  double F = pk;
  double k = 0.0;
  while (!(u < F) && k < n) {
    k = k + 1.0;
    pk = __ddiv_rn(__dmul_rn(pk, __dmul_rn(__dadd_rn(__dadd_rn(n, -k), 1.0), r)), k);
    if (pk == 0.0) break;
    F = __dadd_rn(F, pk);
  }
  return flip ? __dadd_rn(n, -k) : k;
}

__device__ __forceinline__ void dsincospi(double a, double* s_out, double* c_out) {
  const double n = floor(__dadd_rn(__dmul_rn(2.0, a), 0.5));
  const double r = __dadd_rn(a, -__dmul_rn(0.5, n));
  const double y = __dmul_rn(0x1.921fb54442d18p+1, r);
  const double y2 = __dmul_rn(y, y);
  double ps = -0x1.761b41316381ap-75;
  ps = __dadd_rn(__dmul_rn(ps, y2), 0x1.71b8ef6dcf572p-66);
  ps = __dadd_rn(__dmul_rn(ps, y2), -0x1.2f49b46814157p-57);
  ps = __dadd_rn(__dmul_rn(ps, y2), 0x1.952c77030ad4ap-49);
  ps = __dadd_rn(__dmul_rn(ps, y2), -0x1.ae7f3e733b81fp-41);
  ps = __dadd_rn(__dmul_rn(ps, y2), 0x1.6124613a86d09p-33);
  ps = __dadd_rn(__dmul_rn(ps, y2), -0x1.ae64567f544e4p-26);
  ps = __dadd_rn(__dmul_rn(ps, y2), 0x1.71de3a556c734p-19);
  ps = __dadd_rn(__dmul_rn(ps, y2), -0x1.a01a01a01a01ap-13);
  ps = __dadd_rn(__dmul_rn(ps, y2), 0x1.1111111111111p-7);
  ps = __dadd_rn(__dmul_rn(ps, y2), -0x1.5555555555555p-3);
  const double sn = __dadd_rn(y, __dmul_rn(__dmul_rn(y, y2), ps));
  double pc = -0x1.0ce396db7f853p-70;
  pc = __dadd_rn(__dmul_rn(pc, y2), 0x1.e542ba4020225p-62);
  pc = __dadd_rn(__dmul_rn(pc, y2), -0x1.6827863b97d97p-53);
  pc = __dadd_rn(__dmul_rn(pc, y2), 0x1.ae7f3e733b81fp-45);
  pc = __dadd_rn(__dmul_rn(pc, y2), -0x1.93974a8c07c9dp-37);
  pc = __dadd_rn(__dmul_rn(pc, y2), 0x1.1eed8eff8d898p-29);
  pc = __dadd_rn(__dmul_rn(pc, y2), -0x1.27e4fb7789f5cp-22);
  pc = __dadd_rn(__dmul_rn(pc, y2), 0x1.a01a01a01a01ap-16);
  pc = __dadd_rn(__dmul_rn(pc, y2), -0x1.6c16c16c16c17p-10);
  pc = __dadd_rn(__dmul_rn(pc, y2), 0x1.5555555555555p-5);
  pc = __dadd_rn(__dmul_rn(pc, y2), -0.5);
  const double cs = __dadd_rn(1.0, __dmul_rn(y2, pc));
  const int q = static_cast<int>(n) & 3;
  switch (q) {
    case 0: *s_out = sn; *c_out = cs; break;
    case 1: *s_out = cs; *c_out = -sn; break;
    case 2: *s_out = -sn; *c_out = -cs; break;
    default: *s_out = -cs; *c_out = sn; break;
  }
}

// FP64 Gaussian element of a Box-Muller pair (w0, w1); `odd` picks the sin half
__device__ __forceinline__ double dgauss(uint32_t w0, uint32_t w1, bool odd) {
  const double u_open = __dmul_rn(static_cast<double>((w0 >> 8) + 1u), 0x1p-24);
  const double r = __dsqrt_rn(__dmul_rn(-2.0, dlog(u_open)));
  double s, c;
  dsincospi(__dmul_rn(static_cast<double>(w1 >> 8), 0x1p-23), &s, &c);
  return __dmul_rn(r, odd ? s : c);
}

// FP64 Marsaglia-Tsang decision for shape alpha (FP32 input), Gaussian z and
// open uniform u: 1 accept, 0 reject, -1 if t <= 0.  Same operations, same
// order as the reference definition: a = alpha (+1 if alpha < 1),
// d = a - 1/3, c = 1/sqrt(9d), t = 1 + c z, v = (t t) t,
// accept iff log(u) < (0.5 z) z + d ((1 - v) + log(v)).
__device__ __forceinline__ double mt_d64(float alpha_f) {
  const double alpha = static_cast<double>(alpha_f);
  const double a = alpha < 1.0 ? __dadd_rn(alpha, 1.0) : alpha;
  return __dadd_rn(a, -0x1.5555555555555p-2);
}

__device__ __forceinline__ double mt_t64(double d, double z) {
  const double c = __ddiv_rn(1.0, __dsqrt_rn(__dmul_rn(9.0, d)));
  return __dadd_rn(1.0, __dmul_rn(c, z));
}

__device__ __forceinline__ bool mt_accept64(double d, double z, double t, double u_open) {
  const double v = __dmul_rn(__dmul_rn(t, t), t);
  const double lhs = dlog(u_open);
  const double rhs = __dadd_rn(__dmul_rn(__dmul_rn(0.5, z), z),
                               __dmul_rn(d, __dadd_rn(__dadd_rn(1.0, -v), dlog(v))));
  return lhs < rhs;
}


// ---- large means: transformed rejection (Hormann 1993), all FP64 ----------
// The same operations in the same order as the reference definition (IEEE
// sqrt, division and floor, dlog, no contraction), so that every accept
// decision and every count is the reference's.  The kernels run these only
// for the attempts that the FP32 / float-float path (brng_rejection32.cuh)
// leaves undecided, and, in the checked build, to verify the ones it decides.

constexpr double kHalfLog2Pi = 0x1.d67f1c864beb5p-1;  // ln(2 pi) / 2

// Stirling's series of ln Gamma(x) beyond its leading terms, to x^-7 (x >= 17)
__device__ __forceinline__ double dstirling_tail(double x) {
  const double inv = __ddiv_rn(1.0, x);
  const double inv2 = __dmul_rn(inv, inv);
  double t = __dmul_rn(inv2, 1.0 / 1680.0);
  t = __dmul_rn(inv2, __dadd_rn(1.0 / 1260.0, -t));
  t = __dmul_rn(inv2, __dadd_rn(1.0 / 360.0, -t));
  return __dmul_rn(inv, __dadd_rn(1.0 / 12.0, -t));
}

// ln k! for an integer k >= 0: log of the exact product to 15!, Stirling above
__device__ __forceinline__ double dlfact(double k) {
  if (k <= 15.0) {
    double f = 1.0;
    for (double i = 2.0; i <= k; i += 1.0) f = __dmul_rn(f, i);
    return dlog(f);
  }
  const double x = __dadd_rn(k, 1.0);
  return __dadd_rn(__dadd_rn(__dmul_rn(__dadd_rn(x, -0.5), dlog(x)), -x),
                   __dadd_rn(kHalfLog2Pi, dstirling_tail(x)));
}

// f_c(k) = ln k! - (k + 1/2) ln(k + 1) + (k + 1) - ln(2 pi)/2
__device__ __forceinline__ double dstirling_fc(double k) {
  if (k <= 15.0) {
    const double x = __dadd_rn(k, 1.0);
    return __dadd_rn(__dadd_rn(__dadd_rn(dlfact(k), -__dmul_rn(__dadd_rn(k, 0.5), dlog(x))), x), -kHalfLog2Pi);
  }
  return dstirling_tail(__dadd_rn(k, 1.0));
}

// One PTRS attempt for Poisson(lam): u0 = U in [0, 1), v = U' in (0, 1].
// Returns the count, or -1 for a rejection.
__device__ __forceinline__ double ptrs_attempt64(double lam, double u0, double v) {
  const double slam = __dsqrt_rn(lam);
  const double b = __dadd_rn(0.931, __dmul_rn(2.53, slam));
  const double a = __dadd_rn(-0.059, __dmul_rn(0.02483, b));
  const double vr = __dadd_rn(0.9277, -__ddiv_rn(3.6224, __dadd_rn(b, -2.0)));
  const double u = __dadd_rn(u0, -0.5);
  const double us = __dadd_rn(0.5, -fabs(u));
  if (us == 0.0) return -1.0;
  const double k = floor(__dadd_rn(__dadd_rn(__dmul_rn(__dadd_rn(__ddiv_rn(__dmul_rn(2.0, a), us), b), u), lam),
                                   0.43));
  if (us >= 0.07 && v <= vr) return k;
  if (k < 0.0 || (us < 0.013 && v > us)) return -1.0;
  const double inv_alpha = __dadd_rn(1.1239, __ddiv_rn(1.1328, __dadd_rn(b, -3.4)));
  const double lhs = __dadd_rn(__dadd_rn(dlog(v), dlog(inv_alpha)),
                               -dlog(__dadd_rn(__ddiv_rn(a, __dmul_rn(us, us)), b)));
  const double rhs = __dadd_rn(__dadd_rn(-lam, __dmul_rn(k, dlog(lam))), -dlfact(k));
  return lhs <= rhs ? k : -1.0;
}

// One BTRD attempt for Binomial(n, p_in): v0 = U' in (0, 1] (first element),
// u1 = U in [0, 1) (second element, read only when the attempt needs it).
// Returns the count (n - k for p_in > 1/2) or -1 for a rejection; *used gets
// the elements the attempt consumed (1 or 2).
__device__ __forceinline__ double btrd_attempt64(double n, double p_in, double v0, double u1, int* used) {
  const bool flip = p_in > 0.5;
  const double p = flip ? __dadd_rn(1.0, -p_in) : p_in;
  const double q = __dadd_rn(1.0, -p);
  const double spq = __dsqrt_rn(__dmul_rn(__dmul_rn(n, p), q));
  const double b = __dadd_rn(1.15, __dmul_rn(2.53, spq));
  const double a = __dadd_rn(__dadd_rn(-0.0873, __dmul_rn(0.0248, b)), __dmul_rn(0.01, p));
  const double c = __dadd_rn(__dmul_rn(n, p), 0.5);
  const double vr = __dadd_rn(0.92, -__ddiv_rn(4.2, b));
  const double urvr = __dmul_rn(0.86, vr);
  double v = v0, u;
  *used = 1;
  if (v <= urvr) {
    u = __dadd_rn(__ddiv_rn(v, vr), -0.43);
    const double k = floor(__dadd_rn(__dmul_rn(__dadd_rn(__ddiv_rn(__dmul_rn(2.0, a),
                                                                     __dadd_rn(0.5, -fabs(u))), b), u), c));
    return flip ? __dadd_rn(n, -k) : k;
  }
  *used = 2;
  if (v >= vr) {
    u = __dadd_rn(u1, -0.5);
  } else {
    u = __dadd_rn(__ddiv_rn(v, vr), -0.93);
    u = __dadd_rn(u < 0.0 ? -0.5 : 0.5, -u);
    v = __dmul_rn(__dadd_rn(u1, 0x1p-24), vr);
  }
  const double us = __dadd_rn(0.5, -fabs(u));
  if (us == 0.0) return -1.0;
  const double k = floor(__dadd_rn(__dmul_rn(__dadd_rn(__ddiv_rn(__dmul_rn(2.0, a), us), b), u), c));
  if (k < 0.0 || k > n) return -1.0;
  const double m = floor(__dmul_rn(__dadd_rn(n, 1.0), p));
  const double r = __ddiv_rn(p, q);
  const double nr = __dmul_rn(__dadd_rn(n, 1.0), r);
  const double npq = __dmul_rn(__dmul_rn(n, p), q);
  const double alpha = __dmul_rn(__dadd_rn(2.83, __ddiv_rn(5.1, b)), spq);
  v = __ddiv_rn(__dmul_rn(v, alpha), __dadd_rn(__ddiv_rn(a, __dmul_rn(us, us)), b));
  const double km = fabs(__dadd_rn(k, -m));
  const double res = flip ? __dadd_rn(n, -k) : k;
  if (km <= 15.0) {  // f(k)/f(m) by its recursion
    double f = 1.0;
    if (m < k) {
      for (double i = __dadd_rn(m, 1.0); i <= k; i = __dadd_rn(i, 1.0))
        f = __dmul_rn(f, __dadd_rn(__ddiv_rn(nr, i), -r));
    } else if (m > k) {
      for (double i = __dadd_rn(k, 1.0); i <= m; i = __dadd_rn(i, 1.0))
        v = __dmul_rn(v, __dadd_rn(__ddiv_rn(nr, i), -r));
    }
    return v <= f ? res : -1.0;
  }
  v = dlog(v);  // squeeze on the log scale
  const double rho = __dmul_rn(__ddiv_rn(km, npq),
                               __dadd_rn(__ddiv_rn(__dadd_rn(__dmul_rn(__dadd_rn(__ddiv_rn(km, 3.0), 0.625), km),
                                                             1.0 / 6.0),
                                                   npq),
                                         0.5));
  const double t = __ddiv_rn(-__dmul_rn(km, km), __dmul_rn(2.0, npq));
  if (v < __dadd_rn(t, -rho)) return res;
  if (v > __dadd_rn(t, rho)) return -1.0;
  const double nm = __dadd_rn(__dadd_rn(n, -m), 1.0);
  const double h = __dadd_rn(__dadd_rn(__dmul_rn(__dadd_rn(m, 0.5), dlog(__ddiv_rn(__dadd_rn(m, 1.0), __dmul_rn(r, nm)))),
                                       dstirling_fc(m)),
                             dstirling_fc(__dadd_rn(n, -m)));
  const double nk = __dadd_rn(__dadd_rn(n, -k), 1.0);
  const double bound =
      __dadd_rn(__dadd_rn(__dadd_rn(__dadd_rn(h, __dmul_rn(__dadd_rn(n, 1.0), dlog(__ddiv_rn(nm, nk)))),
                                    __dmul_rn(__dadd_rn(k, 0.5), dlog(__ddiv_rn(__dmul_rn(nk, r), __dadd_rn(k, 1.0))))),
                          -dstirling_fc(k)),
                -dstirling_fc(__dadd_rn(n, -k)));
  return v <= bound ? res : -1.0;
}

}  // namespace brng
