// brng_fp32.cuh -- FP32 base conversions and elementary functions for the
// rings' generators, written for instruction count (the Gibbs kernels are
// bound by instruction issue).
//
// Integer-to-float conversions are used only where they replace several
// bit-manipulation instructions (U, U'); measured on GB300 they issue on
// neither the FP64 nor the MUFU pipe.  The log and sin/cos are series
// evaluated with FP32 FMAs after exact integer argument reduction, with one
// MUFU reciprocal in the log.
//
//  u01(w)        U = (w >> 8) 2^-24, exact: the 24-bit integer converts to FP32
//                exactly, and the power-of-two scale is exact.
//  u01_open(w)   U' = ((w >> 8) + 1) 2^-24 in (0, 1], exact: the integer
//                M = (w >> 8) + 1 <= 2^24 converts exactly, and 24 is taken off
//                its exponent field (M >= 1, so the result stays normal).
//  flog(x)       x = m 2^e with m in [sqrt(1/2), sqrt(2)) by subtracting the bit
//                pattern of sqrt(1/2); s = (m-1)/(m+1);
//                ln m = 2s + 2s s^2 (1/3 + s^2/5 + s^4/7 + s^6/9)  (atanh series;
//                |s| <= 0.172, first dropped term < 2e-9 relative);
//                ln x = e ln2_hi + (e ln2_lo + ln m); e enters FP32 exactly
//                through the 1.5*2^23 magic-number addition.  About 3 ulp.
//  fsincospi_k(k) sin and cos of pi k 2^-23 for a 24-bit integer k: the
//                quadrant and the reduced argument r = k - n 2^22, |r| <= 2^21,
//                come from integer arithmetic (exact); y = pi r 2^-23;
//                sin y = y + y^3 P(y^2), cos y = 1 - y^2/2 + y^4 Q(y^2) with P
//                of degree 2 and Q of degree 2, minimax for |y| <= pi/4 (fitted
//                for this library by linear programming over 3,000
//                Chebyshev-spaced points, weighted for relative error, then
//                rounded to FP32: polynomial error below 6.1e-9 and 2.4e-9
//                relative, about 0.1 and 0.04 ulp); quadrant swap and signs.
//                About 2 ulp.
#pragma once

#include <cstdint>

namespace brng {

// exact float of a small integer (|i| < 2^22) without a conversion instruction
__device__ __forceinline__ float small_int_to_float(int i) {
  return __int_as_float(0x4B400000 + i) - 12582912.0f;
}

// U = (w >> 8) 2^-24 in [0, 1), exact
__device__ __forceinline__ float u01(uint32_t w) { return __uint2float_rn(w >> 8) * 0x1p-24f; }
// U' = U + 2^-24 in (0, 1], exact
__device__ __forceinline__ float u01_open(uint32_t w) {
  return __int_as_float(__float_as_int(__uint2float_rn((w >> 8) + 1u)) - (24 << 23));
}

// natural log for finite normal x > 0
__device__ __forceinline__ float flog(float x) {
  const int bits = __float_as_int(x);
  const int t = bits - 0x3F3504F3;  // bits of sqrt(1/2)
  const int e = t >> 23;            // arithmetic shift: floor
  const float m = __int_as_float(bits - (e << 23));
  const float s = __fdividef(m - 1.0f, m + 1.0f);
  const float s2 = s * s;
  float p = 0x1.c71c72p-4f;          // 1/9
  p = fmaf(p, s2, 0x1.24924ap-3f);   // 1/7
  p = fmaf(p, s2, 0x1.99999ap-3f);   // 1/5
  p = fmaf(p, s2, 0x1.555556p-2f);   // 1/3
  const float two_s = 2.0f * s;
  const float lnm = fmaf(two_s * s2, p, two_s);
  const float fe = small_int_to_float(e);
  return fmaf(fe, 0x1.62e400p-1f, fmaf(fe, 0x1.7f7d1cp-20f, lnm));
}

// sin and cos of pi k 2^-23 (0 <= k < 2^24)
__device__ __forceinline__ void fsincospi_k(uint32_t k, float* s_out, float* c_out) {
  const uint32_t n = (k + (1u << 21)) >> 22;  // nearest multiple of 2^22: quadrant count
  const int r = static_cast<int>(k) - static_cast<int>(n << 22);
  const float y = small_int_to_float(r) * 0x1.921fb6p-22f;  // pi r 2^-23, |y| <= pi/4
  const float y2 = y * y;
  float ps = -0x1.994eb4p-13f;             // P: minimax, near -1/7!, 1/5!, -1/3!
  ps = fmaf(ps, y2, 0x1.11076p-7f);
  ps = fmaf(ps, y2, -0x1.555546p-3f);
  const float sn = fmaf(y * y2, ps, y);
  float pc = 0x1.99343p-16f;               // Q: minimax, near 1/8!, -1/6!, 1/4!
  pc = fmaf(pc, y2, -0x1.6c087ep-10f);
  pc = fmaf(pc, y2, 0x1.55553ep-5f);
  pc = fmaf(pc, y2, -0.5f);
  const float cs = fmaf(y2, pc, 1.0f);
  const uint32_t q = n & 3u;
  const float a = (q & 1u) ? cs : sn;  // sin(pi a) up to sign
  const float b = (q & 1u) ? sn : cs;  // cos(pi a) up to sign
  *s_out = (q & 2u) ? -a : a;
  *c_out = ((q + 1u) & 2u) ? -b : b;
}

}  // namespace brng
