// brng_fp32.cuh -- FP32 base conversions and elementary functions written
// without integer<->float conversion instructions.
//
// Why: on GB300 the conversion instructions (I2F/F2I/F2F) share the small FP64
// pipe (2 operations per clock per SM), and the base conversions of the
// method run one or more of them per deviate (U from a word; inside a library
// logf, log1pf or sincospif).  A profile of the Gibbs kernel showed that pipe
// two-thirds busy.  Everything here uses integer/logical operations, FP32
// FMA-pipe arithmetic and at most one MUFU reciprocal.
//
//  u01(w)        U = (w >> 8) 2^-24, exact: the top 23 bits become the mantissa
//                of 1 + f (minus 1, exact), the 24th bit adds 2^-24 (exact).
//  flog(x)       x = m 2^e with m in [sqrt(1/2), sqrt(2)) by subtracting the bit
//                pattern of sqrt(1/2); s = (m-1)/(m+1);
//                ln m = 2s + 2s s^2 (1/3 + s^2/5 + s^4/7 + s^6/9)  (atanh series;
//                |s| <= 0.172, first dropped term < 2e-9 relative);
//                ln x = e ln2_hi + (e ln2_lo + ln m); e enters FP32 exactly
//                through the 1.5*2^23 magic-number addition.  About 3 ulp.
//  fsincospi_k(k) sin and cos of pi k 2^-23 for a 24-bit integer k: the
//                quadrant and the reduced argument r = k - n 2^22, |r| <= 2^21,
//                come from integer arithmetic (exact); y = pi r 2^-23; Taylor
//                series of sin to y^9 and cos to y^10 (|y| <= pi/4: the first
//                dropped terms are below 1.8e-9 and 1.2e-10, i.e. under 0.05
//                ulp of sin y >= 0.9 y and of cos y >= 0.7); quadrant swap and
//                signs.  About 2 ulp.
#pragma once

#include <cstdint>

namespace brng {

// exact float of a small integer (|i| < 2^22) without a conversion instruction
__device__ __forceinline__ float small_int_to_float(int i) {
  return __int_as_float(0x4B400000 + i) - 12582912.0f;
}

// U = (w >> 8) 2^-24 in [0, 1), exact
__device__ __forceinline__ float u01(uint32_t w) {
  const float hi = __uint_as_float(0x3F800000u | (w >> 9)) - 1.0f;    // (w >> 9) 2^-23
  const float lo = __uint_as_float((w & 0x100u) ? 0x33800000u : 0u);  // bit 8 of w: 2^-24
  return hi + lo;
}
// U' = U + 2^-24 in (0, 1], exact
__device__ __forceinline__ float u01_open(uint32_t w) { return u01(w) + 0x1p-24f; }

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
  float ps = 0x1.71de3ap-19f;              //  1/9!
  ps = fmaf(ps, y2, -0x1.a01a02p-13f);     // -1/7!
  ps = fmaf(ps, y2, 0x1.111112p-7f);       //  1/5!
  ps = fmaf(ps, y2, -0x1.555556p-3f);      // -1/3!
  const float sn = fmaf(y * y2, ps, y);
  float pc = -0x1.27e4fcp-22f;             // -1/10!
  pc = fmaf(pc, y2, 0x1.a01a02p-16f);      //  1/8!
  pc = fmaf(pc, y2, -0x1.6c16c2p-10f);     // -1/6!
  pc = fmaf(pc, y2, 0x1.555556p-5f);       //  1/4!
  pc = fmaf(pc, y2, -0.5f);                // -1/2!
  const float cs = fmaf(y2, pc, 1.0f);
  const uint32_t q = n & 3u;
  const float a = (q & 1u) ? cs : sn;  // sin(pi a) up to sign
  const float b = (q & 1u) ? sn : cs;  // cos(pi a) up to sign
  *s_out = (q & 2u) ? -a : a;
  *c_out = ((q + 1u) & 2u) ? -b : b;
}

}  // namespace brng
