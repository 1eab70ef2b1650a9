// brng_gamma.cuh -- Gamma(alpha, 1) attempts by Marsaglia & Tsang (2000),
// the irreducible distribution the paper builds from its Gaussian and uniform
// buffers (Sec. 2.2; its own GetGamma is withheld, Sec. 3 note).
//
// One call is ONE attempt for every lane with `run` (all lanes call it, so
// the ring refills stay warp-wide); callers loop until each lane accepted,
// which lets lanes that accepted move on to their next draw instead of
// idling while a neighbour retries.
//
// Precision: the attempt is computed in FP32 and decided there when its
// margin m = ln-test right side minus ln u' is clearly away from zero.  With
// x = c z (c = 1/sqrt(9d)) the margin is exactly
//     m = -ln u' - 3 d x^4 (1/4 - x/5 + x^2/6 - ... ),
// since z^2/2 = 9 d x^2 / 2 cancels the quadratic term of d (1 - v + ln v);
// for |x| <= 1/4 this series (12 terms, truncation < 2e-8 relative) is used,
// free of the cancellation the textbook form suffers at large shapes.  For
// |x| > 1/4 the form z^2/2 + d (1 - v + 3 ln t) - ln u' with
// 1 - v = -x (3 + x (3 + x)) is used.  The FP32 error of m is a few ulp of the
// magnitudes S of its terms, so the decision is taken in FP32 when
// |m| > tol = 1e-5 (1 + S), and otherwise recomputed in FP64
// (brng_fp64.cuh) from the same Philox bits, in the reference operation
// order.  The sign of t = 1 + x is treated the same way when |t| <= 1e-5.
// Rechecks are counted; a recheck that overturns the FP32 sign records
// |m| / tol (which stays far below 1 if the error bound holds).
#pragma once

#include <cstdint>

#include "brng_fp64.cuh"
#include "brng_ring.cuh"

namespace brng {

constexpr int kGammaMaxAttempts = 64;
constexpr float kTauT = 1e-5f;
constexpr float kTauM = 1e-5f;
constexpr float kSeriesMaxX = 0.25f;

// Device counters (layout = brng_counters_t).
struct DevCounters {
  unsigned long long n_domain, n_reject, n_recheck, n_flip;
  unsigned int max_flip_ratio_bits;  // float bits (non-negative -> monotone as uint)
  unsigned int n_timeout;            // bounded waits that ran out
  unsigned long long n_wasted;       // ring elements generated but unused at exit
};

// warp-aggregated counter increment for lanes with `pred`
__device__ __forceinline__ void count_warp(unsigned long long* ctr, bool pred) {
  const unsigned m = __ballot_sync(kFull, pred);
  if (m && lane_id() == static_cast<unsigned>(__ffs(m) - 1)) atomicAdd(ctr, static_cast<unsigned long long>(__popc(m)));
}

// The paper's buffer waste (Sec. 2.4: a buffer refilled in bulk holds
// deviates that are never used when the stream stops): the elements left in
// this lane's rings when its unit ends, summed over the warp into n_wasted
// (all 32 lanes call).  The next call restarts each stream at its position,
// so these elements are generated again there, not lost to the sequence.
__device__ __forceinline__ void count_waste(DevCounters* cnt, uint32_t n) {
  const uint32_t sum = __reduce_add_sync(kFull, n);
  if (sum && lane_id() == 0) atomicAdd(&cnt->n_wasted, static_cast<unsigned long long>(sum));
}

struct GammaState {
  float alpha;  // the parameter as given
  float d, c;   // a - 1/3 and 1/sqrt(9 d), a = alpha or alpha + 1
  bool boost;   // alpha < 1
};

__device__ __forceinline__ GammaState gamma_setup(float alpha) {
  GammaState g;
  g.alpha = alpha;
  g.boost = alpha < 1.0f;
  const float a = g.boost ? alpha + 1.0f : alpha;
  g.d = a - (1.0f / 3.0f);
  g.c = rsqrtf(9.0f * g.d);
  return g;
}

__device__ __forceinline__ bool gamma_param_ok(float alpha) {
  return isfinite(alpha) && alpha > 0.0f;
}

// Philox with the key schedule computed on the fly from the seed words (for
// the rare out-of-line paths, which then need no round-key table)
__device__ __forceinline__ uint4 philox_keyed(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k0 += kPhiloxW0;
      k1 += kPhiloxW1;
    }
    uint32_t hi0, lo0, hi1, lo1;
    mul_hilo(kPhiloxM0, c.x, hi0, lo0);
    mul_hilo(kPhiloxM1, c.z, hi1, lo1);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

struct Recheck {
  float t;   // t = 1 + c z from the FP64 values (for the output d t^3)
  int pass;  // mode 0: t > 0;  mode 1: the attempt accepts
};

// The FP64 re-decision of one attempt, from the same Philox bits: z of N
// element `zi` (Box-Muller in FP64), d, c, t, then either the sign of t
// (mode 0) or the accept test with U' = uo (mode 1; t > 0 is known).  Kept
// out of line on purpose: GB300's FP64 pipe is narrow, and FP64 code the
// compiler predicated into the attempt instead of branching around would
// occupy it on every attempt rather than on the rare ones that need it.
static __device__ __noinline__ Recheck mt_recheck64(float alpha, uint64_t zi, uint32_t stream,
                                                    uint32_t k0, uint32_t k1, float uo, int mode) {
  const uint4 w = philox_keyed(philox_ctr(zi / 4, kDomN, stream), k0, k1);
  const uint32_t slot = static_cast<uint32_t>(zi % 4);
  const double z64 = slot < 2 ? dgauss(w.x, w.y, slot & 1) : dgauss(w.z, w.w, slot & 1);
  const double d64 = mt_d64(alpha);
  const double t64 = mt_t64(d64, z64);
  Recheck r;
  r.t = static_cast<float>(t64);
  r.pass = mode == 0 ? (t64 > 0.0) : mt_accept64(d64, z64, t64, static_cast<double>(uo));
  return r;
}

static __device__ __noinline__ void record_flip(DevCounters* cnt, float ratio) {
  atomicAdd(&cnt->n_flip, 1ull);
  atomicMax(&cnt->max_flip_ratio_bits, __float_as_uint(ratio));
}

// q = 3 d x^4 (1/4 - x/5 + x^2/6 - ...), the margin's correction term for
// |x| <= 1/4 (12 terms, truncation < 2e-8 relative)
__device__ __forceinline__ float mt_series_q(float d, float x) {
  float p = -0x1.111112p-4f;         // -1/15
  p = fmaf(p, x, 0x1.24924ap-4f);    //  1/14
  p = fmaf(p, x, -0x1.3b13b2p-4f);   // -1/13
  p = fmaf(p, x, 0x1.555556p-4f);    //  1/12
  p = fmaf(p, x, -0x1.745d18p-4f);   // -1/11
  p = fmaf(p, x, 0x1.99999ap-4f);    //  1/10
  p = fmaf(p, x, -0x1.c71c72p-4f);   // -1/9
  p = fmaf(p, x, 0.125f);            //  1/8
  p = fmaf(p, x, -0x1.24924ap-3f);   // -1/7
  p = fmaf(p, x, 0x1.555556p-3f);    //  1/6
  p = fmaf(p, x, -0x1.99999ap-3f);   // -1/5
  p = fmaf(p, x, 0.25f);             //  1/4
  const float x2 = x * x;
  return (3.0f * d) * (x2 * x2) * p;
}

// An upper bound of mt_series_q for |x| <= 1/4: the series alternates with
// decreasing terms for x >= 0 (so it is below its partial sum to x^2/6), and
// for x < 0 its terms from x^3 on sum to at most |x|^3 / (7 (1 - |x|)) <=
// 0.1905 |x|^3.  A log-free accept with it is still sufficient, at a quarter
// of the series' cost; the full series is evaluated only on the slow path.
__device__ __forceinline__ float mt_series_qhi(float d, float x) {
  const float p = fmaf(x, fmaf(x, fmaf(fabsf(x), 0.1905f, 0x1.555556p-3f), -0x1.99999ap-3f), 0.25f);
  const float x2 = x * x;
  return (3.0f * d) * (x2 * x2) * p;
}

// The attempts the log-free accept did not settle: the FP32 margin with its
// tolerance, and the FP64 re-decision when the margin is within it.  Returns
// accept | (rechecked << 1).
__device__ __forceinline__ int mt_slow(float alpha, float d, float x, float z, float t, float uo,
                                       bool series, uint64_t zi, uint32_t stream,
                                       uint32_t k0, uint32_t k1, DevCounters* cnt) {
  const float lnu = flog(uo);
  float m, tol;
  if (series) {
    const float q = mt_series_q(d, x);
    m = -lnu - q;
    tol = kTauM * (1.0f + fabsf(lnu) + q);
  } else {
    const float lnv = 3.0f * flog(t);
    const float omv = -x * fmaf(x, x + 3.0f, 3.0f);  // 1 - (1 + x)^3
    const float h = 0.5f * z * z;
    m = h + d * (omv + lnv) - lnu;
    const float S = h + d * (fabsf(omv) + fabsf(lnv) + __fdividef(3.0f * fabsf(x), t)) + fabsf(lnu);
    tol = kTauM * (1.0f + S);
  }
  if (fabsf(m) > tol) return m > 0.0f ? 1 : 0;
  const bool acc = mt_recheck64(alpha, zi, stream, k0, k1, uo, 1).pass != 0;
  if (isfinite(m) && acc != (m > 0.0f)) record_flip(cnt, fabsf(m) / tol);
  return (acc ? 1 : 0) | 2;
}

// The same, out of line: for large shapes (a few per cent of attempts get
// here), so that none of it is issued, even predicated off, on the common path.
static __device__ __noinline__ int mt_slow_call(float alpha, float d, float x, float z, float t,
                                                float uo, bool series, uint64_t zi,
                                                uint32_t stream, uint32_t k0, uint32_t k1,
                                                DevCounters* cnt) {
  return mt_slow(alpha, d, x, z, t, uo, series, zi, stream, k0, k1, cnt);
}

// Marsaglia & Tsang's squeeze: u' < 1 - 0.0331 z^4 implies the accept test
// for every shape a >= 1 (d >= 2/3), which covers all the shapes used here
// (a shape below 1 is boosted to a + 1).  Near z = 0 the slack is
// (0.0331 - 1/(108 d)) z^4 > 0, and a dense grid over d in [2/3, 2e4] and all
// z finds none below zero.  In FP32 the term is enlarged by 1.00001 (z's own
// error of a few 1e-7 relative enters z^4 four times, plus the rounding of
// the constant and products) and compared against 1 - 2^-22, so an FP32 pass
// is a pass of the exact test: a sufficient condition, it never changes a
// decision, and it spares the logarithms of about 90 % of the attempts that
// the series form does not cover (small shapes).
__device__ __forceinline__ bool mt_squeeze(float z, float uo) {
  const float z2 = z * z;
  return fmaf(0.0331f * 1.00001f, z2 * z2, uo) < 0x1.fffff8p-1f;
}

// One attempt.  Returns true for lanes that accepted; then *dv = d v (FP32).
// *zword gets the raw word of the N element used (for the first-word output).
// kLargeShape: the caller's shapes are large (the series form and the
// log-free accept settle almost every attempt), so the rest is called out of
// line; otherwise it is inline (small shapes take it on most attempts).
template <bool kLargeShape = false, class RN, class RU>
__device__ __forceinline__ bool mt_attempt(bool run, const GammaState& g, RN& N, RU& U,
                                           uint32_t stream, const RoundKeys& rk,
                                           DevCounters* cnt, float* dv, uint32_t* zword) {
  const float z = N.get(run, stream, rk, zword);
  const float x = g.c * z;
  const bool series = fabsf(x) <= kSeriesMaxX;
  float t = 1.0f + x;
  bool tpos = t > 0.0f;
  const bool tclose = run && !series && fabsf(t) <= kTauT;
  if (tclose) {  // rare: the sign of t is re-decided in FP64 (z is N element pos-1)
    const Recheck r = mt_recheck64(g.alpha, N.pos() - 1, stream, rk.k[0][0], rk.k[0][1], 0.0f, 0);
    tpos = r.pass != 0;
    t = r.t;
  }
  const bool needu = run && tpos;
  const float u = U.get(needu, stream, rk);
  bool acc = false;
  bool recheck = false;
  if (needu) {
    const float uo = u + 0x1p-24f;  // U' = U + 2^-24, exact
    // q = 3 d x^4 (1/4 - x/5 + ...) >= 0 and the margin is -ln U' - q.
    // Log-free accept: e^-q >= 1 - q, so U' + q < 1 implies ln U' < -q; with
    // the upper bound q_hi >= q this still holds.  The factor 1.00001 covers
    // q_hi's FP32 error (a few 1e-7 relative) and the bound 1 - 2^-22 the
    // rounding of the sum with room to spare, so a fast accept is also an
    // accept of the exact (and FP64) test.
    const float qh = mt_series_qhi(g.d, x);
    if ((series && fmaf(qh, 1.00001f, uo) < 0x1.fffff8p-1f) || mt_squeeze(z, uo)) {
      acc = true;
    } else {
      const int r = kLargeShape ? mt_slow_call(g.alpha, g.d, x, z, t, uo, series, N.pos() - 1, stream,
                                               rk.k[0][0], rk.k[0][1], cnt)
                                : mt_slow(g.alpha, g.d, x, z, t, uo, series, N.pos() - 1, stream,
                                          rk.k[0][0], rk.k[0][1], cnt);
      acc = (r & 1) != 0;
      recheck = (r & 2) != 0;
    }
    *dv = g.d * (t * t * t);
  }
  count_warp(&cnt->n_recheck, tclose || recheck);
  return acc;
}

// One attempt (as mt_attempt) reading its elements with peek/advance from
// rings that already hold, for each lane with `run`, at least 1 N and 2 U
// elements: z (N), then U' if t > 0, then for a boosted shape U_b after an
// accept, which it folds in: on accept *dv = Gamma(alpha) (FP32).  *zword
// gets z's raw word when the N ring keeps words.  Consumes exactly what
// mt_attempt plus the caller's boost draw consume.
// kLogBoost: leave *dv = d v and return the boost in log form in *lboost
// (ln U_b / alpha, 0 without boost) for callers that work in log space.
// rechecked != nullptr: no warp vote inside (the caller counts the rechecks,
// e.g. after several independent attempts, which then overlap).
template <bool kLargeShape, bool kZWord, bool kLogBoost = false, class RNT, class RUT>
__device__ __forceinline__ bool mt_attempt_peek(bool run, const GammaState& g, RNT& N, RUT& U,
                                                uint32_t stream, const RoundKeys& rk,
                                                DevCounters* cnt, float* dv, uint32_t* zword,
                                                float* lboost = nullptr, bool* rechecked = nullptr) {
  float z = 0.0f;
  if (run) {
    z = N.peek(0);
    if constexpr (kZWord) *zword = N.peek_word(0);
    N.advance(1);
  }
  const float x = g.c * z;
  const bool series = fabsf(x) <= kSeriesMaxX;
  float t = 1.0f + x;
  bool tpos = t > 0.0f;
  const bool tclose = run && !series && fabsf(t) <= kTauT;
  if (tclose) {  // rare: the sign of t is re-decided in FP64 (z is N element pos-1)
    const Recheck r = mt_recheck64(g.alpha, N.pos() - 1, stream, rk.k[0][0], rk.k[0][1], 0.0f, 0);
    tpos = r.pass != 0;
    t = r.t;
  }
  const bool needu = run && tpos;
  bool acc = false, recheck = false;
  if (needu) {
    const float uo = U.peek(0) + 0x1p-24f;  // U' = U + 2^-24, exact
    U.advance(1);
    const float qh = mt_series_qhi(g.d, x);  // the log-free accept of mt_attempt
    if ((series && fmaf(qh, 1.00001f, uo) < 0x1.fffff8p-1f) || mt_squeeze(z, uo)) {
      acc = true;
    } else {
      const int r = kLargeShape ? mt_slow_call(g.alpha, g.d, x, z, t, uo, series, N.pos() - 1, stream,
                                               rk.k[0][0], rk.k[0][1], cnt)
                                : mt_slow(g.alpha, g.d, x, z, t, uo, series, N.pos() - 1, stream,
                                          rk.k[0][0], rk.k[0][1], cnt);
      acc = (r & 1) != 0;
      recheck = (r & 2) != 0;
    }
    float v = g.d * (t * t * t);
    if (acc && g.boost) {  // shapes below 1: Gamma(a + 1) U_b^(1/a), U_b after the accept
      const float ub = U.peek(0);
      U.advance(1);
      const float lb = __fdividef(flog(ub + 0x1p-24f), g.alpha);
      if constexpr (kLogBoost) *lboost = lb;
      else v = v * expf(lb);
    }
    *dv = v;
  }
  if (rechecked) *rechecked = tclose || recheck;
  else count_warp(&cnt->n_recheck, tclose || recheck);
  return acc;
}

}  // namespace brng
