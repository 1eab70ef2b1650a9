// brng_gamma.cuh -- Gamma(alpha, 1) attempts by Marsaglia & Tsang (2000),
// the irreducible distribution the paper builds from its Gaussian and uniform
// buffers (Sec. 2.2; its own GetGamma is withheld, Sec. 3 note).
//
// One call is ONE attempt for every lane with `run` (all lanes call it, so
// the ring refills stay warp-wide); callers loop until each lane accepted,
// which lets lanes that accepted move on to their next draw instead of
// idling while a neighbour retries.
//
// Precision: the attempt is computed in FP32 with the cancellation-free forms
//   1 - v = -x (3 + x (3 + x)),  ln v = 3 log1p(x),  x = c z,
// and its margin m = z^2/2 + d (1 - v + ln v) - ln u' decides when
// |m| > tol = 1e-5 (1 + S), S the sum of the magnitudes of the terms
// (plus d 3|x|/t for the sensitivity to z near t = 0).  The FP32 error of m is
// a few ulp of S (~1e-6 S), so the FP64 decision agrees whenever |m| > tol;
// otherwise the decision is recomputed in FP64 (brng_fp64.cuh) from the same
// Philox bits, in the reference operation order.  The sign of t is treated
// the same way when |t| <= 1e-5.  Both rechecks are counted; a recheck that
// overturns the FP32 sign records |m| / tol (which must stay below 1).
#pragma once

#include <cstdint>

#include "brng_fp64.cuh"
#include "brng_ring.cuh"

namespace brng {

constexpr int kGammaMaxAttempts = 64;
constexpr float kTauT = 1e-5f;
constexpr float kTauM = 1e-5f;

// Device counters (layout = brng_counters_t).
struct DevCounters {
  unsigned long long n_domain, n_reject, n_recheck, n_flip;
  unsigned int max_flip_ratio_bits;  // float bits (non-negative -> monotone as uint)
  unsigned int pad;
};

// warp-aggregated counter increment for lanes with `pred`
__device__ __forceinline__ void count_warp(unsigned long long* ctr, bool pred) {
  const unsigned m = __ballot_sync(kFull, pred);
  if (m && lane_id() == static_cast<unsigned>(__ffs(m) - 1)) atomicAdd(ctr, static_cast<unsigned long long>(__popc(m)));
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

// FP64 value of N element `idx` of `stream` (Box-Muller from its word pair)
__device__ __forceinline__ double gauss64_at(uint64_t idx, uint32_t stream, const RoundKeys& rk) {
  const uint4 w = philox_block(idx / 4, kDomN, stream, rk);
  const uint32_t slot = static_cast<uint32_t>(idx % 4);
  return slot < 2 ? dgauss(w.x, w.y, slot & 1) : dgauss(w.z, w.w, slot & 1);
}

static __device__ __noinline__ void record_flip(DevCounters* cnt, float ratio) {
  atomicAdd(&cnt->n_flip, 1ull);
  atomicMax(&cnt->max_flip_ratio_bits, __float_as_uint(ratio));
}

// One attempt.  Returns true for lanes that accepted; then *dv = d v (FP32).
// *zword gets the raw word of the N element used (for the first-word output).
template <class RN, class RU>
__device__ __forceinline__ bool mt_attempt(bool run, const GammaState& g, RN& N, RU& U,
                                           uint32_t stream, const RoundKeys& rk,
                                           DevCounters* cnt, float* dv, uint32_t* zword) {
  uint64_t zi = 0;
  const float z = N.get(run, stream, rk, zword, &zi);
  const float x = g.c * z;
  float t = 1.0f + x;
  bool tpos = t > 0.0f;
  double z64 = 0.0, d64 = 0.0, t64 = 0.0;
  bool have64 = false;
  const bool tclose = run && fabsf(t) <= kTauT;
  if (tclose) {  // rare: the sign of t is re-decided in FP64
    z64 = gauss64_at(zi, stream, rk);
    d64 = mt_d64(g.alpha);
    t64 = mt_t64(d64, z64);
    tpos = t64 > 0.0;
    have64 = true;
    t = static_cast<float>(t64);
  }
  count_warp(&cnt->n_recheck, tclose);
  const bool needu = run && tpos;
  const float u = U.get(needu, stream, rk);
  bool acc = false;
  bool recheck = false;
  if (needu) {
    const float uo = u + 0x1p-24f;  // U' = U + 2^-24, exact
    const float lnu = logf(uo);
    const float lnv = 3.0f * log1pf(x);
    const float omv = -x * fmaf(x, x + 3.0f, 3.0f);  // 1 - (1 + x)^3
    const float h = 0.5f * z * z;
    const float m = h + g.d * (omv + lnv) - lnu;
    const float S = h + g.d * (fabsf(omv) + fabsf(lnv) + 3.0f * fabsf(x) / t) + fabsf(lnu);
    const float tol = kTauM * (1.0f + S);
    if (fabsf(m) > tol) {
      acc = m > 0.0f;
    } else {
      recheck = true;
      if (!have64) {
        z64 = gauss64_at(zi, stream, rk);
        d64 = mt_d64(g.alpha);
        t64 = mt_t64(d64, z64);
      }
      acc = mt_accept64(d64, z64, t64, static_cast<double>(uo));
      if (isfinite(m) && acc != (m > 0.0f)) record_flip(cnt, fabsf(m) / tol);
    }
    *dv = g.d * (t * t * t);
  }
  count_warp(&cnt->n_recheck, recheck);
  return acc;
}

}  // namespace brng
