// brng_inversion.cuh -- Poisson and Binomial by inversion of one U element
// (the small-mean discrete draws): the FP32 and double-single tiers, as pure
// functions (no FP64, no device state), shared by the bulk kernels and a
// host build of this header that checks them against the FP64 inversion.
//
// A draw is the smallest k with u < F(k), F the CDF summed left to right from
// p_0 by the pmf recurrence; the reference evaluates it in FP64 in a fixed
// operation order (brng_fp64.cuh: poisson_inv64, binomial_inv64).  Each tier
// takes the two comparisons that fix k (u < F(k), u >= F(k-1)) only when u
// lies beyond a band of at least twice its bound on the error of F, relative
// to F (every term is positive and carries p_0's relative error); otherwise it
// returns kUndecided and the caller takes the next tier, FP64 last.  u is a U
// element on the 2^-24 grid; u = 2^-24 below is the FP32 unit roundoff.
//
//   FP32 tier (every draw; a warp runs each search step for all its
//   searching lanes, so a step must be cheap): Poisson p_0 = expf(-lambda)
//   (2 ulp: 4u), p_k = (p_{k-1} lambda) / k, so F(k) is within (4 + 3k) u,
//   band (16 + 8k) u.  Binomial on q = min(p, 1 - p) (n - k when p > 1/2):
//   p_0 = expf(a), a = n log1pf(-q) ((3|a| + 4) u: log1pf 1 ulp, the product,
//   expf), r = q / (1 - q) from the rounded 1 - q (2u), p_k = (p_{k-1}
//   ((n - k + 1) r)) / k (3 roundings more a step), so F(k) is within
//   (3|a| + 4 + 6k) u, band (6|a| + 16 + 14k) u + 2^-30; p_0 below 2^-125
//   (next to the subnormal range, where a rounding is no longer relative)
//   decides nothing.
//
//   Double-single tier (the draws the FP32 tier left, about one in a
//   thousand): a value is hi + lo, each operation's rounding error carried
//   in lo through FMA, so the recurrence and the sums add only O(k u^2) and
//   p_0's own error remains: band 8u + 2^-30 (Poisson) and (6|a| + 8) u +
//   2^-30 (Binomial).
#pragma once

#include <cstdint>

#include "brng_ff.cuh"

namespace brng {

// ---- FP32 tier -----------------------------------------------------------------

// The decision on a finished FP32 search (k, F(k), F(k-1)): k, or kUndecided.
__device__ __forceinline__ float poisson_decide32(float u, float k, float F, float Fprev, bool ran_out) {
  const float rel = (16.0f + 8.0f * k) * 0x1p-24f;
  const bool sure = !ran_out && (F - u > rel * F) && (k == 0.0f || u - Fprev > rel * Fprev);
  return sure ? k : kUndecided;
}

// The whole FP32 search: k, or kUndecided.
__device__ __forceinline__ float poisson_inv32(float lambda, float u, int kmax) {
  float p = expf(-lambda);
  float F = p, Fprev = 0.0f;
  int k = 0;
  bool ran_out = false;
  while (!(u < F)) {
    if (k >= kmax) {
      ran_out = true;
      break;
    }
    ++k;
    p = (p * lambda) / static_cast<float>(k);
    Fprev = F;
    if (p == 0.0f) {
      ran_out = true;
      break;
    }
    F = F + p;
  }
  return poisson_decide32(u, static_cast<float>(k), F, Fprev, ran_out);
}

__device__ __forceinline__ float binomial_q(float p) { return p > 0.5f ? 1.0f - p : p; }  // exact
__device__ __forceinline__ float binomial_ratio(float p) {
  const float q = binomial_q(p);
  return __fdiv_rn(q, 1.0f - q);
}
__device__ __forceinline__ float binomial_p0(float n, float p) { return expf(n * log1pf(-binomial_q(p))); }

// The decision on a finished FP32 search (k counted on q): the draw (n - k
// when p > 1/2), or kUndecided.
__device__ __forceinline__ float binomial_decide32(float n, float p, float u, float k, float F, float Fprev,
                                                   bool ran_out) {
  const float a = n * log1pf(-binomial_q(p));
  const float rel = (6.0f * fabsf(a) + 16.0f + 14.0f * k) * 0x1p-24f + 0x1p-30f;
  const bool sure = !ran_out && (F - u > rel * F) && (k == 0.0f || u - Fprev > rel * Fprev);
  if (!sure) return kUndecided;
  return p > 0.5f ? n - k : k;
}

__device__ __forceinline__ float binomial_inv32(float n, float p, float u) {
  const float r = binomial_ratio(p);
  float pk = binomial_p0(n, p);
  float F = pk, Fprev = 0.0f, k = 0.0f;
  bool ran_out = !(pk >= 0x1p-125f);
  while (!ran_out && !(u < F)) {
    if (k >= n) {
      ran_out = true;
      break;
    }
    k += 1.0f;
    pk = (pk * (((n - k) + 1.0f) * r)) / k;
    Fprev = F;
    if (pk == 0.0f) {
      ran_out = true;
      break;
    }
    F = F + pk;
  }
  return binomial_decide32(n, p, u, k, F, Fprev, ran_out);
}

// ---- double-single tier ----------------------------------------------------------

struct DS {
  float hi, lo;
};
__device__ __forceinline__ DS ds_norm(float a, float b) {  // |a| >= |b|
  const float s = a + b;
  return DS{s, b - (s - a)};
}
__device__ __forceinline__ DS ds_mul(DS x, float b) {  // (x.hi + x.lo) b
  const float p = x.hi * b;
  const float e = fmaf(x.hi, b, -p);  // exact product error
  return ds_norm(p, fmaf(x.lo, b, e));
}
__device__ __forceinline__ DS ds_mul(DS x, DS y) {
  const float p = x.hi * y.hi;
  const float e = fmaf(x.hi, y.hi, -p);
  return ds_norm(p, fmaf(x.hi, y.lo, fmaf(x.lo, y.hi, e)));
}
__device__ __forceinline__ DS ds_div(DS x, float k) {  // (x.hi + x.lo) / k, k > 0
  const float q1 = __fdividef(x.hi, k);
  const float r = fmaf(-q1, k, x.hi) + x.lo;  // remainder (first part exact)
  return ds_norm(q1, __fdividef(r, k));
}
__device__ __forceinline__ DS ds_add(DS x, DS y) {  // both >= 0
  const float s = x.hi + y.hi;
  const float bb = s - x.hi;
  const float e = (x.hi - (s - bb)) + (y.hi - bb);  // exact sum error
  return ds_norm(s, e + x.lo + y.lo);
}
// (u - F) as one float, F = hi + lo
__device__ __forceinline__ float ds_gap(float u, DS F) { return (u - F.hi) - F.lo; }

// The double-single Poisson search: k, or kUndecided.
__device__ __forceinline__ float poisson_inv_ds(float lambda, float u, int kmax) {
  DS pk{expf(-lambda), 0.0f};
  DS F = pk, Fprev{0.0f, 0.0f};
  float k = 0.0f;
  bool ran_out = false;
  while (!(ds_gap(u, F) < 0.0f)) {
    if (k >= static_cast<float>(kmax)) {
      ran_out = true;
      break;
    }
    k += 1.0f;
    pk = ds_div(ds_mul(pk, lambda), k);
    Fprev = F;
    if (pk.hi == 0.0f) {
      ran_out = true;
      break;
    }
    F = ds_add(F, pk);
  }
  const float rel = 8.0f * 0x1p-24f + 0x1p-30f;
  const bool sure = !ran_out && -ds_gap(u, F) > rel * F.hi && (k == 0.0f || ds_gap(u, Fprev) > rel * Fprev.hi);
  return sure ? k : kUndecided;
}

// The double-single Binomial search: the draw, or kUndecided.
__device__ __forceinline__ float binomial_inv_ds(float n, float p, float u) {
  const bool flip = p > 0.5f;
  const float q = flip ? 1.0f - p : p;  // exact for p in (1/2, 1]
  const float a = n * log1pf(-q);
  const float omq_hi = 1.0f - q;
  const DS omq{omq_hi, (1.0f - omq_hi) - q};  // 1 - q exactly
  const float r1 = __fdividef(q, omq.hi);
  const DS r = ds_norm(r1, __fdividef(fmaf(-r1, omq.hi, q) - r1 * omq.lo, omq.hi));
  DS pk{expf(a), 0.0f};
  DS F = pk, Fprev{0.0f, 0.0f};
  float k = 0.0f;
  bool ran_out = false;
  while (!(ds_gap(u, F) < 0.0f)) {
    if (k >= n) {
      ran_out = true;
      break;
    }
    k += 1.0f;
    pk = ds_div(ds_mul(pk, ds_mul(r, (n - k) + 1.0f)), k);
    Fprev = F;
    if (pk.hi == 0.0f) {
      ran_out = true;
      break;
    }
    F = ds_add(F, pk);
  }
  // all terms carry p_0's relative error: the band scales with F
  const float rel = (6.0f * fabsf(a) + 8.0f) * 0x1p-24f + 0x1p-30f;
  const bool sure = !ran_out && -ds_gap(u, F) > rel * F.hi && (k == 0.0f || ds_gap(u, Fprev) > rel * Fprev.hi);
  if (!sure) return kUndecided;
  return flip ? n - k : k;
}

}  // namespace brng
