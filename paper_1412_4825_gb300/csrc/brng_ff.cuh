// brng_ff.cuh -- float-float ("double-word") arithmetic: a value is the
// unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2, about 48
// significant bits, carried in FP32 operations only.
//
// Why: GB300 issues FP64 at a small fraction of its FP32 rate, and the
// large-mean discrete samplers (Hormann's PTRS and BTRD) need a few of their
// per-draw constants and the floor of the hat transform to well beyond FP32
// precision to certify that their result equals an FP64 evaluation.  Every
// operation is written with explicit round-to-nearest intrinsics (no FMA
// contraction, no reassociation), so each is the algorithm as stated.
//
// The algorithms are the classical error-free transforms (Knuth's TwoSum,
// Dekker's FastTwoSum, the FMA product error) and the double-word operations
// analysed by Joldes, Muller and Popescu ("Tight and rigorous error bounds
// for basic building blocks of double-word arithmetic", ACM TOMS 44, 2017),
// with u = 2^-24 the FP32 unit roundoff and no underflow:
//   ff_add (both words, any signs)   relative error <= 3u^2 / (1 - 4u)
//   ff_add_f (word + float)          <= 2u^2
//   ff_mul (word x word, with FMA)   <= 5u^2
//   ff_mul_f (word x float, FMA)     <= 2u^2
//   ff_div_f (word / float)          <= 3u^2
//   ff_div (word / word)             <= 15u^2 + 56u^3
//   ff_sqrt (of a word)              <= 25u^2 / 8
// Callers budget 2^-40 (256 u^2, several times the largest) per operation.
#pragma once

#include <cuda_runtime.h>

namespace brng {

// the result of a certified decision that its error bound did not allow
// (the caller takes the next, more precise tier)
constexpr float kUndecided = -2.0f;

struct FF {
  float hi, lo;
};

// a + b exactly as s + t (any magnitudes)
__device__ __forceinline__ FF two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float ap = __fadd_rn(s, -b);
  const float bp = __fadd_rn(s, -ap);
  const float da = __fadd_rn(a, -ap);
  const float db = __fadd_rn(b, -bp);
  return FF{s, __fadd_rn(da, db)};
}

// a + b exactly as s + t, given |a| >= |b| (or a = 0)
__device__ __forceinline__ FF fast_two_sum(float a, float b) {
  const float s = __fadd_rn(a, b);
  const float z = __fadd_rn(s, -a);
  return FF{s, __fadd_rn(b, -z)};
}

// a b exactly as p + e (FMA gives the product's rounding error)
__device__ __forceinline__ FF two_prod(float a, float b) {
  const float p = __fmul_rn(a, b);
  return FF{p, __fmaf_rn(a, b, -p)};
}

__device__ __forceinline__ FF ff_neg(FF x) { return FF{-x.hi, -x.lo}; }
__device__ __forceinline__ FF ff_abs(FF x) { return x.hi < 0.0f ? ff_neg(x) : x; }
__device__ __forceinline__ FF ff_scale2(FF x) { return FF{__fmul_rn(2.0f, x.hi), __fmul_rn(2.0f, x.lo)}; }  // exact

__device__ __forceinline__ FF ff_add_f(FF x, float y) {
  const FF s = two_sum(x.hi, y);
  return fast_two_sum(s.hi, __fadd_rn(x.lo, s.lo));
}

__device__ __forceinline__ FF ff_add(FF x, FF y) {
  const FF s = two_sum(x.hi, y.hi);
  const FF t = two_sum(x.lo, y.lo);
  const FF v = fast_two_sum(s.hi, __fadd_rn(s.lo, t.hi));
  return fast_two_sum(v.hi, __fadd_rn(t.lo, v.lo));
}

__device__ __forceinline__ FF ff_sub(FF x, FF y) { return ff_add(x, ff_neg(y)); }

__device__ __forceinline__ FF ff_mul_f(FF x, float y) {
  const FF c = two_prod(x.hi, y);
  return fast_two_sum(c.hi, __fmaf_rn(x.lo, y, c.lo));
}

__device__ __forceinline__ FF ff_mul(FF x, FF y) {
  const FF c = two_prod(x.hi, y.hi);
  const float t0 = __fmul_rn(x.lo, y.lo);
  const float t1 = __fmaf_rn(x.hi, y.lo, t0);
  const float c2 = __fmaf_rn(x.lo, y.hi, t1);
  return fast_two_sum(c.hi, __fadd_rn(c.lo, c2));
}

__device__ __forceinline__ FF ff_div_f(FF x, float y) {
  const float th = __fdiv_rn(x.hi, y);
  const FF pi = two_prod(th, y);
  const float dh = __fadd_rn(x.hi, -pi.hi);  // exact
  const float d = __fadd_rn(__fadd_rn(dh, -pi.lo), x.lo);
  return fast_two_sum(th, __fdiv_rn(d, y));
}

__device__ __forceinline__ FF ff_div(FF x, FF y) {
  const float th = __fdiv_rn(x.hi, y.hi);
  const FF r = ff_mul_f(y, th);
  const float ph = __fadd_rn(x.hi, -r.hi);
  const float dl = __fadd_rn(x.lo, -r.lo);
  const float d = __fadd_rn(ph, dl);
  return fast_two_sum(th, __fdiv_rn(d, y.hi));
}

// sqrt(x.hi + x.lo), x > 0: the residual of the rounded root is exact by FMA
__device__ __forceinline__ FF ff_sqrt(FF x) {
  const float sh = __fsqrt_rn(x.hi);
  const float rho = __fadd_rn(__fmaf_rn(-sh, sh, x.hi), x.lo);
  return fast_two_sum(sh, __fdiv_rn(rho, __fmul_rn(2.0f, sh)));
}

__device__ __forceinline__ FF ff_from(float x) { return FF{x, 0.0f}; }

// The double-word nearest a double constant (within 2^-48 relative); used
// for the FP64 constants of the reference formulas.
__host__ __device__ constexpr FF ff_const(double d) {
  return FF{static_cast<float>(d), static_cast<float>(d - static_cast<double>(static_cast<float>(d)))};
}

// floor(x.hi + x.lo) exactly, for |x.hi| < 2^24
__device__ __forceinline__ float ff_floor(FF x) {
  const float f = floorf(x.hi);
  return (f == x.hi && x.lo < 0.0f) ? __fadd_rn(f, -1.0f) : f;
}

// Distance from x to the nearest integer, given fx = ff_floor(x), as a float
// (rounded; callers' bands cover the rounding).
__device__ __forceinline__ float ff_frac_gap(FF x, float fx) {
  const float below = ff_add_f(x, -fx).hi;  // x - floor(x) in [0, 1)
  return fminf(below, __fadd_rn(1.0f, -below));
}

}  // namespace brng
