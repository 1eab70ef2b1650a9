// brng_engine.cuh -- core engine and base conversions on the device.
//
// Core engine: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, "Parallel Random
// Numbers: As Easy as 1, 2, 3", SC'11): ten rounds of two 32x32->64-bit
// multiplies by the published multipliers, XOR of the high halves into the
// other counter words and the round key, key bumped by the published Weyl
// increments.  It plays the part of the paper's vectorised core engine
// (Sec. 2.2); being counter-based, element j of any stream is computable
// directly, so buffers are pure caches of a fixed sequence.
//
// The round keys are computed once per launch on the host and passed in the
// kernel parameter block, so every XOR with a key reads the constant bank.
#pragma once

#include <cstdint>

#include "brng_fp32.cuh"

namespace brng {

constexpr uint32_t kPhiloxM0 = 0xD2511F53u;
constexpr uint32_t kPhiloxM1 = 0xCD9E8D57u;
constexpr uint32_t kPhiloxW0 = 0x9E3779B9u;
constexpr uint32_t kPhiloxW1 = 0xBB67AE85u;

constexpr uint32_t kDomU = 0, kDomN = 1, kDomE = 2, kDomData = 3, kDomU64 = 4;
constexpr uint32_t kDomZ = 5;  // the full LDA step's topic draws

// Round keys (k0 + r W0, k1 + r W1), r = 0..9.
struct RoundKeys {
  uint32_t k[10][2];
};

inline RoundKeys make_round_keys(uint64_t seed) {
  RoundKeys rk;
  uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
  for (int r = 0; r < 10; ++r) {
    rk.k[r][0] = k0;
    rk.k[r][1] = k1;
    k0 += kPhiloxW0;
    k1 += kPhiloxW1;
  }
  return rk;
}

// One 32x32 -> 64-bit product, both halves: written as a widening multiply
// so that it is a single wide multiply-add instruction rather than separate
// high-half and low-half multiplies.
__device__ __forceinline__ void mul_hilo(uint32_t m, uint32_t x, uint32_t& hi, uint32_t& lo) {
  const uint64_t p = static_cast<uint64_t>(m) * x;
  hi = static_cast<uint32_t>(p >> 32);
  lo = static_cast<uint32_t>(p);
}

__device__ __forceinline__ uint4 philox(uint4 c, const RoundKeys& rk) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mul_hilo(kPhiloxM0, c.x, hi0, lo0);
    mul_hilo(kPhiloxM1, c.z, hi1, lo1);
    c = make_uint4(hi1 ^ c.y ^ rk.k[r][0], lo1, hi0 ^ c.w ^ rk.k[r][1], lo0);
  }
  return c;
}

// counter of block `blk` of (domain, stream)
__device__ __forceinline__ uint4 philox_ctr(uint64_t blk, uint32_t dom, uint32_t stream) {
  return make_uint4(static_cast<uint32_t>(blk), dom, stream, static_cast<uint32_t>(blk >> 32));
}

__device__ __forceinline__ uint4 philox_block(uint64_t blk, uint32_t dom, uint32_t stream,
                                              const RoundKeys& rk) {
  return philox(philox_ctr(blk, dom, stream), rk);
}

// Round 0 multiplies counter word 2 (the stream) by M1, so for a fixed
// (domain, stream) its half of round 0's output, (hi(M1 s) ^ dom ^ k0, lo(M1 s)),
// is the same for every block: computed once per stream it leaves one
// multiply and one XOR per block.  philox_block_sh(blk, philox_stream_half(
// dom, s, rk), rk) == philox_block(blk, dom, s, rk) bit for bit.
__device__ __forceinline__ uint2 philox_stream_half(uint32_t dom, uint32_t stream, const RoundKeys& rk) {
  uint32_t hi1, lo1;
  mul_hilo(kPhiloxM1, stream, hi1, lo1);
  return make_uint2(hi1 ^ dom ^ rk.k[0][0], lo1);
}

__device__ __forceinline__ uint4 philox_block_sh(uint64_t blk, uint2 sh, const RoundKeys& rk) {
  const uint32_t lo = static_cast<uint32_t>(blk), hi = static_cast<uint32_t>(blk >> 32);
  uint32_t h0, l0;
  mul_hilo(kPhiloxM0, lo, h0, l0);
  uint4 c = make_uint4(sh.x, sh.y, h0 ^ hi ^ rk.k[0][1], l0);
#pragma unroll
  for (int r = 1; r < 10; ++r) {
    uint32_t hi0, lo0, hi1, lo1;
    mul_hilo(kPhiloxM0, c.x, hi0, lo0);
    mul_hilo(kPhiloxM1, c.z, hi1, lo1);
    c = make_uint4(hi1 ^ c.y ^ rk.k[r][0], lo1, hi0 ^ c.w ^ rk.k[r][1], lo0);
  }
  return c;
}

// ---- FP32 base conversions (brng_fp32.cuh: no conversion instructions) ----
// Box-Muller pair from (w0, w1): radius from U'(w0), angle 2 pi U(w1) =
// pi (w1 >> 8) 2^-23
__device__ __forceinline__ float2 box_muller(uint32_t w0, uint32_t w1) {
  const float q = -2.0f * flog(u01_open(w0));  // >= 0; 0 only for U' = 1
  // sqrt(q) = q / sqrt(q); for U' < 1, q >= -2 ln(1 - 2^-24) > FLT_MIN, and
  // q = 0 gives 0 * rsqrt(FLT_MIN) = 0
  const float r = q * rsqrtf(fmaxf(q, 0x1p-126f));
  float s, c;
  fsincospi_k(w1 >> 8, &s, &c);
  return make_float2(r * c, r * s);
}

__device__ __forceinline__ float exp1(uint32_t w) { return -flog(u01_open(w)); }

// 53-bit uniform from two words: ((w0>>5) 2^26 + (w1>>6)) 2^-53, exact.
// Built from the bits with integer operations only (normalise the 53-bit
// integer m, then set the exponent), since GB300's FP64 pipe is narrow: the
// value m 2^-53 is exactly representable, so this is the same double a
// conversion and a multiply would give.
__device__ __forceinline__ double u53(uint32_t w0, uint32_t w1) {
  const unsigned long long m =
      (static_cast<unsigned long long>(w0 >> 5) << 26) | static_cast<unsigned long long>(w1 >> 6);
  if (m == 0) return 0.0;
  const int sh = __clzll(m) - 11;  // bit 52 becomes the leading one
  const unsigned long long mant = m << sh;
  const unsigned long long bits =
      (static_cast<unsigned long long>(1022 - sh) << 52) | (mant & 0xFFFFFFFFFFFFFull);
  return __longlong_as_double(static_cast<long long>(bits));
}

}  // namespace brng
