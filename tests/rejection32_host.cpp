// Host build of the large-mean discrete attempts (csrc/brng_rejection32.cuh
// and csrc/brng_fp64.cuh) for a CPU check of the certification: every
// attempt the FP32 / float-float path decides must be decided the same way,
// with the same count and the same number of elements, by the FP64 attempt.
//
// The device intrinsics are mapped to IEEE host operations with the same
// rounding (round to nearest, no contraction: build with -ffp-contract=off);
// logf and log1pf are the host library's, which have their own error of
// about one ulp, like CUDA's, so the bands are exercised against a second,
// independent implementation of the two functions.
//
// Usage: rejection32_host {ptrs|btrd} N seed
// Prints one JSON line: attempts, decided, undecided, accepted, mismatches.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#define __device__
#define __host__
#define __forceinline__ inline

static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fdiv_rn(float a, float b) { return a / b; }
static inline float __fsqrt_rn(float a) { return std::sqrt(a); }
static inline float __fmaf_rn(float a, float b, float c) { return std::fma(a, b, c); }
static inline double __dadd_rn(double a, double b) { return a + b; }
static inline double __dmul_rn(double a, double b) { return a * b; }
static inline double __ddiv_rn(double a, double b) { return a / b; }
static inline double __dsqrt_rn(double a) { return std::sqrt(a); }
static inline float __ull2float_rn(unsigned long long v) { return static_cast<float>(v); }
static inline float __ll2float_rn(long long v) { return static_cast<float>(v); }
static inline unsigned long long __float2ull_rn(float v) { return static_cast<unsigned long long>(std::nearbyint(v)); }
static inline uint32_t __float_as_uint(float f) {
  uint32_t u;
  std::memcpy(&u, &f, 4);
  return u;
}
static inline float __uint_as_float(uint32_t u) {
  float f;
  std::memcpy(&f, &u, 4);
  return f;
}
static inline long long __double_as_longlong(double d) {
  long long u;
  std::memcpy(&u, &d, 8);
  return u;
}
static inline double __longlong_as_double(long long u) {
  double d;
  std::memcpy(&d, &u, 8);
  return d;
}
using std::fabs;
using std::floor;

#include "brng_fp64.cuh"
#include "brng_rejection32.cuh"

static uint64_t g_state;
static uint64_t next64() {  // splitmix64
  uint64_t z = (g_state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static double unif() { return static_cast<double>(next64() >> 11) * 0x1p-53; }
static float grid_u() { return static_cast<float>(next64() >> 40) * 0x1p-24f; }  // [0, 1) on 2^-24

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  const bool ptrs = std::strcmp(argv[1], "ptrs") == 0;
  const long long N = std::atoll(argv[2]);
  g_state = std::strtoull(argv[3], nullptr, 10);
  long long decided = 0, undecided = 0, accepted = 0, mismatches = 0;
  for (long long i = 0; i < N; ++i) {
    const float u0 = grid_u(), u1 = grid_u();
    float k32, k64;
    int used32, used64 = 2;
    float p0, p1 = 0.0f;
    if (ptrs) {
      // lambda log-uniform in (64, 1e7], a few at the ends of the range
      p0 = i % 97 == 0 ? 64.00001f : (i % 89 == 0 ? 1e7f : static_cast<float>(64.0 * std::exp(unif() * std::log(1e7 / 64.0))));
      const brng::Attempt32 a = brng::ptrs_attempt32(p0, u0, u1 + 0x1p-24f);
      k32 = a.k;
      used32 = a.used;
      k64 = static_cast<float>(brng::ptrs_attempt64(p0, u0, static_cast<double>(u1) + 0x1p-24));
    } else {
      // n log-uniform in [129, 2^24], p uniform with n min(p, 1-p) > 64
      do {
        p0 = i % 101 == 0 ? 16777216.0f : std::floor(static_cast<float>(129.0 * std::exp(unif() * std::log(16777216.0 / 129.0))));
        p1 = i % 7 == 0 ? 0.5f : static_cast<float>(unif());
      } while (!(static_cast<double>(p0) * std::fmin(static_cast<double>(p1), 1.0 - static_cast<double>(p1)) > 64.0));
      const brng::Attempt32 a = brng::btrd_attempt32(p0, p1, u0, u1);
      k32 = a.k;
      used32 = a.used;
      k64 = static_cast<float>(brng::btrd_attempt64(p0, p1, static_cast<double>(u0) + 0x1p-24, u1, &used64));
    }
    if (k32 == brng::kUndecided) {
      ++undecided;
      continue;
    }
    ++decided;
    if (k32 >= 0.0f) ++accepted;
    if (k32 != k64 || used32 != used64) {
      if (mismatches < 5)
        std::fprintf(stderr, "mismatch p0=%a p1=%a u0=%a u1=%a k32=%.1f k64=%.1f used %d/%d\n", p0, p1, u0, u1,
                     k32, k64, used32, used64);
      ++mismatches;
    }
  }
  std::printf("{\"attempts\": %lld, \"decided\": %lld, \"undecided\": %lld, \"accepted\": %lld, \"mismatches\": %lld}\n",
              N, decided, undecided, accepted, mismatches);
  return 0;
}
