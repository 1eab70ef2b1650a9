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
// Usage: rejection32_host {ptrs|btrd|ptrs_edges|btrd_edges} N seed
// Prints one JSON line: attempts, decided, undecided, accepted, mismatches.
// The *_edges modes place attempts next to the decisions' boundaries.
//
// The small-mean inversions (csrc/brng_inversion.cuh) the same way:
//   rejection32_host {inv|inv_edges} N seed -- N Poisson and N Binomial
//   draws through the FP32 tier, then the double-single tier, each decided
//   draw against the FP64 inversion (inv_edges: u next to a CDF step).
//
// And the float-float arithmetic the certified decisions rest on
// (csrc/brng_ff.cuh): rejection32_host ffops N seed -- the largest relative
// error of each operation on random operands (cancelling sums included),
// against wider arithmetic, in units of u^2 = 2^-48.
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <algorithm>

#define __device__
#define __host__
#define __forceinline__ inline

static inline float __fadd_rn(float a, float b) { return a + b; }
static inline float __fmul_rn(float a, float b) { return a * b; }
static inline float __fdiv_rn(float a, float b) { return a / b; }
static inline float __fdividef(float a, float b) { return a / b; }  // the device one is within 2 ulp
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
#include "brng_inversion.cuh"

static uint64_t g_state;
static uint64_t next64() {  // splitmix64
  uint64_t z = (g_state += 0x9e3779b97f4a7c15ull);
  z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
  z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
  return z ^ (z >> 31);
}
static double unif() { return static_cast<double>(next64() >> 11) * 0x1p-53; }
static float grid_u() { return static_cast<float>(next64() >> 40) * 0x1p-24f; }  // [0, 1) on 2^-24

struct Tally {
  long long attempts = 0, decided = 0, undecided = 0, accepted = 0, mismatches = 0;
  void check(float k32, int used32, float k64, int used64, float p0, float p1, float u0, float u1) {
    ++attempts;
    if (k32 == brng::kUndecided) {
      ++undecided;
      return;
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
};

static float ptrs64(float lam, float u0, float u1) {
  return static_cast<float>(brng::ptrs_attempt64(lam, u0, static_cast<double>(u1) + 0x1p-24));
}
static float btrd64(float n, float p, float u0, float u1, int* used) {
  return static_cast<float>(brng::btrd_attempt64(n, p, static_cast<double>(u0) + 0x1p-24, u1, used));
}
static float grid(uint32_t j) { return static_cast<float>(j) * 0x1p-24f; }

// The smallest grid index j in [lo, hi] at which pred(j) turns true (pred is
// monotone false -> true on the range), or hi + 1.
template <class P>
static uint32_t first_true(uint32_t lo, uint32_t hi, P pred) {
  if (!pred(hi)) return hi + 1;
  while (lo < hi) {
    const uint32_t mid = lo + (hi - lo) / 2;
    if (pred(mid)) hi = mid;
    else lo = mid + 1;
  }
  return lo;
}

// Attempts placed next to the decisions' boundaries, found on the FP64
// attempt by bisection over the 2^-24 grid: where floor(X) steps to the next
// integer, where the squeeze's threshold on v lies, and where the log test
// turns from accept to reject.  Every decided attempt there must still equal
// the FP64 attempt.
static void edges(bool ptrs, long long N, Tally& t) {
  for (long long i = 0; i < N; ++i) {
    const int kind = static_cast<int>(next64() % 3);
    if (ptrs) {
      const float lam = static_cast<float>(64.0 * std::exp(unif() * std::log(1e7 / 64.0)));
      uint32_t j0;
      float u1;
      if (kind == 0) {  // floor(X) steps: X increases with u0; take u0 in the squeeze region, v small
        u1 = 0.0f;
        const float ref = ptrs64(lam, grid(1u << 23), u1);  // k at u0 = 1/2
        const float target = ref + static_cast<float>(static_cast<int>(next64() % 41) - 20);
        j0 = first_true(1174406u, (1u << 24) - 1174406u, [&](uint32_t j) { return ptrs64(lam, grid(j), u1) >= target; });
        for (int d = -3; d <= 3; ++d) {
          const uint32_t j = j0 + d;
          const brng::Attempt32 a = brng::ptrs_attempt32(lam, grid(j), u1 + 0x1p-24f);
          t.check(a.k, a.used, ptrs64(lam, grid(j), u1), 2, lam, 0.0f, grid(j), u1);
        }
      } else if (kind == 1) {  // the squeeze's v <= v_r: accept turns to the log test as v grows
        const float u0 = grid(static_cast<uint32_t>(1174406u + next64() % 6000000u));
        const uint32_t m = first_true(0u, (1u << 24) - 1u, [&](uint32_t m) {
          const brng::Attempt32 a = brng::ptrs_attempt32(lam, u0, grid(m) + 0x1p-24f);
          return a.k == brng::kUndecided || ptrs64(lam, u0, grid(m)) < 0.0f;
        });
        for (int d = -4; d <= 4; ++d) {
          const uint32_t mm = static_cast<uint32_t>(std::min<long long>(std::max<long long>(m + d, 0), (1 << 24) - 1));
          const brng::Attempt32 a = brng::ptrs_attempt32(lam, u0, grid(mm) + 0x1p-24f);
          t.check(a.k, a.used, ptrs64(lam, u0, grid(mm)), 2, lam, 0.0f, u0, grid(mm));
        }
      } else {  // the log test: us in [0.013, 0.07), accept for v below a threshold
        const uint32_t ju = static_cast<uint32_t>(218104u + next64() % (1174406u - 218104u));
        const float u0 = (next64() & 1) ? grid(ju) : grid((1u << 24) - ju);
        const uint32_t m = first_true(0u, (1u << 24) - 1u, [&](uint32_t m) { return ptrs64(lam, u0, grid(m)) < 0.0f; });
        for (int d = -4; d <= 4; ++d) {
          const uint32_t mm = static_cast<uint32_t>(std::min<long long>(std::max<long long>(m + d, 0), (1 << 24) - 1));
          const brng::Attempt32 a = brng::ptrs_attempt32(lam, u0, grid(mm) + 0x1p-24f);
          t.check(a.k, a.used, ptrs64(lam, u0, grid(mm)), 2, lam, 0.0f, u0, grid(mm));
        }
      }
    } else {
      float n, p;
      do {
        n = std::floor(static_cast<float>(129.0 * std::exp(unif() * std::log(16777216.0 / 129.0))));
        p = static_cast<float>(unif());
      } while (!(static_cast<double>(n) * std::fmin(static_cast<double>(p), 1.0 - static_cast<double>(p)) > 64.0));
      int used = 0;
      if (kind == 0) {  // the immediate accept's floor(X) steps: X increases with v (u1 unused)
        const float ref = btrd64(n, p, grid(1u << 22), 0.0f, &used);
        if (ref < 0.0f || used != 1) continue;
        const float base = p > 0.5f ? n - ref : ref;
        const float target = base + static_cast<float>(static_cast<int>(next64() % 21) - 10);
        const uint32_t m = first_true(0u, 1u << 23, [&](uint32_t m) {
          int us = 0;
          const float k = btrd64(n, p, grid(m), 0.0f, &us);
          return us != 1 || (p > 0.5f ? n - k : k) >= target;
        });
        for (int d = -3; d <= 3; ++d) {
          const uint32_t mm = static_cast<uint32_t>(std::max<long long>(m + d, 0));
          int u64 = 0;
          const float k64 = btrd64(n, p, grid(mm), 0.0f, &u64);
          const brng::Attempt32 a = brng::btrd_attempt32(n, p, grid(mm), 0.0f);
          t.check(a.k, a.used, k64, u64, n, p, grid(mm), 0.0f);
        }
      } else {  // the thresholds 0.86 v_r and v_r on v, and the accept test beyond v_r
        const float u1 = grid(static_cast<uint32_t>(next64() >> 40));
        const double pq = p > 0.5f ? 1.0 - static_cast<double>(p) : static_cast<double>(p);
        const double b = 1.15 + 2.53 * std::sqrt(static_cast<double>(n) * pq * (1.0 - pq));
        const double vr = 0.92 - 4.2 / b;
        uint32_t m;
        if (kind == 1) {
          const int which = static_cast<int>(next64() % 2);
          if (which == 0) {  // 0.86 v_r: one element below, two above
            m = first_true(0u, (1u << 24) - 1u, [&](uint32_t mm) {
              int us = 0;
              btrd64(n, p, grid(mm), u1, &us);
              return us == 2;
            });
          } else {  // v_r (v = u0 + 2^-24)
            m = static_cast<uint32_t>(std::ceil(vr * 16777216.0)) - 1u;
          }
        } else {  // beyond v_r the element u1 fixes k; the test turns from accept to reject as v grows
          const uint32_t lo = static_cast<uint32_t>(std::ceil(vr * 16777216.0)) + 1u;
          int us = 0;
          if (btrd64(n, p, grid(lo), u1, &us) < 0.0f) continue;  // k outside or rejected everywhere
          m = first_true(lo, (1u << 24) - 1u, [&](uint32_t mm) {
            int u2 = 0;
            return btrd64(n, p, grid(mm), u1, &u2) < 0.0f;
          });
        }
        for (int d = -4; d <= 4; ++d) {
          const uint32_t mm = static_cast<uint32_t>(std::min<long long>(std::max<long long>(static_cast<long long>(m) + d, 0),
                                                                       (1 << 24) - 1));
          int u64 = 0;
          const float k64 = btrd64(n, p, grid(mm), u1, &u64);
          const brng::Attempt32 a = brng::btrd_attempt32(n, p, grid(mm), u1);
          t.check(a.k, a.used, k64, u64, n, p, grid(mm), u1);
        }
      }
    }
  }
}

// ---- the small-mean inversions -------------------------------------------------
struct InvTally {
  long long draws = 0, decided32 = 0, decided_ds = 0, undecided = 0, mismatches = 0;
  // one draw through both tiers, checked against FP64
  void run(bool poisson, float a, float b, float u) {
    ++draws;
    const float ref = poisson ? static_cast<float>(brng::poisson_inv64(a, u, 1024))
                              : static_cast<float>(brng::binomial_inv64(a, b, u));
    float k = poisson ? brng::poisson_inv32(a, u, 1024) : brng::binomial_inv32(a, b, u);
    if (k != brng::kUndecided) {
      ++decided32;
    } else {
      k = poisson ? brng::poisson_inv_ds(a, u, 1024) : brng::binomial_inv_ds(a, b, u);
      if (k == brng::kUndecided) {
        ++undecided;
        return;
      }
      ++decided_ds;
    }
    if (k != ref) {
      if (mismatches < 5)
        std::fprintf(stderr, "inversion mismatch %s a=%a b=%a u=%a k=%.1f fp64=%.1f\n", poisson ? "poisson" : "binomial",
                     a, b, u, k, ref);
      ++mismatches;
    }
  }
};

// Poisson lambda log-uniform in [0.05, 64]; Binomial n log-uniform integers
// in [1, 2^24] and p uniform with n min(p, 1 - p) <= 64 (a few at the ends)
static float rand_lambda(long long i) {
  if (i % 97 == 0) return 64.0f;
  return static_cast<float>(0.05 * std::exp(unif() * std::log(64.0 / 0.05)));
}
static void rand_binomial(long long i, float* n, float* p) {
  do {
    *n = i % 101 == 0 ? 16777216.0f : std::floor(static_cast<float>(std::exp(unif() * std::log(16777216.0))));
    *p = i % 7 == 0 && *n <= 128.0f ? 0.5f : static_cast<float>(unif());
  } while (!(static_cast<double>(*n) * std::fmin(static_cast<double>(*p), 1.0 - static_cast<double>(*p)) <= 64.0));
}

static void inversions(bool at_steps, long long N, InvTally& t) {
  for (long long i = 0; i < N; ++i) {
    const float lam = rand_lambda(i);
    float n, p;
    rand_binomial(i, &n, &p);
    if (!at_steps) {
      t.run(true, lam, 0.0f, grid_u());
      t.run(false, n, p, grid_u());
      continue;
    }
    // u on the grid points next to a step of the CDF: the first one whose
    // FP64 draw passes a count near the middle of the distribution, and its
    // neighbours
    const uint32_t mid = 1u << 23;
    const float kp = static_cast<float>(brng::poisson_inv64(lam, grid(mid), 1024)) +
                     static_cast<float>(static_cast<int>(next64() % 5) - 2);
    uint32_t j = first_true(0u, (1u << 24) - 1u, [&](uint32_t m) { return brng::poisson_inv64(lam, grid(m), 1024) > kp; });
    for (int d = -3; d <= 3; ++d)
      if (static_cast<long long>(j) + d >= 0 && j + d < (1u << 24)) t.run(true, lam, 0.0f, grid(j + d));
    const bool flip = p > 0.5f;  // the draw falls as u grows when p > 1/2
    const float kb = static_cast<float>(brng::binomial_inv64(n, p, grid(mid))) +
                     static_cast<float>(static_cast<int>(next64() % 5) - 2);
    j = first_true(0u, (1u << 24) - 1u, [&](uint32_t m) {
      const float k = static_cast<float>(brng::binomial_inv64(n, p, grid(m)));
      return flip ? k < kb : k > kb;
    });
    for (int d = -3; d <= 3; ++d)
      if (static_cast<long long>(j) + d >= 0 && j + d < (1u << 24)) t.run(false, n, p, grid(j + d));
  }
}

// ---- float-float operations against wider arithmetic -------------------------------
// The references: a quad-precision type where the compiler has one (the sums
// of nearly cancelling operands need every bit of both words: hi + lo spans
// up to ~110 bits here), else long double; products, quotients and roots
// only need the inputs to ~2^-64, which long double gives.
#if defined(__x86_64__) && defined(__GNUC__)
using wide_t = __float128;
#else
using wide_t = long double;
#endif
// A random double-word: hi with a random exponent in [-30, 30], lo within half
// an ulp of hi and not below 2^-60 of it (normalised through fast_two_sum).
static brng::FF rand_ff() {
  const float hi = static_cast<float>(std::ldexp(1.0 + unif(), static_cast<int>(next64() % 61) - 30)) *
                   ((next64() & 1) ? -1.0f : 1.0f);
  const double frac = std::ldexp(1.0 + unif(), -1 - static_cast<int>(next64() % 36));  // [2^-36, 1) / 2
  const float lo = static_cast<float>(((next64() & 1) ? -frac : frac) * std::ldexp(1.0, std::ilogb(hi) - 23));
  return brng::fast_two_sum(hi, lo);
}
static bool tight(brng::FF x) {  // hi + lo is exact in wide_t
  return x.lo == 0.0f || std::fabs(x.lo) >= std::ldexp(std::fabs(x.hi), -85);
}
static long double ld(brng::FF x) { return static_cast<long double>(x.hi) + static_cast<long double>(x.lo); }
static wide_t wd(brng::FF x) { return static_cast<wide_t>(x.hi) + static_cast<wide_t>(x.lo); }
static long double rel_u2(long double got, long double want) {
  return want == 0.0L ? 0.0L : fabsl((got - want) / want) * 281474976710656.0L;  // / 2^-48
}
static long double rel_u2w(wide_t got, wide_t want) {
  if (want == 0) return 0.0L;
  const wide_t r = (got - want) / want;
  return static_cast<long double>(r < 0 ? -r : r) * 281474976710656.0L;
}

static void ffops(long long N) {
  long double e_add = 0, e_add_f = 0, e_mul = 0, e_mul_f = 0, e_div_f = 0, e_div = 0, e_sqrt = 0;
  long long n_add = 0, n_cancel = 0;  // sums checked, and of them those cancelling below 2^-20 |x|
  for (long long i = 0; i < N; ++i) {
    const brng::FF x = rand_ff();
    brng::FF y = rand_ff();
    if (i % 4 == 0) {  // a nearly cancelling sum: y close to -x
      const float d = static_cast<float>((unif() - 0.5) * std::ldexp(1.0, std::ilogb(x.hi) - static_cast<int>(next64() % 40)));
      y = brng::fast_two_sum(-x.hi, -x.lo + d);
    }
    const float f = rand_ff().hi;
    if (tight(x) && tight(y)) {
      ++n_add;
      if (std::fabs(static_cast<double>(ld(x) + ld(y))) < std::ldexp(std::fabs(x.hi), -20)) ++n_cancel;
      e_add = std::max(e_add, rel_u2w(wd(brng::ff_add(x, y)), wd(x) + wd(y)));
      e_add_f = std::max(e_add_f, rel_u2w(wd(brng::ff_add_f(x, f)), wd(x) + static_cast<wide_t>(f)));
    }
    e_mul = std::max(e_mul, rel_u2(ld(brng::ff_mul(x, y)), ld(x) * ld(y)));
    e_mul_f = std::max(e_mul_f, rel_u2(ld(brng::ff_mul_f(x, f)), ld(x) * f));
    e_div_f = std::max(e_div_f, rel_u2(ld(brng::ff_div_f(x, f)), ld(x) / f));
    e_div = std::max(e_div, rel_u2(ld(brng::ff_div(x, y)), ld(x) / ld(y)));
    const brng::FF ax = brng::ff_abs(x);
    e_sqrt = std::max(e_sqrt, rel_u2(ld(brng::ff_sqrt(ax)), sqrtl(ld(ax))));
  }
  std::printf("{\"add\": %.4Lf, \"add_f\": %.4Lf, \"mul\": %.4Lf, \"mul_f\": %.4Lf, \"div_f\": %.4Lf, "
              "\"div\": %.4Lf, \"sqrt\": %.4Lf, \"sums\": %lld, \"cancelling_sums\": %lld}\n",
              e_add, e_add_f, e_mul, e_mul_f, e_div_f, e_div, e_sqrt, n_add, n_cancel);
}

int main(int argc, char** argv) {
  if (argc != 4) return 2;
  if (std::strcmp(argv[1], "ffops") == 0) {
    g_state = std::strtoull(argv[3], nullptr, 10);
    ffops(std::atoll(argv[2]));
    return 0;
  }
  if (std::strcmp(argv[1], "inv") == 0 || std::strcmp(argv[1], "inv_edges") == 0) {
    g_state = std::strtoull(argv[3], nullptr, 10);
    InvTally t;
    inversions(argv[1][3] == '_', std::atoll(argv[2]), t);
    std::printf("{\"draws\": %lld, \"decided32\": %lld, \"decided_ds\": %lld, \"undecided\": %lld, \"mismatches\": %lld}\n",
                t.draws, t.decided32, t.decided_ds, t.undecided, t.mismatches);
    return 0;
  }
  if (std::strcmp(argv[1], "ptrs_edges") == 0 || std::strcmp(argv[1], "btrd_edges") == 0) {
    g_state = std::strtoull(argv[3], nullptr, 10);
    Tally t;
    edges(argv[1][0] == 'p', std::atoll(argv[2]), t);
    std::printf("{\"attempts\": %lld, \"decided\": %lld, \"undecided\": %lld, \"accepted\": %lld, \"mismatches\": %lld}\n",
                t.attempts, t.decided, t.undecided, t.accepted, t.mismatches);
    return 0;
  }
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
