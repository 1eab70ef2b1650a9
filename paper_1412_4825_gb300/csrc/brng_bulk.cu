// brng_bulk.cu -- varying-parameter streams (the paper's OAAT-with-buffers
// scenario, Sec. 2.3: a parameter is read from memory for every draw and
// every output is written) and the raw core-engine fill.
//
// One lane per stream: warp w serves streams 32w .. 32w+31, and draw i of the
// call belongs to stream i mod S.  Each lane takes its stream's draws m = 0,
// 1, ... in order, one step per iteration (a draw, or one Marsaglia-Tsang
// attempt of a Gamma draw); the lanes stay within a few draws of each other,
// so a warp's parameter loads and output stores (i = s + m S for consecutive
// s) touch few 128-byte rows.  Base deviates come from the warp-shared
// top-up rings (brng_ring.cuh), read by peek/advance.
#include <cuda_runtime.h>

#include <cmath>

#include "brng_gamma.cuh"
#include "brng_inversion.cuh"
#include "brng_rejection32.cuh"
#include "brng_internal.h"

namespace brng {

// TAG: a distribution tag (one distribution per call), kTagMixed (-1: the
// mixed stream, any tag) or kTagMixedContinuous (-2: the mixed stream when no
// Poisson / Binomial tag is present; the same code without the discrete
// draws, so it fits fewer registers).
constexpr int kTagMixedContinuous = -2;

template <int TAG>
struct BulkDomains {
  static constexpr bool kU = TAG < 0 || TAG == BRNG_TAG_UNIFORM || TAG == BRNG_TAG_GAMMA ||
                             TAG == BRNG_TAG_LAPLACE || TAG == BRNG_TAG_POISSON ||
                             TAG == BRNG_TAG_BINOMIAL;
  static constexpr bool kN = TAG < 0 || TAG == BRNG_TAG_NORMAL || TAG == BRNG_TAG_GAMMA;
  static constexpr bool kE = TAG < 0 || TAG == BRNG_TAG_EXPONENTIAL ||
                             TAG == BRNG_TAG_LAPLACE || TAG == BRNG_TAG_WEIBULL;
  static constexpr int kCount = int(kU) + int(kN) + int(kE);
};

__host__ __device__ inline uint32_t bulk_warp_bytes(int n_domains, uint32_t B, bool words) {
  return 128u + static_cast<uint32_t>(n_domains) * B * 32u * 4u * (words ? 2u : 1u);
}

template <int TAG = kTagMixed>
__device__ __forceinline__ bool param_ok(int tag, float p0, float p1) {
  // the continuous-only mixed kernel never runs a discrete draw: if one were
  // dispatched to it, it would be a domain error, not a step that never ends
  if (TAG == kTagMixedContinuous && (tag == BRNG_TAG_POISSON || tag == BRNG_TAG_BINOMIAL)) return false;
  switch (tag) {
    case BRNG_TAG_UNIFORM: return isfinite(p0) && isfinite(p1) && p0 <= p1;
    case BRNG_TAG_NORMAL:
    case BRNG_TAG_LAPLACE: return isfinite(p0) && isfinite(p1) && p1 > 0.0f;
    case BRNG_TAG_EXPONENTIAL:
    case BRNG_TAG_GAMMA: return isfinite(p0) && p0 > 0.0f;
    case BRNG_TAG_WEIBULL: return isfinite(p0) && isfinite(p1) && p0 > 0.0f && p1 > 0.0f;
    case BRNG_TAG_POISSON: return isfinite(p0) && p0 > 0.0f && p0 <= kPoissonMaxLambda;
    case BRNG_TAG_BINOMIAL:
      return isfinite(p0) && p0 >= 0.0f && p0 == floorf(p0) && p0 <= 16777216.0f && isfinite(p1) &&
             p1 >= 0.0f && p1 <= 1.0f;
    default: return false;
  }
}

// Means above kInversionMaxMean take transformed rejection (PTRS, BTRD)
// instead of the O(mean) inversion.  The Binomial mean n min(p, 1 - p) is
// compared exactly: min(p, 1 - p) is a float (1 - p is exact for p > 1/2) and
// the product is held as the exact sum hi + lo.
__device__ __forceinline__ bool discrete_large(int tag, float p0, float p1) {
  if (tag == BRNG_TAG_POISSON) return p0 > kInversionMaxMean;
  const FF m = two_prod(p0, p1 > 0.5f ? __fadd_rn(1.0f, -p1) : p1);
  return m.hi > kInversionMaxMean || (m.hi == kInversionMaxMean && m.lo > 0.0f);
}

// One rejection attempt for a large-mean Poisson or Binomial draw from the
// next U elements u0, u1 of the lane's ring (u1 is consumed only when the
// attempt reads it).  Decided in FP32 and float-float where that provably
// gives the FP64 evaluation's result (brng_rejection32.cuh), else redone in
// FP64.  Out of line: the FP64 code runs on GB300's narrow FP64 pipe and
// must not be issued, even predicated off, on other draws' steps.
struct LargeAttempt {
  float k;        // the count, or -1 for a rejection
  int used;       // U elements consumed (1 or 2)
  bool recheck;   // decided in FP64
};
static __device__ __noinline__ LargeAttempt large_attempt64(bool poisson, float p0, float p1, float u0, float u1) {
  LargeAttempt r;
  r.recheck = true;
  if (poisson) {
    r.used = 2;
    r.k = static_cast<float>(ptrs_attempt64(static_cast<double>(p0), static_cast<double>(u0),
                                            static_cast<double>(u1) + 0x1p-24));
  } else {
    int used = 1;
    r.k = static_cast<float>(btrd_attempt64(static_cast<double>(p0), static_cast<double>(p1),
                                            static_cast<double>(u0) + 0x1p-24, static_cast<double>(u1), &used));
    r.used = used;
  }
  return r;
}
static __device__ __noinline__ LargeAttempt large_attempt(bool poisson, float p0, float p1, float u0, float u1) {
  const Attempt32 c =
      poisson ? ptrs_attempt32(p0, u0, __fadd_rn(u1, 0x1p-24f)) : btrd_attempt32(p0, p1, u0, u1);
  if (c.k == kUndecided) return large_attempt64(poisson, p0, p1, u0, u1);
#ifdef BRNG_DEBUG
  const LargeAttempt e = large_attempt64(poisson, p0, p1, u0, u1);
  BRNG_CHECK(e.k == c.k && e.used == c.used);
#endif
  return LargeAttempt{c.k, c.used, false};
}

// ---- discrete draws by inversion (Poisson, Binomial) ------------------------
// The FP32 and double-single tiers of brng_inversion.cuh, then an FP64 redraw
// in the reference operation order for the draws both leave undecided, so
// every count equals the reference's.  The FP32 tier runs inline; the rest,
// about one draw in a thousand, out of line.
static __device__ __noinline__ float poisson_recheck(float lambda, float u) {
  return static_cast<float>(poisson_inv64(static_cast<double>(lambda), static_cast<double>(u),
                                          kPoissonMaxK));
}
static __device__ __noinline__ float binomial_recheck(float n, float p, float u) {
  return static_cast<float>(binomial_inv64(static_cast<double>(n), static_cast<double>(p),
                                           static_cast<double>(u)));
}

// The double-single tier, then FP64.  *rechecked: the draw was redone in FP64.
static __device__ __noinline__ float poisson_slow(float lambda, float u, bool* rechecked) {
  const float k = poisson_inv_ds(lambda, u, kPoissonMaxK);
  *rechecked = k == kUndecided;
  if (*rechecked) return poisson_recheck(lambda, u);
#ifdef BRNG_DEBUG
  BRNG_CHECK(k == poisson_recheck(lambda, u));  // a decided draw is the FP64 draw
#endif
  return k;
}
static __device__ __noinline__ float binomial_slow(float n, float p, float u, bool* rechecked) {
  const float k = binomial_inv_ds(n, p, u);
  *rechecked = k == kUndecided;
  if (*rechecked) return binomial_recheck(n, p, u);
#ifdef BRNG_DEBUG
  BRNG_CHECK(k == binomial_recheck(n, p, u));
#endif
  return k;
}

// The FP32 tier's result k32 (kUndecided: the slower tiers decide).
__device__ __forceinline__ float poisson_take(float k32, float lambda, float u, bool* rechecked) {
  if (k32 == kUndecided) return poisson_slow(lambda, u, rechecked);
  *rechecked = false;
#ifdef BRNG_DEBUG
  BRNG_CHECK(k32 == poisson_recheck(lambda, u));
#endif
  return k32;
}
__device__ __forceinline__ float binomial_take(float k32, float n, float p, float u, bool* rechecked) {
  if (k32 == kUndecided) return binomial_slow(n, p, u, rechecked);
  *rechecked = false;
#ifdef BRNG_DEBUG
  BRNG_CHECK(k32 == binomial_recheck(n, p, u));
#endif
  return k32;
}

// In the single-distribution kernels the inversion searches run at most
// kInvSteps steps per iteration of the kernel's loop and resume on the next:
// a lane with a long search (a mean near 64) then takes several iterations
// while its neighbours move on to their next draws, instead of the whole warp
// running every step to the largest k among its lanes (GB300, 2^26 draws:
// Poisson means <= 64 3.54 -> 2.28 ms, Binomial 8.1 -> 5.85 ms; 8 and 32
// steps were slower).  The U element is consumed when the search starts, so
// positions and values do not depend on the bound.  The mixed stream, and a
// Binomial warp with BTRD attempts, search to the end in one step: the mixed
// kernel has no registers left for the state, and a warp paying a BTRD
// attempt every iteration loses more to the extra iterations than it gains
// (n log-uniform to 2^24: 11.2 ms one-shot, 13.4 ms resumable).  A Poisson
// warp with PTRS attempts resumes too (lambda log-uniform [0.05, 1e6]:
// 4.42 ms one-shot, 3.70 ms resumable).
constexpr int kInvSteps = 16;

struct InvSearch {  // an FP32-tier search in progress
  float u, k, pk, F, Fprev;
};

__device__ __forceinline__ void poisson_start(InvSearch& s, float lambda, float u) {
  s.u = u;
  s.k = 0.0f;
  s.pk = expf(-lambda);
  s.F = s.pk;
  s.Fprev = 0.0f;
}

// Up to kInvSteps FP32 steps: 1 when u < F(k) (found), -1 when the search ran
// out (k at its cap, or p_k underflowed), 0 to resume later.
__device__ __forceinline__ int poisson_steps(InvSearch& s, float lambda) {
  float p = s.pk, F = s.F, Fprev = s.Fprev, k = s.k;
  int st = 0;
  for (int j = 0; j < kInvSteps; ++j) {
    if (s.u < F) {
      st = 1;
      break;
    }
    if (k >= static_cast<float>(kPoissonMaxK)) {
      st = -1;
      break;
    }
    k += 1.0f;
    p = (p * lambda) / k;
    Fprev = F;
    if (p == 0.0f) {
      st = -1;
      break;
    }
    F = F + p;
  }
  if (st == 0 && s.u < F) st = 1;
  s.pk = p;
  s.F = F;
  s.Fprev = Fprev;
  s.k = k;
  return st;
}

__device__ __forceinline__ float poisson_finish(const InvSearch& s, float lambda, bool ran_out, bool* rechecked) {
  return poisson_take(poisson_decide32(s.u, s.k, s.F, s.Fprev, ran_out), lambda, s.u, rechecked);
}

// The whole search in one step.
__device__ __forceinline__ float poisson_draw(float lambda, float u, bool* rechecked) {
  return poisson_take(poisson_inv32(lambda, u, kPoissonMaxK), lambda, u, rechecked);
}

__device__ __forceinline__ void binomial_start(InvSearch& s, float n, float p, float u) {
  s.u = u;
  s.k = 0.0f;
  s.pk = binomial_p0(n, p);
  s.F = s.pk;
  s.Fprev = 0.0f;
}

// Up to kInvSteps FP32 steps (as poisson_steps)
__device__ __forceinline__ int binomial_steps(InvSearch& s, float n, float p) {
  float pk = s.pk, F = s.F, Fprev = s.Fprev, k = s.k;
  if (k == 0.0f && !(pk >= 0x1p-125f)) return -1;  // p_0 too small to decide in FP32
  const float r = binomial_ratio(p);
  int st = 0;
  for (int j = 0; j < kInvSteps; ++j) {
    if (s.u < F) {
      st = 1;
      break;
    }
    if (k >= n) {
      st = -1;
      break;
    }
    k += 1.0f;
    pk = (pk * (((n - k) + 1.0f) * r)) / k;
    Fprev = F;
    if (pk == 0.0f) {
      st = -1;
      break;
    }
    F = F + pk;
  }
  if (st == 0 && s.u < F) st = 1;
  s.pk = pk;
  s.F = F;
  s.Fprev = Fprev;
  s.k = k;
  return st;
}

__device__ __forceinline__ float binomial_finish(const InvSearch& s, float n, float p, bool ran_out,
                                                 bool* rechecked) {
  return binomial_take(binomial_decide32(n, p, s.u, s.k, s.F, s.Fprev, ran_out), n, p, s.u, rechecked);
}

__device__ __forceinline__ float binomial_draw(float n, float p, float u, bool* rechecked) {
  return binomial_take(binomial_inv32(n, p, u), n, p, u, rechecked);
}

// Register caps (measured on GB300, 2^28 mixed draws / 2^26 discrete draws;
// no spills at 96, a few words at 72): the mixed stream at 96 -- the
// out-of-line rejection attempt had raised it from 89 to 100 registers, one
// occupancy step lower (6.59 ms without the call, 7.85 ms at 100, 6.69 ms
// capped at 96); every single-distribution kernel at 72, seven blocks of 4
// warps per SM (Poisson means <= 64: 2.45 ms at 80 registers, 2.28 at 72,
// 2.72 at 64; Binomial 6.02 / 5.85 / 5.97; the other distributions need
// fewer).  The mixed stream without discrete tags at 64 (a few spilled
// words; 5.88 ms against 5.96 at 80 and 5.99 at 72, with the shared-memory
// carveout at its maximum so that 32 warps fit).
template <int TAG>
constexpr int kBulkMaxRegs = TAG == kTagMixed ? 96 : TAG == kTagMixedContinuous ? 64 : 72;

// Per lane, one step per iteration: the lane's current draw, or for a Gamma
// draw one Marsaglia-Tsang attempt (a rejected attempt leaves the lane on the
// same draw for the next iteration, while its neighbours move on).  Each ring
// is topped up at one point of the iteration, for the most a step can take
// (U: 2 = attempt + boost; N: 1; E: 1), and every read is a peek, so each
// domain's generator code appears once in the kernel.  The next draw's tag
// and parameters are loaded one step ahead.
template <int TAG, bool WORDS>
__global__ void __maxnreg__(kBulkMaxRegs<TAG>) bulk_kernel(const BulkArgs a) {
  using D = BulkDomains<TAG>;
  if constexpr (TAG < 0) {  // both mixed kernels are launched; the flag picks one
    if (a.mixed_flag && (*a.mixed_flag != 0u) != (TAG == kTagMixed)) return;
  }
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned warp = threadIdx.x >> 5;
  const uint32_t wbytes = bulk_warp_bytes(D::kCount, a.B, WORDS);
  unsigned char* base = smem + warp * wbytes + 128;
  const uint32_t ring_bytes = a.B * 32u * 4u;

  const uint64_t gwarp = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
  const uint64_t s64 = gwarp * 32u + lane_id();
  const bool has_stream = s64 < a.S;
  const uint32_t s = static_cast<uint32_t>(s64);

  CRing<GenU, WORDS> RU;
  CRing<GenN, WORDS> RN;
  CRing<GenE, WORDS> RE;
  if constexpr (D::kU) {
    RU.init(reinterpret_cast<float*>(base), WORDS ? reinterpret_cast<uint32_t*>(base + ring_bytes) : nullptr,
            a.B, has_stream ? a.pos[s] : 0);
    base += ring_bytes * (WORDS ? 2 : 1);
  }
  if constexpr (D::kN) {
    RN.init(reinterpret_cast<float*>(base), WORDS ? reinterpret_cast<uint32_t*>(base + ring_bytes) : nullptr,
            a.B, has_stream ? a.pos[static_cast<uint64_t>(a.S) + s] : 0);
    base += ring_bytes * (WORDS ? 2 : 1);
  }
  if constexpr (D::kE) {
    RE.init(reinterpret_cast<float*>(base), WORDS ? reinterpret_cast<uint32_t*>(base + ring_bytes) : nullptr,
            a.B, has_stream ? a.pos[2ull * a.S + s] : 0);
  }

  // current draw (i, tag, p0, p1) and the next one's inputs, loaded ahead
  uint64_t i = s64;
  int tag = TAG, tag_n = TAG;
  float p0 = 0.0f, p1 = 0.0f, p0_n = 0.0f, p1_n = 0.0f;
  auto load = [&](uint64_t k, int& t, float& q0, float& q1) {
    if constexpr (TAG < 0) t = a.tag[k];
    q0 = a.p0[k];
    if (a.p1) q1 = a.p1[k];
  };
  if (has_stream && i < a.n) load(i, tag, p0, p1);
  if (has_stream && i + a.S < a.n) load(i + a.S, tag_n, p0_n, p1_n);
  bool ok = has_stream && i < a.n && param_ok<TAG>(tag, p0, p1);
  count_warp(&a.cnt->n_domain, has_stream && i < a.n && !ok);
  GammaState g = gamma_setup(ok && tag == BRNG_TAG_GAMMA ? p0 : 1.0f);
  int attempts = 0;  // of the current draw (an inversion search: 1 once started)
  InvSearch inv;
  uint32_t word = 0;

  while (true) {
    const bool active = has_stream && i < a.n;
    if (!__any_sync(kFull, active)) break;
    const bool isU = ok && tag == BRNG_TAG_UNIFORM;
    const bool isN = ok && tag == BRNG_TAG_NORMAL;
    const bool isE = ok && (tag == BRNG_TAG_EXPONENTIAL || tag == BRNG_TAG_LAPLACE || tag == BRNG_TAG_WEIBULL);
    const bool isL = ok && tag == BRNG_TAG_LAPLACE;
    const bool isG = ok && tag == BRNG_TAG_GAMMA;
    const bool isP = ok && tag == BRNG_TAG_POISSON;
    const bool isB = ok && tag == BRNG_TAG_BINOMIAL;
    // a stream with draws left is topped up whenever a ring of its warp runs dry
    if constexpr (D::kU) RU.ensure(isU || isL || isG || isP || isB, 2, active, s, a.rk);
    if constexpr (D::kN) RN.ensure(isN || isG, 1, active, s, a.rk);
    if constexpr (D::kE) RE.ensure(isE, 1, active, s, a.rk);

    bool done = active && !ok;  // an invalid parameter: NaN, nothing consumed
    float out = __int_as_float(0x7fc00000);
    if constexpr (D::kU && (TAG < 0 || TAG == BRNG_TAG_UNIFORM)) {
      if (isU) {
        const float u = RU.peek(0);
        if (WORDS) word = RU.peek_word(0);
        RU.advance(1);
        out = fmaf(p1 - p0, u, p0);
        done = true;
      }
    }
    if constexpr (D::kN && (TAG < 0 || TAG == BRNG_TAG_NORMAL)) {
      if (isN) {
        const float z = RN.peek(0);
        if (WORDS) word = RN.peek_word(0);
        RN.advance(1);
        out = fmaf(p1, z, p0);
        done = true;
      }
    }
    if constexpr (D::kE) {
      if (isE) {
        const float e = RE.peek(0);
        if (WORDS) word = RE.peek_word(0);
        RE.advance(1);
        if (tag == BRNG_TAG_EXPONENTIAL) out = e / p0;
        if constexpr (TAG < 0 || TAG == BRNG_TAG_WEIBULL)
          if (tag == BRNG_TAG_WEIBULL) out = p1 * expf(flog(e) / p0);
        if constexpr (D::kU && (TAG < 0 || TAG == BRNG_TAG_LAPLACE)) {
          if (isL) {
            const float u = RU.peek(0);
            RU.advance(1);
            out = u < 0.5f ? fmaf(-p1, e, p0) : fmaf(p1, e, p0);
          }
        }
        done = true;
      }
    }
    if constexpr (D::kU && (TAG == kTagMixed || TAG == BRNG_TAG_POISSON || TAG == BRNG_TAG_BINOMIAL)) {
      if (__builtin_expect(__any_sync(kFull, isP || isB), TAG >= 0)) {  // one vote for both
        bool rc = false, rej = false;
        const bool large = (isP || isB) && discrete_large(tag, p0, p1);
        const bool any_large = __any_sync(kFull, large);
        if (isP || isB) {
          if (!large) {  // inversion of one U
            if (TAG < 0 || (TAG == BRNG_TAG_BINOMIAL && attempts == 0 && any_large)) {  // the whole search now
              const float u = RU.peek(0);
              if (WORDS) word = RU.peek_word(0);
              RU.advance(1);
              if constexpr (TAG < 0 || TAG == BRNG_TAG_POISSON)
                if (isP) out = poisson_draw(p0, u, &rc);
              if constexpr (TAG < 0 || TAG == BRNG_TAG_BINOMIAL)
                if (isB) out = binomial_draw(p0, p1, u, &rc);
              done = true;
            } else if constexpr (TAG >= 0) {  // resumable: at most kInvSteps steps per iteration
              if (attempts == 0) {  // the draw's first step: take its U element
                const float u = RU.peek(0);
                if (WORDS) word = RU.peek_word(0);
                RU.advance(1);
                attempts = 1;
                if constexpr (TAG == BRNG_TAG_POISSON) poisson_start(inv, p0, u);
                if constexpr (TAG == BRNG_TAG_BINOMIAL) binomial_start(inv, p0, p1, u);
              }
              int st = 0;
              if constexpr (TAG == BRNG_TAG_POISSON) st = poisson_steps(inv, p0);
              if constexpr (TAG == BRNG_TAG_BINOMIAL) st = binomial_steps(inv, p0, p1);
              if (st != 0) {
                if constexpr (TAG == BRNG_TAG_POISSON) out = poisson_finish(inv, p0, st < 0, &rc);
                if constexpr (TAG == BRNG_TAG_BINOMIAL) out = binomial_finish(inv, p0, p1, st < 0, &rc);
                done = true;
              }
            }
          } else {  // one transformed-rejection attempt (1 or 2 U elements)
            if (WORDS && attempts == 0) word = RU.peek_word(0);
            const LargeAttempt r = large_attempt(isP, p0, p1, RU.peek(0), RU.peek(1));
            RU.advance(static_cast<uint32_t>(r.used));
            rc = r.recheck;
            ++attempts;
            if (r.k >= 0.0f) {
              out = r.k;
              done = true;
            } else if (attempts >= kGammaMaxAttempts) {
              done = true;  // NaN
              rej = true;
            }
          }
        }
        count_warp(&a.cnt->n_recheck, rc);
        count_warp(&a.cnt->n_reject, rej);
      }
    }
    if constexpr (D::kN && D::kU && (TAG < 0 || TAG == BRNG_TAG_GAMMA)) {
      bool gdone = false, rej = false;
      if (__any_sync(kFull, isG)) {
        float dv = 0.0f;
        uint32_t zw = 0;
        const bool acc = mt_attempt_peek<false, WORDS>(isG, g, RN, RU, s, a.rk, a.cnt, &dv, &zw);
        if (isG) {
          if (attempts == 0) word = zw;
          ++attempts;
          if (acc) {
            out = dv;
            gdone = true;
          } else if (attempts >= kGammaMaxAttempts) {
            gdone = true;  // NaN
            rej = true;
          }
        }
      }
      count_warp(&a.cnt->n_reject, rej);
      done = done || gdone;
    }
    if (done) {  // finish the draw, move to the stream's next one
      a.out[i] = out;
      if (WORDS) a.words[i] = word;
      i += a.S;
      tag = tag_n;
      p0 = p0_n;
      p1 = p1_n;
      if (i + a.S < a.n) load(i + a.S, tag_n, p0_n, p1_n);
      word = 0;
      attempts = 0;
    }
    const bool fresh = done && i < a.n;
    if (__any_sync(kFull, done)) {
      const bool okn = fresh && param_ok<TAG>(tag, p0, p1);
      count_warp(&a.cnt->n_domain, fresh && !okn);
      if (done) {
        ok = okn;
        if constexpr (D::kN && D::kU && (TAG < 0 || TAG == BRNG_TAG_GAMMA))
          if (ok && tag == BRNG_TAG_GAMMA) g = gamma_setup(p0);
      }
    }
  }
  uint32_t left = 0;
  if constexpr (D::kU) left += static_cast<uint32_t>(max(RU.avail(), 0));
  if constexpr (D::kN) left += static_cast<uint32_t>(max(RN.avail(), 0));
  if constexpr (D::kE) left += static_cast<uint32_t>(max(RE.avail(), 0));
  count_waste(a.cnt, has_stream ? left : 0u);
  if (has_stream) {
    if constexpr (D::kU) a.pos[s] = RU.pos();
    if constexpr (D::kN) a.pos[static_cast<uint64_t>(a.S) + s] = RN.pos();
    if constexpr (D::kE) a.pos[2ull * a.S + s] = RE.pos();
  }
}

template <int TAG, bool WORDS>
static cudaError_t launch_bulk_t(const BulkArgs& a, const Geometry& g, cudaStream_t st) {
  using D = BulkDomains<TAG>;
  BulkArgs b = a;
  b.B = a.B < kBulkMinRing ? kBulkMinRing : a.B;  // a step may take 2 U elements: B - 3 >= 2
  const uint32_t threads = 32u * g.warps_per_block;
  const size_t smem = static_cast<size_t>(g.warps_per_block) * bulk_warp_bytes(D::kCount, b.B, WORDS);
  const uint64_t warps = (static_cast<uint64_t>(a.S) + 31) / 32;
  const uint64_t blocks = (warps + g.warps_per_block - 1) / g.warps_per_block;
  cudaError_t e = cudaFuncSetAttribute(bulk_kernel<TAG, WORDS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  if constexpr (TAG < 0)  // room for every warp the register cap allows
    e = cudaFuncSetAttribute(bulk_kernel<TAG, WORDS>, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
  if (e != cudaSuccess) return e;
  bulk_kernel<TAG, WORDS><<<static_cast<unsigned>(blocks), threads, smem, st>>>(b);
  return cudaGetLastError();
}

// The mixed stream's dispatch: one pass over the tags (1 byte per draw, 16
// per load) sets the flag when a Poisson or Binomial tag is present; both
// mixed kernels are then launched and the flag lets one of them run (the
// other's blocks exit at once), so the choice needs no host round trip and
// the call stays asynchronous and capturable.
__global__ void mixed_scan_kernel(const uint8_t* tag, uint64_t n, unsigned int* flag) {
  const uint64_t tid = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  const uint64_t nv = (reinterpret_cast<uintptr_t>(tag) & 15u) == 0 ? n / 16 : 0;
  unsigned hit = 0;
  const uint4* t4 = reinterpret_cast<const uint4*>(tag);
  for (uint64_t i = tid; i < nv; i += stride) {
    const uint4 v = __ldcs(t4 + i);
    // bytes 6 and 7 are exactly those with (b & 0xfe) == 6
    hit |= __vcmpeq4(v.x & 0xfefefefeu, 0x06060606u) | __vcmpeq4(v.y & 0xfefefefeu, 0x06060606u) |
           __vcmpeq4(v.z & 0xfefefefeu, 0x06060606u) | __vcmpeq4(v.w & 0xfefefefeu, 0x06060606u);
  }
  for (uint64_t i = nv * 16 + tid; i < n; i += stride) hit |= (tag[i] & 0xfeu) == 6u;
  if (__any_sync(kFull, hit != 0) && lane_id() == 0) *flag = 1u;
}

static cudaError_t launch_mixed(const BulkArgs& a, const Geometry& g, cudaStream_t st, bool w) {
  cudaError_t e = cudaMemsetAsync(a.mixed_flag, 0, sizeof(unsigned int), st);
  if (e != cudaSuccess) return e;
  if (a.n > 0) {
    mixed_scan_kernel<<<4u * 152u, 256u, 0, st>>>(a.tag, a.n, a.mixed_flag);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  e = w ? launch_bulk_t<kTagMixedContinuous, true>(a, g, st) : launch_bulk_t<kTagMixedContinuous, false>(a, g, st);
  if (e != cudaSuccess) return e;
  return w ? launch_bulk_t<kTagMixed, true>(a, g, st) : launch_bulk_t<kTagMixed, false>(a, g, st);
}

cudaError_t launch_bulk(int tag, const BulkArgs& a, const Geometry& g, cudaStream_t st) {
  const bool w = a.words != nullptr;
  switch (tag) {
    case kTagMixed:
      if (a.mixed_flag) return launch_mixed(a, g, st, w);
      return w ? launch_bulk_t<-1, true>(a, g, st) : launch_bulk_t<-1, false>(a, g, st);
    case BRNG_TAG_UNIFORM: return w ? launch_bulk_t<0, true>(a, g, st) : launch_bulk_t<0, false>(a, g, st);
    case BRNG_TAG_NORMAL: return w ? launch_bulk_t<1, true>(a, g, st) : launch_bulk_t<1, false>(a, g, st);
    case BRNG_TAG_EXPONENTIAL: return w ? launch_bulk_t<2, true>(a, g, st) : launch_bulk_t<2, false>(a, g, st);
    case BRNG_TAG_GAMMA: return w ? launch_bulk_t<3, true>(a, g, st) : launch_bulk_t<3, false>(a, g, st);
    case BRNG_TAG_LAPLACE: return w ? launch_bulk_t<4, true>(a, g, st) : launch_bulk_t<4, false>(a, g, st);
    case BRNG_TAG_WEIBULL: return w ? launch_bulk_t<5, true>(a, g, st) : launch_bulk_t<5, false>(a, g, st);
    case BRNG_TAG_POISSON: return w ? launch_bulk_t<6, true>(a, g, st) : launch_bulk_t<6, false>(a, g, st);
    case BRNG_TAG_BINOMIAL: return w ? launch_bulk_t<7, true>(a, g, st) : launch_bulk_t<7, false>(a, g, st);
    default: return cudaErrorInvalidValue;
  }
}

// ---- raw core-engine fill: one thread per Philox block --------------------
__global__ void philox_words_kernel(const RoundKeys rk, uint32_t dom, uint32_t stream,
                                    uint64_t first_block, uint64_t n_blocks, uint4* out) {
  for (uint64_t b = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; b < n_blocks;
       b += static_cast<uint64_t>(gridDim.x) * blockDim.x)
    out[b] = philox_block(first_block + b, dom, stream, rk);
}

cudaError_t launch_philox_words(const RoundKeys& rk, uint32_t dom, uint32_t stream,
                                uint64_t first_block, size_t n_blocks, uint32_t* out,
                                cudaStream_t st) {
  if (n_blocks == 0) return cudaSuccess;
  int dev = 0, sms = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  uint64_t blocks = (n_blocks + 255) / 256;
  const uint64_t cap = static_cast<uint64_t>(sms) * 16;
  if (blocks > cap) blocks = cap;
  philox_words_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(
      rk, dom, stream, first_block, n_blocks, reinterpret_cast<uint4*>(out));
  return cudaGetLastError();
}

// ---- integer-pipe probe: Philox blocks kept in registers ------------------
// Each thread runs 4 independent counter chains (for instruction-level
// parallelism) for `iters` blocks each, folding the outputs into a checksum
// so nothing is dead code; only one word per thread reaches memory.
__global__ void __launch_bounds__(256) philox_peak_kernel(const RoundKeys rk, uint64_t iters,
                                                          uint32_t* sink) {
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  uint4 c0 = make_uint4(tid, 0u, 1u, 0u), c1 = make_uint4(tid, 1u, 2u, 0u);
  uint4 c2 = make_uint4(tid, 2u, 3u, 0u), c3 = make_uint4(tid, 3u, 4u, 0u);
  uint32_t acc = 0;
  for (uint64_t i = 0; i < iters; ++i) {
    const uint4 a = philox(c0, rk), b = philox(c1, rk), c = philox(c2, rk), d = philox(c3, rk);
    acc ^= a.x ^ a.y ^ a.z ^ a.w ^ b.x ^ b.y ^ b.z ^ b.w ^ c.x ^ c.y ^ c.z ^ c.w ^ d.x ^ d.y ^ d.z ^ d.w;
    ++c0.w; ++c1.w; ++c2.w; ++c3.w;
  }
  sink[tid] = acc;
}

cudaError_t launch_philox_peak(const RoundKeys& rk, uint64_t iters, uint32_t blocks, uint32_t threads,
                               uint32_t* sink, cudaStream_t st) {
  philox_peak_kernel<<<blocks, threads, 0, st>>>(rk, iters, sink);
  return cudaGetLastError();
}

// ---- the FP32 base-conversion functions, one element per thread ----------
__global__ void fp32_eval_kernel(uint32_t fn, uint64_t n, const float* in, float* out) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    if (fn == 0) {
      out[i] = flog(in[i]);
    } else {
      float s, c;
      fsincospi_k(static_cast<uint32_t>(in[i]), &s, &c);
      out[i] = fn == 1 ? s : c;
    }
  }
}

cudaError_t launch_fp32_eval(uint32_t fn, size_t n, const float* in, float* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  fp32_eval_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(fn, n, in, out);
  return cudaGetLastError();
}

// ---- FP64 uniform from the U64 domain (brng_uniform_f64) -------------------
// finite a <= b, decided on the bit patterns with integer operations: GB300's
// FP64 pipe is narrow, and the two FP64 operations of the value (a difference
// and a fused multiply-add) are all a draw should spend there.  Finite: exponent field below 0x7ff.  Order of
// finite doubles: the sign-magnitude pattern mapped to a two's-complement key
// (-0 and +0 both to 0), which orders like the values.
__device__ __forceinline__ int64_t f64_order_key(uint64_t bits) {
  const int64_t mag = static_cast<int64_t>(bits & 0x7fffffffffffffffull);
  return (bits >> 63) ? -mag : mag;
}
__device__ __forceinline__ bool f64_interval_ok(double lo, double hi) {
  const uint64_t a = static_cast<uint64_t>(__double_as_longlong(lo));
  const uint64_t b = static_cast<uint64_t>(__double_as_longlong(hi));
  const bool finite = ((a >> 52) & 0x7ffu) != 0x7ffu && ((b >> 52) & 0x7ffu) != 0x7ffu;
  return finite && f64_order_key(a) <= f64_order_key(b);
}

// One thread per stream walks that stream's draws i = s, s + S, ... in order
// (reads and writes of a warp's 32 streams are consecutive, so coalesced).  A
// draw takes the stream's next U64 element, two per Philox block; the block is
// kept in registers between its two elements, so there is no ring.
__global__ void __launch_bounds__(256) uniform64_kernel(const Uniform64Args a) {
  constexpr int kU = 4;  // draws whose loads are in flight together
  const uint64_t s = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (s >= a.S || s >= a.n) return;
  const uint32_t stream = static_cast<uint32_t>(s);
  const uint64_t S = a.S;
  uint64_t j = a.pos64[s];
  uint64_t have = ~0ull;  // Philox block held in w
  uint4 w = make_uint4(0, 0, 0, 0);
  uint32_t bad = 0;
  for (uint64_t i0 = s; i0 < a.n; i0 += kU * S) {
    double lo[kU], hi[kU];
#pragma unroll
    for (int k = 0; k < kU; ++k) {  // streaming loads: every input is read once
      const uint64_t i = i0 + k * S;
      lo[k] = i < a.n ? __ldcs(a.a + i) : 0.0;
      hi[k] = i < a.n ? __ldcs(a.b + i) : 0.0;
    }
#pragma unroll
    for (int k = 0; k < kU; ++k) {
      const uint64_t i = i0 + k * S;
      if (i >= a.n) break;
      double v = __longlong_as_double(0x7ff8000000000000ll);
      uint32_t first = 0;
      if (f64_interval_ok(lo[k], hi[k])) {
        const uint64_t blk = j >> 1;
        if (blk != have) {
          w = philox_block(blk, kDomU64, stream, a.rk);
          have = blk;
        }
        const bool second = (j & 1) != 0;
        first = second ? w.z : w.x;
        const double u = u53(first, second ? w.w : w.y);
        v = __fma_rn(__dadd_rn(hi[k], -lo[k]), u, lo[k]);  // fma(b - a, U64, a), as the oracle
        ++j;
      } else {
        ++bad;
      }
      __stcs(a.out + i, v);
      if (a.words) __stcs(a.words + i, first);
    }
  }
  a.pos64[s] = j;
  if (bad) atomicAdd(&a.cnt->n_domain, static_cast<unsigned long long>(bad));
}

cudaError_t launch_uniform64(const Uniform64Args& a, cudaStream_t st) {
  const uint64_t threads = a.n < a.S ? a.n : a.S;
  if (threads == 0) return cudaSuccess;
  const uint64_t blocks = (threads + 255) / 256;
  uniform64_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(a);
  return cudaGetLastError();
}

// ---- the FP64 recheck functions, one element per thread -------------------
__global__ void fp64_eval_kernel(uint32_t fn, uint64_t n, const double* in, double* out) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    double s, c;
    if (fn == 0) {
      out[i] = dlog(in[i]);
    } else if (fn == 3) {
      out[i] = dexp(in[i]);
    } else {
      dsincospi(in[i], &s, &c);
      out[i] = fn == 1 ? s : c;
    }
  }
}

cudaError_t launch_fp64_eval(uint32_t fn, size_t n, const double* in, double* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  uint64_t blocks = (n + 255) / 256;
  if (blocks > 65535) blocks = 65535;
  fp64_eval_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(fn, n, in, out);
  return cudaGetLastError();
}

}  // namespace brng
