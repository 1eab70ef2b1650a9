// brng_gibbs.cuh -- the Gibbs models' per-unit bodies (one warp runs one unit),
// shared by the one-kernel-per-job launches (brng_gibbs.cu) and the batched
// persistent kernel (brng_batch.cu).
#pragma once

#include <cmath>

#include "brng_gamma.cuh"
#include "brng_internal.h"
#include "brng_pc.cuh"

namespace brng {

// ---------------------------------------------------------------------------
// Triangle (Eq. 1, Fig. 1): x <- (1 - y) U64, y <- (1 - x) U64, FP64 with
// every operation an explicit __d*_rn intrinsic (never contracted, i.e. the
// same as compiling with -fmad=false).  NC chains per warp: with NC < 32 the
// other lanes only help refill the rings (lanes per chain = 32 / NC), which
// spreads the few chains of a small ensemble over more warps and SMs.
// ---------------------------------------------------------------------------
__host__ __device__ inline uint32_t triangle_warp_bytes(uint32_t NC, uint32_t B) {
  return 128u + B * NC * 8u;
}

// One work unit: NC chains (unit * NC .. unit * NC + NC - 1), one warp.
// `base`: this warp's shared memory (triangle_warp_bytes(NC, a.B) bytes).
//
// With L = 32 / NC lanes per chain, the L lanes of a chain (one per group
// g = lane / NC) all read the chain's U64 elements (a shared-memory broadcast)
// and run the same x, y updates, and group g keeps the running sums
// m_g, m_{g+L}, ... of the five moments (x, y, x^2, y^2, x y).  On GB300 the
// FP64 pipe issues a warp instruction over many cycles, so what counts is FP64
// warp instructions per sweep: 4 for the updates plus 2 per moment slot --
// 5 slots with one lane per chain, 1 with eight or more.  Group 0 owns the
// ring refills (the other groups read its columns in step).
template <int NC>
__device__ __forceinline__ void triangle_unit(const TriangleArgs& a, uint64_t unit,
                                              unsigned char* base) {
  constexpr int L = 32 / NC;                  // lanes per chain
  constexpr int SLOTS = (5 + L - 1) / L;      // moments per lane
  const unsigned lane = lane_id();
  const unsigned col = lane % NC;
  const unsigned grp = lane / NC;
  uint32_t* list = reinterpret_cast<uint32_t*>(base);
  double* ring = reinterpret_cast<double*>(base + 128);
  if (unit * NC >= a.n_chains) return;  // whole warp
  const uint64_t c = unit * NC + col;
  const bool live = c < a.n_chains;
  const bool owner = live && grp == 0;
  const uint32_t stream = static_cast<uint32_t>(a.chain_offset + c);

  double x = 0.0, y = 0.0;
  double m[SLOTS];
  uint64_t pos = 0;
  if (live) {
    const brng_triangle_state_t s = a.state[c];
    x = s.x;
    y = s.y;
    pos = s.pos;
  }
#pragma unroll
  for (int k = 0; k < SLOTS; ++k) {
    const unsigned j = grp + k * L;  // moment index of this slot
    m[k] = (live && j < 5) ? a.moments[5 * c + j] : 0.0;
  }
  Ring<GenU64, NC, false> R;
  R.init(ring, nullptr, list, a.B, pos);
  for (uint32_t it = 0; it < a.n_sweeps; ++it) {
    const double ux = R.get(live, stream, a.rk, nullptr, nullptr, grp == 0);
    x = __dmul_rn(__dadd_rn(1.0, -y), ux);
    const double uy = R.get(live, stream, a.rk, nullptr, nullptr, grp == 0);
    y = __dmul_rn(__dadd_rn(1.0, -x), uy);
    if constexpr (L == 1) {  // one lane per chain: all five sums here
      m[0] = __dadd_rn(m[0], x);
      m[1] = __dadd_rn(m[1], y);
      m[2] = __dadd_rn(m[2], __dmul_rn(x, x));
      m[3] = __dadd_rn(m[3], __dmul_rn(y, y));
      m[4] = __dadd_rn(m[4], __dmul_rn(x, y));
    } else {
#pragma unroll
      for (int k = 0; k < SLOTS; ++k) {
        // moment j = grp + k L: x*1, y*1, x*x, y*y, x*y (times 1.0 is exact)
        const unsigned j = grp + k * L;
        const double f0 = (j == 1 || j == 3) ? y : x;
        const double f1 = j < 2 ? 1.0 : (j == 2 ? x : y);
        m[k] = __dadd_rn(m[k], __dmul_rn(f0, f1));
      }
    }
  }
  count_waste(a.cnt, owner && R.valid > R.rp ? R.valid - R.rp : 0u);
  if (owner) {
    brng_triangle_state_t s;
    s.x = x;
    s.y = y;
    s.pos = R.pos();
    s.pad = 0;
    a.state[c] = s;
  }
#pragma unroll
  for (int k = 0; k < SLOTS; ++k) {
    const unsigned j = grp + k * L;
    if (live && j < 5) a.moments[5 * c + j] = m[k];
  }
  __syncwarp();  // the ring is reused by the warp's next unit
}

// ---------------------------------------------------------------------------
// Normal-gamma Gibbs: per sweep tau | mu ~ Gamma(a0 + n/2, rate b0 + SS/2),
// SS = S + n (xbar - mu)^2, then mu | tau ~ N((prec0 mu0 + tau n xbar)/P, 1/P),
// P = prec0 + n tau.  The sweeps run in speculative rounds (ng_sweeps below);
// moments are compensated FP32 sums added into FP64 at the end.
// ---------------------------------------------------------------------------
// The warp's N and U rings: circular, with mirrored heads as deep as a round's
// lookahead (2W N and W U elements, W <= 8), so every read is one load.
using NgRingN = CRing<GenN, false, 16>;
using NgRingU = CRing<GenU, false, 8>;

__host__ __device__ inline uint32_t normal_gamma_warp_bytes(uint32_t B) {
  return 128u + (NgRingN::ring_slots(B) + NgRingU::ring_slots(B)) * 32u * 4u;
}

// Compensated (Kahan) FP32 running sum: accurate to a few FP32 ulp of the
// total over any number of terms, with no FP64 arithmetic in the loop.
struct Kahan {
  float s = 0.0f, c = 0.0f;
  __device__ __forceinline__ void add(float v) {
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
  }
  __device__ __forceinline__ double value() const {
    return static_cast<double>(s) - static_cast<double>(c);
  }
};

// Sweep moments of one chain (sum mu, tau, mu^2, tau^2).  The sweeps of a run
// are taken in groups of kMomGroup consecutive sweeps, counted from the run's
// first: within a group plain FP32 sums (one add or FMA per moment and
// sweep), and each finished group's sums go into compensated FP32 sums, which
// go into the FP64 moments at the end of the run.  The error stays within
// (kMomGroup + 2) FP32 ulp of the sum of magnitudes over any number of
// sweeps, and since the grouping depends only on the sweep count, every ring
// length, round width and producer layout gives the same bits.
constexpr uint32_t kMomGroup = 8;
struct SweepMoments {
  float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;  // the open group's sums
  Kahan k[4];
  __device__ __forceinline__ void add(float mu, float tau) {
    p0 += mu;
    p1 += tau;
    p2 = fmaf(mu, mu, p2);
    p3 = fmaf(tau, tau, p3);
  }
  // close the open group
  __device__ __forceinline__ void fold() {
    k[0].add(p0);
    k[1].add(p1);
    k[2].add(p2);
    k[3].add(p3);
    p0 = p1 = p2 = p3 = 0.0f;
  }
};

// Chain state of one lane, read from and written back to global memory.
struct NgChain {
  float n, xb, S, mu, tau;
  uint64_t pn, pu;
  double d0, d1, d2, d3;  // FP64 moments (sum mu, tau, mu^2, tau^2)
  SweepMoments m;         // this run's sums, not yet in d
};

// Adds the run's sums (the last, possibly partial, group included) into the
// FP64 moments.
__device__ __forceinline__ void ng_fold_moments(NgChain& s) {
  s.m.fold();
  s.d0 += s.m.k[0].value();
  s.d1 += s.m.k[1].value();
  s.d2 += s.m.k[2].value();
  s.d3 += s.m.k[3].value();
  s.m = SweepMoments{};
}

__device__ __forceinline__ NgChain ng_load(const NormalGammaArgs& a, uint64_t c, bool active) {
  NgChain s{};
  if (active) {
    s.n = a.nobs[c];
    s.xb = a.xbar[c];
    s.S = a.sc[c];
    const brng_normal_gamma_state_t st = a.state[c];
    s.mu = st.mu;
    s.tau = st.tau;
    s.pn = st.pos_n;
    s.pu = st.pos_u;
    const double* m = a.moments + 4 * c;
    s.d0 = m[0]; s.d1 = m[1]; s.d2 = m[2]; s.d3 = m[3];
  }
  return s;
}

__device__ __forceinline__ void ng_store(const NormalGammaArgs& a, uint64_t c, bool active,
                                         const NgChain& s) {
  if (active) {
    brng_normal_gamma_state_t st;
    st.mu = s.mu;
    st.tau = s.tau;
    st.pos_n = s.pn;
    st.pos_u = s.pu;
    a.state[c] = st;
    double* m = a.moments + 4 * c;
    m[0] = s.d0; m[1] = s.d1; m[2] = s.d2; m[3] = s.d3;
  }
}

template <class R>
__device__ __forceinline__ bool ring_failed(const R&) { return false; }

// mu | tau after tau = G / (b0 + SS/2): the sweep's state update (FP32)
__device__ __forceinline__ void ng_update(const NormalGammaArgs& a, float n, float xb, float S,
                                          float nxb, float prior_num, float G, float z, float& mu,
                                          float& tau) {
  const float dm = xb - mu;
  const float SS = fmaf(n * dm, dm, S);
  tau = __fdividef(G, fmaf(0.5f, SS, a.b0));
  const float P = fmaf(n, tau, a.prec0);
  const float mean = __fdividef(fmaf(tau, nxb, prior_num), P);
  mu = fmaf(z, rsqrtf(P), mean);
}

// The sweeps of one warp's 32 chains from the rings RN (N domain) and RU (U
// domain): the warp's own circular rings or rings that producer warps fill
// (brng_pc.cuh).  Leaves the final positions in s.pn, s.pu.
//
// The Gamma shape a0 + n/2 does not depend on the chain state, only the rate
// does, so the Gamma(shape, 1) draws of a chain -- and the positions of the
// normal and uniform elements each consumes -- follow from its streams alone.
// Each round therefore evaluates W Marsaglia-Tsang attempts at once (ILP W),
// speculating that each earlier one accepts: attempt i reads N element 2i (z)
// and U element i, and its sweep's mu | tau normal is N element 2i + 1.  The
// first k attempts that the log-free test accepts are exactly the sweeps the
// one-at-a-time loop would run (same elements, same FP32 operations); the
// cheap state recursion then runs over them.  The attempt after them is
// usually a rejection, which a log-free reject test settles: its z and U'
// are consumed and the next round speculates from there.  One that neither
// test settles (a few per million at shape 52) puts the lane in exact mode:
// one attempt the exact way per round, in the same round and the following
// ones, until one accepts and its sweep ends.
// Shapes below 1 (boosted) stay in exact mode.  Each ring is refilled at one
// point of the round only (its refill code is large, and the instruction
// cache small): the round's 2W N and W U elements cover both parts, since
// a lane that leaves the speculative part after k < W sweeps still has
// 2W - 2k >= 2 N and W - k >= 1 U elements for its exact attempt, and a lane
// in exact mode from the start needs at most 2 of each (boosted lanes never
// speculate).
template <int W, class RNT, class RUT>
__device__ __forceinline__ void ng_sweeps(const NormalGammaArgs& a, uint32_t n_sweeps, uint32_t stream,
                                          bool active, NgChain& s, RNT& RN, RUT& RU) {
  static_assert(W >= 2, "the speculative form needs W >= 2");
  const GammaState g = gamma_setup(a.a0 + 0.5f * s.n);
  const float prior_num = a.prec0 * a.mu0;
  const float nxb = s.n * s.xb;
  const float n = s.n, xb = s.xb, S = s.S;
  float mu = s.mu, tau = s.tau;
  SweepMoments& mom = s.m;
  bool exact = g.boost;  // per lane: the next attempt is taken the exact way
  int att = 0;
  uint32_t sweep = 0;
  bool rejected = false;
  while (true) {
    const bool run = active && sweep < n_sweeps && !ring_failed(RN) && !ring_failed(RU);
    if (!__any_sync(kFull, run)) break;
    RN.ensure(run, 2 * W, run, stream, a.rk);
    RU.ensure(run, W, run, stream, a.rk);
    const bool spec = run && !exact;
    if (__any_sync(kFull, spec)) {
      float G[W], zm[W];
      uint32_t fast = 0;
#pragma unroll
      for (int i = 0; i < W; ++i) {
        const float z = RN.peek(2 * i);
        zm[i] = RN.peek(2 * i + 1);
        const float uo = RU.peek(i) + 0x1p-24f;  // U' = U + 2^-24, exact
        const float x = g.c * z;
        // q_hi >= q (mt_series_qhi): U' + q_hi < 1 is still a sufficient
        // condition of the accept test, so a fast accept stays an exact
        // accept, and an attempt it does not settle goes to the fast reject
        // or the exact path.  q_hi exceeds q by ~3 d |x|^7 / 7, far below U's
        // resolution at the |x| that occur.
        const float q = mt_series_qhi(g.d, x);
        const float t = 1.0f + x;
        G[i] = g.d * (t * t * t);
        const bool ok = fabsf(x) <= kSeriesMaxX && fmaf(q, 1.00001f, uo) < 0x1.fffff8p-1f;
        fast |= static_cast<uint32_t>(ok) << i;
      }
      if (!spec) fast = 0;
      uint32_t k = static_cast<uint32_t>(__ffs(~fast)) - 1u;  // leading accepted attempts
      k = min(k, static_cast<uint32_t>(W));
      k = min(k, n_sweeps - min(sweep, n_sweeps));
      const uint32_t kspec = k;
      k = min(k, kMomGroup - sweep % kMomGroup);  // a round ends at a moment-group boundary
#pragma unroll
      for (int i = 0; i < W; ++i) {
        if (static_cast<uint32_t>(i) < k) {
          ng_update(a, n, xb, S, nxb, prior_num, G[i], zm[i], mu, tau);
          mom.add(mu, tau);
        }
      }
      if (spec) {
        RN.advance(2 * k);
        RU.advance(k);
        sweep += k;
        if (k > 0) {
          att = 0;
          if (sweep % kMomGroup == 0) mom.fold();
        }
        if (k == kspec && k < W && sweep < n_sweeps) {
          // The attempt after the k sweeps was not settled by the fast accept;
          // it now sits at the read points (N element 0, U element 0).  Fast
          // reject: q_lo = 3 d x^4 (1/4 - x/5) <= q for |x| < 1 (the margin
          // series alternates with decreasing terms for x >= 0 and has only
          // positive terms for x < 0), and U' (1 + q) >= 1 gives
          // ln U' >= -ln(1 + q) >= -q, a rejection.  In FP32 q_lo is shrunk by
          // 1e-5 and the product compared with 1 + 2^-22, covering q_lo's and
          // z's rounding as the fast accept's margins do; so a fast reject is
          // an exact (and FP64) reject.  It consumes the attempt's z and U'
          // and the sweep goes on speculatively from the next elements; an
          // attempt settled by neither test goes to the exact path.
          const float z = RN.peek(0);
          const float uo = RU.peek(0) + 0x1p-24f;  // U' = U + 2^-24, exact
          const float x = g.c * z;
          const float x2 = x * x;
          const float ql = ((3.0f * g.d) * (x2 * x2)) * fmaf(x, -0.2f, 0.25f);
          const bool rej = fabsf(x) <= kSeriesMaxX && att + 1 < kGammaMaxAttempts &&
                           fmaf(uo, ql * 0.99999f, uo) >= 0x1.000004p+0f;
          if (rej) {
            RN.advance(1);
            RU.advance(1);
            ++att;
          } else {
            exact = true;
          }
        }
      }
    }
    const bool ex = run && exact && sweep < n_sweeps;
    if (__any_sync(kFull, ex)) {
      float G = 0.0f;
      const bool acc = mt_attempt_peek<true, false>(ex, g, RN, RU, stream, a.rk, a.cnt, &G, nullptr);
      bool finish = false;
      if (ex) {
        ++att;
        if (acc) {
          finish = true;
        } else if (att >= kGammaMaxAttempts) {
          G = __int_as_float(0x7fc00000);
          finish = true;
          rejected = true;
        }
      }
      if (finish) {
        const float z = RN.peek(0);
        RN.advance(1);
        ng_update(a, n, xb, S, nxb, prior_num, G, z, mu, tau);
        mom.add(mu, tau);
        ++sweep;
        if (sweep % kMomGroup == 0) mom.fold();
        att = 0;
        exact = g.boost;
      }
    }
  }
  count_warp(&a.cnt->n_reject, rejected);
  if (ring_failed(RN) || ring_failed(RU)) mu = tau = __int_as_float(0x7fc00000);
  s.mu = mu;
  s.tau = tau;
  s.pn = RN.pos();
  s.pu = RU.pos();
}

// Ring length 4 (one block): no room to look ahead, one exact attempt per
// iteration with refill-on-demand reads.
template <class RNT, class RUT>
__device__ __forceinline__ void ng_sweeps_plain(const NormalGammaArgs& a, uint32_t n_sweeps, uint32_t stream,
                                                bool active, NgChain& s, RNT& RN, RUT& RU) {
  const GammaState g = gamma_setup(a.a0 + 0.5f * s.n);
  const float prior_num = a.prec0 * a.mu0;
  const float nxb = s.n * s.xb;
  const float n = s.n, xb = s.xb, S = s.S;
  float mu = s.mu, tau = s.tau;
  SweepMoments& mom = s.m;
  uint32_t sweep = 0;
  int att = 0;
  bool rejected = false;
  while (true) {
    const bool run = active && sweep < n_sweeps && !ring_failed(RN) && !ring_failed(RU);
    if (!__any_sync(kFull, run)) break;
    float dv = 0.0f;
    uint32_t zw;
    const bool acc = mt_attempt<true>(run, g, RN, RU, stream, a.rk, a.cnt, &dv, &zw);
    const bool boost_now = run && acc && g.boost;
    if (__any_sync(kFull, boost_now)) {  // shapes below 1 only
      const float ub = RU.get(boost_now, stream, a.rk);
      if (boost_now) dv = dv * expf(flog(ub + 0x1p-24f) / g.alpha);
    }
    bool finish = false;
    if (run) {
      ++att;
      if (acc) {
        finish = true;
      } else if (att >= kGammaMaxAttempts) {
        dv = __int_as_float(0x7fc00000);
        finish = true;
        rejected = true;
      }
    }
    const float z = RN.get(finish, stream, a.rk);
    if (finish) {
      ng_update(a, n, xb, S, nxb, prior_num, dv, z, mu, tau);
      mom.add(mu, tau);
      ++sweep;
      if (sweep % kMomGroup == 0) mom.fold();
      att = 0;
    }
  }
  count_warp(&a.cnt->n_reject, rejected);
  if (ring_failed(RN) || ring_failed(RU)) mu = tau = __int_as_float(0x7fc00000);
  s.mu = mu;
  s.tau = tau;
  s.pn = RN.pos();
  s.pu = RU.pos();
}

// Speculation width for ring length B (elements per lane and domain): the
// N ring must hold 2W elements past the read point (B >= 4W).
__host__ __device__ constexpr int ng_width(uint32_t B) { return B >= 32 ? 8 : B >= 16 ? 4 : B >= 8 ? 2 : 0; }

// Runs n_sweeps sweeps of the lane's chain (all lanes call).
template <class RNT, class RUT>
__device__ __forceinline__ void ng_sweeps_any(const NormalGammaArgs& a, uint32_t n_sweeps, uint32_t stream,
                                              bool active, NgChain& s, RNT& RN, RUT& RU) {
  switch (ng_width(a.B)) {  // warp-uniform
    case 8: ng_sweeps<8>(a, n_sweeps, stream, active, s, RN, RU); break;
    case 4: ng_sweeps<4>(a, n_sweeps, stream, active, s, RN, RU); break;
    case 2: ng_sweeps<2>(a, n_sweeps, stream, active, s, RN, RU); break;
    default: ng_sweeps_plain(a, n_sweeps, stream, active, s, RN, RU); break;
  }
}

// One work unit: 32 chains (unit * 32 ..), one warp; `base` holds
// normal_gamma_warp_bytes(a.B) bytes of this warp's shared memory.
__device__ __forceinline__ void normal_gamma_unit(const NormalGammaArgs& a, uint64_t unit,
                                                  unsigned char* base) {
  const unsigned lane = lane_id();
  float* ringN = reinterpret_cast<float*>(base + 128);
  float* ringU = ringN + NgRingN::ring_slots(a.B) * 32u;
  if (unit * 32 >= a.n_chains) return;  // whole warp
  const uint64_t c = unit * 32 + lane;
  const bool active = c < a.n_chains;
  const uint32_t stream = static_cast<uint32_t>(a.chain_offset + c);
  NgChain s = ng_load(a, c, active);
  NgRingN RN;
  NgRingU RU;
  RN.init(ringN, nullptr, a.B, s.pn);
  RU.init(ringU, nullptr, a.B, s.pu);
  ng_sweeps_any(a, a.n_sweeps, stream, active, s, RN, RU);
  count_waste(a.cnt, active ? static_cast<uint32_t>(RN.avail() + RU.avail()) : 0u);
  ng_fold_moments(s);
  ng_store(a, c, active, s);
  __syncwarp();  // the rings are reused by the warp's next unit
}

}  // namespace brng
