// brng_gibbs.cuh -- the Gibbs models' per-unit bodies (one warp runs one unit),
// shared by the one-kernel-per-job launches (brng_gibbs.cu) and the batched
// persistent kernel (brng_batch.cu).
#pragma once

#include <cmath>

#include "brng_gamma.cuh"
#include "brng_internal.h"

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
template <int NC>
__device__ __forceinline__ void triangle_unit(const TriangleArgs& a, uint64_t unit,
                                              unsigned char* base) {
  const unsigned lane = lane_id();
  uint32_t* list = reinterpret_cast<uint32_t*>(base);
  double* ring = reinterpret_cast<double*>(base + 128);
  if (unit * NC >= a.n_chains) return;  // whole warp
  const uint64_t c = unit * NC + lane;
  const bool consumer = lane < static_cast<unsigned>(NC) && c < a.n_chains;
  const uint32_t stream = static_cast<uint32_t>(a.chain_offset + c);

  double x = 0.0, y = 0.0;
  double m0 = 0.0, m1 = 0.0, m2 = 0.0, m3 = 0.0, m4 = 0.0;
  uint64_t pos = 0;
  if (consumer) {
    const brng_triangle_state_t s = a.state[c];
    x = s.x;
    y = s.y;
    pos = s.pos;
    const double* m = a.moments + 5 * c;
    m0 = m[0]; m1 = m[1]; m2 = m[2]; m3 = m[3]; m4 = m[4];
  }
  Ring<GenU64, NC, false> R;
  R.init(ring, nullptr, list, a.B, pos);
  for (uint32_t it = 0; it < a.n_sweeps; ++it) {
    const double ux = R.get(consumer, stream, a.rk);
    x = __dmul_rn(__dadd_rn(1.0, -y), ux);
    const double uy = R.get(consumer, stream, a.rk);
    y = __dmul_rn(__dadd_rn(1.0, -x), uy);
    m0 = __dadd_rn(m0, x);
    m1 = __dadd_rn(m1, y);
    m2 = __dadd_rn(m2, __dmul_rn(x, x));
    m3 = __dadd_rn(m3, __dmul_rn(y, y));
    m4 = __dadd_rn(m4, __dmul_rn(x, y));
  }
  if (consumer) {
    brng_triangle_state_t s;
    s.x = x;
    s.y = y;
    s.pos = R.pos();
    s.pad = 0;
    a.state[c] = s;
    double* m = a.moments + 5 * c;
    m[0] = m0; m[1] = m1; m[2] = m2; m[3] = m3; m[4] = m4;
  }
  __syncwarp();  // the ring is reused by the warp's next unit
}

// ---------------------------------------------------------------------------
// Normal-gamma Gibbs: per sweep tau | mu ~ Gamma(a0 + n/2, rate b0 + SS/2),
// SS = S + n (xbar - mu)^2, then mu | tau ~ N((prec0 mu0 + tau n xbar)/P, 1/P),
// P = prec0 + n tau.  The Gamma shape does not depend on the state, so a lane
// runs one Marsaglia-Tsang attempt per loop iteration and, when it accepts,
// finishes its sweep (draws mu) in the same iteration: lanes never idle while
// a neighbour retries.  Moments: FP32 partials over 64 iterations (the warp
// flushes together) added into FP64 accumulators.
// ---------------------------------------------------------------------------
__host__ __device__ inline uint32_t normal_gamma_warp_bytes(uint32_t B) {
  return 128u + 2u * B * 32u * 4u;
}

// One work unit: 32 chains (unit * 32 ..), one warp; `base` holds
// normal_gamma_warp_bytes(a.B) bytes of this warp's shared memory.
__device__ __forceinline__ void normal_gamma_unit(const NormalGammaArgs& a, uint64_t unit,
                                                  unsigned char* base) {
  const unsigned lane = lane_id();
  uint32_t* list = reinterpret_cast<uint32_t*>(base);
  float* ringN = reinterpret_cast<float*>(base + 128);
  float* ringU = ringN + a.B * 32u;
  if (unit * 32 >= a.n_chains) return;  // whole warp
  const uint64_t c = unit * 32 + lane;
  const bool active = c < a.n_chains;
  const uint32_t stream = static_cast<uint32_t>(a.chain_offset + c);

  float n = 0.0f, xb = 0.0f, S = 0.0f, mu = 0.0f, tau = 0.0f;
  uint64_t pn = 0, pu = 0;
  double d0 = 0.0, d1 = 0.0, d2 = 0.0, d3 = 0.0;
  if (active) {
    n = a.nobs[c];
    xb = a.xbar[c];
    S = a.sc[c];
    const brng_normal_gamma_state_t s = a.state[c];
    mu = s.mu;
    tau = s.tau;
    pn = s.pos_n;
    pu = s.pos_u;
    const double* m = a.moments + 4 * c;
    d0 = m[0]; d1 = m[1]; d2 = m[2]; d3 = m[3];
  }
  Ring<GenN, 32, false> RN;
  Ring<GenU, 32, false> RU;
  RN.init(ringN, nullptr, list, a.B, pn);
  RU.init(ringU, nullptr, list, a.B, pu);
  const GammaState g = gamma_setup(a.a0 + 0.5f * n);
  const float prior_num = a.prec0 * a.mu0;
  const float nxb = n * xb;

  float p0 = 0.0f, p1 = 0.0f, p2 = 0.0f, p3 = 0.0f;
  uint32_t sweep = 0;
  int att = 0;
  bool rejected = false;
  bool more = true;
  while (more) {
    // at most 64 attempts per lane into the FP32 partials, then one FP64 flush
    // outside the inner loop (so no FP64 instruction sits in the hot loop)
    for (uint32_t j = 0; j < 64; ++j) {
      const bool run = active && sweep < a.n_sweeps;
      more = __any_sync(kFull, run);
      if (!more) break;
      float dv = 0.0f;
      uint32_t zw;
      const bool acc = mt_attempt(run, g, RN, RU, stream, a.rk, a.cnt, &dv, &zw);
      const bool boost_now = run && acc && g.boost;
      float G = dv;
      if (__any_sync(kFull, boost_now)) {  // warp-uniform: shapes below 1 only
        const float ub = RU.get(boost_now, stream, a.rk);
        if (boost_now) G = dv * expf(flog(ub + 0x1p-24f) / g.alpha);
      }
      bool finish = false;
      if (run) {
        ++att;
        if (acc) {
          finish = true;
        } else if (att >= kGammaMaxAttempts) {
          G = __int_as_float(0x7fc00000);
          finish = true;
          rejected = true;
        }
      }
      const float z = RN.get(finish, stream, a.rk);
      if (finish) {
        const float dm = xb - mu;
        const float SS = fmaf(n * dm, dm, S);
        tau = __fdividef(G, fmaf(0.5f, SS, a.b0));
        const float P = fmaf(n, tau, a.prec0);
        const float mean = __fdividef(fmaf(tau, nxb, prior_num), P);
        mu = fmaf(z, rsqrtf(P), mean);
        p0 += mu;
        p1 += tau;
        p2 = fmaf(mu, mu, p2);
        p3 = fmaf(tau, tau, p3);
        ++sweep;
        att = 0;
      }
    }
    d0 += p0; d1 += p1; d2 += p2; d3 += p3;
    p0 = p1 = p2 = p3 = 0.0f;
  }
  count_warp(&a.cnt->n_reject, rejected);
  if (active) {
    brng_normal_gamma_state_t s;
    s.mu = mu;
    s.tau = tau;
    s.pos_n = RN.pos();
    s.pos_u = RU.pos();
    a.state[c] = s;
    double* m = a.moments + 4 * c;
    m[0] = d0; m[1] = d1; m[2] = d2; m[3] = d3;
  }
  __syncwarp();  // the rings are reused by the warp's next unit
}

}  // namespace brng
