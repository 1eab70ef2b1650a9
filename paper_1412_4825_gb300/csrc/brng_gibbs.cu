// brng_gibbs.cu -- Markov-dependent consumers: the triangle Gibbs sampler of
// Eq. 1 / Fig. 1 and the normal-gamma Gibbs sampler.  Each chain is a Philox
// stream (global chain id) and a lane; its state stays in registers for the
// whole run and its base deviates come from the warp-shared rings.
#include <cuda_runtime.h>

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

template <int NC>
__global__ void __launch_bounds__(512) triangle_kernel(const TriangleArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = lane_id();
  const unsigned warp = threadIdx.x >> 5;
  unsigned char* base = smem + warp * triangle_warp_bytes(NC, a.B);
  uint32_t* list = reinterpret_cast<uint32_t*>(base);
  double* ring = reinterpret_cast<double*>(base + 128);

  const uint64_t unit = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
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
}

template <int NC>
static cudaError_t launch_tri_t(const TriangleArgs& a, const Geometry& g, cudaStream_t st) {
  const uint64_t units = (static_cast<uint64_t>(a.n_chains) + NC - 1) / NC;
  if (units == 0) return cudaSuccess;
  const uint32_t threads = 32u * g.warps_per_block;
  const size_t smem = static_cast<size_t>(g.warps_per_block) * triangle_warp_bytes(NC, a.B);
  const uint64_t blocks = (units + g.warps_per_block - 1) / g.warps_per_block;
  cudaError_t e = cudaFuncSetAttribute(triangle_kernel<NC>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  triangle_kernel<NC><<<static_cast<unsigned>(blocks), threads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_triangle(const TriangleArgs& a, const Geometry& g, uint32_t lanes_per_chain,
                            cudaStream_t st) {
  switch (lanes_per_chain) {
    case 1: return launch_tri_t<32>(a, g, st);
    case 2: return launch_tri_t<16>(a, g, st);
    case 4: return launch_tri_t<8>(a, g, st);
    case 8: return launch_tri_t<4>(a, g, st);
    case 16: return launch_tri_t<2>(a, g, st);
    case 32: return launch_tri_t<1>(a, g, st);
    default: return cudaErrorInvalidValue;
  }
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

__global__ void __launch_bounds__(512) normal_gamma_kernel(const NormalGammaArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = lane_id();
  const unsigned warp = threadIdx.x >> 5;
  unsigned char* base = smem + warp * normal_gamma_warp_bytes(a.B);
  uint32_t* list = reinterpret_cast<uint32_t*>(base);
  float* ringN = reinterpret_cast<float*>(base + 128);
  float* ringU = ringN + a.B * 32u;

  const uint64_t unit = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
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
}

cudaError_t launch_normal_gamma(const NormalGammaArgs& a, const Geometry& g, cudaStream_t st) {
  const uint64_t units = (static_cast<uint64_t>(a.n_chains) + 31) / 32;
  if (units == 0) return cudaSuccess;
  const uint32_t threads = 32u * g.warps_per_block;
  const size_t smem = static_cast<size_t>(g.warps_per_block) * normal_gamma_warp_bytes(a.B);
  const uint64_t blocks = (units + g.warps_per_block - 1) / g.warps_per_block;
  cudaError_t e = cudaFuncSetAttribute(normal_gamma_kernel,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  normal_gamma_kernel<<<static_cast<unsigned>(blocks), threads, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace brng
