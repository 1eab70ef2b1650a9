// brng_bulk.cu -- varying-parameter streams (the paper's OAAT-with-buffers
// scenario, Sec. 2.3: a parameter is read from memory for every draw and
// every output is written) and the raw core-engine fill.
//
// One lane per stream: warp w serves streams 32w .. 32w+31, and draw i of the
// call belongs to stream i mod S.  The warp walks its streams' draws m = 0, 1,
// ... in lockstep, so each parameter load and output store of a warp is one
// contiguous 128-byte access (i = s + m S for consecutive s).  Base deviates
// come from the warp-shared rings (brng_ring.cuh); a Gamma draw loops over
// Marsaglia-Tsang attempts until every lane of the warp has accepted.
#include <cuda_runtime.h>

#include <cmath>

#include "brng_gamma.cuh"
#include "brng_internal.h"

namespace brng {

template <int TAG>
struct BulkDomains {
  static constexpr bool kU = TAG < 0 || TAG == BRNG_TAG_UNIFORM || TAG == BRNG_TAG_GAMMA ||
                             TAG == BRNG_TAG_LAPLACE;
  static constexpr bool kN = TAG < 0 || TAG == BRNG_TAG_NORMAL || TAG == BRNG_TAG_GAMMA;
  static constexpr bool kE = TAG < 0 || TAG == BRNG_TAG_EXPONENTIAL ||
                             TAG == BRNG_TAG_LAPLACE || TAG == BRNG_TAG_WEIBULL;
  static constexpr int kCount = int(kU) + int(kN) + int(kE);
};

__host__ __device__ inline uint32_t bulk_warp_bytes(int n_domains, uint32_t B, bool words) {
  return 128u + static_cast<uint32_t>(n_domains) * B * 32u * 4u * (words ? 2u : 1u);
}

__device__ __forceinline__ bool param_ok(int tag, float p0, float p1) {
  switch (tag) {
    case BRNG_TAG_UNIFORM: return isfinite(p0) && isfinite(p1) && p0 <= p1;
    case BRNG_TAG_NORMAL:
    case BRNG_TAG_LAPLACE: return isfinite(p0) && isfinite(p1) && p1 > 0.0f;
    case BRNG_TAG_EXPONENTIAL:
    case BRNG_TAG_GAMMA: return isfinite(p0) && p0 > 0.0f;
    case BRNG_TAG_WEIBULL: return isfinite(p0) && isfinite(p1) && p0 > 0.0f && p1 > 0.0f;
    default: return false;
  }
}

template <int TAG, bool WORDS>
__global__ void __launch_bounds__(512) bulk_kernel(const BulkArgs a) {
  using D = BulkDomains<TAG>;
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = lane_id();
  const unsigned warp = threadIdx.x >> 5;
  const uint32_t wbytes = bulk_warp_bytes(D::kCount, a.B, WORDS);
  unsigned char* base = smem + warp * wbytes;
  uint32_t* list = reinterpret_cast<uint32_t*>(base);
  base += 128;
  const uint32_t ring_bytes = a.B * 32u * 4u;

  const uint64_t gwarp = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
  const uint64_t s64 = gwarp * 32u + lane;
  const bool has_stream = s64 < a.S;
  const uint32_t s = static_cast<uint32_t>(s64);

  Ring<GenU, 32, WORDS> RU;
  Ring<GenN, 32, WORDS> RN;
  Ring<GenE, 32, WORDS> RE;
  if constexpr (D::kU) {
    RU.init(reinterpret_cast<float*>(base), WORDS ? reinterpret_cast<uint32_t*>(base + ring_bytes) : nullptr,
            list, a.B, has_stream ? a.pos[s] : 0);
    base += ring_bytes * (WORDS ? 2 : 1);
  }
  if constexpr (D::kN) {
    RN.init(reinterpret_cast<float*>(base), WORDS ? reinterpret_cast<uint32_t*>(base + ring_bytes) : nullptr,
            list, a.B, has_stream ? a.pos[static_cast<uint64_t>(a.S) + s] : 0);
    base += ring_bytes * (WORDS ? 2 : 1);
  }
  if constexpr (D::kE) {
    RE.init(reinterpret_cast<float*>(base), WORDS ? reinterpret_cast<uint32_t*>(base + ring_bytes) : nullptr,
            list, a.B, has_stream ? a.pos[2ull * a.S + s] : 0);
  }

  for (uint64_t m = 0;; ++m) {
    const uint64_t i = s64 + m * a.S;
    const bool active = has_stream && i < a.n;
    if (!__any_sync(kFull, active)) break;
    int tag = TAG;
    float p0 = 0.0f, p1 = 0.0f;
    if (active) {
      if constexpr (TAG < 0) tag = a.tag[i];
      p0 = a.p0[i];
      if (a.p1) p1 = a.p1[i];
    }
    const bool ok = active && param_ok(tag, p0, p1);
    count_warp(&a.cnt->n_domain, active && !ok);
    float out = __int_as_float(0x7fc00000);  // NaN unless drawn
    uint32_t word = 0;

    if constexpr (D::kU && (TAG < 0 || TAG == BRNG_TAG_UNIFORM)) {
      const bool w = ok && tag == BRNG_TAG_UNIFORM;
      uint32_t wd = 0;
      const float u = RU.get(w, s, a.rk, &wd);
      if (w) {
        out = fmaf(p1 - p0, u, p0);
        word = wd;
      }
    }
    if constexpr (D::kN && (TAG < 0 || TAG == BRNG_TAG_NORMAL)) {
      const bool w = ok && tag == BRNG_TAG_NORMAL;
      uint32_t wd = 0;
      const float z = RN.get(w, s, a.rk, &wd);
      if (w) {
        out = fmaf(p1, z, p0);
        word = wd;
      }
    }
    if constexpr (D::kE && (TAG < 0 || TAG == BRNG_TAG_EXPONENTIAL || TAG == BRNG_TAG_LAPLACE ||
                            TAG == BRNG_TAG_WEIBULL)) {
      const bool w = ok && (tag == BRNG_TAG_EXPONENTIAL || tag == BRNG_TAG_LAPLACE ||
                            tag == BRNG_TAG_WEIBULL);
      uint32_t wd = 0;
      const float e = RE.get(w, s, a.rk, &wd);
      if constexpr (TAG < 0 || TAG == BRNG_TAG_LAPLACE) {
        const bool wl = ok && tag == BRNG_TAG_LAPLACE;
        const float u = RU.get(wl, s, a.rk);
        if (wl) out = u < 0.5f ? fmaf(-p1, e, p0) : fmaf(p1, e, p0);
      }
      if (w) {
        word = wd;
        if (tag == BRNG_TAG_EXPONENTIAL) out = e / p0;
        if (tag == BRNG_TAG_WEIBULL) out = p1 * expf(flog(e) / p0);
      }
    }
    if constexpr (D::kN && D::kU && (TAG < 0 || TAG == BRNG_TAG_GAMMA)) {
      bool pending = ok && tag == BRNG_TAG_GAMMA;
      GammaState g = gamma_setup(pending ? p0 : 1.0f);
      int attempts = 0;
      bool rejected = false;
      while (__any_sync(kFull, pending)) {
        float dv = 0.0f;
        uint32_t zw = 0;
        const bool acc = mt_attempt(pending, g, RN, RU, s, a.rk, a.cnt, &dv, &zw);
        if (pending && attempts == 0) word = zw;
        const bool boost_now = pending && acc && g.boost;
        if (__any_sync(kFull, boost_now)) {  // warp-uniform: shapes below 1 only
          const float ub = RU.get(boost_now, s, a.rk);
          if (boost_now) dv *= expf(flog(ub + 0x1p-24f) / g.alpha);
        }
        if (pending) {
          ++attempts;
          if (acc) {
            out = dv;
            pending = false;
          } else if (attempts >= kGammaMaxAttempts) {
            pending = false;
            rejected = true;
          }
        }
      }
      count_warp(&a.cnt->n_reject, rejected);
    }
    if (active) {
      a.out[i] = out;
      if (WORDS) a.words[i] = word;
    }
  }
  if (has_stream) {
    if constexpr (D::kU) a.pos[s] = RU.pos();
    if constexpr (D::kN) a.pos[static_cast<uint64_t>(a.S) + s] = RN.pos();
    if constexpr (D::kE) a.pos[2ull * a.S + s] = RE.pos();
  }
}

template <int TAG, bool WORDS>
static cudaError_t launch_bulk_t(const BulkArgs& a, const Geometry& g, cudaStream_t st) {
  using D = BulkDomains<TAG>;
  const uint32_t threads = 32u * g.warps_per_block;
  const size_t smem = static_cast<size_t>(g.warps_per_block) * bulk_warp_bytes(D::kCount, a.B, WORDS);
  const uint64_t warps = (static_cast<uint64_t>(a.S) + 31) / 32;
  const uint64_t blocks = (warps + g.warps_per_block - 1) / g.warps_per_block;
  cudaError_t e = cudaFuncSetAttribute(bulk_kernel<TAG, WORDS>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  bulk_kernel<TAG, WORDS><<<static_cast<unsigned>(blocks), threads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_bulk(int tag, const BulkArgs& a, const Geometry& g, cudaStream_t st) {
  const bool w = a.words != nullptr;
  switch (tag) {
    case kTagMixed: return w ? launch_bulk_t<-1, true>(a, g, st) : launch_bulk_t<-1, false>(a, g, st);
    case BRNG_TAG_UNIFORM: return w ? launch_bulk_t<0, true>(a, g, st) : launch_bulk_t<0, false>(a, g, st);
    case BRNG_TAG_NORMAL: return w ? launch_bulk_t<1, true>(a, g, st) : launch_bulk_t<1, false>(a, g, st);
    case BRNG_TAG_EXPONENTIAL: return w ? launch_bulk_t<2, true>(a, g, st) : launch_bulk_t<2, false>(a, g, st);
    case BRNG_TAG_GAMMA: return w ? launch_bulk_t<3, true>(a, g, st) : launch_bulk_t<3, false>(a, g, st);
    case BRNG_TAG_LAPLACE: return w ? launch_bulk_t<4, true>(a, g, st) : launch_bulk_t<4, false>(a, g, st);
    case BRNG_TAG_WEIBULL: return w ? launch_bulk_t<5, true>(a, g, st) : launch_bulk_t<5, false>(a, g, st);
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

// ---- the FP64 recheck functions, one element per thread -------------------
__global__ void fp64_eval_kernel(uint32_t fn, uint64_t n, const double* in, double* out) {
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < n;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    double s, c;
    if (fn == 0) {
      out[i] = dlog(in[i]);
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
