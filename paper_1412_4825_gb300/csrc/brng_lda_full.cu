// brng_lda_full.cu -- the full LDA Gibbs step's topic draws (Sec. 1, the LDA
// paragraph: the Dirichlet parameters of the document-topic draw change every
// iteration because the topic assignments do).  One warp per document.
//
// Per token t of document d (word w, current topic zo), in token order:
//   weights   w_k = ((float(n_dk') + alpha) * (float(n_kw') + beta)) * inv_k,
//             inv_k = 1 / (float(n_k') + V beta), ' = without token t;
//             n_kw', n_k' = the sweep's snapshot plus the document's own
//             changes so far (for n_kw of word w: the earlier tokens of the
//             document with word w, reached through the prev links);
//             every operation IEEE round-to-nearest FP32 (no contraction),
//             so that the oracle, doing the same operations, gets the same
//             bits;
//   integers  q_k = trunc(w_k 2^(b - 1 - e)), 2^e <= max w < 2^(e+1),
//             b = 32 - ceil(log2 K), so that the K weights sum below 2^32;
//   draw      the smallest k with C_k > (r Q) >> 24, C the inclusive sums of
//             q (32-bit warp scan), Q = C_(K-1), r = top 24 bits of the
//             document's next Z word: exact integer arithmetic, so the choice
//             is the oracle's.
// The maximum weight and the pick (the number of topics whose inclusive sum
// is <= (r Q) >> 24) are one warp reduction each (redux on the weights' bits,
// which order as unsigned since the weights are non-negative, and on the
// lanes' counts); the inclusive sums are each lane's own topics in order plus
// an exclusive scan of the lanes' totals.
// Lane l holds topics l KP .. l KP + KP - 1 (KP = ceil(K / 32)): its
// document-topic counts, its topic totals and their two reciprocals (with and
// without the token itself) live in registers; a reciprocal is recomputed only
// when its topic's total changes.  The word's snapshot row is loaded one token
// ahead, so its latency overlaps the current draw.  The Z words come from
// 32 Philox blocks at a time, one per lane, into the warp's 128-word buffer.
// The document's count changes go to dnkw (word-topic, two atomic adds per
// changed token) and, at the end, dnk; the snapshot is never written.
#include <cuda_runtime.h>

#include "brng_internal.h"
#include "brng_ring.cuh"

namespace brng {

constexpr uint32_t kLdaNone = BRNG_LDA_NONE;
constexpr uint32_t kLdaWarps = 1;  // warps (documents) per block: one, so that a block retires with its document (lengths vary 10x)

__global__ void __launch_bounds__(32 * kLdaWarps) lda_index_kernel(uint32_t n_docs,
                                                                   const uint32_t* __restrict__ doc_ptr,
                                                                   const uint32_t* __restrict__ words,
                                                                   uint32_t* __restrict__ prev) {
  const uint32_t d = blockIdx.x * kLdaWarps + (threadIdx.x >> 5);
  if (d >= n_docs) return;
  const uint32_t t0 = doc_ptr[d], t1 = doc_ptr[d + 1];
  for (uint32_t t = t0 + lane_id(); t < t1; t += 32) {
    const uint32_t w = words[t];
    uint32_t p = kLdaNone;
    for (uint32_t j = t; j > t0; --j) {
      if (words[j - 1] == w) {
        p = j - 1;
        break;
      }
    }
    prev[t] = p;
  }
}

__device__ __forceinline__ float lda_inv(int32_t n, float vbeta) {
  return __frcp_rn(__fadd_rn(__int2float_rn(n), vbeta));
}

// One step of an inclusive warp scan: v plus the value `off` lanes below,
// where there is one.  The shuffle's own predicate (the source lane lies in
// the warp) guards the add, so a step is two instructions.
__device__ __forceinline__ uint32_t scan_step_up(uint32_t v, uint32_t off) {
  uint32_t r;
  asm volatile(
      "{\n\t.reg .pred p;\n\t.reg .u32 t;\n\t"
      "mov.u32 %0, %1;\n\t"
      "shfl.sync.up.b32 t|p, %1, %2, 0, 0xffffffff;\n\t"
      "@p add.u32 %0, %0, t;\n\t}"
      : "=r"(r)
      : "r"(v), "r"(off));
  return r;
}

// The lane's KP consecutive topics of a word-topic row (one 8- or 16-byte
// load when every lane's topics are all inside the row).  FULL: K = 32 KP.
template <int KP, bool FULL>
__device__ __forceinline__ void load_row(const int32_t* rowp, uint32_t gl, uint32_t K, bool vec, int32_t* out) {
  if constexpr (KP == 2) {
    if (vec) {
      const int2 v = __ldg(reinterpret_cast<const int2*>(rowp) + gl);
      out[0] = v.x;
      out[1] = v.y;
      return;
    }
  } else if constexpr (KP == 4) {
    if (vec) {
      const int4 v = __ldg(reinterpret_cast<const int4*>(rowp) + gl);
      out[0] = v.x;
      out[1] = v.y;
      out[2] = v.z;
      out[3] = v.w;
      return;
    }
  }
#pragma unroll
  for (int p = 0; p < KP; ++p) {
    const uint32_t k = gl * KP + p;
    out[p] = FULL || k < K ? __ldg(rowp + k) : 0;
  }
}

// One warp per document, G = 32 lanes, KP = ceil(K / 32) topics per lane;
// FULL: K = 32 KP, every lane's topics exist (no bounds tests per token).
// (Two documents per warp, 16 lanes each, was measured slower: the two
// documents' control flow diverges, and the per-token reductions are single
// instructions here already.)
template <int KP, bool FULL>
__global__ void __launch_bounds__(32 * kLdaWarps) lda_z_kernel(const LdaZArgs a) {
  constexpr uint32_t G = 32;
  constexpr unsigned gmask = kFull;
  __shared__ uint32_t zbuf[kLdaWarps][4 * G];
  const uint32_t wid = threadIdx.x >> 5;
  const uint32_t gl = lane_id();
  const uint32_t slot = blockIdx.x * kLdaWarps + wid;
  const uint32_t d = a.order && slot < a.n_docs ? a.order[slot] : slot;
  if (d >= a.n_docs) return;  // whole warp
  uint32_t* zw = zbuf[wid];
  const uint32_t K = a.K;
  const uint32_t t0 = __ldg(a.doc_ptr + d), t1 = __ldg(a.doc_ptr + d + 1);
  const uint32_t stream = static_cast<uint32_t>(a.doc_offset + d);
  const uint2 sh = philox_stream_half(kDomZ, stream, a.rk);

  int32_t nd[KP], nks[KP], own[KP];
  float inv_c[KP], inv_m[KP];
  float xc[KP], xm[KP];  // float(n_dk) + alpha with and without the token itself
#pragma unroll
  for (int p = 0; p < KP; ++p) {
    const uint32_t k = gl * KP + p;
    const bool on = FULL || k < K;
    nd[p] = on ? a.ndk[static_cast<uint64_t>(d) * K + k] : 0;
    nks[p] = on ? a.nk[k] : 0;
    own[p] = 0;
    inv_c[p] = lda_inv(nks[p], a.vbeta);
    inv_m[p] = lda_inv(nks[p] - 1, a.vbeta);
    xc[p] = __fadd_rn(__int2float_rn(nd[p]), a.alpha);
    xm[p] = __fadd_rn(__int2float_rn(nd[p] - 1), a.alpha);
  }
  // a lane's topics are consecutive: with every lane full and the table
  // aligned to the vector, one vector load per row
  const bool vec = FULL && (KP == 2 || KP == 4) && (reinterpret_cast<uintptr_t>(a.nkw) % (4u * KP)) == 0;
  const uint64_t zp0 = a.zpos[d];
  uint32_t zoff = 4u * G;  // the next Z element's slot in zw (4G: refill first)

  int32_t row[KP];
#pragma unroll
  for (int p = 0; p < KP; ++p) row[p] = 0;
  uint32_t w = 0, zo = 0, pv = kLdaNone;  // the token's word, start topic and same-word link
  if (t0 < t1) {
    w = __ldg(a.words + t0);
    zo = a.z[t0];
    pv = __ldg(a.prev + t0);
    load_row<KP, FULL>(a.nkw + static_cast<uint64_t>(w) * K, gl, K, vec, row);
  }
  for (uint32_t t = t0; t < t1; ++t) {
    // the next token's word, snapshot row, topic (not yet redrawn: only this
    // warp writes it, at that token) and link, independent of this draw
    int32_t row_n[KP];
#pragma unroll
    for (int p = 0; p < KP; ++p) row_n[p] = 0;
    uint32_t w_n = 0, zo_n = 0, pv_n = kLdaNone;
    if (t + 1 < t1) {
      w_n = __ldg(a.words + t + 1);
      zo_n = a.z[t + 1];
      pv_n = __ldg(a.prev + t + 1);
      load_row<KP, FULL>(a.nkw + static_cast<uint64_t>(w_n) * K, gl, K, vec, row_n);
    }
    // this draw's Z word (element zp0 + (t - t0) of the document's stream);
    // zw holds the 4G elements from the block of the element that refilled it
    if (zoff >= 4u * G) {
      const uint64_t e = zp0 + (t - t0);
      zoff = static_cast<uint32_t>(e & 3u);
      const uint4 v = philox_block_sh(e / 4u + gl, sh, a.rk);
      __syncwarp(gmask);
      zw[4u * gl + 0u] = v.x;
      zw[4u * gl + 1u] = v.y;
      zw[4u * gl + 2u] = v.z;
      zw[4u * gl + 3u] = v.w;
      __syncwarp(gmask);
    }
    const uint32_t r24 = zw[zoff++] >> 8;
    // the document's own changes of this word's counts in this sweep
    int32_t ow[KP];
#pragma unroll
    for (int p = 0; p < KP; ++p) ow[p] = 0;
    for (uint32_t j = pv; j != kLdaNone; j = __ldg(a.prev + j)) {
      const uint32_t zs = __ldcg(a.z_start + j), zc = __ldcg(a.z + j);
      if (zs != zc) {
#pragma unroll
        for (int p = 0; p < KP; ++p) {
          const uint32_t k = gl * KP + p;
          ow[p] += (k == zc ? 1 : 0) - (k == zs ? 1 : 0);
        }
      }
    }
    // FP32 weights, their maximum, integer weights, inclusive sums
    float wk[KP];
    float m = 0.0f;
#pragma unroll
    for (int p = 0; p < KP; ++p) {
      const uint32_t k = gl * KP + p;
      const int32_t self = k == zo ? 1 : 0;
      const float x = self ? xm[p] : xc[p];
      const float y = __fadd_rn(__int2float_rn(row[p] + ow[p] - self), a.beta);
      wk[p] = FULL || k < K ? __fmul_rn(__fmul_rn(x, y), self ? inv_m[p] : inv_c[p]) : 0.0f;
      m = fmaxf(m, wk[p]);
    }
    // the maximum (weights are non-negative, so their bits order as unsigned)
    m = __uint_as_float(__reduce_max_sync(gmask, __float_as_uint(m)));
    const uint32_t ef = (__float_as_uint(m) >> 23) & 0xFFu;
    const float scale = __uint_as_float((253u + a.qbits - ef) << 23);
    // inclusive sums in topic order: the lane's own topics, then an exclusive
    // scan of the lanes' totals
    uint32_t c[KP];
    uint32_t run = 0;
#pragma unroll
    for (int p = 0; p < KP; ++p) {
      run += __float2uint_rz(__fmul_rn(wk[p], scale));
      c[p] = run;
    }
    uint32_t incl = run;
#pragma unroll
    for (unsigned off = 1; off < G; off <<= 1) incl = scan_step_up(incl, off);
    const uint32_t excl = incl - run;
    const uint32_t base = __shfl_sync(gmask, incl, G - 1, G);
    const uint32_t tt = static_cast<uint32_t>((static_cast<uint64_t>(r24) * base) >> 24);
    uint32_t below = 0;  // this lane's topics whose inclusive sum is <= tt
#pragma unroll
    for (int p = 0; p < KP; ++p) below += ((FULL || gl * KP + p < K) && excl + c[p] <= tt) ? 1u : 0u;
    const uint32_t zn = __reduce_add_sync(gmask, below);
    if (zn != zo) {
#pragma unroll
      for (int p = 0; p < KP; ++p) {
        const uint32_t k = gl * KP + p;
        const int32_t dlt = (k == zn ? 1 : 0) - (k == zo ? 1 : 0);
        // a count moving by one turns the "with" term into the "without" one
        // (or back): one new reciprocal and one new n_dk term per change,
        // taken without a branch so that the lanes of zo and zn share them
        if (dlt != 0) {
          const bool up = dlt > 0;
          nd[p] += dlt;
          own[p] += dlt;
          const float r = lda_inv(nks[p] + own[p] - (up ? 0 : 1), a.vbeta);
          const float xn = __fadd_rn(__int2float_rn(nd[p] - (up ? 0 : 1)), a.alpha);
          const float ic = inv_c[p], im = inv_m[p], c = xc[p], m = xm[p];
          inv_c[p] = up ? r : im;
          inv_m[p] = up ? ic : r;
          xc[p] = up ? xn : m;
          xm[p] = up ? c : xn;
        }
      }
      if (gl == 0) {
        atomicAdd(a.dnkw + static_cast<uint64_t>(w) * K + zo, -1);
        atomicAdd(a.dnkw + static_cast<uint64_t>(w) * K + zn, 1);
      }
    }
    if (gl == 0) {
      a.z_start[t] = static_cast<uint8_t>(zo);
      a.z[t] = static_cast<uint8_t>(zn);
    }
    __syncwarp(gmask);  // this token's z and z_start are visible to the next tokens' walks
    w = w_n;
    zo = zo_n;
    pv = pv_n;
#pragma unroll
    for (int p = 0; p < KP; ++p) row[p] = row_n[p];
  }
  if (gl == 0) a.zpos[d] = zp0 + (t1 - t0);
#pragma unroll
  for (int p = 0; p < KP; ++p) {
    const uint32_t k = gl * KP + p;
    if (k < K) {
      a.ndk[static_cast<uint64_t>(d) * K + k] = nd[p];
      a.dir_alpha[static_cast<uint64_t>(d) * K + k] = __fadd_rn(a.alpha, __int2float_rn(nd[p]));
      if (own[p] != 0) atomicAdd(a.dnkw + static_cast<uint64_t>(a.V) * K + k, own[p]);
    }
  }
}

__global__ void lda_apply_kernel(uint64_t n_kw, uint32_t K, int32_t* __restrict__ nkw, int32_t* __restrict__ nk,
                                 int32_t* __restrict__ dnkw) {
  const uint64_t total = n_kw + K;
  for (uint64_t i = static_cast<uint64_t>(blockIdx.x) * blockDim.x + threadIdx.x; i < total;
       i += static_cast<uint64_t>(gridDim.x) * blockDim.x) {
    const int32_t v = dnkw[i];
    if (v != 0) {
      if (i < n_kw) nkw[i] += v;
      else nk[i - n_kw] += v;
      dnkw[i] = 0;
    }
  }
}

cudaError_t launch_lda_index(uint32_t n_docs, const uint32_t* doc_ptr, const uint32_t* words, uint32_t* prev,
                             cudaStream_t st) {
  if (n_docs == 0) return cudaSuccess;
  lda_index_kernel<<<(n_docs + kLdaWarps - 1) / kLdaWarps, 32 * kLdaWarps, 0, st>>>(n_docs, doc_ptr, words, prev);
  return cudaGetLastError();
}

cudaError_t launch_lda_z(const LdaZArgs& a, cudaStream_t st) {
  if (a.n_docs == 0) return cudaSuccess;
  const uint32_t blocks = (a.n_docs + kLdaWarps - 1) / kLdaWarps;
  if (a.K == 32) lda_z_kernel<1, true><<<blocks, 32 * kLdaWarps, 0, st>>>(a);
  else if (a.K == 64) lda_z_kernel<2, true><<<blocks, 32 * kLdaWarps, 0, st>>>(a);
  else if (a.K == 128) lda_z_kernel<4, true><<<blocks, 32 * kLdaWarps, 0, st>>>(a);
  else if (a.K < 32) lda_z_kernel<1, false><<<blocks, 32 * kLdaWarps, 0, st>>>(a);
  else if (a.K < 64) lda_z_kernel<2, false><<<blocks, 32 * kLdaWarps, 0, st>>>(a);
  else if (a.K < 128) lda_z_kernel<4, false><<<blocks, 32 * kLdaWarps, 0, st>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

cudaError_t launch_lda_apply(uint32_t K, uint32_t V, int32_t* nkw, int32_t* nk, int32_t* dnkw, cudaStream_t st) {
  int dev = 0, sms = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const uint64_t total = static_cast<uint64_t>(V) * K + K;
  uint64_t blocks = (total + 255) / 256;
  if (blocks > static_cast<uint64_t>(sms) * 8) blocks = static_cast<uint64_t>(sms) * 8;
  lda_apply_kernel<<<static_cast<unsigned>(blocks), 256, 0, st>>>(static_cast<uint64_t>(V) * K, K, nkw, nk, dnkw);
  return cudaGetLastError();
}

}  // namespace brng
