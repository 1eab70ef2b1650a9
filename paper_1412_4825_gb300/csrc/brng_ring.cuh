// brng_ring.cuh -- the paper's per-distribution buffers (Sec. 2.2
// buffer_length / buffer / buffer_counter) as warp-shared rings.
//
// One ring holds, for each of NC consumer columns of a warp (a column is one
// stream: a chain, a stream of a bulk call, or one Dirichlet component), the
// next B elements of one domain of that stream.  Layout in shared memory is
// column-minor, val[slot * NC + col], so a warp reading one element per
// column hits NC distinct banks whatever each column's read pointer is.
//
// Refill-on-empty (Sec. 2.2), done by the whole warp: every get() is called
// by all 32 lanes at the same program point with a per-lane `want`; lanes
// whose ring is exhausted vote (ballot), the warp lists them, and all 32 lanes
// generate the needed Philox blocks round-robin over the needy columns (item
// q -> column list[q mod k], block q div k), converting to the domain's
// deviates and storing into the needy columns' rings.  Generation is thus
// always 32-wide, however the consumers have drifted apart (rejection
// sampling consumes unevenly), which is the GPU form of the paper's batch
// refill by the vectorised core engine.
//
// Per-lane state: blk = Philox block of ring slot 0, rp = read pointer,
// valid = filled slots (0 before the first refill).  The stream position is
// blk * EPB + rp (EPB elements per block), so a ring can start at any element.
#pragma once

#include <cstdint>

#include "brng_engine.cuh"

namespace brng {

constexpr unsigned kFull = 0xffffffffu;

__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ uint64_t shfl_u64(uint64_t v, int src) {
  const uint32_t lo = __shfl_sync(kFull, static_cast<uint32_t>(v), src);
  const uint32_t hi = __shfl_sync(kFull, static_cast<uint32_t>(v >> 32), src);
  return (static_cast<uint64_t>(hi) << 32) | lo;
}

// ---- domain generators: one Philox block -> EPB elements ------------------
struct GenU {  // 4 x U[0,1) (U' = U + 2^-24 is formed by the consumer)
  using T = float;
  static constexpr uint32_t kDom = kDomU;
  static constexpr uint32_t kEPB = 4;
  __device__ __forceinline__ static void gen(uint4 w, T* v) {
    v[0] = u01(w.x); v[1] = u01(w.y); v[2] = u01(w.z); v[3] = u01(w.w);
  }
};
struct GenN {  // 2 Box-Muller pairs -> 4 x N(0,1): (cos, sin) of (w0,w1), then of (w2,w3)
  using T = float;
  static constexpr uint32_t kDom = kDomN;
  static constexpr uint32_t kEPB = 4;
  __device__ __forceinline__ static void gen(uint4 w, T* v) {
    const float2 a = box_muller(w.x, w.y);
    const float2 b = box_muller(w.z, w.w);
    v[0] = a.x; v[1] = a.y; v[2] = b.x; v[3] = b.y;
  }
};
struct GenE {  // 4 x Exp(1) = -ln U'
  using T = float;
  static constexpr uint32_t kDom = kDomE;
  static constexpr uint32_t kEPB = 4;
  __device__ __forceinline__ static void gen(uint4 w, T* v) {
    v[0] = exp1(w.x); v[1] = exp1(w.y); v[2] = exp1(w.z); v[3] = exp1(w.w);
  }
};
struct GenU64 {  // 2 x 53-bit U[0,1)
  using T = double;
  static constexpr uint32_t kDom = kDomU64;
  static constexpr uint32_t kEPB = 2;
  __device__ __forceinline__ static void gen(uint4 w, T* v) {
    v[0] = u53(w.x, w.y); v[1] = u53(w.z, w.w);
  }
};

__device__ __forceinline__ uint32_t word_of(uint4 w, uint32_t i) {
  return i == 0 ? w.x : i == 1 ? w.y : i == 2 ? w.z : w.w;
}

// A ring of NC columns.  kWords: also keep each element's raw word (its own
// slot word; the first word of the pair for U64).
template <class Gen, int NC, bool kWords>
struct Ring {
  using T = typename Gen::T;
  static constexpr uint32_t kEPB = Gen::kEPB;
  T* val;          // shared: [B][NC]
  uint32_t* wrd;   // shared: [B][NC] when kWords
  uint32_t* list;  // shared: 32 entries, scratch for the needy-column list
  uint64_t blk;    // Philox block held by slot 0
  uint32_t rp;     // read pointer
  uint32_t valid;  // slots filled
  uint32_t B;      // ring length (multiple of kEPB), warp-uniform

  __device__ __forceinline__ void init(T* v, uint32_t* w, uint32_t* l, uint32_t len, uint64_t pos) {
    val = v; wrd = w; list = l; B = len;
    blk = pos / kEPB;
    rp = static_cast<uint32_t>(pos % kEPB);
    valid = 0;
  }
  __device__ __forceinline__ uint64_t pos() const { return blk * kEPB + rp; }

  // Refill the rings of the columns in `mask` (all 32 lanes call this).
  // `col` is this lane's column (== lane for lane < NC), `stream` its stream.
  __device__ __forceinline__ void refill(unsigned mask, bool need, uint32_t stream,
                                      const RoundKeys& rk) {
    const unsigned lane = lane_id();
    if (need) {
      blk += rp / kEPB;
      rp %= kEPB;
      valid = B;
      list[__popc(mask & ((1u << lane) - 1u))] = lane;
    }
    __syncwarp();
    const uint32_t k = __popc(mask);
    const uint32_t nblk = B / kEPB;
    const uint32_t total = k * nblk;
    uint32_t rank = lane % k, b = lane / k;
    const uint32_t step_r = 32u % k, step_b = 32u / k;
    for (uint32_t q0 = 0; q0 < total; q0 += 32) {
      const uint32_t tgt = list[rank];
      const uint64_t tblk = shfl_u64(blk, static_cast<int>(tgt));
      const uint32_t tstream = __shfl_sync(kFull, stream, static_cast<int>(tgt));
      if (q0 + lane < total) {
        const uint4 w = philox_block(tblk + b, Gen::kDom, tstream, rk);
        T v[kEPB];
        Gen::gen(w, v);
#pragma unroll
        for (uint32_t i = 0; i < kEPB; ++i) {
          val[(b * kEPB + i) * NC + tgt] = v[i];
          if (kWords) wrd[(b * kEPB + i) * NC + tgt] = word_of(w, kEPB == 4 ? i : 2 * i);
        }
      }
      rank += step_r;
      b += step_b;
      if (rank >= k) {
        rank -= k;
        b += 1;
      }
    }
    __syncwarp();
  }

  // Next element for lanes with `want` (all 32 lanes call this).  Optional
  // outputs: the element's raw word and its index in the stream.
  __device__ __forceinline__ T get(bool want, uint32_t stream, const RoundKeys& rk,
                                   uint32_t* word = nullptr, uint64_t* index = nullptr) {
    const bool need = want && rp >= valid;
    const unsigned mask = __ballot_sync(kFull, need);
    if (mask) refill(mask, need, stream, rk);
    T v = T(0);
    if (want) {
      const unsigned lane = lane_id();
      v = val[rp * NC + lane];
      if (kWords && word) *word = wrd[rp * NC + lane];
      if (index) *index = blk * kEPB + rp;
      ++rp;
    }
    return v;
  }
};

}  // namespace brng
