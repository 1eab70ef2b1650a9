// brng_ring.cuh -- the paper's per-distribution buffers (Sec. 2.2
// buffer_length / buffer / buffer_counter) as warp-shared rings.
//
// One ring holds, for each of NC consumer columns of a warp (a column is one
// stream: a chain, a stream of a bulk call, or one Dirichlet component), the
// next B elements of one domain of that stream.  Layout in shared memory is
// column-minor, val[slot * NC + col], so a warp reading one element per
// column hits NC distinct banks whatever each column's read pointer is.
//
// Two forms: Ring (below; the triangle sampler's U64 rings, NC columns) and
// CRing (further down; 32 columns, circular, top-up refills and lookahead,
// used by every other kernel).
//
// Ring: refill-on-empty (Sec. 2.2), done by the whole warp: every get() is called
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

#include "brng_debug.cuh"
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

  // Refill the rings of the needy columns (all 32 lanes call this).  Lanes
  // with `need` restart their ring; those that also have `gen` (one lane per
  // column, lane == column) put their column on the list to generate.
  // `stream` is this lane's stream.
  __device__ __forceinline__ void refill(bool need, bool gen, uint32_t stream, const RoundKeys& rk) {
    const unsigned lane = lane_id();
    const unsigned mask = __ballot_sync(kFull, need && gen);
    if (need) {
      blk += rp / kEPB;
      rp %= kEPB;
      valid = B;
      if (gen) list[__popc(mask & ((1u << lane) - 1u))] = lane;
    }
    __syncwarp();
    const uint32_t k = __popc(mask);
    if (k == 0) return;
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
  // outputs: the element's raw word and its index in the stream.  `gen`:
  // this lane generates its column when it runs dry (false for lanes that
  // read a column another lane of the warp owns, in step with it).
  __device__ __forceinline__ T get(bool want, uint32_t stream, const RoundKeys& rk,
                                   uint32_t* word = nullptr, uint64_t* index = nullptr,
                                   bool gen = true) {
    const bool need = want && rp >= valid;
    if (__any_sync(kFull, need)) refill(need, gen, stream, rk);
    T v = T(0);
    if (want) {
      BRNG_CHECK(rp < valid && valid <= B);  // the slot was filled by this refill
      const unsigned lane = lane_id();
      v = val[rp * NC + (lane % NC)];
      if (kWords && word) *word = wrd[rp * NC + (lane % NC)];
      if (index) *index = blk * kEPB + rp;
      ++rp;
    }
    return v;
  }
};

// A circular ring of 32 columns (one per lane) for lookahead consumers.
// Element r (counted from the first element of Philox block b0) of a lane
// lives in slot r mod B.  Unlike Ring, a refill appends blocks after the
// last one generated instead of restarting the ring, so nothing is thrown
// away, and a consumer may read (peek) any of the next avail = filled - rp
// elements before it commits to consuming them (advance).
//
// Refill is a top-up: when any lane with `want` has fewer than k elements
// (ensure), every live lane appends as many whole blocks as its free slots
// hold, nb = floor((rp + B - filled) / 4), generating its own column (no
// shuffles, no lists).  Afterwards every live lane has at least B - 3
// elements, so k <= B - 3 is always met by one top-up, even for a ring that
// starts inside a block (rp > filled = 0).  Lanes that consume at different
// rates (tags of a mixed stream, rejections) are thus refilled together, and
// each refill does nearly a full ring of work per lane instead of a few
// blocks for the few lanes that ran dry.  kWords: also keep each element's
// raw Philox word.
//
// kHead > 0: the first min(kHead, B) slots are mirrored after the ring (slot
// s < kHead is also stored at s + B), so the next kHead elements lie in
// consecutive slots from the read point on: a lookahead read is one
// shared-memory load at a constant offset from the read point, with no wrap
// arithmetic.  The ring then occupies B + min(kHead, B) slots (ring_slots).
template <class Gen, bool kWords = false, uint32_t kHead = 0>
struct CRing {
  using T = typename Gen::T;
  static constexpr uint32_t kEPB = Gen::kEPB;
  static_assert(kEPB == 4, "four elements per block");
  static_assert(kHead % kEPB == 0, "whole blocks are mirrored");
  T* val;          // shared: [ring_slots][32]
  uint32_t* wrd;   // shared: [ring_slots][32] when kWords
  uint64_t b0;     // Philox block of relative element 0
  uint32_t rp;     // next relative element to consume
  uint32_t filled; // relative elements generated (multiple of 4)
  uint32_t mask;   // B - 1
  bool live = false;  // get(): also top up this lane when another runs dry

  __host__ __device__ static constexpr uint32_t ring_slots(uint32_t len) {
    return len + (kHead < len ? kHead : len);
  }
  __device__ __forceinline__ void init(T* v, uint32_t* w, uint32_t len, uint64_t pos) {
    val = v; wrd = w; mask = len - 1;
    b0 = pos / kEPB;
    rp = static_cast<uint32_t>(pos % kEPB);
    filled = 0;
  }
  __device__ __forceinline__ uint64_t pos() const { return b0 * kEPB + rp; }
  __device__ __forceinline__ int32_t avail() const { return static_cast<int32_t>(filled - rp); }
  __device__ __forceinline__ uint32_t slot_of(uint32_t i) const {
    if constexpr (kHead > 0) {
      BRNG_CHECK(i < kHead || i <= mask);  // within the mirrored head
      return (rp & mask) + i;
    } else {
      return (rp + i) & mask;
    }
  }
  __device__ __forceinline__ T peek(uint32_t i) const { return val[slot_of(i) * 32u + lane_id()]; }
  __device__ __forceinline__ uint32_t peek_word(uint32_t i) const { return wrd[slot_of(i) * 32u + lane_id()]; }
  __device__ __forceinline__ void advance(uint32_t n) {
    BRNG_CHECK(avail() >= static_cast<int32_t>(n));  // every consumed element was generated
    rp += n;
  }

  __device__ __forceinline__ void gen_own(uint64_t blk, uint32_t slot, uint2 sh, const RoundKeys& rk) {
    const uint4 w = philox_block_sh(blk, sh, rk);
    T v[kEPB];
    Gen::gen(w, v);
#pragma unroll
    for (uint32_t i = 0; i < kEPB; ++i) {
      val[(slot + i) * 32u + lane_id()] = v[i];
      if (kWords) wrd[(slot + i) * 32u + lane_id()] = word_of(w, i);
    }
    if constexpr (kHead > 0) {
      if (slot < kHead) {  // the mirror copy (slot is a multiple of 4, as kHead is)
        const uint32_t m = slot + mask + 1u;
#pragma unroll
        for (uint32_t i = 0; i < kEPB; ++i) {
          val[(m + i) * 32u + lane_id()] = v[i];
          if (kWords) wrd[(m + i) * 32u + lane_id()] = word_of(w, i);
        }
      }
    }
  }

  // Lanes with `live` fill every free slot (inline: the round keys stay
  // kernel parameters, read from the constant bank).
  __device__ __forceinline__ void topup(bool live, uint32_t stream, const RoundKeys& rk) {
    if (!live) return;
    if (filled >= rp) {  // keep the relative counters small: drop whole rings already read
      const uint32_t D = rp & ~mask;
      b0 += D / kEPB;
      rp -= D;
      filled -= D;
    }
    const uint32_t nb = (rp + mask + 1u - filled) / kEPB;
    const uint64_t first = b0 + filled / kEPB;
    BRNG_CHECK(static_cast<int32_t>(filled + nb * kEPB - rp) <= static_cast<int32_t>(mask + 1u));  // no unread slot overwritten
    // one block per iteration, not unrolled: the generator code (Philox and
    // Box-Muller) is long and the instruction cache small; measured on GB300,
    // two blocks in flight (more ILP, three copies of the code) were 5-18 %
    // slower in every kernel
    const uint2 sh = philox_stream_half(Gen::kDom, stream, rk);
#pragma unroll 1
    for (uint32_t j = 0; j < nb; ++j) gen_own(first + j, (filled + j * kEPB) & mask, sh, rk);
    filled += nb * kEPB;
  }

  // At least k <= B - 3 elements for every lane with `want` (all 32 lanes call).
  __device__ __forceinline__ void ensure(bool want, uint32_t k, bool live, uint32_t stream,
                                         const RoundKeys& rk) {
    const bool need = want && avail() < static_cast<int32_t>(k);
    if (__any_sync(kFull, need)) topup(live || need, stream, rk);
    BRNG_CHECK(!want || avail() >= static_cast<int32_t>(k));  // one top-up meets k <= B - 3
  }

  // Next element for lanes with `want` (all 32 lanes call this); `live`: the
  // lane's stream is still in use (topped up along with the needy ones).
  __device__ __forceinline__ T take(bool want, bool live, uint32_t stream, const RoundKeys& rk,
                                    uint32_t* word = nullptr) {
    ensure(want, 1, live, stream, rk);
    T v = T(0);
    if (want) {
      v = peek(0);
      if (kWords && word) *word = peek_word(0);
      ++rp;
    }
    return v;
  }
  // Ring::get's call shape; the lane is topped up when it wants or is `live`.
  __device__ __forceinline__ T get(bool want, uint32_t stream, const RoundKeys& rk,
                                   uint32_t* word = nullptr, uint64_t* = nullptr) {
    return take(want, want || live, stream, rk, word);
  }
};

}  // namespace brng
