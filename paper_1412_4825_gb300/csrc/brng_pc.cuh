// brng_pc.cuh -- asynchronous replenishment of the buffers: producer warps
// keep the rings filled while consumer warps run the sampler (the paper's
// closing idea of refilling the buffers in the background, Sec. 3 item 3, in its
// GPU form: warp specialisation inside one block).
//
// A block holds Wc consumer warps (32 chains each, as in the inline form) and
// Wp producer warps.  Each consumer lane has, per domain, a ring of B slots
// in shared memory (column-minor, val[slot * 32 + lane]) and two counters in
// the warp's control block: `tail` (elements written, set by the producer)
// and `head` (elements read, set by the consumer), both counted from the
// first element of the Philox block that held the lane's start position.
// Element r of the lane's sequence lives in slot r mod B; the producer may
// write block [t, t + 4) once t + 4 <= head + B.  Tail is published with a
// release store after the values, head after the reads it covers, and both
// are read with acquire loads, so a slot is never read before it is written
// or overwritten before it is read.  Values are still a pure function of the
// position (counter-based generator), so results equal the inline form's.
//
// Producer lane l of producer warp j serves lane l of consumer warps
// j, j + Wp, j + 2 Wp, ...; it generates a block for every ring of its lanes
// that has room, round after round, and stops when its consumer warps say
// they are done.  Every wait is bounded: a consumer that sees no new element,
// or a producer that finds no room anywhere, for kPcWaitNs of the global
// timer gives up, counts a timeout and returns (the consumer's chains then
// end with NaN state).
#pragma once

#include <cstdint>

#include "brng_gamma.cuh"

namespace brng {

constexpr uint64_t kPcWaitNs = 1000000000ull;  // 1 s without progress

__device__ __forceinline__ uint64_t global_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ uint32_t ld_acquire_cta(const uint32_t* p) {
  uint32_t v;
  asm volatile("ld.acquire.cta.shared.u32 %0, [%1];" : "=r"(v) : "r"(smem_addr(p)) : "memory");
  return v;
}

__device__ __forceinline__ void st_release_cta(uint32_t* p, uint32_t v) {
  asm volatile("st.release.cta.shared.u32 [%0], %1;" ::"r"(smem_addr(p)), "r"(v) : "memory");
}

// Per consumer warp: counters of its 32 lanes for two domains, and its flag.
struct PcCtl {
  uint32_t tail[2][32];
  uint32_t head[2][32];
  uint32_t done;
  uint32_t pad[31];
};

// Consumer side of one ring (one domain of one lane).  Same calls as CRing
// (ensure / peek / advance / get) so that the samplers' bodies take either.
// Positions are 64-bit; the counters shared with the producer are their low
// 32 bits (differences stay far below 2^31).
template <class Gen>
struct PcRing {
  using T = typename Gen::T;
  static constexpr uint32_t kEPB = Gen::kEPB;
  T* val;            // shared: [B][32]
  uint32_t* tail_p;  // this lane's tail
  uint32_t* head_p;  // this lane's head
  uint64_t b0;       // Philox block of relative element 0
  uint64_t p;        // next relative element
  uint32_t seen;     // last tail read
  uint32_t mask;     // B - 1
  DevCounters* cnt;
  bool failed;       // warp-uniform: a wait ran out

  // Before the block barrier that starts the producers.
  __device__ __forceinline__ void init(T* v, PcCtl* ctl, int dom, uint32_t len, uint64_t pos,
                                       DevCounters* c) {
    const unsigned lane = lane_id();
    val = v;
    tail_p = &ctl->tail[dom][lane];
    head_p = &ctl->head[dom][lane];
    b0 = pos / kEPB;
    p = pos % kEPB;
    seen = 0;
    mask = len - 1;
    cnt = c;
    failed = false;
    *tail_p = 0;
    *head_p = static_cast<uint32_t>(p);
  }
  __device__ __forceinline__ uint64_t pos() const { return b0 * kEPB + p; }
  __device__ __forceinline__ T peek(uint32_t i) const {
    return failed ? T(NAN) : val[((static_cast<uint32_t>(p) + i) & mask) * 32u + lane_id()];
  }
  // Commits n elements and hands their slots back to the producer.
  __device__ __forceinline__ void advance(uint32_t n) {
    BRNG_CHECK(failed || static_cast<int32_t>(seen - static_cast<uint32_t>(p)) >= static_cast<int32_t>(n));
    p += n;
    st_release_cta(head_p, static_cast<uint32_t>(p));
  }

  // Waits until k elements are available to every lane with `want` (all 32
  // lanes call this; k <= B - 3, since the producer writes whole blocks).
  __device__ __forceinline__ void ensure(bool want, uint32_t k, bool = false, uint32_t = 0,
                                         const RoundKeys& = RoundKeys{}) {
    bool need = want && static_cast<int32_t>(seen - static_cast<uint32_t>(p)) < static_cast<int32_t>(k);
    if (!__any_sync(kFull, need)) return;
    // the producer must see every slot this lane has read before it waits
    st_release_cta(head_p, static_cast<uint32_t>(p));
    uint64_t t0 = 0;
    while (true) {
      if (need) {
        seen = ld_acquire_cta(tail_p);
        need = static_cast<int32_t>(seen - static_cast<uint32_t>(p)) < static_cast<int32_t>(k);
      }
      if (!__any_sync(kFull, need)) break;
      const uint64_t now = shfl_u64(global_ns(), 0);  // one clock for the warp
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > kPcWaitNs) {
        failed = true;
        if (lane_id() == 0) atomicAdd(&cnt->n_timeout, 1u);
        break;
      }
    }
    BRNG_CHECK(failed || !want || static_cast<int32_t>(seen - static_cast<uint32_t>(p)) >= static_cast<int32_t>(k));
  }

  // Next element for lanes with `want` (all 32 lanes call this).
  __device__ __forceinline__ T get(bool want, uint32_t = 0, const RoundKeys& = RoundKeys{},
                                   uint32_t* = nullptr, uint64_t* = nullptr) {
    ensure(want, 1);
    T v = T(0);
    if (want) {
      v = peek(0);
      ++p;
      if ((p & 3u) == 0) st_release_cta(head_p, static_cast<uint32_t>(p));  // every block
    }
    return v;
  }

  // Publishes the final head (so a producer never waits on a stale one).
  __device__ __forceinline__ void flush() { st_release_cta(head_p, static_cast<uint32_t>(p)); }
};

template <class G>
__device__ __forceinline__ bool ring_failed(const PcRing<G>& r) { return r.failed; }

// One producer lane's view of one ring it fills.
struct PcFill {
  uint64_t b0;      // Philox block of relative element 0
  uint64_t t;       // elements written (multiple of 4)
  uint32_t stream;  // Philox stream
  bool on;          // this lane's column has a chain
};

// Fills one block into a ring if it has room; returns whether it did.
template <class Gen>
__device__ __forceinline__ bool pc_fill_one(PcFill& f, typename Gen::T* val, uint32_t* tail_p,
                                            const uint32_t* head_p, uint32_t B, const RoundKeys& rk) {
  if (!f.on) return false;
  const uint32_t h = ld_acquire_cta(head_p);
  if (static_cast<int32_t>(static_cast<uint32_t>(f.t) + 4u - (h + B)) > 0) return false;
  const uint4 w = philox_block(f.b0 + f.t / 4u, Gen::kDom, f.stream, rk);
  typename Gen::T v[4];
  Gen::gen(w, v);
  const uint32_t lane = lane_id();
  const uint32_t s = static_cast<uint32_t>(f.t) & (B - 1u);
#pragma unroll
  for (uint32_t i = 0; i < 4; ++i) val[(s + i) * 32u + lane] = v[i];
  f.t += 4u;
  st_release_cta(tail_p, static_cast<uint32_t>(f.t));
  return true;
}

}  // namespace brng
