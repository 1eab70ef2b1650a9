// brng_gibbs_pc.cu -- the normal-gamma Gibbs sampler with asynchronous
// replenishment (brng_pc.cuh): per block, Wc consumer warps run the sweeps of
// 32 chains each (the same body as the inline form, brng_gibbs.cuh) from
// rings that Wp producer warps keep filled.  Results equal the inline form's
// bit for bit; only who generates the base deviates, and when, differs.
#include <cuda_runtime.h>

#include "brng_gibbs.cuh"
#include "brng_pc.cuh"

namespace brng {

__host__ __device__ inline uint32_t normal_gamma_pc_warp_bytes(uint32_t B) {
  return static_cast<uint32_t>(sizeof(PcCtl)) + 2u * B * 32u * 4u;
}

// PER: consumer warps served by one producer warp (>= ceil(Wc / Wp)).
template <int PER>
__global__ void __launch_bounds__(512) normal_gamma_pc_kernel(const NormalGammaArgs a, uint32_t Wc,
                                                              uint32_t Wp, uint32_t stall) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = lane_id();
  const unsigned warp = threadIdx.x >> 5;
  const uint32_t B = a.B;
  PcCtl* ctl = reinterpret_cast<PcCtl*>(smem);
  float* rings = reinterpret_cast<float*>(smem + Wc * sizeof(PcCtl));
  auto ringN = [&](uint32_t w) { return rings + static_cast<size_t>(w) * 2u * B * 32u; };
  auto ringU = [&](uint32_t w) { return rings + (static_cast<size_t>(w) * 2u + 1u) * B * 32u; };
  const uint64_t unit0 = static_cast<uint64_t>(blockIdx.x) * Wc;

  if (warp < Wc) {
    // ---- consumer: 32 chains ----
    const uint64_t unit = unit0 + warp;
    const bool has = unit * 32 < a.n_chains;  // warp-uniform
    const uint64_t c = unit * 32 + lane;
    const bool active = c < a.n_chains;
    const uint32_t stream = static_cast<uint32_t>(a.chain_offset + c);
    NgChain s = ng_load(a, c, active);
    PcRing<GenN> RN;
    PcRing<GenU> RU;
    RN.init(ringN(warp), &ctl[warp], 0, B, s.pn, a.cnt);
    RU.init(ringU(warp), &ctl[warp], 1, B, s.pu, a.cnt);
    if (lane == 0) ctl[warp].done = has ? 0u : 1u;
    __syncthreads();  // counters and flags set; producers have read positions
    if (has) {
      ng_sweeps_any(a, a.n_sweeps, stream, active, s, RN, RU);
      ng_fold_moments(s);
      RN.flush();
      RU.flush();
      ng_store(a, c, active, s);
      __syncwarp();
      if (lane == 0) st_release_cta(&ctl[warp].done, 1u);
    }
    return;
  }

  // ---- producer: lane l fills lane l of consumer warps j, j + Wp, ... ----
  const uint32_t j = warp - Wc;
  PcFill fN[PER], fU[PER];
  bool alive[PER];
#pragma unroll
  for (int k = 0; k < PER; ++k) {
    const uint32_t w = j + static_cast<uint32_t>(k) * Wp;
    const uint64_t unit = unit0 + w;
    alive[k] = w < Wc && unit * 32 < a.n_chains;
    const uint64_t c = unit * 32 + lane;
    const bool on = alive[k] && c < a.n_chains;
    uint64_t pn = 0, pu = 0;
    if (on) {
      const brng_normal_gamma_state_t st = a.state[c];
      pn = st.pos_n;
      pu = st.pos_u;
    }
    const uint32_t stream = static_cast<uint32_t>(a.chain_offset + c);
    fN[k] = PcFill{pn / 4u, 0ull, stream, on};
    fU[k] = PcFill{pu / 4u, 0ull, stream, on};
  }
  __syncthreads();
  if (stall) return;  // failure-path test: the consumers' waits must run out
  uint64_t t0 = 0;
  while (true) {
    bool progress = false, any = false;
#pragma unroll
    for (int k = 0; k < PER; ++k) {
      if (!alive[k]) continue;
      const uint32_t w = j + static_cast<uint32_t>(k) * Wp;
      // lane 0's view of the flag decides for the warp (the loop stays uniform)
      if (__shfl_sync(kFull, ld_acquire_cta(&ctl[w].done), 0)) {
        alive[k] = false;
        continue;
      }
      any = true;
      progress |= pc_fill_one<GenN>(fN[k], ringN(w), &ctl[w].tail[0][lane], &ctl[w].head[0][lane], B, a.rk);
      progress |= pc_fill_one<GenU>(fU[k], ringU(w), &ctl[w].tail[1][lane], &ctl[w].head[1][lane], B, a.rk);
    }
    if (!any) break;
    if (__any_sync(kFull, progress)) {
      t0 = 0;
    } else {
      const uint64_t now = shfl_u64(global_ns(), 0);
      if (t0 == 0) {
        t0 = now;
      } else if (now - t0 > kPcWaitNs) {  // consumers stopped reading: give up
        if (lane == 0) atomicAdd(&a.cnt->n_timeout, 1u);
        break;
      }
      __nanosleep(64);
    }
  }
}

template <int PER>
static cudaError_t launch_pc_t(const NormalGammaArgs& a, uint32_t Wc, uint32_t Wp, size_t smem,
                               uint64_t blocks, cudaStream_t st, bool stall) {
  cudaError_t e = cudaFuncSetAttribute(normal_gamma_pc_kernel<PER>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  normal_gamma_pc_kernel<PER><<<static_cast<unsigned>(blocks), 32u * (Wc + Wp), smem, st>>>(a, Wc, Wp,
                                                                                          stall ? 1u : 0u);
  return cudaGetLastError();
}

cudaError_t launch_normal_gamma_pc(const NormalGammaArgs& a, uint32_t Wc, uint32_t Wp, cudaStream_t st,
                                   bool stall) {
  const uint64_t units = (static_cast<uint64_t>(a.n_chains) + 31) / 32;
  if (units == 0) return cudaSuccess;
  if (Wc < 1 || Wp < 1 || Wc + Wp > 16 || a.B < 4 || (a.B & (a.B - 1)) != 0) return cudaErrorInvalidValue;
  const size_t smem = static_cast<size_t>(Wc) * normal_gamma_pc_warp_bytes(a.B);
  const uint64_t blocks = (units + Wc - 1) / Wc;
  const uint32_t per = (Wc + Wp - 1) / Wp;
  if (per <= 1) return launch_pc_t<1>(a, Wc, Wp, smem, blocks, st, stall);
  if (per <= 2) return launch_pc_t<2>(a, Wc, Wp, smem, blocks, st, stall);
  if (per <= 4) return launch_pc_t<4>(a, Wc, Wp, smem, blocks, st, stall);
  if (per <= 8) return launch_pc_t<8>(a, Wc, Wp, smem, blocks, st, stall);
  return cudaErrorInvalidValue;  // a producer warp serves at most 8 consumer warps
}

size_t normal_gamma_pc_bytes_per_warp(uint32_t B) { return normal_gamma_pc_warp_bytes(B); }

}  // namespace brng
