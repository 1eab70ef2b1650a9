// brng_batch.cu -- uneven ensembles of Gibbs jobs in one persistent kernel.
//
// A job is one brng_gibbs_run (model, chains, sweeps, seed); its work splits
// into units of one warp each (32 triangle or normal-gamma chains, one LDA
// document).  The host lays the jobs out in a device table in decreasing
// per-unit cost (longest units first) with prefix offsets; a grid of
// resident warps then claims global unit indices from one atomic counter,
// finds the job by binary search and runs the same per-unit body the
// one-kernel-per-job launches run (brng_gibbs.cuh, brng_dirichlet.cuh).  So a
// job's results are identical in a batch and alone, small jobs no longer
// leave the GPU idle (one launch instead of one per job, no per-job tail),
// and the launch is a single kernel after a counter reset, which a CUDA graph
// can capture and replay.
#include <cuda_runtime.h>

#include "brng_dirichlet.cuh"
#include "brng_gibbs.cuh"
#include "brng_internal.h"

namespace brng {

template <int P>
__global__ void __launch_bounds__(512) batch_kernel(const BatchArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned lane = lane_id();
  const unsigned warp = threadIdx.x >> 5;
  unsigned char* base = smem + warp * a.warp_bytes;
  while (true) {
    unsigned long long u = 0;
    if (lane == 0) u = atomicAdd(a.counter, 1ull);
    u = shfl_u64(u, 0);
    if (u >= a.total_units) break;
    uint32_t lo = 0, hi = a.n_jobs - 1;  // last job with first_unit <= u
    while (lo < hi) {
      const uint32_t mid = (lo + hi + 1) >> 1;
      if (a.jobs[mid].first_unit <= u) lo = mid;
      else hi = mid - 1;
    }
    const BatchJob* J = a.jobs + lo;
    const uint64_t local = u - J->first_unit;
    BRNG_CHECK(J->first_unit <= u && local < J->n_units);  // the unit belongs to the job found
    switch (J->model) {
      case BRNG_MODEL_TRIANGLE: {
        const TriangleArgs ta = J->tri;
        triangle_unit<32>(ta, local, base);
        break;
      }
      case BRNG_MODEL_NORMAL_GAMMA: {
        const NormalGammaArgs na = J->ng;
        normal_gamma_unit(na, local, base);
        break;
      }
      default: {
        const DirichletArgs da = J->lda;
        dirichlet_unit<P, true>(da, local, base);
        break;
      }
    }
  }
}

size_t batch_warp_bytes(bool tri, bool ng, bool lda, uint32_t B, uint32_t P, uint32_t Q) {
  size_t w = 128;
  if (tri && triangle_warp_bytes(32, B) > w) w = triangle_warp_bytes(32, B);
  if (ng && normal_gamma_warp_bytes(B) > w) w = normal_gamma_warp_bytes(B);
  if (lda && dirichlet_warp_bytes(P, ring_len_min8(B), Q) > w) w = dirichlet_warp_bytes(P, ring_len_min8(B), Q);
  return w;
}

// Host set-up of a launch (shared-memory attribute, occupancy): done when a
// batch is planned, so that the launch itself is only stream work.
template <int P>
static cudaError_t grid_t(const BatchArgs& a, uint32_t warps_per_block, uint32_t* blocks_out) {
  const size_t smem = static_cast<size_t>(warps_per_block) * a.warp_bytes;
  cudaError_t e = cudaFuncSetAttribute(batch_kernel<P>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 0, per_sm = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_kernel<P>,
                                                    static_cast<int>(32u * warps_per_block), smem);
  if (e != cudaSuccess || per_sm < 1) per_sm = 1;
  // every resident warp claims units: one full wave, fewer if there are fewer units
  uint64_t blocks = static_cast<uint64_t>(sms) * per_sm;
  const uint64_t need = (a.total_units + warps_per_block - 1) / warps_per_block;
  if (need < blocks) blocks = need;
  *blocks_out = static_cast<uint32_t>(blocks);
  return cudaSuccess;
}

cudaError_t batch_grid(const BatchArgs& a, uint32_t P, uint32_t warps_per_block, uint32_t* blocks) {
  if (P <= 1) return grid_t<1>(a, warps_per_block, blocks);
  if (P == 2) return grid_t<2>(a, warps_per_block, blocks);
  if (P <= 4) return grid_t<4>(a, warps_per_block, blocks);
  return cudaErrorInvalidValue;
}

cudaError_t launch_batch(const BatchArgs& a, uint32_t P, uint32_t warps_per_block, uint32_t blocks,
                         cudaStream_t st) {
  if (a.total_units == 0 || blocks == 0) return cudaSuccess;
  const size_t smem = static_cast<size_t>(warps_per_block) * a.warp_bytes;
  const uint32_t threads = 32u * warps_per_block;
  if (P <= 1) batch_kernel<1><<<blocks, threads, smem, st>>>(a);
  else if (P == 2) batch_kernel<2><<<blocks, threads, smem, st>>>(a);
  else if (P <= 4) batch_kernel<4><<<blocks, threads, smem, st>>>(a);
  else return cudaErrorInvalidValue;
  return cudaGetLastError();
}

}  // namespace brng
