// brng_gibbs.cu -- one-kernel-per-job launches of the triangle Gibbs sampler of
// Eq. 1 / Fig. 1 and of the normal-gamma Gibbs sampler (bodies in brng_gibbs.cuh).  Each chain is a Philox
// stream (global chain id) and a lane; its state stays in registers for the
// whole run and its base deviates come from the warp-shared rings.
#include <cuda_runtime.h>

#include <cmath>

#include "brng_gibbs.cuh"

namespace brng {

template <int NC>
__global__ void __launch_bounds__(512) triangle_kernel(const TriangleArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned warp = threadIdx.x >> 5;
  const uint64_t unit = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
  triangle_unit<NC>(a, unit, smem + warp * triangle_warp_bytes(NC, a.B));
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

__global__ void __maxnreg__(128) normal_gamma_kernel(const NormalGammaArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned warp = threadIdx.x >> 5;
  const uint64_t unit = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
  normal_gamma_unit(a, unit, smem + warp * normal_gamma_warp_bytes(a.B));
}

size_t normal_gamma_bytes_per_warp(uint32_t B) { return normal_gamma_warp_bytes(B); }

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
