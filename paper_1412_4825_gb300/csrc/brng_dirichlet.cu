// brng_dirichlet.cu -- launches of the Dirichlet-row and LDA kernels (bodies in
// brng_dirichlet.cuh).
#include <cuda_runtime.h>

#include "brng_dirichlet.cuh"

namespace brng {

// Register cap: up to two components per lane at 80 (a few spilled words at
// P = 2; the K = 64 LDA step, 16,384 documents x 500 sweeps, measured on
// GB300: 9.83 ms at its natural 107 registers, 9.12 at 96, 8.77 at 80 with
// rings of 16 and lookahead 4, 8.87 at 72, 9.66 at 64), four at 128.
template <int P>
constexpr int kDirichletMaxRegs = P >= 4 ? 128 : 80;

template <int P, bool LDA>
__global__ void __maxnreg__(kDirichletMaxRegs<P>) dirichlet_kernel(const DirichletArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned warp = threadIdx.x >> 5;
  const uint64_t unit = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
  dirichlet_unit<P, LDA>(a, unit, smem + warp * dirichlet_warp_bytes(P, a.B, a.lookahead));
}

template <int P, bool LDA>
static cudaError_t launch_dir_t(const DirichletArgs& a, const Geometry& g, cudaStream_t st) {
  const uint64_t n_units = LDA ? a.n_docs : (a.n_rows < a.R ? a.n_rows : a.R);
  if (n_units == 0) return cudaSuccess;
  const uint32_t threads = 32u * g.warps_per_block;
  const size_t smem = static_cast<size_t>(g.warps_per_block) * dirichlet_warp_bytes(P, a.B, a.lookahead);
  const uint64_t blocks = (n_units + g.warps_per_block - 1) / g.warps_per_block;
  cudaError_t e = cudaFuncSetAttribute(dirichlet_kernel<P, LDA>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  dirichlet_kernel<P, LDA><<<static_cast<unsigned>(blocks), threads, smem, st>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_dirichlet(const DirichletArgs& a, const Geometry& g, bool lda, cudaStream_t st) {
  const uint32_t P = (a.K + 31) / 32;
  if (P == 1) return lda ? launch_dir_t<1, true>(a, g, st) : launch_dir_t<1, false>(a, g, st);
  if (P == 2) return lda ? launch_dir_t<2, true>(a, g, st) : launch_dir_t<2, false>(a, g, st);
  if (P <= 4) return lda ? launch_dir_t<4, true>(a, g, st) : launch_dir_t<4, false>(a, g, st);
  return cudaErrorInvalidValue;
}

}  // namespace brng
