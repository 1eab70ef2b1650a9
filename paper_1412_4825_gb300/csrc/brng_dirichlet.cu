// brng_dirichlet.cu -- launches of the Dirichlet-row and LDA kernels (bodies in
// brng_dirichlet.cuh).
#include <cuda_runtime.h>

#include "brng_dirichlet.cuh"

namespace brng {

// Two register budgets.  The natural one (107 registers at two components
// per lane) lets about 16 warps share an SM; capped at 80 (a few spilled
// words), 24 -- which pays only when the warps' rings and row queues leave
// shared memory for them.  Measured on GB300, the K = 64 LDA step, 16,384
// documents x 500 sweeps, 4 warps per block: rings of 16 with lookahead 4,
// 10.03 ms uncapped and 8.77 capped (9.12 at 96, 8.87 at 72, 11.29 at 64);
// lookahead 8, 9.85 and 9.32; lookahead 16 (room for 18 warps), 9.83 and
// 10.38; rings of 32, 11.83 and 12.49.  So the launch takes the capped kernel
// when shared memory holds at least 20 of its warps; four components per
// lane always take the natural budget.
constexpr int kDirichletTightRegs = 80;
constexpr uint32_t kDirichletTightWarps = 20;

template <int P, bool LDA, bool TIGHT>
__global__ void __maxnreg__(TIGHT ? kDirichletTightRegs : 128) dirichlet_kernel(const DirichletArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const unsigned warp = threadIdx.x >> 5;
  const uint64_t unit = static_cast<uint64_t>(blockIdx.x) * (blockDim.x >> 5) + warp;
  dirichlet_unit<P, LDA>(a, unit, smem + warp * dirichlet_warp_bytes(P, a.B, a.lookahead));
}

template <int P, bool LDA, bool TIGHT>
static cudaError_t launch_dir_k(const DirichletArgs& a, uint64_t blocks, uint32_t threads, size_t smem,
                                cudaStream_t st) {
  cudaError_t e = cudaFuncSetAttribute(dirichlet_kernel<P, LDA, TIGHT>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  dirichlet_kernel<P, LDA, TIGHT><<<static_cast<unsigned>(blocks), threads, smem, st>>>(a);
  return cudaGetLastError();
}

template <int P, bool LDA>
static cudaError_t launch_dir_t(const DirichletArgs& a, const Geometry& g, cudaStream_t st) {
  const uint64_t n_units = LDA ? a.n_docs : (a.n_rows < a.R ? a.n_rows : a.R);
  if (n_units == 0) return cudaSuccess;
  const uint32_t threads = 32u * g.warps_per_block;
  const size_t per_warp = dirichlet_warp_bytes(P, a.B, a.lookahead);
  const size_t smem = static_cast<size_t>(g.warps_per_block) * per_warp;
  const uint64_t blocks = (n_units + g.warps_per_block - 1) / g.warps_per_block;
  if constexpr (P <= 2) {
    int dev = 0, smem_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (e != cudaSuccess) return e;
    if (per_warp * kDirichletTightWarps <= static_cast<size_t>(smem_sm))
      return launch_dir_k<P, LDA, true>(a, blocks, threads, smem, st);
  }
  return launch_dir_k<P, LDA, false>(a, blocks, threads, smem, st);
}

cudaError_t launch_dirichlet(const DirichletArgs& a, const Geometry& g, bool lda, cudaStream_t st) {
  const uint32_t P = (a.K + 31) / 32;
  if (P == 1) return lda ? launch_dir_t<1, true>(a, g, st) : launch_dir_t<1, false>(a, g, st);
  if (P == 2) return lda ? launch_dir_t<2, true>(a, g, st) : launch_dir_t<2, false>(a, g, st);
  if (P <= 4) return lda ? launch_dir_t<4, true>(a, g, st) : launch_dir_t<4, false>(a, g, st);
  return cudaErrorInvalidValue;
}

}  // namespace brng
