// brng_internal.h -- declarations shared by the library's translation units
// (host launchers of the kernels and the handle layout).
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

#include "brng.h"
#include <nvtx3/nvToolsExt.h>
#include "brng_engine.cuh"

namespace brng {

// An NVTX range over a host-side call or phase: Nsight tools show the
// library's calls by name (and ncu --nvtx can filter on them); without a tool
// attached a push/pop costs a few nanoseconds.
struct TraceRange {
  explicit TraceRange(const char* name) { nvtxRangePushA(name); }
  ~TraceRange() { nvtxRangePop(); }
  TraceRange(const TraceRange&) = delete;
  TraceRange& operator=(const TraceRange&) = delete;
};


struct DevCounters;

constexpr uint32_t kDefaultBufLen = 32;
constexpr uint32_t kMaxBufLen = 512;
constexpr uint32_t kDefaultWarpsPerBlock = 4;
constexpr uint32_t kDefaultLookahead = 8;
constexpr uint32_t kDefaultProducerWarps = BRNG_PRODUCERS_NONE;
constexpr int kTagMixed = -1;
constexpr float kPoissonMaxLambda = 1e7f;   // Poisson: 0 < lambda <= this
constexpr float kInversionMaxMean = 64.0f;  // Poisson / Binomial by inversion up to this mean, PTRS / BTRD above
constexpr int kPoissonMaxK = 1024;          // the inversion's search stops here at the latest
constexpr uint32_t kBulkMinRing = 8;  // bulk streams and Dirichlet rows use rings of at least this length
// (a step may take 2 U elements from a top-up ring, which guarantees B - 3)
inline uint32_t ring_len_min8(uint32_t B) { return B < kBulkMinRing ? kBulkMinRing : B; }

// Launch geometry shared by all kernels: warps per block and ring length.
struct Geometry {
  uint32_t warps_per_block;
  uint32_t buf_len;
};

// ---- bulk varying-parameter streams (brng_bulk.cu) ----
struct BulkArgs {
  RoundKeys rk;
  uint64_t n;
  uint32_t S;
  uint32_t B;
  const uint8_t* tag;
  const float* p0;
  const float* p1;
  float* out;
  uint32_t* words;
  uint64_t* pos;  // SoA: pos[d * S + s], d = U, N, E
  DevCounters* cnt;
  unsigned int* mixed_flag = nullptr;  // mixed stream: device word, 1 if a Poisson/Binomial tag is present
};
cudaError_t launch_bulk(int tag, const BulkArgs& a, const Geometry& g, cudaStream_t st);
cudaError_t launch_philox_words(const RoundKeys& rk, uint32_t dom, uint32_t stream,
                                uint64_t first_block, size_t n_blocks, uint32_t* out,
                                cudaStream_t st);

cudaError_t launch_philox_peak(const RoundKeys& rk, uint64_t iters, uint32_t blocks, uint32_t threads,
                               uint32_t* sink, cudaStream_t st);
cudaError_t launch_fp32_eval(uint32_t fn, size_t n, const float* in, float* out, cudaStream_t st);
cudaError_t launch_fp64_eval(uint32_t fn, size_t n, const double* in, double* out, cudaStream_t st);

// ---- Dirichlet rows and LDA sweeps (brng_dirichlet.cu) ----
struct DirichletArgs {
  RoundKeys rk;
  uint32_t K;
  uint32_t B;
  uint32_t lookahead;
  // bulk rows: rows i = r + m R of row-stream r, component streams r K + k
  uint64_t n_rows;
  uint32_t R;
  const float* alpha;  // [rows][K]
  float* out;          // [rows][K] (bulk) or last theta (LDA)
  uint64_t* pos;       // bulk: SoA [3][S]; LDA: [docs][K][2] (N, U)
  uint32_t S;          // bulk: stream count
  // LDA
  uint64_t stream_base;  // LDA: (chain_offset) -> component stream (base + d) K + k
  uint32_t n_docs;
  uint32_t n_sweeps;
  double* moments;  // LDA: [docs][K]
  DevCounters* cnt;
};
cudaError_t launch_dirichlet(const DirichletArgs& a, const Geometry& g, bool lda, cudaStream_t st);

// FP64 uniform from the U64 domain, one thread per stream (brng_bulk.cu)
struct Uniform64Args {
  RoundKeys rk;
  uint64_t n;
  uint32_t S;
  const double *a, *b;
  double* out;
  uint32_t* words;
  uint64_t* pos64;  // [S]
  DevCounters* cnt;
};
cudaError_t launch_uniform64(const Uniform64Args& a, cudaStream_t st);

// ---- Gibbs models (brng_gibbs.cu) ----
struct TriangleArgs {
  RoundKeys rk;
  uint64_t chain_offset;
  uint32_t n_chains, n_sweeps, B;
  brng_triangle_state_t* state;
  double* moments;
  DevCounters* cnt;
};
cudaError_t launch_triangle(const TriangleArgs& a, const Geometry& g, uint32_t lanes_per_chain,
                            cudaStream_t st);

struct NormalGammaArgs {
  RoundKeys rk;
  uint64_t chain_offset;
  uint32_t n_chains, n_sweeps, B;
  float a0, b0, mu0, prec0;
  const float *nobs, *xbar, *sc;
  brng_normal_gamma_state_t* state;
  double* moments;
  DevCounters* cnt;
};
cudaError_t launch_normal_gamma(const NormalGammaArgs& a, const Geometry& g, cudaStream_t st);
// With Wc consumer and Wp producer warps per block (brng_gibbs_pc.cu).
// `stall` (failure-path tests only): the producers write nothing, so every
// consumer wait runs out after its bound.
cudaError_t launch_normal_gamma_pc(const NormalGammaArgs& a, uint32_t Wc, uint32_t Wp, cudaStream_t st,
                                   bool stall = false);
size_t normal_gamma_bytes_per_warp(uint32_t B);     // shared memory per warp (inline rings)
size_t normal_gamma_pc_bytes_per_warp(uint32_t B);  // shared memory per consumer warp

// ---- full LDA step: topic draws per token (brng_lda_full.cu) ----
struct LdaZArgs {
  RoundKeys rk;
  uint64_t doc_offset;       // global id of document 0 (its Z stream id)
  uint32_t n_docs, K, V;
  float alpha, beta, vbeta;  // vbeta = float(V) * beta, rounded once on the host
  uint32_t qbits;            // bits per integer weight: 32 - ceil(log2 K)
  const uint32_t* doc_ptr;   // [n_docs + 1]
  const uint32_t* words;     // [tokens]
  const uint32_t* prev;      // [tokens]
  const uint32_t* order;     // [n_docs] processing order, or null (identity)
  uint8_t* z;                // [tokens]
  uint8_t* z_start;          // [tokens]
  int32_t* ndk;              // [n_docs][K]
  const int32_t* nkw;        // [V][K] snapshot
  const int32_t* nk;         // [K] snapshot
  int32_t* dnkw;             // [V*K + K] changes
  float* dir_alpha;          // [n_docs][K]
  uint64_t* zpos;            // [n_docs]
};
cudaError_t launch_lda_index(uint32_t n_docs, const uint32_t* doc_ptr, const uint32_t* words, uint32_t* prev,
                             cudaStream_t st);
cudaError_t launch_lda_z(const LdaZArgs& a, cudaStream_t st);
cudaError_t launch_lda_apply(uint32_t K, uint32_t V, int32_t* nkw, int32_t* nk, int32_t* dnkw, cudaStream_t st);

// ---- batched persistent kernel (brng_batch.cu) ----
struct BatchJob {
  uint32_t model;       // brng_model_t
  uint32_t pad;
  uint64_t first_unit;  // global index of the job's first unit (prefix sum)
  uint64_t n_units;
  TriangleArgs tri;
  NormalGammaArgs ng;
  DirichletArgs lda;
};
struct BatchArgs {
  const BatchJob* jobs;  // device, ordered by first_unit
  uint32_t n_jobs;
  uint32_t warp_bytes;   // shared memory per warp (max over the models present)
  uint64_t total_units;
  unsigned long long* counter;  // device, zeroed before each launch
};
size_t batch_warp_bytes(bool tri, bool ng, bool lda, uint32_t B, uint32_t P, uint32_t Q);
cudaError_t batch_grid(const BatchArgs& a, uint32_t P, uint32_t warps_per_block, uint32_t* blocks);
// Plans `jobs` with the handle's tuning and launches them as one batch on
// `st`, using (and growing) the caller's device table and counter.
int batch_launch_into(brng_t* h, const brng_job_t* jobs, uint32_t n_jobs, BatchJob** d_table,
                      size_t* cap, unsigned long long** d_counter, cudaStream_t st);
cudaError_t launch_batch(const BatchArgs& a, uint32_t P, uint32_t warps_per_block, uint32_t blocks,
                         cudaStream_t st);

}  // namespace brng
