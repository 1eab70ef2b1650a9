// brng_api.cu -- the C ABI (include/brng.h): handle, argument checks,
// dispatch to the kernels.  Plain pointers and sizes only; all compute runs in
// the kernels of brng_bulk.cu, brng_dirichlet.cu and brng_gibbs.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "brng.h"
#include "brng_gamma.cuh"
#include "brng_internal.h"

#ifdef BRNG_DEBUG
namespace brng {
namespace {
std::vector<unsigned long long (*)(bool)>& debug_readers() {
  static std::vector<unsigned long long (*)(bool)> r;  // filled at library load
  return r;
}
}  // namespace
void register_debug_reader(unsigned long long (*read)(bool reset)) { debug_readers().push_back(read); }
}  // namespace brng
#endif

struct brng_handle {
  uint64_t seed;
  uint32_t S;
  brng_tuning_t tune;
  brng::RoundKeys rk;
  uint64_t* d_pos;            // SoA [3][S]: U, N, E positions of every stream
  uint64_t* d_pos64;          // [S]: U64-domain positions (brng_uniform_f64)
  brng::DevCounters* d_cnt;   // device counters
  unsigned int* d_flag;       // the mixed stream's dispatch word (discrete tags present)
  int device;
  brng::BatchJob* d_batch_jobs = nullptr;        // brng_gibbs_batch job table
  size_t batch_cap = 0;
  unsigned long long* d_batch_counter = nullptr;  // brng_gibbs_batch unit counter
};

namespace {

bool pow2_in(uint32_t v, uint32_t lo, uint32_t hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; }

int cuda_status(cudaError_t e) {
  if (e == cudaSuccess) return BRNG_OK;
  if (e == cudaErrorMemoryAllocation) return BRNG_ENOMEM;
  if (e == cudaErrorInvalidValue) return BRNG_EINVAL;
  return BRNG_ECUDA;
}

// Launch geometry for a kernel needing `per_warp` bytes of shared memory per
// warp: the tuned warps per block, reduced until a block fits the device's
// opt-in shared memory (values never depend on it).  warps_per_block = 0 if
// not even one warp fits.
brng::Geometry geometry(const brng_t* h, size_t per_warp) {
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  uint32_t w = h->tune.warps_per_block;
  while (w > 0 && per_warp * w > static_cast<size_t>(optin)) --w;
  return brng::Geometry{w, h->tune.buf_len};
}

const char* bulk_name(int tag) {
  static const char* const names[] = {"brng_uniform", "brng_normal", "brng_exponential", "brng_gamma",
                                      "brng_laplace", "brng_weibull", "brng_poisson", "brng_binomial"};
  return (tag >= 0 && tag < 8) ? names[tag] : "brng_mixed";
}

int bulk(brng_t* h, int tag, size_t n, const uint8_t* tagv, const float* p0, const float* p1,
         float* out, uint32_t* words, cudaStream_t st) {
  const brng::TraceRange trace(bulk_name(tag));
  if (!h) return BRNG_EINVAL;
  if (n == 0) return BRNG_OK;
  if (!p0 || !out || (tag == brng::kTagMixed && !tagv)) return BRNG_EINVAL;
  const bool two = tag == brng::kTagMixed || tag == BRNG_TAG_UNIFORM || tag == BRNG_TAG_NORMAL ||
                   tag == BRNG_TAG_LAPLACE || tag == BRNG_TAG_WEIBULL || tag == BRNG_TAG_BINOMIAL;
  if (two && tag != brng::kTagMixed && !p1) return BRNG_EINVAL;
  const int ndom = (tag == brng::kTagMixed) ? 3 : (tag == BRNG_TAG_GAMMA || tag == BRNG_TAG_LAPLACE) ? 2 : 1;
  const size_t per_warp =
      128u + static_cast<size_t>(ndom) * std::max(h->tune.buf_len, brng::kBulkMinRing) * 128u * (words ? 2 : 1);
  const brng::Geometry g = geometry(h, per_warp);
  if (g.warps_per_block == 0) return BRNG_EINVAL;
  brng::BulkArgs a;
  a.rk = h->rk;
  a.n = n;
  a.S = h->S;
  a.B = h->tune.buf_len;
  a.tag = tagv;
  a.p0 = p0;
  a.p1 = p1;
  a.out = out;
  a.words = words;
  a.pos = h->d_pos;
  a.cnt = h->d_cnt;
  a.mixed_flag = h->d_flag;
  return cuda_status(brng::launch_bulk(tag, a, g, st));
}

}  // namespace

extern "C" {

int brng_create(uint64_t seed, uint32_t n_streams, uint32_t buf_len, brng_t** out) {
  const brng::TraceRange trace("brng_create");
  if (!out || n_streams == 0) return BRNG_EINVAL;
  if (buf_len == 0) buf_len = brng::kDefaultBufLen;
  if (!pow2_in(buf_len, 4, brng::kMaxBufLen)) return BRNG_EINVAL;
  brng_t* h = new (std::nothrow) brng_t();
  if (!h) return BRNG_ENOMEM;
  h->seed = seed;
  h->S = n_streams;
  h->tune.buf_len = buf_len;
  h->tune.warps_per_block = brng::kDefaultWarpsPerBlock;
  h->tune.lanes_per_chain = 1;
  h->tune.lookahead = brng::kDefaultLookahead;
  h->tune.producer_warps = brng::kDefaultProducerWarps;
  h->rk = brng::make_round_keys(seed);
  cudaGetDevice(&h->device);
  const size_t pos_bytes = sizeof(uint64_t) * 3ull * n_streams;
  h->d_pos = nullptr;
  h->d_pos64 = nullptr;
  h->d_cnt = nullptr;
  h->d_flag = nullptr;
  cudaError_t e = cudaMalloc(&h->d_pos, pos_bytes);
  if (e == cudaSuccess) e = cudaMalloc(&h->d_pos64, sizeof(uint64_t) * static_cast<size_t>(n_streams));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_cnt, sizeof(brng::DevCounters));
  if (e == cudaSuccess) e = cudaMalloc(&h->d_flag, sizeof(unsigned int));
  if (e == cudaSuccess) e = cudaMemset(h->d_pos, 0, pos_bytes);
  if (e == cudaSuccess) e = cudaMemset(h->d_pos64, 0, sizeof(uint64_t) * static_cast<size_t>(n_streams));
  if (e == cudaSuccess) e = cudaMemset(h->d_cnt, 0, sizeof(brng::DevCounters));
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(h->d_pos);
    cudaFree(h->d_pos64);
    cudaFree(h->d_cnt);
    cudaFree(h->d_flag);
    delete h;
    return cuda_status(e);
  }
  *out = h;
  return BRNG_OK;
}

int brng_destroy(brng_t* h) {
  if (!h) return BRNG_OK;
  cudaFree(h->d_batch_jobs);
  cudaFree(h->d_batch_counter);
  cudaFree(h->d_pos64);
  cudaFree(h->d_flag);
  cudaError_t e1 = cudaFree(h->d_pos);
  cudaError_t e2 = cudaFree(h->d_cnt);
  delete h;
  return e1 != cudaSuccess ? cuda_status(e1) : cuda_status(e2);
}

int brng_set_tuning(brng_t* h, const brng_tuning_t* t) {
  if (!h || !t) return BRNG_EINVAL;
  brng_tuning_t n = h->tune;
  if (t->buf_len) n.buf_len = t->buf_len;
  if (t->warps_per_block) n.warps_per_block = t->warps_per_block;
  if (t->lanes_per_chain) n.lanes_per_chain = t->lanes_per_chain;
  if (t->lookahead) n.lookahead = t->lookahead;
  if (t->producer_warps) n.producer_warps = t->producer_warps;
  if (!pow2_in(n.buf_len, 4, brng::kMaxBufLen)) return BRNG_EINVAL;
  if (n.warps_per_block < 1 || n.warps_per_block > 16) return BRNG_EINVAL;
  if (!pow2_in(n.lanes_per_chain, 1, 32)) return BRNG_EINVAL;
  if (n.lookahead < 1 || n.lookahead > 16) return BRNG_EINVAL;
  if (n.producer_warps != BRNG_PRODUCERS_NONE && (n.producer_warps < 1 || n.producer_warps > 8))
    return BRNG_EINVAL;
  h->tune = n;
  return BRNG_OK;
}

int brng_get_tuning(const brng_t* h, brng_tuning_t* t) {
  if (!h || !t) return BRNG_EINVAL;
  *t = h->tune;
  return BRNG_OK;
}

uint32_t brng_n_streams(const brng_t* h) { return h ? h->S : 0; }
uint64_t brng_seed(const brng_t* h) { return h ? h->seed : 0; }

int brng_get_positions(brng_t* h, uint64_t* host_pos) {
  if (!h || !host_pos) return BRNG_EINVAL;
  std::vector<uint64_t> soa(3ull * h->S);
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(soa.data(), h->d_pos, sizeof(uint64_t) * soa.size(), cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) return cuda_status(e);
  for (uint64_t s = 0; s < h->S; ++s)
    for (int d = 0; d < 3; ++d) host_pos[3 * s + d] = soa[d * static_cast<uint64_t>(h->S) + s];
  return BRNG_OK;
}

int brng_set_positions(brng_t* h, const uint64_t* host_pos) {
  if (!h || !host_pos) return BRNG_EINVAL;
  std::vector<uint64_t> soa(3ull * h->S);
  for (uint64_t s = 0; s < h->S; ++s)
    for (int d = 0; d < 3; ++d) soa[d * static_cast<uint64_t>(h->S) + s] = host_pos[3 * s + d];
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_pos, soa.data(), sizeof(uint64_t) * soa.size(), cudaMemcpyHostToDevice);
  return cuda_status(e);
}

int brng_get_positions_u64(brng_t* h, uint64_t* host_pos) {
  if (!h || !host_pos) return BRNG_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(host_pos, h->d_pos64, sizeof(uint64_t) * static_cast<size_t>(h->S), cudaMemcpyDeviceToHost);
  return cuda_status(e);
}

int brng_set_positions_u64(brng_t* h, const uint64_t* host_pos) {
  if (!h || !host_pos) return BRNG_EINVAL;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess)
    e = cudaMemcpy(h->d_pos64, host_pos, sizeof(uint64_t) * static_cast<size_t>(h->S), cudaMemcpyHostToDevice);
  return cuda_status(e);
}

int brng_read_counters(brng_t* h, brng_stream_t stream, brng_counters_t* out, int reset) {
  if (!h) return BRNG_EINVAL;
  static_assert(sizeof(brng_counters_t) == sizeof(brng::DevCounters), "counter layout");
  brng_counters_t c;
  cudaError_t e = cudaStreamSynchronize(reinterpret_cast<cudaStream_t>(stream));
  if (e == cudaSuccess) e = cudaMemcpy(&c, h->d_cnt, sizeof c, cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && reset) e = cudaMemset(h->d_cnt, 0, sizeof(brng::DevCounters));
  if (e == cudaSuccess && reset) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e);
  if (out) *out = c;
  if (c.n_timeout) return BRNG_ETIMEOUT;
  if (c.n_domain) return BRNG_EDOMAIN;
  if (c.n_reject) return BRNG_EREJECT;
  return BRNG_OK;
}

int brng_philox_words(brng_t* h, uint32_t domain, uint32_t stream_id, uint64_t first_block,
                      size_t n_blocks, uint32_t* out, brng_stream_t stream) {
  if (!h) return BRNG_EINVAL;
  if (n_blocks == 0) return BRNG_OK;
  if (!out || (reinterpret_cast<uintptr_t>(out) & 15u)) return BRNG_EINVAL;
  return cuda_status(brng::launch_philox_words(h->rk, domain, stream_id, first_block, n_blocks, out,
                                               reinterpret_cast<cudaStream_t>(stream)));
}

int brng_philox_peak(uint64_t iters, uint32_t blocks, uint32_t threads, uint32_t* sink,
                     brng_stream_t stream) {
  if (!sink || blocks == 0 || threads == 0 || threads > 256 || iters == 0) return BRNG_EINVAL;
  return cuda_status(brng::launch_philox_peak(brng::make_round_keys(0x243F6A8885A308D3ull), iters,
                                              blocks, threads, sink, reinterpret_cast<cudaStream_t>(stream)));
}

int brng_fp32_eval(uint32_t fn, size_t n, const float* in, float* out, brng_stream_t stream) {
  if (fn > 3) return BRNG_EINVAL;
  if (n == 0) return BRNG_OK;
  if (!in || !out) return BRNG_EINVAL;
  return cuda_status(brng::launch_fp32_eval(fn, n, in, out, reinterpret_cast<cudaStream_t>(stream)));
}

int brng_fp64_eval(uint32_t fn, size_t n, const double* in, double* out, brng_stream_t stream) {
  if (fn > 3) return BRNG_EINVAL;
  if (n == 0) return BRNG_OK;
  if (!in || !out) return BRNG_EINVAL;
  return cuda_status(brng::launch_fp64_eval(fn, n, in, out, reinterpret_cast<cudaStream_t>(stream)));
}

int brng_uniform(brng_t* h, size_t n, const float* a, const float* b, float* out, uint32_t* words,
                 brng_stream_t stream) {
  return bulk(h, BRNG_TAG_UNIFORM, n, nullptr, a, b, out, words, reinterpret_cast<cudaStream_t>(stream));
}
int brng_uniform_f64(brng_t* h, size_t n, const double* a, const double* b, double* out,
                     uint32_t* words, brng_stream_t stream) {
  const brng::TraceRange trace("brng_uniform_f64");
  if (!h) return BRNG_EINVAL;
  if (n == 0) return BRNG_OK;
  if (!a || !b || !out) return BRNG_EINVAL;
  brng::Uniform64Args u;
  u.rk = h->rk;
  u.n = n;
  u.S = h->S;
  u.a = a;
  u.b = b;
  u.out = out;
  u.words = words;
  u.pos64 = h->d_pos64;
  u.cnt = h->d_cnt;
  return cuda_status(brng::launch_uniform64(u, reinterpret_cast<cudaStream_t>(stream)));
}
int brng_normal(brng_t* h, size_t n, const float* mu, const float* sigma, float* out,
                uint32_t* words, brng_stream_t stream) {
  return bulk(h, BRNG_TAG_NORMAL, n, nullptr, mu, sigma, out, words, reinterpret_cast<cudaStream_t>(stream));
}
int brng_exponential(brng_t* h, size_t n, const float* lambda, float* out, uint32_t* words,
                     brng_stream_t stream) {
  return bulk(h, BRNG_TAG_EXPONENTIAL, n, nullptr, lambda, nullptr, out, words,
              reinterpret_cast<cudaStream_t>(stream));
}
int brng_gamma(brng_t* h, size_t n, const float* alpha, float* out, uint32_t* words,
               brng_stream_t stream) {
  return bulk(h, BRNG_TAG_GAMMA, n, nullptr, alpha, nullptr, out, words, reinterpret_cast<cudaStream_t>(stream));
}
int brng_laplace(brng_t* h, size_t n, const float* mu, const float* b, float* out, uint32_t* words,
                 brng_stream_t stream) {
  return bulk(h, BRNG_TAG_LAPLACE, n, nullptr, mu, b, out, words, reinterpret_cast<cudaStream_t>(stream));
}
int brng_weibull(brng_t* h, size_t n, const float* k, const float* lambda, float* out,
                 uint32_t* words, brng_stream_t stream) {
  return bulk(h, BRNG_TAG_WEIBULL, n, nullptr, k, lambda, out, words, reinterpret_cast<cudaStream_t>(stream));
}
int brng_poisson(brng_t* h, size_t n, const float* lambda, float* out, uint32_t* words,
                 brng_stream_t stream) {
  return bulk(h, BRNG_TAG_POISSON, n, nullptr, lambda, nullptr, out, words,
              reinterpret_cast<cudaStream_t>(stream));
}
int brng_binomial(brng_t* h, size_t n, const float* trials, const float* prob, float* out,
                  uint32_t* words, brng_stream_t stream) {
  return bulk(h, BRNG_TAG_BINOMIAL, n, nullptr, trials, prob, out, words,
              reinterpret_cast<cudaStream_t>(stream));
}
int brng_mixed(brng_t* h, size_t n, const uint8_t* tag, const float* p0, const float* p1,
               float* out, uint32_t* words, brng_stream_t stream) {
  if (n && !p1) return BRNG_EINVAL;
  return bulk(h, brng::kTagMixed, n, tag, p0, p1, out, words, reinterpret_cast<cudaStream_t>(stream));
}

int brng_dirichlet(brng_t* h, size_t n_rows, uint32_t K, const float* alpha, float* out,
                   brng_stream_t stream) {
  const brng::TraceRange trace("brng_dirichlet");
  if (!h || K == 0 || K > 128 || h->S % K != 0) return BRNG_EINVAL;
  if (n_rows == 0) return BRNG_OK;
  if (!alpha || !out) return BRNG_EINVAL;
  const uint32_t P = K <= 32 ? 1 : K <= 64 ? 2 : 4;
  const uint32_t B = brng::ring_len_min8(h->tune.buf_len);
  const size_t per_warp = 128u + h->tune.lookahead * 32u * P * 4u + 2u * P * B * 128u;
  const brng::Geometry g = geometry(h, per_warp);
  if (g.warps_per_block == 0) return BRNG_EINVAL;
  brng::DirichletArgs a{};
  a.rk = h->rk;
  a.K = K;
  a.B = B;
  a.lookahead = h->tune.lookahead;
  a.n_rows = n_rows;
  a.R = h->S / K;
  a.alpha = alpha;
  a.out = out;
  a.pos = h->d_pos;
  a.S = h->S;
  a.cnt = h->d_cnt;
  return cuda_status(brng::launch_dirichlet(a, g, false, reinterpret_cast<cudaStream_t>(stream)));
}

}  // extern "C"

namespace {

// Validates one Gibbs job and fills its kernel arguments (model args of a
// BatchJob; the other two model slots are left zero).  `seed_rk`: the job's
// round keys.
int make_job(const brng_t* h, brng_model_t model, const brng::RoundKeys& rk, uint64_t chain_offset,
             uint32_t n_chains, uint32_t n_sweeps, const void* params, void* state, double* moments,
             brng::BatchJob* j) {
  if (!state || !moments) return BRNG_EINVAL;
  *j = brng::BatchJob{};
  j->model = static_cast<uint32_t>(model);
  switch (model) {
    case BRNG_MODEL_TRIANGLE: {
      if (chain_offset + n_chains > 0x100000000ull) return BRNG_EINVAL;
      brng::TriangleArgs& a = j->tri;
      a.rk = rk;
      a.chain_offset = chain_offset;
      a.n_chains = n_chains;
      a.n_sweeps = n_sweeps;
      a.B = h->tune.buf_len;
      a.state = static_cast<brng_triangle_state_t*>(state);
      a.moments = moments;
      a.cnt = h->d_cnt;
      j->n_units = (static_cast<uint64_t>(n_chains) + 31) / 32;
      return BRNG_OK;
    }
    case BRNG_MODEL_NORMAL_GAMMA: {
      const brng_normal_gamma_params_t* p = static_cast<const brng_normal_gamma_params_t*>(params);
      if (!p || !p->nobs || !p->xbar || !p->sc) return BRNG_EINVAL;
      if (chain_offset + n_chains > 0x100000000ull) return BRNG_EINVAL;
      brng::NormalGammaArgs& a = j->ng;
      a.rk = rk;
      a.chain_offset = chain_offset;
      a.n_chains = n_chains;
      a.n_sweeps = n_sweeps;
      a.B = h->tune.buf_len;
      a.a0 = p->a0;
      a.b0 = p->b0;
      a.mu0 = p->mu0;
      a.prec0 = p->prec0;
      a.nobs = p->nobs;
      a.xbar = p->xbar;
      a.sc = p->sc;
      a.state = static_cast<brng_normal_gamma_state_t*>(state);
      a.moments = moments;
      a.cnt = h->d_cnt;
      j->n_units = (static_cast<uint64_t>(n_chains) + 31) / 32;
      return BRNG_OK;
    }
    case BRNG_MODEL_LDA: {
      const brng_lda_params_t* p = static_cast<const brng_lda_params_t*>(params);
      const brng_lda_state_t* s = static_cast<const brng_lda_state_t*>(state);
      if (!p || !p->alpha || p->K == 0 || p->K > 128 || !s->theta || !s->pos) return BRNG_EINVAL;
      if ((chain_offset + n_chains) * static_cast<uint64_t>(p->K) > 0x100000000ull) return BRNG_EINVAL;
      brng::DirichletArgs& a = j->lda;
      a.rk = rk;
      a.K = p->K;
      a.B = brng::ring_len_min8(h->tune.buf_len);
      a.lookahead = h->tune.lookahead;
      a.alpha = p->alpha;
      a.out = s->theta;
      a.pos = s->pos;
      a.stream_base = chain_offset;
      a.n_docs = n_chains;
      a.n_sweeps = n_sweeps;
      a.moments = moments;
      a.cnt = h->d_cnt;
      j->n_units = n_chains;
      return BRNG_OK;
    }
    default:
      return BRNG_EINVAL;
  }
}

uint32_t lda_p(uint32_t K) { return K <= 32 ? 1 : K <= 64 ? 2 : 4; }

// relative cost of one unit-sweep by model (orders the batch: longest first)
double unit_cost(const brng::BatchJob& j) {
  switch (j.model) {
    case BRNG_MODEL_TRIANGLE: return 1.0 * j.tri.n_sweeps;
    case BRNG_MODEL_NORMAL_GAMMA: return 3.0 * j.ng.n_sweeps;
    default: return 0.25 * j.lda.K * j.lda.n_sweeps;
  }
}

}  // namespace

struct brng_batch {
  brng::BatchJob* d_jobs;
  unsigned long long* d_counter;
  brng::BatchArgs args;
  uint32_t P;
  uint32_t warps_per_block;
  uint32_t blocks;  // grid, fixed when planned
};

namespace {

// Builds the ordered job table of a batch on the host.
int plan_batch(const brng_t* h, const brng_job_t* jobs, uint32_t n_jobs,
               std::vector<brng::BatchJob>* table, uint32_t* P, uint32_t* wpb, uint32_t* warp_bytes) {
  if (!h || (n_jobs && !jobs)) return BRNG_EINVAL;
  table->clear();
  table->reserve(n_jobs);
  bool tri = false, ng = false, lda = false;
  uint32_t maxP = 1;
  for (uint32_t i = 0; i < n_jobs; ++i) {
    const brng_job_t& jb = jobs[i];
    if (jb.n_chains == 0) continue;
    brng::BatchJob j;
    const int st = make_job(h, jb.model, brng::make_round_keys(jb.seed), jb.chain_offset, jb.n_chains,
                            jb.n_sweeps, jb.params, jb.state, jb.moments, &j);
    if (st != BRNG_OK) return st;
    tri |= jb.model == BRNG_MODEL_TRIANGLE;
    ng |= jb.model == BRNG_MODEL_NORMAL_GAMMA;
    if (jb.model == BRNG_MODEL_LDA) {
      lda = true;
      maxP = std::max(maxP, lda_p(j.lda.K));
    }
    table->push_back(j);
  }
  std::stable_sort(table->begin(), table->end(), [](const brng::BatchJob& a, const brng::BatchJob& b) {
    return unit_cost(a) > unit_cost(b);
  });
  uint64_t first = 0;
  for (auto& j : *table) {
    j.first_unit = first;
    first += j.n_units;
  }
  const size_t per_warp = brng::batch_warp_bytes(tri, ng, lda, h->tune.buf_len, maxP, h->tune.lookahead);
  const brng::Geometry g = geometry(h, per_warp);
  if (g.warps_per_block == 0) return BRNG_EINVAL;
  *P = maxP;
  *wpb = g.warps_per_block;
  *warp_bytes = static_cast<uint32_t>(per_warp);
  return BRNG_OK;
}

// The full LDA step, n_sweeps times: topic draws (one warp per document),
// the count changes added into the corpus counts (unless the caller exchanges
// them across devices first), then theta ~ Dirichlet(alpha + n_d) through the
// LDA model's own launch, on the same stream.
int lda_full_run(brng_t* h, uint64_t doc_offset, uint32_t n_docs, uint32_t n_sweeps,
                 const brng_lda_full_params_t* p, const brng_lda_full_state_t* s, double* moments,
                 brng_stream_t stream);

uint64_t total_units(const std::vector<brng::BatchJob>& t) {
  return t.empty() ? 0 : t.back().first_unit + t.back().n_units;
}

int lda_full_run(brng_t* h, uint64_t doc_offset, uint32_t n_docs, uint32_t n_sweeps,
                 const brng_lda_full_params_t* p, const brng_lda_full_state_t* s, double* moments,
                 brng_stream_t stream) {
  if (!p || !s || !moments) return BRNG_EINVAL;
  if (p->K == 0 || p->K > 128 || p->V == 0 || !p->doc_ptr || !p->words || !p->prev) return BRNG_EINVAL;
  if (!(p->alpha >= 1e-6f && p->alpha <= 1e6f && p->beta >= 1e-6f && p->beta <= 1e6f)) return BRNG_EINVAL;
  if (!s->z || !s->z_start || !s->ndk || !s->nkw || !s->nk || !s->dnkw || !s->dir_alpha || !s->zpos ||
      !s->theta || !s->pos)
    return BRNG_EINVAL;
  if (p->exchange > 1 || (p->exchange == 1 && n_sweeps != 1)) return BRNG_EINVAL;
  if ((doc_offset + n_docs) * static_cast<uint64_t>(p->K) > 0x100000000ull) return BRNG_EINVAL;
  if (n_docs == 0 || n_sweeps == 0) return BRNG_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  brng::LdaZArgs a;
  a.rk = h->rk;
  a.doc_offset = doc_offset;
  a.n_docs = n_docs;
  a.K = p->K;
  a.V = p->V;
  a.alpha = p->alpha;
  a.beta = p->beta;
  a.vbeta = static_cast<float>(p->V) * p->beta;  // one FP32 rounding, as the oracle
  uint32_t lg = 0;
  while ((1u << lg) < p->K) ++lg;
  a.qbits = 32u - lg;
  a.doc_ptr = p->doc_ptr;
  a.order = p->order;
  a.words = p->words;
  a.prev = p->prev;
  a.z = s->z;
  a.z_start = s->z_start;
  a.ndk = s->ndk;
  a.nkw = s->nkw;
  a.nk = s->nk;
  a.dnkw = s->dnkw;
  a.dir_alpha = s->dir_alpha;
  a.zpos = s->zpos;
  brng_lda_params_t lp;
  lp.K = p->K;
  lp.alpha = s->dir_alpha;
  brng_lda_state_t ls;
  ls.theta = s->theta;
  ls.pos = s->pos;
  for (uint32_t sweep = 0; sweep < n_sweeps; ++sweep) {
    int rc = cuda_status(brng::launch_lda_z(a, st));
    if (rc != BRNG_OK) return rc;
    if (p->exchange == 0) {
      rc = cuda_status(brng::launch_lda_apply(p->K, p->V, s->nkw, s->nk, s->dnkw, st));
      if (rc != BRNG_OK) return rc;
    }
    rc = brng_gibbs_run(h, BRNG_MODEL_LDA, doc_offset, n_docs, 1, &lp, &ls, moments, stream);
    if (rc != BRNG_OK) return rc;
  }
  return BRNG_OK;
}

}  // namespace

extern "C" {

int brng_lda_index(uint32_t n_docs, const uint32_t* doc_ptr, const uint32_t* words, uint32_t* prev,
                   brng_stream_t stream) {
  if (n_docs == 0) return BRNG_OK;
  if (!doc_ptr || !words || !prev) return BRNG_EINVAL;
  return cuda_status(brng::launch_lda_index(n_docs, doc_ptr, words, prev, reinterpret_cast<cudaStream_t>(stream)));
}

int brng_lda_apply(uint32_t K, uint32_t V, int32_t* nkw, int32_t* nk, int32_t* dnkw, brng_stream_t stream) {
  if (K == 0 || K > 128 || V == 0 || !nkw || !nk || !dnkw) return BRNG_EINVAL;
  return cuda_status(brng::launch_lda_apply(K, V, nkw, nk, dnkw, reinterpret_cast<cudaStream_t>(stream)));
}

int brng_gibbs_run(brng_t* h, brng_model_t model, uint64_t chain_offset, uint32_t n_chains,
                   uint32_t n_sweeps, const void* params, void* state, double* moments,
                   brng_stream_t stream) {
  const brng::TraceRange trace("brng_gibbs_run");
  if (!h) return BRNG_EINVAL;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  if (model == BRNG_MODEL_LDA_FULL)
    return lda_full_run(h, chain_offset, n_chains, n_sweeps, static_cast<const brng_lda_full_params_t*>(params),
                        static_cast<const brng_lda_full_state_t*>(state), moments, stream);
  if (n_chains == 0) return BRNG_OK;
  brng::BatchJob j;
  const int rc = make_job(h, model, h->rk, chain_offset, n_chains, n_sweeps, params, state, moments, &j);
  if (rc != BRNG_OK) return rc;
  switch (model) {
    case BRNG_MODEL_TRIANGLE: {
      const uint32_t nc = 32 / h->tune.lanes_per_chain;
      const brng::Geometry g = geometry(h, 128u + static_cast<size_t>(h->tune.buf_len) * nc * 8u);
      if (g.warps_per_block == 0) return BRNG_EINVAL;
      return cuda_status(brng::launch_triangle(j.tri, g, h->tune.lanes_per_chain, st));
    }
    case BRNG_MODEL_NORMAL_GAMMA: {
      const uint32_t Wp = h->tune.producer_warps;
      if (Wp != BRNG_PRODUCERS_NONE) {  // consumer warps + producer warps per block
        const brng::Geometry g = geometry(h, brng::normal_gamma_pc_bytes_per_warp(h->tune.buf_len));
        const uint32_t Wc = std::min({g.warps_per_block, 16u - Wp, 8u * Wp});
        if (Wc == 0) return BRNG_EINVAL;
        return cuda_status(brng::launch_normal_gamma_pc(j.ng, Wc, Wp, st));
      }
      const brng::Geometry g = geometry(h, brng::normal_gamma_bytes_per_warp(h->tune.buf_len));
      if (g.warps_per_block == 0) return BRNG_EINVAL;
      return cuda_status(brng::launch_normal_gamma(j.ng, g, st));
    }
    default: {
      const uint32_t P = lda_p(j.lda.K);
      const size_t per_warp = 128u + h->tune.lookahead * 32u * P * 4u + 2u * P * j.lda.B * 128u;
      const brng::Geometry g = geometry(h, per_warp);
      if (g.warps_per_block == 0) return BRNG_EINVAL;
      return cuda_status(brng::launch_dirichlet(j.lda, g, true, st));
    }
  }
}

int brng_debug_violations(uint64_t* count, int reset) {
#ifdef BRNG_DEBUG
  if (!count) return BRNG_EINVAL;
  const cudaError_t e = cudaDeviceSynchronize();
  if (e != cudaSuccess) return cuda_status(e);
  uint64_t total = 0;
  for (auto read : brng::debug_readers()) total += read(reset != 0);
  *count = total;
  return BRNG_OK;
#else
  (void)count;
  (void)reset;
  return BRNG_EINVAL;
#endif
}

int brng_test_pc_stall(brng_t* h, uint32_t n_chains, uint32_t n_sweeps, const void* params, void* state,
                       double* moments, brng_stream_t stream) {
  const brng::TraceRange trace("brng_test_pc_stall");
  if (!h) return BRNG_EINVAL;
  if (n_chains == 0) return BRNG_OK;
  brng::BatchJob j;
  const int rc = make_job(h, BRNG_MODEL_NORMAL_GAMMA, h->rk, 0, n_chains, n_sweeps, params, state, moments, &j);
  if (rc != BRNG_OK) return rc;
  const uint32_t Wp = h->tune.producer_warps == BRNG_PRODUCERS_NONE ? 1u : h->tune.producer_warps;
  const brng::Geometry g = geometry(h, brng::normal_gamma_pc_bytes_per_warp(h->tune.buf_len));
  const uint32_t Wc = std::min({g.warps_per_block, 16u - Wp, 8u * Wp});
  if (Wc == 0) return BRNG_EINVAL;
  return cuda_status(brng::launch_normal_gamma_pc(j.ng, Wc, Wp, reinterpret_cast<cudaStream_t>(stream), true));
}

int brng_batch_create(brng_t* h, const brng_job_t* jobs, uint32_t n_jobs, brng_batch_t** out) {
  const brng::TraceRange trace("brng_batch_create");
  if (!out) return BRNG_EINVAL;
  std::vector<brng::BatchJob> table;
  uint32_t P = 1, wpb = 1, wbytes = 128;
  const int rc = plan_batch(h, jobs, n_jobs, &table, &P, &wpb, &wbytes);
  if (rc != BRNG_OK) return rc;
  brng_batch_t* b = new (std::nothrow) brng_batch_t();
  if (!b) return BRNG_ENOMEM;
  cudaError_t e = cudaMalloc(&b->d_counter, sizeof(unsigned long long));
  if (e == cudaSuccess && !table.empty())
    e = cudaMalloc(&b->d_jobs, sizeof(brng::BatchJob) * table.size());
  if (e == cudaSuccess && !table.empty())
    e = cudaMemcpy(b->d_jobs, table.data(), sizeof(brng::BatchJob) * table.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(b->d_counter);
    cudaFree(b->d_jobs);
    delete b;
    return cuda_status(e);
  }
  b->args.jobs = b->d_jobs;
  b->args.n_jobs = static_cast<uint32_t>(table.size());
  b->args.warp_bytes = wbytes;
  b->args.total_units = total_units(table);
  b->args.counter = b->d_counter;
  b->P = P;
  b->warps_per_block = wpb;
  e = brng::batch_grid(b->args, P, wpb, &b->blocks);
  if (e != cudaSuccess) {
    brng_batch_destroy(b);
    return cuda_status(e);
  }
  *out = b;
  return BRNG_OK;
}

int brng_batch_launch(brng_batch_t* b, brng_stream_t stream) {
  const brng::TraceRange trace("brng_batch_launch");
  if (!b) return BRNG_EINVAL;
  if (b->args.total_units == 0) return BRNG_OK;
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(b->d_counter, 0, sizeof(unsigned long long), st);
  if (e == cudaSuccess) e = brng::launch_batch(b->args, b->P, b->warps_per_block, b->blocks, st);
  return cuda_status(e);
}

int brng_batch_destroy(brng_batch_t* b) {
  if (!b) return BRNG_OK;
  cudaError_t e1 = cudaFree(b->d_jobs);
  cudaError_t e2 = cudaFree(b->d_counter);
  delete b;
  return e1 != cudaSuccess ? cuda_status(e1) : cuda_status(e2);
}

int brng_gibbs_batch(brng_t* h, const brng_job_t* jobs, uint32_t n_jobs, brng_stream_t stream) {
  const brng::TraceRange trace("brng_gibbs_batch");
  if (!h) return BRNG_EINVAL;
  return brng::batch_launch_into(h, jobs, n_jobs, &h->d_batch_jobs, &h->batch_cap,
                                 &h->d_batch_counter, reinterpret_cast<cudaStream_t>(stream));
}

}  // extern "C"

namespace brng {

int batch_launch_into(brng_t* h, const brng_job_t* jobs, uint32_t n_jobs, BatchJob** d_table,
                      size_t* cap, unsigned long long** d_counter, cudaStream_t st) {
  std::vector<BatchJob> table;
  uint32_t P = 1, wpb = 1, wbytes = 128;
  const int rc = plan_batch(h, jobs, n_jobs, &table, &P, &wpb, &wbytes);
  if (rc != BRNG_OK) return rc;
  if (table.empty()) return BRNG_OK;
  cudaError_t e = cudaSuccess;
  if (table.size() > *cap) {  // grow the table (cudaFree waits for the device)
    cudaFree(*d_table);
    *d_table = nullptr;
    *cap = 0;
    e = cudaMalloc(d_table, sizeof(BatchJob) * table.size());
    if (e != cudaSuccess) return cuda_status(e);
    *cap = table.size();
  }
  if (!*d_counter) {
    e = cudaMalloc(d_counter, sizeof(unsigned long long));
    if (e != cudaSuccess) return cuda_status(e);
  }
  // from pageable memory: the call returns once the table is staged, so the
  // vector may go; the copy is ordered on `st` before the kernel
  e = cudaMemcpyAsync(*d_table, table.data(), sizeof(BatchJob) * table.size(), cudaMemcpyHostToDevice,
                      st);
  if (e == cudaSuccess) e = cudaMemsetAsync(*d_counter, 0, sizeof(unsigned long long), st);
  if (e != cudaSuccess) return cuda_status(e);
  BatchArgs a;
  a.jobs = *d_table;
  a.n_jobs = static_cast<uint32_t>(table.size());
  a.warp_bytes = wbytes;
  a.total_units = total_units(table);
  a.counter = *d_counter;
  uint32_t blocks = 0;
  e = batch_grid(a, P, wpb, &blocks);
  if (e != cudaSuccess) return cuda_status(e);
  return cuda_status(launch_batch(a, P, wpb, blocks, st));
}

}  // namespace brng
