/*
 * oracle.h -- the CPU oracle of the batched varying-parameter RNG method.
 *
 * TEST INFRASTRUCTURE ONLY.  This is a plain, slow, FP64 restatement of the
 * method (Mahani & Sharabiani, "Efficient SIMD RNG for Varying-Parameter
 * Streams: C++ Class BatchRNG", arXiv 1412.4825), written to check the CUDA
 * path.  Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline and
 * reference legs may load it.  It shares no code, header, table or constant
 * with the CUDA library; the two agree only through the definitions below.
 *
 * Conventions (the paper leaves the engine open, Sec. 2.2; these are the
 * readings this project fixes):
 *   - core engine: Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11),
 *     key = (seed & 0xffffffff, seed >> 32),
 *     counter = (block & 0xffffffff, domain, stream, block >> 32);
 *   - a stream is one BatchRNG object (Sec. 2.2); each reducible
 *     distribution ("domain") has its own element sequence, element j of a
 *     4-word domain living in block j/4, word j%4 (U64: block j/2, words
 *     2(j%2), 2(j%2)+1);
 *   - buffers (Sec. 2.2 "buffer_length", "buffer", "buffer_counter") hold a
 *     window of that sequence and are refilled when the counter reaches the
 *     end, so every value is independent of the buffer length.
 */
#ifndef BRNG_ORACLE_H
#define BRNG_ORACLE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* domain tags (counter word 1) */
#define OR_DOM_U 0u    /* 24-bit uniforms, one word per element           */
#define OR_DOM_N 1u    /* Box-Muller Gaussians, a word pair per two elems  */
#define OR_DOM_E 2u    /* exponentials -ln U', one word per element        */
#define OR_DOM_DATA 3u /* reserved for synthetic data / set-up draws       */
#define OR_DOM_U64 4u  /* 53-bit uniforms, two words per element           */
#define OR_NDOM 5      /* domains a buffered stream object holds            */
#define OR_DOM_Z 5u    /* LDA topic draws: one word per element (top 24 bits) */

/* status bits returned by the bulk and Gibbs functions */
#define OR_OK 0
#define OR_EDOMAIN 4
#define OR_EREJECT 5
#define OR_EINVAL 1

/* Marsaglia-Tsang attempts before a Gamma draw gives up (NaN + EREJECT) */
#define OR_GAMMA_MAX_ATTEMPTS 64
/* Poisson: 0 < lambda <= this; inversion (sequential search, O(lambda) steps)
 * up to OR_INVERSION_MAX_MEAN, transformed rejection (PTRS) above */
#define OR_POISSON_MAX_LAMBDA 1e7f
/* Poisson and Binomial means (n min(p, 1-p)) up to this: inversion of one U */
#define OR_INVERSION_MAX_MEAN 64.0
/* the search stops here at the latest (far beyond any 24-bit uniform's reach) */
#define OR_POISSON_MAX_K 1024

/* ---- core engine ------------------------------------------------------ */
void or_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]);
void or_philox_words(uint64_t seed, uint32_t domain, uint32_t stream,
                     uint64_t first_block, uint64_t n_blocks, uint32_t *out);

/* ---- FP64 elementary functions written for the oracle ----------------- */
double or_log(double x);
double or_exp(double x);
void or_exp_many(uint64_t n, const double *x, double *out);
void or_sincospi(double a, double *s, double *c);
void or_log_many(uint64_t n, const double *x, double *out);
void or_sincospi_many(uint64_t n, const double *a, double *s, double *c);

/* ---- element accessors: element j of a domain, straight from the engine */
uint32_t or_elem_word(uint64_t seed, uint32_t domain, uint32_t stream, uint64_t j);
double or_elem_value(uint64_t seed, uint32_t domain, uint32_t stream, uint64_t j);
void or_elem_values(uint64_t seed, uint32_t domain, uint32_t stream, uint64_t j0,
                    uint64_t n, double *out, uint32_t *words);

/* ---- bulk varying-parameter streams (Sec. 2.3: per-draw parameters read
 *      from memory, every output written).  Draw i goes to stream i mod S.
 *      pos[3*s + {0,1,2}] = next U, N, E element of stream s (in/out).   */
int or_uniform(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *a,
               const float *b, double *out, uint32_t *words, uint32_t buf_len);
/* U[a, b) in FP64 from the U64 domain; pos64: one U64 position per stream */
int or_uniform_f64(uint64_t seed, uint32_t S, uint64_t *pos64, uint64_t n, const double *a,
                   const double *b, double *out, uint32_t *words, uint32_t buf_len);
int or_normal(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *mu,
              const float *sigma, double *out, uint32_t *words, uint32_t buf_len);
int or_exponential(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *lambda,
                   double *out, uint32_t *words, uint32_t buf_len);
/* cond (nullable): per draw 3|c z|/t of the accepted attempt plus |ln(u_b)/alpha|
 * when boosted -- the relative conditioning of the result, for FP32 checks */
int or_gamma(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *alpha,
             double *out, uint32_t *words, double *cond, uint32_t buf_len);
int or_laplace(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *mu,
               const float *scale, double *out, uint32_t *words, uint32_t buf_len);
int or_weibull(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *shape,
               const float *scale, double *out, uint32_t *words, double *cond, uint32_t buf_len);
/* rows of K components; S % K == 0; component k of row i draws from stream
 * (i mod (S/K))*K + k; logs (nullable) gets each component's log-Gamma */
int or_dirichlet(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n_rows, uint32_t K,
                 const float *alpha, double *out, double *logs, double *cond, uint32_t buf_len);
/* Poisson(lambda = p0) by inversion of one U: the smallest k with U < F(k),
 * F(k) = sum_{j<=k} p_j, p_0 = e^-lambda (or_exp), p_j = (p_{j-1} lambda) / j,
 * F accumulated left to right, all in FP64 (the draw's value is k) */
double or_poisson_inv(double lambda, double u);
int or_poisson(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *lambda,
               double *out, uint32_t *words, uint32_t buf_len);
/* Binomial(n = p0, p = p1) by inversion of one U on q = min(p, 1-p): the
 * smallest k with U < F(k), F the Binomial(n, q) CDF summed left to right from
 * p_0 = exp(n log(1 - q)) (or_exp, or_log), p_k = (p_{k-1} ((n - k + 1) r)) / k,
 * r = q / (1 - q), all FP64; the draw is k, or n - k when p > 1/2 */
double or_binomial_inv(double n, double p, double u);
/* ln k! of an integer k >= 0 (exact product's log to 15!, Stirling above) */
double or_lfact(double k);
int or_binomial(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const float *trials,
                const float *prob, double *out, uint32_t *words, uint32_t buf_len);
/* tag 0 U(p0,p1), 1 N(p0,p1), 2 Exp(rate p0), 3 Gamma(p0), 4 Laplace(p0,p1),
 * 5 Weibull(shape p0, scale p1), 6 Poisson(p0), 7 Binomial(n = p0, p = p1) */
int or_mixed(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const uint8_t *tag,
             const float *p0, const float *p1, double *out, uint32_t *words, double *cond,
             uint32_t buf_len);
/* the same, for the streams in [s_begin, s_end) only (sampled parity) */
int or_mixed_streams(uint64_t seed, uint32_t S, uint32_t s_begin, uint32_t s_end, uint64_t *pos,
                     uint64_t n, const uint8_t *tag, const float *p0, const float *p1,
                     double *out, uint32_t *words, double *cond, uint32_t buf_len);

/* ---- Gibbs models (Markov-dependent consumers) ------------------------ */
/* Eq. 1 / Fig. 1: xy[2c] = x, xy[2c+1] = y; pos[c] = next U64 element;
 * mom[5c..5c+4] += (x, y, x^2, y^2, xy) per sweep. */
int or_gibbs_triangle(uint64_t seed, uint64_t chain_offset, uint32_t n_chains, uint32_t n_sweeps,
                      double *xy, uint64_t *pos, double *mom, uint32_t buf_len);
/* Normal model with unknown mean and precision, semi-conjugate priors
 * mu ~ N(mu0, 1/prec0), tau ~ Gamma(a0, rate b0).  prior = {a0, b0, mu0, prec0}.
 * state[2c] = mu, state[2c+1] = tau; pos[2c] = N, pos[2c+1] = U;
 * mom[4c..4c+3] += (mu, tau, mu^2, tau^2).
 * trace (nullable): per chain c and sweep t, trace[5 (c n_sweeps + t) + i] =
 * (G, its conditioning as or_gamma's cond, the Gaussian z of mu's draw, tau,
 * mu) -- the trajectory that FP32 error bounds are propagated along. */
int or_gibbs_normal_gamma(uint64_t seed, uint64_t chain_offset, uint32_t n_chains,
                          uint32_t n_sweeps, const float *prior, const float *nobs,
                          const float *xbar, const float *sc, double *state, uint64_t *pos,
                          double *mom, double *trace, uint32_t buf_len);
/* LDA-style document-topic draws theta_d ~ Dir(alpha_d) every sweep; component
 * (d, k) is stream (doc_offset + d)*K + k; pos[2(dK+k)] = N, [..+1] = U;
 * theta = last draw, logs (nullable) = its log-Gammas; mom[dK+k] += theta_dk
 * per sweep.  trace (nullable): per document d, sweep t and component k,
 * trace[2 ((d n_sweeps + t) K + k) + i] = (log-Gamma, its conditioning). */
int or_gibbs_lda(uint64_t seed, uint64_t doc_offset, uint32_t n_docs, uint32_t K,
                 uint32_t n_sweeps, const float *alpha, double *theta, double *logs,
                 double *cond, uint64_t *pos, double *mom, double *trace, uint32_t buf_len);

/* ---- full LDA step (or_lda.c): topic assignments resampled per token ---- */
/* The FP32 weights w_k of one token's collapsed conditional and their
 * integer form q_k (see or_lda.c): ndk, nkw_w, nk are the counts including
 * the token itself, whose current topic is z_old. */
void or_lda_weights(uint32_t K, float alpha, float beta, float vbeta, const int32_t *ndk,
                    const int32_t *nkw_w, const int32_t *nk, uint32_t z_old, float *w_out,
                    uint32_t *q_out);
/* the topic for a 24-bit uniform integer r24: smallest k with C_k > (r24 Q) >> 24 */
uint32_t or_lda_pick(uint32_t K, const uint32_t *q, uint32_t r24);
/* One sweep of topic draws over documents [0, n_docs) (global ids doc_offset +
 * d): tokens doc_ptr[d] .. doc_ptr[d+1]-1 with words[t] < V and topics z[t]
 * (in/out), document-topic counts ndk [n_docs][K] (in/out), word-topic and
 * topic counts nkw [V][K], nk [K] of the start of the sweep (read only); the
 * sweep's changes are added to dnkw [V][K] and dnk [K]; zpos[d] = the
 * document's next Z-domain element (in/out).  K <= 255. */
int or_lda_z_sweep(uint64_t seed, uint64_t doc_offset, uint32_t n_docs, uint32_t K, uint32_t V,
                   float alpha, float beta, const uint32_t *doc_ptr, const uint32_t *words,
                   uint8_t *z, int32_t *ndk, const int32_t *nkw, const int32_t *nk,
                   int32_t *dnkw, int32_t *dnk, uint64_t *zpos);
int or_lda_z_sweep_mt(uint64_t seed, uint64_t doc_offset, uint32_t n_docs, uint32_t K, uint32_t V,
                      float alpha, float beta, const uint32_t *doc_ptr, const uint32_t *words,
                      uint8_t *z, int32_t *ndk, const int32_t *nkw, const int32_t *nk,
                      int32_t *dnkw, int32_t *dnk, uint64_t *zpos, int nthreads);
/* n_sweeps topic sweeps (document ids from 0), each followed by adding its
 * changes into nkw and nk; zhist (nullable) [n_tokens][K] += 1 at the topic of
 * each token after each sweep. */
int or_lda_z_run(uint64_t seed, uint32_t n_sweeps, uint32_t n_docs, uint32_t K, uint32_t V,
                 float alpha, float beta, const uint32_t *doc_ptr, const uint32_t *words,
                 uint8_t *z, int32_t *ndk, int32_t *nkw, int32_t *nk, uint64_t *zpos,
                 uint32_t *zhist);

/* the same on `nthreads` host threads over contiguous chain ranges */
int or_gibbs_triangle_mt(uint64_t seed, uint64_t chain_offset, uint32_t n_chains,
                         uint32_t n_sweeps, double *xy, uint64_t *pos, double *mom,
                         uint32_t buf_len, int nthreads);
int or_gibbs_normal_gamma_mt(uint64_t seed, uint64_t chain_offset, uint32_t n_chains,
                             uint32_t n_sweeps, const float *prior, const float *nobs,
                             const float *xbar, const float *sc, double *state, uint64_t *pos,
                             double *mom, double *trace, uint32_t buf_len, int nthreads);
int or_gibbs_lda_mt(uint64_t seed, uint64_t doc_offset, uint32_t n_docs, uint32_t K,
                    uint32_t n_sweeps, const float *alpha, double *theta, double *logs,
                    double *cond, uint64_t *pos, double *mom, double *trace, uint32_t buf_len,
                    int nthreads);
int or_mixed_mt(uint64_t seed, uint32_t S, uint64_t *pos, uint64_t n, const uint8_t *tag,
                const float *p0, const float *p1, double *out, uint32_t *words, double *cond,
                uint32_t buf_len, int nthreads);

/* Marsaglia-Tsang acceptance test of one attempt, exactly as the Gamma
 * sampler takes it (for tests): returns 1 accept, 0 reject, -1 if t <= 0. */
int or_mt_accept(double alpha, double z, double u_open);

#ifdef __cplusplus
}
#endif
#endif
