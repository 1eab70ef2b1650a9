/*
 * brng.h -- C ABI of libbrng.so, the GB300 (sm_103a) implementation of the
 * batched varying-parameter RNG method of Mahani & Sharabiani, "Efficient
 * SIMD RNG for Varying-Parameter Streams: C++ Class BatchRNG" (arXiv
 * 1412.4825).
 *
 * The paper's object (Sec. 2.2) keeps, per reducible distribution (uniform,
 * Gaussian, exponential), a buffer of base deviates that the vectorised core
 * engine fills in bulk; Get* calls consume it one draw at a time with
 * per-draw parameters and refill it when the counter reaches the end.  Here
 * every stream is a GPU lane, the core engine is Philox4x32-10 (Salmon et al.,
 * SC'11), buffers are shared-memory rings that a whole warp refills at once,
 * and all state stays on the device.
 *
 * Stream conventions (fixed; every value depends only on these):
 *   key     = (seed & 0xffffffff, seed >> 32)
 *   counter = (block & 0xffffffff, domain, stream, block >> 32)
 *   element j of domain U, N or E lives in block j/4, word j%4;
 *   element j of domain U64 lives in block j/2, words 2(j%2), 2(j%2)+1.
 *   U = (w>>8) 2^-24 in [0,1);  U' = ((w>>8)+1) 2^-24 in (0,1];
 *   N: (w0, w1) -> sqrt(-2 ln U'(w0)) * (cos, sin)(2 pi U(w1)), cos first;
 *   E = -ln U'(w);  U64 = ((w0>>5) 2^26 + (w1>>6)) 2^-53.
 * Values never depend on buffer length, block size, lanes per chain, call
 * splitting or how chains are sharded over calls or devices.
 *
 * Memory: every array argument marked "device" is caller-owned device memory
 * (e.g. a torch CUDA tensor), read or written asynchronously on `stream`; the
 * call returns once the work is enqueued.  "host" arrays are read or written
 * before the call returns.  Parameter arrays are float32 and contiguous
 * (float64 for brng_uniform_f64).
 *
 * Errors: every call returns a brng_status_t.  Argument errors are detected
 * on the host before any launch (BRNG_EINVAL); CUDA launch/alloc failures give
 * BRNG_ECUDA / BRNG_ENOMEM.  Invalid per-draw parameters are *not* an error
 * of the call: the draw's output is NaN, it consumes nothing, and the
 * handle's device counters record it; brng_read_counters() synchronises the
 * stream and reports BRNG_ETIMEOUT / BRNG_EDOMAIN / BRNG_EREJECT from those
 * counters.  Calls on one handle must be ordered on one stream (they share its
 * stream positions and counters).
 */
#ifndef BRNG_H
#define BRNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct brng_handle brng_t;
typedef struct CUstream_st *brng_stream_t; /* a cudaStream_t; NULL = legacy default stream */

typedef enum {
  BRNG_OK = 0,
  BRNG_EINVAL = 1,   /* bad argument (NULL pointer, size, unsupported option)     */
  BRNG_ENOMEM = 2,   /* device allocation failed / memory budget exceeded         */
  BRNG_ECUDA = 3,    /* a CUDA runtime call failed                                */
  BRNG_EDOMAIN = 4,  /* some per-draw parameter was invalid (outputs NaN)         */
  BRNG_EREJECT = 5,  /* some Gamma draw hit the 64-attempt cap (output NaN)       */
  BRNG_ETIMEOUT = 6, /* a bounded device wait expired                             */
  BRNG_EAGAIN = 7,   /* not done yet / not admitted yet                           */
  BRNG_ENOTFOUND = 8 /* unknown job id                                            */
} brng_status_t;

/* domain tags (counter word 1); Z: the full LDA step's topic draws, one word
 * (its top 24 bits) per draw, stream = global document id */
enum { BRNG_DOMAIN_U = 0, BRNG_DOMAIN_N = 1, BRNG_DOMAIN_E = 2, BRNG_DOMAIN_DATA = 3,
       BRNG_DOMAIN_U64 = 4, BRNG_DOMAIN_Z = 5 };

/* distribution tags of the mixed stream */
enum { BRNG_TAG_UNIFORM = 0, BRNG_TAG_NORMAL = 1, BRNG_TAG_EXPONENTIAL = 2, BRNG_TAG_GAMMA = 3,
       BRNG_TAG_LAPLACE = 4, BRNG_TAG_WEIBULL = 5, BRNG_TAG_POISSON = 6, BRNG_TAG_BINOMIAL = 7 };
#define BRNG_POISSON_MAX_LAMBDA 1e7f      /* Poisson: 0 < lambda <= this                     */
#define BRNG_INVERSION_MAX_MEAN 64.0f     /* discrete means up to this: inversion; above: rejection */

/* Gibbs models */
typedef enum {
  BRNG_MODEL_TRIANGLE = 0,     /* Sec. 1, Eq. 1 and Fig. 1                              */
  BRNG_MODEL_NORMAL_GAMMA = 1, /* mean/precision of a normal sample, Gamma + Normal steps */
  BRNG_MODEL_LDA = 2,          /* LDA document-topic Dirichlet step (Sec. 1, footnote)   */
  BRNG_MODEL_LDA_FULL = 3      /* full LDA step: topic draws per token, then the Dirichlet */
} brng_model_t;

/* Device-side counters of a handle (brng_read_counters). */
typedef struct {
  uint64_t n_domain;   /* draws with an invalid parameter (NaN output)               */
  uint64_t n_reject;   /* Gamma draws that hit the attempt cap (NaN output)           */
  uint64_t n_recheck;  /* Gamma tests, discrete draws and rejection attempts re-decided
                          in FP64 (the FP32 result within its error bound of a boundary) */
  uint64_t n_flip;     /* ... of which the FP64 decision differed from the FP32 sign  */
  float max_flip_ratio;/* max |FP32 margin| / tolerance over the flips (must stay < 1) */
  uint32_t n_timeout;  /* bounded device waits that ran out (chains ended with NaN)  */
  uint64_t n_wasted;   /* base deviates generated into buffers but unused when a call
                          ended (Sec. 2.4's buffer waste; regenerated by the next call) */
} brng_counters_t;

/* Tuning knobs; zero fields mean "library default". */
typedef struct {
  uint32_t buf_len;         /* ring length per lane and domain, elements, power of 2 in [4, 512] */
  uint32_t warps_per_block; /* 1..16                                                         */
  uint32_t lanes_per_chain; /* triangle model only: 1, 2, 4, 8, 16 or 32                       */
  uint32_t lookahead;       /* Dirichlet/LDA: sweeps a component may run ahead, 1..16         */
  uint32_t producer_warps;  /* normal-gamma brng_gibbs_run: warps per block that only refill  */
                            /* the rings while the others sample (asynchronous replenishment, */
                            /* Sec. 3 item 3), 1..8, or BRNG_PRODUCERS_NONE: each warp refills */
                            /* its own rings when they run dry (Sec. 2.2).  Same results.    */
} brng_tuning_t;
#define BRNG_PRODUCERS_NONE 0xffffffffu

/* ---- handle (Sec. 2.2 constructor / destructor) ---------------------------
 * brng_create: a handle with `n_streams` streams (>= 1, < 2^32) keyed by
 * `seed`, buffer length `buf_len` (0 = default 32; power of two, 4..512),
 * on the current CUDA device.  It owns per-stream positions (4 x uint64 per
 * stream: the U, N, E domains and the U64 domain of brng_uniform_f64; all
 * zero = every stream at its start) and the counters.  The
 * paper's constructor fills the buffers at once; here rings are filled lazily
 * inside each kernel, which gives the same values.  *out is set only on
 * BRNG_OK.  brng_destroy frees it (NULL is a no-op); no call on the handle
 * may be in flight.  Calls on one handle must be ordered on the device (one
 * CUDA stream, or streams ordered by events): they read and advance the same
 * stream positions (and brng_mixed its dispatch word). */
int brng_create(uint64_t seed, uint32_t n_streams, uint32_t buf_len, brng_t **out);
int brng_destroy(brng_t *h);
int brng_set_tuning(brng_t *h, const brng_tuning_t *t); /* host struct */
int brng_get_tuning(const brng_t *h, brng_tuning_t *t);
uint32_t brng_n_streams(const brng_t *h);
uint64_t brng_seed(const brng_t *h);

/* Checkpoint / resume of the stream positions: host array of 3*n_streams
 * uint64, laid out [stream][U, N, E].  Synchronous (device-wide sync). */
int brng_get_positions(brng_t *h, uint64_t *host_pos);
int brng_set_positions(brng_t *h, const uint64_t *host_pos);
/* The same for the streams' U64-domain positions (brng_uniform_f64): host
 * array of n_streams uint64.  Synchronous (device-wide sync). */
int brng_get_positions_u64(brng_t *h, uint64_t *host_pos);
int brng_set_positions_u64(brng_t *h, const uint64_t *host_pos);

/* Reads (and if `reset`, zeroes) the device counters after synchronising
 * `stream`.  Returns BRNG_ETIMEOUT if n_timeout > 0 (a bounded device wait ran
 * out), else BRNG_EDOMAIN if n_domain > 0, else BRNG_EREJECT if n_reject > 0,
 * else BRNG_OK (or a CUDA error).  `out` (host) may be NULL. */
int brng_read_counters(brng_t *h, brng_stream_t stream, brng_counters_t *out, int reset);

/* ---- core engine (Sec. 2.2 "vectorized RNG for uniform distribution") ----
 * Raw Philox4x32-10 words of blocks [first_block, first_block + n_blocks) of
 * (domain, stream_id) under the handle's key: out (device, 4*n_blocks uint32)
 * gets the 4 words of each block in order.  Stateless. */
int brng_philox_words(brng_t *h, uint32_t domain, uint32_t stream_id, uint64_t first_block,
                      size_t n_blocks, uint32_t *out, brng_stream_t stream);

/* ===== TEST AND MEASUREMENT HOOKS =========================================
 * brng_philox_peak, brng_fp32_eval, brng_fp64_eval (below), brng_test_pc_stall
 * and brng_debug_violations (end of file) are not part of the sampling
 * interface: they exist for the parity tests, the roofline probe and the
 * failure-detection test, and a user of the library does not need them. */

/* ---- integer-pipe probe (test/measurement hook) -------------------------------
 * Runs `blocks` x `threads` (<= 256) threads, each generating 4 x `iters`
 * Philox4x32-10 blocks in registers (4 independent counter chains) and
 * writing one checksum word to sink[thread] (device, blocks*threads uint32).
 * Timing it gives the Philox generation rate of the device: the integer-pipe
 * roofline of the method (no memory traffic on the measured path). */
int brng_philox_peak(uint64_t iters, uint32_t blocks, uint32_t threads, uint32_t *sink,
                     brng_stream_t stream);

/* ---- FP32 elementary functions of the base conversions (test hook) -----------
 * out[i] = f(in[i]) on the device for fn = 0: natural log (the FP32 log of
 * the exponential and Box-Muller buffers and of the Gamma test), 1: sin and
 * 2: cos of pi k 2^-23 for the integer k = in[i] in [0, 2^24) (the Box-Muller
 * angle).  Written without integer/float conversion instructions; exposed so
 * their error can be bounded against a reference.  in, out: device float[n]. */
int brng_fp32_eval(uint32_t fn, size_t n, const float *in, float *out, brng_stream_t stream);

/* ---- FP64 elementary functions of the Gamma and Poisson rechecks (test hook) -
 * out[i] = f(in[i]) on the device for fn = 0: log, 1: sin(pi x), 2: cos(pi x),
 * 3: exp (Taylor through r^16 after reduction by ln 2),
 * the fixed-operation-order FP64 functions the Gamma sampler uses when it
 * re-decides an accept test in FP64 (log by the atanh series, sin/cos(pi x) by
 * exact reduction and Taylor series).  Exposed so that their bits can be
 * checked against a reference.  in, out: device double[n]. */
int brng_fp64_eval(uint32_t fn, size_t n, const double *in, double *out, brng_stream_t stream);
/* ===== end of the first group of test hooks ================================ */

/* ---- varying-parameter streams (Sec. 2.2 Get* functions; Sec. 2.3 method:
 * parameters read from memory per draw, every output written) -------------
 * Draw i (0 <= i < n) goes to stream i mod n_streams and takes that stream's
 * next elements; draws of one stream are taken in increasing i, and the
 * positions persist in the handle, so a later call continues every stream.
 * out (device, n float32) gets the deviate; words (device, n uint32, or
 * NULL) gets the raw Philox word of the first element the draw consumed
 * (0 if none).  An invalid parameter gives NaN, consumes nothing and counts
 * in n_domain. */
/* U[a, b):  a + (b - a) U.  Needs finite a <= b. */
int brng_uniform(brng_t *h, size_t n, const float *a, const float *b, float *out,
                 uint32_t *words, brng_stream_t stream);
/* U[a, b) in FP64 (Sec. 2.2 GetUniform at double precision): a + (b - a) U64,
 * rounded as fma(b - a, U64, a),
 * with the 53-bit uniform U64 = ((w0 >> 5) 2^26 + (w1 >> 6)) 2^-53 of domain 4,
 * element j of a stream in Philox block j/2, words (w0, w1) = (2(j%2),
 * 2(j%2)+1).  Each stream has its own U64 position (brng_get_positions_u64),
 * apart from its U, N, E positions; draw i -> stream i mod n_streams as above.
 * a, b, out: device, n float64 each; words: the pair's first word.  The same
 * two FP64 roundings as the oracle: bit-exact with it.
 * Needs finite a <= b. */
int brng_uniform_f64(brng_t *h, size_t n, const double *a, const double *b, double *out,
                     uint32_t *words, brng_stream_t stream);
/* N(mu, sigma): mu + sigma z.  Needs finite mu, finite sigma > 0. */
int brng_normal(brng_t *h, size_t n, const float *mu, const float *sigma, float *out,
                uint32_t *words, brng_stream_t stream);
/* Exp(rate lambda): E / lambda.  Needs finite lambda > 0. */
int brng_exponential(brng_t *h, size_t n, const float *lambda, float *out, uint32_t *words,
                     brng_stream_t stream);
/* Gamma(alpha, 1) by Marsaglia-Tsang (the paper withholds its GetGamma,
 * Sec. 3 note): per attempt one N element z, t = 1 + z/sqrt(9d), d = a - 1/3,
 * a = alpha (alpha >= 1) or alpha + 1; if t > 0 one U element u' and accept
 * iff ln u' < z^2/2 + d (1 - t^3 + ln t^3), result d t^3; alpha < 1 takes one
 * more U element u_b after the accept and multiplies by u_b^(1/alpha).  The
 * accept test runs in FP32 and is re-decided in FP64 (from the same Philox
 * bits) when the FP32 margin lies within its error bound.  Needs finite
 * alpha > 0; 64 rejected attempts give NaN (n_reject). */
int brng_gamma(brng_t *h, size_t n, const float *alpha, float *out, uint32_t *words,
               brng_stream_t stream);
/* Laplace(mu, b): one E element e, then one U element u; mu - b e if
 * u < 1/2 else mu + b e.  Needs finite mu, finite b > 0. */
int brng_laplace(brng_t *h, size_t n, const float *mu, const float *b, float *out,
                 uint32_t *words, brng_stream_t stream);
/* Weibull(shape k, scale lambda): lambda E^(1/k).  Needs finite k, lambda > 0. */
int brng_weibull(brng_t *h, size_t n, const float *k, const float *lambda, float *out,
                 uint32_t *words, brng_stream_t stream);
/* Poisson(lambda), a discrete distribution of the expanded library (Sec. 3
 * item 1), drawn from the same U buffer: one U element u per draw, the result
 * the smallest k with u < F(k), F the Poisson CDF summed left to right from
 * p_0 = e^-lambda, p_k = p_{k-1} lambda / k (inversion by sequential search,
 * O(lambda) steps).  The search runs in FP32; when u lies within the FP32
 * error bound of a CDF step it is repeated in double-single FP32, and when u
 * lies within that bound too, in FP64 (own exp, fixed operation order), so
 * every k equals the FP64 reference's.  That holds for
 * lambda <= BRNG_INVERSION_MAX_MEAN; above it the draw is Hormann's transformed
 * rejection PTRS (Insurance: Math. Econ. 12, 1993): per attempt U in [0, 1)
 * and V = U' from the same buffer, k = floor((2a/u_s + b)(U - 1/2) + lambda +
 * 0.43) with u_s = 1/2 - |U - 1/2|, a squeeze accept, and otherwise the test
 * ln(V / alpha'(u_s)) <= k ln lambda - lambda - ln k!.  The reference is the
 * FP64 evaluation (own log, IEEE sqrt/division, Stirling's series for ln k!);
 * each attempt is decided in FP32 and float-float where that provably gives
 * the same result, else in FP64, so every count equals the reference's.  out
 * gets k as a float (exact).  Needs finite 0 < lambda <=
 * BRNG_POISSON_MAX_LAMBDA; FP64 redraws of the inversion and attempts redone
 * in FP64 count in n_recheck; a rejection draw that runs out of attempts (64)
 * is NaN and counts in n_reject. */
int brng_poisson(brng_t *h, size_t n, const float *lambda, float *out, uint32_t *words,
                 brng_stream_t stream);
/* Binomial(n, p), the second discrete distribution of the expanded library
 * (Sec. 3 item 1): one U element u per draw; with q = min(p, 1 - p), the
 * smallest k with u < F(k), F the Binomial(n, q) CDF summed left to right
 * from (1 - q)^n, p_k = p_{k-1} (n - k + 1) q / ((1 - q) k); the draw is k, or
 * n - k when p > 1/2.  FP32 search, repeated in double-single FP32 near a
 * CDF step and in FP64 (own log and exp, fixed operation order) nearer
 * still, so every count equals the FP64 reference's (FP64 redraws count in
 * n_recheck).  Above n min(p, 1-p) = BRNG_INVERSION_MAX_MEAN the draw is
 * Hormann's BTRD (J. Statist. Comput. Simul. 46, 1993) on min(p, 1-p): per
 * attempt one U' (V), and unless V falls in the immediate-accept region one
 * more element (U when V >= v_r, else V' = U' v_r), then the recursive
 * evaluation of f(k)/f(m) for |k - m| <= 15 or a log-scale squeeze and the
 * Stirling-corrected log test; the reference is their FP64 evaluation, and
 * each attempt is decided in FP32 / float-float only where that provably
 * gives its result (else in FP64; counted in n_recheck).  trials: device
 * float[n] holding integers 0 <= n <= 2^24; prob: device float[n] in [0, 1]. */
int brng_binomial(brng_t *h, size_t n, const float *trials, const float *prob, float *out,
                  uint32_t *words, brng_stream_t stream);
/* Mixed stream: draw i is distribution tag[i] (BRNG_TAG_*) with parameters
 * (p0[i], p1[i]) as in the calls above (Gamma, Exponential, Poisson ignore p1).
 * Unknown tags give NaN (n_domain).  tag: device uint8[n]. */
int brng_mixed(brng_t *h, size_t n, const uint8_t *tag, const float *p0, const float *p1,
               float *out, uint32_t *words, brng_stream_t stream);
/* ---- Gamma draws without device allocation ----------------------------------
 * No counterpart in the paper: this entry point exists for callers that cannot
 * call cudaMalloc -- code running inside another framework's memory pool,
 * which must own every device allocation, or a loop that must not stall on the
 * device-wide synchronisation that cudaMalloc/cudaFree imply.
 * brng_gamma_static(seed, n_streams, n, alpha, out, words, stream) gives what
 * brng_create(seed, n_streams, 0, &h); brng_gamma(h, n, alpha, out, words,
 * stream); brng_destroy(h) would give -- every stream starting at its first
 * element -- but allocates nothing: its per-stream positions and counters live
 * in one fixed array in the library's device memory, which every GPU that
 * loads the library holds (about 1.5 MB) until the process exits.
 * Limits and rules:
 *   - 1 <= n_streams <= BRNG_STATIC_MAX_STREAMS, else BRNG_EINVAL (nothing is
 *     enqueued);
 *   - alpha, out (and words, if not NULL) are caller-owned device arrays of n
 *     elements, as for brng_gamma; invalid alpha gives NaN in out (no counter
 *     can be read back through this entry point);
 *   - the first call on a device looks up the array's device address (a
 *     one-time set-up per device); make that first call before any stream
 *     capture.  The address is kept for the life of the process: after a
 *     cudaDeviceReset it no longer belongs to the device's context, so a
 *     process that resets a device must not call this entry point again;
 *   - every call clears the array on `stream` before its kernel, and all calls
 *     share it: calls whose work overlaps on the GPU (other streams, other
 *     host threads) race and give wrong results.  Order them on one stream.
 * Enqueued on `stream`; returns BRNG_OK, BRNG_EINVAL or BRNG_ECUDA. */
#define BRNG_STATIC_MAX_STREAMS 65536u
int brng_gamma_static(uint64_t seed, uint32_t n_streams, size_t n, const float *alpha,
                      float *out, uint32_t *words, brng_stream_t stream);

/* Dirichlet rows (Sec. 1 footnote: K Gammas, normalised).  alpha and out are
 * device float32 [n_rows][K].  Needs K >= 1, K <= 128 and n_streams % K == 0:
 * component k of row i draws its Gamma from stream (i mod (n_streams/K))*K + k.
 * A row with any invalid alpha is all NaN and consumes nothing. */
int brng_dirichlet(brng_t *h, size_t n_rows, uint32_t K, const float *alpha, float *out,
                   brng_stream_t stream);

/* ---- Gibbs models (Markov-dependent consumers; Sec. 1) ----------------------
 * Runs `n_sweeps` sweeps of chains chain_offset .. chain_offset+n_chains-1
 * (global chain id = Philox stream id; chains never share draws, so any split
 * of a chain range over calls or devices gives identical results).  Uses the
 * handle's seed and tuning, not its stream positions: each chain's positions
 * are part of its device state, so a run continues from where the previous
 * one stopped (checkpoint = copy the state arrays).  All arrays are device
 * memory, per chain, contiguous:
 *
 * TRIANGLE (Eq. 1, Fig. 1): per sweep x <- (1 - y) U64, then y <- (1 - x) U64,
 *   FP64 without contraction.  params: NULL.  state: brng_triangle_state_t[n].
 *   moments: double[n][5] += (x, y, x^2, y^2, x y) per sweep.
 * NORMAL_GAMMA: tau | mu ~ Gamma(a0 + n/2, rate b0 + SS/2), SS = S + n (xbar -
 *   mu)^2, then mu | tau ~ N((prec0 mu0 + tau n xbar)/P, 1/P), P = prec0 + n tau.
 *   params: brng_normal_gamma_params_t (host struct, copied at the call).
 *   state: brng_normal_gamma_state_t[n].  moments: double[n][4] += (mu, tau,
 *   mu^2, tau^2) per sweep.  FP32 arithmetic, FP64 accumulators.
 * LDA: per sweep theta_d ~ Dirichlet(alpha_d); here a "chain" is a document
 *   and component (d, k) is stream (chain_offset + d)*K + k.  params:
 *   brng_lda_params_t (host struct).  state: brng_lda_state_t view (below).
 *   moments: double[n][K] += theta per sweep.
 */
typedef struct {
  double x, y;  /* current point, start (0.5, 0.5) */
  uint64_t pos; /* next U64 element of the chain */
  uint64_t pad;
} brng_triangle_state_t;

typedef struct {
  float a0, b0, mu0, prec0; /* priors: tau ~ Gamma(a0, rate b0), mu ~ N(mu0, 1/prec0) */
  const float *nobs;        /* device [n]: number of observations of each chain       */
  const float *xbar;        /* device [n]: their mean                                  */
  const float *sc;          /* device [n]: sum of squared deviations from the mean     */
} brng_normal_gamma_params_t;

typedef struct {
  float mu, tau;     /* current values; start mu = mu0 (tau is drawn first) */
  uint64_t pos_n;    /* next N element                                      */
  uint64_t pos_u;    /* next U element                                      */
} brng_normal_gamma_state_t;

typedef struct {
  uint32_t K;          /* topics, 1..128                                        */
  const float *alpha;  /* device [n][K]: Dirichlet parameter of each document   */
} brng_lda_params_t;

typedef struct {
  float *theta;   /* device [n][K]: last draw (output)                          */
  uint64_t *pos;  /* device [n][K][2]: next (N, U) element of each component      */
} brng_lda_state_t;

/* LDA_FULL (Sec. 1, the LDA paragraph: the Dirichlet's parameters change from
 *   one Gibbs iteration to the next): per sweep, for every document d (a
 *   "chain"; global id chain_offset + d), (1) each token's topic is redrawn
 *   from the collapsed conditional
 *       p(z = k) proportional to (n_dk' + alpha)(n_kw' + beta)/(n_k' + V beta)
 *   (' = without the token itself), with the word-topic counts n_kw, n_k of
 *   the start of the sweep plus the document's own changes so far (the
 *   distributed sampler of Newman et al., JMLR 2009, one document per worker;
 *   exact sequential collapsed Gibbs for a one-document corpus); the weights
 *   are FP32 in a fixed operation order, made integers (q_k = trunc(w_k
 *   2^(b-1-e)), 2^e <= max w < 2^(e+1), b = 32 - ceil(log2 K)) and the topic
 *   is the smallest k whose
 *   cumulative q exceeds (r Q) >> 24, r the top 24 bits of the document's
 *   next Z-domain word; (2) theta_d ~ Dirichlet(alpha + n_d) exactly as the
 *   LDA model (alpha + n_dk formed in FP32; component k on stream
 *   (chain_offset + d) K + k).  After the sweep the documents' count changes
 *   are added into n_kw and n_k (exchange = 0).  params:
 *   brng_lda_full_params_t (host struct).  state: brng_lda_full_state_t
 *   (host struct of device pointers).  moments: double[n][K] += theta per
 *   sweep.  z, the counts and every position are bit-exact integer results;
 *   theta is FP32.  Not available in brng_gibbs_batch.  Errors: BRNG_EINVAL
 *   for K outside 1..128, V = 0, alpha or beta not in [1e-6, 1e6], a NULL
 *   array, or exchange = 1 with n_sweeps != 1. */
#define BRNG_LDA_NONE 0xFFFFFFFFu
typedef struct {
  uint32_t K, V;            /* topics (1..128), vocabulary size (words < V)             */
  float alpha, beta;        /* symmetric document-topic and topic-word priors           */
  const uint32_t *doc_ptr;  /* device [n+1]: document d holds tokens doc_ptr[d] ..
                               doc_ptr[d+1]-1 (offsets into words, prev and z)           */
  const uint32_t *words;    /* device [tokens]: word of each token                      */
  const uint32_t *prev;     /* device [tokens]: the document's previous token with the
                               same word, or BRNG_LDA_NONE (brng_lda_index makes it)      */
  uint32_t exchange;        /* 0: every sweep's count changes are added into nkw, nk
                               before the next; 1 (n_sweeps = 1 only): they are left in
                               dnkw for the caller to sum over devices, then
                               brng_lda_apply adds them                                  */
  const uint32_t *order;    /* device [n] or NULL: the order in which the documents'
                               topic draws are started (a permutation of 0..n-1;
                               longest first balances the uneven lengths).  Speed only:
                               no value depends on it.  NULL: 0, 1, ..., n-1             */
} brng_lda_full_params_t;

typedef struct {
  uint8_t *z;         /* device [tokens]: topic of each token (in/out)              */
  uint8_t *z_start;   /* device [tokens]: workspace (each token's topic at the start
                         of the sweep)                                               */
  int32_t *ndk;       /* device [n][K]: document-topic counts (in/out)              */
  int32_t *nkw;       /* device [V][K]: word-topic counts of the whole corpus        */
  int32_t *nk;        /* device [K]: topic totals of the whole corpus                */
  int32_t *dnkw;      /* device [V*K + K]: count changes (word-topic, then topic);
                         zero on entry and, with exchange = 0, on return              */
  float *dir_alpha;   /* device [n][K]: workspace (alpha + n_dk of the theta draw)   */
  uint64_t *zpos;     /* device [n]: next Z-domain element of each document          */
  float *theta;       /* device [n][K]: last theta draw (output)                     */
  uint64_t *pos;      /* device [n][K][2]: next (N, U) element of each component     */
} brng_lda_full_state_t;

int brng_gibbs_run(brng_t *h, brng_model_t model, uint64_t chain_offset, uint32_t n_chains,
                   uint32_t n_sweeps, const void *params, void *state, double *moments,
                   brng_stream_t stream);

/* The LDA_FULL model's helpers (no counterpart in the paper: corpus indexing
 * and the count exchange of the distributed sampler).  brng_lda_index fills
 * prev[t] (above) for the tokens of n_docs documents (device doc_ptr [n+1],
 * words); one pass, O(L^2) per document of L tokens.  brng_lda_apply adds the
 * changes dnkw [V*K + K] into nkw [V][K] and nk [K] and zeroes dnkw.  Both are
 * asynchronous on `stream`; BRNG_EINVAL for NULL arrays or K outside 1..128. */
int brng_lda_index(uint32_t n_docs, const uint32_t *doc_ptr, const uint32_t *words, uint32_t *prev,
                   brng_stream_t stream);
int brng_lda_apply(uint32_t K, uint32_t V, int32_t *nkw, int32_t *nk, int32_t *dnkw,
                   brng_stream_t stream);

/* ---- batched Gibbs jobs: uneven ensembles in one persistent kernel ---------
 * Batching/serving (the paper's asynchronous-service idea, Sec. 3 item 3): a
 * job is the argument list of one brng_gibbs_run plus its own seed.  All jobs
 * of a batch run in ONE launch: each job splits into units of one warp (32
 * triangle or normal-gamma chains, one LDA document); resident warps claim
 * units from a counter, longest units first.  Every job's results are
 * identical to brng_gibbs_run on a handle created with the job's seed and the
 * same tuning (lanes_per_chain is 1 inside a batch), because each unit runs
 * the same code on the same streams.  Jobs of one batch must not share state
 * or output memory. */
typedef struct {
  brng_model_t model;
  uint32_t n_chains;     /* chains (documents for LDA); 0 = empty job      */
  uint32_t n_sweeps;
  uint32_t pad;
  uint64_t seed;         /* the job's Philox key                             */
  uint64_t chain_offset; /* global chain id of the job's first chain         */
  const void *params;    /* as brng_gibbs_run (host struct or NULL), read at */
  void *state;           /*   planning time; device state / moments as       */
  double *moments;       /*   brng_gibbs_run                                  */
} brng_job_t;

typedef struct brng_batch brng_batch_t;

/* brng_batch_create: validate the jobs and upload their table (synchronous;
 * allocates device memory); brng_batch_launch: reset the unit counter and
 * launch the persistent kernel on `stream` (two stream operations, no host
 * synchronisation: it can be captured in a CUDA graph and replayed, each
 * replay continuing every job's chains); brng_batch_destroy frees it (no
 * launch may be in flight).  Errors: BRNG_EINVAL for a bad job (the first
 * one found), else CUDA errors. */
int brng_batch_create(brng_t *h, const brng_job_t *jobs, uint32_t n_jobs, brng_batch_t **out);
int brng_batch_launch(brng_batch_t *b, brng_stream_t stream);
int brng_batch_destroy(brng_batch_t *b);

/* brng_gibbs_batch: plan + launch in one call, using table memory owned by
 * the handle (grown as needed); asynchronous on `stream`.  Calls on one
 * handle must be ordered (one stream). */
int brng_gibbs_batch(brng_t *h, const brng_job_t *jobs, uint32_t n_jobs, brng_stream_t stream);

/* ---- serving: continuous batching of Gibbs jobs ------------------------------
 * A server owns a scheduler thread on the current device.  brng_serve_submit
 * queues a job (copying its host inputs) and returns at once.  The scheduler
 * admits queued jobs in arrival order while their device memory (state,
 * moments, inputs) fits `mem_budget` bytes, and launches every admitted job
 * not yet running as one batch on one of `max_inflight` streams, so work that
 * arrives while earlier batches run starts at once and overlaps with them on
 * the device.  A served job gives exactly the results of brng_gibbs_run for
 * it alone (its own seed, start state x = y = 0.5 / mu = mu0 / empty LDA
 * positions, zero moments).  Results stay on the device until
 * brng_serve_result copies them to the host (state as in brng_gibbs_run; for
 * LDA the last theta, float [n][K]) and returns the memory to the budget:
 * collect every job, or admission stalls.  A job larger than the whole budget
 * fails with BRNG_ENOMEM. */
typedef struct brng_server brng_server_t;

typedef struct {
  brng_model_t model;
  uint32_t n_chains;     /* chains (documents for LDA), >= 1                  */
  uint32_t n_sweeps;
  uint32_t K;            /* LDA topics                                        */
  uint64_t seed;
  uint64_t chain_offset;
  const float *nobs;     /* host [n] (NORMAL_GAMMA), copied at submit          */
  const float *xbar;     /* host [n]                                          */
  const float *sc;       /* host [n]                                          */
  const float *alpha;    /* host [n][K] (LDA), copied at submit               */
  float a0, b0, mu0, prec0; /* NORMAL_GAMMA priors                             */
  uint32_t flags;        /* BRNG_SERVE_BORROW_INPUTS: the host arrays stay valid */
  uint32_t pad;          /*   until the job finishes and are read at admission  */
} brng_request_t;        /*   instead of being copied at submit                  */

#define BRNG_SERVE_BORROW_INPUTS 1u

typedef struct {
  uint64_t submitted_ns, admitted_ns, launched_ns, completed_ns; /* steady clock */
  uint64_t device_bytes;
  int32_t status;
  uint32_t pad;
} brng_job_info_t;

typedef struct {
  uint64_t submitted, admitted, completed, refused, batches, queued, device_bytes_in_use;
  uint64_t cancelled;  /* by brng_serve_cancel, or still queued at close */
} brng_serve_stats_t;

int brng_serve_open(uint64_t mem_budget, uint32_t max_inflight, const brng_tuning_t *tuning,
                    brng_server_t **out);
int brng_serve_submit(brng_server_t *s, const brng_request_t *req, uint64_t *job_id);
/* *done = 1 once finished (or failed; the return value is then its status) */
int brng_serve_poll(brng_server_t *s, uint64_t job_id, int *done);
/* blocks up to timeout_s; BRNG_EAGAIN on timeout */
int brng_serve_wait(brng_server_t *s, uint64_t job_id, double timeout_s);
/* host_state / host_moments may be NULL; BRNG_EAGAIN if not finished; the
 * job is forgotten afterwards (BRNG_ENOTFOUND on a second call) */
int brng_serve_result(brng_server_t *s, uint64_t job_id, void *host_state, double *host_moments,
                      brng_job_info_t *info);
int brng_serve_stats(brng_server_t *s, brng_serve_stats_t *out);
/* Withdraws a job that still waits for memory: it is forgotten (later calls
 * on its id give BRNG_ENOTFOUND) and counted as cancelled.  BRNG_EAGAIN once
 * it has been admitted (it then runs to the end), BRNG_ENOTFOUND for an
 * unknown id. */
int brng_serve_cancel(brng_server_t *s, uint64_t job_id);
/* cancels the jobs still waiting for memory or for a launch, lets the batches
 * already launched finish, frees everything; uncollected results are lost */
int brng_serve_close(brng_server_t *s);

/* ---- test hook: failure detection without a GPU fault ----------------------
 * Runs brng_gibbs_run's normal-gamma sampler (chain_offset 0) in the
 * producer/consumer form (the handle's producer_warps, 1 if none) with
 * producer warps that write nothing, so that every consumer wait for ring
 * elements runs out after its bound (1 s of the global timer): the chains end
 * with NaN state, n_timeout counts the expired waits and brng_read_counters
 * returns BRNG_ETIMEOUT.  Nothing hangs; the context stays usable.
 * Asynchronous on `stream`; arguments as brng_gibbs_run. */
int brng_test_pc_stall(brng_t *h, uint32_t n_chains, uint32_t n_sweeps, const void *params, void *state,
                       double *moments, brng_stream_t stream);

/* Test hook.  Checked build (compiled with -DBRNG_DEBUG): the number of failed protocol
 * checks -- a ring element read or consumed before it was generated, a refill
 * over unread slots, a batch unit outside its job -- counted on the device
 * since the last reset (nothing traps).  Synchronous.  BRNG_EINVAL in the
 * normal build, which has no checks. */
int brng_debug_violations(uint64_t *count, int reset);

#ifdef __cplusplus
}
#endif
#endif /* BRNG_H */
