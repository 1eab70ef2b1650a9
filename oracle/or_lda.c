/*
 * or_lda.c -- the full LDA Gibbs step: topic assignments resampled per token,
 * so that the document-topic counts, and with them the Dirichlet parameters
 * of the next theta draw, change every sweep (Sec. 1, the LDA paragraph: the
 * Dirichlet's parameters change from one Gibbs iteration to the next; its
 * footnote: Dirichlet from normalised Gammas).
 * TEST INFRASTRUCTURE ONLY (see oracle.h).
 *
 * The topic of token i of document d (word w, current topic z) is drawn from
 * the collapsed conditional of LDA (Griffiths & Steyvers, PNAS 2004):
 *
 *     p(z_i = k | rest) proportional to
 *         (n_dk' + alpha) (n_kw' + beta) / (n_k' + V beta),
 *
 * where ' marks counts without token i itself.  Documents are sampled in
 * parallel against the word-topic counts n_kw, n_k of the start of the sweep
 * (a snapshot), each seeing its own changes of the sweep at once (n_dk always,
 * and its own word-topic changes on top of the snapshot), and the changes of
 * all documents are added into n_kw and n_k when the sweep ends -- the
 * approximate distributed sampler of Newman, Asuncion, Smyth & Welling (JMLR
 * 2009) with one document per worker.  For a corpus of one document this is
 * the exact sequential collapsed Gibbs sampler.
 *
 * The draw is decided in FP32 (the precision of the CUDA path, so that both
 * decide identically):
 *     inv_k = 1 / (float(n_k') + Vbeta),  Vbeta = float(V) * beta,
 *     w_k = ((float(n_dk') + alpha) * (float(n_kw') + beta)) * inv_k,
 * each operation rounded to FP32 in this order; the weights are then made
 * integers q_k = trunc(w_k 2^(b - 1 - e)), with 2^e <= max_k w_k < 2^(e+1)
 * and b = 32 - ceil(log2 K) bits per weight (so q_k < 2^b and the K weights
 * sum below 2^32), and the topic is the smallest k whose integer cumulative
 * sum C_k exceeds floor(r Q / 2^24), Q = C_(K-1), r = the top 24 bits of the
 * token's word from the document's Z-domain stream (domain 5, stream = global
 * document id, one element per token draw).  Everything after the weights is
 * exact integer arithmetic.
 */
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include "oracle.h"
#include "or_internal.h"

static float f32_of_bits(uint32_t b) {
  float f;
  memcpy(&f, &b, 4);
  return f;
}

static uint32_t bits_of_f32(float f) {
  uint32_t b;
  memcpy(&b, &f, 4);
  return b;
}

void or_lda_weights(uint32_t K, float alpha, float beta, float vbeta, const int32_t *ndk,
                    const int32_t *nkw_w, const int32_t *nk, uint32_t z_old, float *w_out,
                    uint32_t *q_out) {
  float m = 0.0f;
  for (uint32_t k = 0; k < K; ++k) {
    int32_t self = k == z_old ? 1 : 0;
    float inv = 1.0f / ((float)(nk[k] - self) + vbeta);
    float a = (float)(ndk[k] - self) + alpha;
    float b = (float)(nkw_w[k] - self) + beta;
    float w = (a * b) * inv;
    w_out[k] = w;
    if (w > m) m = w;
  }
  /* 2^e <= m < 2^(e+1) with e = exponent field - 127; b = 32 - ceil(log2 K);
   * scale = 2^(b - 1 - e), exponent field 127 + b - 1 - e = 253 + b - field */
  uint32_t lg = 0;
  while ((1u << lg) < K) ++lg;
  uint32_t b = 32u - lg;
  uint32_t ef = (bits_of_f32(m) >> 23) & 0xFFu;
  float scale = f32_of_bits((253u + b - ef) << 23);
  for (uint32_t k = 0; k < K; ++k) q_out[k] = (uint32_t)(w_out[k] * scale);
}

uint32_t or_lda_pick(uint32_t K, const uint32_t *q, uint32_t r24) {
  uint64_t Q = 0;
  for (uint32_t k = 0; k < K; ++k) Q += q[k];
  uint64_t t = ((uint64_t)r24 * Q) >> 24;
  uint64_t c = 0;
  for (uint32_t k = 0; k < K; ++k) {
    c += q[k];
    if (c > t) return k;
  }
  return K - 1; /* not reached: C_(K-1) = Q > t */
}

int or_lda_z_sweep(uint64_t seed, uint64_t doc_offset, uint32_t n_docs, uint32_t K, uint32_t V,
                   float alpha, float beta, const uint32_t *doc_ptr, const uint32_t *words,
                   uint8_t *z, int32_t *ndk, const int32_t *nkw, const int32_t *nk,
                   int32_t *dnkw, int32_t *dnk, uint64_t *zpos) {
  if (K == 0 || K > 255 || V == 0 || !(alpha > 0.0f) || !(beta > 0.0f)) return OR_EINVAL;
  const float vbeta = (float)V * beta;
  /* the running document's own word-topic changes, dense, cleared per document */
  int32_t *own = (int32_t *)calloc((size_t)V * K, sizeof(int32_t));
  int32_t *own_k = (int32_t *)malloc(sizeof(int32_t) * K);
  int32_t *nkw_w = (int32_t *)malloc(sizeof(int32_t) * K);
  int32_t *nk_cur = (int32_t *)malloc(sizeof(int32_t) * K);
  float *w = (float *)malloc(sizeof(float) * K);
  uint32_t *q = (uint32_t *)malloc(sizeof(uint32_t) * K);
  for (uint32_t d = 0; d < n_docs; ++d) {
    const uint32_t t0 = doc_ptr[d], t1 = doc_ptr[d + 1];
    const uint32_t stream = (uint32_t)(doc_offset + d);
    int32_t *nd = ndk + (uint64_t)d * K;
    memset(own_k, 0, sizeof(int32_t) * K);
    for (uint32_t t = t0; t < t1; ++t) {
      const uint32_t wd = words[t];
      const uint32_t zo = z[t];
      for (uint32_t k = 0; k < K; ++k) {
        nkw_w[k] = nkw[(uint64_t)wd * K + k] + own[(uint64_t)wd * K + k];
        nk_cur[k] = nk[k] + own_k[k];
      }
      or_lda_weights(K, alpha, beta, vbeta, nd, nkw_w, nk_cur, zo, w, q);
      const uint32_t r24 = or_elem_word(seed, OR_DOM_Z, stream, zpos[d]++) >> 8;
      const uint32_t zn = or_lda_pick(K, q, r24);
      if (zn != zo) {
        nd[zo] -= 1;
        nd[zn] += 1;
        own_k[zo] -= 1;
        own_k[zn] += 1;
        own[(uint64_t)wd * K + zo] -= 1;
        own[(uint64_t)wd * K + zn] += 1;
        dnkw[(uint64_t)wd * K + zo] -= 1;
        dnkw[(uint64_t)wd * K + zn] += 1;
        z[t] = (uint8_t)zn;
      }
    }
    for (uint32_t k = 0; k < K; ++k) dnk[k] += own_k[k];
    for (uint32_t t = t0; t < t1; ++t) /* clear the rows this document touched */
      memset(own + (uint64_t)words[t] * K, 0, sizeof(int32_t) * K);
  }
  free(own);
  free(own_k);
  free(nkw_w);
  free(nk_cur);
  free(w);
  free(q);
  return OR_OK;
}

/* ---- thread harness: contiguous document ranges, private change arrays -- */

typedef struct {
  uint64_t seed, doc_offset;
  uint32_t n_docs, K, V;
  float alpha, beta;
  const uint32_t *doc_ptr, *words;
  uint8_t *z;
  int32_t *ndk;
  const int32_t *nkw, *nk;
  int32_t *dnkw, *dnk;
  uint64_t *zpos;
  int status;
} or_zjob;

static void *or_zrun(void *arg) {
  or_zjob *j = (or_zjob *)arg;
  j->status = or_lda_z_sweep(j->seed, j->doc_offset, j->n_docs, j->K, j->V, j->alpha, j->beta,
                             j->doc_ptr, j->words, j->z, j->ndk, j->nkw, j->nk, j->dnkw, j->dnk,
                             j->zpos);
  return NULL;
}

int or_lda_z_sweep_mt(uint64_t seed, uint64_t doc_offset, uint32_t n_docs, uint32_t K, uint32_t V,
                      float alpha, float beta, const uint32_t *doc_ptr, const uint32_t *words,
                      uint8_t *z, int32_t *ndk, const int32_t *nkw, const int32_t *nk,
                      int32_t *dnkw, int32_t *dnk, uint64_t *zpos, int nthreads) {
  if (nthreads < 1) nthreads = 1;
  if ((uint32_t)nthreads > n_docs) nthreads = n_docs ? (int)n_docs : 1;
  or_zjob *jobs = (or_zjob *)calloc(nthreads, sizeof(or_zjob));
  pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nthreads);
  for (int t = 0; t < nthreads; ++t) {
    uint32_t b = (uint32_t)((uint64_t)n_docs * t / nthreads);
    uint32_t e = (uint32_t)((uint64_t)n_docs * (t + 1) / nthreads);
    jobs[t] = (or_zjob){.seed = seed, .doc_offset = doc_offset + b, .n_docs = e - b, .K = K, .V = V,
                        .alpha = alpha, .beta = beta, .doc_ptr = doc_ptr + b, .words = words,
                        .z = z, .ndk = ndk + (uint64_t)b * K, .nkw = nkw, .nk = nk,
                        .dnkw = t ? (int32_t *)calloc((size_t)V * K, sizeof(int32_t)) : dnkw,
                        .dnk = t ? (int32_t *)calloc(K, sizeof(int32_t)) : dnk,
                        .zpos = zpos + b};
  }
  for (int t = 0; t < nthreads; ++t) pthread_create(&th[t], NULL, or_zrun, &jobs[t]);
  int status = OR_OK;
  for (int t = 0; t < nthreads; ++t) {
    pthread_join(th[t], NULL);
    if (jobs[t].status != OR_OK && status == OR_OK) status = jobs[t].status;
  }
  /* integer sums: the order of the additions does not matter */
  for (int t = 1; t < nthreads; ++t) {
    for (uint64_t i = 0; i < (uint64_t)V * K; ++i) dnkw[i] += jobs[t].dnkw[i];
    for (uint32_t k = 0; k < K; ++k) dnk[k] += jobs[t].dnk[k];
    free(jobs[t].dnkw);
    free(jobs[t].dnk);
  }
  free(th);
  free(jobs);
  return status;
}

int or_lda_z_run(uint64_t seed, uint32_t n_sweeps, uint32_t n_docs, uint32_t K, uint32_t V,
                 float alpha, float beta, const uint32_t *doc_ptr, const uint32_t *words,
                 uint8_t *z, int32_t *ndk, int32_t *nkw, int32_t *nk, uint64_t *zpos,
                 uint32_t *zhist) {
  int32_t *dnkw = (int32_t *)calloc((size_t)V * K, sizeof(int32_t));
  int32_t *dnk = (int32_t *)calloc(K, sizeof(int32_t));
  int status = OR_OK;
  const uint32_t n_tok = doc_ptr[n_docs];
  for (uint32_t s = 0; s < n_sweeps && status == OR_OK; ++s) {
    status = or_lda_z_sweep(seed, 0, n_docs, K, V, alpha, beta, doc_ptr, words, z, ndk, nkw, nk,
                            dnkw, dnk, zpos);
    for (uint64_t i = 0; i < (uint64_t)V * K; ++i) {
      nkw[i] += dnkw[i];
      dnkw[i] = 0;
    }
    for (uint32_t k = 0; k < K; ++k) {
      nk[k] += dnk[k];
      dnk[k] = 0;
    }
    if (zhist)
      for (uint32_t t = 0; t < n_tok; ++t) zhist[(uint64_t)t * K + z[t]] += 1;
  }
  free(dnkw);
  free(dnk);
  return status;
}
