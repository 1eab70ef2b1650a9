"""Seeded synthetic inputs shaped like the paper's workloads.

This module holds no arithmetic of the method itself (no generator, no
transform, no Gibbs update): it only draws the *inputs* -- per-draw parameter
arrays, observation summaries, topic counts -- with numpy's own seeded
generator.  The CUDA path and the oracle are both fed from here.

Workloads (arXiv 1412.4825):
  * triangle Gibbs of Eq. 1 / Fig. 1 needs no input beyond the start (0.5, 0.5);
  * normal-gamma Gibbs: per chain n observations ~ N(mean, sd^2), reduced to
    (n, xbar, S = sum (x - xbar)^2) in FP64 and handed over as FP32;
  * LDA document-topic step (Sec. 1, LDA paragraph): per document a topic mix
    phi ~ Dir(prior * 1_K), a length L ~ U{len_lo..len_hi}, counts ~ Mult(L, phi),
    and the Dirichlet parameter alpha = prior + counts formed in FP32;
  * full LDA step (topic draws per token): a synthetic corpus from LDA's own
    generative model (topic-word distributions ~ Dir(word_prior), per
    document a topic mix ~ Dir(doc_prior), a length ~ U{len_lo..len_hi}, per
    token a topic from the mix and a word from that topic), a uniformly random
    initial topic per token and the count tables of that assignment;
  * varying-parameter streams (Sec. 2.3, parameters read from memory per
    draw): log-uniform parameters, and for the mixed stream a tag per draw.
"""
from __future__ import annotations

import numpy as np

TAG_UNIFORM, TAG_NORMAL, TAG_EXPONENTIAL, TAG_GAMMA, TAG_LAPLACE, TAG_WEIBULL, TAG_POISSON, TAG_BINOMIAL = (
    0, 1, 2, 3, 4, 5, 6, 7)


def log_uniform(rng: np.random.Generator, lo: float, hi: float, n: int) -> np.ndarray:
    return np.exp(rng.uniform(np.log(lo), np.log(hi), n)).astype(np.float32)


def normal_gamma_data(n_chains: int, n_obs: int = 100, mean: float = 1.5, sd: float = 2.0,
                      seed: int = 42, chunk: int = 8192):
    """Per-chain sufficient statistics (nobs, xbar, S) as float32 arrays."""
    rng = np.random.default_rng(seed)
    nobs = np.full(n_chains, n_obs, dtype=np.float32)
    xbar = np.empty(n_chains, dtype=np.float32)
    sc = np.empty(n_chains, dtype=np.float32)
    for c0 in range(0, n_chains, chunk):
        c1 = min(n_chains, c0 + chunk)
        x = rng.normal(mean, sd, size=(c1 - c0, n_obs))
        xb = x.mean(axis=1)
        xbar[c0:c1] = xb
        sc[c0:c1] = ((x - xb[:, None]) ** 2).sum(axis=1)
    return nobs, xbar, sc


def lda_alpha(n_docs: int, K: int = 64, len_lo: int = 50, len_hi: int = 500, prior: float = 0.1,
              seed: int = 42):
    """(alpha float32 [n_docs, K], counts uint32 [n_docs, K], lengths)."""
    rng = np.random.default_rng(seed)
    phi = rng.dirichlet(np.full(K, prior), size=n_docs)
    lengths = rng.integers(len_lo, len_hi + 1, size=n_docs)
    counts = np.stack([rng.multinomial(int(L), p) for L, p in zip(lengths, phi)]).astype(np.uint32)
    alpha = (np.float32(prior) + counts.astype(np.float32)).astype(np.float32)
    return alpha, counts, lengths


def lda_corpus(n_docs: int, K: int = 64, V: int = 4096, len_lo: int = 50, len_hi: int = 500,
               doc_prior: float = 0.1, word_prior: float = 0.05, seed: int = 42):
    """A corpus drawn from LDA's generative model: dict(K, V, doc_ptr uint32
    [n_docs + 1] token offsets, words uint32 [n_tokens])."""
    rng = np.random.default_rng(seed)
    phi = rng.dirichlet(np.full(V, word_prior), size=K)          # topic-word
    lengths = rng.integers(len_lo, len_hi + 1, size=n_docs)
    doc_ptr = np.zeros(n_docs + 1, dtype=np.uint32)
    np.cumsum(lengths, out=doc_ptr[1:])
    n_tok = int(doc_ptr[-1])
    mix = rng.dirichlet(np.full(K, doc_prior), size=n_docs)      # document-topic
    # per token: topic by inversion of its document's mix, word by inversion
    # of its topic's distribution
    cmix = np.cumsum(mix, axis=1)
    cmix[:, -1] = 1.0
    doc_of = np.repeat(np.arange(n_docs), lengths)
    u = rng.random(n_tok)
    # row-wise inversion: rows shifted by their document index, one search
    flat = (cmix + np.arange(n_docs)[:, None]).ravel()
    topic = np.searchsorted(flat, u + doc_of, side="right") - doc_of * K
    topic = np.clip(topic, 0, K - 1)
    cphi = np.cumsum(phi, axis=1)
    cphi[:, -1] = 1.0
    words = np.empty(n_tok, dtype=np.uint32)
    v = rng.random(n_tok)
    for k in range(K):
        idx = np.nonzero(topic == k)[0]
        words[idx] = np.minimum(np.searchsorted(cphi[k], v[idx], side="right"), V - 1)
    return dict(K=K, V=V, doc_ptr=doc_ptr, words=words)


def lda_initial_state(corpus: dict, seed: int = 7):
    """Uniformly random initial topics and the count tables they imply:
    dict(z uint8 [n_tokens], ndk int32 [n_docs, K], nkw int32 [V, K],
    nk int32 [K], zpos uint64 [n_docs] (next topic-draw element per
    document), pos uint64 [n_docs, K, 2] (Dirichlet component positions),
    mom float64 [n_docs, K], theta float64 [n_docs, K])."""
    K, V = corpus["K"], corpus["V"]
    doc_ptr, words = corpus["doc_ptr"], corpus["words"]
    n_docs = doc_ptr.size - 1
    rng = np.random.default_rng(seed)
    z = rng.integers(0, K, size=words.size, dtype=np.uint8)
    doc_of = np.repeat(np.arange(n_docs), np.diff(doc_ptr.astype(np.int64)))
    ndk = np.bincount(doc_of * K + z, minlength=n_docs * K).reshape(n_docs, K).astype(np.int32)
    nkw = np.bincount(words.astype(np.int64) * K + z, minlength=V * K).reshape(V, K).astype(np.int32)
    nk = np.bincount(z, minlength=K).astype(np.int32)
    return dict(z=z, ndk=ndk, nkw=nkw, nk=nk, zpos=np.zeros(n_docs, dtype=np.uint64),
                pos=np.zeros((n_docs, K, 2), dtype=np.uint64), mom=np.zeros((n_docs, K)),
                theta=np.zeros((n_docs, K)))


def uniform_params(n: int, seed: int = 42, lo: float = 1e-3, hi: float = 1e3):
    rng = np.random.default_rng(seed)
    a = log_uniform(rng, lo, hi, n)
    b = log_uniform(rng, lo, hi, n)
    return np.minimum(a, b), np.maximum(a, b)


def normal_params(n: int, seed: int = 42):
    rng = np.random.default_rng(seed)
    mu = log_uniform(rng, 1e-3, 1e3, n) * np.where(rng.random(n) < 0.5, -1, 1).astype(np.float32)
    sigma = log_uniform(rng, 1e-2, 1e2, n)
    return mu.astype(np.float32), sigma


def rate_params(n: int, seed: int = 42):
    return log_uniform(np.random.default_rng(seed), 1e-2, 1e2, n)


def shape_params(n: int, seed: int = 42, lo: float = 0.05, hi: float = 50.0):
    return log_uniform(np.random.default_rng(seed), lo, hi, n)


def mixed_stream_torch(n: int, seed: int = 42, n_tags: int = 4, device="cuda"):
    """The mixed stream's inputs drawn on the device with a seeded torch
    generator (same distributions as mixed_stream; different draws), for
    sizes where host generation and transfer would dominate (2^28 draws)."""
    import torch

    g = torch.Generator(device=device)
    g.manual_seed(seed)

    def logu(lo, hi):
        u = torch.rand(n, generator=g, device=device, dtype=torch.float32)
        return torch.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * u)

    tag = torch.randint(0, n_tags, (n,), generator=g, device=device, dtype=torch.uint8)
    a, b = logu(1e-3, 1e3), logu(1e-3, 1e3)
    sign = torch.where(torch.rand(n, generator=g, device=device) < 0.5, -1.0, 1.0)
    p0 = torch.where(tag == TAG_UNIFORM, torch.minimum(a, b), a * sign)
    p1 = torch.where(tag == TAG_UNIFORM, torch.maximum(a, b), logu(1e-2, 1e2))
    del a, b, sign
    p0 = torch.where(tag == TAG_EXPONENTIAL, logu(1e-2, 1e2), p0)
    p0 = torch.where(tag == TAG_GAMMA, logu(0.05, 50.0), p0)
    p1 = torch.where((tag == TAG_EXPONENTIAL) | (tag == TAG_GAMMA), torch.zeros_like(p1), p1)
    if n_tags > TAG_WEIBULL:
        p0 = torch.where(tag == TAG_WEIBULL, logu(0.5, 5.0), p0)
    if n_tags > TAG_POISSON:
        p0 = torch.where(tag == TAG_POISSON, logu(0.05, 64.0), p0)
        p1 = torch.where(tag == TAG_POISSON, torch.zeros_like(p1), p1)
    if n_tags > TAG_BINOMIAL:  # as binomial_params: trials log-U integers [1, 1000], mean <= 64
        trials = torch.floor(logu(1.0, 1001.0))
        prob = torch.rand(n, generator=g, device=device, dtype=torch.float32)
        q = torch.minimum(prob, 1.0 - prob)
        cap = 0.999 * 64.0 / torch.clamp(trials, min=1.0)
        prob = torch.where(trials * q > 64.0, torch.where(prob <= 0.5, cap, 1.0 - cap), prob)
        p0 = torch.where(tag == TAG_BINOMIAL, trials, p0)
        p1 = torch.where(tag == TAG_BINOMIAL, prob, p1)
    return tag, p0.contiguous(), p1.contiguous()


def mixed_stream(n: int, seed: int = 42, n_tags: int = 4):
    """Tag per draw (uniform over the first n_tags distributions) and its
    parameters (p0, p1): U(a,b) a,b log-U[1e-3,1e3] sorted; N(mu, sigma)
    mu = +-log-U[1e-3,1e3], sigma log-U[1e-2,1e2]; Exp(rate) log-U[1e-2,1e2];
    Gamma(alpha) log-U[0.05, 50]; Laplace(mu, b) like Normal; Weibull(k, lambda)
    k log-U[0.5, 5], lambda log-U[1e-2, 1e2]; Poisson(lambda) log-U[0.05, 64];
    Binomial(n, p) as binomial_params."""
    rng = np.random.default_rng(seed)
    tag = rng.integers(0, n_tags, size=n, dtype=np.uint8)
    p0 = np.empty(n, dtype=np.float32)
    p1 = np.zeros(n, dtype=np.float32)
    for t in range(n_tags):
        idx = np.nonzero(tag == t)[0]
        m = idx.size
        if t == TAG_UNIFORM:
            a = log_uniform(rng, 1e-3, 1e3, m)
            b = log_uniform(rng, 1e-3, 1e3, m)
            p0[idx], p1[idx] = np.minimum(a, b), np.maximum(a, b)
        elif t in (TAG_NORMAL, TAG_LAPLACE):
            sign = np.where(rng.random(m) < 0.5, -1.0, 1.0).astype(np.float32)
            p0[idx] = log_uniform(rng, 1e-3, 1e3, m) * sign
            p1[idx] = log_uniform(rng, 1e-2, 1e2, m)
        elif t == TAG_EXPONENTIAL:
            p0[idx] = log_uniform(rng, 1e-2, 1e2, m)
        elif t == TAG_GAMMA:
            p0[idx] = log_uniform(rng, 0.05, 50.0, m)
        elif t == TAG_WEIBULL:
            p0[idx] = log_uniform(rng, 0.5, 5.0, m)
            p1[idx] = log_uniform(rng, 1e-2, 1e2, m)
        elif t == TAG_POISSON:
            p0[idx] = log_uniform(rng, 0.05, 64.0, m)
        elif t == TAG_BINOMIAL:
            p0[idx], p1[idx] = binomial_params(m, rng=rng)
    return tag, p0, p1


def poisson_params(n: int, seed: int = 42, lo: float = 0.05, hi: float = 64.0):
    return log_uniform(np.random.default_rng(seed), lo, hi, n)


def binomial_params(n: int, seed: int = 42, max_trials: int = 1000, rng=None):
    """(trials, prob): trials log-uniform integers in [1, max_trials] (some 0),
    prob uniform in [0, 1], clipped so that trials * min(p, 1-p) <= 64."""
    rng = rng if rng is not None else np.random.default_rng(seed)
    trials = np.floor(np.exp(rng.uniform(0.0, np.log(max_trials + 1), n))).astype(np.float32)
    trials[rng.random(n) < 0.02] = 0.0
    prob = rng.random(n).astype(np.float32)
    q = np.minimum(prob, 1.0 - prob)
    over = trials.astype(np.float64) * q > 64.0
    cap = (64.0 / np.maximum(trials, 1.0)).astype(np.float32) * np.float32(0.999)
    prob = np.where(over, np.where(prob <= 0.5, cap, np.float32(1.0) - cap), prob).astype(np.float32)
    return trials, prob
