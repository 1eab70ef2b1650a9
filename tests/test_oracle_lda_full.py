"""Pins of the oracle's full LDA step (topic draws per token, then theta).

* The topic weights equal the collapsed conditional derived independently
  from the joint p(w, z) of LDA with theta and phi integrated out
  (Dirichlet-multinomial marginals, evaluated with log-Gamma functions), at
  the first token of a sweep, where the snapshot counts are the current ones.
* The integer pick inverts the cumulative sums exactly: every 24-bit uniform
  maps to the topic whose interval holds it, so each topic is chosen for
  exactly its share of the 2^24 values.
* Count invariants after sweeps: document rows sum to the lengths, columns to
  the topic totals, the word-topic table is the histogram of (word, topic).
* For a corpus of one document the sampler is the sequential collapsed Gibbs
  sampler, so its long-run topic frequencies per token equal the posterior
  marginals p(z_i = k | w) by brute-force enumeration of every assignment.
* Threads and document-range shards give the same draws and count changes.
"""
import itertools

import numpy as np
import pytest
from scipy.special import gammaln

from paper_1412_4825_gb300 import inputs


def _log_joint(doc_ptr, words, z, K, V, alpha, beta):
    """log p(w, z) of LDA with symmetric priors, theta and phi integrated out."""
    lp = 0.0
    for d in range(doc_ptr.size - 1):
        zd = z[doc_ptr[d]:doc_ptr[d + 1]]
        n = np.bincount(zd, minlength=K)
        lp += gammaln(K * alpha) - gammaln(zd.size + K * alpha) + np.sum(gammaln(n + alpha) - gammaln(alpha))
    nkw = np.zeros((K, V))
    np.add.at(nkw, (z, words), 1)
    for k in range(K):
        lp += gammaln(V * beta) - gammaln(nkw[k].sum() + V * beta) + np.sum(gammaln(nkw[k] + beta) - gammaln(beta))
    return lp


def _tiny_corpus(rng, n_docs, K, V, lo=2, hi=6):
    lengths = rng.integers(lo, hi + 1, n_docs)
    doc_ptr = np.zeros(n_docs + 1, dtype=np.uint32)
    np.cumsum(lengths, out=doc_ptr[1:])
    words = rng.integers(0, V, doc_ptr[-1]).astype(np.uint32)
    return dict(K=K, V=V, doc_ptr=doc_ptr, words=words)


@pytest.mark.parametrize("case", range(6))
def test_weights_equal_conditional_from_joint(oracle, case):
    rng = np.random.default_rng(100 + case)
    K, V = int(rng.integers(2, 7)), int(rng.integers(2, 9))
    alpha, beta = float(np.float32(rng.uniform(0.05, 2.0))), float(np.float32(rng.uniform(0.01, 1.0)))
    c = _tiny_corpus(rng, 3, K, V)
    st = inputs.lda_initial_state(c, seed=case)
    z = st["z"].astype(np.int64)
    words = c["words"].astype(np.int64)
    for t in range(int(c["doc_ptr"][-1])):
        d = int(np.searchsorted(c["doc_ptr"], t, side="right") - 1)
        logp = []
        for k in range(K):
            zz = z.copy()
            zz[t] = k
            logp.append(_log_joint(c["doc_ptr"], words, zz, K, V, alpha, beta))
        p = np.exp(np.array(logp) - max(logp))
        p /= p.sum()
        w, q = oracle.lda_weights(K, alpha, beta, V, st["ndk"][d], st["nkw"][words[t]], st["nk"], int(z[t]))
        wn = w.astype(np.float64) / w.astype(np.float64).sum()
        assert np.allclose(wn, p, rtol=1e-5, atol=0), (t, wn, p)
        qn = q.astype(np.float64) / q.astype(np.float64).sum()
        assert np.allclose(qn, p, rtol=1e-5, atol=2.0 ** -24)


def test_pick_inverts_integer_cdf_exactly(oracle):
    rng = np.random.default_rng(5)
    r = np.arange(1 << 24, dtype=np.uint64)
    for K in (1, 2, 5, 64):
        q = rng.integers(0, 1 << 32, K, dtype=np.uint64).astype(np.uint32)
        q[rng.random(K) < 0.2] = 0  # topics with no weight are never picked
        if q.sum() == 0:
            q[0] = 1
        C = np.cumsum(q.astype(np.uint64))
        Q = int(C[-1])
        t = (r * np.uint64(Q)) >> np.uint64(24)
        topic = np.searchsorted(C, t, side="right")  # smallest k with C_k > t
        counts = np.bincount(topic, minlength=K)
        # each topic is chosen for a share of the 2^24 values within one value of q_k / Q
        assert np.all(np.abs(counts - q.astype(np.float64) / Q * 2 ** 24) <= 1.0)
        assert np.all(counts[q == 0] == 0)
        for rr in rng.integers(0, 1 << 24, 200):
            assert oracle.lda_pick(q, int(rr)) == int(topic[rr])


def test_count_invariants_after_sweeps(oracle):
    c = inputs.lda_corpus(40, K=16, V=300, len_lo=5, len_hi=60, seed=9)
    st = inputs.lda_initial_state(c, seed=10)
    oracle.lda_full(3, 7, c, st, alpha=0.2, beta=0.05, nthreads=3)
    K, V = c["K"], c["V"]
    lengths = np.diff(c["doc_ptr"].astype(np.int64))
    doc_of = np.repeat(np.arange(lengths.size), lengths)
    assert np.array_equal(st["ndk"].sum(axis=1), lengths)
    assert np.array_equal(st["ndk"].sum(axis=0), st["nk"])
    hist = np.bincount(c["words"].astype(np.int64) * K + st["z"], minlength=V * K).reshape(V, K)
    assert np.array_equal(st["nkw"], hist)
    assert np.array_equal(st["ndk"], np.bincount(doc_of * K + st["z"], minlength=lengths.size * K).reshape(-1, K))
    assert np.array_equal(st["zpos"], 7 * lengths.astype(np.uint64))
    # theta: one Dirichlet draw per document per sweep, rows on the simplex
    assert np.allclose(st["theta"].sum(axis=1), 1.0, atol=1e-12)
    assert np.all(st["pos"][:, :, 0] > 0)


def test_single_document_posterior_marginals_brute_force(oracle):
    """One document: the topic frequencies of each token over many sweeps
    match p(z_i = k | w) from enumerating all K^L assignments."""
    K, V, alpha, beta = 2, 3, 0.5, 0.3
    words = np.array([0, 0, 1, 2, 1], dtype=np.uint32)
    c = dict(K=K, V=V, doc_ptr=np.array([0, words.size], dtype=np.uint32), words=words)
    L = words.size
    logs, confs = [], []
    for zz in itertools.product(range(K), repeat=L):
        zz = np.array(zz)
        confs.append(zz)
        logs.append(_log_joint(c["doc_ptr"], words.astype(np.int64), zz, K, V, alpha, beta))
    pz = np.exp(np.array(logs) - max(logs))
    pz /= pz.sum()
    marg = np.array([[pz[[cf[t] == k for cf in confs]].sum() for k in range(K)] for t in range(L)])
    n_batches, per = 100, 2000
    est = np.zeros((n_batches, L))
    st = inputs.lda_initial_state(c, seed=1)
    for b in range(n_batches):
        h = oracle.lda_z_run(11, per, c, st, alpha=alpha, beta=beta, zhist=True)
        est[b] = h[:, 0] / per
    mean = est.mean(axis=0)
    se = est.std(axis=0, ddof=1) / np.sqrt(n_batches)
    assert np.all(np.abs(mean - marg[:, 0]) < 5 * se + 1e-3), (mean, marg[:, 0], se)
    # the sampler is not trivially at its start: frequencies are far from 0 and 1
    assert np.all((mean > 0.05) & (mean < 0.95))


def test_threads_and_shards_exact(oracle):
    c = inputs.lda_corpus(30, K=8, V=100, len_lo=3, len_hi=40, seed=2)
    base = inputs.lda_initial_state(c, seed=3)

    def run(nthreads):
        st = {k: v.copy() for k, v in base.items()}
        d = oracle.lda_z_sweep(5, c, st, 0.1, 0.01, nthreads=nthreads)
        return st, d

    a, da = run(1)
    b, db = run(4)
    assert np.array_equal(a["z"], b["z"]) and np.array_equal(a["ndk"], b["ndk"])
    assert np.array_equal(da[0], db[0]) and np.array_equal(da[1], db[1])
    # documents [0, 12) and [12, 30) as two shards against the same snapshot
    parts = []
    for lo, hi in [(0, 12), (12, 30)]:
        sub = dict(K=c["K"], V=c["V"], doc_ptr=c["doc_ptr"][lo:hi + 1], words=c["words"])
        st = {k: v.copy() for k, v in base.items()}
        st["ndk"] = np.ascontiguousarray(st["ndk"][lo:hi])
        st["zpos"] = np.ascontiguousarray(st["zpos"][lo:hi])
        parts.append((st, oracle.lda_z_sweep(5, sub, st, 0.1, 0.01, doc_offset=lo)))
    t0, t1 = int(c["doc_ptr"][12]), int(c["doc_ptr"][30])
    assert np.array_equal(parts[0][0]["z"][:t0], a["z"][:t0]) and np.array_equal(parts[1][0]["z"][t0:t1], a["z"][t0:t1])
    assert np.array_equal(np.concatenate([parts[0][0]["ndk"], parts[1][0]["ndk"]]), a["ndk"])
    assert np.array_equal(parts[0][1][0] + parts[1][1][0], da[0])
    assert np.array_equal(parts[0][1][1] + parts[1][1][1], da[1])
