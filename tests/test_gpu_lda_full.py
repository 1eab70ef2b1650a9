"""Parity of the full LDA step (topic draws per token, then theta) on the GPU
with the oracle.

Bars: every topic assignment, every count table (document-topic, word-topic,
topic totals) and every stream position bit-exact -- the draw is decided by
integer arithmetic on FP32 weights both sides compute with the same IEEE
operations -- and theta (FP32) within the Dirichlet bound of the parity tests
(per draw, and summed over the sweeps for the moments).
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1412_4825_gb300 import inputs

import gibbs_bounds

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_4825_gb300 import brng as B  # noqa: E402

NT = os.cpu_count() or 1
RTOL = 2e-6
FLT_MIN = float(np.finfo(np.float32).tiny)
SEED = 42


def _prev_host(corpus):
    """For each token: the previous token of its document with the same word."""
    doc_ptr, words = corpus["doc_ptr"].astype(np.int64), corpus["words"]
    prev = np.full(words.size, B.LDA_NONE, dtype=np.uint32)
    for d in range(doc_ptr.size - 1):
        last = {}
        for t in range(doc_ptr[d], doc_ptr[d + 1]):
            w = int(words[t])
            if w in last:
                prev[t] = last[w]
            last[w] = t
    return prev


def _check(g, ref, what, theta=True):
    for key in ("z", "ndk", "nkw", "nk", "zpos"):
        a, b = g[key], ref[key]
        assert np.array_equal(a.astype(np.int64), b.astype(np.int64)), "%s: %s differs (%d entries)" % (
            what, key, int((a.astype(np.int64) != b.astype(np.int64)).sum()))
    assert not g["dnkw"].any()  # the changes were applied and cleared
    if not theta:
        return
    assert np.array_equal(g["pos"], ref["pos"]), what + ": Dirichlet positions"
    th, scale = gibbs_bounds.dirichlet_scale(ref["logs"], ref["cond"])
    err = np.abs(g["theta"].astype(np.float64) - ref["theta"])
    bound = RTOL * scale + 2 * FLT_MIN
    print("%s theta: max err/bound = %.3g" % (what, np.max(err / bound)))
    assert np.all(err <= bound)
    mb = gibbs_bounds.lda_mom_bound(ref["trace"], RTOL) + 2 * FLT_MIN
    merr = np.abs(g["mom"] - ref["mom"])
    print("%s sum theta: max err/bound = %.3g" % (what, np.max(merr / mb)))
    assert np.all(merr <= mb)


def _run_pair(corpus, n_sweeps, alpha=0.1, beta=0.01, seed_state=7, calls=None, buf_len=0, doc_offset=0):
    st0 = inputs.lda_initial_state(corpus, seed=seed_state)
    m = B.LdaFull(corpus, st0, alpha=alpha, beta=beta)
    h = B.Handle(SEED, 1, buf_len)
    for n in (calls or [n_sweeps]):
        m.run(h, n, doc_offset=doc_offset)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    g = m.host()
    ref = {k: v.copy() for k, v in st0.items()}
    O.lda_full(SEED, n_sweeps, corpus, ref, alpha=alpha, beta=beta, doc_offset=doc_offset, nthreads=NT,
               trace=True)
    h.close()
    return g, ref


def test_index_links_match_host():
    c = inputs.lda_corpus(200, K=8, V=40, len_lo=1, len_hi=300, seed=1)
    st = inputs.lda_initial_state(c, seed=2)
    m = B.LdaFull(c, st)
    torch.cuda.synchronize()
    assert np.array_equal(m.host()["prev"], _prev_host(c))


@pytest.mark.parametrize("K,V", [(64, 512), (5, 50), (17, 300), (32, 1000), (100, 200), (128, 64), (1, 10)])
def test_lda_full_bit_exact(K, V):
    """Small vocabularies: many repeated words per document, so the walks over
    the document's own changes are exercised; K spans one to four topics per
    lane and ragged lane counts."""
    c = inputs.lda_corpus(301, K=K, V=V, len_lo=1, len_hi=400, seed=K + V)
    g, ref = _run_pair(c, 6, alpha=0.1, beta=0.01)
    _check(g, ref, "K=%d V=%d" % (K, V))


def test_lda_full_priors_offset_and_split_calls():
    c = inputs.lda_corpus(150, K=64, V=700, seed=3)
    g, ref = _run_pair(c, 5, alpha=0.7, beta=0.3, calls=[2, 1, 2], buf_len=8, doc_offset=1000)
    _check(g, ref, "priors 0.7/0.3, offset 1000, calls 2+1+2")


def test_lda_full_one_long_document():
    """One document of 3,000 tokens over 20 words: long chains of earlier
    tokens with the same word (the sequential collapsed sampler exactly)."""
    rng = np.random.default_rng(4)
    words = rng.integers(0, 20, 3000).astype(np.uint32)
    c = dict(K=12, V=20, doc_ptr=np.array([0, words.size], dtype=np.uint32), words=words)
    g, ref = _run_pair(c, 4, alpha=0.5, beta=0.1)
    _check(g, ref, "one document")


def test_lda_full_exchange_mode_equals_internal_apply():
    """exchange = 1 leaves each sweep's count changes for the caller (to sum
    across devices); applying them with brng_lda_apply gives the same run."""
    c = inputs.lda_corpus(120, K=64, V=900, seed=5)
    st0 = inputs.lda_initial_state(c, seed=6)
    a = B.LdaFull(c, st0)
    b = B.LdaFull(c, st0)
    ha, hb = B.Handle(SEED, 1), B.Handle(SEED, 1)
    a.run(ha, 3)
    for _ in range(3):
        b.run(hb, 1, exchange=1)
        assert b.dnkw.abs().sum().item() > 0
        B.brng_lda_apply(b.K, b.V, b.nkw, b.nk, b.dnkw)
    ga, gb = a.host(), b.host()
    for key in ("z", "ndk", "nkw", "nk", "zpos", "pos", "theta", "mom"):
        assert np.array_equal(ga[key], gb[key]), key
    with pytest.raises(B.BrngError):
        b.run(hb, 2, exchange=1)


def test_lda_full_full_size_sampled():
    """16,384 documents, K = 64, V = 4,096, lengths U{50..500} (4.5 M tokens):
    three sweeps; every assignment and count bit-exact, theta within bound."""
    c = inputs.lda_corpus(16384, K=64, V=4096, seed=SEED)
    g, ref = _run_pair(c, 3)
    _check(g, ref, "16384 docs")


def test_lda_full_document_order_changes_nothing():
    """The documents' start order (longest first by default, the identity, a
    random permutation) is speed only: every output is bit-identical."""
    c = inputs.lda_corpus(300, K=16, V=200, len_lo=5, len_hi=400, seed=21)
    st0 = inputs.lda_initial_state(c, seed=22)
    outs = []
    for mode in ("longest", "identity", "random"):
        m = B.LdaFull(c, st0)
        if mode == "random":
            perm = np.random.default_rng(5).permutation(m.n_docs).astype(np.uint32)
            m.order = torch.from_numpy(perm.view(np.int32)).to(m.order.device)
        h = B.Handle(SEED, 1)
        m.run(h, 3, ordered=(mode != "identity"))
        code, cnt = h.counters()
        assert code == B.BRNG_OK, cnt
        outs.append(m.host())
        h.close()
    for other in outs[1:]:
        for key in ("z", "ndk", "nkw", "nk", "zpos", "pos", "theta", "mom"):
            assert np.array_equal(outs[0][key], other[key]), key


def test_lda_full_run_with_a_handle_made_in_the_call():
    """A Handle created in the argument list stays alive for the whole call
    (the binding must not drop its last reference before the library runs)."""
    c = inputs.lda_corpus(50, K=8, V=64, len_lo=5, len_hi=40, seed=31)
    st0 = inputs.lda_initial_state(c, seed=32)
    m = B.LdaFull(c, st0)
    m.run(B.Handle(SEED, 1), 2)
    ref = {k: v.copy() for k, v in st0.items()}
    O.lda_full(SEED, 2, c, ref, alpha=0.1, beta=0.01, nthreads=NT)
    g = m.host()
    for key in ("z", "ndk", "nkw", "nk", "zpos"):
        assert np.array_equal(g[key].astype(np.int64), ref[key].astype(np.int64)), key
