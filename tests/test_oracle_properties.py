"""Randomised properties of the oracle's buffer semantics (Sec. 2.2: values
never depend on buffer_length, and the buffer counters persist across calls),
for every bulk distribution and the mixed stream, over random seeds, stream
counts, draw counts, buffer lengths, parameters (invalid ones included) and
split points: one call equals two chained calls with the positions carried,
and equals the same call with another buffer length -- values, words and
positions alike."""
import numpy as np
import pytest

import oracle as O

hyp = pytest.importorskip("hypothesis")
st = pytest.importorskip("hypothesis.strategies")

FNS = {
    "uniform": lambda rng, n: [np.sort(rng.uniform(-5, 5, (2, n)), axis=0)[0], None],
    "normal": lambda rng, n: [rng.uniform(-5, 5, n), rng.uniform(0.01, 5, n)],
    "exponential": lambda rng, n: [rng.uniform(0.01, 5, n)],
    "gamma": lambda rng, n: [np.exp(rng.uniform(np.log(0.05), np.log(60.0), n))],
    "laplace": lambda rng, n: [rng.uniform(-5, 5, n), rng.uniform(0.01, 5, n)],
    "weibull": lambda rng, n: [rng.uniform(0.3, 5, n), rng.uniform(0.01, 5, n)],
    "poisson": lambda rng, n: [rng.uniform(0.01, 64.0, n)],
    "binomial": lambda rng, n: [np.floor(rng.uniform(0, 60, n)), rng.uniform(0, 1, n)],
}


def _params(fn, rng, n):
    ps = FNS[fn](rng, n)
    if fn == "uniform":  # a <= b
        b = ps[0] + rng.uniform(0, 3, n)
        ps = [ps[0], b]
    ps = [np.asarray(p, dtype=np.float32) for p in ps]
    bad = rng.random(n) < 0.05  # a few invalid parameters: NaN, consume nothing
    ps[0] = np.where(bad, np.float32(np.nan), ps[0]).astype(np.float32)
    return ps


@hyp.settings(max_examples=40, deadline=None)
@hyp.given(fn=st.sampled_from(sorted(FNS)), seed=st.integers(0, 2**64 - 1), S=st.integers(1, 40),
           n=st.integers(0, 600), cut=st.floats(0.0, 1.0), L=st.sampled_from([1, 2, 3, 5, 8, 64, 1000]),
           pseed=st.integers(0, 10**6))
def test_split_and_buffer_length_invariance(fn, seed, S, n, cut, L, pseed):
    rng = np.random.default_rng(pseed)
    ps = _params(fn, rng, n)
    call = getattr(O, fn)
    whole = call(seed, S, *ps, buf_len=64)
    other = call(seed, S, *ps, buf_len=L)
    for a, b in zip(whole[:3], other[:3]):
        assert np.array_equal(a, b, equal_nan=a.dtype.kind == "f")
    k = int(cut * n) // S * S  # a multiple of S keeps draw i on stream i mod S in both parts
    first = call(seed, S, *[p[:k] for p in ps], buf_len=L)
    second = call(seed, S, *[p[k:] for p in ps], pos=first[2], buf_len=L)
    assert np.array_equal(np.concatenate([first[0], second[0]]), whole[0], equal_nan=True)
    assert np.array_equal(np.concatenate([first[1], second[1]]), whole[1])
    assert np.array_equal(second[2], whole[2])


@hyp.settings(max_examples=25, deadline=None)
@hyp.given(seed=st.integers(0, 2**64 - 1), S=st.integers(1, 50), n=st.integers(0, 800),
           n_tags=st.sampled_from([4, 6, 8]), L=st.sampled_from([1, 4, 7, 64]), pseed=st.integers(0, 10**6))
def test_mixed_stream_equals_its_single_distribution_calls(seed, S, n, n_tags, L, pseed):
    """The mixed stream with one tag everywhere is that distribution's call,
    and any mix is invariant to the buffer length."""
    from paper_1412_4825_gb300 import inputs
    tag, p0, p1 = inputs.mixed_stream(n, seed=pseed % 1000, n_tags=n_tags)
    a = O.mixed(seed, S, tag, p0, p1, buf_len=64)
    b = O.mixed(seed, S, tag, p0, p1, buf_len=L)
    for x, y in zip(a[:3], b[:3]):
        assert np.array_equal(x, y, equal_nan=x.dtype.kind == "f")
    lam = np.abs(p0).astype(np.float32) % np.float32(60.0) + np.float32(0.01)
    single = O.poisson(seed, S, lam, buf_len=L)
    mixed = O.mixed(seed, S, np.full(n, 6, np.uint8), lam, np.zeros(n, np.float32), buf_len=L)
    for x, y in zip(single[:3], mixed[:3]):
        assert np.array_equal(x, y, equal_nan=x.dtype.kind == "f")


@hyp.settings(max_examples=30, deadline=None)
@hyp.given(model=st.sampled_from([0, 1, 2]), n=st.integers(1, 30), sweeps=st.integers(1, 50),
           cut=st.floats(0.0, 1.0), shard=st.floats(0.0, 1.0), L=st.sampled_from([1, 3, 8, 64, 256]),
           seed=st.integers(0, 2**64 - 1), offset=st.integers(0, 10**6))
def test_gibbs_resume_shard_and_buffer_length(model, n, sweeps, cut, shard, L, seed, offset):
    """Each Gibbs model: a run split in two with the state carried equals one
    run, chain (document) ranges run separately equal one run over all of
    them, and the buffer length changes nothing -- states, positions and
    moments bit for bit."""
    from paper_1412_4825_gb300 import inputs
    s1, k = int(cut * sweeps), int(shard * n)

    def run(lo, hi, nsw, start=None, L_=L):
        if model == 0:
            kw = {} if start is None else dict(xy=start["xy"].ravel(), pos=start["pos"], mom=start["mom"].ravel())
            r = O.gibbs_triangle(seed, hi - lo, nsw, chain_offset=offset + lo, buf_len=L_, **kw)
            return r, (r["xy"], r["pos"], r["mom"])
        if model == 1:
            nobs, xbar, sc = (a[lo:hi] for a in inputs.normal_gamma_data(n, seed=7))
            kw = {} if start is None else dict(state=start["state"].ravel(), pos=start["pos"].ravel(),
                                               mom=start["mom"].ravel())
            r = O.gibbs_normal_gamma(seed, nsw, nobs, xbar, sc, chain_offset=offset + lo, buf_len=L_, **kw)
            return r, (r["state"], r["pos"], r["mom"])
        alpha = inputs.lda_alpha(n, K=12, seed=7)[0][lo:hi]
        kw = {} if start is None else dict(pos=start["pos"].ravel(), mom=start["mom"])
        r = O.gibbs_lda(seed, nsw, alpha, doc_offset=offset + lo, buf_len=L_, **kw)
        return r, (r["theta"] if nsw else None, r["pos"], r["mom"])

    whole, w = run(0, n, sweeps, L_=64)
    first, _ = run(0, n, s1)
    _, resumed = run(0, n, sweeps - s1, start=first)
    for a, b in zip(w[1:], resumed[1:]):
        assert np.array_equal(a, b)
    if model != 2 or sweeps - s1 > 0:  # LDA's theta is the last sweep's
        assert np.array_equal(w[0], resumed[0])
    parts = [run(lo, hi, sweeps)[1] for lo, hi in ((0, k), (k, n)) if hi > lo]
    for j in range(3):
        assert np.array_equal(np.concatenate([p[j] for p in parts]), w[j])
