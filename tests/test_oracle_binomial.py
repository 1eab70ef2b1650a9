"""Pins of the oracle's Binomial draws (the second discrete distribution
from the same U buffer).

* the inversion equals the smallest k with u < F(k) for the exact Binomial
  CDF of q = min(p, 1 - p) (60-digit arithmetic), reflected to n - k when
  p > 1/2, on a grid of (n, p) and 24-bit u's;
* goodness of fit against scipy's pmf, mean and variance, a randomised PIT
  with per-draw (n, p); special cases n = 0, p = 0, p = 1; one U per valid
  draw; invalid parameters -> NaN with nothing consumed; mixed tag 7 equal
  to the single-distribution call.
"""
import math

import numpy as np
import pytest

import oracle as O

stats = pytest.importorskip("scipy.stats")
mpmath = pytest.importorskip("mpmath")


def _exact_cdf(n, p, kmax):
    """Binomial(n, q) CDF steps F(0..kmax), q = min(p, 1-p), in 60-digit
    arithmetic (q is the float's exact value), and whether to reflect."""
    mpmath.mp.dps = 60
    p = mpmath.mpf(p)
    flip = p > mpmath.mpf(1) / 2
    q = 1 - p if flip else p
    F, out = mpmath.mpf(0), []
    for k in range(min(n, kmax) + 1):
        F += mpmath.binomial(n, k) * q ** k * (1 - q) ** (n - k)
        out.append(F)
    return out, flip


def _exact(cdf, flip, n, u):
    """Smallest k with u < F(k), and the distance of u to the nearest step."""
    u = mpmath.mpf(u)
    prev = mpmath.mpf(0)
    for k, F in enumerate(cdf):
        if u < F:
            gap = min(abs(F - u), abs(u - prev))
            return (n - k if flip else k), float(gap)
        prev = F
    return None, 0.0


@pytest.mark.parametrize("n,p", [(1, 0.5), (10, 0.3), (10, 0.7), (40, 0.5), (1000, 0.01),
                                 (1000, 0.99), (100000, 0.0002), (7, 1.0), (7, 0.0)])
def test_inversion_matches_exact_cdf(n, p):
    p = float(np.float32(p))
    rng = np.random.default_rng(n + 3)
    us = (rng.integers(0, 1 << 24, 120) * 2.0 ** -24).tolist() + [0.0, 1.0 - 2.0 ** -24]
    cdf, flip = _exact_cdf(n, p, int(n * min(p, 1 - p) + 40 * math.sqrt(n * min(p, 1 - p) + 1) + 40))
    for u in us:
        k, gap = _exact(cdf, flip, n, u)
        assert k is not None
        got = O.binomial_inv(n, p, u)
        if got != k:  # only a u within FP64 rounding of a CDF step may differ
            assert gap < 1e-12, (n, p, u, got, k)


@pytest.mark.parametrize("n,p", [(1, 0.5), (20, 0.25), (20, 0.9), (128, 0.5), (5000, 0.004)])
def test_goodness_of_fit(n, p):
    p = float(np.float32(p))
    N, S = 200_000, 1000
    out, words, pos, st = O.binomial(13, S, np.full(N, n, np.float32), np.full(N, p, np.float32))
    assert st == O.OK
    x = out.astype(np.int64)
    assert np.all(out == x) and x.min() >= 0 and x.max() <= n
    k = np.arange(n + 1)
    e = stats.binom.pmf(k, n, p) * N
    o = np.bincount(x, minlength=n + 1)
    keep = e >= 5
    lo, hi = np.argmax(keep), len(keep) - np.argmax(keep[::-1])
    E = np.concatenate([[e[:lo].sum()], e[lo:hi], [e[hi:].sum()]])
    Obs = np.concatenate([[o[:lo].sum()], o[lo:hi], [o[hi:].sum()]])
    m = E > 0
    chi2 = ((Obs[m] - E[m]) ** 2 / E[m]).sum()
    assert stats.chi2.sf(chi2, max(1, m.sum() - 1)) > 1e-4, (n, p, chi2)
    mean, var = n * p, n * p * (1 - p)
    assert abs(x.mean() - mean) < 5 * math.sqrt(var / N) + 1e-12


def test_varying_parameters_randomised_pit():
    N, S = 200_000, 4096
    rng = np.random.default_rng(6)
    n = rng.integers(0, 200, N).astype(np.float32)
    p = rng.random(N).astype(np.float32)
    mean = n * np.minimum(p, 1 - p)
    p = np.where(mean > 64.0, np.float32(0.3), p).astype(np.float32)
    out, words, pos, st = O.binomial(4, S, n, p)
    assert st == O.OK
    k = out.astype(np.int64)
    lo = stats.binom.cdf(k - 1, n.astype(np.int64), p.astype(np.float64))
    pk = stats.binom.pmf(k, n.astype(np.int64), p.astype(np.float64))
    pit = lo + rng.random(N) * pk
    assert stats.kstest(pit, "uniform").pvalue > 1e-4


def test_special_cases_words_and_consumption():
    S, N = 5, 500
    rng = np.random.default_rng(2)
    n = rng.integers(0, 60, N).astype(np.float32)
    p = rng.random(N).astype(np.float32)
    n[:5], p[:5] = 0.0, 0.5          # n = 0 -> 0
    n[5:10], p[5:10] = 9.0, 0.0      # p = 0 -> 0
    n[10:15], p[10:15] = 9.0, 1.0    # p = 1 -> n
    out, words, pos, st = O.binomial(31, S, n, p)
    assert st == O.OK
    assert np.all(out[:10] == 0) and np.all(out[10:15] == 9)
    for s in range(S):
        idx = np.arange(s, N, S)
        vals, w = O.elements(31, O.DOM_U, s, 0, idx.size)
        assert np.array_equal(words[idx], w)  # one U element per draw, in order
        for i, u in zip(idx[:15], vals[:15]):
            assert out[i] == O.binomial_inv(float(n[i]), float(p[i]), float(u))


def test_invalid_parameters_consume_nothing():
    n = np.array([10, 2.5, -1, np.nan, 10, 10, 10, 2.0e7, 10], np.float32)
    p = np.array([0.5, 0.5, 0.5, 0.5, -0.1, 1.5, np.nan, 0.5, 0.25], np.float32)
    out, words, pos, st = O.binomial(2, 1, n, p)
    assert st == O.EDOMAIN
    assert np.isnan(out[1:8]).all() and np.all(words[1:8] == 0)
    ok, _, pos_ok, _ = O.binomial(2, 1, n[[0, 8]], p[[0, 8]])
    assert out[0] == ok[0] and out[8] == ok[1] and np.array_equal(pos, pos_ok)


def test_mixed_tag_seven_equals_single_call():
    N, S = 5000, 64
    rng = np.random.default_rng(8)
    n = rng.integers(0, 100, N).astype(np.float32)
    p = rng.random(N).astype(np.float32) * 0.5
    single, sw, spos, _ = O.binomial(8, S, n, p)
    mixed, mw, mpos, _ = O.mixed(8, S, np.full(N, 7, np.uint8), n, p)
    assert np.array_equal(single, mixed) and np.array_equal(sw, mw) and np.array_equal(spos, mpos)
