"""Pins of the oracle's Poisson draws (discrete distributions, from the same
U buffer) and of its own FP64 exp.

* exp: within 1 ulp of 50-digit mpmath over [-708, 0], exact at 0;
* the inversion: the oracle's k is the smallest k with u < F(k) for the exact
  Poisson CDF (50-digit arithmetic), on a grid of lambdas and 24-bit u's;
* the bulk stream: goodness of fit against scipy's Poisson pmf, mean and
  variance, a randomised PIT with per-draw lambda, one U per draw (word and
  position), invalid lambda -> NaN with nothing consumed, and the mixed
  stream's tag 6 equal to the single-distribution call.
"""
import math

import numpy as np
import pytest

import oracle as O

mpmath = pytest.importorskip("mpmath")
stats = pytest.importorskip("scipy.stats")


def ulp(x):
    return np.spacing(np.abs(x))


def test_exp_within_one_ulp():
    rng = np.random.default_rng(1)
    xs = np.concatenate([rng.uniform(-708.0, 0.0, 3000), rng.uniform(-64.0, 0.0, 3000),
                         -np.exp(rng.uniform(-40, 0, 1000)), [0.0, -1e-300, -0.5, -1.0, -64.0, -700.0]])
    got = O.exp(xs)
    mpmath.mp.dps = 50
    ref = np.array([float(mpmath.exp(mpmath.mpf(float(x)))) for x in xs])
    err = np.abs(got - ref) / ulp(ref)
    assert err.max() <= 1.0, (err.max(), xs[err.argmax()])
    assert O.exp(np.array([0.0]))[0] == 1.0
    assert np.isnan(O.exp(np.array([np.nan]))[0])


def _exact_k(lam, u):
    """Smallest k with u < F(k), F the exact Poisson(lam) CDF (50 digits)."""
    mpmath.mp.dps = 50
    lam = mpmath.mpf(lam)
    u = mpmath.mpf(u)
    p = mpmath.exp(-lam)
    F = p
    k = 0
    while not (u < F):
        k += 1
        p = p * lam / k
        F += p
    return k, float(F - u), float(u - (F - p))


@pytest.mark.parametrize("lam", [0.01, 0.5, 1.0, 4.5, 17.0, 64.0])
def test_inversion_matches_exact_cdf(lam):
    lam = float(np.float32(lam))
    rng = np.random.default_rng(int(lam * 100) + 7)
    us = (rng.integers(0, 1 << 24, 400) * 2.0 ** -24).tolist() + [0.0, 1.0 - 2.0 ** -24]
    for u in us:
        k, above, below = _exact_k(lam, u)
        got = O.poisson_inv(lam, u)
        if got != k:  # only a u within FP64 rounding of a CDF step may differ
            assert min(abs(above), abs(below)) < 1e-13, (lam, u, got, k)


def _draw(lam_value, n=200_000, S=1000, seed=11):
    lam = np.full(n, lam_value, np.float32)
    out, words, pos, st = O.poisson(seed, S, lam)
    assert st == O.OK
    return out


@pytest.mark.parametrize("lam", [0.1, 1.0, 4.5, 30.0, 64.0])
def test_goodness_of_fit(lam):
    lam32 = float(np.float32(lam))
    x = _draw(lam32)
    assert np.all(x == np.floor(x)) and x.min() >= 0
    k = np.arange(0, int(lam32 + 12 * math.sqrt(lam32) + 12))
    pmf = stats.poisson.pmf(k, lam32)
    obs = np.bincount(x.astype(np.int64), minlength=k.size)[: k.size]
    # pool bins with expected count < 5 at both ends
    exp_counts = pmf * x.size
    keep = exp_counts >= 5
    lo, hi = np.argmax(keep), len(keep) - np.argmax(keep[::-1])
    e = np.concatenate([[exp_counts[:lo].sum()], exp_counts[lo:hi], [x.size - exp_counts[:hi].sum()]])
    o = np.concatenate([[obs[:lo].sum()], obs[lo:hi], [x.size - obs[:hi].sum()]])
    m = e > 0
    chi2 = ((o[m] - e[m]) ** 2 / e[m]).sum()
    p = stats.chi2.sf(chi2, m.sum() - 1)
    assert p > 1e-4, (lam, chi2, p)
    se = math.sqrt(lam32 / x.size)
    assert abs(x.mean() - lam32) < 5 * se
    assert abs(x.var() - lam32) < 5 * lam32 * math.sqrt(2.0 / x.size) + 5 * se


def test_varying_lambda_randomised_pit():
    n, S = 200_000, 4096
    rng = np.random.default_rng(5)
    lam = np.exp(rng.uniform(np.log(0.05), np.log(64.0), n)).astype(np.float32)
    out, words, pos, st = O.poisson(3, S, lam)
    assert st == O.OK
    k = out.astype(np.int64)
    lo = stats.poisson.cdf(k - 1, lam.astype(np.float64))
    pk = stats.poisson.pmf(k, lam.astype(np.float64))
    v = rng.random(n)
    pit = lo + v * pk
    assert stats.kstest(pit, "uniform").pvalue > 1e-4


def test_one_uniform_per_draw_and_words():
    S, n = 7, 700
    rng = np.random.default_rng(9)
    lam = rng.uniform(0.1, 64.0, n).astype(np.float32)
    out, words, pos, st = O.poisson(21, S, lam)
    assert st == O.OK
    for s in range(S):
        idx = np.arange(s, n, S)
        vals, w = O.elements(21, O.DOM_U, s, 0, idx.size)
        assert np.array_equal(words[idx], w)  # draw m of stream s consumed U element m
        for i, u in zip(idx[:20], vals[:20]):
            assert out[i] == O.poisson_inv(float(lam[i]), float(u))
    assert np.array_equal(pos.reshape(S, 3)[:, 0], [len(range(s, n, S)) for s in range(S)])
    assert np.all(pos.reshape(S, 3)[:, 1:] == 0)


def test_invalid_lambda_consumes_nothing():
    lam = np.array([1.0, 0.0, -2.0, np.nan, np.inf, 2.0e7, 3.0], np.float32)
    out, words, pos, st = O.poisson(2, 1, lam)
    assert st == O.EDOMAIN
    assert np.isnan(out[1:6]).all() and np.all(words[1:6] == 0)
    ok, _, pos_ok, _ = O.poisson(2, 1, lam[[0, 6]])
    assert out[0] == ok[0] and out[6] == ok[1]
    assert np.array_equal(pos, pos_ok)


def test_mixed_tag_six_equals_single_call():
    n, S = 5000, 64
    rng = np.random.default_rng(4)
    lam = rng.uniform(0.1, 40.0, n).astype(np.float32)
    single, sw, spos, _ = O.poisson(8, S, lam)
    tag = np.full(n, 6, np.uint8)
    mixed, mw, mpos, _ = O.mixed(8, S, tag, lam, np.zeros(n, np.float32))
    assert np.array_equal(single, mixed) and np.array_equal(sw, mw) and np.array_equal(spos, mpos)
