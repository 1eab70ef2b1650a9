"""Pins of the oracle's large-mean discrete samplers: Poisson by PTRS and
Binomial by BTRD (Hormann 1993, transformed rejection), used above mean 64.

* ln k! (the rejection tests' only special function) against 40-digit
  arithmetic for k up to 2^24.
* The samples follow the exact distribution: a chi-square test on bins of
  near-equal exact probability (scipy's regularised incomplete Gamma / Beta
  CDFs, accurate to ~1e-14, far below the test's resolution) at means from
  just above 64 to 10^6, and the first two moments within 5 standard errors.
* The stream bookkeeping: the first consumed word is reported, the mixed
  stream's tags 6 and 7 equal the single-distribution calls, and means on
  both sides of 64 switch between inversion and rejection as documented.
"""
import numpy as np
import pytest
from scipy import stats

from paper_1412_4825_gb300 import inputs


def test_lfact_against_high_precision(oracle):
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    ks = list(range(0, 64)) + [100, 1000, 12345, 10 ** 6, 10 ** 7, 2 ** 24 - 1]
    for k in ks:
        want = float(mp.loggamma(k + 1))
        got = oracle.lfact(k)
        assert abs(got - want) <= 4e-16 * max(1.0, abs(want)), (k, got, want)


def _chi2_pvalue(samples, cdf, n_bins=40):
    """Chi-square goodness of fit on integer bins cut at the exact
    distribution's quantiles."""
    lo, hi = samples.min(), samples.max()
    grid = np.arange(lo - 1, hi + 2)
    c = cdf(grid)
    edges = [grid[0]]
    targets = np.linspace(0, 1, n_bins + 1)[1:-1]
    for t in targets:
        k = grid[np.searchsorted(c, t)]
        if k > edges[-1]:
            edges.append(k)
    edges.append(grid[-1] + 1)
    edges = np.array(edges)
    obs = np.histogram(samples, bins=np.concatenate([[-np.inf], edges[1:-1] + 0.5, [np.inf]]))[0]
    probs = np.diff(np.concatenate([[0.0], cdf(edges[1:-1]), [1.0]]))
    exp = probs * samples.size
    keep = exp > 5
    chi2 = ((obs[keep] - exp[keep]) ** 2 / exp[keep]).sum()
    dof = keep.sum() - 1
    return stats.chi2.sf(chi2, dof)


@pytest.mark.parametrize("lam", [64.5, 100.0, 777.0, 1e4, 1e5, 1e6])
def test_poisson_ptrs_matches_exact_distribution(oracle, lam):
    n, S = 200000, 1000
    lam_arr = np.full(n, lam, np.float32)
    out, words, pos, st = oracle.poisson(int(lam) + 3, S, lam_arr)
    assert st == oracle.OK and not np.isnan(out).any()
    x = out.astype(np.int64)
    lam32 = float(np.float32(lam))
    p = _chi2_pvalue(x, lambda k: stats.poisson.cdf(k, lam32))
    assert p > 1e-4, p
    se_mean = np.sqrt(lam32 / n)
    assert abs(x.mean() - lam32) < 5 * se_mean
    # variance: SE of the sample variance ~ sqrt((mu4 - sigma^4)/n), mu4 = 3 lam^2 + lam
    se_var = np.sqrt((2 * lam32 ** 2 + lam32) / n)
    assert abs(x.var() - lam32) < 5 * se_var
    # 2 uniforms per attempt: consumption is even and about 2 per draw
    used = pos.reshape(S, 3)[:, 0]
    assert np.all(used % 2 == 0) and 2.0 <= used.sum() / n < 2.6


@pytest.mark.parametrize("trials,prob", [(1000, 0.3), (100000, 0.01), (2 ** 24, 0.5), (500, 0.9),
                                          (130, 0.5), (3000, 0.97)])
def test_binomial_btrd_matches_exact_distribution(oracle, trials, prob):
    n, S = 200000, 1000
    t = np.full(n, trials, np.float32)
    p = np.full(n, prob, np.float32)
    out, words, pos, st = oracle.binomial(trials % 97 + 5, S, t, p)
    assert st == oracle.OK and not np.isnan(out).any()
    x = out.astype(np.int64)
    p32 = float(np.float32(prob))
    pv = _chi2_pvalue(x, lambda k: stats.binom.cdf(k, trials, p32))
    assert pv > 1e-4, pv
    mean, var = trials * p32, trials * p32 * (1 - p32)
    assert abs(x.mean() - mean) < 5 * np.sqrt(var / n)
    assert abs(x.var() - var) < 5 * np.sqrt((2 * var ** 2 + var) / n) + 1e-9
    assert x.min() >= 0 and x.max() <= trials


def test_switch_at_mean_64_and_words(oracle):
    """Means up to 64 take one uniform per draw (inversion); above, the first
    word of each draw is its first attempt's uniform."""
    S = 3
    lam = np.array([64.0, 64.5, 63.9, 500.0, 1e6, 10.0], np.float32)
    out, words, pos, st = oracle.poisson(5, S, lam)
    assert st == oracle.OK
    # stream 0 draws: 64.0 (inversion: 1 U), then 500 (PTRS: 2 per attempt)
    vals, w = oracle.elements(5, oracle.DOM_U, 0, 0, 1)
    assert words[0] == w[0] and out[0] == oracle.poisson_inv(64.0, float(vals[0]))
    _, w = oracle.elements(5, oracle.DOM_U, 0, 1, 1)
    assert words[3] == w[0]
    assert (pos.reshape(S, 3)[0, 0] - 1) % 2 == 0
    trials = np.array([128, 129, 1000], np.float32)
    prob = np.array([0.5, 0.5, 0.06], np.float32)  # means 64 (inversion), 64.5, 60 (inversion)
    out, words, pos, st = oracle.binomial(6, 1, trials, prob)
    assert st == oracle.OK
    vals, w = oracle.elements(6, oracle.DOM_U, 0, 0, 1)
    assert out[0] == oracle.binomial_inv(128.0, 0.5, float(vals[0])) and words[0] == w[0]


def test_mixed_tags_large_means_equal_single_calls(oracle):
    n, S = 6000, 50
    rng = np.random.default_rng(12)
    lam = inputs.log_uniform(rng, 0.05, 1e6, n)
    single, sw, spos, _ = oracle.poisson(8, S, lam)
    mixed, mw, mpos, _ = oracle.mixed(8, S, np.full(n, 6, np.uint8), lam, np.zeros(n, np.float32))
    assert np.array_equal(single, mixed) and np.array_equal(sw, mw) and np.array_equal(spos, mpos)
    trials = np.floor(inputs.log_uniform(rng, 1.0, 1.6e7, n)).astype(np.float32)
    prob = rng.random(n).astype(np.float32)
    single, sw, spos, _ = oracle.binomial(9, S, trials, prob)
    mixed, mw, mpos, _ = oracle.mixed(9, S, np.full(n, 7, np.uint8), trials, prob)
    assert np.array_equal(single, mixed) and np.array_equal(sw, mw) and np.array_equal(spos, mpos)
    assert np.all((single >= 0) & (single <= trials))
