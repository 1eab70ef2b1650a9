"""Pins of the oracle's varying-parameter distributions (Sec. 2.1-2.2).

Distribution pins: Kolmogorov-Smirnov against scipy at fixed parameters,
probability-integral-transform KS for per-draw parameters, closed-form
moments, the special case Gamma(1) = Exp(1), and Dirichlet invariants.  Buffer
semantics pins (Sec. 2.2): every value is independent of buffer_length and of
how draws are split across calls; consumption is sequential with no skips.
"""
import mpmath as mp
import numpy as np
import pytest
from scipy import stats

from paper_1412_4825_gb300 import inputs

KS_P = 1e-4  # a correct sampler fails one KS test with probability 1e-4


def _const(n, v):
    return np.full(n, v, dtype=np.float32)


def test_uniform_ks(oracle):
    n = 200000
    out, words, pos, st = oracle.uniform(1, 64, _const(n, -2.0), _const(n, 3.0))
    assert st == 0
    assert stats.kstest(out, stats.uniform(-2.0, 5.0).cdf).pvalue > KS_P
    assert out.min() >= -2.0 and out.max() < 3.0


def test_normal_ks_and_moments(oracle):
    n = 200000
    out, _, _, st = oracle.normal(2, 128, _const(n, 1.5), _const(n, 2.0))
    assert st == 0
    assert stats.kstest(out, stats.norm(1.5, 2.0).cdf).pvalue > KS_P
    assert abs(out.mean() - 1.5) < 5 * 2.0 / np.sqrt(n)
    assert abs(out.var() - 4.0) < 5 * 4.0 * np.sqrt(2.0 / n)


def test_gaussian_pairs_uncorrelated(oracle):
    vals, _ = oracle.elements(3, 1, 0, 0, 400000)
    z0, z1 = vals[0::2], vals[1::2]  # cos and sin halves of each Box-Muller pair
    assert abs(np.corrcoef(z0, z1)[0, 1]) < 5 / np.sqrt(z0.size)
    assert abs(np.corrcoef(z0 ** 2, z1 ** 2)[0, 1]) < 5 / np.sqrt(z0.size)


def test_exponential_ks(oracle):
    n = 200000
    out, _, _, st = oracle.exponential(3, 64, _const(n, 0.5))
    assert st == 0
    assert stats.kstest(out, stats.expon(scale=2.0).cdf).pvalue > KS_P


@pytest.mark.parametrize("alpha", [0.05, 0.1, 0.5, 1.0, 1.1, 5.2, 52.0, 500.0])
def test_gamma_ks_and_moments(oracle, alpha):
    n = 100000
    out, _, pos, st = oracle.gamma(4, 100, _const(n, alpha))
    assert st == 0
    assert stats.kstest(out, stats.gamma(alpha).cdf).pvalue > KS_P
    assert abs(out.mean() - alpha) < 5 * np.sqrt(alpha / n)
    # acceptance: N elements consumed per draw = attempts (Marsaglia-Tsang
    # accepts with probability > 0.95 for every shape >= 1)
    attempts = pos.reshape(-1, 3)[:, 1].sum() / n
    assert 1.0 <= attempts < 1.06


def test_gamma_one_is_exponential(oracle):
    n = 100000
    out, _, _, _ = oracle.gamma(5, 64, _const(n, 1.0))
    assert stats.kstest(out, stats.expon().cdf).pvalue > KS_P


def test_gamma_varying_parameters_pit(oracle):
    n = 100000
    alpha = inputs.shape_params(n, seed=6)
    out, _, _, st = oracle.gamma(6, 1000, alpha)
    assert st == 0
    pit = stats.gamma.cdf(out, alpha.astype(np.float64))
    assert stats.kstest(pit, "uniform").pvalue > KS_P


def test_mt_accept_against_exact_arithmetic(oracle):
    """The FP64 acceptance test equals the exact one except within 1e-12 of
    the boundary."""
    mp.mp.prec = 100
    rng = np.random.default_rng(8)
    checked = 0
    for _ in range(3000):
        alpha = float(np.exp(rng.uniform(np.log(0.05), np.log(500.0))))
        z = float(rng.normal())
        u = float((rng.integers(0, 1 << 24) + 1) * 2.0**-24)
        got = oracle.mt_accept(alpha, z, u)
        a = mp.mpf(alpha) + (1 if alpha < 1 else 0)
        d = a - mp.mpf(1) / 3
        c = 1 / mp.sqrt(9 * d)
        t = 1 + c * z
        if t <= 0:
            assert got == -1
            continue
        v = t ** 3
        margin = mp.mpf(z) ** 2 / 2 + d * (1 - v + mp.log(v)) - mp.log(u)
        if abs(margin) > 1e-12 * (1 + d):
            assert got == (1 if margin > 0 else 0)
            checked += 1
    assert checked > 2500


def test_mt_squeeze_implies_accept(oracle):
    """Marsaglia & Tsang's squeeze, as the GPU takes it (u' + 0.0331 (1 + 1e-5)
    z^4 < 1 - 2^-22), is a sufficient condition of the exact accept test for
    every shape a >= 1 (boosted shapes included): checked in 100-bit
    arithmetic and against the oracle's FP64 test, with z drawn over the
    squeeze's whole range and near 0, where its slack is smallest."""
    mp.mp.prec = 100
    rng = np.random.default_rng(21)
    zmax = (1 / 0.0331) ** 0.25
    passed = 0
    for i in range(4000):
        alpha = float(np.exp(rng.uniform(np.log(0.01), np.log(2e4))))
        z = float(rng.uniform(-zmax, zmax)) if i % 4 else float(rng.normal() * 1e-2)
        bound = 1.0 - 0.0331 * 1.00001 * z ** 4 - 2.0 ** -22
        if bound <= 2.0 ** -24:
            continue
        u = float(rng.integers(1, int(bound * 2**24) + 1) * 2.0 ** -24)  # u' < bound on the 24-bit grid
        a = mp.mpf(alpha) + (1 if alpha < 1 else 0)
        d = a - mp.mpf(1) / 3
        t = 1 + z / mp.sqrt(9 * d)
        assert t > 0
        v = t ** 3
        margin = mp.mpf(z) ** 2 / 2 + d * (1 - v + mp.log(v)) - mp.log(u)
        assert margin > 0, (alpha, z, u)
        assert oracle.mt_accept(alpha, z, u) == 1
        passed += 1
    assert passed > 3000


def test_laplace_ks(oracle):
    n = 200000
    out, _, _, st = oracle.laplace(9, 64, _const(n, 1.0), _const(n, 0.5))
    assert st == 0
    assert stats.kstest(out, stats.laplace(1.0, 0.5).cdf).pvalue > KS_P


def test_weibull_ks(oracle):
    n = 200000
    out, _, _, st = oracle.weibull(10, 64, _const(n, 1.7), _const(n, 3.0))
    assert st == 0
    assert stats.kstest(out, stats.weibull_min(1.7, scale=3.0).cdf).pvalue > KS_P


def test_varying_parameter_pit_all(oracle):
    n = 60000
    a, b = inputs.uniform_params(n, seed=11)
    out, _, _, _ = oracle.uniform(11, 500, a, b)
    wide = b > a
    pit = (out[wide] - a[wide]) / (b[wide].astype(np.float64) - a[wide])
    assert stats.kstest(pit, "uniform").pvalue > KS_P
    mu, sigma = inputs.normal_params(n, seed=12)
    out, _, _, _ = oracle.normal(12, 500, mu, sigma)
    assert stats.kstest(stats.norm.cdf(out, mu, sigma), "uniform").pvalue > KS_P
    lam = inputs.rate_params(n, seed=13)
    out, _, _, _ = oracle.exponential(13, 500, lam)
    assert stats.kstest(stats.expon.cdf(out * lam), "uniform").pvalue > KS_P


def test_dirichlet_invariants(oracle):
    K = 8
    alpha_row = np.array([0.1, 0.5, 1.0, 2.0, 3.5, 0.05, 10.0, 1.1], dtype=np.float32)
    n = 40000
    alpha = np.tile(alpha_row, (n, 1))
    th, pos, st = oracle.dirichlet(14, 64 * K, alpha)
    assert st == 0
    assert np.max(np.abs(th.sum(axis=1) - 1.0)) < 1e-13
    a0 = float(alpha_row.astype(np.float64).sum())
    for k in range(K):
        ak = float(alpha_row[k])
        mean = ak / a0
        var = ak * (a0 - ak) / (a0 * a0 * (a0 + 1))
        assert abs(th[:, k].mean() - mean) < 5 * np.sqrt(var / n)
        assert stats.kstest(th[:, k], stats.beta(ak, a0 - ak).cdf).pvalue > KS_P


# ---- buffer semantics (Sec. 2.2) ---------------------------------------------

@pytest.mark.parametrize("fn", ["uniform", "normal", "exponential", "gamma", "laplace", "weibull"])
def test_buffer_length_invariance(oracle, fn):
    n = 3000
    p0 = inputs.shape_params(n, seed=15) if fn in ("gamma", "weibull") else _const(n, 1.0)
    p1 = _const(n, 2.0)
    args = [p0] if fn in ("exponential", "gamma") else [p0, p1]
    ref = None
    for L in (1, 3, 4, 64, 1000):
        out, words, pos, st = getattr(oracle, fn)(16, 37, *args, buf_len=L)
        if ref is None:
            ref = (out, words, pos)
        else:
            assert np.array_equal(out, ref[0]) and np.array_equal(words, ref[1])
            assert np.array_equal(pos, ref[2])


@pytest.mark.parametrize("fn", ["normal", "gamma", "laplace"])
def test_call_splitting(oracle, fn):
    """Two calls continuing the streams equal one call (counters persist)."""
    S = 16
    n = S * 50
    p0 = inputs.shape_params(n, seed=17)
    p1 = _const(n, 1.0)
    args = [p0] if fn == "gamma" else [p0, p1]
    whole, wwhole, pos_whole, _ = getattr(oracle, fn)(18, S, *args, buf_len=8)
    k = S * 20
    first, w1, pos1, _ = getattr(oracle, fn)(18, S, *[a[:k] for a in args], buf_len=8)
    second, w2, pos2, _ = getattr(oracle, fn)(18, S, *[a[k:] for a in args], pos=pos1, buf_len=8)
    assert np.array_equal(np.concatenate([first, second]), whole)
    assert np.array_equal(np.concatenate([w1, w2]), wwhole)
    assert np.array_equal(pos2, pos_whole)


def test_sequential_consumption(oracle):
    """Draw m of stream s consumes element m of that stream's domain."""
    S, m = 8, 40
    n = S * m
    out, words, pos, _ = oracle.exponential(19, S, _const(n, 1.0))
    pos = pos.reshape(S, 3)
    assert np.all(pos[:, 2] == m) and np.all(pos[:, 0] == 0) and np.all(pos[:, 1] == 0)
    for s in range(S):
        vals, w = oracle.elements(19, 2, s, 0, m)
        assert np.array_equal(out[s::S], vals) and np.array_equal(words[s::S], w)


def test_gamma_consumption_and_words(oracle):
    S, m = 4, 200
    n = S * m
    alpha = _const(n, 0.3)
    out, words, pos, _ = oracle.gamma(20, S, alpha)
    pos = pos.reshape(S, 3)
    for s in range(S):
        _, wn = oracle.elements(20, 1, s, 0, int(pos[s, 1]))
        # the first word of every draw is the word of an N element, in order
        idx = [int(np.nonzero(wn == w)[0][0]) for w in words[s::S]]
        assert idx[0] == 0 and all(b > a for a, b in zip(idx, idx[1:]))
        # alpha < 1: each draw takes one extra U' after the accept
        assert pos[s, 1] >= m and pos[s, 0] >= 2 * m


def test_invalid_parameters(oracle):
    a = np.array([0.0, 1.0, np.nan, 2.0], dtype=np.float32)
    b = np.array([1.0, 0.5, 1.0, np.inf], dtype=np.float32)
    out, words, pos, st = oracle.uniform(21, 1, a, b)
    assert st == 4
    assert np.isfinite(out[0]) and np.all(np.isnan(out[1:]))
    assert pos[0] == 1  # invalid draws consume nothing
    out, _, pos, st = oracle.gamma(21, 1, np.array([-1.0, 0.0, 2.0], dtype=np.float32))
    assert st == 4 and np.isnan(out[0]) and np.isnan(out[1]) and out[2] > 0


def test_mixed_matches_single_distributions(oracle):
    n = 4000
    S = 40
    for tagv, fn in [(0, "uniform"), (1, "normal"), (2, "exponential"), (3, "gamma"),
                     (4, "laplace"), (5, "weibull")]:
        p0 = inputs.shape_params(n, seed=22)
        p1 = p0 + np.float32(1.0)
        tag = np.full(n, tagv, dtype=np.uint8)
        mo, mw, mpos, _ = oracle.mixed(23, S, tag, p0, p1)
        args = [p0] if fn in ("exponential", "gamma") else [p0, p1]
        so, sw, spos, _ = getattr(oracle, fn)(23, S, *args)
        assert np.array_equal(mo, so) and np.array_equal(mw, sw) and np.array_equal(mpos, spos)


def test_mixed_sampled_streams_equal_full(oracle):
    n = 20000
    S = 100
    tag, p0, p1 = inputs.mixed_stream(n, seed=24, n_tags=6)
    full, fw, fpos, _ = oracle.mixed(25, S, tag, p0, p1, nthreads=4)
    part, pw, ppos, _ = oracle.mixed(25, S, tag, p0, p1, streams=(10, 20))
    idx = np.nonzero((np.arange(n) % S >= 10) & (np.arange(n) % S < 20))[0]
    assert np.array_equal(part[idx], full[idx]) and np.array_equal(pw[idx], fw[idx])
    assert np.array_equal(ppos.reshape(S, 3)[10:20], fpos.reshape(S, 3)[10:20])
