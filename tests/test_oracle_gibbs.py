"""Pins of the oracle's Gibbs models.

Triangle (Eq. 1, Fig. 1): the first sweep recomputed by hand from the raw
Philox words, the closed-form moments of the uniform density on the triangle
(E X = E Y = 1/3, Var = 1/18, Cov = -1/36), and the support X + Y < 1 checked
in exact rational arithmetic.  Normal-gamma: chain means against the
stationary marginals computed by 1-D quadrature.  LDA: Dirichlet means.
Structure: threads, chain-range sharding and checkpoint/resume are exact.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate

from paper_1412_4825_gb300 import inputs


def _u64(wa, wb):
    return ((int(wa) >> 5) * 2**26 + (int(wb) >> 6)) / 2**53


def test_triangle_first_sweeps_by_hand(oracle):
    seed, chain = 42, 5
    r = oracle.gibbs_triangle(seed, 1, 3, chain_offset=chain)
    w = oracle.philox_words(seed, 4, chain, 0, 3)  # U64 domain, 2 elements per block
    u = [_u64(w[2 * j], w[2 * j + 1]) for j in range(6)]
    x, y = 0.5, 0.5
    sx = sy = 0.0
    for it in range(3):
        x = (1.0 - y) * u[2 * it]  # Fig. 1: x first, from U[0, 1-y)
        y = (1.0 - x) * u[2 * it + 1]
        sx += x
        sy += y
    assert r["xy"][0, 0] == x and r["xy"][0, 1] == y
    assert r["mom"][0, 0] == sx and r["mom"][0, 1] == sy
    assert r["pos"][0] == 6


def test_triangle_support_exact(oracle):
    """Every state lies in the triangle: x, y >= 0 and x + y < 1 exactly."""
    xy = None
    pos = None
    for _ in range(300):
        r = oracle.gibbs_triangle(7, 64, 1, xy=xy, pos=pos)
        xy, pos = r["xy"].ravel(), r["pos"]
        for x, y in r["xy"]:
            assert x >= 0.0 and y >= 0.0
            assert Fraction(x) + Fraction(y) < 1


def test_triangle_closed_form_moments(oracle):
    n_chains, n_sweeps = 256, 4000
    r = oracle.gibbs_triangle(42, n_chains, n_sweeps, nthreads=4)
    m = r["mom"] / n_sweeps  # per-chain time averages
    ex, ey = m[:, 0], m[:, 1]
    vx = m[:, 2] - ex ** 2
    cxy = m[:, 4] - ex * ey
    # chains are independent: the spread of per-chain averages gives the SE
    for est, truth in [(ex, 1 / 3), (ey, 1 / 3), (vx, 1 / 18), (cxy, -1 / 36)]:
        se = est.std(ddof=1) / np.sqrt(n_chains)
        assert abs(est.mean() - truth) < 5 * se + 1e-4, (est.mean(), truth, se)


def test_triangle_threads_and_shards_exact(oracle):
    a = oracle.gibbs_triangle(3, 100, 50, nthreads=1)
    b = oracle.gibbs_triangle(3, 100, 50, nthreads=7)
    assert np.array_equal(a["xy"], b["xy"]) and np.array_equal(a["mom"], b["mom"])
    s1 = oracle.gibbs_triangle(3, 40, 50, chain_offset=0)
    s2 = oracle.gibbs_triangle(3, 60, 50, chain_offset=40)
    assert np.array_equal(np.concatenate([s1["xy"], s2["xy"]]), a["xy"])


def test_triangle_resume_exact(oracle):
    whole = oracle.gibbs_triangle(9, 16, 100, buf_len=256)
    h = oracle.gibbs_triangle(9, 16, 37, buf_len=256)
    rest = oracle.gibbs_triangle(9, 16, 63, xy=h["xy"].ravel(), pos=h["pos"], mom=h["mom"].ravel(),
                                 buf_len=5)
    assert np.array_equal(rest["xy"], whole["xy"]) and np.array_equal(rest["mom"], whole["mom"])


def _ng_stationary(n, xbar, S, prior=(2.0, 1.0, 0.0, 0.01)):
    a0, b0, mu0, prec0 = prior
    shape = a0 + n / 2

    def logp(mu):
        SS = S + n * (xbar - mu) ** 2
        return -0.5 * prec0 * (mu - mu0) ** 2 - shape * np.log(b0 + SS / 2)

    sd = np.sqrt(S / n / n) + 1e-3
    lo, hi = xbar - 30 * sd, xbar + 30 * sd
    c = logp(xbar)
    Z = integrate.quad(lambda m: np.exp(logp(m) - c), lo, hi, limit=200)[0]
    Emu = integrate.quad(lambda m: m * np.exp(logp(m) - c), lo, hi, limit=200)[0] / Z
    Etau = integrate.quad(lambda m: shape / (b0 + (S + n * (xbar - m) ** 2) / 2) * np.exp(logp(m) - c),
                          lo, hi, limit=200)[0] / Z
    return Emu, Etau


def test_normal_gamma_stationary_means(oracle):
    n_chains, n_sweeps = 64, 3000
    nobs, xbar, sc = inputs.normal_gamma_data(1, seed=3)
    nobs, xbar, sc = (np.repeat(a, n_chains) for a in (nobs, xbar, sc))
    r = oracle.gibbs_normal_gamma(42, n_sweeps, nobs, xbar, sc, nthreads=4)
    Emu, Etau = _ng_stationary(float(nobs[0]), float(xbar[0]), float(sc[0]))
    m = r["mom"] / n_sweeps
    for est, truth in [(m[:, 0], Emu), (m[:, 1], Etau)]:
        se = est.std(ddof=1) / np.sqrt(n_chains)
        assert abs(est.mean() - truth) < 5 * se, (est.mean(), truth, se)
    assert 0.15 < Etau < 0.4  # data sd 2: the precision is near 1/4


def test_normal_gamma_structure_exact(oracle):
    nobs, xbar, sc = inputs.normal_gamma_data(50, seed=4)
    a = oracle.gibbs_normal_gamma(5, 40, nobs, xbar, sc, nthreads=1)
    b = oracle.gibbs_normal_gamma(5, 40, nobs, xbar, sc, nthreads=3, buf_len=3)
    assert np.array_equal(a["state"], b["state"]) and np.array_equal(a["mom"], b["mom"])
    h = oracle.gibbs_normal_gamma(5, 15, nobs, xbar, sc)
    rest = oracle.gibbs_normal_gamma(5, 25, nobs, xbar, sc, state=h["state"].ravel(),
                                     pos=h["pos"].ravel(), mom=h["mom"].ravel())
    assert np.array_equal(rest["state"], a["state"]) and np.array_equal(rest["mom"], a["mom"])
    s2 = oracle.gibbs_normal_gamma(5, 40, nobs[20:], xbar[20:], sc[20:], chain_offset=20)
    assert np.array_equal(s2["state"], a["state"][20:])
    # per sweep: one Gaussian for mu plus one per Gamma attempt (>= 1)
    assert np.all(a["pos"][:, 0] >= 80) and np.all(a["pos"][:, 1] >= 40)


def test_lda_dirichlet_means(oracle):
    alpha, counts, _ = inputs.lda_alpha(4, K=16, len_lo=50, len_hi=500, seed=5)
    n_sweeps = 4000
    r = oracle.gibbs_lda(42, n_sweeps, alpha, nthreads=4)
    assert np.max(np.abs(r["theta"].sum(axis=1) - 1.0)) < 1e-13
    a = alpha.astype(np.float64)
    a0 = a.sum(axis=1, keepdims=True)
    mean = a / a0
    var = a * (a0 - a) / (a0 ** 2 * (a0 + 1))
    est = r["mom"] / n_sweeps  # sweeps are independent draws (counts fixed)
    assert np.all(np.abs(est - mean) < 5 * np.sqrt(var / n_sweeps) + 1e-12)


def test_lda_structure_exact(oracle):
    alpha, _, _ = inputs.lda_alpha(6, K=8, seed=6)
    a = oracle.gibbs_lda(7, 30, alpha, nthreads=1)
    b = oracle.gibbs_lda(7, 30, alpha, nthreads=4, buf_len=5)
    assert np.array_equal(a["theta"], b["theta"]) and np.array_equal(a["mom"], b["mom"])
    s = oracle.gibbs_lda(7, 30, alpha[2:], doc_offset=2)
    assert np.array_equal(s["theta"], a["theta"][2:])
    # one LDA sweep is one Dirichlet draw from the documents' component streams
    d = oracle.gibbs_lda(8, 1, alpha)
    S = alpha.shape[0] * alpha.shape[1]
    th, _, _ = oracle.dirichlet(8, S, alpha)
    assert np.allclose(d["theta"], th, rtol=0, atol=0)
