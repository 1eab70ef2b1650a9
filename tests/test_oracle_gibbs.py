"""Pins of the oracle's Gibbs models.

Triangle (Eq. 1, Fig. 1): the first sweep recomputed by hand from the raw
Philox words, the closed-form moments of the uniform density on the triangle
(E X = E Y = 1/3, Var = 1/18, Cov = -1/36), and the support X + Y < 1 checked
in exact rational arithmetic.  Normal-gamma: chain means and second moments
against the stationary marginals computed by 1-D quadrature; the sweep map's
partial derivatives (which the FP32 error bounds propagate along) against
finite differences of the oracle's own sweep.  LDA: Dirichlet means.
Structure: threads, chain-range sharding and checkpoint/resume are exact.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy import integrate

from paper_1412_4825_gb300 import inputs

import gibbs_bounds


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
    """E[mu], E[tau], E[mu^2], E[tau^2] under the joint posterior, the
    stationary law of the Gibbs chain.  Integrating tau out of
    N(mu; mu0, 1/prec0) Gamma(tau; a0, b0) prod_i N(x_i; mu, 1/tau) leaves
    p(mu | x) proportional to N(mu; mu0, 1/prec0) r(mu)^-(a0 + n/2) with
    r(mu) = b0 + (S + n (xbar - mu)^2)/2, and tau | mu, x ~ Gamma(a, r(mu)),
    a = a0 + n/2, whose first two moments are a/r and a (a + 1)/r^2."""
    a0, b0, mu0, prec0 = prior
    shape = a0 + n / 2

    def rate(mu):
        return b0 + (S + n * (xbar - mu) ** 2) / 2

    def logp(mu):
        return -0.5 * prec0 * (mu - mu0) ** 2 - shape * np.log(rate(mu))

    sd = np.sqrt(S / n / n) + 1e-3
    lo, hi = xbar - 30 * sd, xbar + 30 * sd
    c = logp(xbar)

    def E(f):
        return integrate.quad(lambda m: f(m) * np.exp(logp(m) - c), lo, hi, limit=200)[0]

    Z = E(lambda m: 1.0)
    return dict(mu=E(lambda m: m) / Z, tau=E(lambda m: shape / rate(m)) / Z,
                mu2=E(lambda m: m * m) / Z, tau2=E(lambda m: shape * (shape + 1) / rate(m) ** 2) / Z)


def _ng_long_run(oracle):
    n_chains, n_sweeps = 64, 3000
    nobs, xbar, sc = inputs.normal_gamma_data(1, seed=3)
    nobs, xbar, sc = (np.repeat(a, n_chains) for a in (nobs, xbar, sc))
    r = oracle.gibbs_normal_gamma(42, n_sweeps, nobs, xbar, sc, nthreads=4)
    truth = _ng_stationary(float(nobs[0]), float(xbar[0]), float(sc[0]))
    return r["mom"] / n_sweeps, truth, n_chains


def test_normal_gamma_stationary_means(oracle):
    m, truth, n_chains = _ng_long_run(oracle)
    for est, want in [(m[:, 0], truth["mu"]), (m[:, 1], truth["tau"])]:
        se = est.std(ddof=1) / np.sqrt(n_chains)
        assert abs(est.mean() - want) < 5 * se, (est.mean(), want, se)
    assert 0.15 < truth["tau"] < 0.4  # data sd 2: the precision is near 1/4


def test_normal_gamma_stationary_second_moments(oracle):
    """E[mu^2] and E[tau^2] (hence Var[mu | x] and Var[tau | x]) of the chain
    time averages against quadrature.  A wrong spread in either conditional
    fails here even when the means stay right: drawing mu with standard
    deviation 1/P instead of 1/sqrt(P) (P ~ 25 here) shrinks Var[mu] from
    ~0.04 to ~0.002, about 25 standard errors of this estimate."""
    m, truth, n_chains = _ng_long_run(oracle)
    for est, want in [(m[:, 2], truth["mu2"]), (m[:, 3], truth["tau2"])]:
        se = est.std(ddof=1) / np.sqrt(n_chains)
        assert abs(est.mean() - want) < 5 * se, (est.mean(), want, se)
    var_mu = truth["mu2"] - truth["mu"] ** 2
    var_tau = truth["tau2"] - truth["tau"] ** 2
    assert 0.02 < var_mu < 0.08 and 0.0005 < var_tau < 0.003  # sd(mu) ~ 2/sqrt(100)
    # the estimate resolves the variance itself, not only the second moment
    se_var = (m[:, 2] - m[:, 0] ** 2).std(ddof=1) / np.sqrt(n_chains)
    assert abs((m[:, 2] - m[:, 0] ** 2).mean() - var_mu) < 0.2 * var_mu + 5 * se_var


def test_normal_gamma_trace_matches_run(oracle):
    """The traced trajectory is the run itself: its last (tau, mu) is the
    final state and its column sums are the sweep moments."""
    nobs, xbar, sc = inputs.normal_gamma_data(20, seed=8)
    r = oracle.gibbs_normal_gamma(3, 30, nobs, xbar, sc, trace=True)
    tr = r["trace"]
    assert np.array_equal(tr[:, -1, 3], r["state"][:, 1]) and np.array_equal(tr[:, -1, 4], r["state"][:, 0])
    assert np.allclose(tr[:, :, 4].sum(axis=1), r["mom"][:, 0], rtol=1e-13)
    assert np.allclose((tr[:, :, 3] ** 2).sum(axis=1), r["mom"][:, 3], rtol=1e-13)
    # G / rate = tau, rate from the previous mu
    mu_prev = np.concatenate([np.zeros((20, 1)), tr[:, :-1, 4]], axis=1)
    w = gibbs_bounds.ng_sweep_terms(nobs[:, None], xbar[:, None], sc[:, None], (2.0, 1.0, 0.0, 0.01),
                                    mu_prev, tr[:, :, 0], tr[:, :, 2])
    assert np.allclose(w["tau"], tr[:, :, 3], rtol=1e-14)
    assert np.all(tr[:, :, 1] >= 0.0)


@pytest.mark.parametrize("prior,nobs_set", [((2.0, 1.0, 0.0, 0.01), None), ((0.4, 1.0, 0.5, 0.2), 1.0),
                                            ((3.0, 2.0, -1.0, 1.0), 7.0)])
def test_normal_gamma_sweep_derivatives(oracle, prior, nobs_set):
    """The partial derivatives of the sweep map that the FP32 error bounds
    propagate along agree with central finite differences of the oracle's own
    FP64 sweep: one sweep from mu and from mu +- h with the same stream
    positions (the Gamma shape does not depend on mu, so the same draws are
    consumed and only the rate and the mean move)."""
    nobs, xbar, sc = inputs.normal_gamma_data(40, seed=11)
    if nobs_set is not None:
        nobs = np.full_like(nobs, nobs_set)
    r0 = oracle.gibbs_normal_gamma(7, 9, nobs, xbar, sc, prior=prior)
    st, pos = r0["state"], r0["pos"]
    h = 1e-5 * (1.0 + np.abs(st[:, 0]))
    runs = []
    for sgn in (-1.0, 0.0, 1.0):
        s = st.copy()
        s[:, 0] += sgn * h
        runs.append(oracle.gibbs_normal_gamma(7, 1, nobs, xbar, sc, prior=prior, state=s.ravel(),
                                              pos=pos.ravel(), trace=True))
    for r in runs[1:]:
        assert np.array_equal(r["pos"], runs[0]["pos"])
    tr = runs[1]["trace"][:, 0]
    w = gibbs_bounds.ng_sweep_terms(nobs, xbar, sc, prior, st[:, 0], tr[:, 0], tr[:, 2])
    fd_tau = (runs[2]["state"][:, 1] - runs[0]["state"][:, 1]) / (2 * h)
    fd_mu = (runs[2]["state"][:, 0] - runs[0]["state"][:, 0]) / (2 * h)
    assert np.allclose(w["dtau_dmu"], fd_tau, rtol=1e-4, atol=1e-9 * np.abs(tr[:, 3]).max())
    chain = w["dmu_dtau"] * w["dtau_dmu"]
    assert np.allclose(chain, fd_mu, rtol=1e-4, atol=1e-9)
    # d mu / d tau alone, where tau moves enough to divide by
    ok = np.abs(fd_tau) > 1e-3 * np.abs(fd_tau).max()
    assert ok.sum() >= 10
    assert np.allclose(w["dmu_dtau"][ok], (fd_mu / fd_tau)[ok], rtol=1e-3)


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
