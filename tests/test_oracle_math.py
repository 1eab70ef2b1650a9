"""Pins of the oracle's FP64 log and sincospi, and of the base conversions.

log and sincospi are checked against mpmath (50+ digits) for an error bound,
exhaustively over every argument the Gaussian/exponential buffers can feed
them (all 2^24 values of U' and of 2U), and on exact special values.  The
conversions are checked against their definitions evaluated independently in
Python integers / mpmath from the raw words.
"""
import math

import mpmath as mp
import numpy as np
import pytest

mp.mp.prec = 120


def _ulps(got, exact):
    exact_f = float(exact)
    if exact_f == 0.0:
        return 0.0 if got == 0.0 else math.inf
    return float(abs(mp.mpf(float(got)) - exact) / mp.mpf(float(np.spacing(abs(exact_f)))))


def test_log_error_bound_vs_mpmath(oracle):
    rng = np.random.default_rng(3)
    xs = np.concatenate([
        rng.uniform(0.0, 1.0, 3000),
        np.exp(rng.uniform(-700.0, 700.0, 3000)),
        1.0 + rng.uniform(-1e-6, 1e-6, 1000),
        rng.uniform(0.5, 2.0, 1000) ** 3,  # the v = t^3 range of the Gamma test
        [5e-324, 2.2250738585072014e-308, 1.0000000000000002, 0.9999999999999999, 1e308],
    ])
    xs = xs[xs > 0]
    got = oracle.log(xs)
    worst = max(_ulps(g, mp.log(mp.mpf(float(x)))) for x, g in zip(xs, got))
    assert worst <= 2.0, worst


def test_log_exhaustive_over_open_uniforms(oracle):
    k = np.arange(1 << 24, dtype=np.float64)
    u = (k + 1.0) * 2.0**-24
    got = oracle.log(u)
    ref = np.log(u)  # libm, within 1 ulp of the true value
    ulp = np.spacing(np.abs(ref))
    bad = (np.abs(got - ref) > 2.0 * ulp) & (ref != 0.0)
    assert not bad.any(), u[bad][:5]
    assert got[-1] == 0.0  # ln 1 = 0 exactly


def test_log_special_values(oracle):
    assert oracle.log(np.array([1.0]))[0] == 0.0
    for e in (-1074, -1022, -60, -1, 1, 60, 1023):
        x = math.ldexp(1.0, e)
        assert _ulps(oracle.log(np.array([x]))[0], e * mp.log(2)) <= 1.0
    out = oracle.log(np.array([0.0, -1.0, np.inf]))
    assert out[0] == -np.inf and np.isnan(out[1]) and out[2] == np.inf


def test_sincospi_exhaustive_dyadic(oracle):
    a = np.arange(1 << 24, dtype=np.float64) * 2.0**-23  # every 2U the Gaussian buffer uses
    s, c = oracle.sincospi(a)
    # numpy evaluates sin(fl(pi*a)); fl(pi*a) is off by <= 2^-53 * 2pi absolute
    assert np.max(np.abs(s - np.sin(np.pi * a))) < 1.5e-15
    assert np.max(np.abs(c - np.cos(np.pi * a))) < 1.5e-15
    assert np.max(np.abs(s * s + c * c - 1.0)) < 5e-16
    # exact values at multiples of 1/2, and the symmetric values at 1/4
    for q, (sv, cv) in enumerate([(0, 1), (1, 0), (0, -1), (-1, 0)]):
        i = q << 22
        assert s[i] == sv and c[i] == cv
    r = math.sqrt(0.5)
    for q in range(4):
        i = (2 * q + 1) << 21
        assert abs(abs(s[i]) - r) <= 2.3e-16 and abs(abs(c[i]) - r) <= 2.3e-16


def test_sincospi_error_bound_vs_mpmath(oracle):
    rng = np.random.default_rng(5)
    a = rng.integers(0, 1 << 24, 3000).astype(np.float64) * 2.0**-23
    s, c = oracle.sincospi(a)
    worst = 0.0
    for ai, si, ci in zip(a, s, c):
        x = mp.mpf(float(ai))
        worst = max(worst, _ulps(si, mp.sinpi(x)), _ulps(ci, mp.cospi(x)))
    # fl(pi*r) adds up to 1/2 ulp to the series evaluation error
    assert worst <= 2.0, worst


# ---- base conversions, from the raw words ---------------------------------

def test_uniform_conversion_exact(oracle):
    vals, words = oracle.elements(42, 0, 3, 0, 50000)
    k = (words >> 8).astype(np.float64)
    assert np.array_equal(vals, k * 2.0**-24)
    assert vals.min() >= 0.0 and vals.max() < 1.0


def test_u64_conversion_exact(oracle):
    vals, _ = oracle.elements(42, 4, 5, 0, 4000)
    w = oracle.philox_words(42, 4, 5, 0, 2000)
    for j in range(4000):
        wa, wb = int(w[2 * j]), int(w[2 * j + 1])
        want = ((wa >> 5) * 2**26 + (wb >> 6)) / 2**53  # exact: 53-bit integer
        assert vals[j] == want
    assert vals.min() >= 0.0 and vals.max() < 1.0


def test_exponential_conversion(oracle):
    vals, words = oracle.elements(42, 2, 1, 0, 3000)
    for v, w in zip(vals, words):
        u = mp.mpf(int(w >> 8) + 1) / 2**24
        assert _ulps(v, -mp.log(u)) <= 2.0 or (v == 0.0 and int(w >> 8) == 2**24 - 1)


def test_gaussian_conversion(oracle):
    vals, _ = oracle.elements(42, 1, 2, 0, 4000)
    w = oracle.philox_words(42, 1, 2, 0, 1000)
    for j in range(4000):
        b, slot = divmod(j, 4)
        pair = slot // 2
        w0, w1 = int(w[4 * b + 2 * pair]), int(w[4 * b + 2 * pair + 1])
        r = mp.sqrt(-2 * mp.log(mp.mpf((w0 >> 8) + 1) / 2**24))
        ang = mp.mpf(w1 >> 8) / 2**23
        z = r * (mp.cospi(ang) if slot % 2 == 0 else mp.sinpi(ang))
        # r carries the error of log+sqrt (<= 2 ulp), cos/sin <= 1.5 ulp
        assert abs(mp.mpf(float(vals[j])) - z) <= 6 * 2.0**-53 * max(abs(z), r * 2.0**-20), j


def test_gaussian_tail_truncation(oracle):
    # |z| <= sqrt(-2 ln 2^-24): the 24-bit U' bounds the Box-Muller radius
    vals, _ = oracle.elements(7, 1, 0, 0, 200000)
    assert np.max(np.abs(vals)) <= math.sqrt(2 * 24 * math.log(2)) + 1e-12
