"""Pins of the oracle's FP64 uniform (Sec. 2.2 GetUniform at double precision,
from the 53-bit U64 domain).

* brute force: every output equals fma(b - a, u53, a) -- the difference
  rounded to double, then the product and sum rounded once, computed here in
  exact rational arithmetic -- with u53 built in Python integers from Philox
  words of a Python-int Philox (the Salmon et al. round function restated
  here, independent of the oracle's C), element j of stream s in block j/2,
  words 2(j%2) and 2(j%2)+1; the word output is the pair's first word;
* closed forms: mean (a+b)/2 and variance (b-a)^2/12, KS against U(0, 1);
  u53 values are multiples of 2^-53 in [0, 1);
* consumption: invalid (a, b) give NaN, word 0 and consume nothing; positions
  advance by the valid draws per stream; a call split in two (positions
  carried) equals one call; values do not depend on the buffer length.
"""
from fractions import Fraction

import numpy as np
import pytest
from scipy import stats

import oracle as O

M0, M1, W0, W1 = 0xD2511F53, 0xCD9E8D57, 0x9E3779B9, 0xBB67AE85


def _philox(ctr, seed):
    c = list(ctr)
    k0, k1 = seed & 0xFFFFFFFF, seed >> 32
    for _ in range(10):
        p0 = M0 * c[0]
        p1 = M1 * c[2]
        c = [(p1 >> 32) ^ c[1] ^ k0, p1 & 0xFFFFFFFF, (p0 >> 32) ^ c[3] ^ k1, p0 & 0xFFFFFFFF]
        k0 = (k0 + W0) & 0xFFFFFFFF
        k1 = (k1 + W1) & 0xFFFFFFFF
    return c


def _u53_element(seed, stream, j):
    """Element j of the U64 domain (4) of `stream`: (value, first word)."""
    blk = j // 2
    w = _philox([blk & 0xFFFFFFFF, 4, stream, blk >> 32], seed)
    wa, wb = w[2 * (j % 2)], w[2 * (j % 2) + 1]
    m = ((wa >> 5) << 26) | (wb >> 6)
    return m * 2.0 ** -53, wa


def test_brute_force_against_python_philox():
    seed, S, n = 0x1234ABCD9876, 5, 37
    rng = np.random.default_rng(1)
    a = rng.uniform(-10, 10, n)
    b = a + rng.uniform(0, 5, n)
    pos0 = np.array([0, 1, 7, 2**32 + 3, 11], dtype=np.uint64)  # odd and beyond-32-bit starts
    out, words, pos, st = O.uniform_f64(seed, S, a, b, pos0)
    assert st == O.OK
    for s in range(S):
        j = int(pos0[s])
        for i in range(s, n, S):
            u, w0 = _u53_element(seed, s, j)
            d = float(b[i]) - float(a[i])  # rounded once
            want = float(Fraction(d) * Fraction(u) + Fraction(float(a[i])))  # one more rounding
            assert out[i] == want
            assert words[i] == w0
            j += 1
        assert pos[s] == j


def test_closed_forms_and_resolution():
    n, S = 400_000, 1000
    out, words, pos, st = O.uniform_f64(7, S, np.zeros(n), np.ones(n))
    assert st == O.OK
    assert out.min() >= 0.0 and out.max() < 1.0
    k = out * 2.0 ** 53
    assert np.all(k == np.floor(k))  # multiples of 2^-53
    assert abs(out.mean() - 0.5) < 5 * np.sqrt(1 / 12 / n)
    assert abs(out.var() - 1 / 12) < 5 * np.sqrt((1 / 80 - 1 / 144) / n)
    assert stats.kstest(out, "uniform").pvalue > 1e-4
    # a general interval: mean (a+b)/2, variance (b-a)^2/12
    o2, _, _, st = O.uniform_f64(8, S, np.full(n, -3.0), np.full(n, 5.0))
    assert st == O.OK and o2.min() >= -3.0 and o2.max() < 5.0
    assert abs(o2.mean() - 1.0) < 5 * np.sqrt(64 / 12 / n)
    assert abs(o2.var() - 64 / 12) < 5 * 64 * np.sqrt((1 / 80 - 1 / 144) / n)


def test_invalid_parameters_consume_nothing():
    a = np.array([0.0, np.nan, 1.0, -np.inf, 2.0, 0.5, 3.0])
    b = np.array([1.0, 1.0, 0.5, 1.0, np.inf, 0.5, 4.0])  # b < a, infinite, a == b
    out, words, pos, st = O.uniform_f64(3, 1, a, b)
    assert st == O.EDOMAIN
    assert np.isnan(out[[1, 2, 3, 4]]).all() and np.all(words[[1, 2, 3, 4]] == 0)
    assert out[5] == 0.5  # a == b is valid
    ok, okw, okpos, _ = O.uniform_f64(3, 1, a[[0, 5, 6]], b[[0, 5, 6]])
    assert np.array_equal(out[[0, 5, 6]], ok) and np.array_equal(words[[0, 5, 6]], okw)
    assert np.array_equal(pos, okpos) and pos[0] == 3


@pytest.mark.parametrize("buf_len", [1, 3, 64])
def test_split_calls_and_buffer_length(buf_len):
    n, S = 5000, 17
    rng = np.random.default_rng(4)
    a = rng.uniform(-1, 0, n)
    b = rng.uniform(0, 1, n)
    whole, ww, wpos, _ = O.uniform_f64(5, S, a, b, buf_len=64)
    cut = 1700  # a multiple of S keeps draw i on stream i mod S in both halves
    cut -= cut % S
    o1, w1, p1, _ = O.uniform_f64(5, S, a[:cut], b[:cut], buf_len=buf_len)
    o2, w2, p2, _ = O.uniform_f64(5, S, a[cut:], b[cut:], p1, buf_len=buf_len)
    assert np.array_equal(np.concatenate([o1, o2]), whole)
    assert np.array_equal(np.concatenate([w1, w2]), ww) and np.array_equal(p2, wpos)
