"""The log-free Marsaglia-Tsang tests of the CUDA path rest on two bounds of
the margin's series p(x) = sum_k (-x)^k / (k + 4) (the margin is
-ln U' - 3 d x^4 p(x), |x| <= 1/4):
    p_lo(x) = 1/4 - x/5                       <= p(x)
    p_hi(x) = 1/4 - x/5 + x^2/6 + 0.1905 |x|^3 >= p(x)
checked here on a dense grid against the series summed exactly (mpmath), with
the FP32 constants the kernels use, and with room for their 1e-5 margins."""
import numpy as np
import pytest


def _p_exact(x, mp):
    # closed form of the series: p(x) = (ln(1+x) - x + x^2/2 - x^3/3) / (-x^4)
    x = mp.mpf(x)
    if x == 0:
        return mp.mpf(1) / 4
    return (mp.log1p(x) - x + x ** 2 / 2 - x ** 3 / 3) / (-(x ** 4))


def test_series_bounds_hold_on_the_series_range():
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 50
    c6 = float(np.float32(float.fromhex("0x1.555556p-3")))  # 1/6 as the kernels round it
    c5 = float(np.float32(float.fromhex("0x1.99999ap-3")))  # 1/5
    xs = np.concatenate([np.linspace(-0.25, 0.25, 20001), [-0.25, 0.25, 1e-6, -1e-6]])
    worst_hi, worst_lo = np.inf, np.inf
    for x in xs:
        p = _p_exact(x, mp)
        hi = 0.25 - c5 * x + c6 * x * x + 0.1905 * abs(x) ** 3
        lo = 0.25 - 0.2 * x
        worst_hi = min(worst_hi, float((hi - p) / p))
        worst_lo = min(worst_lo, float((p - lo) / p))
    # both hold with far more than the 1e-5 relative slack the kernels add
    assert worst_hi > -1e-7, worst_hi
    assert worst_lo >= 0.0, worst_lo
    # and the series check: the closed form equals the series at small x
    x = mp.mpf("0.01")
    ser = mp.nsum(lambda k: (-x) ** k / (k + 4), [0, mp.inf])
    assert abs(ser - _p_exact(x, mp)) < mp.mpf(10) ** -40
