"""The three tiers of the Poisson and Binomial inversion searches on GB300.

A draw is decided by the plain FP32 search when its uniform lies far enough
from the CDF steps, else by the double-single search, else redone in FP64
(the bounds are stated beside each tier in brng_bulk.cu).  Here each selected
draw's uniform is placed, by choosing its parameter, at a relative distance
from a CDF step that the FP32 tier cannot certify but the double-single tier
can (computed from the float32 parameter actually passed, with scipy's CDF):
every count must equal the oracle's, and the FP64 path must not run at all.
"""
import numpy as np
import pytest

import oracle as O

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on a CPU host only with -m gpu
    pytest.skip("no CUDA device", allow_module_level=True)
stats = pytest.importorskip("scipy.stats")

from paper_1412_4825_gb300 import brng as B  # noqa: E402

DEV = torch.device("cuda:0")
UR = 2.0 ** -24  # FP32 unit roundoff


def _run(fn, seed, S, params, n):
    h = B.Handle(seed, S)
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    w = torch.empty(n, dtype=torch.int32, device=DEV)
    getattr(B, "brng_" + fn)(h.h, *[torch.from_numpy(np.ascontiguousarray(p)).to(DEV) for p in params], out, w)
    torch.cuda.synchronize()
    code, cnt = h.counters()
    pos = h.positions()
    h.close()
    return out.cpu().numpy().astype(np.float64), w.cpu().numpy().view(np.uint32), pos, code, cnt


def _bisect(f, lo, hi, target, iters=90):
    """The root of the decreasing function f - target on [lo, hi]."""
    for _ in range(iters):
        mid = 0.5 * (lo + hi)
        if f(mid) > target:
            lo = mid
        else:
            hi = mid
    return 0.5 * (lo + hi)


def _f32_near(x, d_of, want):
    """Of the float32 values within 4 ulp of x, the one whose distance d_of
    is closest to want."""
    x = np.float32(x)
    cands = [x]
    up = dn = x
    for _ in range(4):
        up = np.nextafter(up, np.float32(np.inf))
        dn = np.nextafter(dn, np.float32(0))
        cands += [up, dn]
    return min(cands, key=lambda c: abs(d_of(float(c)) - want))


def test_poisson_draws_between_the_fp32_and_double_single_bands():
    seed, S, per = 91, 32, 16
    n = S * per
    rng = np.random.default_rng(11)
    lam = np.full(n, 3.0, np.float32)
    chosen = 0
    for i in range(n):
        u = float(O.elements(seed, O.DOM_U, i % S, i // S, 1)[0][0])
        k = int(rng.integers(6, 14))
        sgn = 1.0 if rng.random() < 0.5 else -1.0  # u below F(k) (draw k) or above it (draw k + 1)
        kf = k if sgn > 0 else k + 1  # the draw, which sets the FP32 band
        lo_d, hi_d = 16.0 * UR, (8.0 + 5.0 * kf) * UR  # DS certain beyond 12 u; FP32 uncertain below (12 + 5k) u
        want = 0.5 * (lo_d + hi_d)
        target = u * (1.0 + sgn * want)
        if not (stats.poisson.cdf(k, 64.0) < target < stats.poisson.cdf(k, 1e-3)):
            continue
        lm = _bisect(lambda x: stats.poisson.cdf(k, x), 1e-3, 64.0, target)
        d_of = lambda x: sgn * (stats.poisson.cdf(k, x) - u) / stats.poisson.cdf(k, x)  # noqa: E731
        lf = _f32_near(lm, d_of, want)
        if lo_d <= d_of(float(lf)) <= hi_d:
            lam[i] = lf
            chosen += 1
    assert chosen > n // 2
    out, w, pos, code, cnt = _run("poisson", seed, S, [lam], n)
    assert code == B.BRNG_OK, cnt
    ro, rw, rpos, _ = O.poisson(seed, S, lam)
    assert np.array_equal(out, ro)
    assert np.array_equal(w, rw) and np.array_equal(pos, rpos)
    assert cnt["n_recheck"] == 0, cnt  # the double-single tier decided them all


def test_binomial_draws_between_the_fp32_and_double_single_bands():
    seed, S, per = 92, 32, 16
    n = S * per
    rng = np.random.default_rng(12)
    trials = rng.integers(20, 200, n).astype(np.float32)
    prob = np.full(n, 0.01, np.float32)
    chosen = 0
    for i in range(n):
        u = float(O.elements(seed, O.DOM_U, i % S, i // S, 1)[0][0])
        t = int(trials[i])
        k = int(rng.integers(4, 13))
        sgn = 1.0 if rng.random() < 0.5 else -1.0
        kf = k if sgn > 0 else k + 1
        target = u * (1.0 + sgn * 40.0 * UR)
        if not (stats.binom.cdf(k, t, 0.5) < target < stats.binom.cdf(k, t, 1e-6)):
            continue
        q = _bisect(lambda x: stats.binom.cdf(k, t, x), 1e-6, 0.5, target)
        a = abs(t * np.log1p(-q))
        # DS certain beyond (9|a| + 12) u, FP32 uncertain below (3|a| + 12 + 8k) u
        lo_d, hi_d = (9.0 * a + 14.0) * UR, (3.0 * a + 10.0 + 8.0 * kf) * UR
        if not lo_d < hi_d or t * q > 64.0:
            continue
        want = 0.5 * (lo_d + hi_d)
        q = _bisect(lambda x: stats.binom.cdf(k, t, x), 1e-6, 0.5, u * (1.0 + sgn * want))
        d_of = lambda x: sgn * (stats.binom.cdf(k, t, x) - u) / stats.binom.cdf(k, t, x)  # noqa: E731
        qf = _f32_near(q, d_of, want)
        if lo_d <= d_of(float(qf)) <= hi_d:
            prob[i] = qf
            chosen += 1
    assert chosen > n // 8
    out, w, pos, code, cnt = _run("binomial", seed, S, [trials, prob], n)
    assert code == B.BRNG_OK, cnt
    ro, rw, rpos, _ = O.binomial(seed, S, trials, prob)
    assert np.array_equal(out, ro)
    assert np.array_equal(w, rw) and np.array_equal(pos, rpos)
    assert cnt["n_recheck"] == 0, cnt
