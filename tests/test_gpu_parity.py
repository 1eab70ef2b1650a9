"""Parity of the CUDA path (through the C ABI) with the FP64 oracle.

Bars:
  * integer work -- Philox words, first-consumed words, stream positions
    (hence every Gamma accept decision and attempt count) -- bit-exact;
  * FP64 paths -- the triangle Gibbs sampler of Eq. 1 and the FP64
    elementary functions of the Gamma recheck -- bit-exact;
  * FP32 transforms within 2e-6 relative error of the FP64 oracle fed the same
    Philox bits.  "Relative" is to the magnitude the FP32 arithmetic works
    at: |a|+|b| for a+(b-a)U, |mu|+|sigma z| for mu+sigma z, and the result
    times its conditioning for results built through a power or a
    logarithm (the oracle reports the Gamma's 3|cz|/t and boost exponent
    |ln(u_b)/alpha|, the Weibull exponent |ln(E)/k|, the Dirichlet log-Gammas);
    results below FLT_MIN compare absolutely (2 FLT_MIN).
Sizes span several warps and a ragged tail; the full-size workloads are
checked on sampled streams/chains the oracle recomputes one by one.
"""
import os

import numpy as np
import pytest

import oracle as O
from paper_1412_4825_gb300 import inputs

import gibbs_bounds

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():  # collected on a CPU host only with -m gpu
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_4825_gb300 import brng as B  # noqa: E402

DEV = torch.device("cuda:0")
FLT_MIN = float(np.finfo(np.float32).tiny)
RTOL = 2e-6
NT = os.cpu_count() or 1


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def H(t):
    return t.detach().cpu().numpy()


def words_np(t):
    return H(t).view(np.uint32)


def assert_close(got, want, scale, rtol=RTOL, what=""):
    got = np.asarray(got, np.float64).ravel()
    want = np.asarray(want, np.float64).ravel()
    scale = np.asarray(scale, np.float64)
    scale = scale.ravel() if scale.size == want.size else np.broadcast_to(scale, want.shape)
    nan_ok = np.isnan(got) & np.isnan(want)
    err = np.abs(got - want)
    bound = rtol * scale + 2 * FLT_MIN
    bad = ~nan_ok & ~(err <= bound)
    norm = np.where(nan_ok, 0.0, err / np.maximum(bound, 1e-300))
    print("%s: max err/bound = %.3g over %d values" % (what, np.nanmax(norm) if norm.size else 0, got.size))
    assert not bad.any(), "%s: %d mismatches, idx %s got %s want %s scale %s" % (
        what, bad.sum(), np.nonzero(bad)[0][:4], got[bad][:4], want[bad][:4], scale[bad][:4])


def handle(seed, S, buf_len=0, **tune):
    h = B.Handle(seed, S, buf_len)
    if tune:
        h.tune(**tune)
    return h


# ---- core engine and FP64 recheck functions ---------------------------------

@pytest.mark.parametrize("domain", [0, 1, 2, 3, 4])
def test_philox_words_bit_exact(domain):
    h = handle(0xDEADBEEF12345678, 1)
    for stream_id, first in [(0, 0), (7, 12345), (2**32 - 1, 2**32 - 3)]:
        n = 1001
        out = torch.empty(4 * n, dtype=torch.int32, device=DEV)
        B.brng_philox_words(h.h, domain, stream_id, first, n, out)
        ref = O.philox_words(0xDEADBEEF12345678, domain, stream_id, first, n)
        assert np.array_equal(words_np(out), ref)


def test_fp64_log_bit_exact_exhaustive():
    k = np.arange(1 << 24, dtype=np.float64)
    rng = np.random.default_rng(1)
    t = rng.uniform(0.05, 2.5, 1 << 20)
    x = np.concatenate([(k + 1) * 2.0**-24, t * t * t, np.exp(rng.uniform(-700, 700, 1 << 16)),
                        [5e-324, 1e-310, 2.2250738585072014e-308, 1.0, 2.0, 0.5]])
    out = torch.empty(x.size, dtype=torch.float64, device=DEV)
    B.brng_fp64_eval(0, T(x), out)
    assert np.array_equal(H(out).view(np.int64), O.log(x).view(np.int64))


def test_fp64_sincospi_bit_exact_exhaustive():
    a = np.arange(1 << 24, dtype=np.float64) * 2.0**-23
    s_ref, c_ref = O.sincospi(a)
    out = torch.empty(a.size, dtype=torch.float64, device=DEV)
    B.brng_fp64_eval(1, T(a), out)
    assert np.array_equal(H(out).view(np.int64), s_ref.view(np.int64))
    B.brng_fp64_eval(2, T(a), out)
    assert np.array_equal(H(out).view(np.int64), c_ref.view(np.int64))


def _ulp32(v):
    return np.spacing(np.abs(v).astype(np.float32)).astype(np.float64)


def test_fp32_log_error_bound():
    """The FP32 log of the base conversions (no conversion instructions):
    within 4 ulp of the true value over every U' the buffers produce and over
    the t = 1 + cz and d v ranges of the Gamma test."""
    k = np.arange(1 << 24, dtype=np.float64)
    rng = np.random.default_rng(2)
    x = np.concatenate([(k + 1) * 2.0**-24, rng.uniform(0.05, 3.0, 1 << 20),
                        np.exp(rng.uniform(-30, 30, 1 << 18))]).astype(np.float32)
    out = torch.empty(x.size, dtype=torch.float32, device=DEV)
    B.brng_fp32_eval(0, T(x), out)
    ref = O.log(x.astype(np.float64))
    err = np.abs(H(out).astype(np.float64) - ref)
    ratio = err / np.maximum(_ulp32(ref), 1e-45)
    print("flog max error %.2f ulp" % ratio.max())
    assert ratio.max() <= 4.0
    assert H(out)[(1 << 24) - 1] == 0.0  # log 1 = 0 exactly


def test_fp32_sincospi_error_bound():
    """sin/cos of pi k 2^-23 over every 24-bit k (every Box-Muller angle):
    within 2 ulp of the true value; exact at multiples of pi/2."""
    k = np.arange(1 << 24, dtype=np.float32)
    s_ref, c_ref = O.sincospi(np.arange(1 << 24, dtype=np.float64) * 2.0**-23)
    out = torch.empty(k.size, dtype=torch.float32, device=DEV)
    for fn, ref in ((1, s_ref), (2, c_ref)):
        B.brng_fp32_eval(fn, T(k), out)
        g = H(out).astype(np.float64)
        ratio = np.abs(g - ref) / np.maximum(_ulp32(ref), 1e-45)
        print("sincospi fn %d max error %.2f ulp" % (fn, ratio.max()))
        assert ratio.max() <= 2.0
        for q in range(4):
            assert g[q << 22] == np.round(ref[q << 22])


# ---- varying-parameter streams ----------------------------------------------

def _params(fn, n, seed):
    if fn == "uniform":
        return list(inputs.uniform_params(n, seed))
    if fn in ("normal", "laplace"):
        return list(inputs.normal_params(n, seed))
    if fn == "exponential":
        return [inputs.rate_params(n, seed)]
    if fn == "gamma":
        return [inputs.shape_params(n, seed)]
    if fn == "weibull":
        return [inputs.log_uniform(np.random.default_rng(seed), 0.5, 5.0, n), inputs.rate_params(n, seed + 1)]
    raise ValueError(fn)


def _scale(fn, out, params, cond=None):
    """Magnitude the FP32 arithmetic of `fn` works at (see the module doc)."""
    out = np.abs(out)
    if fn == "uniform":
        return np.maximum(np.abs(params[0]), np.abs(params[1])).astype(np.float64)
    if fn in ("normal", "laplace"):
        mu = np.abs(params[0].astype(np.float64))
        return mu + np.abs(out - mu)
    if fn == "exponential":
        return out
    return out * np.maximum(1.0, cond)


def _run_bulk(fn, h, params, n, words=True):
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    w = torch.empty(n, dtype=torch.int32, device=DEV) if words else None
    getattr(B, "brng_" + fn)(h.h, *[T(p) for p in params], out, w)
    return out, w


BULK = ["uniform", "normal", "exponential", "gamma", "laplace", "weibull"]


@pytest.mark.parametrize("fn", BULK)
def test_bulk_parity(fn):
    seed, S, n = 42, 1000, 20011  # 31.25 warps of streams; 20 or 21 draws each
    params = _params(fn, n, 7)
    h = handle(seed, S)
    out, w = _run_bulk(fn, h, params, n)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    res = getattr(O, fn)(seed, S, *params, **({"with_cond": True} if fn in ("gamma", "weibull") else {}))
    ro, rw, rpos = res[0], res[1], res[2]
    cond = res[4] if fn in ("gamma", "weibull") else None
    assert np.array_equal(words_np(w), rw)
    assert np.array_equal(h.positions(), rpos)
    g = H(out).astype(np.float64)
    if fn in ("normal", "laplace"):
        mu = params[0].astype(np.float64)
        scale = np.abs(mu) + np.abs(ro - mu)
    else:
        scale = _scale(fn, ro, params, cond)
    assert_close(g, ro, scale, what=fn)


def _uniform_f64_gpu(h, a, b):
    n = len(a)
    out = torch.empty(n, dtype=torch.float64, device=DEV)
    w = torch.empty(n, dtype=torch.int32, device=DEV)
    B.brng_uniform_f64(h.h, T(a), T(b), out, w)
    return out, w


@pytest.mark.parametrize("S,n", [(1000, 20011), (1, 77), (4099, 4099), (64, 1 << 16)])
def test_uniform_f64_bit_exact(S, n):
    """FP64 uniform from the U64 domain: values, words and U64 positions equal
    the oracle's bit for bit (ragged draws per stream, odd start positions
    through the checkpoint call, invalid parameters), and the U, N, E
    positions stay untouched."""
    rng = np.random.default_rng(S + n)
    a = rng.uniform(-1e3, 1e3, n)
    b = a + rng.exponential(10.0, n)
    a[::97] = b[::97]          # a == b
    b[5::211] = a[5::211] - 1  # b < a: invalid
    a[7::307] = np.nan
    h = handle(42, S)
    start = rng.integers(0, 1 << 40, S).astype(np.uint64)
    h.set_positions_u64(start)
    out, w = _uniform_f64_gpu(h, a, b)
    ro, rw, rpos, st = O.uniform_f64(42, S, a, b, start)
    code, cnt = h.counters()
    assert code == (B.BRNG_EDOMAIN if st == O.EDOMAIN else B.BRNG_OK)
    g = H(out)
    assert np.array_equal(np.isnan(g), np.isnan(ro))
    assert np.array_equal(g[~np.isnan(g)].view(np.uint64), ro[~np.isnan(ro)].view(np.uint64))
    assert np.array_equal(words_np(w), rw)
    assert np.array_equal(h.positions_u64(), rpos)
    assert not h.positions().any()


def test_uniform_f64_special_parameters():
    """The validity rule (finite a <= b, taken on the bit patterns on the
    GPU) agrees with the oracle on signed zeros, subnormals, infinities, NaN
    and the largest finite values, in every pairing."""
    sp = np.array([0.0, -0.0, 5e-324, -5e-324, 2.2e-308, -2.2e-308, 1.0, -1.0, 1e308, -1e308,
                   np.inf, -np.inf, np.nan])
    a, b = np.repeat(sp, sp.size), np.tile(sp, sp.size)
    h = handle(3, 7)
    out, w = _uniform_f64_gpu(h, a, b)
    ro, rw, rpos, st = O.uniform_f64(3, 7, a, b)
    g = H(out)
    assert np.array_equal(np.isnan(g), np.isnan(ro))
    assert np.array_equal(g[~np.isnan(g)].view(np.uint64), ro[~np.isnan(ro)].view(np.uint64))
    assert np.array_equal(words_np(w), rw) and np.array_equal(h.positions_u64(), rpos)
    code, cnt = h.counters()
    assert cnt["n_domain"] == int(np.isnan(ro).sum())


def test_uniform_f64_call_splitting_and_full_size_sampled():
    """Two calls continue every stream; at 2^26 draws over 2^20 streams a
    sample of whole streams equals the oracle."""
    S = 333
    rng = np.random.default_rng(5)
    a = rng.uniform(0, 1, 3 * S + 17)
    b = a + 1.0
    h = handle(9, S)
    o1, w1 = _uniform_f64_gpu(h, a[: 2 * S], b[: 2 * S])
    o2, w2 = _uniform_f64_gpu(h, a[2 * S:], b[2 * S:])
    r1 = O.uniform_f64(9, S, a[: 2 * S], b[: 2 * S])
    r2 = O.uniform_f64(9, S, a[2 * S:], b[2 * S:], r1[2])
    assert np.array_equal(H(o1), r1[0]) and np.array_equal(H(o2), r2[0])
    assert np.array_equal(words_np(w2), r2[1]) and np.array_equal(h.positions_u64(), r2[2])
    S, n = 1 << 20, 1 << 26
    a = torch.zeros(n, dtype=torch.float64, device=DEV)
    b = torch.ones(n, dtype=torch.float64, device=DEV)
    out = torch.empty(n, dtype=torch.float64, device=DEV)
    h = handle(42, S)
    B.brng_uniform_f64(h.h, a, b, out)
    torch.cuda.synchronize()
    pos = h.positions_u64()
    assert np.all(pos == n // S)
    for s in [0, 1, 12345, S - 1]:
        vals, _ = O.elements(42, O.DOM_U64, s, 0, n // S)
        assert np.array_equal(H(out[s::S]), vals)


@pytest.mark.parametrize("case", range(12))
def test_bulk_random_configurations(case):
    """Seeded random configurations of the bulk calls: distribution, seed,
    stream count, draw count, ring length, warps per block and a split of the
    draws into two calls (each call maps its draw i to stream i mod S and
    continues the streams): words and positions bit-exact, values within the
    tolerance of the module doc."""
    rng = np.random.default_rng(1000 + case)
    fn = BULK[case % len(BULK)]
    S = int(rng.integers(1, 3000))
    n = int(rng.integers(1, 40000))
    seed = int(rng.integers(0, 2**63))
    h = handle(seed, S, buf_len=int(rng.choice([4, 8, 16, 32, 64, 128])),
               warps_per_block=int(rng.choice([1, 2, 4, 8, 16])))
    params = _params(fn, n, case + 50)
    cut = int(rng.integers(0, n + 1))
    parts = [[p[:cut] for p in params], [p[cut:] for p in params]]
    outs, ws = [], []
    pos = None
    refs = []
    for part in parts:
        m = len(part[0])
        if m == 0:
            continue
        o, w = _run_bulk(fn, h, part, m)
        outs.append(H(o).astype(np.float64))
        ws.append(words_np(w))
        kw = {"with_cond": True} if fn in ("gamma", "weibull") else {}
        r = getattr(O, fn)(seed, S, *part, pos=pos, **kw)
        pos = r[2]
        refs.append(r)
    assert np.array_equal(np.concatenate(ws), np.concatenate([r[1] for r in refs]))
    assert np.array_equal(h.positions(), pos)
    ro = np.concatenate([r[0] for r in refs])
    cond = np.concatenate([r[4] for r in refs]) if fn in ("gamma", "weibull") else None
    if fn in ("normal", "laplace"):
        mu = params[0].astype(np.float64)
        scale = np.abs(mu) + np.abs(ro - mu)
    else:
        scale = _scale(fn, ro, params, cond)
    assert_close(np.concatenate(outs), ro, scale, what="%s random case %d" % (fn, case))


def test_gamma_decisions_many():
    """4M Gamma draws over alpha in [0.05, 500] and near 1: every attempt
    count (hence every accept decision) equals the oracle's."""
    seed, S, n = 9, 1 << 14, 1 << 22
    rng = np.random.default_rng(3)
    alpha = np.exp(rng.uniform(np.log(0.05), np.log(500.0), n)).astype(np.float32)
    alpha[::7] = np.float32(1.0)
    alpha[1::7] = np.nextafter(np.float32(1.0), np.float32(0.0))
    h = handle(seed, S)
    out, w = _run_bulk("gamma", h, [alpha], n)
    code, cnt = h.counters()
    assert code == B.BRNG_OK
    ro, rw, rpos, _, cond = O.gamma(seed, S, alpha, with_cond=True)
    assert np.array_equal(h.positions(), rpos)
    assert np.array_equal(words_np(w), rw)
    assert_close(H(out), ro, np.abs(ro) * np.maximum(1.0, cond), what="gamma 4M")
    print("rechecks", cnt)
    # FP32 decisions overturned in FP64 lie deep inside the tolerance band
    assert cnt["n_flip"] == 0 or cnt["max_flip_ratio"] < 0.25


@pytest.mark.parametrize("buf_len,wpb", [(4, 1), (16, 16), (128, 2), (256, 1)])
def test_bulk_tuning_invariance(buf_len, wpb):
    seed, S, n = 5, 333, 10000
    tag, p0, p1 = inputs.mixed_stream(n, seed=5, n_tags=6)
    outs = []
    for tune in [dict(), dict(buf_len=buf_len, warps_per_block=wpb)]:
        h = handle(seed, S, **tune)
        out = torch.empty(n, dtype=torch.float32, device=DEV)
        w = torch.empty(n, dtype=torch.int32, device=DEV)
        B.brng_mixed(h.h, T(tag), T(p0), T(p1), out, w)
        outs.append((H(out), words_np(w), h.positions()))
    for a, b in zip(outs[0], outs[1]):
        assert np.array_equal(a.view(np.uint32) if a.dtype == np.float32 else a,
                              b.view(np.uint32) if b.dtype == np.float32 else b)


def test_call_splitting():
    seed, S = 11, 64
    n1, n2 = 64 * 7 + 5, 64 * 9 + 33
    alpha = inputs.shape_params(n1 + n2, seed=2)
    h = handle(seed, S)
    o1, w1 = _run_bulk("gamma", h, [alpha[:n1]], n1)
    o2, w2 = _run_bulk("gamma", h, [alpha[n1:]], n2)
    pos1 = O.new_positions(S)
    r1 = O.gamma(seed, S, alpha[:n1])
    r2 = O.gamma(seed, S, alpha[n1:], pos=r1[2])
    assert np.array_equal(words_np(w1), r1[1]) and np.array_equal(words_np(w2), r2[1])
    assert np.array_equal(h.positions(), r2[2])
    # checkpoint / resume of positions
    h2 = handle(seed, S)
    h2.set_positions(r1[2])
    o2b, w2b = _run_bulk("gamma", h2, [alpha[n1:]], n2)
    assert np.array_equal(words_np(w2b), r2[1])
    assert np.array_equal(H(o2b).view(np.uint32), H(o2).view(np.uint32))
    del pos1


# ---- Poisson (discrete; counts must equal the oracle's exactly) -------------

def test_fp64_exp_bit_exact():
    rng = np.random.default_rng(12)
    x = np.concatenate([rng.uniform(-708.0, 0.0, 1 << 16), -rng.uniform(0.0, 64.0, 1 << 16),
                        [0.0, -1e-300, -64.0, -708.0]])
    out = torch.empty(x.size, dtype=torch.float64, device=DEV)
    B.brng_fp64_eval(3, T(x), out)
    assert np.array_equal(H(out).view(np.uint64), O.exp(x).view(np.uint64))


@pytest.mark.parametrize("lo,hi", [(0.05, 64.0), (0.001, 0.5), (30.0, 64.0)])
def test_poisson_parity(lo, hi):
    seed, S, n = 42, 1000, 200011
    lam = inputs.poisson_params(n, seed=3, lo=lo, hi=hi)
    h = handle(seed, S)
    out, w = _run_bulk("poisson", h, [lam], n)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    ro, rw, rpos, _ = O.poisson(seed, S, lam)
    assert np.array_equal(H(out).astype(np.float64), ro)
    assert np.array_equal(words_np(w), rw)
    assert np.array_equal(h.positions(), rpos)
    print("poisson rechecks", cnt["n_recheck"])


def test_poisson_near_cdf_steps_redraw_in_fp64():
    """Lambdas chosen so that each draw's uniform sits next to a step of the
    Poisson CDF (within a few 2^-24): the FP32 search cannot certify those
    comparisons and redraws in FP64; every count still equals the oracle's."""
    from scipy import stats
    seed, S, per = 77, 32, 8
    n = S * per
    rng = np.random.default_rng(1)
    lam = np.empty(n, np.float32)
    for i in range(n):
        s_, m = i % S, i // S
        u = float(O.elements(seed, O.DOM_U, s_, m, 1)[0][0])
        k = int(rng.integers(0, 12))
        if not (stats.poisson.cdf(k, 64.0) < u < stats.poisson.cdf(k, 1e-3)):
            lam[i] = np.float32(3.0)
            continue
        lo, hi = 1e-3, 64.0  # F(k; lambda) falls from ~1 to ~0 as lambda grows
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            if stats.poisson.cdf(k, mid) > u:
                lo = mid
            else:
                hi = mid
        lam[i] = np.float32(lo)
    h = handle(seed, S)
    out, w = _run_bulk("poisson", h, [lam], n)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    ro, rw, rpos, _ = O.poisson(seed, S, lam)
    assert np.array_equal(H(out).astype(np.float64), ro)
    assert np.array_equal(words_np(w), rw)
    assert np.array_equal(h.positions(), rpos)
    assert cnt["n_recheck"] > n // 4, cnt  # the FP64 path ran


def test_mixed_with_discrete_tags():
    seed, S, n = 42, 2048, 100003
    tag, p0, p1 = inputs.mixed_stream(n, seed=seed, n_tags=8)
    assert (tag == 6).any() and (tag == 7).any()
    h = handle(seed, S)
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    w = torch.empty(n, dtype=torch.int32, device=DEV)
    B.brng_mixed(h.h, T(tag), T(p0), T(p1), out, w)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    ro, rw, rpos, _, cond = O.mixed(seed, S, tag, p0, p1, nthreads=NT, with_cond=True)
    assert np.array_equal(words_np(w), rw)
    assert np.array_equal(h.positions(), rpos)
    pois = (tag == 6) | (tag == 7)  # discrete: counts exact
    assert np.array_equal(H(out)[pois].astype(np.float64), ro[pois])
    rest = ~pois
    assert_close(H(out)[rest], ro[rest], _mixed_scale(tag[rest], p0[rest], p1[rest], ro[rest], cond[rest]),
                 what="mixed with Poisson")


@pytest.mark.parametrize("lo,hi,S", [(64.0, 1e6, 1000), (0.05, 1e7, 777), (60.0, 70.0, 64)])
def test_poisson_large_means_bit_exact(lo, hi, S):
    """Means above 64 take PTRS (FP64 transformed rejection, 2 U per attempt):
    every count, first word and stream position equals the oracle's, across
    the switch at 64 and up to lambda = 1e7."""
    seed, n = 42, 100003
    lam = inputs.poisson_params(n, seed=11, lo=lo, hi=hi)
    h = handle(seed, S)
    out, w = _run_bulk("poisson", h, [lam], n)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    ro, rw, rpos, _ = O.poisson(seed, S, lam)
    assert np.array_equal(H(out).astype(np.float64), ro)
    assert np.array_equal(words_np(w), rw)
    assert np.array_equal(h.positions(), rpos)


@pytest.mark.parametrize("max_trials,S", [(1 << 24, 1000), (3000, 513)])
def test_binomial_large_means_bit_exact(max_trials, S):
    """n min(p, 1-p) above 64 takes BTRD (1 or 2 U per attempt, recursion,
    log squeeze and the Stirling test, FP64): counts, words and positions
    bit-exact, reflected (p > 1/2) draws included."""
    seed, n = 42, 100003
    rng = np.random.default_rng(12)
    trials = np.floor(np.exp(rng.uniform(0.0, np.log(max_trials), n))).astype(np.float32)
    prob = rng.random(n).astype(np.float32)
    prob[::5] = np.float32(0.5)
    h = handle(seed, S)
    out, w = _run_bulk("binomial", h, [trials, prob], n)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    ro, rw, rpos, _ = O.binomial(seed, S, trials, prob)
    assert (trials.astype(np.float64) * np.minimum(prob, 1 - prob) > 64).mean() > 0.2  # both paths run
    assert np.array_equal(H(out).astype(np.float64), ro)
    assert np.array_equal(words_np(w), rw)
    assert np.array_equal(h.positions(), rpos)


@pytest.mark.parametrize("which", ["poisson", "binomial", "poisson_small", "binomial_small"])
def test_large_means_full_size_sampled(which):
    """The bench's discrete lines in their launch configuration, 2^26 draws
    over 2^20 streams: Poisson with lambda log-uniform [64, 1e6] (PTRS) and
    Binomial with n log-uniform integers to 2^24 and p uniform (BTRD above
    mean 64, inversion below), ring 8, 4 warps per block; Poisson with lambda
    log-uniform [0.05, 64] and Binomial with n to 1,000, means capped below 64
    (the resumable inversion searches), ring 8, 2 warps per block.  4,096
    whole streams recomputed by the oracle: counts, first words and positions
    bit-exact."""
    seed, S, n = 42, 1 << 20, 1 << 26
    g = torch.Generator(device=DEV)
    g.manual_seed(3)
    wpb = 4
    if which == "poisson":
        p0 = torch.exp(np.log(64.0) + np.log(1e6 / 64.0) * torch.rand(n, generator=g, device=DEV)).contiguous()
        p1 = torch.zeros_like(p0)
    elif which == "poisson_small":
        p0 = torch.exp(np.log(0.05) + np.log(64 / 0.05) * torch.rand(n, generator=g, device=DEV)).contiguous()
        p1 = torch.zeros_like(p0)
        wpb = 2
    elif which == "binomial":
        p0 = torch.floor(torch.exp(np.log(2.0 ** 24) * torch.rand(n, generator=g, device=DEV))).contiguous()
        p1 = torch.rand(n, generator=g, device=DEV).contiguous()
    else:
        p0 = torch.floor(torch.exp(np.log(1001.0) * torch.rand(n, generator=g, device=DEV)))
        pr = torch.rand(n, generator=g, device=DEV)
        q = torch.minimum(pr, 1.0 - pr)
        cap = 0.999 * 64.0 / torch.clamp(p0, min=1.0)
        p1 = torch.where(p0 * q > 64.0, torch.where(pr <= 0.5, cap, 1.0 - cap), pr).contiguous()
        p0 = p0.contiguous()
        wpb = 2
    tag = 6 if which.startswith("poisson") else 7
    which = which.split("_")[0]
    h = handle(seed, S, 8, warps_per_block=wpb)
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    w = torch.empty(n, dtype=torch.int32, device=DEV)
    if which == "poisson":
        B.brng_poisson(h.h, p0, out, w)
    else:
        B.brng_binomial(h.h, p0, p1, out, w)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    p0_h, p1_h, out_h, w_h = H(p0), H(p1), H(out), words_np(w)
    tags = np.full(n, tag, np.uint8)
    pos_gpu = h.positions().reshape(S, 3)
    starts = np.random.default_rng(10).choice(np.arange(1, S // 64 - 1), 62, replace=False) * 64
    ranges = [(0, 64), (S - 64, S)] + [(int(s0), int(s0) + 64) for s0 in starts]
    ro, rw, rpos, _ = O.mixed(seed, S, tags, p0_h, p1_h, streams=ranges)
    sel = np.concatenate([np.arange(s0, s1) for s0, s1 in ranges])
    idx = (np.arange(n // S)[:, None] * S + sel[None, :]).ravel()
    assert np.array_equal(out_h[idx].astype(np.float64), ro[idx])
    assert np.array_equal(w_h[idx], rw[idx])
    assert np.array_equal(pos_gpu[sel], rpos.reshape(S, 3)[sel])
    print("%s: %d attempts or draws redone in FP64 over %d draws" % (which, cnt["n_recheck"], n))


def test_mixed_with_large_discrete_means():
    """All eight tags, Poisson means log-uniform up to 1e6 and Binomial trials
    up to 2^24: discrete counts exact, continuous values within tolerance."""
    seed, S, n = 42, 2048, 100003
    tag, p0, p1 = inputs.mixed_stream(n, seed=seed, n_tags=8)
    rng = np.random.default_rng(13)
    big = rng.random(n) < 0.5
    p0 = p0.copy()
    p1 = p1.copy()
    sel = (tag == 6) & big
    p0[sel] = inputs.log_uniform(rng, 64.0, 1e6, int(sel.sum()))
    sel = (tag == 7) & big
    p0[sel] = np.floor(inputs.log_uniform(rng, 130.0, 1.6e7, int(sel.sum())))
    h = handle(seed, S)
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    w = torch.empty(n, dtype=torch.int32, device=DEV)
    B.brng_mixed(h.h, T(tag), T(p0), T(p1), out, w)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    ro, rw, rpos, _, cond = O.mixed(seed, S, tag, p0, p1, nthreads=NT, with_cond=True)
    assert np.array_equal(words_np(w), rw)
    assert np.array_equal(h.positions(), rpos)
    disc = (tag == 6) | (tag == 7)
    assert np.array_equal(H(out)[disc].astype(np.float64), ro[disc])
    rest = ~disc
    assert_close(H(out)[rest], ro[rest], _mixed_scale(tag[rest], p0[rest], p1[rest], ro[rest], cond[rest]),
                 what="mixed with large discrete means")


def test_buffer_waste_counter():
    """n_wasted counts the ring elements generated but unused when a call ends
    (Sec. 2.4's buffer-length trade-off): at most one ring per stream and
    domain, more for longer rings, and none that the next call loses (it
    restarts each stream at its position, bit-exact as the parity tests show)."""
    S, n = 1000, 20011
    a, b = inputs.uniform_params(n, seed=3)
    waste = {}
    for buf_len in (8, 64):
        h = handle(7, S, buf_len=buf_len)
        _run_bulk("uniform", h, [a, b], n)
        code, cnt = h.counters()
        assert code == B.BRNG_OK
        waste[buf_len] = cnt["n_wasted"]
        assert 0 < cnt["n_wasted"] <= S * buf_len
    assert waste[64] > waste[8]
    nobs, xbar, sc = inputs.normal_gamma_data(333, seed=2)
    for buf_len in (8, 32):
        st, m, cnt = _ng_gpu(nobs, xbar, sc, 50, buf_len=buf_len)
        assert 0 < cnt["n_wasted"] <= 333 * 2 * buf_len


def test_poisson_invalid_lambda():
    lam = np.array([1.0, 0.0, -2.0, np.nan, np.inf, 2.0e7, 3.0], np.float32)
    h = handle(2, 1)
    out, w = _run_bulk("poisson", h, [lam], lam.size)
    code, cnt = h.counters()
    assert code == B.BRNG_EDOMAIN and cnt["n_domain"] == 5
    ro, rw, rpos, _ = O.poisson(2, 1, lam)
    g = H(out).astype(np.float64)
    assert np.isnan(g[1:6]).all() and np.array_equal(g[[0, 6]], ro[[0, 6]])
    assert np.array_equal(h.positions(), rpos)


def test_binomial_parity():
    seed, S, n = 42, 1000, 200011
    trials, prob = inputs.binomial_params(n, seed=4)
    h = handle(seed, S)
    out, w = _run_bulk("binomial", h, [trials, prob], n)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    ro, rw, rpos, _ = O.binomial(seed, S, trials, prob)
    assert np.array_equal(H(out).astype(np.float64), ro)
    assert np.array_equal(words_np(w), rw)
    assert np.array_equal(h.positions(), rpos)
    print("binomial rechecks", cnt["n_recheck"])


def test_binomial_near_cdf_steps_redraw_in_fp64():
    """Probabilities chosen so that each draw's uniform sits next to a step
    of the Binomial CDF: those draws are redone in FP64; every count still
    equals the oracle's."""
    from scipy import stats
    seed, S, per = 78, 32, 8
    n = S * per
    rng = np.random.default_rng(2)
    trials = rng.integers(1, 120, n).astype(np.float32)
    prob = np.full(n, 0.25, np.float32)
    for i in range(n):
        s_, m = i % S, i // S
        u = float(O.elements(seed, O.DOM_U, s_, m, 1)[0][0])
        t = int(trials[i])
        k = int(rng.integers(0, min(t, 20) + 1))
        lo, hi = 0.0, 0.5  # F(k; t, q) falls as q grows
        if not (stats.binom.cdf(k, t, hi) < u < stats.binom.cdf(k, t, lo)):
            continue
        for _ in range(80):
            mid = 0.5 * (lo + hi)
            if stats.binom.cdf(k, t, mid) > u:
                lo = mid
            else:
                hi = mid
        if t * lo <= 64.0:
            prob[i] = np.float32(lo)
    h = handle(seed, S)
    out, w = _run_bulk("binomial", h, [trials, prob], n)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    ro, rw, rpos, _ = O.binomial(seed, S, trials, prob)
    assert np.array_equal(H(out).astype(np.float64), ro)
    assert np.array_equal(words_np(w), rw)
    assert cnt["n_recheck"] > n // 4, cnt  # the FP64 path ran


def test_discrete_extremes():
    """Largest allowed means and trials, tiny means, p at 0 and 1."""
    S = 64
    lam = np.array([64.0, 1e-30, 63.999, 32.0] * 256, np.float32)
    h = handle(5, S)
    out, w = _run_bulk("poisson", h, [lam], lam.size)
    ro, rw, rpos, st = O.poisson(5, S, lam)
    assert st == O.OK and np.array_equal(H(out).astype(np.float64), ro)
    assert np.all(ro[1::4] == 0)
    trials = np.array([16777216, 16777216, 1000, 128, 7, 0] * 200, np.float32)
    prob = np.array([3.8e-6, 1 - 3.8e-6, 0.0639, 0.5, 1.0, 0.3] * 200, np.float32)
    h = handle(6, S)
    out, w = _run_bulk("binomial", h, [trials, prob], trials.size)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    ro, rw, rpos, st = O.binomial(6, S, trials, prob)
    assert st == O.OK and np.array_equal(H(out).astype(np.float64), ro)
    assert np.array_equal(words_np(w), rw) and np.array_equal(h.positions(), rpos)
    assert np.all(ro[4::6] == 7) and np.all(ro[5::6] == 0)


def test_normal_gamma_zero_sweeps():
    nobs, xbar, sc = inputs.normal_gamma_data(70, seed=2)
    st, m, _ = _ng_gpu(nobs, xbar, sc, 0)
    mu, tau, pn, pu = B.normal_gamma_unpack(st)
    assert np.all(pn == 0) and np.all(pu == 0) and np.all(H(m) == 0)


def test_binomial_invalid_parameters():
    trials = np.array([10, 2.5, -1, np.nan, 10, 10, 10, 2.0e7, 10], np.float32)
    prob = np.array([0.5, 0.5, 0.5, 0.5, -0.1, 1.5, np.nan, 0.5, 0.25], np.float32)
    h = handle(2, 1)
    out, w = _run_bulk("binomial", h, [trials, prob], trials.size)
    code, cnt = h.counters()
    assert code == B.BRNG_EDOMAIN and cnt["n_domain"] == 7
    ro, rw, rpos, _ = O.binomial(2, 1, trials, prob)
    g = H(out).astype(np.float64)
    assert np.isnan(g[1:8]).all() and np.array_equal(g[[0, 8]], ro[[0, 8]])
    assert np.array_equal(h.positions(), rpos)


def _mixed_scale(tag, p0, p1, ro, cond):
    p0 = p0.astype(np.float64)
    p1 = p1.astype(np.float64)
    sc = np.abs(ro) * np.maximum(1.0, cond)
    sc = np.where(tag == 0, np.maximum(np.abs(p0), np.abs(p1)), sc)
    sc = np.where((tag == 1) | (tag == 4), np.abs(p0) + np.abs(ro - p0), sc)
    sc = np.where(tag == 2, np.abs(ro), sc)
    return sc


def test_mixed_parity():
    seed, S, n = 42, 2048, 200003
    tag, p0, p1 = inputs.mixed_stream(n, seed=seed, n_tags=6)
    h = handle(seed, S)
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    w = torch.empty(n, dtype=torch.int32, device=DEV)
    B.brng_mixed(h.h, T(tag), T(p0), T(p1), out, w)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    ro, rw, rpos, _, cond = O.mixed(seed, S, tag, p0, p1, nthreads=NT, with_cond=True)
    assert np.array_equal(words_np(w), rw)
    assert np.array_equal(h.positions(), rpos)
    assert_close(H(out), ro, _mixed_scale(tag, p0, p1, ro, cond), what="mixed")


def test_mixed_dispatch_across_calls():
    """A call's kernel is picked on the device from its tags (the 96-register
    kernel when a Poisson or Binomial tag is present, the continuous-only one
    otherwise): calls that alternate between the two, on one handle, continue
    every stream exactly as one oracle run over the concatenated draws."""
    seed, S = 7, 1000
    parts = []
    for n_tags, n, sd in [(8, 30011, 1), (6, 20011, 2), (4, 25013, 3), (8, 10007, 4)]:
        tag, p0, p1 = inputs.mixed_stream(n, seed=sd, n_tags=n_tags)
        parts.append((tag, p0, p1))
    h = handle(seed, S)
    pos = O.new_positions(S)
    for tag, p0, p1 in parts:
        n = tag.size
        out = torch.empty(n, dtype=torch.float32, device=DEV)
        w = torch.empty(n, dtype=torch.int32, device=DEV)
        B.brng_mixed(h.h, T(tag), T(p0), T(p1), out, w)
        code, cnt = h.counters(reset=True)
        assert code == B.BRNG_OK, cnt
        ro, rw, pos, _, cond = O.mixed(seed, S, tag, p0, p1, pos=pos, nthreads=NT, with_cond=True)
        assert np.array_equal(words_np(w), rw)
        assert np.array_equal(h.positions(), pos)
        disc = (tag == 6) | (tag == 7)
        assert np.array_equal(H(out)[disc].astype(np.float64), ro[disc])
        rest = ~disc
        assert_close(H(out)[rest], ro[rest], _mixed_scale(tag[rest], p0[rest], p1[rest], ro[rest], cond[rest]),
                     what="mixed call with %d tags" % int(tag.max() + 1))


@pytest.mark.parametrize("offset,where", [(0, "tail"), (1, "tail"), (3, "head"), (0, "middle")])
def test_mixed_dispatch_finds_a_single_discrete_tag(offset, where):
    """The tag scan reads 16 tags per load when the array is 16-byte aligned
    and one at a time otherwise (and for the tail): a single Poisson tag
    anywhere, with the tag array at any byte offset, still selects the kernel
    with the discrete draws (the continuous-only one would report it as a
    domain error)."""
    seed, S, n = 11, 64, 4099
    tag, p0, p1 = inputs.mixed_stream(n, seed=5, n_tags=6)
    idx = {"tail": n - 1, "head": 0, "middle": n // 2}[where]
    tag = tag.copy()
    p0 = p0.copy()
    p1 = p1.copy()
    tag[idx], p0[idx], p1[idx] = 6, np.float32(3.5), np.float32(0.0)
    buf = torch.zeros(n + 16, dtype=torch.uint8, device=DEV)
    buf[offset:offset + n] = T(tag)
    tview = buf[offset:offset + n]
    assert (tview.data_ptr() % 16 == 0) == (offset == 0)
    h = handle(seed, S)
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    w = torch.empty(n, dtype=torch.int32, device=DEV)
    B.brng_mixed(h.h, tview, T(p0), T(p1), out, w)
    code, cnt = h.counters()
    assert code == B.BRNG_OK and cnt["n_domain"] == 0, cnt
    ro, rw, rpos, _ = O.mixed(seed, S, tag, p0, p1)
    assert H(out)[idx] == ro[idx] and np.array_equal(words_np(w), rw)
    assert np.array_equal(h.positions(), rpos)


def test_mixed_full_size_sampled():
    """2^28 draws over 2^20 streams (the mixed-stream workload); 4,096 whole
    streams recomputed by the oracle: the first and last 64 and 62 blocks of
    64 at seeded random offsets."""
    seed, S, n = 42, 1 << 20, 1 << 28
    tag, p0, p1 = inputs.mixed_stream_torch(n, seed=seed, device=DEV)
    h = handle(seed, S)
    out = torch.empty(n, dtype=torch.float32, device=DEV)
    w = torch.empty(n, dtype=torch.int32, device=DEV)
    B.brng_mixed(h.h, tag, p0, p1, out, w)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    tag_h, p0_h, p1_h = H(tag), H(p0), H(p1)
    out_h, w_h = H(out), words_np(w)
    pos_gpu = h.positions().reshape(S, 3)
    starts = np.random.default_rng(9).choice(np.arange(1, S // 64 - 1), 62, replace=False) * 64
    ranges = [(0, 64), (S - 64, S)] + [(int(s0), int(s0) + 64) for s0 in starts]
    ro, rw, rpos, _, cond = O.mixed(seed, S, tag_h, p0_h, p1_h, streams=ranges, with_cond=True)
    sel = np.concatenate([np.arange(s0, s1) for s0, s1 in ranges])
    idx = (np.arange(n // S)[:, None] * S + sel[None, :]).ravel()
    assert np.array_equal(w_h[idx], rw[idx])
    assert np.array_equal(pos_gpu[sel], rpos.reshape(S, 3)[sel])
    assert_close(out_h[idx], ro[idx], _mixed_scale(tag_h[idx], p0_h[idx], p1_h[idx], ro[idx], cond[idx]),
                 what="mixed 2^28, %d streams" % sel.size)


# ---- Dirichlet --------------------------------------------------------------

def _dir_scale(th, logs, cond):
    mag = np.abs(logs) + np.nanmax(np.abs(logs), axis=1, keepdims=True)
    kap = cond + np.nanmax(cond, axis=1, keepdims=True)
    return np.abs(th) * (1.0 + mag + kap)


@pytest.mark.parametrize("K,rows,R", [(1, 100, 100), (5, 333, 333), (64, 500, 100), (100, 40, 7),
                                      (128, 64, 64), (64, 2000, 2000)])
def test_dirichlet_parity(K, rows, R):
    seed = 13
    rng = np.random.default_rng(K)
    alpha = np.exp(rng.uniform(np.log(0.05), np.log(20.0), (rows, K))).astype(np.float32)
    h = handle(seed, R * K)
    out = torch.empty((rows, K), dtype=torch.float32, device=DEV)
    B.brng_dirichlet(h.h, T(alpha), out)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    th, rpos, st, logs, cond = O.dirichlet(seed, R * K, alpha, with_logs=True)
    assert np.array_equal(h.positions(), rpos)
    g = H(out).astype(np.float64)
    assert_close(g, th, _dir_scale(th, logs, cond), what="dirichlet K=%d" % K)
    assert np.max(np.abs(g.sum(axis=1) - 1.0)) < 1e-5


@pytest.mark.parametrize("K", [5, 64])
def test_dirichlet_tuning_invariance(K):
    """Short rings and a short row queue (the register-capped kernel, chosen
    when shared memory holds enough of its warps) give the same bits as the
    default tuning (the natural register budget)."""
    rng = np.random.default_rng(K + 1)
    rows, R = 700, 350
    alpha = np.exp(rng.uniform(np.log(0.05), np.log(20.0), (rows, K))).astype(np.float32)
    outs, poss = [], []
    for tune in [{}, dict(buf_len=8, lookahead=2), dict(buf_len=16, lookahead=4, warps_per_block=2)]:
        h = handle(21, R * K, **tune)
        out = torch.empty((rows, K), dtype=torch.float32, device=DEV)
        B.brng_dirichlet(h.h, T(alpha), out)
        code, cnt = h.counters()
        assert code == B.BRNG_OK, cnt
        outs.append(out)
        poss.append(h.positions())
    for o, p in zip(outs[1:], poss[1:]):
        assert torch.equal(o, outs[0]) and np.array_equal(p, poss[0])


def test_dirichlet_invalid_rows():
    seed, K, rows = 3, 40, 30
    alpha = np.full((rows, K), 0.7, dtype=np.float32)
    alpha[4, 7] = -1.0
    alpha[9, 39] = np.nan
    h = handle(seed, 10 * K)  # R = 10: row-streams serve 3 rows each
    out = torch.empty((rows, K), dtype=torch.float32, device=DEV)
    B.brng_dirichlet(h.h, T(alpha), out)
    code, cnt = h.counters()
    assert code == B.BRNG_EDOMAIN and cnt["n_domain"] == 2
    th, rpos, st = O.dirichlet(seed, 10 * K, alpha)
    assert st == O.EDOMAIN
    g = H(out)
    assert np.all(np.isnan(g[4])) and np.all(np.isnan(g[9]))
    assert np.array_equal(h.positions(), rpos)


# ---- Gibbs models -----------------------------------------------------------

def _triangle_gpu(n_chains, n_sweeps, lanes=1, buf_len=256, wpb=4, state=None, mom=None, offset=0):
    h = handle(42, 1, buf_len, lanes_per_chain=lanes, warps_per_block=wpb)
    st = B.triangle_state(n_chains, device=DEV) if state is None else state
    m = torch.zeros((n_chains, 5), dtype=torch.float64, device=DEV) if mom is None else mom
    B.brng_gibbs_run(h.h, B.MODEL_TRIANGLE, offset, n_chains, n_sweeps, None, st, m)
    torch.cuda.synchronize()
    return st, m


def test_triangle_full_size_bit_exact():
    """Eq. 1 / Fig. 1 workload: 1,024 chains x 10,000 sweeps, FP64, bit-exact."""
    n_chains, n_sweeps = 1024, 10000
    st, m = _triangle_gpu(n_chains, n_sweeps)
    x, y, pos = B.triangle_unpack(st)
    ref = O.gibbs_triangle(42, n_chains, n_sweeps, nthreads=NT)
    assert np.array_equal(x.view(np.int64), ref["xy"][:, 0].view(np.int64))
    assert np.array_equal(y.view(np.int64), ref["xy"][:, 1].view(np.int64))
    assert np.array_equal(pos, ref["pos"])
    assert np.array_equal(H(m).view(np.int64), ref["mom"].view(np.int64))


@pytest.mark.parametrize("lanes,buf_len,wpb", [(2, 64, 4), (4, 4, 16), (32, 512, 1), (8, 256, 2)])
def test_triangle_layout_invariance(lanes, buf_len, wpb):
    a, ma = _triangle_gpu(300, 777)
    b, mb = _triangle_gpu(300, 777, lanes=lanes, buf_len=buf_len, wpb=wpb)
    assert torch.equal(a, b) and torch.equal(ma, mb)


def test_triangle_resume_and_shard():
    whole, mw = _triangle_gpu(100, 500)
    st, m = _triangle_gpu(100, 123)
    st, m = _triangle_gpu(100, 377, state=st, mom=m, buf_len=8)
    assert torch.equal(st, whole) and torch.equal(m, mw)
    a, ma = _triangle_gpu(40, 500)
    b, mb = _triangle_gpu(60, 500, offset=40)
    assert torch.equal(torch.cat([a, b]), whole) and torch.equal(torch.cat([ma, mb]), mw)


PRIOR_NG = (2.0, 1.0, 0.0, 0.01)


def _ng_state(mu, tau, pos):
    """brng_normal_gamma_state_t[n] from FP32 (mu, tau) and the oracle's
    positions [n, 2] = (N, U)."""
    n = len(mu)
    s = torch.zeros((n, 3), dtype=torch.int64)
    f = s.view(torch.float32).view(n, 6)
    f[:, 0] = torch.from_numpy(np.asarray(mu, np.float32))
    f[:, 1] = torch.from_numpy(np.asarray(tau, np.float32))
    s[:, 1] = torch.from_numpy(np.asarray(pos[:, 0], np.uint64).view(np.int64))
    s[:, 2] = torch.from_numpy(np.asarray(pos[:, 1], np.uint64).view(np.int64))
    return s.to(DEV)


def _ng_gpu(nobs, xbar, sc, n_sweeps, offset=0, state=None, mom=None, prior=PRIOR_NG, **tune):
    n = nobs.size
    h = handle(42, 1, **tune)
    t = [T(nobs), T(xbar), T(sc)]
    params = B.brng_normal_gamma_params_t(*prior, *[x.data_ptr() for x in t])
    st = B.normal_gamma_state(n, device=DEV) if state is None else state
    m = torch.zeros((n, 4), dtype=torch.float64, device=DEV) if mom is None else mom
    B.brng_gibbs_run(h.h, B.MODEL_NORMAL_GAMMA, offset, n, n_sweeps, params, st, m)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    return st, m, cnt


def assert_bound(got, want, bound, what):
    """|got - want| <= bound element by element (NaN only where both are)."""
    assert_close(got, want, np.asarray(bound, np.float64) / RTOL, what=what)


def _ng_check(st, m, ref, nobs, xbar, sc, what, prior=PRIOR_NG, mu_start=0.0, mom_start=None):
    """Positions bit-exact; final (mu, tau) and the sweep moments within the
    FP32 bound propagated along the oracle's trajectory (gibbs_bounds: the
    per-draw 2e-6 of each sweep carried through the sweep map)."""
    mu, tau, pn, pu = B.normal_gamma_unpack(st)
    assert np.array_equal(pn, ref["pos"][:, 0]) and np.array_equal(pu, ref["pos"][:, 1])
    bnd = gibbs_bounds.ng_bounds(nobs, xbar, sc, prior, mu_start, ref["trace"], RTOL)
    assert_bound(mu, ref["state"][:, 0], bnd["mu"], what + " mu")
    assert_bound(tau, ref["state"][:, 1], bnd["tau"], what + " tau")
    g = H(m)
    base = 0.0 if mom_start is None else mom_start
    for j, name in enumerate(["sum mu", "sum tau", "sum mu^2", "sum tau^2"]):
        assert_bound(g[:, j] - base[:, j] if mom_start is not None else g[:, j],
                     ref["mom"][:, j] - (base[:, j] if mom_start is not None else 0.0),
                     bnd["mom"][:, j], what + " " + name)


def test_normal_gamma_parity_small():
    nobs, xbar, sc = inputs.normal_gamma_data(1000, seed=5)
    st, m, cnt = _ng_gpu(nobs, xbar, sc, 300)
    ref = O.gibbs_normal_gamma(42, 300, nobs, xbar, sc, nthreads=NT, trace=True)
    _ng_check(st, m, ref, nobs, xbar, sc, "normal-gamma 1000x300")


def test_normal_gamma_full_size_sampled():
    """65,536 chains x 2,000 sweeps; 256 chains recomputed by the oracle."""
    n_chains, n_sweeps = 65536, 2000
    nobs, xbar, sc = inputs.normal_gamma_data(n_chains, seed=42)
    st, m, cnt = _ng_gpu(nobs, xbar, sc, n_sweeps)
    print("counters", cnt)
    for c0, c1 in [(0, 128), (n_chains - 128, n_chains)]:
        sl = slice(c0, c1)
        ref = O.gibbs_normal_gamma(42, n_sweeps, nobs[sl], xbar[sl], sc[sl], chain_offset=c0,
                                   nthreads=NT, trace=True)
        _ng_check(st[c0:c1], m[c0:c1], ref, nobs[sl], xbar[sl], sc[sl],
                  "normal-gamma chains %d..%d" % (c0, c1))


@pytest.mark.parametrize("case", ["shape52", "boosted", "mixed_prior"])
@pytest.mark.parametrize("buf_len", [32, 8, 4])
def test_normal_gamma_one_sweep_from_shared_state(case, buf_len):
    """One sweep from the same FP32 state on both sides isolates the per-draw
    FP32 error from its propagation: the oracle runs k sweeps, its state is
    rounded to FP32 and handed, with the same stream positions, to the GPU
    (one sweep) and back to the oracle (one sweep).  tau and mu must then be
    within 2e-6 of the magnitude each draw's FP32 arithmetic works at
    (|tau| (1 + kappa) for tau = G / rate, |mean| + |z| / sqrt(P) for mu),
    mu also carrying tau's bound through d mu / d tau."""
    n = 4096 + 77
    nobs, xbar, sc = inputs.normal_gamma_data(n, seed=21)
    prior = PRIOR_NG
    if case == "boosted":
        nobs = nobs.copy()
        nobs[::3] = 0.0  # shape 0.4: boosted
        nobs[1::3] = 1.0  # shape 0.9: boosted
        prior = (0.4, 1.0, 0.0, 0.01)
    elif case == "mixed_prior":
        nobs = np.floor(np.random.default_rng(4).uniform(0, 400, n)).astype(np.float32)
        prior = (3.0, 2.0, -1.0, 1.0)
    k = 57
    ref0 = O.gibbs_normal_gamma(42, k, nobs, xbar, sc, prior=prior, nthreads=NT)
    mu32 = ref0["state"][:, 0].astype(np.float32)
    tau32 = ref0["state"][:, 1].astype(np.float32)
    st = _ng_state(mu32, tau32, ref0["pos"])
    st, m, cnt = _ng_gpu(nobs, xbar, sc, 1, state=st, prior=prior, buf_len=buf_len)
    start = np.stack([mu32, tau32], axis=1).astype(np.float64)
    ref1 = O.gibbs_normal_gamma(42, 1, nobs, xbar, sc, prior=prior, state=start.ravel(),
                                pos=ref0["pos"].ravel(), nthreads=NT, trace=True)
    _ng_check(st, m, ref1, nobs, xbar, sc, "one sweep %s B=%d" % (case, buf_len), prior=prior,
              mu_start=mu32.astype(np.float64))


def test_normal_gamma_invariance_and_resume():
    nobs, xbar, sc = inputs.normal_gamma_data(200, seed=6)
    a, ma, _ = _ng_gpu(nobs, xbar, sc, 100)
    b, mb, _ = _ng_gpu(nobs, xbar, sc, 100, buf_len=4, warps_per_block=16)
    assert torch.equal(a, b) and torch.equal(ma, mb)
    c, mc, _ = _ng_gpu(nobs, xbar, sc, 37)
    c, mc, _ = _ng_gpu(nobs, xbar, sc, 63, state=c, mom=mc, buf_len=128)
    assert torch.equal(a[:, 1:], c[:, 1:])  # positions identical
    mu_a, tau_a, _, _ = B.normal_gamma_unpack(a)
    mu_c, tau_c, _, _ = B.normal_gamma_unpack(c)
    assert np.array_equal(mu_a, mu_c) and np.array_equal(tau_a, tau_c)


@pytest.mark.parametrize("wpb,wp,buf_len", [(4, 1, 32), (4, 2, 32), (8, 2, 8), (2, 2, 4), (12, 4, 64), (1, 1, 16)])
def test_normal_gamma_producers_equal_inline(wpb, wp, buf_len):
    """Asynchronous replenishment (producer warps) gives the inline form's
    bits, for ragged chain counts and every block shape."""
    nobs, xbar, sc = inputs.normal_gamma_data(1000, seed=9)
    a, ma, _ = _ng_gpu(nobs, xbar, sc, 150)
    b, mb, cnt = _ng_gpu(nobs, xbar, sc, 150, buf_len=buf_len, warps_per_block=wpb, producer_warps=wp)
    assert cnt["n_timeout"] == 0, cnt
    assert torch.equal(a, b) and torch.equal(ma, mb)


def test_normal_gamma_producers_oracle_and_resume():
    nobs, xbar, sc = inputs.normal_gamma_data(333, seed=10)
    ref = O.gibbs_normal_gamma(42, 120, nobs, xbar, sc, nthreads=NT, trace=True)
    st, m, _ = _ng_gpu(nobs, xbar, sc, 120, producer_warps=2)
    _ng_check(st, m, ref, nobs, xbar, sc, "normal-gamma producers 333x120")
    # resume from mid-block positions (the rings then start inside a block)
    c, mc, _ = _ng_gpu(nobs, xbar, sc, 41, producer_warps=1)
    c, mc, cnt = _ng_gpu(nobs, xbar, sc, 79, state=c, mom=mc, producer_warps=3, buf_len=8)
    assert cnt["n_timeout"] == 0
    assert torch.equal(st, c)
    # the FP32 partial sums are flushed at other iterations when a run is split:
    # each part's compensated sum is within SUM_ERR of its exact value
    bnd = gibbs_bounds.ng_bounds(nobs, xbar, sc, PRIOR_NG, 0.0, ref["trace"], RTOL)["mom"]
    assert_bound(H(mc), H(m), 2 * bnd, "split-run moments")


def test_normal_gamma_producers_full_size_sampled():
    """65,536 chains x 2,000 sweeps with producer warps; 128 chains at each
    end recomputed by the oracle."""
    n_chains, n_sweeps = 65536, 2000
    nobs, xbar, sc = inputs.normal_gamma_data(n_chains, seed=42)
    st, m, cnt = _ng_gpu(nobs, xbar, sc, n_sweeps, producer_warps=2)
    assert cnt["n_timeout"] == 0, cnt
    for c0, c1 in [(0, 128), (n_chains - 128, n_chains)]:
        sl = slice(c0, c1)
        ref = O.gibbs_normal_gamma(42, n_sweeps, nobs[sl], xbar[sl], sc[sl], chain_offset=c0,
                                   nthreads=NT, trace=True)
        _ng_check(st[c0:c1], m[c0:c1], ref, nobs[sl], xbar[sl], sc[sl],
                  "normal-gamma producers chains %d..%d" % (c0, c1))


@pytest.mark.parametrize("buf_len", [32, 8, 4])
def test_normal_gamma_small_shapes_boosted(buf_len):
    """Prior shape a0 = 0.4 and chains without observations: shapes below 1
    take the boosted exact path (an extra U after each accept) in every round
    structure (speculative width 8, 2, and the plain loop)."""
    nobs, xbar, sc = inputs.normal_gamma_data(400, seed=12)
    nobs = nobs.copy()
    nobs[::3] = 0.0  # shape 0.4
    nobs[1::3] = 1.0  # shape 0.9
    prior = (0.4, 1.0, 0.0, 0.01)
    st, m, cnt = _ng_gpu(nobs, xbar, sc, 120, prior=prior, buf_len=buf_len)
    ref = O.gibbs_normal_gamma(42, 120, nobs, xbar, sc, prior=prior, nthreads=NT, trace=True)
    _ng_check(st, m, ref, nobs, xbar, sc, "boosted B=%d" % buf_len, prior=prior)


def _lda_gpu(alpha, n_sweeps, offset=0, pos0=None, **tune):
    n_docs, K = alpha.shape
    h = handle(42, 1, **tune)
    a = T(alpha)
    theta = torch.zeros((n_docs, K), dtype=torch.float32, device=DEV)
    if pos0 is None:
        pos = torch.zeros((n_docs, K, 2), dtype=torch.int64, device=DEV)
    else:
        pos = T(np.asarray(pos0, np.uint64).view(np.int64).reshape(n_docs, K, 2))
    mom = torch.zeros((n_docs, K), dtype=torch.float64, device=DEV)
    params = B.brng_lda_params_t(K, a.data_ptr())
    state = B.brng_lda_state_t(theta.data_ptr(), pos.data_ptr())
    B.brng_gibbs_run(h.h, B.MODEL_LDA, offset, n_docs, n_sweeps, params, state, mom)
    code, cnt = h.counters()
    assert code == B.BRNG_OK, cnt
    return theta, pos, mom


def _lda_check(theta, pos, mom, ref, what):
    """Positions bit-exact; the last draw within the per-draw bound; the sweep
    sums within the per-draw bounds of every sweep summed (the sweeps are
    independent draws from fixed counts, so nothing propagates) plus the
    compensated sum's own error."""
    assert np.array_equal(H(pos).view(np.uint64), ref["pos"])
    assert_close(H(theta), ref["theta"], _dir_scale(ref["theta"], ref["logs"], ref["cond"]),
                 what=what + " theta")
    assert_bound(H(mom), ref["mom"], gibbs_bounds.lda_mom_bound(ref["trace"], RTOL), what + " sum theta")


def test_lda_parity_small():
    alpha, _, _ = inputs.lda_alpha(96, K=64, seed=7)
    theta, pos, mom = _lda_gpu(alpha, 40)
    ref = O.gibbs_lda(42, 40, alpha, nthreads=NT, trace=True)
    _lda_check(theta, pos, mom, ref, "lda 96x64x40")


@pytest.mark.parametrize("buf_len", [64, 16, 4])
def test_lda_one_sweep_from_shared_positions(buf_len):
    """One LDA sweep from the positions the oracle reached after k sweeps
    (resuming inside Philox blocks): theta and its sum within the per-draw
    bound."""
    alpha, _, _ = inputs.lda_alpha(300, K=64, seed=17)
    ref0 = O.gibbs_lda(42, 13, alpha, nthreads=NT)
    theta, pos, mom = _lda_gpu(alpha, 1, pos0=ref0["pos"], buf_len=buf_len)
    ref1 = O.gibbs_lda(42, 1, alpha, pos=ref0["pos"].ravel(), nthreads=NT, trace=True)
    _lda_check(theta, pos, mom, ref1, "lda one sweep B=%d" % buf_len)


def test_lda_full_size_sampled():
    """16,384 documents x K=64 x 500 sweeps; 8 documents recomputed."""
    alpha, _, _ = inputs.lda_alpha(16384, K=64, seed=42)
    theta, pos, mom = _lda_gpu(alpha, 500)
    for d0, d1 in [(0, 4), (16380, 16384)]:
        ref = O.gibbs_lda(42, 500, alpha[d0:d1], doc_offset=d0, nthreads=NT, trace=True)
        _lda_check(theta[d0:d1], pos[d0:d1], mom[d0:d1], ref, "lda docs %d..%d" % (d0, d1))


@pytest.mark.parametrize("case", range(9))
def test_gibbs_random_configurations(case):
    """Seeded random configurations of the three Gibbs models -- chain or
    document counts, sweeps, chain offset, ring length, warps per block,
    lanes per chain (triangle), K and lookahead (LDA), a run split in two
    with other tunings (triangle) -- against the oracle: triangle bit-exact,
    normal-gamma and LDA positions bit-exact and values within tolerance."""
    rng = np.random.default_rng(2000 + case)
    model = case % 3
    pick = lambda xs: int(rng.choice(xs))  # noqa: E731
    offset = int(rng.integers(0, 100000))
    if model == 0:
        n, sweeps = int(rng.integers(1, 700)), int(rng.integers(2, 400))
        s1 = int(rng.integers(1, sweeps))
        st, m = _triangle_gpu(n, s1, lanes=pick([1, 2, 4, 8, 16, 32]), buf_len=pick([4, 8, 64, 256, 512]),
                              wpb=pick([1, 2, 4, 8, 16]), offset=offset)
        st, m = _triangle_gpu(n, sweeps - s1, lanes=pick([1, 2, 4, 8, 16, 32]), buf_len=pick([4, 16, 128]),
                              wpb=pick([1, 4, 16]), state=st, mom=m, offset=offset)
        x, y, pos = B.triangle_unpack(st)
        ref = O.gibbs_triangle(42, n, sweeps, chain_offset=offset, nthreads=NT)
        assert np.array_equal(x.view(np.int64), ref["xy"][:, 0].view(np.int64))
        assert np.array_equal(y.view(np.int64), ref["xy"][:, 1].view(np.int64))
        assert np.array_equal(pos, ref["pos"])
        assert np.array_equal(H(m).view(np.int64), ref["mom"].view(np.int64))
    elif model == 1:
        n, sweeps = int(rng.integers(1, 1500)), int(rng.integers(1, 200))
        nobs, xbar, sc = inputs.normal_gamma_data(n, seed=case)
        st, m, cnt = _ng_gpu(nobs, xbar, sc, sweeps, offset=offset, buf_len=pick([4, 8, 16, 32, 64]),
                             warps_per_block=pick([1, 2, 4, 8, 16]))
        ref = O.gibbs_normal_gamma(42, sweeps, nobs, xbar, sc, chain_offset=offset, nthreads=NT,
                                   trace=True)
        _ng_check(st, m, ref, nobs, xbar, sc, "normal-gamma random case %d" % case)
    else:
        docs, K, sweeps = int(rng.integers(1, 120)), pick([5, 17, 32, 64, 100]), int(rng.integers(1, 30))
        alpha, _, _ = inputs.lda_alpha(docs, K=K, seed=case)
        theta, pos, mom = _lda_gpu(alpha, sweeps, offset=offset, buf_len=pick([4, 8, 16, 32]),
                                   lookahead=pick([1, 2, 4, 8, 16]), warps_per_block=pick([1, 2, 4]))
        ref = O.gibbs_lda(42, sweeps, alpha, doc_offset=offset, nthreads=NT, trace=True)
        _lda_check(theta, pos, mom, ref, "lda random case %d" % case)


@pytest.mark.parametrize("tune", [dict(lookahead=1), dict(lookahead=16, buf_len=4), dict(warps_per_block=1, buf_len=128)])
def test_lda_tuning_invariance(tune):
    alpha, _, _ = inputs.lda_alpha(50, K=64, seed=8)
    a = _lda_gpu(alpha, 25)
    b = _lda_gpu(alpha, 25, **tune)
    for x, y in zip(a, b):
        assert torch.equal(x, y)


# ---- edge cases and errors --------------------------------------------------

def test_edge_cases():
    h = handle(1, 10)
    empty = torch.empty(0, dtype=torch.float32, device=DEV)
    assert B.brng_gamma(h.h, empty, empty) == B.BRNG_OK
    # fewer draws than streams; single stream
    for S, n in [(10, 3), (1, 257)]:
        h = handle(2, S)
        alpha = np.full(n, 0.5, np.float32)
        out, w = _run_bulk("gamma", h, [alpha], n)
        ro, rw, rpos, _ = O.gamma(2, S, alpha)
        assert np.array_equal(words_np(w), rw) and np.array_equal(h.positions(), rpos)
    # invalid parameters: NaN, nothing consumed, counted
    h = handle(3, 4)
    a = np.array([0, 1, np.nan, 2, 5, 5], np.float32)
    b = np.array([1, 0.5, 1, np.inf, 5, 6], np.float32)
    out, w = _run_bulk("uniform", h, [a, b], 6)
    code, cnt = h.counters(reset=True)
    assert code == B.BRNG_EDOMAIN and cnt["n_domain"] == 3
    ro, rw, rpos, st = O.uniform(3, 4, a, b)
    g = H(out)
    assert np.array_equal(np.isnan(g), np.isnan(ro)) and np.array_equal(h.positions(), rpos)
    assert g[4] == 5.0
    code, cnt = h.counters()
    assert code == B.BRNG_OK and cnt["n_domain"] == 0
    # unknown tag
    tag = np.array([0, 9, 3], np.uint8)
    p = np.ones(3, np.float32)
    o = torch.empty(3, dtype=torch.float32, device=DEV)
    B.brng_mixed(h.h, T(tag), T(p), T(p + 1), o)
    code, cnt = h.counters()
    assert code == B.BRNG_EDOMAIN and np.isnan(H(o)[1])


def test_argument_errors():
    with pytest.raises(B.BrngError):
        B.brng_create(1, 0)
    with pytest.raises(B.BrngError):
        B.brng_create(1, 4, 48)  # not a power of two
    h = handle(1, 10)
    with pytest.raises(B.BrngError):
        h.tune(warps_per_block=17)
    with pytest.raises(B.BrngError):
        h.tune(producer_warps=9)
    with pytest.raises(B.BrngError):
        B.brng_dirichlet(h.h, torch.ones((2, 3), device=DEV), torch.empty((2, 3), device=DEV))  # 10 % 3
    with pytest.raises(B.BrngError):
        h.tune(buf_len=512, warps_per_block=16)
        a = torch.ones(100, device=DEV)
        # 3 rings x 512 elements x 32 lanes x (value + word): not even one warp fits
        B.brng_mixed(h.h, torch.zeros(100, dtype=torch.uint8, device=DEV), a, a, torch.empty(100, device=DEV),
                     torch.empty(100, dtype=torch.int32, device=DEV))
