"""Python face of the CPU oracle (plain C, FP64) -- TEST INFRASTRUCTURE ONLY.

The oracle restates the batched varying-parameter RNG method of Mahani &
Sharabiani (arXiv 1412.4825, Sec. 2) in plain, slow FP64 C.  Only tests/,
``__graft_entry__.smoke()`` and bench.py's CPU-baseline / reference legs may
import it; the product path (the CUDA library and its binding) never does.
Every function takes numpy arrays and returns new numpy arrays; stream
positions are passed in and returned, so calls can be chained exactly like
the stateful object of Sec. 2.2.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

DOM_U, DOM_N, DOM_E, DOM_DATA, DOM_U64 = 0, 1, 2, 3, 4
OK, EINVAL, EDOMAIN, EREJECT = 0, 1, 4, 5
GAMMA_MAX_ATTEMPTS = 64
POISSON_MAX_LAMBDA = 1e7
POISSON_MAX_K = 1024
INVERSION_MAX_MEAN = 64.0  # Poisson / Binomial means above this: PTRS / BTRD

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        u32, u64, i32, dbl = C.c_uint32, C.c_uint64, C.c_int, C.c_double
        vp = C.c_void_p
        L.or_philox4x32_10.argtypes = [vp, vp, vp]
        L.or_philox_words.argtypes = [u64, u32, u32, u64, u64, vp]
        L.or_log.argtypes = [dbl]
        L.or_log.restype = dbl
        L.or_log_many.argtypes = [u64, vp, vp]
        L.or_exp_many.argtypes = [u64, vp, vp]
        L.or_poisson_inv.argtypes = [dbl, dbl]
        L.or_poisson_inv.restype = dbl
        L.or_poisson.argtypes = [u64, u32, vp, u64, vp, vp, vp, u32]
        L.or_poisson.restype = i32
        L.or_binomial_inv.argtypes = [dbl, dbl, dbl]
        L.or_binomial_inv.restype = dbl
        L.or_lfact.argtypes = [dbl]
        L.or_lfact.restype = dbl
        L.or_binomial.argtypes = [u64, u32, vp, u64, vp, vp, vp, vp, u32]
        L.or_binomial.restype = i32
        L.or_sincospi_many.argtypes = [u64, vp, vp, vp]
        L.or_elem_values.argtypes = [u64, u32, u32, u64, u64, vp, vp]
        for name in ("or_uniform", "or_normal", "or_laplace"):
            getattr(L, name).argtypes = [u64, u32, vp, u64, vp, vp, vp, vp, u32]
            getattr(L, name).restype = i32
        L.or_uniform_f64.argtypes = [u64, u32, vp, u64, vp, vp, vp, vp, u32]
        L.or_uniform_f64.restype = i32
        L.or_weibull.argtypes = [u64, u32, vp, u64, vp, vp, vp, vp, vp, u32]
        L.or_weibull.restype = i32
        L.or_exponential.argtypes = [u64, u32, vp, u64, vp, vp, vp, u32]
        L.or_exponential.restype = i32
        L.or_gamma.argtypes = [u64, u32, vp, u64, vp, vp, vp, vp, u32]
        L.or_gamma.restype = i32
        L.or_dirichlet.argtypes = [u64, u32, vp, u64, u32, vp, vp, vp, vp, u32]
        L.or_dirichlet.restype = i32
        L.or_mixed_streams.argtypes = [u64, u32, u32, u32, vp, u64, vp, vp, vp, vp, vp, vp, u32]
        L.or_mixed_streams.restype = i32
        L.or_mixed_mt.argtypes = [u64, u32, vp, u64, vp, vp, vp, vp, vp, vp, u32, i32]
        L.or_mixed_mt.restype = i32
        L.or_gibbs_triangle_mt.argtypes = [u64, u64, u32, u32, vp, vp, vp, u32, i32]
        L.or_gibbs_triangle_mt.restype = i32
        L.or_gibbs_normal_gamma_mt.argtypes = [u64, u64, u32, u32, vp, vp, vp, vp, vp, vp, vp, vp, u32, i32]
        L.or_gibbs_normal_gamma_mt.restype = i32
        L.or_gibbs_lda_mt.argtypes = [u64, u64, u32, u32, u32, vp, vp, vp, vp, vp, vp, vp, u32, i32]
        L.or_gibbs_lda_mt.restype = i32
        f32 = C.c_float
        L.or_lda_weights.argtypes = [u32, f32, f32, f32, vp, vp, vp, u32, vp, vp]
        L.or_lda_pick.argtypes = [u32, vp, u32]
        L.or_lda_pick.restype = u32
        L.or_lda_z_sweep_mt.argtypes = [u64, u64, u32, u32, u32, f32, f32, vp, vp, vp, vp, vp, vp, vp, vp,
                                        vp, i32]
        L.or_lda_z_sweep_mt.restype = i32
        L.or_lda_z_run.argtypes = [u64, u32, u32, u32, u32, f32, f32, vp, vp, vp, vp, vp, vp, vp, vp]
        L.or_lda_z_run.restype = i32
        L.or_mt_accept.argtypes = [dbl, dbl, dbl]
        L.or_mt_accept.restype = i32
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f32(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float32)


def _threads(nthreads):
    return os.cpu_count() or 1 if nthreads is None else int(nthreads)


# ---- core engine and elementary functions --------------------------------

def philox4x32_10(ctr, key):
    """One Philox4x32-10 block: 4 counter words, 2 key words -> 4 words."""
    c = np.ascontiguousarray(ctr, dtype=np.uint32)
    k = np.ascontiguousarray(key, dtype=np.uint32)
    out = np.zeros(4, dtype=np.uint32)
    lib().or_philox4x32_10(_p(c), _p(k), _p(out))
    return out


def philox_words(seed, domain, stream, first_block, n_blocks):
    out = np.zeros(4 * n_blocks, dtype=np.uint32)
    lib().or_philox_words(seed, domain, stream, first_block, n_blocks, _p(out))
    return out


def log(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    lib().or_log_many(x.size, _p(x), _p(out))
    return out


def exp(x):
    x = np.ascontiguousarray(x, dtype=np.float64)
    out = np.empty_like(x)
    lib().or_exp_many(x.size, _p(x), _p(out))
    return out


def poisson_inv(lam, u):
    return lib().or_poisson_inv(float(lam), float(u))


def sincospi(a):
    a = np.ascontiguousarray(a, dtype=np.float64)
    s = np.empty_like(a)
    c = np.empty_like(a)
    lib().or_sincospi_many(a.size, _p(a), _p(s), _p(c))
    return s, c


def elements(seed, domain, stream, j0, n):
    """Elements j0..j0+n-1 of one domain of one stream: (values, words)."""
    out = np.empty(n, dtype=np.float64)
    words = np.empty(n, dtype=np.uint32)
    lib().or_elem_values(seed, domain, stream, j0, n, _p(out), _p(words))
    return out, words


def mt_accept(alpha, z, u_open):
    return lib().or_mt_accept(float(alpha), float(z), float(u_open))


# ---- bulk varying-parameter streams ---------------------------------------

def new_positions(n_streams):
    return np.zeros(3 * n_streams, dtype=np.uint64)


def _bulk(name, seed, S, pos, n, params, buf_len, with_cond=False):
    pos = np.array(pos if pos is not None else new_positions(S), dtype=np.uint64, copy=True)
    out = np.empty(n, dtype=np.float64)
    words = np.zeros(n, dtype=np.uint32)
    ps = [_f32(p) for p in params]
    extra = []
    cond = None
    if name in ("or_gamma", "or_weibull"):
        cond = np.zeros(n, dtype=np.float64)
        extra = [_p(cond)]
    st = getattr(lib(), name)(seed, S, _p(pos), n, *[_p(p) for p in ps], _p(out), _p(words), *extra,
                              buf_len)
    if with_cond:
        return out, words, pos, st, cond
    return out, words, pos, st


def uniform(seed, S, a, b, pos=None, buf_len=64):
    return _bulk("or_uniform", seed, S, pos, len(a), [a, b], buf_len)


def uniform_f64(seed, S, a, b, pos64=None, buf_len=64):
    """U[a, b) in FP64 from the 53-bit U64 domain; pos64 holds one U64
    position per stream (separate from the U, N, E positions)."""
    pos = np.array(pos64 if pos64 is not None else np.zeros(S, dtype=np.uint64), dtype=np.uint64, copy=True)
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    n = len(a)
    out = np.empty(n, dtype=np.float64)
    words = np.zeros(n, dtype=np.uint32)
    st = lib().or_uniform_f64(seed, S, _p(pos), n, _p(a), _p(b), _p(out), _p(words), buf_len)
    return out, words, pos, st


def normal(seed, S, mu, sigma, pos=None, buf_len=64):
    return _bulk("or_normal", seed, S, pos, len(mu), [mu, sigma], buf_len)


def exponential(seed, S, lam, pos=None, buf_len=64):
    return _bulk("or_exponential", seed, S, pos, len(lam), [lam], buf_len)


def gamma(seed, S, alpha, pos=None, buf_len=64, with_cond=False):
    return _bulk("or_gamma", seed, S, pos, len(alpha), [alpha], buf_len, with_cond)


def laplace(seed, S, mu, scale, pos=None, buf_len=64):
    return _bulk("or_laplace", seed, S, pos, len(mu), [mu, scale], buf_len)


def weibull(seed, S, shape, scale, pos=None, buf_len=64, with_cond=False):
    return _bulk("or_weibull", seed, S, pos, len(shape), [shape, scale], buf_len, with_cond)


def poisson(seed, S, lam, pos=None, buf_len=64):
    return _bulk("or_poisson", seed, S, pos, len(lam), [lam], buf_len)


def lfact(k):
    return lib().or_lfact(float(k))


def binomial_inv(n, p, u):
    return lib().or_binomial_inv(float(n), float(p), float(u))


def binomial(seed, S, trials, prob, pos=None, buf_len=64):
    return _bulk("or_binomial", seed, S, pos, len(trials), [trials, prob], buf_len)


def dirichlet(seed, S, alpha, pos=None, buf_len=64, with_logs=False):
    alpha = _f32(alpha)
    n_rows, K = alpha.shape
    pos = np.array(pos if pos is not None else new_positions(S), dtype=np.uint64, copy=True)
    out = np.empty((n_rows, K), dtype=np.float64)
    logs = np.empty((n_rows, K), dtype=np.float64)
    cond = np.zeros((n_rows, K), dtype=np.float64)
    st = lib().or_dirichlet(seed, S, _p(pos), n_rows, K, _p(alpha), _p(out), _p(logs), _p(cond),
                            buf_len)
    if with_logs:
        return out, pos, st, logs, cond
    return out, pos, st


def mixed(seed, S, tag, p0, p1, pos=None, buf_len=64, streams=None, nthreads=1, with_cond=False):
    """Mixed-tag stream; `streams=(s0, s1)` restricts to those streams only
    (the other outputs stay NaN / 0); a list of such pairs computes each range."""
    tag = np.ascontiguousarray(tag, dtype=np.uint8)
    p0, p1 = _f32(p0), _f32(p1)
    n = tag.size
    pos = np.array(pos if pos is not None else new_positions(S), dtype=np.uint64, copy=True)
    out = np.full(n, np.nan, dtype=np.float64)
    words = np.zeros(n, dtype=np.uint32)
    cond = np.zeros(n, dtype=np.float64)
    if streams is None:
        st = lib().or_mixed_mt(seed, S, _p(pos), n, _p(tag), _p(p0), _p(p1), _p(out), _p(words),
                               _p(cond), buf_len, _threads(nthreads))
    else:
        ranges = [streams] if np.isscalar(streams[0]) else list(streams)
        st = 0
        for s0, s1 in ranges:
            st = lib().or_mixed_streams(seed, S, int(s0), int(s1), _p(pos), n, _p(tag), _p(p0),
                                        _p(p1), _p(out), _p(words), _p(cond), buf_len)
            if st:
                break
    if with_cond:
        return out, words, pos, st, cond
    return out, words, pos, st


# ---- Gibbs models ---------------------------------------------------------

def gibbs_triangle(seed, n_chains, n_sweeps, chain_offset=0, xy=None, pos=None, mom=None,
                   buf_len=256, nthreads=1):
    xy = np.full(2 * n_chains, 0.5) if xy is None else np.array(xy, dtype=np.float64, copy=True)
    pos = np.zeros(n_chains, np.uint64) if pos is None else np.array(pos, np.uint64, copy=True)
    mom = np.zeros(5 * n_chains) if mom is None else np.array(mom, dtype=np.float64, copy=True)
    st = lib().or_gibbs_triangle_mt(seed, chain_offset, n_chains, n_sweeps, _p(xy), _p(pos),
                                    _p(mom), buf_len, _threads(nthreads))
    return dict(xy=xy.reshape(n_chains, 2), pos=pos, mom=mom.reshape(n_chains, 5), status=st)


def gibbs_normal_gamma(seed, n_sweeps, nobs, xbar, sc, prior=(2.0, 1.0, 0.0, 0.01),
                       chain_offset=0, state=None, pos=None, mom=None, buf_len=64, nthreads=1,
                       trace=False):
    """trace=True adds "trace": [n_chains, n_sweeps, 5] = per sweep (G, the
    Gamma draw's conditioning, the Gaussian z of mu's draw, tau, mu)."""
    nobs, xbar, sc = _f32(nobs), _f32(xbar), _f32(sc)
    n_chains = nobs.size
    prior = np.ascontiguousarray(prior, dtype=np.float32)
    state = np.zeros(2 * n_chains) if state is None else np.array(state, np.float64, copy=True)
    pos = np.zeros(2 * n_chains, np.uint64) if pos is None else np.array(pos, np.uint64, copy=True)
    mom = np.zeros(4 * n_chains) if mom is None else np.array(mom, np.float64, copy=True)
    tr = np.zeros((n_chains, n_sweeps, 5)) if trace else None
    st = lib().or_gibbs_normal_gamma_mt(seed, chain_offset, n_chains, n_sweeps, _p(prior),
                                        _p(nobs), _p(xbar), _p(sc), _p(state), _p(pos), _p(mom),
                                        _p(tr), buf_len, _threads(nthreads))
    out = dict(state=state.reshape(n_chains, 2), pos=pos.reshape(n_chains, 2),
               mom=mom.reshape(n_chains, 4), status=st)
    if trace:
        out["trace"] = tr
    return out


def gibbs_lda(seed, n_sweeps, alpha, doc_offset=0, pos=None, mom=None, buf_len=64, nthreads=1,
              trace=False):
    """trace=True adds "trace": [n_docs, n_sweeps, K, 2] = per sweep and
    component (log-Gamma, its conditioning)."""
    alpha = _f32(alpha)
    n_docs, K = alpha.shape
    theta = np.zeros((n_docs, K))
    logs = np.zeros((n_docs, K))
    cond = np.zeros((n_docs, K))
    pos = np.zeros(2 * n_docs * K, np.uint64) if pos is None else np.array(pos, np.uint64, copy=True)
    mom = np.zeros((n_docs, K)) if mom is None else np.array(mom, np.float64, copy=True)
    tr = np.zeros((n_docs, n_sweeps, K, 2)) if trace else None
    st = lib().or_gibbs_lda_mt(seed, doc_offset, n_docs, K, n_sweeps, _p(alpha), _p(theta),
                               _p(logs), _p(cond), _p(pos), _p(mom), _p(tr), buf_len,
                               _threads(nthreads))
    out = dict(theta=theta, logs=logs, cond=cond, pos=pos.reshape(n_docs, K, 2), mom=mom,
               status=st)
    if trace:
        out["trace"] = tr
    return out


# ---- full LDA step: topic draws per token, then theta ~ Dir(alpha + n_d) --

DOM_Z = 5


def lda_weights(K, alpha, beta, V, ndk, nkw_w, nk, z_old):
    """FP32 weights and their integer form for one token (counts include the
    token itself, whose topic is z_old); Vbeta = float32(V) * beta."""
    ndk, nkw_w, nk = (np.ascontiguousarray(a, dtype=np.int32) for a in (ndk, nkw_w, nk))
    w = np.empty(K, dtype=np.float32)
    q = np.empty(K, dtype=np.uint32)
    vbeta = float(np.float32(V) * np.float32(beta))
    lib().or_lda_weights(K, alpha, beta, vbeta, _p(ndk), _p(nkw_w), _p(nk), z_old, _p(w), _p(q))
    return w, q


def lda_pick(q, r24):
    q = np.ascontiguousarray(q, dtype=np.uint32)
    return int(lib().or_lda_pick(q.size, _p(q), r24))


def lda_z_sweep(seed, corpus, state, alpha, beta, doc_offset=0, nthreads=1):
    """One sweep of topic draws over the corpus's documents (state updated in
    place: z, ndk, zpos); returns (dnkw, dnk), the sweep's word-topic and topic
    count changes, which the caller adds into nkw and nk (the sweep's
    snapshot is state["nkw"], state["nk"], left untouched)."""
    K, V = corpus["K"], corpus["V"]
    n_docs = corpus["doc_ptr"].size - 1
    dnkw = np.zeros((V, K), dtype=np.int32)
    dnk = np.zeros(K, dtype=np.int32)
    st = lib().or_lda_z_sweep_mt(seed, doc_offset, n_docs, K, V, alpha, beta, _p(corpus["doc_ptr"]),
                                 _p(corpus["words"]), _p(state["z"]), _p(state["ndk"]), _p(state["nkw"]),
                                 _p(state["nk"]), _p(dnkw), _p(dnk), _p(state["zpos"]), _threads(nthreads))
    if st != OK:
        raise ValueError("or_lda_z_sweep: status %d" % st)
    return dnkw, dnk


def lda_z_run(seed, n_sweeps, corpus, state, alpha=0.1, beta=0.01, zhist=False):
    """n_sweeps topic sweeps without theta draws, all in C (documents from id
    0); state updated in place; returns the per-token topic histogram
    [n_tokens, K] over the sweeps when zhist."""
    K, V = corpus["K"], corpus["V"]
    n_docs = corpus["doc_ptr"].size - 1
    h = np.zeros((corpus["words"].size, K), dtype=np.uint32) if zhist else None
    st = lib().or_lda_z_run(seed, n_sweeps, n_docs, K, V, alpha, beta, _p(corpus["doc_ptr"]),
                            _p(corpus["words"]), _p(state["z"]), _p(state["ndk"]), _p(state["nkw"]),
                            _p(state["nk"]), _p(state["zpos"]), _p(h))
    if st != OK:
        raise ValueError("or_lda_z_run: status %d" % st)
    return h


def lda_full(seed, n_sweeps, corpus, state, alpha=0.1, beta=0.01, doc_offset=0, nthreads=1, buf_len=64,
             theta_draws=True, trace=False):
    """The full LDA Gibbs step, n_sweeps times: topic draws for every token
    (lda_z_sweep), the sweep's count changes added into nkw and nk, then per
    document theta_d ~ Dirichlet(alpha + n_d) with alpha + n_dk formed in FP32
    (the Dirichlet of Sec. 1's LDA paragraph, from Gammas per its footnote),
    its components on streams (doc_offset + d) K + k as in gibbs_lda.
    `state` (dict of numpy arrays: z, ndk, nkw, nk, zpos, pos [n_docs, K, 2],
    mom [n_docs, K], theta) is updated in place and returned; trace=True
    appends every theta draw's log-Gammas and conditioning to state["trace"]."""
    K = corpus["K"]
    a32 = np.float32(alpha)
    for _ in range(n_sweeps):
        dnkw, dnk = lda_z_sweep(seed, corpus, state, alpha, beta, doc_offset, nthreads)
        state["nkw"] += dnkw
        state["nk"] += dnk
        if theta_draws:
            dir_alpha = (a32 + state["ndk"].astype(np.float32)).astype(np.float32)
            r = gibbs_lda(seed, 1, dir_alpha, doc_offset=doc_offset, pos=state["pos"].ravel(),
                          mom=state["mom"], buf_len=buf_len, nthreads=nthreads, trace=trace)
            state["pos"] = r["pos"]
            state["mom"] = r["mom"]
            state["theta"] = r["theta"]
            state["logs"], state["cond"] = r["logs"], r["cond"]
            if trace:  # [n_docs, sweeps, K, 2]: every theta draw's log-Gammas and conditioning
                prev = state.get("trace")
                state["trace"] = r["trace"] if prev is None else np.concatenate([prev, r["trace"]], axis=1)
    assert K == state["ndk"].shape[1]
    return state
