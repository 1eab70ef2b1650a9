"""ctypes binding of libbrng.so (include/brng.h), argument marshalling only.

Every ``brng_*`` function here has the name and argument order of the C
call; device arrays are torch CUDA tensors (their ``data_ptr()`` is passed),
``stream`` is a ``torch.cuda.Stream`` or None (the current torch stream).
Every step of the computation runs in the library's CUDA kernels; there is no
CPU fallback: importing this module fails loudly if the library is missing.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BRNG_LIB selects another build of the same library (the checked build,
# libbrng_debug.so); the default is the in-tree libbrng.so
LIB_PATH = os.environ.get("BRNG_LIB") or os.path.join(_HERE, "libbrng.so")

BRNG_OK, BRNG_EINVAL, BRNG_ENOMEM, BRNG_ECUDA, BRNG_EDOMAIN, BRNG_EREJECT, BRNG_ETIMEOUT, \
    BRNG_EAGAIN, BRNG_ENOTFOUND = range(9)
STATUS_NAMES = ["OK", "EINVAL", "ENOMEM", "ECUDA", "EDOMAIN", "EREJECT", "ETIMEOUT", "EAGAIN",
                "ENOTFOUND"]
DOMAIN_U, DOMAIN_N, DOMAIN_E, DOMAIN_DATA, DOMAIN_U64, DOMAIN_Z = 0, 1, 2, 3, 4, 5
TAG_UNIFORM, TAG_NORMAL, TAG_EXPONENTIAL, TAG_GAMMA, TAG_LAPLACE, TAG_WEIBULL, TAG_POISSON, TAG_BINOMIAL = range(8)
POISSON_MAX_LAMBDA = 1e7
INVERSION_MAX_MEAN = 64.0
MODEL_TRIANGLE, MODEL_NORMAL_GAMMA, MODEL_LDA, MODEL_LDA_FULL = 0, 1, 2, 3
LDA_NONE = 0xFFFFFFFF
BRNG_STATIC_MAX_STREAMS = 65536


class BrngError(RuntimeError):
    def __init__(self, call, code):
        super().__init__("%s failed: %s (%d)" % (call, STATUS_NAMES[code] if 0 <= code < 9 else "?", code))
        self.code = code


class brng_tuning_t(C.Structure):
    _fields_ = [("buf_len", C.c_uint32), ("warps_per_block", C.c_uint32),
                ("lanes_per_chain", C.c_uint32), ("lookahead", C.c_uint32),
                ("producer_warps", C.c_uint32)]


PRODUCERS_NONE = 0xFFFFFFFF


class brng_counters_t(C.Structure):
    _fields_ = [("n_domain", C.c_uint64), ("n_reject", C.c_uint64), ("n_recheck", C.c_uint64),
                ("n_flip", C.c_uint64), ("max_flip_ratio", C.c_float), ("n_timeout", C.c_uint32),
                ("n_wasted", C.c_uint64)]

    def as_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_ if f != "pad"}


class brng_normal_gamma_params_t(C.Structure):
    _fields_ = [("a0", C.c_float), ("b0", C.c_float), ("mu0", C.c_float), ("prec0", C.c_float),
                ("nobs", C.c_void_p), ("xbar", C.c_void_p), ("sc", C.c_void_p)]


class brng_lda_params_t(C.Structure):
    _fields_ = [("K", C.c_uint32), ("alpha", C.c_void_p)]


class brng_lda_state_t(C.Structure):
    _fields_ = [("theta", C.c_void_p), ("pos", C.c_void_p)]


class brng_lda_full_params_t(C.Structure):
    _fields_ = [("K", C.c_uint32), ("V", C.c_uint32), ("alpha", C.c_float), ("beta", C.c_float),
                ("doc_ptr", C.c_void_p), ("words", C.c_void_p), ("prev", C.c_void_p), ("exchange", C.c_uint32),
                ("order", C.c_void_p)]


class brng_lda_full_state_t(C.Structure):
    _fields_ = [("z", C.c_void_p), ("z_start", C.c_void_p), ("ndk", C.c_void_p), ("nkw", C.c_void_p),
                ("nk", C.c_void_p), ("dnkw", C.c_void_p), ("dir_alpha", C.c_void_p), ("zpos", C.c_void_p),
                ("theta", C.c_void_p), ("pos", C.c_void_p)]


class brng_job_t(C.Structure):
    _fields_ = [("model", C.c_int), ("n_chains", C.c_uint32), ("n_sweeps", C.c_uint32),
                ("pad", C.c_uint32), ("seed", C.c_uint64), ("chain_offset", C.c_uint64),
                ("params", C.c_void_p), ("state", C.c_void_p), ("moments", C.c_void_p)]


class brng_request_t(C.Structure):
    _fields_ = [("model", C.c_int), ("n_chains", C.c_uint32), ("n_sweeps", C.c_uint32), ("K", C.c_uint32),
                ("seed", C.c_uint64), ("chain_offset", C.c_uint64), ("nobs", C.c_void_p),
                ("xbar", C.c_void_p), ("sc", C.c_void_p), ("alpha", C.c_void_p), ("a0", C.c_float),
                ("b0", C.c_float), ("mu0", C.c_float), ("prec0", C.c_float), ("flags", C.c_uint32),
                ("pad", C.c_uint32)]


SERVE_BORROW_INPUTS = 1


class brng_job_info_t(C.Structure):
    _fields_ = [("submitted_ns", C.c_uint64), ("admitted_ns", C.c_uint64), ("launched_ns", C.c_uint64),
                ("completed_ns", C.c_uint64), ("device_bytes", C.c_uint64), ("status", C.c_int32),
                ("pad", C.c_uint32)]


class brng_serve_stats_t(C.Structure):
    _fields_ = [("submitted", C.c_uint64), ("admitted", C.c_uint64), ("completed", C.c_uint64),
                ("refused", C.c_uint64), ("batches", C.c_uint64), ("queued", C.c_uint64),
                ("device_bytes_in_use", C.c_uint64), ("cancelled", C.c_uint64)]


def _load():
    if not os.path.exists(LIB_PATH):
        raise ImportError("libbrng.so not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = C.CDLL(LIB_PATH)
    vp, u32, u64, sz, i32 = C.c_void_p, C.c_uint32, C.c_uint64, C.c_size_t, C.c_int
    sig = {
        "brng_create": ([u64, u32, u32, C.POINTER(vp)], i32),
        "brng_destroy": ([vp], i32),
        "brng_set_tuning": ([vp, C.POINTER(brng_tuning_t)], i32),
        "brng_get_tuning": ([vp, C.POINTER(brng_tuning_t)], i32),
        "brng_n_streams": ([vp], u32),
        "brng_seed": ([vp], u64),
        "brng_get_positions": ([vp, vp], i32),
        "brng_set_positions": ([vp, vp], i32),
        "brng_get_positions_u64": ([vp, vp], i32),
        "brng_set_positions_u64": ([vp, vp], i32),
        "brng_read_counters": ([vp, vp, C.POINTER(brng_counters_t), i32], i32),
        "brng_philox_words": ([vp, u32, u32, u64, sz, vp, vp], i32),
        "brng_fp64_eval": ([u32, sz, vp, vp, vp], i32),
        "brng_fp32_eval": ([u32, sz, vp, vp, vp], i32),
        "brng_philox_peak": ([u64, u32, u32, vp, vp], i32),
        "brng_uniform": ([vp, sz, vp, vp, vp, vp, vp], i32),
        "brng_uniform_f64": ([vp, sz, vp, vp, vp, vp, vp], i32),
        "brng_normal": ([vp, sz, vp, vp, vp, vp, vp], i32),
        "brng_exponential": ([vp, sz, vp, vp, vp, vp], i32),
        "brng_gamma": ([vp, sz, vp, vp, vp, vp], i32),
        "brng_laplace": ([vp, sz, vp, vp, vp, vp, vp], i32),
        "brng_weibull": ([vp, sz, vp, vp, vp, vp, vp], i32),
        "brng_poisson": ([vp, sz, vp, vp, vp, vp], i32),
        "brng_binomial": ([vp, sz, vp, vp, vp, vp, vp], i32),
        "brng_mixed": ([vp, sz, vp, vp, vp, vp, vp, vp], i32),
        "brng_dirichlet": ([vp, sz, u32, vp, vp, vp], i32),
        "brng_gamma_static": ([u64, u32, sz, vp, vp, vp, vp], i32),
        "brng_gibbs_run": ([vp, i32, u64, u32, u32, vp, vp, vp, vp], i32),
        "brng_lda_index": ([u32, vp, vp, vp, vp], i32),
        "brng_lda_apply": ([u32, u32, vp, vp, vp, vp], i32),
        "brng_batch_create": ([vp, vp, u32, C.POINTER(vp)], i32),
        "brng_batch_launch": ([vp, vp], i32),
        "brng_batch_destroy": ([vp], i32),
        "brng_gibbs_batch": ([vp, vp, u32, vp], i32),
        "brng_serve_open": ([u64, u32, vp, C.POINTER(vp)], i32),
        "brng_serve_submit": ([vp, C.POINTER(brng_request_t), C.POINTER(u64)], i32),
        "brng_serve_poll": ([vp, u64, C.POINTER(C.c_int)], i32),
        "brng_serve_wait": ([vp, u64, C.c_double], i32),
        "brng_serve_result": ([vp, u64, vp, vp, C.POINTER(brng_job_info_t)], i32),
        "brng_serve_stats": ([vp, C.POINTER(brng_serve_stats_t)], i32),
        "brng_serve_close": ([vp], i32),
        "brng_serve_cancel": ([vp, u64], i32),
        "brng_debug_violations": ([C.POINTER(u64), i32], i32),
        "brng_test_pc_stall": ([vp, u32, u32, vp, vp, vp, vp], i32),
    }
    for name, (args, res) in sig.items():
        fn = getattr(L, name)
        fn.argtypes = args
        fn.restype = res
    return L


lib = _load()


# ---- marshalling helpers ----------------------------------------------------

def _ptr(t, dtype=None, name="array"):
    """Device pointer of a contiguous torch CUDA tensor (None -> NULL)."""
    if t is None:
        return None
    if isinstance(t, int):
        return t
    import torch
    if not t.is_cuda:
        raise ValueError("%s must be a CUDA tensor" % name)
    if dtype is not None and t.dtype != dtype:
        raise ValueError("%s must be %s, got %s" % (name, dtype, t.dtype))
    if not t.is_contiguous():
        raise ValueError("%s must be contiguous" % name)
    return t.data_ptr()


def _stream(stream):
    import torch
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    if isinstance(stream, int):
        return stream
    return stream.cuda_stream


def _check(call, code, ok=(BRNG_OK,)):
    if code not in ok:
        raise BrngError(call, code)
    return code


def _f32():
    import torch
    return torch.float32


# ---- the C calls, same names --------------------------------------------------

def brng_create(seed, n_streams, buf_len=0):
    h = C.c_void_p()
    _check("brng_create", lib.brng_create(int(seed) & (2**64 - 1), int(n_streams), int(buf_len), C.byref(h)))
    return h


def brng_destroy(h):
    return _check("brng_destroy", lib.brng_destroy(h))


def brng_set_tuning(h, buf_len=0, warps_per_block=0, lanes_per_chain=0, lookahead=0, producer_warps=0):
    t = brng_tuning_t(buf_len, warps_per_block, lanes_per_chain, lookahead, producer_warps)
    return _check("brng_set_tuning", lib.brng_set_tuning(h, C.byref(t)))


def brng_get_tuning(h):
    t = brng_tuning_t()
    _check("brng_get_tuning", lib.brng_get_tuning(h, C.byref(t)))
    return {f: getattr(t, f) for f, _ in t._fields_}


def brng_get_positions(h):
    out = np.zeros(3 * lib.brng_n_streams(h), dtype=np.uint64)
    _check("brng_get_positions", lib.brng_get_positions(h, out.ctypes.data_as(C.c_void_p)))
    return out


def brng_get_positions_u64(h):
    out = np.zeros(lib.brng_n_streams(h), dtype=np.uint64)
    _check("brng_get_positions_u64", lib.brng_get_positions_u64(h, out.ctypes.data_as(C.c_void_p)))
    return out


def brng_set_positions_u64(h, pos):
    pos = np.ascontiguousarray(pos, dtype=np.uint64)
    return _check("brng_set_positions_u64", lib.brng_set_positions_u64(h, pos.ctypes.data_as(C.c_void_p)))


def brng_set_positions(h, pos):
    pos = np.ascontiguousarray(pos, dtype=np.uint64)
    return _check("brng_set_positions", lib.brng_set_positions(h, pos.ctypes.data_as(C.c_void_p)))


def brng_read_counters(h, stream=None, reset=False):
    c = brng_counters_t()
    code = lib.brng_read_counters(h, _stream(stream), C.byref(c), int(bool(reset)))
    _check("brng_read_counters", code, ok=(BRNG_OK, BRNG_EDOMAIN, BRNG_EREJECT, BRNG_ETIMEOUT))
    return code, c.as_dict()


def brng_philox_words(h, domain, stream_id, first_block, n_blocks, out, stream=None):
    import torch
    return _check("brng_philox_words", lib.brng_philox_words(
        h, domain, stream_id, first_block, n_blocks, _ptr(out, torch.int32, "out"), _stream(stream)))


def brng_philox_peak(iters, blocks, threads, sink, stream=None):
    import torch
    return _check("brng_philox_peak", lib.brng_philox_peak(
        int(iters), int(blocks), int(threads), _ptr(sink, torch.int32, "sink"), _stream(stream)))


def brng_fp32_eval(fn, x, out, stream=None):
    return _check("brng_fp32_eval", lib.brng_fp32_eval(
        int(fn), x.numel(), _ptr(x, _f32(), "in"), _ptr(out, _f32(), "out"), _stream(stream)))


def brng_fp64_eval(fn, x, out, stream=None):
    import torch
    return _check("brng_fp64_eval", lib.brng_fp64_eval(
        int(fn), x.numel(), _ptr(x, torch.float64, "in"), _ptr(out, torch.float64, "out"), _stream(stream)))


def brng_uniform(h, a, b, out, words=None, stream=None):
    import torch
    return _check("brng_uniform", lib.brng_uniform(
        h, out.numel(), _ptr(a, _f32(), "a"), _ptr(b, _f32(), "b"), _ptr(out, _f32(), "out"),
        _ptr(words, torch.int32, "words"), _stream(stream)))


def brng_uniform_f64(h, a, b, out, words=None, stream=None):
    import torch
    return _check("brng_uniform_f64", lib.brng_uniform_f64(
        h, out.numel(), _ptr(a, torch.float64, "a"), _ptr(b, torch.float64, "b"),
        _ptr(out, torch.float64, "out"), _ptr(words, torch.int32, "words"), _stream(stream)))


def brng_normal(h, mu, sigma, out, words=None, stream=None):
    import torch
    return _check("brng_normal", lib.brng_normal(
        h, out.numel(), _ptr(mu, _f32(), "mu"), _ptr(sigma, _f32(), "sigma"), _ptr(out, _f32(), "out"),
        _ptr(words, torch.int32, "words"), _stream(stream)))


def brng_poisson(h, lam, out, words=None, stream=None):
    import torch
    return _check("brng_poisson", lib.brng_poisson(
        h, out.numel(), _ptr(lam, _f32(), "lambda"), _ptr(out, _f32(), "out"),
        _ptr(words, torch.int32, "words"), _stream(stream)))


def brng_binomial(h, trials, prob, out, words=None, stream=None):
    import torch
    return _check("brng_binomial", lib.brng_binomial(
        h, out.numel(), _ptr(trials, _f32(), "trials"), _ptr(prob, _f32(), "prob"), _ptr(out, _f32(), "out"),
        _ptr(words, torch.int32, "words"), _stream(stream)))


def brng_exponential(h, lam, out, words=None, stream=None):
    import torch
    return _check("brng_exponential", lib.brng_exponential(
        h, out.numel(), _ptr(lam, _f32(), "lambda"), _ptr(out, _f32(), "out"),
        _ptr(words, torch.int32, "words"), _stream(stream)))


def brng_gamma(h, alpha, out, words=None, stream=None):
    import torch
    return _check("brng_gamma", lib.brng_gamma(
        h, out.numel(), _ptr(alpha, _f32(), "alpha"), _ptr(out, _f32(), "out"),
        _ptr(words, torch.int32, "words"), _stream(stream)))


def brng_laplace(h, mu, b, out, words=None, stream=None):
    import torch
    return _check("brng_laplace", lib.brng_laplace(
        h, out.numel(), _ptr(mu, _f32(), "mu"), _ptr(b, _f32(), "b"), _ptr(out, _f32(), "out"),
        _ptr(words, torch.int32, "words"), _stream(stream)))


def brng_weibull(h, k, lam, out, words=None, stream=None):
    import torch
    return _check("brng_weibull", lib.brng_weibull(
        h, out.numel(), _ptr(k, _f32(), "k"), _ptr(lam, _f32(), "lambda"), _ptr(out, _f32(), "out"),
        _ptr(words, torch.int32, "words"), _stream(stream)))


def brng_mixed(h, tag, p0, p1, out, words=None, stream=None):
    import torch
    return _check("brng_mixed", lib.brng_mixed(
        h, out.numel(), _ptr(tag, torch.uint8, "tag"), _ptr(p0, _f32(), "p0"), _ptr(p1, _f32(), "p1"),
        _ptr(out, _f32(), "out"), _ptr(words, torch.int32, "words"), _stream(stream)))


def brng_gamma_static(seed, n_streams, alpha, out, words=None, stream=None):
    """Gamma draws with no device allocation (see include/brng.h): for
    callers that must not call cudaMalloc.  Streams start at their first
    element on every call; calls must not overlap on the GPU."""
    import torch
    return _check("brng_gamma_static", lib.brng_gamma_static(
        int(seed) & (2**64 - 1), int(n_streams), out.numel(), _ptr(alpha, _f32(), "alpha"),
        _ptr(out, _f32(), "out"), _ptr(words, torch.int32, "words"), _stream(stream)))


def brng_dirichlet(h, alpha, out, stream=None):
    n_rows, K = alpha.shape
    return _check("brng_dirichlet", lib.brng_dirichlet(
        h, n_rows, K, _ptr(alpha, _f32(), "alpha"), _ptr(out, _f32(), "out"), _stream(stream)))


def brng_lda_index(doc_ptr, words, prev, stream=None):
    import torch
    return _check("brng_lda_index", lib.brng_lda_index(
        doc_ptr.numel() - 1, _ptr(doc_ptr, torch.int32, "doc_ptr"), _ptr(words, torch.int32, "words"),
        _ptr(prev, torch.int32, "prev"), _stream(stream)))


def brng_lda_apply(K, V, nkw, nk, dnkw, stream=None):
    import torch
    return _check("brng_lda_apply", lib.brng_lda_apply(
        int(K), int(V), _ptr(nkw, torch.int32, "nkw"), _ptr(nk, torch.int32, "nk"),
        _ptr(dnkw, torch.int32, "dnkw"), _stream(stream)))


class LdaFull:
    """Device arrays of the LDA_FULL model for one corpus (torch tensors; the
    32-bit unsigned arrays are held as int32 and passed by pointer):
    doc_ptr, words, prev, z, z_start, ndk, nkw, nk, dnkw, dir_alpha, zpos,
    theta, pos, mom.  `corpus`/`state` are the numpy dicts of
    inputs.lda_corpus / inputs.lda_initial_state; prev is built on the device
    with brng_lda_index."""

    def __init__(self, corpus, state, alpha=0.1, beta=0.01, device="cuda", stream=None):
        import torch

        def dev(a, dtype):
            return torch.from_numpy(np.ascontiguousarray(a).view(dtype)).to(device)

        self.K, self.V = int(corpus["K"]), int(corpus["V"])
        self.alpha, self.beta = float(alpha), float(beta)
        self.n_docs = corpus["doc_ptr"].size - 1
        n_tok = corpus["words"].size
        self.doc_ptr = dev(corpus["doc_ptr"].astype(np.uint32), np.int32)
        self.words = dev(corpus["words"].astype(np.uint32), np.int32)
        self.prev = torch.empty(n_tok, dtype=torch.int32, device=device)
        self.z = dev(state["z"].astype(np.uint8), np.uint8)
        self.z_start = torch.empty(n_tok, dtype=torch.uint8, device=device)
        self.ndk = dev(state["ndk"].astype(np.int32), np.int32)
        self.nkw = dev(state["nkw"].astype(np.int32), np.int32)
        self.nk = dev(state["nk"].astype(np.int32), np.int32)
        self.dnkw = torch.zeros(self.V * self.K + self.K, dtype=torch.int32, device=device)
        self.dir_alpha = torch.empty((self.n_docs, self.K), dtype=torch.float32, device=device)
        self.zpos = dev(state["zpos"].astype(np.uint64), np.int64)
        self.theta = torch.zeros((self.n_docs, self.K), dtype=torch.float32, device=device)
        self.pos = dev(state["pos"].astype(np.uint64), np.int64)
        self.mom = dev(state["mom"].astype(np.float64), np.float64)
        # documents start longest first (speed only: the draws do not depend on it)
        lengths = np.diff(corpus["doc_ptr"].astype(np.int64))
        self.order = dev(np.argsort(-lengths, kind="stable").astype(np.uint32), np.int32)
        brng_lda_index(self.doc_ptr, self.words, self.prev, stream)

    def params(self, exchange=0, ordered=True):
        return brng_lda_full_params_t(self.K, self.V, self.alpha, self.beta, self.doc_ptr.data_ptr(),
                                      self.words.data_ptr(), self.prev.data_ptr(), int(exchange),
                                      self.order.data_ptr() if ordered else None)

    def state(self):
        return brng_lda_full_state_t(*[t.data_ptr() for t in (
            self.z, self.z_start, self.ndk, self.nkw, self.nk, self.dnkw, self.dir_alpha, self.zpos,
            self.theta, self.pos)])

    def run(self, h, n_sweeps, doc_offset=0, stream=None, exchange=0, ordered=True):
        """h: a Handle or a raw brng_t* (its seed keys the draws; its tuning
        sets the theta draw's rings, which never changes a value: that draw
        runs one sweep per launch, so Handle.tune(buf_len=8, lookahead=1,
        warps_per_block=2) wastes least -- about 8 % faster per sweep than
        the defaults at 16,384 documents).  `h` stays referenced for the
        whole call, so a Handle made in the argument list is not destroyed
        under it."""
        raw = getattr(h, "h", h)
        return brng_gibbs_run(raw, MODEL_LDA_FULL, doc_offset, self.n_docs, n_sweeps, self.params(exchange, ordered),
                              self.state(), self.mom, stream)

    def host(self):
        """The state as numpy arrays (the oracle's dict layout)."""
        g = lambda t: t.detach().cpu().numpy()  # noqa: E731
        return dict(z=g(self.z), ndk=g(self.ndk), nkw=g(self.nkw).reshape(self.V, self.K), nk=g(self.nk),
                    zpos=g(self.zpos).view(np.uint64), pos=g(self.pos).view(np.uint64), mom=g(self.mom),
                    theta=g(self.theta), dnkw=g(self.dnkw), prev=g(self.prev).view(np.uint32))


def brng_gibbs_run(h, model, chain_offset, n_chains, n_sweeps, params, state, moments, stream=None):
    """`params` / `state`: ctypes structures (passed by reference) or device
    tensors, as include/brng.h specifies per model."""
    import torch

    def ref(x):
        if x is None:
            return None
        if isinstance(x, C.Structure):
            return C.cast(C.byref(x), C.c_void_p)
        return _ptr(x, None, "state")

    return _check("brng_gibbs_run", lib.brng_gibbs_run(
        h, int(model), int(chain_offset), int(n_chains), int(n_sweeps), ref(params), ref(state),
        _ptr(moments, torch.float64, "moments"), _stream(stream)))


def make_job(model, n_chains, n_sweeps, seed, params, state, moments, chain_offset=0):
    """A brng_job_t; `params` / `state` as for brng_gibbs_run (a ctypes
    structure is referenced by address, so keep it alive while the job is
    used).  Returns (job, keepalive)."""
    def addr(x):
        if x is None:
            return None
        if isinstance(x, C.Structure):
            return C.addressof(x)
        return _ptr(x, None, "state")
    j = brng_job_t(int(model), int(n_chains), int(n_sweeps), 0, int(seed) & (2**64 - 1),
                   int(chain_offset), addr(params), addr(state), _ptr(moments, None, "moments"))
    return j, (params, state, moments)


def _job_array(jobs):
    arr = (brng_job_t * len(jobs))(*jobs)
    return arr


def brng_gibbs_batch(h, jobs, stream=None):
    arr = _job_array(jobs)
    return _check("brng_gibbs_batch", lib.brng_gibbs_batch(h, C.cast(arr, C.c_void_p), len(jobs),
                                                           _stream(stream)))


def brng_batch_create(h, jobs):
    arr = _job_array(jobs)
    b = C.c_void_p()
    _check("brng_batch_create", lib.brng_batch_create(h, C.cast(arr, C.c_void_p), len(jobs), C.byref(b)))
    return b


def brng_batch_launch(b, stream=None):
    return _check("brng_batch_launch", lib.brng_batch_launch(b, _stream(stream)))


def brng_batch_destroy(b):
    return _check("brng_batch_destroy", lib.brng_batch_destroy(b))


def brng_serve_open(mem_budget, max_inflight=4, buf_len=0, warps_per_block=0, lookahead=0):
    s = C.c_void_p()
    t = brng_tuning_t(buf_len, warps_per_block, 0, lookahead, 0)
    _check("brng_serve_open", lib.brng_serve_open(int(mem_budget), int(max_inflight), C.byref(t), C.byref(s)))
    return s


def brng_serve_submit(s, req):
    """`req`: a brng_request_t whose host arrays stay alive until the call returns."""
    jid = C.c_uint64()
    _check("brng_serve_submit", lib.brng_serve_submit(s, C.byref(req), C.byref(jid)))
    return jid.value


def brng_serve_poll(s, job_id):
    done = C.c_int()
    code = lib.brng_serve_poll(s, job_id, C.byref(done))
    return code, bool(done.value)


def brng_serve_wait(s, job_id, timeout_s):
    return lib.brng_serve_wait(s, job_id, float(timeout_s))


def brng_serve_result(s, job_id, host_state=None, host_moments=None):
    """host_state / host_moments: writable numpy arrays (or None)."""
    info = brng_job_info_t()
    ps = None if host_state is None else host_state.ctypes.data_as(C.c_void_p)
    pm = None if host_moments is None else host_moments.ctypes.data_as(C.c_void_p)
    code = lib.brng_serve_result(s, job_id, ps, pm, C.byref(info))
    return code, {f: getattr(info, f) for f, _ in info._fields_ if f != "pad"}


def brng_serve_stats(s):
    st = brng_serve_stats_t()
    code = lib.brng_serve_stats(s, C.byref(st))
    return code, {f: getattr(st, f) for f, _ in st._fields_}


def brng_serve_close(s):
    return _check("brng_serve_close", lib.brng_serve_close(s))


def brng_serve_cancel(s, job_id):
    """BRNG_OK (withdrawn), BRNG_EAGAIN (already admitted) or BRNG_ENOTFOUND."""
    return lib.brng_serve_cancel(s, int(job_id))


def brng_debug_violations(reset=False):
    """Failed protocol checks of the checked build since the last reset, or
    None for the normal build."""
    n = C.c_uint64()
    code = lib.brng_debug_violations(C.byref(n), int(bool(reset)))
    return n.value if code == BRNG_OK else None


def brng_test_pc_stall(h, n_chains, n_sweeps, params, state, moments, stream=None):
    """Failure-path test hook: the producer/consumer sampler with producers
    that write nothing (every consumer wait runs out after its bound)."""
    return _check("brng_test_pc_stall", lib.brng_test_pc_stall(
        h, int(n_chains), int(n_sweeps), C.cast(C.byref(params), C.c_void_p) if params is not None else None,
        _ptr(state, None, "state"), _ptr(moments, None, "moments"), _stream(stream)))


# ---- state layouts (marshalling of the C structs held in device tensors) ------

def triangle_state(n, x0=0.5, y0=0.5, device="cuda"):
    """brng_triangle_state_t[n] as a float64 tensor [n, 4]: x, y, pos bits, pad."""
    import torch
    s = torch.zeros((n, 4), dtype=torch.float64, device=device)
    s[:, 0] = x0
    s[:, 1] = y0
    return s


def triangle_unpack(s):
    a = s.detach().cpu()
    return a[:, 0].numpy(), a[:, 1].numpy(), a[:, 2].view(__import__("torch").int64).numpy().view(np.uint64)


def normal_gamma_state(n, mu0=0.0, device="cuda"):
    """brng_normal_gamma_state_t[n] (24 bytes: mu, tau as float32; pos_n, pos_u
    as uint64) as an int64 tensor [n, 3]."""
    import torch
    s = torch.zeros((n, 3), dtype=torch.int64, device=device)
    f = s.view(torch.float32).view(n, 6)
    f[:, 0] = mu0
    return s


def normal_gamma_unpack(s):
    import torch
    a = s.detach().cpu()
    f = a.view(torch.float32).view(-1, 6)
    return (f[:, 0].numpy().copy(), f[:, 1].numpy().copy(),
            a[:, 1].numpy().view(np.uint64).copy(), a[:, 2].numpy().view(np.uint64).copy())


class Handle:
    """Owns a brng_t*; a convenience wrapper over the brng_* calls."""

    def __init__(self, seed, n_streams, buf_len=0):
        self.h = brng_create(seed, n_streams, buf_len)
        self.n_streams = n_streams
        self.seed = seed

    def close(self):
        if self.h:
            brng_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def tune(self, **kw):
        brng_set_tuning(self.h, **kw)
        return self

    @property
    def tuning(self):
        return brng_get_tuning(self.h)

    def positions(self):
        return brng_get_positions(self.h)

    def set_positions(self, pos):
        brng_set_positions(self.h, pos)

    def positions_u64(self):
        return brng_get_positions_u64(self.h)

    def set_positions_u64(self, pos):
        brng_set_positions_u64(self.h, pos)

    def counters(self, stream=None, reset=False):
        return brng_read_counters(self.h, stream, reset)
