"""Workloads run through one build of the library (the in-tree libbrng.so, or
the checked build named by BRNG_LIB) by tests/test_gpu_checked_build.py:
prints one JSON line with a digest of every workload's outputs and the
checked build's count of failed protocol checks (None for the normal build).

Small sizes, but every ring path: the normal-gamma sampler at every
speculation width (ring 32, 16, 8) and the plain loop (ring 4), boosted
shapes, producer warps, a run resumed from mid-block positions; the triangle
sampler at 1, 4 and 16 lanes per chain; LDA at K = 64 and K = 100; the mixed
stream with all eight tags; bulk Gamma, Dirichlet, Poisson, Binomial (small
and large means) and FP64
uniforms; one batch of all three models.
"""
import hashlib
import json
import os
import sys

import numpy as np
import torch

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
from paper_1412_4825_gb300 import brng as B  # noqa: E402
from paper_1412_4825_gb300 import inputs  # noqa: E402

DEV = torch.device("cuda:0")
out = {}


def digest(*tensors):
    h = hashlib.sha1()
    for t in tensors:
        h.update(t.detach().cpu().contiguous().numpy().tobytes())
    return h.hexdigest()[:16]


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


def ng(name, n, sweeps, prior=(2.0, 1.0, 0.0, 0.01), split=None, **tune):
    nobs, xbar, sc = inputs.normal_gamma_data(n, seed=7)
    d = [T(nobs), T(xbar), T(sc)]
    p = B.brng_normal_gamma_params_t(*prior, *[x.data_ptr() for x in d])
    h = B.Handle(42, 1)
    h.tune(**tune)
    st = B.normal_gamma_state(n, device=DEV)
    m = torch.zeros((n, 4), dtype=torch.float64, device=DEV)
    for part in (split or [sweeps]):
        B.brng_gibbs_run(h.h, B.MODEL_NORMAL_GAMMA, 0, n, part, p, st, m)
    out[name] = digest(st, m)
    h.close()


def tri(name, lanes):
    n = 256
    h = B.Handle(42, 1)
    h.tune(lanes_per_chain=lanes, buf_len=64)
    st = B.triangle_state(n, device=DEV)
    m = torch.zeros((n, 5), dtype=torch.float64, device=DEV)
    B.brng_gibbs_run(h.h, B.MODEL_TRIANGLE, 0, n, 300, None, st, m)
    out[name] = digest(st, m)
    h.close()


def lda(name, K):
    docs = 200
    alpha = (0.1 + np.random.default_rng(K).poisson(1.0, (docs, K))).astype(np.float32)
    a = T(alpha)
    theta = torch.zeros((docs, K), dtype=torch.float32, device=DEV)
    pos = torch.zeros((docs, K, 2), dtype=torch.int64, device=DEV)
    mom = torch.zeros((docs, K), dtype=torch.float64, device=DEV)
    h = B.Handle(42, 1)
    B.brng_gibbs_run(h.h, B.MODEL_LDA, 0, docs, 20, B.brng_lda_params_t(K, a.data_ptr()),
                     B.brng_lda_state_t(theta.data_ptr(), pos.data_ptr()), mom)
    out[name] = digest(theta, pos, mom)
    h.close()


def main():
    for bl in (32, 16, 8, 4):
        ng("ng_ring%d" % bl, 3000, 60, buf_len=bl, warps_per_block=8)
    ng("ng_boosted", 1000, 60, prior=(0.4, 1.0, 0.0, 0.01), buf_len=32)
    ng("ng_producers", 3000, 60, buf_len=32, producer_warps=2)
    ng("ng_resumed", 3000, 60, split=[17, 43], buf_len=32)
    for lanes in (1, 4, 16):
        tri("triangle_lanes%d" % lanes, lanes)
    lda("lda_k64", 64)
    lda("lda_k100", 100)
    n, S = 1 << 18, 1 << 12
    tag, p0, p1 = inputs.mixed_stream(n, seed=3, n_tags=8)
    for bl in (8, 16):
        h = B.Handle(9, S)
        h.tune(buf_len=bl)
        o = torch.empty(n, dtype=torch.float32, device=DEV)
        w = torch.empty(n, dtype=torch.int32, device=DEV)
        B.brng_mixed(h.h, T(tag), T(p0), T(p1), o, w)
        out["mixed_ring%d" % bl] = digest(o, w) + ":" + hashlib.sha1(h.positions().tobytes()).hexdigest()[:8]
        h.close()
    h = B.Handle(11, 1000)
    alpha = T(inputs.shape_params(50000, seed=1))
    o = torch.empty(50000, dtype=torch.float32, device=DEV)
    B.brng_gamma(h.h, alpha, o)
    out["gamma"] = digest(o)
    lam = T(inputs.poisson_params(50000, seed=2))
    B.brng_poisson(h.h, lam, o)
    out["poisson"] = digest(o)
    tr, pr = inputs.binomial_params(50000, seed=3)
    B.brng_binomial(h.h, T(tr), T(pr), o)
    out["binomial"] = digest(o)
    # large means (PTRS / BTRD): the checked build redoes every attempt the
    # FP32 path decided in FP64 and counts a differing result as a violation
    rng = np.random.default_rng(4)
    lam = T(inputs.log_uniform(rng, 64.0, 1e7, 50000))
    B.brng_poisson(h.h, lam, o)
    out["poisson_large"] = digest(o)
    tr = np.floor(inputs.log_uniform(rng, 130.0, 16777216.0, 50000)).astype(np.float32)
    pr = rng.random(50000).astype(np.float32)
    pr[::3] = np.float32(0.5)
    B.brng_binomial(h.h, T(tr), T(pr), o)
    out["binomial_large"] = digest(o)
    da = T(np.random.default_rng(4).uniform(0.05, 3.0, (1000, 10)).astype(np.float32))
    do = torch.empty((1000, 10), dtype=torch.float32, device=DEV)
    B.brng_dirichlet(h.h, da, do)
    out["dirichlet"] = digest(do)
    a64 = T(np.random.default_rng(5).uniform(-1, 0, 50000))
    o64 = torch.empty(50000, dtype=torch.float64, device=DEV)
    B.brng_uniform_f64(h.h, a64, a64 + 1.0, o64)
    out["uniform_f64"] = digest(o64)
    h.close()
    # one batch of the three models
    hb = B.Handle(1, 1)
    nobs, xbar, sc = inputs.normal_gamma_data(700, seed=8)
    d = [T(nobs), T(xbar), T(sc)]
    p = B.brng_normal_gamma_params_t(2.0, 1.0, 0.0, 0.01, *[x.data_ptr() for x in d])
    s1 = B.triangle_state(500, device=DEV)
    m1 = torch.zeros((500, 5), dtype=torch.float64, device=DEV)
    s2 = B.normal_gamma_state(700, device=DEV)
    m2 = torch.zeros((700, 4), dtype=torch.float64, device=DEV)
    alpha = T((0.1 + np.random.default_rng(6).poisson(1.0, (90, 64))).astype(np.float32))
    th = torch.zeros((90, 64), dtype=torch.float32, device=DEV)
    ps = torch.zeros((90, 64, 2), dtype=torch.int64, device=DEV)
    m3 = torch.zeros((90, 64), dtype=torch.float64, device=DEV)
    lp = B.brng_lda_params_t(64, alpha.data_ptr())
    ls = B.brng_lda_state_t(th.data_ptr(), ps.data_ptr())
    jobs, keep = [], []
    for args in [(B.MODEL_TRIANGLE, 500, 40, 21, None, s1, m1), (B.MODEL_NORMAL_GAMMA, 700, 50, 22, p, s2, m2),
                 (B.MODEL_LDA, 90, 10, 23, lp, ls, m3)]:
        j, k = B.make_job(*args)
        jobs.append(j)
        keep.append(k)
    B.brng_gibbs_batch(hb.h, jobs)
    out["batch"] = digest(s1, m1, s2, m2, th, ps, m3)
    hb.close()
    torch.cuda.synchronize()
    print(json.dumps({"digests": out, "violations": B.brng_debug_violations()}), flush=True)


if __name__ == "__main__":
    main()
