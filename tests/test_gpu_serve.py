"""The library's server (continuous batching) through the C ABI.

A job gives the same results served -- admitted under a memory budget that
forces queueing, batched with whatever else is waiting, overlapping with other
batches -- as run alone with brng_gibbs_run; a job larger than the budget is
refused; the Poisson driver completes a small sub-capacity mix.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_4825_gb300 import brng as B  # noqa: E402
from paper_1412_4825_gb300 import serve  # noqa: E402

DEV = torch.device("cuda:0")


def _solo(pool, model, n, sweeps, seed):
    h = B.Handle(seed, 1)
    if model == B.MODEL_TRIANGLE:
        st = B.triangle_state(n, device=DEV)
        mom = torch.zeros((n, 5), dtype=torch.float64, device=DEV)
        B.brng_gibbs_run(h.h, model, 0, n, sweeps, None, st, mom)
        state = st.cpu().numpy()
    elif model == B.MODEL_NORMAL_GAMMA:
        d = [torch.from_numpy(a[:n].copy()).to(DEV) for a in (pool.nobs, pool.xbar, pool.sc)]
        p = B.brng_normal_gamma_params_t(2.0, 1.0, 0.0, 0.01, *[x.data_ptr() for x in d])
        st = B.normal_gamma_state(n, device=DEV)
        mom = torch.zeros((n, 4), dtype=torch.float64, device=DEV)
        B.brng_gibbs_run(h.h, model, 0, n, sweeps, p, st, mom)
        state = st.cpu().numpy()
    else:
        a = torch.from_numpy(pool.alpha[:n].copy()).to(DEV)
        theta = torch.zeros((n, pool.K), dtype=torch.float32, device=DEV)
        pos = torch.zeros((n, pool.K, 2), dtype=torch.int64, device=DEV)
        mom = torch.zeros((n, pool.K), dtype=torch.float64, device=DEV)
        B.brng_gibbs_run(h.h, model, 0, n, sweeps, B.brng_lda_params_t(pool.K, a.data_ptr()),
                         B.brng_lda_state_t(theta.data_ptr(), pos.data_ptr()), mom)
        state = theta.cpu().numpy()
    torch.cuda.synchronize()
    h.close()
    return state, mom.cpu().numpy()


def _host_buffers(pool, model, n):
    if model == B.MODEL_TRIANGLE:
        return np.zeros((n, 4), np.float64), np.zeros((n, 5), np.float64)
    if model == B.MODEL_NORMAL_GAMMA:
        return np.zeros((n, 3), np.int64), np.zeros((n, 4), np.float64)
    return np.zeros((n, pool.K), np.float32), np.zeros((n, pool.K), np.float64)


def test_served_equals_solo_under_tight_budget():
    pool = serve.InputPool(4096, 64, 11)
    rng = np.random.default_rng(3)
    jobs = []
    for i in range(24):
        model = [B.MODEL_TRIANGLE, B.MODEL_NORMAL_GAMMA, B.MODEL_LDA][i % 3]
        n = int(np.exp(rng.uniform(0, np.log(4000 if model != B.MODEL_LDA else 200))))
        jobs.append((model, max(1, n), int(rng.integers(10, 200)), 1000 + i))
    # admission must queue: the largest jobs take ~0.3-0.4 MB each
    budget = 700_000  # every job fits alone; only a few at a time
    srv = B.brng_serve_open(budget, max_inflight=3)
    ids = [B.brng_serve_submit(srv, serve.make_request(pool, *j)) for j in jobs]
    for jid, (model, n, sweeps, seed) in zip(ids, jobs):
        assert B.brng_serve_wait(srv, jid, 120.0) == B.BRNG_OK
        hs, hm = _host_buffers(pool, model, n)
        code, info = B.brng_serve_result(srv, jid, hs, hm)
        assert code == B.BRNG_OK
        assert info["submitted_ns"] <= info["admitted_ns"] <= info["launched_ns"] <= info["completed_ns"]
        ss, sm = _solo(pool, model, n, sweeps, seed)
        assert np.array_equal(hs.view(np.uint8), ss.view(np.uint8)), (model, n, sweeps)
        assert np.array_equal(hm.view(np.uint8), sm.view(np.uint8)), (model, n, sweeps)
    code, st = B.brng_serve_stats(srv)
    assert code == B.BRNG_OK and st["completed"] == len(jobs) and st["device_bytes_in_use"] == 0
    assert st["batches"] >= 2
    B.brng_serve_close(srv)


def test_serve_refuses_job_larger_than_budget():
    pool = serve.InputPool(1024, 64, 12)
    srv = B.brng_serve_open(1 << 16)
    jid = B.brng_serve_submit(srv, serve.make_request(pool, B.MODEL_LDA, 1000, 10, 5))
    assert B.brng_serve_wait(srv, jid, 30.0) == B.BRNG_ENOMEM
    code, info = B.brng_serve_result(srv, jid)
    assert code == B.BRNG_ENOMEM
    assert B.brng_serve_result(srv, jid)[0] == B.BRNG_ENOTFOUND
    B.brng_serve_close(srv)


def test_poisson_mix_small():
    spec = serve.MixSpec(rate=200.0, duration=1.0, chains=(1, 2048), sweeps=(10, 200), seed=5)
    res = serve.run_mix(spec, mem_budget=1 << 30, max_inflight=4)
    s = res.summary()
    print("served mix", s)
    assert res.submitted > 100 and res.failed == 0
    assert res.completed + s["censored"] + res.cancelled == res.submitted
    assert s["completed_fraction"] > 0.8
    assert s["p99_s"] >= s["p50_s"] > 0
