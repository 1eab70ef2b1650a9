"""Failure detection without a GPU fault.

* Device: the producer/consumer sampler's ring waits are bounded.  A test hook
  runs it with producers that write nothing (a flag that nothing sets), so
  every consumer wait runs out after its bound: the call ends in a few
  seconds, the chains are NaN, n_timeout counts the expired waits,
  brng_read_counters returns BRNG_ETIMEOUT, and the next run on the same
  handle and context is correct.
* Host (the server): malformed requests are refused at submit; a queued job
  can be cancelled, an admitted one cannot; closing with jobs still queued
  cancels them and returns; a submitting thread that dies mid-way leaves the
  other clients' jobs unaffected.
"""
import threading
import time

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_4825_gb300 import brng as B  # noqa: E402
from paper_1412_4825_gb300 import inputs, serve  # noqa: E402

DEV = torch.device("cuda:0")


def _ng(n):
    nobs, xbar, sc = inputs.normal_gamma_data(n, seed=3)
    d = [torch.from_numpy(a).to(DEV) for a in (nobs, xbar, sc)]
    p = B.brng_normal_gamma_params_t(2.0, 1.0, 0.0, 0.01, *[x.data_ptr() for x in d])
    return p, d


def test_bounded_wait_runs_out_and_context_survives():
    n, sweeps = 64, 50
    p, keep = _ng(n)
    h = B.Handle(42, 1)
    h.tune(producer_warps=1, warps_per_block=2)
    st = B.normal_gamma_state(n, device=DEV)
    mom = torch.zeros((n, 4), dtype=torch.float64, device=DEV)
    t0 = time.monotonic()
    B.brng_test_pc_stall(h.h, n, sweeps, p, st, mom)
    code, cnt = h.counters(reset=True)
    elapsed = time.monotonic() - t0
    assert code == B.BRNG_ETIMEOUT and cnt["n_timeout"] >= 2, cnt  # two consumer warps
    assert elapsed < 30.0
    mu, tau, _, _ = B.normal_gamma_unpack(st)
    assert np.isnan(mu).all() and np.isnan(tau).all()
    # the same handle and context go on working: a normal run equals a fresh handle's
    runs = []
    for hh in (h, B.Handle(42, 1)):
        s2 = B.normal_gamma_state(n, device=DEV)
        m2 = torch.zeros((n, 4), dtype=torch.float64, device=DEV)
        B.brng_gibbs_run(hh.h, B.MODEL_NORMAL_GAMMA, 0, n, sweeps, p, s2, m2)
        runs.append((s2, m2))
    code, cnt = h.counters()
    assert code == B.BRNG_OK and cnt["n_timeout"] == 0
    assert torch.equal(runs[0][0], runs[1][0]) and torch.equal(runs[0][1], runs[1][1])


def test_serve_rejects_malformed_requests():
    pool = serve.InputPool(256, 64, 1)
    srv = B.brng_serve_open(1 << 26)
    bad = []
    r = serve.make_request(pool, B.MODEL_TRIANGLE, 10, 5, 1)
    r.model = 9
    bad.append(r)
    bad.append(serve.make_request(pool, B.MODEL_TRIANGLE, 0, 5, 1))  # no chains
    r = serve.make_request(pool, B.MODEL_NORMAL_GAMMA, 10, 5, 1)
    r.nobs = None
    bad.append(r)
    for k in (0, 200):
        r = serve.make_request(pool, B.MODEL_LDA, 10, 5, 1)
        r.K = k
        bad.append(r)
    for r in bad:
        with pytest.raises(B.BrngError):
            B.brng_serve_submit(srv, r)
    assert B.brng_serve_wait(srv, 12345, 0.1) == B.BRNG_ENOTFOUND
    assert B.brng_serve_poll(srv, 12345)[0] == B.BRNG_ENOTFOUND
    assert B.brng_serve_cancel(srv, 12345) == B.BRNG_ENOTFOUND
    code, st = B.brng_serve_stats(srv)
    assert code == B.BRNG_OK and st["submitted"] == 0
    B.brng_serve_close(srv)


def test_serve_cancel_queued_jobs():
    """A budget that admits one job at a time: the first job runs, the queued
    ones can be cancelled (and are then unknown), the rest complete."""
    pool = serve.InputPool(4096, 64, 2)
    req = lambda seed: serve.make_request(pool, B.MODEL_NORMAL_GAMMA, 4096, 2000, seed)  # noqa: E731
    one = B.brng_serve_open(1 << 30)
    jid = B.brng_serve_submit(one, req(0))
    assert B.brng_serve_wait(one, jid, 60.0) == B.BRNG_OK
    per_job = B.brng_serve_result(one, jid)[1]["device_bytes"]
    B.brng_serve_close(one)
    srv = B.brng_serve_open(per_job + per_job // 2)
    ids = [B.brng_serve_submit(srv, req(10 + i)) for i in range(6)]
    # the first job finishes; its memory returns only when its result is
    # collected, so the other five are still waiting for memory
    assert B.brng_serve_wait(srv, ids[0], 60.0) == B.BRNG_OK
    assert B.brng_serve_stats(srv)[1]["queued"] == 5
    assert B.brng_serve_cancel(srv, ids[0]) == B.BRNG_EAGAIN  # ran: cannot be withdrawn
    cancelled = ids[3:]
    for i in cancelled:
        assert B.brng_serve_cancel(srv, i) == B.BRNG_OK
        assert B.brng_serve_cancel(srv, i) == B.BRNG_ENOTFOUND
    for i in ids:
        if i in cancelled:
            assert B.brng_serve_wait(srv, i, 1.0) == B.BRNG_ENOTFOUND
            assert B.brng_serve_result(srv, i)[0] == B.BRNG_ENOTFOUND
        else:
            assert B.brng_serve_wait(srv, i, 120.0) == B.BRNG_OK
            assert B.brng_serve_result(srv, i)[0] == B.BRNG_OK
    code, st = B.brng_serve_stats(srv)
    assert st["cancelled"] == len(cancelled) and st["completed"] == len(ids) - len(cancelled)
    B.brng_serve_close(srv)


def test_serve_close_cancels_queue_and_returns():
    pool = serve.InputPool(4096, 64, 3)
    srv = B.brng_serve_open(1 << 21)  # a few of these jobs at a time
    ids = [B.brng_serve_submit(srv, serve.make_request(pool, B.MODEL_TRIANGLE, 4096, 20000, i))
           for i in range(40)]
    code, st = B.brng_serve_stats(srv)
    assert st["submitted"] == len(ids)
    t0 = time.monotonic()
    B.brng_serve_close(srv)  # finishes the launched batches, cancels the rest
    assert time.monotonic() - t0 < 60.0


def test_serve_survives_a_dying_submitter():
    """One client thread raises after two submissions; another keeps
    submitting; every submitted job completes with the results it has alone."""
    pool = serve.InputPool(2048, 64, 4)
    srv = B.brng_serve_open(1 << 28, max_inflight=2)
    ids, errors, lock = [], [], threading.Lock()

    def client(seeds, die_after):
        try:
            for k, sd in enumerate(seeds):
                if k == die_after:
                    raise RuntimeError("client failure")
                jid = B.brng_serve_submit(srv, serve.make_request(pool, B.MODEL_NORMAL_GAMMA, 2048, 300, sd))
                with lock:
                    ids.append((jid, sd))
        except RuntimeError as e:
            errors.append(e)

    ta = threading.Thread(target=client, args=([101, 102, 103, 104], 2))
    tb = threading.Thread(target=client, args=([201, 202, 203], None))
    ta.start(); tb.start(); ta.join(); tb.join()
    assert len(errors) == 1 and len(ids) == 5
    for jid, sd in ids:
        assert B.brng_serve_wait(srv, jid, 120.0) == B.BRNG_OK
        hs, hm = np.zeros((2048, 3), np.int64), np.zeros((2048, 4), np.float64)
        assert B.brng_serve_result(srv, jid, hs, hm)[0] == B.BRNG_OK
        h = B.Handle(sd, 1)
        d = [torch.from_numpy(a[:2048].copy()).to(DEV) for a in (pool.nobs, pool.xbar, pool.sc)]
        p = B.brng_normal_gamma_params_t(2.0, 1.0, 0.0, 0.01, *[x.data_ptr() for x in d])
        st = B.normal_gamma_state(2048, device=DEV)
        mom = torch.zeros((2048, 4), dtype=torch.float64, device=DEV)
        B.brng_gibbs_run(h.h, B.MODEL_NORMAL_GAMMA, 0, 2048, 300, p, st, mom)
        assert np.array_equal(hs.view(np.uint8), st.cpu().numpy().view(np.uint8))
        assert np.array_equal(hm, mom.cpu().numpy())
        h.close()
    code, st = B.brng_serve_stats(srv)
    assert st["completed"] == 5
    B.brng_serve_close(srv)
