"""Served mix: Poisson arrivals of Gibbs jobs into the library's server.

A host driver for brng_serve_* (include/brng.h): jobs arrive as a Poisson
process, each one of the three Gibbs models chosen uniformly, with a
log-uniform chain count and a uniform sweep count and its own seed; a
collector thread fetches results as jobs finish and records per-job latency
(completion minus submission, steady clock of the library).  All scheduling,
admission by memory budget and batching happens inside the C++ server; this
module only generates arrivals and reads results.
"""
from __future__ import annotations

import threading
import time
from dataclasses import dataclass, field

import numpy as np

from . import brng as B
from . import inputs


@dataclass
class MixSpec:
    rate: float = 2000.0         # jobs per second
    duration: float = 60.0       # seconds of arrivals
    chains: tuple = (1, 65536)   # log-uniform
    sweeps: tuple = (100, 10000) # uniform
    models: tuple = (B.MODEL_TRIANGLE, B.MODEL_NORMAL_GAMMA, B.MODEL_LDA)
    K: int = 64
    seed: int = 42


@dataclass
class MixResult:
    submitted: int = 0
    completed: int = 0
    failed: int = 0
    cancelled: int = 0
    updates: float = 0.0
    latencies: list = field(default_factory=list)      # completed jobs: completion - submission
    censored_ages: list = field(default_factory=list)  # unfinished at the window's end: their age then
    window: float = 0.0                                 # arrival window (s)
    wall: float = 0.0
    stats: dict = field(default_factory=dict)

    def summary(self):
        """Latency percentiles over ALL submitted jobs: a job still unfinished
        when the arrival window closes enters with its age at that moment (a
        right-censored latency, a lower bound of its true latency), so the
        percentiles are lower bounds whenever they fall among censored jobs,
        and never survivor-biased.  The completed-only percentiles are kept
        beside them, with the completed fraction."""
        lat = np.array(self.latencies)
        both = np.concatenate([lat, np.array(self.censored_ages)])
        pct = (lambda a, q: float(np.percentile(a, q)) if a.size else float("nan"))
        n_all = max(1, self.submitted)
        return {"submitted": self.submitted, "completed": self.completed, "failed": self.failed,
                "censored": len(self.censored_ages), "completed_fraction": self.completed / n_all,
                "p50_s": pct(both, 50), "p99_s": pct(both, 99),
                "p50_completed_s": pct(lat, 50), "p99_completed_s": pct(lat, 99),
                "updates_per_s": self.updates / max(self.window, 1e-9),
                "jobs_completed_per_s": self.completed / max(self.window, 1e-9),
                "window_s": self.window, "wall_s": self.wall, "server": self.stats}


class InputPool:
    """Pre-generated inputs sliced per job (generation stays out of the loop)."""

    def __init__(self, max_chains, K, seed):
        self.nobs, self.xbar, self.sc = inputs.normal_gamma_data(max_chains, seed=seed)
        n_docs = min(max_chains, 65536)
        self.alpha, _, _ = inputs.lda_alpha(n_docs, K=K, seed=seed)
        self.K = K


def updates_of(model, n_chains, n_sweeps):
    """Gibbs updates of a job: 2 per chain-sweep (triangle, normal-gamma), 1
    Dirichlet draw per document-sweep (LDA)."""
    return (1 if model == B.MODEL_LDA else 2) * n_chains * n_sweeps


def make_request(pool, model, n, sweeps, seed, borrow=True):
    """A brng_request_t over slices of the pool (which outlives the server, so
    its arrays are lent to the server rather than copied at submit)."""
    r = B.brng_request_t()
    r.model, r.n_chains, r.n_sweeps, r.K, r.seed, r.chain_offset = model, n, sweeps, pool.K, seed, 0
    r.a0, r.b0, r.mu0, r.prec0 = 2.0, 1.0, 0.0, 0.01
    r.flags = B.SERVE_BORROW_INPUTS if borrow else 0
    if model == B.MODEL_NORMAL_GAMMA:
        r.nobs = pool.nobs.ctypes.data
        r.xbar = pool.xbar.ctypes.data
        r.sc = pool.sc.ctypes.data
    elif model == B.MODEL_LDA:
        r.alpha = pool.alpha.ctypes.data
    return r


def run_mix(spec: MixSpec, mem_budget=40_000_000_000, max_inflight=4, pool=None, max_jobs=None):
    """Drive the server with Poisson arrivals for spec.duration seconds.
    Results are collected (and their memory released) as jobs finish; when
    the window closes, every job not yet finished is recorded with its age
    (censored), and the server is closed (admitted jobs finish, queued ones
    are cancelled; neither enters the completed counts).  Throughput is the
    updates of jobs completed within the window over the window."""
    rng = np.random.default_rng(spec.seed)
    pool = pool or InputPool(spec.chains[1], spec.K, spec.seed)
    srv = B.brng_serve_open(mem_budget, max_inflight)
    res = MixResult()
    pending = {}
    lock = threading.Lock()
    stop = threading.Event()

    def collect():
        while not stop.is_set():
            with lock:
                ids = list(pending.items())
            progressed = False
            for jid, (model, n, sw, _) in ids:
                if stop.is_set():
                    break
                code, done = B.brng_serve_poll(srv, jid)
                if not done:
                    continue
                code, info = B.brng_serve_result(srv, jid)
                with lock:
                    if stop.is_set() or pending.pop(jid, None) is None:
                        continue  # the window closed first: counted as censored
                    progressed = True
                    if code == B.BRNG_OK:
                        res.completed += 1
                        res.updates += updates_of(model, n, sw)
                        res.latencies.append((info["completed_ns"] - info["submitted_ns"]) / 1e9)
                    elif code == B.BRNG_EAGAIN:
                        res.cancelled += 1
                    else:
                        res.failed += 1
            if not progressed:
                time.sleep(0.0005)

    th = threading.Thread(target=collect, daemon=True)
    th.start()
    t0 = time.perf_counter()
    t_next = t0
    n_total = 0
    while True:
        t_next += rng.exponential(1.0 / spec.rate)
        if t_next - t0 > spec.duration or (max_jobs is not None and n_total >= max_jobs):
            break
        while time.perf_counter() < t_next:
            pass
        model = int(rng.choice(spec.models))
        n = int(np.exp(rng.uniform(np.log(spec.chains[0]), np.log(spec.chains[1] + 1))))
        n = max(spec.chains[0], min(n, spec.chains[1]))
        sw = int(rng.integers(spec.sweeps[0], spec.sweeps[1] + 1))
        req = make_request(pool, model, n, sw, seed=int(rng.integers(0, 2**63)))
        t_sub = time.perf_counter()
        jid = B.brng_serve_submit(srv, req)
        with lock:
            pending[jid] = (model, n, sw, t_sub)
        n_total += 1
    # the window ends at the last arrival slot (spec.duration, or the job cap)
    while time.perf_counter() - t0 < spec.duration and (max_jobs is None or n_total < max_jobs):
        time.sleep(0.001)
    t_end = time.perf_counter()
    with lock:
        stop.set()
        res.censored_ages = [t_end - t_sub for (_, _, _, t_sub) in pending.values()]
        pending.clear()
    th.join()
    res.submitted = n_total
    res.window = t_end - t0
    code, res.stats = B.brng_serve_stats(srv)
    B.brng_serve_close(srv)
    res.wall = time.perf_counter() - t0
    res.stats["arrival_window_s"] = res.window
    return res
