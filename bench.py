#!/usr/bin/env python3
"""Benchmark of the batched varying-parameter RNG hot path on GB300.

Workload (one step): the normal-gamma Gibbs sampler -- 65,536 chains, each
with n = 100 synthetic observations ~ N(1.5, 2^2), 2,000 sweeps of
tau | mu ~ Gamma(52, rate) (Marsaglia-Tsang from the Gaussian and uniform
rings) and mu | tau ~ Normal -- one library call, one kernel launch.  The
metric is Gibbs updates per second (2 updates per chain-sweep), whole job over
all ranks; every rank runs its own 65,536 chains (global chain ids offset by
rank: weak scaling, no collective on the data path).

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl gb300|reference]

--impl reference times the FP64 CPU oracle on this host's cores on a bounded
sample of the same workload (the oracle is the reference of this project; the
paper's own code is not available).  Prints one JSON line (rank 0).
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_CHAINS = 65536
N_SWEEPS = 2000
N_OBS = 100
SEED = 42
PRIOR = (2.0, 1.0, 0.0, 0.01)
UPDATES_PER_STEP = 2 * N_CHAINS * N_SWEEPS
WORKLOAD = ("normal-gamma Gibbs: 65,536 chains x 2,000 sweeps, n=100 obs/chain ~N(1.5,2^2), "
            "tau|mu ~ Gamma(52, 1+SS/2) (Marsaglia-Tsang) then mu|tau ~ Normal, Philox4x32-10 seed 42")
METRIC = "Gibbs updates/s (normal-gamma, varying-parameter Gamma+Normal draws)"
UNIT = "updates/s"
L2_FLUSH_BYTES = 512 << 20  # > 129 MB L2
PHILOX_MULS_PER_BLOCK = 20
# DRAM traffic of one headline launch, as an ncu capture recorded it, keyed by
# a hash of the kernel sources it was taken on; reported only while the
# sources still hash the same (a changed kernel reports null traffic)
TRAFFIC_RECORD = os.path.join(ROOT, "profiles", "normal_gamma_kernel_traffic.txt")


def kernel_sources_hash():
    """sha256 (16 hex digits) over the CUDA sources and the public header."""
    import hashlib
    csrc = os.path.join(ROOT, "paper_1412_4825_gb300", "csrc")
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        if name.endswith((".cu", ".cuh", ".h")):
            h.update(name.encode())
            h.update(open(os.path.join(csrc, name), "rb").read())
    h.update(open(os.path.join(ROOT, "include", "brng.h"), "rb").read())
    return h.hexdigest()[:16]


def recorded_traffic():
    """(dram bytes per launch, note) from the capture record, or (None, why)."""
    try:
        rec = dict(line.strip().split("=", 1) for line in open(TRAFFIC_RECORD)
                   if "=" in line and not line.startswith("#"))
    except OSError:
        return None, "no capture record"
    if rec.get("sources_sha16") != kernel_sources_hash():
        return None, "kernel sources changed since the capture"
    return int(rec["dram_bytes_per_launch"]), "ncu dram__bytes_read.sum + dram__bytes_write.sum, " + \
        rec.get("captured", "?")


def _clock_sampler(uuid):
    q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")
    cmd = ["nvidia-smi", "--query-gpu=" + q, "--format=csv,noheader,nounits", "-lms", "50"]
    if uuid:
        cmd += ["-i", uuid]
    try:
        return subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
    except OSError:
        return None


def _clock_summary(proc):
    if proc is None:
        return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
    proc.terminate()
    try:
        out, _ = proc.communicate(timeout=5)
    except subprocess.TimeoutExpired:
        proc.kill()
        out, _ = proc.communicate()
    sm, smax, reasons, power = [], [], set(), []
    names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
    for line in out.strip().splitlines():
        f = [x.strip() for x in line.split(",")]
        if len(f) < 9:
            continue
        try:
            sm.append(float(f[1]))
            smax.append(float(f[2]))
            power.append(float(f[3]))
        except ValueError:
            continue
        for name, v in zip(names, f[5:9]):
            if v.lower() == "active":
                reasons.add(name)
    return {"sm_mhz": statistics.median(sm) if sm else None,
            "sm_max_mhz": max(smax) if smax else None,
            "power_w_max": max(power) if power else None,
            "samples": len(sm), "reasons": sorted(reasons)}


def _dist():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def _oracle_sample(n_chains, n_sweeps, nthreads, seed=SEED):
    """The oracle on `n_chains` chains (a bounded sample of the workload)."""
    import oracle as O
    from paper_1412_4825_gb300 import inputs
    nobs, xbar, sc = inputs.normal_gamma_data(n_chains, n_obs=N_OBS, seed=seed)
    O.lib()
    t0 = time.perf_counter()
    O.gibbs_normal_gamma(seed, n_sweeps, nobs, xbar, sc, prior=PRIOR, nthreads=nthreads)
    return time.perf_counter() - t0


def cpu_baseline(n_chains=8192, n_sweeps=N_SWEEPS):
    cores = os.cpu_count() or 1
    dt = _oracle_sample(n_chains, n_sweeps, cores)
    # the same oracle on one core, on an eighth of the sample
    n1 = max(1, n_chains // 8)
    dt1 = _oracle_sample(n1, n_sweeps, 1)
    return {"value": 2.0 * n_chains * n_sweeps / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": "%d of the 65,536 chains x %d sweeps (FP64 C oracle, %d threads, %.1f s)"
                      % (n_chains, n_sweeps, cores, dt),
            "single_core_value": 2.0 * n1 * n_sweeps / dt1,
            "single_core_sample": "%d chains x %d sweeps, 1 thread, %.1f s" % (n1, n_sweeps, dt1)}


def run_reference(args):
    rank, world, _ = _dist()
    if rank != 0:
        return 0
    cores = os.cpu_count() or 1
    n_chains = 2048
    for _ in range(args.warmup):
        _oracle_sample(256, 200, cores)
    times = [_oracle_sample(n_chains, N_SWEEPS, cores) for _ in range(args.steps)]
    upd = 2.0 * n_chains * N_SWEEPS
    value = upd * len(times) / sum(times)
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * sum(times) / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "sample_chains_per_step": n_chains},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": "%d chains x %d sweeps per step, %d threads" % (n_chains, N_SWEEPS, cores)},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def _time_s(fn, stream, reps=3, warm=1):
    """Median seconds of `fn` (which enqueues on `stream`), CUDA events."""
    import torch
    for _ in range(warm):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a, b in ev:
        a.record(stream)
        fn()
        b.record(stream)
    torch.cuda.synchronize()
    return statistics.median(a.elapsed_time(b) for a, b in ev) / 1e3


def extras(dev, stream, peaks, args):
    """Secondary workloads of the method (not the headline): the triangle
    Gibbs sampler of Eq. 1 (1,024 chains x 10,000 sweeps, FP64), the LDA
    document-topic step (16,384 documents x K=64 x 500 sweeps), the mixed
    varying-parameter stream (2^28 draws over 2^20 streams, with its HBM
    roofline), one uneven ensemble run batched vs one kernel per job, and the
    served Poisson mix (2,000 jobs/s and a sub-capacity rate)."""
    import numpy as np
    import torch

    from paper_1412_4825_gb300 import brng as B
    from paper_1412_4825_gb300 import inputs, serve

    out = {}
    from paper_1412_4825_gb300 import autotune as AT
    # integer-pipe roofline of a workload: the Philox blocks one call consumed
    # (from the stream positions before and after it) per second, against the
    # measured Philox probe, as the headline's
    peak_blocks = philox_probe(B, dev, stream)

    def philox_roofline(run, positions, per_block, seconds):
        before = positions()
        with torch.cuda.stream(stream):
            run()
        torch.cuda.synchronize(dev)
        blocks = float((positions() - before).astype(np.float64).sum()) / per_block
        return {"philox_blocks_per_call": blocks, "philox_blocks_per_s": blocks / seconds,
                "philox_frac": blocks / seconds / peak_blocks}

    # -- triangle (Eq. 1, Fig. 1): FP64, 1,024 chains; tuning chosen by the autotuner
    h = B.Handle(SEED, 1)
    st = B.triangle_state(1024, device=dev)
    mom = torch.zeros((1024, 5), dtype=torch.float64, device=dev)
    run_tri = lambda: B.brng_gibbs_run(h.h, B.MODEL_TRIANGLE, 0, 1024, 10000, None, st, mom, stream)  # noqa: E731
    tune, _, table = AT.autotune(h, run_tri, AT.SPACES["triangle"], stream, "triangle-1024x10000")
    t = _time_s(run_tri, stream)
    out["triangle_1024x10000"] = {"updates_per_s": 2 * 1024 * 10000 / t, "ms": t * 1e3, "tuning": tune,
                                  "autotune_ms": table}
    out["triangle_1024x10000"].update(philox_roofline(
        run_tri, lambda: st.view(torch.int64)[:, 2].cpu().numpy().astype(np.uint64), 2.0, t))
    h.close()
    # -- LDA document-topic Dirichlet step
    alpha, _, _ = inputs.lda_alpha(16384, K=64, seed=SEED)
    a = torch.from_numpy(alpha).to(dev)
    theta = torch.zeros((16384, 64), dtype=torch.float32, device=dev)
    pos = torch.zeros((16384, 64, 2), dtype=torch.int64, device=dev)
    mom = torch.zeros((16384, 64), dtype=torch.float64, device=dev)
    h = B.Handle(SEED, 1)
    lp = B.brng_lda_params_t(64, a.data_ptr())
    ls = B.brng_lda_state_t(theta.data_ptr(), pos.data_ptr())
    run_lda = lambda: B.brng_gibbs_run(h.h, B.MODEL_LDA, 0, 16384, 500, lp, ls, mom, stream)  # noqa: E731
    tune, _, table = AT.autotune(h, run_lda, AT.SPACES["lda"], stream, "lda-16384x64x500", reps=2)
    t = _time_s(run_lda, stream)
    out["lda_16384x64x500"] = {"dirichlet_updates_per_s": 16384 * 500 / t,
                               "gamma_deviates_per_s": 16384 * 64 * 500 / t, "ms": t * 1e3,
                               "tuning": tune, "autotune_ms": table}
    out["lda_16384x64x500"].update(philox_roofline(run_lda, lambda: pos.cpu().numpy().astype(np.uint64), 4.0, t))
    h.close()
    del a, theta, pos, mom
    # -- full LDA step: topic draw per token (collapsed conditional), count
    # exchange, theta ~ Dir(alpha + n_d); the same corpus size, 20 sweeps
    out["lda_full_16384x64"] = lda_full_extra(B, inputs, dev, stream, sweeps=20)
    # -- mixed varying-parameter stream, 17 B per draw through HBM
    n, S = 1 << 28, 1 << 20
    tag, p0, p1 = inputs.mixed_stream_torch(n, seed=SEED, device=dev)
    o = torch.empty(n, dtype=torch.float32, device=dev)
    w = torch.empty(n, dtype=torch.int32, device=dev)
    hm = B.Handle(SEED, S)
    run_mixed = lambda: B.brng_mixed(hm.h, tag, p0, p1, o, w, stream)  # noqa: E731
    tune, _, table = AT.autotune(hm, run_mixed, AT.SPACES["mixed"], stream, "mixed-2^28-2^20", reps=2)
    t = _time_s(run_mixed, stream)
    gbs = 17.0 * n / t / 1e9
    out["mixed_2^28"] = {"deviates_per_s": n / t, "ms": t * 1e3, "tuning": tune, "autotune_ms": table,
                         "hbm_achieved_gbs": gbs, "hbm_peak_gbs": peaks.get("hbm_gbs"),
                         "hbm_frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None}
    out["mixed_2^28"].update(philox_roofline(run_mixed, hm.positions, 4.0, t))
    # -- buffer length (the paper's vectorisation-vs-waste trade-off, Sec. 2.4):
    # the mixed stream and the normal-gamma sampler at every ring length whose
    # rings fit in shared memory (values never depend on it)
    sweep = {}
    for bl in (4, 8, 16, 32, 64, 128, 256, 512):
        try:
            hm.tune(buf_len=bl, warps_per_block=2)
            tb = _time_s(run_mixed, stream, reps=2)
            sweep[str(bl)] = {"ms": tb * 1e3, "hbm_frac": 17.0 * n / tb / 1e9 / peaks["hbm_gbs"]
                              if peaks.get("hbm_gbs") else None}
        except B.BrngError:
            sweep[str(bl)] = "rings do not fit in shared memory"
    out["buffer_length_sweep_mixed_2^28"] = sweep
    hm.close()
    ng = [torch.from_numpy(x).to(dev) for x in inputs.normal_gamma_data(65536, seed=SEED)]
    ngp = B.brng_normal_gamma_params_t(2.0, 1.0, 0.0, 0.01, *[x.data_ptr() for x in ng])
    ngs = B.normal_gamma_state(65536, device=dev)
    ngm = torch.zeros((65536, 4), dtype=torch.float64, device=dev)
    hn = B.Handle(SEED, 1)
    run_ng = lambda: B.brng_gibbs_run(hn.h, B.MODEL_NORMAL_GAMMA, 0, 65536, 2000, ngp, ngs, ngm, stream)  # noqa: E731
    sweep = {}
    for bl in (4, 8, 16, 32, 64, 128, 256):
        try:
            hn.tune(buf_len=bl, warps_per_block=8)
            sweep[str(bl)] = {"ms": _time_s(run_ng, stream, reps=2) * 1e3}
        except B.BrngError:
            sweep[str(bl)] = "rings do not fit in shared memory"
    out["buffer_length_sweep_normal_gamma_65536x2000"] = sweep
    hn.close()
    del ng, ngs, ngm
    del tag, p0, p1, o, w
    torch.cuda.empty_cache()
    # -- the paper's per-distribution table (Sec. 2.4) in GPU form: each of its six
    # distributions over 2^26 draws (2^20 streams) with per-draw (varying)
    # parameters -- the BatchRNG column -- and with one constant parameter set
    # -- the batch column; SM-cycles per sample (time x SM clock x SMs / draws)
    # beside the paper's cycles per sample; and one draw per call through the
    # C ABI, the one-at-a-time column
    n, S = 1 << 26, 1 << 20
    gd = torch.Generator(device=dev)
    gd.manual_seed(SEED + 7)

    def logu(lo, hi):
        return torch.exp(np.log(lo) + (np.log(hi) - np.log(lo)) * torch.rand(n, generator=gd, device=dev))

    ones = torch.ones(n, device=dev)
    zeros = torch.zeros(n, device=dev)
    a_u = logu(1e-3, 1e3)
    b_u = a_u + logu(1e-3, 1e3)
    mu = logu(1e-3, 1e3) * torch.where(torch.rand(n, generator=gd, device=dev) < 0.5, -1.0, 1.0)
    sig, lam, alpha, kw = logu(1e-2, 1e2), logu(1e-2, 1e2), logu(0.05, 50.0), logu(0.5, 5.0)
    dists = {"uniform": (B.brng_uniform, [a_u, b_u], [zeros, ones]),
             "normal": (B.brng_normal, [mu, sig], [zeros, ones]),
             "exponential": (B.brng_exponential, [lam], [ones]),
             "gamma": (B.brng_gamma, [alpha], [ones * 2.0]),
             "laplace": (B.brng_laplace, [mu, sig], [zeros, ones]),
             "weibull": (B.brng_weibull, [kw, lam], [ones * 1.5, ones])}
    o = torch.empty(n, device=dev)
    hd = B.Handle(SEED, S)
    hd.tune(buf_len=8, warps_per_block=2)
    sm_cycles_per_s = float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 * torch.cuda.get_device_properties(dev).multi_processor_count
    table = {}
    for name, (fn, pv, pf) in dists.items():
        tv = _time_s(lambda: fn(hd.h, *pv, o, None, stream), stream)
        tf = _time_s(lambda: fn(hd.h, *pf, o, None, stream), stream)
        nbytes = 4.0 * (len(pv) + 1) * n  # parameters read, value written
        table[name] = {"varying_deviates_per_s": n / tv, "fixed_deviates_per_s": n / tf,
                       "varying_sm_cycles_per_sample": tv * sm_cycles_per_s / n,
                       "fixed_sm_cycles_per_sample": tf * sm_cycles_per_s / n,
                       "varying_hbm_frac": nbytes / tv / 1e9 / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None}
    h1 = B.Handle(SEED, 1)
    a1, o1 = alpha[:1].clone(), torch.empty(1, device=dev)
    calls = 2000
    t1 = _time_s(lambda: [B.brng_gamma(h1.h, a1, o1, None, stream) for _ in range(calls)], stream, reps=2)
    table["gamma_one_draw_per_call"] = {"deviates_per_s": calls / t1, "us_per_draw": t1 / calls * 1e6}
    out["per_distribution_2^26"] = table
    hd.close()
    h1.close()
    del ones, zeros, a_u, b_u, mu, sig, lam, alpha, kw, o, dists
    torch.cuda.empty_cache()
    # -- Poisson draws (discrete, by inversion of one U), lambda log-uniform in [0.05, 64]
    n, S = 1 << 26, 1 << 20
    g = torch.Generator(device=dev)
    g.manual_seed(SEED)
    lam = torch.exp(np.log(0.05) + (np.log(64.0) - np.log(0.05)) *
                    torch.rand(n, generator=g, device=dev, dtype=torch.float32))
    o = torch.empty(n, dtype=torch.float32, device=dev)
    w = torch.empty(n, dtype=torch.int32, device=dev)
    hp = B.Handle(SEED, S)
    run_p = lambda: B.brng_poisson(hp.h, lam, o, w, stream)  # noqa: E731
    tune, _, table = AT.autotune(hp, run_p, AT.SPACES["mixed"], stream, "poisson-2^26-2^20", reps=2)
    t = _time_s(run_p, stream)

    def rechecks_per_call(fn, h):  # FP64 redraws of one call (the counters accumulate)
        before = h.counters()[1]["n_recheck"]
        fn()
        torch.cuda.synchronize()
        return h.counters()[1]["n_recheck"] - before

    out["poisson_2^26"] = {"deviates_per_s": n / t, "ms": t * 1e3, "lambda": "log-uniform [0.05, 64]",
                           "tuning": tune, "fp64_redraws_per_call": rechecks_per_call(run_p, hp)}
    # -- Binomial draws: trials log-uniform integers in [1, 1000], p uniform, mean <= 64
    tr = torch.floor(torch.exp(np.log(1001.0) * torch.rand(n, generator=g, device=dev)))
    pr = torch.rand(n, generator=g, device=dev)
    q = torch.minimum(pr, 1.0 - pr)
    cap = 0.999 * 64.0 / torch.clamp(tr, min=1.0)
    pr = torch.where(tr * q > 64.0, torch.where(pr <= 0.5, cap, 1.0 - cap), pr).contiguous()
    del q, cap
    run_b = lambda: B.brng_binomial(hp.h, tr, pr, o, w, stream)  # noqa: E731
    t = _time_s(run_b, stream)
    out["binomial_2^26"] = {"deviates_per_s": n / t, "ms": t * 1e3,
                            "params": "n log-uniform integers [1, 1000], p uniform, n min(p, 1-p) <= 64",
                            "tuning": hp.tuning, "fp64_redraws_per_call": rechecks_per_call(run_b, hp)}
    # -- large means: Poisson by PTRS (lambda log-uniform [64, 1e6]) and
    # Binomial by BTRD (n log-uniform integers up to 2^24, p uniform); each
    # attempt decided in FP32 / float-float, undecided attempts in FP64
    lam = torch.exp(np.log(64.0) + np.log(1e6 / 64.0) * torch.rand(n, generator=g, device=dev)).contiguous()
    t = _time_s(run_p, stream)
    out["poisson_large_2^26"] = {"deviates_per_s": n / t, "ms": t * 1e3, "lambda": "log-uniform [64, 1e6]",
                                 "method": "PTRS, certified FP32 attempts",
                                 "fp64_attempts_per_call": rechecks_per_call(run_p, hp)}
    # both methods in one call: lambda log-uniform [0.05, 1e6] (inversion below
    # mean 64, PTRS above, in the same warps)
    lam = torch.exp(np.log(0.05) + np.log(1e6 / 0.05) * torch.rand(n, generator=g, device=dev)).contiguous()
    t = _time_s(run_p, stream)
    out["poisson_wide_2^26"] = {"deviates_per_s": n / t, "ms": t * 1e3, "lambda": "log-uniform [0.05, 1e6]",
                                "method": "inversion below mean 64, PTRS above",
                                "fp64_redraws_per_call": rechecks_per_call(run_p, hp)}
    tr = torch.floor(torch.exp(np.log(2.0 ** 24) * torch.rand(n, generator=g, device=dev))).contiguous()
    pr = torch.rand(n, generator=g, device=dev).contiguous()
    t = _time_s(run_b, stream)
    out["binomial_large_2^26"] = {"deviates_per_s": n / t, "ms": t * 1e3,
                                  "params": "n log-uniform integers [1, 2^24], p uniform (BTRD above mean 64)",
                                  "method": "BTRD, certified FP32 attempts",
                                  "fp64_attempts_per_call": rechecks_per_call(run_b, hp)}
    hp.close()
    del lam, o, w, tr, pr
    torch.cuda.empty_cache()
    # -- FP64 uniform from the U64 domain: 2^27 draws over 2^20 streams, an
    # HBM-bound stream (a, b read, value and word written: 28 B/draw)
    n64 = 1 << 27
    h64 = B.Handle(SEED, 1 << 20)
    a64 = torch.rand(n64, generator=g, device=dev, dtype=torch.float64)
    b64 = a64 + torch.rand(n64, generator=g, device=dev, dtype=torch.float64)
    o64 = torch.empty(n64, dtype=torch.float64, device=dev)
    w64 = torch.empty(n64, dtype=torch.int32, device=dev)
    t = _time_s(lambda: B.brng_uniform_f64(h64.h, a64, b64, o64, w64, stream), stream)
    gbs = 28.0 * n64 / t / 1e9
    out["uniform_f64_2^27"] = {"deviates_per_s": n64 / t, "ms": t * 1e3, "hbm_achieved_gbs": gbs,
                               "hbm_peak_gbs": peaks.get("hbm_gbs"),
                               "hbm_frac": gbs / peaks["hbm_gbs"] if peaks.get("hbm_gbs") else None,
                               "bytes_per_draw": 28}
    h64.close()
    del a64, b64, o64, w64
    torch.cuda.empty_cache()
    # -- uneven ensembles: batched (one persistent launch) vs one kernel per job
    pool = serve.InputPool(65536, 64, SEED)
    d_nobs, d_xbar, d_sc = (torch.from_numpy(x).to(dev) for x in (pool.nobs, pool.xbar, pool.sc))
    d_alpha = torch.from_numpy(pool.alpha).to(dev)

    def ensemble(n_jobs, max_chains, sweeps, seed):
        rng = np.random.default_rng(seed)
        specs = []
        for i in range(n_jobs):
            model = int(rng.integers(0, 3))
            nch = int(min(max_chains, max(1, np.exp(rng.uniform(0, np.log(max_chains + 1))))))
            specs.append((model, nch, int(rng.integers(sweeps[0], sweeps[1] + 1)), seed + 1 + i))
        keep = []

        positions = []  # per job of the last fresh_jobs(): (its stream positions, elements per block)

        def fresh_jobs():
            jobs = []
            positions.clear()
            for model, nch, sw, sd in specs:
                if model == B.MODEL_TRIANGLE:
                    st = B.triangle_state(nch, device=dev)
                    mm, prm, sarg = torch.zeros((nch, 5), dtype=torch.float64, device=dev), None, st
                    positions.append((st.view(torch.int64)[:, 2], 2.0))
                elif model == B.MODEL_NORMAL_GAMMA:
                    st = B.normal_gamma_state(nch, device=dev)
                    mm = torch.zeros((nch, 4), dtype=torch.float64, device=dev)
                    prm = B.brng_normal_gamma_params_t(2.0, 1.0, 0.0, 0.01, d_nobs.data_ptr(), d_xbar.data_ptr(),
                                                       d_sc.data_ptr())
                    sarg = st
                    positions.append((st[:, 1:3], 4.0))
                else:
                    th = torch.zeros((nch, 64), dtype=torch.float32, device=dev)
                    ps = torch.zeros((nch, 64, 2), dtype=torch.int64, device=dev)
                    mm = torch.zeros((nch, 64), dtype=torch.float64, device=dev)
                    prm = B.brng_lda_params_t(64, d_alpha.data_ptr())
                    sarg = B.brng_lda_state_t(th.data_ptr(), ps.data_ptr())
                    keep.append((th, ps))
                    positions.append((ps, 4.0))
                keep.append((sarg, mm, prm))
                jobs.append((model, nch, sw, sd, prm, sarg, mm))
            return jobs

        def consumed_blocks():
            return sum(float(p.cpu().numpy().astype(np.float64).sum()) / k for p, k in positions)

        upd = sum((1 if m == B.MODEL_LDA else 2) * c * sw for m, c, sw, _ in specs)
        hb = B.Handle(SEED, 1)
        handles = {sd: B.Handle(sd, 1) for _, _, _, sd in specs}
        jobs = fresh_jobs()

        def plain():
            for model, nch, sw, sd, prm, sarg, mm in jobs:
                B.brng_gibbs_run(handles[sd].h, model, 0, nch, sw, prm, sarg, mm, stream)

        t_plain = _time_s(plain, stream, reps=2, warm=1)
        # a measured bound on what batching can gain: each job timed alone
        # (one launch), each model's best time per unit-sweep (a unit = 32
        # chains or one document: the work of one warp) taken from its jobs
        # that fill the GPU best, and the mix's ideal time = its unit-sweeps at
        # those costs; plain time / ideal time bounds batched / plain
        ev = []
        with torch.cuda.stream(stream):
            for model, nch, sw, sd, prm, sarg, mm in jobs:
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                B.brng_gibbs_run(handles[sd].h, model, 0, nch, sw, prm, sarg, mm, stream)
                e1.record(stream)
                ev.append((e0, e1))
        torch.cuda.synchronize(dev)
        unit_sweeps = [((nch + 31) // 32 if m != B.MODEL_LDA else nch) * sw for m, nch, sw, _ in specs]
        t_job = [a.elapsed_time(b) / 1e3 for a, b in ev]
        best = {}
        for (m, _, _, _), us, tj in zip(specs, unit_sweeps, t_job):
            best[m] = min(best.get(m, float("inf")), tj / us)
        t_ideal = sum(best[m] * us for (m, _, _, _), us in zip(specs, unit_sweeps))
        t_alone = sum(t_job)
        jobs = fresh_jobs()
        bjobs = [B.make_job(m, c, sw, sd, prm, sarg, mm)[0] for m, c, sw, sd, prm, sarg, mm in jobs]
        t_batch = _time_s(lambda: B.brng_gibbs_batch(hb.h, bjobs, stream), stream, reps=2, warm=1)
        # the persistent kernel's integer-pipe roofline: the Philox blocks one
        # batched call consumed (every job's stream positions before and after)
        b0 = consumed_blocks()
        with torch.cuda.stream(stream):
            B.brng_gibbs_batch(hb.h, bjobs, stream)
        torch.cuda.synchronize(dev)
        batch_blocks = consumed_blocks() - b0
        # the same batch planned once and captured in a CUDA graph; each replay
        # continues every job's chains by its sweeps
        jobs = fresh_jobs()
        plan = B.brng_batch_create(hb.h, [B.make_job(m, c, sw, sd, prm, sarg, mm)[0]
                                          for m, c, sw, sd, prm, sarg, mm in jobs])
        graph = torch.cuda.CUDAGraph()
        torch.cuda.synchronize()
        with torch.cuda.graph(graph, stream=stream):
            B.brng_batch_launch(plan, stream)

        def replay():
            with torch.cuda.stream(stream):
                graph.replay()

        t_graph = _time_s(replay, stream, reps=2, warm=1)
        del graph
        B.brng_batch_destroy(plan)
        for hh in handles.values():
            hh.close()
        hb.close()
        keep.clear()
        torch.cuda.synchronize()
        return {"jobs": len(specs), "chains": "log-uniform [1, %d]" % max_chains,
                "sweeps": "uniform [%d, %d]" % sweeps, "updates": upd,
                "plain_updates_per_s": upd / t_plain, "batched_updates_per_s": upd / t_batch,
                "batched_over_plain": t_plain / t_batch, "plain_ms": t_plain * 1e3, "batched_ms": t_batch * 1e3,
                "bound_batched_over_plain": t_alone / t_ideal, "ideal_ms": t_ideal * 1e3,
                "jobs_alone_ms": t_alone * 1e3,
                "share_of_plain_in_largest_3_jobs": sum(sorted(t_job)[-3:]) / t_alone,
                "graph_updates_per_s": upd / t_graph, "graph_over_plain": t_plain / t_graph,
                "graph_ms": t_graph * 1e3, "batch_philox_blocks_per_s": batch_blocks / t_batch,
                "batch_philox_frac": batch_blocks / t_batch / peak_blocks}

    out["ensemble_48_jobs"] = ensemble(48, 65536, (100, 10000), SEED)
    out["ensemble_256_small_jobs"] = ensemble(256, 2048, (100, 1000), SEED + 1000)
    torch.cuda.empty_cache()
    # -- served Poisson mix under a 40e9-byte budget: 2,000 jobs/s for the
    # configured 60 s (far over capacity), then 0.8 x the job rate it sustained
    # (near capacity), then 10 jobs/s (idle); latency percentiles over every
    # submitted job, unfinished ones at their age when the window closes
    full = serve.run_mix(serve.MixSpec(rate=2000.0, duration=args.serve_seconds, seed=SEED), pool=pool)
    fs = full.summary()
    out["served_2000_per_s"] = fs
    near_rate = max(1.0, 0.8 * fs["jobs_completed_per_s"])
    near = serve.run_mix(serve.MixSpec(rate=near_rate, duration=args.serve_near_seconds, seed=SEED + 2), pool=pool)
    out["served_near_capacity"] = dict(near.summary(), rate_jobs_per_s=near_rate)
    sub = serve.run_mix(serve.MixSpec(rate=10.0, duration=10.0, seed=SEED + 1), pool=pool)
    out["served_10_per_s"] = sub.summary()
    return out


# The full LDA step's theta draw runs one sweep per launch, so short rings
# and no lookahead waste least (measured on GB300, 20 sweeps of the 16,384-
# document corpus: 19.1 ms with the handle's defaults, 17.5 ms with these).
LDA_FULL_TUNING = dict(buf_len=8, lookahead=1, warps_per_block=2)


def lda_full_extra(B, inputs, dev, stream, sweeps=20, n_docs=16384):
    """The full LDA step on the synthetic corpus (K = 64, V = 4,096, lengths
    U{50..500}): token topic updates per second over `sweeps` sweeps in one
    call (3 launches per sweep), and the z kernel's share."""
    import torch
    corpus = inputs.lda_corpus(n_docs, K=64, V=4096, seed=SEED)
    st = inputs.lda_initial_state(corpus, seed=7)
    m = B.LdaFull(corpus, st, alpha=0.1, beta=0.01, stream=stream)
    h = B.Handle(SEED, 1)
    h.tune(**LDA_FULL_TUNING)
    n_tok = int(corpus["doc_ptr"][-1])
    run = lambda: m.run(h, sweeps, stream=stream)  # noqa: E731
    t = _time_s(run, stream, reps=2, warm=1)
    # the topic draws alone, one sweep, with the changes left unapplied
    lp = m.params(exchange=1)
    ls = m.state()
    zrun = lambda: B.brng_gibbs_run(h.h, B.MODEL_LDA_FULL, 0, n_docs, 1, lp, ls, m.mom, stream)  # noqa: E731
    t1 = _time_s(zrun, stream, reps=3, warm=1)
    B.brng_lda_apply(m.K, m.V, m.nkw, m.nk, m.dnkw, stream)
    torch.cuda.synchronize()
    h.close()
    return {"token_updates_per_s": n_tok * sweeps / t, "dirichlet_updates_per_s": n_docs * sweeps / t,
            "ms_per_sweep": t * 1e3 / sweeps, "tokens": n_tok, "sweeps": sweeps,
            "ms_one_sweep_without_apply": t1 * 1e3,
            "corpus": "%d docs, K=64, V=4096, lengths U{50..500}, LDA generative model" % n_docs}


def philox_probe(B, dev, stream):
    """Measured integer-pipe peak: Philox4x32-10 blocks per second of a
    register-only kernel (8 blocks of 256 threads per SM, 2,048 blocks per
    thread), timed with CUDA events on `stream` after a warm-up launch."""
    import torch
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    sink = torch.empty(sm_count * 8 * 256, dtype=torch.int32, device=dev)
    B.brng_philox_peak(64, sm_count * 8, 256, sink, stream)
    pe0, pe1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    pe0.record(stream)
    B.brng_philox_peak(2048, sm_count * 8, 256, sink, stream)
    pe1.record(stream)
    torch.cuda.synchronize(dev)
    return 4.0 * 2048 * sm_count * 8 * 256 / (pe0.elapsed_time(pe1) / 1e3)


def run_gpu(args):
    import numpy as np
    import torch

    rank, world, local = _dist()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=dev)
        pg = dist

    from paper_1412_4825_gb300 import build_lib
    build_lib.build()
    from paper_1412_4825_gb300 import brng as B
    from paper_1412_4825_gb300 import inputs, shard

    # weak scaling: rank r runs global chains [r*N, (r+1)*N) on its slice of
    # one global data set, so any rank count reproduces the one-GPU chains
    chain_offset, _ = shard.weak_range(N_CHAINS, rank)
    nobs, xbar, sc = (a[chain_offset:chain_offset + N_CHAINS] for a in
                      inputs.normal_gamma_data(chain_offset + N_CHAINS, n_obs=N_OBS, seed=SEED))
    stream = torch.cuda.Stream(device=dev)
    h = B.Handle(SEED, 1)
    fixed = bool(args.buf_len or args.warps_per_block)
    if fixed:
        h.tune(buf_len=args.buf_len, warps_per_block=args.warps_per_block)
    # one device buffer [nobs | xbar | sc | state | moments] (4+4+4+24+32 B per
    # chain): the end-to-end leg moves the inputs in one copy and the results
    # in one copy
    n4 = 4 * N_CHAINS
    dbuf = torch.empty(17 * n4, dtype=torch.uint8, device=dev)
    d_nobs, d_xbar, d_sc = (dbuf[i * n4:(i + 1) * n4].view(torch.float32) for i in range(3))
    state = dbuf[3 * n4:9 * n4].view(torch.int64).view(N_CHAINS, 3)
    mom = dbuf[9 * n4:17 * n4].view(torch.float64).view(N_CHAINS, 4)
    for d, a in ((d_nobs, nobs), (d_xbar, xbar), (d_sc, sc)):
        d.copy_(torch.from_numpy(np.ascontiguousarray(a)))
    state.copy_(B.normal_gamma_state(N_CHAINS, mu0=PRIOR[2], device="cpu"))
    mom.zero_()
    params = B.brng_normal_gamma_params_t(*PRIOR, d_nobs.data_ptr(), d_xbar.data_ptr(), d_sc.data_ptr())
    flush = torch.empty(L2_FLUSH_BYTES, dtype=torch.uint8, device=dev)

    def step():
        B.brng_gibbs_run(h.h, B.MODEL_NORMAL_GAMMA, chain_offset, N_CHAINS, N_SWEEPS, params, state, mom,
                         stream)

    def barrier():
        torch.cuda.synchronize(dev)
        if pg is not None:
            pg.barrier()
        torch.cuda.synchronize(dev)

    autotune_table = None
    if not fixed:  # launch knobs picked by measurement (results do not depend on them)
        from paper_1412_4825_gb300 import autotune as AT
        _, _, autotune_table = AT.autotune(h, step, AT.SPACES["normal_gamma"], stream,
                                           "normal-gamma-%dx%d" % (N_CHAINS, N_SWEEPS))
    with torch.cuda.stream(stream):
        for _ in range(args.warmup):
            step()
    barrier()
    # consumption of one step (exact count of Philox blocks the method used),
    # and the ring elements generated but unused when it ended (Sec. 2.4's
    # buffer waste, from the handle's counter)
    before = state.clone()
    h.counters(stream, reset=True)
    with torch.cuda.stream(stream):
        step()
    torch.cuda.synchronize(dev)
    _, waste_cnt = h.counters(stream, reset=True)
    _, _, pn0, pu0 = B.normal_gamma_unpack(before)
    _, _, pn1, pu1 = B.normal_gamma_unpack(state)
    consumed = float((pn1 - pn0).astype(np.float64).sum() + (pu1 - pu0).astype(np.float64).sum())
    blocks_per_step = consumed / 4.0
    buffer_waste = {"elements_per_step": int(waste_cnt["n_wasted"]),
                    "per_chain": waste_cnt["n_wasted"] / N_CHAINS,
                    "fraction_of_consumed": waste_cnt["n_wasted"] / consumed,
                    "ring_len": h.tuning["buf_len"]}

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(dev).uuid)
    except Exception:
        pass
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    sampler = _clock_sampler(uuid) if rank == 0 else None
    time.sleep(0.2 if sampler else 0)
    barrier()
    wall0 = time.perf_counter()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xFF)  # between timed steps: write > L2
            ev[k][0].record(stream)
            step()
            ev[k][1].record(stream)
    barrier()
    wall = time.perf_counter() - wall0
    clocks = _clock_summary(sampler) if rank == 0 else None
    ms = [a.elapsed_time(b) for a, b in ev]
    total_s = sum(ms) / 1e3
    if pg is not None:
        total_s = shard.max_over_ranks(pg, total_s, device=dev)
    value = world * UPDATES_PER_STEP * args.steps / total_s

    # end to end through the public API: host inputs -> device -> run -> host
    # results, every step: the inputs (data and start state) in one copy from
    # pinned memory, the results (state and moments) in one copy back
    h_in = torch.empty(9 * n4, dtype=torch.uint8).pin_memory()
    for i, a in enumerate((nobs, xbar, sc)):
        h_in[i * n4:(i + 1) * n4].view(torch.float32).copy_(torch.from_numpy(np.ascontiguousarray(a)))
    h_in[3 * n4:].view(torch.int64).view(N_CHAINS, 3).copy_(B.normal_gamma_state(N_CHAINS, mu0=PRIOR[2],
                                                                                  device="cpu"))
    h_out = torch.empty(14 * n4, dtype=torch.uint8).pin_memory()
    d_in, d_out = dbuf[:9 * n4], dbuf[3 * n4:]
    h2d = h_in.numel()
    d2h = h_out.numel()
    e_ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(args.steps)]
    barrier()
    with torch.cuda.stream(stream):
        for k in range(args.steps):
            flush.fill_(k & 0xFF)
            e_ev[k][0].record(stream)
            d_in.copy_(h_in, non_blocking=True)
            mom.zero_()
            step()
            h_out.copy_(d_out, non_blocking=True)
            e_ev[k][1].record(stream)
    barrier()
    e_s = sum(a.elapsed_time(b) for a, b in e_ev) / 1e3
    if pg is not None:
        e_s = shard.max_over_ranks(pg, e_s, device=dev)
    e2e_value = world * UPDATES_PER_STEP * args.steps / e_s

    # integer-pipe roofline: Philox blocks the step consumed / kernel time,
    # against 152 SMs x (64 32-bit multiply results per clock per SM / 2 per
    # 64-bit product / 20 products per block) x SM clock
    sm_count = torch.cuda.get_device_properties(dev).multi_processor_count
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except Exception:
        pass
    sm_max = float(peaks.get("sm_max_mhz", 2070.0))
    derived_blocks = sm_count * (64.0 / 2.0 / PHILOX_MULS_PER_BLOCK) * sm_max * 1e6
    kernel_s = total_s / args.steps  # one launch per step, events bracket it alone
    achieved = blocks_per_step / kernel_s
    probe_blocks_s = philox_probe(B, dev, stream)
    traffic, traffic_note = recorded_traffic()

    if rank != 0:
        if pg is not None:
            pg.barrier()
        return 0
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": 1e3 * total_s / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "chains_per_gpu": N_CHAINS, "sweeps": N_SWEEPS,
                   "updates_per_step_per_gpu": UPDATES_PER_STEP, "parallelism": "chains sharded by rank",
                   "l2": "flushed between timed steps (512 MB write)", "tuning": h.tuning,
                   "autotune_ms": autotune_table},
        "clocks": clocks,
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
        "gpu_launches": args.steps,
        "roofline": {"bound": "alu", "achieved": achieved / 1e9, "peak": probe_blocks_s / 1e9,
                     "unit": "GPhilox-block/s", "frac": achieved / probe_blocks_s, "traffic": traffic,
                     "traffic_source": traffic_note, "kernel": "normal_gamma_kernel",
                     "peak_source": "measured: register-only Philox4x32-10 probe on this GPU, same launch",
                     "derived_peak": derived_blocks / 1e9,
                     "note": "integer pipe: 20 32x32->64 multiplies per Philox4x32-10 block; blocks = "
                             "exact consumption of the step (N+U elements / 4)"},
        "wall_s_timed": wall,
        "buffer_waste": buffer_waste,
    }
    if world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline()
    if world == 1 and not args.no_extras:
        try:
            line["extra"] = extras(dev, stream, peaks, args)
        except Exception as exc:  # the headline line is printed regardless
            line["extra"] = {"error": repr(exc)}
    print(json.dumps(line), flush=True)
    if pg is not None:
        pg.barrier()
    return 0


def run_case(args):
    """One secondary workload at a chosen size, timed with CUDA events (for
    profiling commands): prints {"case", "ms": [...], ...}."""
    import numpy as np
    import torch

    from paper_1412_4825_gb300 import build_lib
    build_lib.build()
    from paper_1412_4825_gb300 import brng as B
    from paper_1412_4825_gb300 import inputs

    dev = torch.device("cuda", 0)
    stream = torch.cuda.Stream(device=dev)
    reps = max(1, args.steps)
    info = {"case": args.case}
    if args.case == "mixed":
        n, S = 1 << args.log2n, 1 << args.log2s
        tag, p0, p1 = inputs.mixed_stream_torch(n, seed=SEED, n_tags=args.tags, device=dev)
        o = torch.empty(n, dtype=torch.float32, device=dev)
        w = torch.empty(n, dtype=torch.int32, device=dev)
        h = B.Handle(SEED, S)
        h.tune(buf_len=args.buf_len or 8, warps_per_block=args.warps_per_block)
        fn = lambda: B.brng_mixed(h.h, tag, p0, p1, o, w, stream)  # noqa: E731
        info.update(draws=n, streams=S, bytes_per_launch=17 * n)
    elif args.case == "lda":
        alpha, _, _ = inputs.lda_alpha(args.docs, K=64, seed=SEED)
        a = torch.from_numpy(alpha).to(dev)
        theta = torch.zeros((args.docs, 64), dtype=torch.float32, device=dev)
        pos = torch.zeros((args.docs, 64, 2), dtype=torch.int64, device=dev)
        mom = torch.zeros((args.docs, 64), dtype=torch.float64, device=dev)
        h = B.Handle(SEED, 1)
        h.tune(buf_len=args.buf_len or 16, lookahead=4, warps_per_block=args.warps_per_block or 4)
        lp = B.brng_lda_params_t(64, a.data_ptr())
        ls = B.brng_lda_state_t(theta.data_ptr(), pos.data_ptr())
        fn = lambda: B.brng_gibbs_run(h.h, B.MODEL_LDA, 0, args.docs, args.sweeps, lp, ls, mom, stream)  # noqa: E731
        info.update(docs=args.docs, sweeps=args.sweeps, K=64)
    elif args.case == "ng":  # the headline model at a chosen size (profiling)
        nobs, xbar, sc = (torch.from_numpy(a).to(dev) for a in
                          inputs.normal_gamma_data(args.chains, n_obs=N_OBS, seed=SEED))
        st = B.normal_gamma_state(args.chains, device=dev)
        mom = torch.zeros((args.chains, 4), dtype=torch.float64, device=dev)
        h = B.Handle(SEED, 1)
        h.tune(buf_len=args.buf_len or 32, warps_per_block=args.warps_per_block or 8)
        prm = B.brng_normal_gamma_params_t(*PRIOR, nobs.data_ptr(), xbar.data_ptr(), sc.data_ptr())
        fn = lambda: B.brng_gibbs_run(h.h, B.MODEL_NORMAL_GAMMA, 0, args.chains, args.sweeps, prm, st, mom,  # noqa: E731
                                      stream)
        info.update(chains=args.chains, sweeps=args.sweeps)
    elif args.case == "lda_full":  # the full LDA step, one call of `sweeps` sweeps
        corpus = inputs.lda_corpus(args.docs, K=64, V=4096, seed=SEED)
        m = B.LdaFull(corpus, inputs.lda_initial_state(corpus, seed=7), stream=stream)
        h = B.Handle(SEED, 1)
        h.tune(**LDA_FULL_TUNING)
        fn = lambda: m.run(h, args.sweeps, stream=stream)  # noqa: E731
        info.update(docs=args.docs, sweeps=args.sweeps, tokens=int(corpus["doc_ptr"][-1]))
    elif args.case == "poisson_large":  # PTRS: lambda log-uniform [64, 1e6]
        n, S = 1 << args.log2n, 1 << args.log2s
        g = torch.Generator(device=dev)
        g.manual_seed(SEED)
        lam = torch.exp(np.log(64.0) + np.log(1e6 / 64.0) * torch.rand(n, generator=g, device=dev)).contiguous()
        o = torch.empty(n, dtype=torch.float32, device=dev)
        w = torch.empty(n, dtype=torch.int32, device=dev)
        h = B.Handle(SEED, S)
        h.tune(buf_len=args.buf_len or 8, warps_per_block=args.warps_per_block or 4)
        fn = lambda: B.brng_poisson(h.h, lam, o, w, stream)  # noqa: E731
        info.update(draws=n, streams=S)
    elif args.case == "binomial_large":  # BTRD: n log-uniform integers [1, 2^24], p uniform
        n, S = 1 << args.log2n, 1 << args.log2s
        g = torch.Generator(device=dev)
        g.manual_seed(SEED)
        tr = torch.floor(torch.exp(np.log(2.0 ** 24) * torch.rand(n, generator=g, device=dev))).contiguous()
        pr = torch.rand(n, generator=g, device=dev).contiguous()
        o = torch.empty(n, dtype=torch.float32, device=dev)
        w = torch.empty(n, dtype=torch.int32, device=dev)
        h = B.Handle(SEED, S)
        h.tune(buf_len=args.buf_len or 8, warps_per_block=args.warps_per_block or 4)
        fn = lambda: B.brng_binomial(h.h, tr, pr, o, w, stream)  # noqa: E731
        info.update(draws=n, streams=S)
    elif args.case == "triangle":
        h = B.Handle(SEED, 1)
        h.tune(buf_len=256, lanes_per_chain=16)
        st = B.triangle_state(1024, device=dev)
        mom = torch.zeros((1024, 5), dtype=torch.float64, device=dev)
        fn = lambda: B.brng_gibbs_run(h.h, B.MODEL_TRIANGLE, 0, 1024, args.sweeps, None, st, mom, stream)  # noqa: E731
        info.update(chains=1024, sweeps=args.sweeps)
    elif args.case == "uniform64":
        n, S = 1 << args.log2n, 1 << args.log2s
        g = torch.Generator(device=dev)
        g.manual_seed(SEED)
        a = torch.rand(n, generator=g, device=dev, dtype=torch.float64)
        b = a + torch.rand(n, generator=g, device=dev, dtype=torch.float64)
        o = torch.empty(n, dtype=torch.float64, device=dev)
        w = torch.empty(n, dtype=torch.int32, device=dev)
        h = B.Handle(SEED, S)
        fn = lambda: B.brng_uniform_f64(h.h, a, b, o, w, stream)  # noqa: E731
        info.update(draws=n, streams=S, bytes_per_launch=28 * n)
    else:
        raise SystemExit("unknown case %r" % args.case)
    for _ in range(args.warmup):
        fn()
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(reps)]
    for a0, a1 in ev:
        a0.record(stream)
        fn()
        a1.record(stream)
    torch.cuda.synchronize()
    info["ms"] = [round(a0.elapsed_time(a1), 4) for a0, a1 in ev]
    info["counters"] = h.counters()[1]
    print(json.dumps(info), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser(description=__doc__, formatter_class=argparse.RawDescriptionHelpFormatter)
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["gb300", "reference"], default="gb300")
    ap.add_argument("--buf-len", type=int, default=0)
    ap.add_argument("--warps-per-block", type=int, default=0,
                    help="fix the warps per block (with --buf-len: no autotuning of the headline)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the secondary workloads (triangle, LDA, mixed stream, batched vs plain, served mix)")
    ap.add_argument("--serve-seconds", type=float, default=60.0,
                    help="arrival window of the served mix at 2,000 jobs/s")
    ap.add_argument("--serve-near-seconds", type=float, default=20.0,
                    help="arrival window of the served mix near its measured capacity")
    ap.add_argument("--case", choices=["mixed", "lda", "triangle", "uniform64", "ng", "lda_full", "poisson_large",
                                       "binomial_large"],
                    default=None,
                    help="time one workload at a chosen size instead (profiling): mixed, lda, triangle, "
                         "uniform64, or ng (the headline normal-gamma model)")
    ap.add_argument("--log2n", type=int, default=28, help="--case mixed / uniform64 / poisson_large / binomial_large: log2 of the draws")
    ap.add_argument("--log2s", type=int, default=20, help="--case mixed / uniform64 / poisson_large / binomial_large: log2 of the streams")
    ap.add_argument("--tags", type=int, default=4,
                    help="--case mixed: the draws' tags are uniform over the first TAGS distributions")
    ap.add_argument("--docs", type=int, default=16384, help="--case lda / lda_full: documents")
    ap.add_argument("--chains", type=int, default=N_CHAINS, help="--case ng: chains")
    ap.add_argument("--sweeps", type=int, default=500, help="--case lda/triangle/ng/lda_full: sweeps")
    args = ap.parse_args()
    if args.case:
        return run_case(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
