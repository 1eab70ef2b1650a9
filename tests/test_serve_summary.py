"""Host-side latency accounting of the served mix (no GPU): percentiles over
every submitted job, unfinished jobs entering with their age at the end of
the window (right-censored), beside the completed-only percentiles."""
import numpy as np

from paper_1412_4825_gb300 import serve


def test_censored_jobs_enter_the_percentiles():
    r = serve.MixResult()
    r.latencies = [0.01] * 10           # 10 fast completions
    r.censored_ages = [5.0] * 90        # 90 jobs still waiting after 5 s
    r.submitted, r.completed, r.window = 100, 10, 10.0
    s = r.summary()
    assert s["completed_fraction"] == 0.1 and s["censored"] == 90
    assert s["p50_s"] == 5.0 and s["p99_s"] == 5.0       # lower bounds, not the survivors'
    assert s["p50_completed_s"] == 0.01                  # what a survivor-only count would say
    assert s["jobs_completed_per_s"] == 1.0


def test_no_censoring_reduces_to_plain_percentiles():
    r = serve.MixResult()
    rng = np.random.default_rng(1)
    r.latencies = list(rng.exponential(0.1, 1000))
    r.submitted, r.completed, r.window = 1000, 1000, 5.0
    s = r.summary()
    assert s["censored"] == 0 and s["completed_fraction"] == 1.0
    assert s["p50_s"] == s["p50_completed_s"] and s["p99_s"] == s["p99_completed_s"]
    assert np.isclose(s["p99_s"], np.percentile(r.latencies, 99))
