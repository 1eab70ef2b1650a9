"""Batched Gibbs jobs (one persistent kernel over a job table) through the C ABI.

Each job of an uneven batch -- mixed models, chain counts from 1 to thousands,
different sweep counts and seeds -- must give exactly (bit for bit) what
brng_gibbs_run gives for that job alone on a handle with the job's seed; a
batch captured in a CUDA graph and replayed twice must equal two solo runs.
"""
import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

from paper_1412_4825_gb300 import brng as B  # noqa: E402
from paper_1412_4825_gb300 import inputs  # noqa: E402

DEV = torch.device("cuda:0")


def T(a):
    return torch.from_numpy(np.ascontiguousarray(a)).to(DEV)


class Job:
    """Device state of one Gibbs job plus its brng_job_t."""

    def __init__(self, model, n, sweeps, seed, offset=0, K=64):
        self.model, self.n, self.sweeps, self.seed, self.offset = model, n, sweeps, seed, offset
        self.keep = []
        if model == B.MODEL_TRIANGLE:
            self.state = B.triangle_state(n, device=DEV)
            self.mom = torch.zeros((n, 5), dtype=torch.float64, device=DEV)
            self.params = None
            self.state_arg = self.state
        elif model == B.MODEL_NORMAL_GAMMA:
            nobs, xbar, sc = inputs.normal_gamma_data(n, seed=seed % 1000)
            self.data = [T(nobs), T(xbar), T(sc)]
            self.params = B.brng_normal_gamma_params_t(2.0, 1.0, 0.0, 0.01, *[d.data_ptr() for d in self.data])
            self.state = B.normal_gamma_state(n, device=DEV)
            self.mom = torch.zeros((n, 4), dtype=torch.float64, device=DEV)
            self.state_arg = self.state
        else:
            alpha, _, _ = inputs.lda_alpha(n, K=K, seed=seed % 1000)
            self.alpha = T(alpha)
            self.params = B.brng_lda_params_t(K, self.alpha.data_ptr())
            self.theta = torch.zeros((n, K), dtype=torch.float32, device=DEV)
            self.pos = torch.zeros((n, K, 2), dtype=torch.int64, device=DEV)
            self.mom = torch.zeros((n, K), dtype=torch.float64, device=DEV)
            self.state_arg = B.brng_lda_state_t(self.theta.data_ptr(), self.pos.data_ptr())
            self.state = self.theta

    def job(self):
        j, keep = B.make_job(self.model, self.n, self.sweeps, self.seed, self.params, self.state_arg,
                             self.mom, chain_offset=self.offset)
        self.keep.append(keep)
        return j

    def solo(self, **tune):
        h = B.Handle(self.seed, 1)
        if tune:
            h.tune(**tune)
        B.brng_gibbs_run(h.h, self.model, self.offset, self.n, self.sweeps, self.params, self.state_arg,
                         self.mom)
        torch.cuda.synchronize()
        h.close()

    def snapshot(self):
        out = [self.state.clone(), self.mom.clone()]
        if self.model == B.MODEL_LDA:
            out.append(self.pos.clone())
        return out


def _jobs(seed0=100):
    rng = np.random.default_rng(seed0)
    jobs = []
    for i in range(18):
        model = [B.MODEL_TRIANGLE, B.MODEL_NORMAL_GAMMA, B.MODEL_LDA][i % 3]
        n = int(np.exp(rng.uniform(0, np.log(3000 if model != B.MODEL_LDA else 300))))
        sweeps = int(rng.integers(5, 120))
        jobs.append(Job(model, n, sweeps, seed=seed0 + i, offset=int(rng.integers(0, 1000))))
    jobs.append(Job(B.MODEL_NORMAL_GAMMA, 1, 50, seed=7))  # a single chain
    jobs.append(Job(B.MODEL_LDA, 3, 20, seed=8, K=5))      # K < 32
    return jobs


def test_batch_equals_solo_runs():
    solo = _jobs()
    for j in solo:
        j.solo()
    batch = _jobs()
    h = B.Handle(1, 1)
    B.brng_gibbs_batch(h.h, [j.job() for j in batch])
    torch.cuda.synchronize()
    for a, b in zip(solo, batch):
        for x, y in zip(a.snapshot(), b.snapshot()):
            assert torch.equal(x, y), (a.model, a.n, a.sweeps)


def test_batch_with_large_k_equals_solo_runs():
    """LDA jobs with K = 100 and 128 put the whole batch on the four-components-
    per-lane kernel; every job (LDA, triangle, normal-gamma) still equals its
    solo run."""
    def jobs():
        return [Job(B.MODEL_LDA, 37, 15, seed=31, K=100), Job(B.MODEL_LDA, 20, 12, seed=32, K=128),
                Job(B.MODEL_LDA, 50, 10, seed=33, K=64), Job(B.MODEL_TRIANGLE, 700, 40, seed=34),
                Job(B.MODEL_NORMAL_GAMMA, 900, 30, seed=35, offset=77)]
    solo = jobs()
    for j in solo:
        j.solo()
    batch = jobs()
    h = B.Handle(1, 1)
    B.brng_gibbs_batch(h.h, [j.job() for j in batch])
    torch.cuda.synchronize()
    for a, b in zip(solo, batch):
        for x, y in zip(a.snapshot(), b.snapshot()):
            assert torch.equal(x, y), (a.model, a.n, a.sweeps)


def test_batch_tuning_and_plan_reuse():
    solo = _jobs(300)
    for j in solo:
        j.solo()
    batch = _jobs(300)
    h = B.Handle(1, 1)
    h.tune(buf_len=8, warps_per_block=2, lookahead=3)
    B.brng_gibbs_batch(h.h, [j.job() for j in batch])
    torch.cuda.synchronize()
    for a, b in zip(solo, batch):
        for x, y in zip(a.snapshot(), b.snapshot()):
            assert torch.equal(x, y)


def test_batch_graph_capture_replay():
    """One batch plan captured in a CUDA graph; two replays continue every
    job's chains exactly as two solo runs do."""
    solo = _jobs(500)
    for _ in range(2):
        for j in solo:
            j.solo()
    batch = _jobs(500)
    h = B.Handle(1, 1)
    plan = B.brng_batch_create(h.h, [j.job() for j in batch])
    s = torch.cuda.Stream()
    torch.cuda.synchronize()
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=s):
        B.brng_batch_launch(plan, s)
    g.replay()
    g.replay()
    torch.cuda.synchronize()
    for a, b in zip(solo, batch):
        for x, y in zip(a.snapshot(), b.snapshot()):
            assert torch.equal(x, y)
    B.brng_batch_destroy(plan)


def test_batch_rejects_bad_job():
    h = B.Handle(1, 1)
    good = Job(B.MODEL_TRIANGLE, 10, 5, seed=1)
    bad, keep = B.make_job(B.MODEL_NORMAL_GAMMA, 10, 5, 1, None, good.state, good.mom)  # no params
    with pytest.raises(B.BrngError):
        B.brng_gibbs_batch(h.h, [good.job(), bad])
    assert B.brng_gibbs_batch(h.h, []) == B.BRNG_OK
