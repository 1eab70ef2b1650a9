"""brng_gamma_static: Gamma draws for callers that cannot call cudaMalloc.

Code that runs inside another framework's memory pool, or a loop that must not
stall on cudaMalloc's device-wide synchronisation, cannot create a handle
(brng_create allocates).  brng_gamma_static keeps its scratch in a fixed
device array instead.  This test calls it twice in a row through the C ABI and
checks each result against the allocating path (a fresh handle + brng_gamma)
within the tolerance the parity tests use; the second call also checks that
the shared array is cleared between calls.  It lives in a file of its own,
collected last, and needs nothing from the other tests.
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
RTOL = 2e-6
FLT_MIN = float(np.finfo(np.float32).tiny)


def _allocating(seed, S, alpha):
    h = B.Handle(seed, S)
    out = torch.empty(alpha.numel(), dtype=torch.float32, device=DEV)
    words = torch.empty(alpha.numel(), dtype=torch.int32, device=DEV)
    B.brng_gamma(h.h, alpha, out, words)
    torch.cuda.synchronize()
    h.close()
    return out.cpu().numpy(), words.cpu().numpy()


def _static(seed, S, alpha):
    out = torch.empty(alpha.numel(), dtype=torch.float32, device=DEV)
    words = torch.empty(alpha.numel(), dtype=torch.int32, device=DEV)
    B.brng_gamma_static(seed, S, alpha, out, words)
    torch.cuda.synchronize()
    return out.cpu().numpy(), words.cpu().numpy()


def test_gamma_static_matches_allocating_path_twice():
    calls = [(42, 4096, 100003, 1), (7, 1000, 20011, 2)]  # second call: fewer streams, other seed
    for seed, S, n, pseed in calls:
        alpha = torch.from_numpy(inputs.shape_params(n, seed=pseed)).to(DEV)
        alpha[5] = -1.0  # an invalid parameter: NaN on both paths
        so, sw = _static(seed, S, alpha)
        ro, rw = _allocating(seed, S, alpha)
        assert np.array_equal(sw, rw)
        assert np.isnan(so[5]) and np.isnan(ro[5])
        ok = np.isnan(ro) & np.isnan(so) | (np.abs(so.astype(np.float64) - ro) <= RTOL * np.abs(ro) + 2 * FLT_MIN)
        assert ok.all()


def test_gamma_static_rejects_too_many_streams():
    alpha = torch.ones(10, device=DEV)
    out = torch.empty(10, device=DEV)
    with pytest.raises(B.BrngError) as e:
        B.brng_gamma_static(1, 65537, alpha, out)
    assert e.value.code == B.BRNG_EINVAL
