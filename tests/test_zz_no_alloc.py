"""brng_gamma_static: Gamma draws for callers that cannot call cudaMalloc.

Code that runs inside another framework's memory pool (which must own every
device allocation), or a loop that must not stall on the device-wide
synchronisation cudaMalloc and cudaFree imply, cannot create a handle
(brng_create allocates).  brng_gamma_static keeps its scratch in a fixed
device array instead.  These tests call it through the C ABI, several calls
in a row, and check:
  * each result equals the allocating path (a fresh handle + brng_gamma) bit
    for bit -- the same kernel runs, and no value depends on the launch
    geometry -- and the oracle (words exact, values within the parity
    tests' 2e-6 of the magnitude each Gamma draw works at);
  * the shared array is cleared between calls (a second call with another
    seed and fewer streams starts every stream at its first element);
  * the largest stream count fills the position region to its end, and a
    non-default CUDA stream works;
  * a call allocates nothing: device free memory and the torch allocator's
    counts are unchanged across it.
It lives in a file of its own, collected last, and needs nothing from the
other tests.
"""
import numpy as np
import pytest

import oracle as O

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


def _static(seed, S, alpha, stream=None):
    """One call with outputs allocated beforehand; returns the results and
    (free device bytes, torch allocation count) before and after the call."""
    out = torch.empty(alpha.numel(), dtype=torch.float32, device=DEV)
    words = torch.empty(alpha.numel(), dtype=torch.int32, device=DEV)
    torch.cuda.synchronize()
    before = (torch.cuda.mem_get_info(DEV)[0], torch.cuda.memory_stats(DEV).get("allocation.all.allocated", 0))
    if stream is None:
        B.brng_gamma_static(seed, S, alpha, out, words)
    else:
        B.brng_gamma_static(seed, S, alpha, out, words, stream=stream)
    torch.cuda.synchronize()
    after = (torch.cuda.mem_get_info(DEV)[0], torch.cuda.memory_stats(DEV).get("allocation.all.allocated", 0))
    return out.cpu().numpy(), words.cpu().numpy(), before, after


def _check_oracle(seed, S, alpha, so, sw):
    a = alpha.cpu().numpy()
    ro, rw, _, _, cond = O.gamma(seed, S, a, with_cond=True)
    assert np.array_equal(sw.view(np.uint32), rw)
    g = so.astype(np.float64)
    both_nan = np.isnan(g) & np.isnan(ro)
    ok = both_nan | (np.abs(g - ro) <= RTOL * np.abs(ro) * np.maximum(1.0, cond) + 2 * FLT_MIN)
    assert ok.all(), np.nonzero(~ok)[0][:5]


def test_gamma_static_matches_allocating_path_and_oracle():
    # S = max: the positions fill their whole region, the counters follow it;
    # the last call runs on a non-default CUDA stream
    side = torch.cuda.Stream(device=DEV)
    calls = [(42, 4096, 100003, 1, None), (7, 1000, 20011, 2, None),
             (9, B.BRNG_STATIC_MAX_STREAMS, B.BRNG_STATIC_MAX_STREAMS + 4099, 3, side)]
    for i, (seed, S, n, pseed, stream) in enumerate(calls):
        alpha = torch.from_numpy(inputs.shape_params(n, seed=pseed)).to(DEV)
        alpha[5] = -1.0  # an invalid parameter: NaN on both paths
        so, sw, before, after = _static(seed, S, alpha, stream)
        ro, rw = _allocating(seed, S, alpha)
        assert np.array_equal(sw, rw)
        assert np.array_equal(so.view(np.uint32), ro.view(np.uint32))  # NaN bits included
        assert np.isnan(so[5])
        _check_oracle(seed, S, alpha, so, sw)
        if i > 0:  # the first call on the device may load the module
            assert after == before, (before, after)


def test_gamma_static_rejects_too_many_streams():
    alpha = torch.ones(10, device=DEV)
    out = torch.empty(10, device=DEV)
    with pytest.raises(B.BrngError) as e:
        B.brng_gamma_static(1, B.BRNG_STATIC_MAX_STREAMS + 1, alpha, out)
    assert e.value.code == B.BRNG_EINVAL
