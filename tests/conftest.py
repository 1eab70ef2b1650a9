import os
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)


def pytest_configure(config):
    config.addinivalue_line("markers", "gpu: needs a CUDA GPU (GB300, sm_103a) and the built library")
    config.addinivalue_line("markers", "slow: longer CPU test")
    # Several CPU tests load the library (its exports, host-side argument
    # checks, the autotuner's host logic), some at import: build it before
    # collection when it is missing or older than its sources (nvcc
    # cross-compiles without a GPU; a no-op when it is current).  Not with
    # BRNG_LIB, which names a build made elsewhere (the checked build).
    if not os.environ.get("BRNG_LIB"):
        import shutil
        if shutil.which("nvcc") or os.path.exists("/usr/local/cuda/bin/nvcc"):
            from paper_1412_4825_gb300 import build_lib
            build_lib.build()


@pytest.fixture(scope="session")
def oracle():
    import oracle as O
    O.lib()
    return O


@pytest.fixture(autouse=True)
def _checked_build_guard(request):
    """With BRNG_CHECKED_RUN=1 (and BRNG_LIB naming the checked build), every
    GPU test also asserts that the checked build counted no failed check while
    it ran: ring protocol, table lookups, and every large-mean Poisson/Binomial
    attempt the FP32 path decided, redone in FP64."""
    if os.environ.get("BRNG_CHECKED_RUN") != "1" or request.node.get_closest_marker("gpu") is None:
        yield
        return
    from paper_1412_4825_gb300 import brng as B
    if B.brng_debug_violations() is None:
        pytest.fail("BRNG_CHECKED_RUN=1 needs the checked build (BRNG_LIB)")
    B.brng_debug_violations(reset=True)
    yield
    assert B.brng_debug_violations() == 0, "the checked build counted failed checks"
