"""The checked build (-DBRNG_DEBUG: ring-protocol and table-lookup checks
counted on the device, csrc/brng_debug.cuh) in place of a sanitizer: every
workload of tests/checked_workload.py runs through it without a failed check
and gives the same bits as the normal build.  Each build runs in its own
process (BRNG_LIB selects the library)."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

HERE = os.path.dirname(os.path.abspath(__file__))


def _run(lib):
    env = dict(os.environ)
    if lib:
        env["BRNG_LIB"] = lib
    else:
        env.pop("BRNG_LIB", None)
    r = subprocess.run([sys.executable, os.path.join(HERE, "checked_workload.py")], env=env,
                       capture_output=True, text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    return json.loads(r.stdout.strip().splitlines()[-1])


def test_checked_build_no_violation_same_bits():
    from paper_1412_4825_gb300 import build_lib
    debug_lib = build_lib.build(debug=True)
    checked = _run(debug_lib)
    normal = _run(None)
    assert normal["violations"] is None  # the normal build has no checks
    assert checked["violations"] == 0, checked
    assert checked["digests"] == normal["digests"]
    assert len(normal["digests"]) >= 20
