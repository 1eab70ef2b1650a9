"""CPU check of the certified FP32 attempts of the large-mean discrete
samplers (PTRS for Poisson, BTRD for Binomial): the kernel headers are built
for the host (tests/rejection32_host.cpp maps each device intrinsic to the
IEEE host operation with the same rounding) and every attempt the FP32 /
float-float path decides must give the count and element use of the FP64
attempt, on random parameters over the whole large-mean range and random
elements on the 2^-24 grid.  The FP32 path must also decide almost every
attempt, else the FP64 pipe would still set the speed.

The host's logf and log1pf are not CUDA's (both within about one ulp), so
this also checks that the bands do not depend on one implementation of the
two functions; the checked GPU build repeats the comparison with CUDA's.
Random attempts rarely fall near a boundary, so a second mode places them
there on purpose.

The float-float operations themselves are checked against their stated
error bounds.  The small-mean inversions (csrc/brng_inversion.cuh) are
checked the same way as the attempts: each draw that the FP32 tier or the double-single tier decides must
equal the FP64 inversion, at random and on the grid points next to the CDF's
steps.
"""
import json
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_1412_4825_gb300", "csrc")


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++") or shutil.which("c++")
    if cxx is None:
        pytest.skip("no C++ compiler")
    d = tmp_path_factory.mktemp("rejection32")
    (d / "fake").mkdir()
    (d / "fake" / "cuda_runtime.h").write_text("")  # the headers need nothing from it on the host
    exe = str(d / "rejection32_host")
    subprocess.run([cxx, "-O2", "-std=c++17", "-ffp-contract=off", "-I", str(d / "fake"), "-I", CSRC,
                    os.path.join(HERE, "rejection32_host.cpp"), "-o", exe], check=True)
    return exe


@pytest.mark.parametrize("method,seed", [("ptrs_edges", 5), ("btrd_edges", 6)])
def test_certified_attempts_at_the_boundaries(harness, method, seed):
    """Attempts placed next to each decision's boundary (found on the FP64
    attempt by bisection over the 2^-24 grid: the steps of floor(X), the
    thresholds on v, the turn from accept to reject of the log and product
    tests): still no decided attempt differs from FP64, and the boundaries
    are reached (many attempts there are left undecided, as the bands
    intend)."""
    r = subprocess.run([harness, method, "60000", str(seed)], capture_output=True, text=True, check=True)
    res = json.loads(r.stdout)
    assert res["mismatches"] == 0, r.stderr
    assert res["undecided"] > 0.05 * res["attempts"], res
    assert res["decided"] > 0.3 * res["attempts"], res


@pytest.mark.parametrize("method,seed", [("ptrs", 1), ("ptrs", 2), ("btrd", 3), ("btrd", 4)])
def test_certified_attempts_equal_fp64(harness, method, seed):
    n = 3_000_000
    r = subprocess.run([harness, method, str(n), str(seed)], capture_output=True, text=True, check=True)
    res = json.loads(r.stdout)
    assert res["mismatches"] == 0, r.stderr
    assert res["attempts"] == n
    assert res["undecided"] <= 3e-3 * n, res  # FP64 for a few attempts in a thousand at most
    assert 0.8 * n < res["accepted"] < 0.95 * n, res  # both outcomes are exercised


def test_inversion_tiers_equal_fp64(harness):
    """Poisson (lambda log-uniform [0.05, 64]) and Binomial (n to 2^24, mean
    <= 64) draws: the FP32 tier decides nearly all, the double-single tier
    most of the rest, and every decided draw is the FP64 draw."""
    r = subprocess.run([harness, "inv", "1000000", "8"], capture_output=True, text=True, check=True)
    res = json.loads(r.stdout)
    assert res["mismatches"] == 0, r.stderr
    assert res["decided_ds"] > 300, res
    assert res["undecided"] <= 5e-4 * res["draws"], res


def test_inversion_tiers_at_cdf_steps(harness):
    """u on the grid points next to a step of the CDF (within one 2^-24 of
    it): the FP32 tier abstains on nearly all, the tiers decide only what
    their bounds allow, and no decided draw differs from FP64."""
    r = subprocess.run([harness, "inv_edges", "30000", "9"], capture_output=True, text=True, check=True)
    res = json.loads(r.stdout)
    assert res["mismatches"] == 0, r.stderr
    assert res["draws"] > 100000, res
    assert res["decided32"] < 0.2 * res["draws"], res
    assert res["decided_ds"] > 1000, res


def test_float_float_error_bounds(harness):
    """The float-float operations the certified decisions rest on
    (csrc/brng_ff.cuh) stay within the relative error bounds their header
    states (Joldes, Muller and Popescu), in units of u^2 = 2^-48, on random
    operands over 60 binades, 14 % of the sums cancelling below 2^-20 of
    their operands; checked against quad-precision sums and long-double
    products, quotients and roots."""
    r = subprocess.run([harness, "ffops", "3000000", "3"], capture_output=True, text=True, check=True)
    res = json.loads(r.stdout)
    bounds = {"add": 3.0 / (1 - 4 * 2.0 ** -24), "add_f": 2.0, "mul": 5.0, "mul_f": 2.0, "div_f": 3.0,
              "div": 15.0 + 56 * 2.0 ** -24, "sqrt": 25.0 / 8.0}
    for op, b in bounds.items():
        assert res[op] <= b, (op, res)
    assert res["sums"] > 2_000_000 and res["cancelling_sums"] > 100_000, res
