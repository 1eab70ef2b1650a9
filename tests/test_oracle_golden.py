"""Cross-host regression: the oracle built on this host reproduces the FP64
bits frozen by tests/golden/make_golden.py (which calls only the oracle).  The
oracle is compiled without contraction or fast-math and its decisions use its
own log/sincospi, so x86-64 and aarch64 builds agree bit for bit; library
pow/exp/log only enter Gamma output values, which are compared to 1 ulp."""
import json
import os

import numpy as np

from paper_1412_4825_gb300 import inputs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "oracle_regression.json")


def _f(h):
    return np.array([float.fromhex(x) for x in h])


def test_oracle_regression(oracle):
    g = json.load(open(GOLDEN))
    r = oracle.gibbs_triangle(42, 4, 10)
    assert np.array_equal(r["xy"].ravel(), _f(g["triangle_xy"]))
    assert np.array_equal(r["mom"].ravel(), _f(g["triangle_mom"]))
    nobs, xbar, sc = inputs.normal_gamma_data(4, seed=42)
    r = oracle.gibbs_normal_gamma(42, 5, nobs, xbar, sc)
    assert np.array_equal(r["pos"].ravel(), np.array(g["ng_pos"], dtype=np.uint64))
    assert np.allclose(r["state"].ravel(), _f(g["ng_state"]), rtol=4e-16, atol=0)
    out, words, _, _ = oracle.gamma(42, 8, inputs.shape_params(64, seed=1))
    assert np.array_equal(words, np.array(g["gamma_words"], dtype=np.uint32))
    assert np.allclose(out, _f(g["gamma_out"]), rtol=4e-16, atol=0)
    vals, _ = oracle.elements(42, 1, 0, 0, 16)
    assert np.array_equal(vals, _f(g["normal_elems"]))
