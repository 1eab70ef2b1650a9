"""Write tests/golden/oracle_regression.json from the oracle alone.

The file freezes a few small oracle results (hex floats) so that a build of
the oracle on another host (x86-64 or aarch64) can be checked to give the same
FP64 bits.  It calls only oracle/ and paper_1412_4825_gb300.inputs.
"""
import json
import os
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import oracle as O  # noqa: E402
from paper_1412_4825_gb300 import inputs  # noqa: E402


def hx(a):
    return [float(v).hex() for v in np.asarray(a, dtype=np.float64).ravel()]


def main():
    g = {}
    r = O.gibbs_triangle(42, 4, 10)
    g["triangle_xy"] = hx(r["xy"])
    g["triangle_mom"] = hx(r["mom"])
    nobs, xbar, sc = inputs.normal_gamma_data(4, seed=42)
    r = O.gibbs_normal_gamma(42, 5, nobs, xbar, sc)
    g["ng_state"] = hx(r["state"])
    g["ng_pos"] = [int(v) for v in r["pos"].ravel()]
    out, words, pos, _ = O.gamma(42, 8, inputs.shape_params(64, seed=1))
    g["gamma_out"] = hx(out)
    g["gamma_words"] = [int(v) for v in words]
    vals, words = O.elements(42, 1, 0, 0, 16)
    g["normal_elems"] = hx(vals)
    with open(os.path.join(HERE, "oracle_regression.json"), "w") as f:
        json.dump(g, f, indent=1)


if __name__ == "__main__":
    main()
