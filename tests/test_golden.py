"""The oracle still reproduces its frozen tiny fixture (tests/golden/tiny_fp64.txt)."""
import os

import numpy as np

import oracle
from tests.golden.make_golden import PARAMS, X, Y

HERE = os.path.dirname(os.path.abspath(__file__))


def load_fixture():
    s2, T = {}, []
    for line in open(os.path.join(HERE, "golden", "tiny_fp64.txt")):
        if line.startswith("#"):
            continue
        parts = line.split()
        if parts[0] == "T":
            T.append([float(v) for v in parts[1:]])
        else:
            s2[parts[0]] = float(parts[1])
    return s2, np.array(T)


def test_oracle_reproduces_fixture():
    s2, T = load_fixture()
    r = oracle.register(X, Y, **PARAMS)
    assert abs(r["sigma2_0"] - s2["sigma2_0"]) <= 1e-14 * s2["sigma2_0"]
    for k in range(PARAMS["n_iter"]):
        ref = s2[f"sigma2_{k + 1}"]
        assert abs(r["sigma2_hist"][k] - ref) <= 1e-12 * ref
    np.testing.assert_allclose(r["T"], T, rtol=0, atol=1e-13)
