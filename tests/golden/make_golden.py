"""Writes tests/golden/tiny_fp64.txt from the FP64 oracle only.

Input: five model points and seven scene points typed by hand (short
decimals, so the input is exact on every machine); omega = 0.1, lambda = 2,
beta = 2, sigma2_0 from the data, five EM iterations of the full-basis update
(Eq. 4, Eq. 5, Eq. 17, Eq. 18).  The fixture freezes the oracle's output so a
later change to its arithmetic shows up as a failing test.

Run from the repository root:  python tests/golden/make_golden.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)
import oracle  # noqa: E402

X = np.array([[-0.5, -0.25, 0.0], [0.25, -0.5, 0.125], [0.5, 0.5, -0.25],
              [-0.25, 0.75, 0.5], [0.0, 0.0, -0.75]])
Y = np.array([[-0.375, -0.25, 0.125], [0.375, -0.375, 0.25], [0.625, 0.5, -0.125],
              [-0.125, 0.875, 0.5], [0.125, 0.0, -0.625], [1.0, -1.0, 1.0], [0.0, 0.25, 0.0]])
PARAMS = dict(w=0.1, beta=2.0, lam_reg=2.0, n_iter=5)


def main():
    r = oracle.register(X, Y, **PARAMS)
    assert r["status"] == 0
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_fp64.txt")
    with open(path, "w") as f:
        f.write("# FP64 oracle output; written by tests/golden/make_golden.py (Eq. 4, 5, 17, 18)\n")
        f.write("# params w=0.1 beta=2 lambda=2 n_iter=5 sigma2_0=from data\n")
        f.write(f"sigma2_0 {r['sigma2_0']:.17e}\n")
        for k, s in enumerate(r["sigma2_hist"]):
            f.write(f"sigma2_{k + 1} {s:.17e}\n")
        for m in range(X.shape[0]):
            f.write("T " + " ".join(f"{v:.17e}" for v in r["T"][m]) + "\n")


if __name__ == "__main__":
    main()
