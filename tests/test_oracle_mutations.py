"""The oracle pins must catch plausible slips.

Each mutant below is a copy of the oracle's C source with one plausible
mistake planted (on the CPU, in a temporary directory).  The pin suite
(test_oracle_pins.py) is run against each mutant in a subprocess and must
fail.  This shows the pins are not vacuous.
"""
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
SRC = os.path.join(ROOT, "oracle", "cpd_oracle.c")

MUTANTS = {
    "drop_outlier_constant": ("dn[n] = s + c;", "dn[n] = s;"),
    "exponent_missing_factor_2": ("return exp(-d2 / (2.0 * sigma2));", "return exp(-d2 / sigma2);"),
    "no_row_normalisation": ("Ytil[m * D + d] = py[d] / p1;", "Ytil[m * D + d] = py[d];"),
    "outlier_ratio_inverted": ("((double)M / (double)N)", "((double)N / (double)M)"),
    "gram_width_wrong": ("exp(-d2 / (2.0 * beta * beta))", "exp(-d2 / (beta * beta))"),
    "mstep_missing_eigenvalue_factor": ("sdiag[i] = lam[i] * dinv[i];", "sdiag[i] = dinv[i];"),
    "mstep_drops_X": ("T[m * D + d] = X[m * D + d] + t;", "T[m * D + d] = t;"),
    "mstep_residual_sign": ("A[i * D + d] += u * (Ytil[m * D + d] - X[m * D + d]);",
                            "A[i * D + d] += u * (X[m * D + d] - Ytil[m * D + d]);"),
    "sigma2_cross_term_sign": ("(t1 - 2.0 * t2 + t3)", "(t1 + 2.0 * t2 + t3)"),
    "sigma2_normaliser": ("return (t1 - 2.0 * t2 + t3) / ((double)D * (double)M);",
                          "return (t1 - 2.0 * t2 + t3) / ((double)M);"),
    "sigma2_uses_P1_not_row_normalised": ("t1 += S[m] / P1[m];", "t1 += S[m];"),
    "mstep_uses_initial_sigma2": ("fcpd_oracle_mstep(U, lam, M, K, X, Ytil, D, lambda, sigma2, T, W, A);",
                                  "fcpd_oracle_mstep(U, lam, M, K, X, Ytil, D, lambda, sigma2_0, T, W, A);"),
    "sigma2_init_denominator": ("return total / ((double)D * (double)M * (double)N);",
                                "return total / ((double)M * (double)N);"),
    "second_moment_wrong": ("yy += Y[n * D + d] * Y[n * D + d];", "yy += Y[n * D + d];"),
    "rmse_missing_root": ("return sqrt(s / (double)M);", "return s / (double)M;"),
    "rmse_per_coordinate_mean": ("return sqrt(s / (double)M);", "return sqrt(s / ((double)D * (double)M));"),
    "loglik_prior_term_sign": ("ll += (double)N * log((1.0 - w) / (double)M)",
                               "ll -= (double)N * log((1.0 - w) / (double)M)"),
}


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_pins_catch_mutant(name, tmp_path):
    old, new = MUTANTS[name]
    src = open(SRC).read()
    assert src.count(old) == 1, f"mutation anchor for {name} not unique/present"
    mutated = tmp_path / "mutant.c"
    mutated.write_text(src.replace(old, new))
    lib = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-fopenmp", "-fPIC", "-shared", "-ffp-contract=off",
                    "-std=c11", "-D_DEFAULT_SOURCE", "-o", str(lib), str(mutated), "-lm"],
                   check=True)
    env = dict(os.environ, FCPD_ORACLE_LIB=str(lib), OMP_NUM_THREADS="2")
    r = subprocess.run([sys.executable, "-m", "pytest", "-q", "-x", "-p", "no:cacheprovider",
                        os.path.join(ROOT, "tests", "test_oracle_pins.py")],
                       env=env, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert r.returncode != 0, f"mutant {name} survived the pins:\n{r.stdout[-2000:]}"
