"""The spectral-trim rule of the M-step, checked on the FP64 oracle (CPU).

Direction k of the eigenbasis enters T (Eq. 17) through s_k a_k with
s_k = l_k / (l_k + lambda sigma2) and a = U^T (Ytil - X).  Keeping only the
directions with s_k >= eps is the top-K M-step (Eq. 20) with K = that count
(s_k decreases with k), and the dropped part has norm <= eps |Ytil - X|
because U is orthonormal.  These tests pin that rule -- the one the GPU's
trimmed M-step relies on -- with the oracle's own eigendecomposition and
M-step.
"""
import numpy as np
import pytest

import oracle
from paper_2006_06281_gb300 import datagen

EPS = 2.0 ** -24
LAM_REG = 2.0


@pytest.fixture(scope="module")
def case():
    ps = datagen.gen(400, n_out=0, amp=0.15, noise=0.01, seed=41)
    U, lam = oracle.eig(ps.X, 2.0)
    # a posterior mean from the oracle's own E-step at a moderate variance
    e = oracle.estep(ps.X, ps.Y, 0.01, 0.1)
    return ps.X, e["Ytil"], U, lam


@pytest.mark.parametrize("sigma2", [0.3, 1e-2, 1e-3, 1e-4])
def test_dropping_directions_below_eps_moves_T_by_at_most_eps_R(case, sigma2):
    X, Yt, U, lam = case
    M = X.shape[0]
    s = lam / (lam + LAM_REG * sigma2)
    assert np.all(np.diff(s) <= 0)                       # the kept set is a leading block
    k = int((s >= EPS).sum())
    T_full, _, _ = oracle.mstep(U, lam, X, Yt, LAM_REG, sigma2)
    T_trim, _, _ = oracle.mstep(U[:, :k], lam[:k], X, Yt, LAM_REG, sigma2)
    R = np.linalg.norm(Yt - X)
    d = np.linalg.norm(T_trim - T_full)
    print(f"sigma2 {sigma2:g}: {k} of {M} directions kept; |dT| = {d:.3e}, eps |R| = {EPS * R:.3e}")
    assert d <= EPS * R + 1e-13 * np.linalg.norm(T_full)
    # the spectrum decays fast: most directions are below one FP32 rounding
    assert k < M // 2


def test_the_setup_threshold_covers_every_sigma2_above_the_floor(case):
    # k_cap keeps every l_k >= eps lambda s2f / (1 - eps): then for any
    # sigma2 >= s2f the largest dropped eigenvalue has s < eps
    X, _, U, lam = case
    s2f = 1e-4 * X.var(axis=0).mean()
    thr = EPS * LAM_REG * s2f / (1.0 - EPS)
    k_cap = int((lam >= thr).sum())
    k_cap = (k_cap + 15) // 16 * 16
    assert k_cap < X.shape[0]
    l_drop = lam[k_cap]
    for sigma2 in (s2f, 2 * s2f, 1e-2, 1.0):
        assert l_drop / (l_drop + LAM_REG * sigma2) < EPS
    # and below the floor the test can fail: the full M-step must then run
    tiny = l_drop / (EPS * LAM_REG) * 1e-3
    assert not (l_drop / (l_drop + LAM_REG * tiny) < EPS) or l_drop == 0.0
