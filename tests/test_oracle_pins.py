"""Pins for the FP64 oracle (no GPU).

Each test checks the oracle against something other than itself: a closed
form, an invariant the paper states, a textbook solve, a brute-force
evaluation of a different formula for the same quantity, or a symmetry.
The aim is that a plausible slip anywhere in the oracle (a dropped term, a
wrong sign or index, a transposed operand, the wrong sigma2 in the M-step)
fails at least one of them.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2006_06281_gb300 import datagen


def _rng_points(seed, M, N, spread=1.0):
    s = datagen.Stream(seed)
    X = (s.uniform(3 * M).reshape(M, 3) * 2 - 1) * spread
    Y = (s.uniform(3 * N).reshape(N, 3) * 2 - 1) * spread
    return X, Y


def _gmm_posterior(T, Y, sigma2, w):
    """Posterior of component m given y_n for the mixture of Eq. 2, written
    with Bayes' rule: prior (1-w)/M times the normalised Gaussian density g of
    Eq. 1, divided by the mixture density p(y_n) (uniform part w/N).  This is
    a different formula from Eq. 4 (no constant c): agreement pins c."""
    M, D = T.shape
    N = Y.shape[0]
    d2 = ((Y[None, :, :] - T[:, None, :]) ** 2).sum(-1)           # (M, N)
    g = np.exp(-d2 / (2 * sigma2)) / (2 * math.pi * sigma2) ** (D / 2)
    joint = (1 - w) / M * g
    p_y = w / N + joint.sum(0)
    return joint / p_y[None, :], p_y


# ---------------------------------------------------------------- Eq. 11
def test_gram_matrix_values():
    X = np.array([[0.0, 0.0, 0.0], [1.0, 0.0, 0.0], [0.0, 2.0, 0.0]])
    Phi = oracle.gram(X, beta=2.0)
    assert np.allclose(np.diag(Phi), 1.0, rtol=0, atol=0)
    assert np.array_equal(Phi, Phi.T)
    # |x0-x1|^2 = 1, |x0-x2|^2 = 4, |x1-x2|^2 = 5 ; 2 beta^2 = 8
    assert Phi[0, 1] == pytest.approx(math.exp(-1 / 8), rel=1e-15)
    assert Phi[0, 2] == pytest.approx(math.exp(-4 / 8), rel=1e-15)
    assert Phi[1, 2] == pytest.approx(math.exp(-5 / 8), rel=1e-15)


# ---------------------------------------------------------------- Eq. 16 / 19
def test_eigendecomposition_reconstructs_gram():
    X, _ = _rng_points(1, 200, 1)
    Phi = oracle.gram(X, 2.0)
    U, lam = oracle.eig(X, 2.0)
    assert np.all(np.diff(lam) <= 0), "descending order"
    assert np.all(lam >= 0), "clamped at zero"
    rec = (U * lam) @ U.T
    assert np.linalg.norm(rec - Phi) / np.linalg.norm(Phi) < 1e-13
    assert np.abs(U.T @ U - np.eye(200)).max() < 1e-12
    # columns are eigenvectors: Phi u_i = l_i u_i (absolute, scale of l_max)
    assert np.abs(Phi @ U - U * lam).max() < 1e-11 * lam[0]
    # top-K is the leading block of the full basis
    Uk, lk = oracle.eig(X, 2.0, K=17)
    assert Uk.shape == (200, 17) and np.array_equal(lk, lam[:17])
    assert np.array_equal(Uk, U[:, :17])
    # trace of Phi is M (unit diagonal): the spectrum must sum to M
    assert lam.sum() == pytest.approx(200.0, rel=1e-12)


# ---------------------------------------------------------------- Eq. 4
def test_outlier_constant_special_values():
    # (2 pi sigma2)^(D/2) = 1 when sigma2 = 1/(2 pi): c = w/(1-w) M/N
    assert oracle.outlier_c(1 / (2 * math.pi), 0.5, 2, 4, 3) == pytest.approx(0.5, rel=1e-15)
    assert oracle.outlier_c(0.3, 0.0, 10, 10, 3) == 0.0
    # D/2 exponent: D = 2, sigma2 = 1 -> 2 pi
    assert oracle.outlier_c(1.0, 0.5, 1, 1, 2) == pytest.approx(2 * math.pi, rel=1e-15)


@pytest.mark.parametrize("w", [0.0, 0.1, 0.7])
def test_estep_is_bayes_posterior_of_the_mixture(w):
    T, Y = _rng_points(2, 37, 53, spread=0.5)
    sigma2 = 0.07
    e = oracle.estep(T, Y, sigma2, w)
    assert e["status"] == oracle.OK
    P, p_y = _gmm_posterior(T, Y, sigma2, w)
    # column invariant of Eq. 4: sum_m p_mn + c / den_n = 1
    c = oracle.outlier_c(sigma2, w, 37, 53, 3)
    np.testing.assert_allclose(P.sum(0) + c / e["den"], 1.0, rtol=0, atol=1e-14)
    # row quantities of the posterior
    np.testing.assert_allclose(e["P1"], P.sum(1), rtol=1e-12)
    np.testing.assert_allclose(e["PY"], P @ Y, rtol=1e-12, atol=1e-15)
    np.testing.assert_allclose(e["S"], P @ (Y * Y).sum(1), rtol=1e-12)
    # Eq. 3 log-likelihood straight from the mixture density
    assert e["loglik"] == pytest.approx(np.log(p_y).sum(), rel=1e-12)


# ---------------------------------------------------------------- Eq. 5
def test_corresponding_constraint_normalises_rows_not_columns():
    T, Y = _rng_points(3, 29, 41, spread=0.6)
    e = oracle.estep(T, Y, 0.05, 0.2)
    P, _ = _gmm_posterior(T, Y, 0.05, 0.2)
    Phat = P / P.sum(1, keepdims=True)               # each row sums to 1
    np.testing.assert_allclose(Phat.sum(1), 1.0, atol=1e-15)
    np.testing.assert_allclose(e["Ytil"], Phat @ Y, rtol=1e-12, atol=1e-14)
    # without the row rescaling of Eq. 5 the estimate would be P Y, which
    # differs on this input (rows of P do not sum to 1)
    assert np.abs(P.sum(1) - 1).max() > 1e-2
    assert np.abs(e["Ytil"] - P @ Y).max() > 1e-3
    # Ytil is a convex combination of scene points
    assert np.all(e["Ytil"] >= Y.min(0) - 1e-15) and np.all(e["Ytil"] <= Y.max(0) + 1e-15)


def test_estep_reports_row_underflow():
    T = np.array([[0.0, 0.0, 0.0], [100.0, 0.0, 0.0]])
    Y = np.array([[0.01, 0.0, 0.0], [0.0, 0.02, 0.0]])
    e = oracle.estep(T, Y, 1e-3, 0.1)
    assert e["status"] == oracle.ENUMERIC


# ---------------------------------------------------------------- Eq. 15 / 17 / 21
@pytest.mark.parametrize("sigma2", [0.3, 0.02])
def test_mstep_equals_dense_solve_of_normal_equations(sigma2):
    X, _ = _rng_points(4, 48, 1, spread=0.8)
    s = datagen.Stream(44)
    Ytil = X + 0.1 * s.normal(48 * 3).reshape(48, 3)
    lam_reg = 2.0
    Phi = oracle.gram(X, 2.0)
    U, lam = oracle.eig(X, 2.0)
    T, W, A = oracle.mstep(U, lam, X, Ytil, lam_reg, sigma2)
    # Eq. 15 solved directly (Cholesky) -- no eigendecomposition involved
    L = np.linalg.cholesky(Phi + lam_reg * sigma2 * np.eye(48))
    Wd = np.linalg.solve(L.T, np.linalg.solve(L, Ytil - X))
    np.testing.assert_allclose(W, Wd, rtol=1e-9, atol=1e-10 * np.abs(Wd).max())
    np.testing.assert_allclose(T, X + Phi @ Wd, rtol=0, atol=1e-12)
    np.testing.assert_allclose(A, U.T @ (Ytil - X), atol=1e-13)


def test_cpd_update_with_normalised_posterior_reduces_to_fast_update():
    """Eq. 21 (CPD) fed with the row-normalised posterior (d(P1) = I) is Eq. 15."""
    X, Y = _rng_points(5, 31, 40, spread=0.7)
    sigma2, w, lam_reg = 0.04, 0.1, 3.0
    P, _ = _gmm_posterior(X, Y, sigma2, w)
    Phat = P / P.sum(1, keepdims=True)
    P1 = Phat.sum(1)
    Phi = oracle.gram(X, 2.0)
    Wcpd = np.linalg.solve(Phi + lam_reg * sigma2 * np.diag(1 / P1), (Phat @ Y) / P1[:, None] - X)
    e = oracle.estep(X, Y, sigma2, w)
    U, lam = oracle.eig(X, 2.0)
    T, W, _ = oracle.mstep(U, lam, X, e["Ytil"], lam_reg, sigma2)
    np.testing.assert_allclose(W, Wcpd, rtol=1e-8, atol=1e-10 * np.abs(Wcpd).max())
    np.testing.assert_allclose(T, X + Phi @ Wcpd, atol=1e-12)


# ---------------------------------------------------------------- Eq. 19 / 20
def test_lowrank_update():
    X, _ = _rng_points(6, 60, 1)
    s = datagen.Stream(66)
    Ytil = X + 0.05 * s.normal(180).reshape(60, 3)
    Phi = oracle.gram(X, 2.0)
    U, lam = oracle.eig(X, 2.0)
    Tf, Wf, _ = oracle.mstep(U, lam, X, Ytil, 2.0, 0.01)
    # K = M is the full basis
    Uk, lk = oracle.eig(X, 2.0, K=60)
    Tk, Wk, _ = oracle.mstep(Uk, lk, X, Ytil, 2.0, 0.01)
    np.testing.assert_allclose(Tk, Tf, atol=1e-15)
    # K < M: W~ = U~ (L~ + lambda sigma2)^-1 U~^T (Ytil - X) and T = X + Phi W~
    U8, l8 = oracle.eig(X, 2.0, K=8)
    T8, W8, _ = oracle.mstep(U8, l8, X, Ytil, 2.0, 0.01)
    W8_direct = U8 @ ((U8.T @ (Ytil - X)) / (l8 + 2.0 * 0.01)[:, None])
    np.testing.assert_allclose(W8, W8_direct, atol=1e-13)
    np.testing.assert_allclose(T8, X + Phi @ W8_direct, atol=1e-12)
    # the truncated update differs from the full one (rank matters here)
    assert np.abs(T8 - Tf).max() > 1e-6


# ---------------------------------------------------------------- Eq. 18
def test_sigma2_update_matches_bruteforce_definition():
    X, Y = _rng_points(7, 23, 35, spread=0.6)
    sigma2, w = 0.05, 0.1
    e = oracle.estep(X, Y, sigma2, w)
    U, lam = oracle.eig(X, 2.0)
    T, _, _ = oracle.mstep(U, lam, X, e["Ytil"], 2.0, sigma2)
    P, _ = _gmm_posterior(X, Y, sigma2, w)
    Phat = P / P.sum(1, keepdims=True)
    d2 = ((Y[None, :, :] - T[:, None, :]) ** 2).sum(-1)
    brute = (Phat * d2).sum() / (3 * 23)
    assert oracle.sigma2_update(e["S"], e["P1"], e["Ytil"], T) == pytest.approx(brute, rel=1e-12)


def test_sigma2_init_definition():
    assert oracle.sigma2_init(np.zeros((1, 3)), np.array([[1.0, 0, 0]])) == pytest.approx(1 / 3)
    X, Y = _rng_points(8, 19, 27)
    closed = (27 * (X ** 2).sum() + 19 * (Y ** 2).sum() - 2 * X.sum(0) @ Y.sum(0)) / (3 * 19 * 27)
    assert oracle.sigma2_init(X, Y) == pytest.approx(closed, rel=1e-13)


# ---------------------------------------------------------------- the loop
@pytest.mark.parametrize("lam_reg,w", [(2.0, 0.1), (10.0, 0.7), (0.5, 0.0)])
def test_single_point_closed_form(lam_reg, w):
    """M = N = 1: Phi = [1], p^ = 1, Ytil = y, t = x + (y - x)/(1 + lambda sigma2),
    sigma2' = (lambda sigma2 / (1 + lambda sigma2))^2 |y - x|^2 / D, with the
    OLD sigma2 in the M-step.  The pair is far apart so sigma2 stays well above
    the rounding floor of Eq. 18's expanded form during the six iterations."""
    x = np.array([[0.1, -0.2, 0.3]])
    y = np.array([[2.1, 1.8, -1.7]])
    r2 = float(((y - x) ** 2).sum())
    res = oracle.register(x, y, w=w, beta=2.0, lam_reg=lam_reg, n_iter=6)
    assert res["status"] == oracle.OK and res["iters"] == 6
    s2 = r2 / 3
    assert res["sigma2_0"] == pytest.approx(s2, rel=1e-15)
    for k in range(6):
        f = lam_reg * s2 / (1 + lam_reg * s2)
        s2 = f * f * r2 / 3
        assert res["sigma2_hist"][k] == pytest.approx(s2, rel=1e-11)
    f_last = 1 / (1 + lam_reg * res["sigma2_hist"][-2])
    np.testing.assert_allclose(res["T"], x + (y - x) * f_last, rtol=1e-13)


def test_identity_pair_converges_to_itself():
    ps = datagen.gen(150, amp=0.0, noise=0.0, seed=9)
    X = ps.X
    res = oracle.register(X, X.copy(), w=0.1, beta=2.0, lam_reg=2.0, n_iter=50)
    assert res["status"] == oracle.OK
    h = np.concatenate([[res["sigma2_0"]], res["sigma2_hist"]])
    assert np.all(np.diff(h) <= 1e-15), "sigma2 non-increasing"
    assert h[-1] < 1e-3 * h[0]
    assert np.sqrt(((res["T"] - X) ** 2).sum(1).mean()) < 1e-3


def test_rigid_motion_equivariance_and_permutations():
    ps = datagen.gen(80, amp=0.1, noise=0.01, seed=10)
    X, Y = ps.X, ps.Y
    base = oracle.register(X, Y, w=0.1, beta=2.0, lam_reg=2.0, n_iter=10)
    th = 0.7
    R = np.array([[math.cos(th), -math.sin(th), 0], [math.sin(th), math.cos(th), 0], [0, 0, 1.0]])
    t = np.array([0.3, -0.2, 0.5])
    moved = oracle.register(X @ R.T + t, Y @ R.T + t, w=0.1, beta=2.0, lam_reg=2.0, n_iter=10)
    np.testing.assert_allclose(moved["T"], base["T"] @ R.T + t, atol=1e-10)
    assert moved["sigma2"] == pytest.approx(base["sigma2"], rel=1e-9)
    # permuting the scene leaves T unchanged
    p = np.random.default_rng(0).permutation(Y.shape[0])
    perm_y = oracle.register(X, Y[p], w=0.1, beta=2.0, lam_reg=2.0, n_iter=10)
    np.testing.assert_allclose(perm_y["T"], base["T"], atol=1e-11)
    # permuting the model permutes T
    q = np.random.default_rng(1).permutation(X.shape[0])
    perm_x = oracle.register(X[q], Y, w=0.1, beta=2.0, lam_reg=2.0, n_iter=10)
    np.testing.assert_allclose(perm_x["T"], base["T"][q], atol=1e-10)


def test_recovers_synthetic_deformation():
    """Eq. 22 on the generator: the registration error drops well below the
    initial misalignment (qualitative, like the paper's accuracy claims)."""
    cfg = datagen.WORKLOADS["fp64_m500"]
    ps = datagen.gen(cfg["M"], cfg["n_out"], cfg["amp"], cfg["noise"], cfg["seed"])
    res = oracle.register(ps.X, ps.Y, w=cfg["omega"], beta=cfg["beta"], lam_reg=cfg["lam"],
                          n_iter=cfg["iters"])
    assert res["status"] == oracle.OK
    before = oracle.rmse(ps.X, ps.Yhat)
    after = oracle.rmse(res["T"], ps.Yhat)
    assert after < 0.25 * before
    assert after < 0.02


# ---------------------------------------------------------------- Eq. 22
def test_rmse_hand_values():
    """Eq. 22: the root of the mean over the M model points of the squared
    Euclidean error (not a mean over the D M coordinates, not squared).  Two
    points, one off by (3, 4, 0) and one exact: sqrt(25 / 2)."""
    T = np.array([[3.0, 4.0, 0.0], [1.0, -2.0, 0.5]])
    Yhat = np.array([[0.0, 0.0, 0.0], [1.0, -2.0, 0.5]])
    assert oracle.rmse(T, Yhat) == pytest.approx(math.sqrt(25.0 / 2.0), rel=1e-15)
    # the same error in two dimensions: the divisor is M, whatever D
    assert oracle.rmse(T[:, :2], Yhat[:, :2]) == pytest.approx(math.sqrt(25.0 / 2.0), rel=1e-15)


def test_rmse_of_a_translation_is_its_length():
    """A rigid translation by v moves every point by |v|: RMSE = |v| for any
    point set (here 37 points, v = (0.3, -1.2, 0.4), |v| = 1.3)."""
    X, _ = _rng_points(11, 37, 1)
    v = np.array([0.3, -1.2, 0.4])
    assert oracle.rmse(X + v, X) == pytest.approx(1.3, rel=1e-13)
    assert oracle.rmse(X, X) == 0.0


def test_lanczos_top_k_equals_dense_top_k():
    """eig_top (Lanczos) gives the dense solver's leading eigenvalues, and
    the low-rank registration (Eq. 20) on either basis gives the same T:
    the eigenvectors agree up to sign (and rotation inside the noise-level
    tail, which enters T with weight s_k ~ 0)."""
    X, Y = _rng_points(12, 300, 320)
    U0, l0 = oracle.eig(X, 2.0, 30)
    U1, l1 = oracle.eig_top(X, 2.0, 30)
    np.testing.assert_allclose(l1, l0, rtol=0, atol=1e-11 * l0[0])
    a = oracle.register(X, Y, w=0.1, beta=2.0, lam_reg=2.0, n_iter=8, eigpairs=(U0, l0))
    b = oracle.register(X, Y, w=0.1, beta=2.0, lam_reg=2.0, n_iter=8, eigpairs=(U1, l1))
    assert np.linalg.norm(a["T"] - b["T"]) <= 1e-10 * np.linalg.norm(a["T"])
